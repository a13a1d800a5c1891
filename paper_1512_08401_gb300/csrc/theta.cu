// Construction of Theta_K (Algorithm 2 + Sec. 3.7) and of the preconditioner diagonals
// (Sec. 4.2, 4.3), FP64 on the device.
//
//  1. probes: for every subband b, psi_b = IDWT(e_{b,0}); H psi_b and H^T psi_b by cuFFT
//     (D2Z, multiply by h^ or conj(h^), Z2D); one forward DWT each (Algorithm 2).
//  2. candidates: block (a, b) takes column taps col[b] restricted to subband a when
//     level(a) <= level(b), otherwise row taps row[a] restricted to subband b (Thm 3).
//  3. selection: keys (score desc, candidate index asc) with score |sigma_b v|; a weighted
//     radix select over the 128-bit composite key (8-bit digits, histogram weights =
//     multiplicities) finds the first tap whose entries would exceed K; everything before
//     it in key order is kept. Numerical zeros (|v| <= 1e-14 max|v|) never enter.
//  4. packing (host): kept taps -> gather-form tap lists of Theta_K and Theta_K^T, tiled
//     into the shared-memory plans of tile.cu (autotuned on the GPU).
//  5. diag(M), diag(M^2), M = Theta_K^T Theta_K, per phase class by comb probes: impulses of
//     one phase class spaced further apart than the reach of M^2, one Theta_K and one
//     Theta_K^T application, norms divided by the number of impulses.
//  6. step: power iteration for lambda_max(P^-1/2 M P^-1/2) from a splitmix64 start vector.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <tuple>

#include "device_util.cuh"
#include "fftops.cuh"
#include "subband_ops.cuh"
#include "select.cuh"
#include "theta_impl.h"

namespace wdb {

namespace {

struct CandPair {
    const double* src;     // tap array (rows x cols, row-major) inside a probe vector
    int rows, cols;
    long long base;        // global candidate index of element 0
    unsigned long long mult;
    double sigma;
};

__device__ __forceinline__ bool cand_key(const CandPair& P, int e, double thr, unsigned long long& hi,
                                         unsigned long long& lo, double& v) {
    v = P.src[e];
    const double av = fabs(v);
    if (!(av > thr)) return false;
    const double score = av * P.sigma;
    hi = ~(unsigned long long)__double_as_longlong(score);
    lo = (unsigned long long)(P.base + e);
    return true;
}

__global__ void vmax_kernel(const CandPair* __restrict__ pairs, SelState* sel) {
    const CandPair P = pairs[blockIdx.y];
    const int n = P.rows * P.cols;
    double m = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) m = fmax(m, fabs(P.src[e]));
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(&sel->vmax_bits, (unsigned long long)__double_as_longlong(m));
}

// One digit pass of the weighted radix select. Passes 0..7 take 8-bit digits of the score
// part (high to low), passes 8.. digits of the index part (ibits bits, a multiple of 8).
__global__ void sel_hist_kernel(const CandPair* __restrict__ pairs, SelState* sel, int pass, int ibits) {
    __shared__ unsigned long long h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0ull;
    __syncthreads();
    const bool skip = sel->keep_all != 0;
    const CandPair P = pairs[blockIdx.y];
    const int n = P.rows * P.cols;
    const double thr = 1e-14 * __longlong_as_double((long long)sel->vmax_bits);
    const unsigned long long phi = sel->prefix_hi, plo = sel->prefix_lo;
    if (!skip) {
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
            unsigned long long hi, lo;
            double v;
            if (!cand_key(P, e, thr, hi, lo, v)) continue;
            int d;
            if (pass < 8) {
                if (pass > 0 && (hi >> (64 - 8 * pass)) != phi) continue;
                d = (int)((hi >> (56 - 8 * pass)) & 255ull);
            } else {
                const int q = pass - 8;
                if (hi != phi) continue;
                if (q > 0 && (lo >> (ibits - 8 * q)) != plo) continue;
                d = (int)((lo >> (ibits - 8 - 8 * q)) & 255ull);
            }
            atomicAdd(&h[d], P.mult);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(&sel->hist[i], h[i]);
}

__global__ void sel_emit_kernel(const CandPair* __restrict__ pairs, SelState* sel, int* out_pair, int* out_e,
                                double* out_v, unsigned long long cap) {
    const CandPair P = pairs[blockIdx.y];
    const int n = P.rows * P.cols;
    const SelState s = *sel;
    const double thr = 1e-14 * __longlong_as_double((long long)s.vmax_bits);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        unsigned long long hi, lo;
        double v;
        if (!cand_key(P, e, thr, hi, lo, v) || !kept(s, hi, lo)) continue;
        const unsigned long long slot = atomicAdd(&sel->count, 1ull);
        if (out_pair && slot < cap) {
            out_pair[slot] = blockIdx.y;
            out_e[slot] = e;
            out_v[slot] = v;
        }
    }
}

__global__ void set_value_kernel(double* p, long long idx, double v) { p[idx] = v; }

// comb of impulses of one phase class (value v) in subband sb
template <typename T>
__global__ void comb_kernel(T* __restrict__ vec, long long off, int cols, int phy, int phx, int step, int ty, int tx,
                            T v) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ty * tx) return;
    int ky = t / tx, kx = t - ky * tx;
    vec[off + (size_t)(phy + ky * step) * cols + (phx + kx * step)] = v;
}

int wrap_signed(int v, int n) {
    int m = ((v % n) + n) % n;
    return (m >= n - n / 2) ? m - n : m;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Handle helpers
// ---------------------------------------------------------------------------------------
template <typename T>
wdb_status th_alloc(wdb_theta* th, T** p, size_t n) {
    void* q = nullptr;
    WDB_CK(cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)));
    th->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return WDB_OK;
}
template wdb_status th_alloc<float>(wdb_theta*, float**, size_t);
template wdb_status th_alloc<double>(wdb_theta*, double**, size_t);
template wdb_status th_alloc<int>(wdb_theta*, int**, size_t);

template <typename T>
static wdb_status upload(wdb_theta* th, const std::vector<T>& h, T** d, cudaStream_t st) {
    WDB_TRY(th_alloc(th, reinterpret_cast<T**>(d), h.size()));
    if (!h.empty()) WDB_CK(cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return WDB_OK;
}

SubbandArgs subband_args(const wdb_theta* th) {
    SubbandArgs A;
    A.sb = th->d_sb;
    A.vb_start = th->d_vb_start;
    A.S = th->lay.S;
    A.nvb = th->sched.nvb;
    return A;
}

RedTarget th_red(const wdb_theta* th, double* out) { return RedTarget{th->d_counter, th->d_red_part, out}; }

// ---------------------------------------------------------------------------------------
// Kept taps in gather form, one list per operator (Theta_K, Theta_K^T)
//   down pair (input finer or equal, ratio r = 2^lg): out[p] += v * in[r p + d]
//   up pair   (input coarser, r = 2^lg):  out[r P + phi] += v * in[P + d] for taps of phase phi
// ---------------------------------------------------------------------------------------
struct PEntry {
    int out, in, up, lg, phase, dy, dx;
    double v;
    bool operator<(const PEntry& o) const {
        return std::tie(out, in, up, lg, phase, dy, dx) < std::tie(o.out, o.in, o.up, o.lg, o.phase, o.dy, o.dx);
    }
};

// Kept taps -> gather-form entries of Theta_K (te[0]) and Theta_K^T (te[1]), sorted (host).
void gather_entries(const Layout& L, const std::vector<Tap>& taps, std::vector<TileEntry> (&te)[2]) {
    std::vector<PEntry> F, A;
    F.reserve(taps.size());
    A.reserve(taps.size());
    for (const Tap& t : taps) {
        const SubbandDev &sa = L.sb[t.a], &sb = L.sb[t.b];
        if (sa.level <= sb.level) {  // column form: tap array in subband a
            const int lg = sb.level - sa.level;
            if (lg == 0) {
                F.push_back({t.a, t.b, 0, 0, 0, wrap_signed(-t.oy, sb.rows), wrap_signed(-t.ox, sb.cols), t.v});
            } else {
                const int m = (1 << lg) - 1;
                const int ph = ((t.oy & m) << lg) | (t.ox & m);
                F.push_back({t.a, t.b, 1, lg, ph, wrap_signed(-(t.oy >> lg), sb.rows), wrap_signed(-(t.ox >> lg), sb.cols),
                             t.v});
            }
            A.push_back({t.b, t.a, 0, lg, 0, wrap_signed(t.oy, sa.rows), wrap_signed(t.ox, sa.cols), t.v});
        } else {  // row form: tap array in subband b
            const int lg = sa.level - sb.level;
            F.push_back({t.a, t.b, 0, lg, 0, wrap_signed(t.oy, sb.rows), wrap_signed(t.ox, sb.cols), t.v});
            const int m = (1 << lg) - 1;
            const int ph = ((t.oy & m) << lg) | (t.ox & m);
            A.push_back({t.b, t.a, 1, lg, ph, wrap_signed(-(t.oy >> lg), sa.rows), wrap_signed(-(t.ox >> lg), sa.cols),
                         t.v});
        }
    }
    std::sort(F.begin(), F.end());
    std::sort(A.begin(), A.end());
    for (int op = 0; op < 2; ++op) {
        const std::vector<PEntry>& src = op ? A : F;
        te[op].resize(src.size());
        for (size_t i = 0; i < src.size(); ++i)
            te[op][i] = TileEntry{src[i].out, src[i].in, src[i].up, src[i].lg, src[i].phase, src[i].dy, src[i].dx, src[i].v};
    }
}

static void build_ops(wdb_theta* th) {
    const Layout& L = th->lay;
    gather_entries(L, th->taps, th->tent);
    // the tiles are shared by about 3 resident CTAs per SM
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ctas = 3 * std::max(sms, 1);
    th->plan_ctas = ctas;
    for (int op = 0; op < 2; ++op) {
        th->tplan[op][0] = make_tile_plan(L, th->tent[op], 4, kTileSmemBudget, ctas);
        th->tplan[op][1] = make_tile_plan(L, th->tent[op], 8, kTileSmemBudget, ctas);
    }
}

namespace {

// Device copy of a candidate plan, freed after it has been timed.
struct TempPlan {
    std::vector<void*> bufs;
    TileArgs a{};
    ~TempPlan() {
        for (void* p : bufs) cudaFree(p);
    }
};

template <typename T>
wdb_status temp_copy(TempPlan& d, const std::vector<T>& h, const T** out, cudaStream_t st) {
    void* p = nullptr;
    WDB_CK(cudaMalloc(&p, std::max<size_t>(h.size(), 1) * sizeof(T)));
    d.bufs.push_back(p);
    if (!h.empty()) WDB_CK(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    *out = static_cast<const T*>(p);
    return WDB_OK;
}

wdb_status temp_plan(const wdb_theta* th, const TilePlanHost& h, TempPlan& d, cudaStream_t st) {
    TilePlanDev& p = d.a.plan;
    WDB_TRY(temp_copy(d, h.pairs, &p.pairs, st));
    WDB_TRY(temp_copy(d, h.pair_sm, &p.pair_sm, st));
    WDB_TRY(temp_copy(d, h.subs, &p.subs, st));
    WDB_TRY(temp_copy(d, h.batches, &p.batches, st));
    WDB_TRY(temp_copy(d, h.items, &p.items, st));
    WDB_TRY(temp_copy(d, h.tap_off, &p.tap_off, st));
    WDB_TRY(temp_copy(d, h.tap_lin, &p.tap_lin, st));
    WDB_TRY(temp_copy(d, h.tap_v, &p.tap_v, st));
    WDB_TRY(temp_copy(d, h.tap_v64, &p.tap_v64, st));
    WDB_TRY(temp_copy(d, h.tap_ov, &p.tap_ov, st));
    if (h.n_split > 0) {   // split tiles: zeroed arrival counters and the partial sums
        void* c = nullptr;
        void* b = nullptr;
        WDB_CK(cudaMalloc(&c, sizeof(unsigned int) * h.n_split));
        d.bufs.push_back(c);
        WDB_CK(cudaMemsetAsync(c, 0, sizeof(unsigned int) * h.n_split, st));
        WDB_CK(cudaMalloc(&b, (size_t)h.esize * h.split_elems));
        d.bufs.push_back(b);
        p.split_ctr = static_cast<unsigned int*>(c);
        p.split_buf = b;
        WDB_TRY(temp_copy(d, h.split_base, &p.split_base, st));
    }
    p.n_items = (int)h.items.size();
    p.n_sup = h.n_sup;
    p.n_grp = h.n_grp;
    p.buf_elems = h.buf_elems;
    p.smem_bytes = h.smem_bytes;
    d.a.sb = th->d_sb;
    void* q = nullptr;
    WDB_CK(cudaMalloc(&q, sizeof(TileQueue)));
    d.bufs.push_back(q);
    WDB_CK(cudaMemsetAsync(q, 0, sizeof(TileQueue), st));
    d.a.queue = static_cast<TileQueue*>(q);
    d.a.grid = std::max(1, std::min(p.n_items, tile_grid(h.smem_bytes)));
    return WDB_OK;
}

}  // namespace

// Autotuned FP32 tile plans: for every output level, each candidate (tile side, 1 or 4
// outputs per thread) is planned for that level's tiles alone and applied on this GPU (best
// of 3 after a warm-up); the per-level winners form one plan, which then competes, over the
// whole operator, with the planner's own plans (per-tile cost caps of 1, 2 and 4 per-CTA
// shares, which balance the levels against each other, and staging buffers of 24, 32 and
// 48 KB, which trade batches per tile against resident CTAs). The fastest is kept.
static wdb_status autotune_plans(wdb_theta* th, cudaStream_t st) {
    const Layout& L = th->lay;
    const long long N = L.N;
    float *in = nullptr, *out = nullptr;
    double* part = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    wdb_status s = WDB_OK;
    auto fail = [&](wdb_status v) {
        if (s == WDB_OK) s = v;
    };
    if (cudaMalloc(&in, sizeof(float) * N) != cudaSuccess || cudaMalloc(&out, sizeof(float) * N) != cudaSuccess ||
        cudaMalloc(&part, sizeof(double) * 2 * 8192) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        fail(set_error(WDB_ENOMEM, "autotune workspace"));
    if (s == WDB_OK && cudaMemsetAsync(in, 0, sizeof(float) * N, st) != cudaSuccess) fail(set_error(WDB_ECUDA, "memset"));
    // milliseconds of one application of plan h (1e30 on error)
    auto time_plan = [&](const TilePlanHost& h) {
        float ms = 1e30f;
        TempPlan d;
        wdb_status r = temp_plan(th, h, d, st);
        if (r != WDB_OK) {
            fail(r);
            return ms;
        }
        for (int rep = 0; rep < 4 && s == WDB_OK; ++rep) {
            if (cudaEventRecord(e0, st) != cudaSuccess) fail(set_error(WDB_ECUDA, "event"));
            // timed with kernel 1's epilogue (read x0, write r, reduce ||r||^2), so that plans
            // are ranked with a solve's per-output loads and stores
            r = tile_resnorm(d.a, in, in, out, part + 2 * 8192 - 1, part, st);
            if (r != WDB_OK) fail(r);
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
                fail(set_error(WDB_ECUDA, "autotune timing"));
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms = std::min(ms, t);   // the first application is a warm-up
        }
        return ms;
    };
    for (int op = 0; op < 2 && s == WDB_OK; ++op) {
        std::vector<TileTune> best(L.S, TileTune{0, 0});
        for (int lev = 1; lev <= L.J && s == WDB_OK; ++lev) {
            int side = 1;
            for (int o = 0; o < L.S; ++o)
                if (L.sb[o].level == lev) side = std::max(side, std::max(L.sb[o].rows, L.sb[o].cols));
            int tsmax = 1;
            while (tsmax < side && tsmax < 32) tsmax <<= 1;
            float best_ms = 1e30f;
            TileTune pick{0, 0};
            for (int ts = tsmax; ts >= 1 && s == WDB_OK; ts >>= 1)
                for (int e4 = 1; e4 >= 0; --e4) {
                    if ((e4 && ts < 8) || (!e4 && ts == 32)) continue;
                    std::vector<TileTune> tune(L.S, TileTune{0, 0});
                    for (int o = 0; o < L.S; ++o)
                        if (L.sb[o].level == lev) tune[o] = TileTune{ts, e4};
                    const TilePlanHost h =
                        make_tile_plan(L, th->tent[op], 4, kTileSmemBudget, th->plan_ctas, &tune, lev);
                    if (h.items.empty()) continue;
                    const float ms = time_plan(h);
                    if (ms < best_ms) {
                        best_ms = ms;
                        pick = TileTune{ts, e4};
                    }
                }
            for (int o = 0; o < L.S; ++o)
                if (L.sb[o].level == lev) best[o] = pick;
        }
        if (s != WDB_OK) break;
        th->tune_levels[op] = best;
        std::vector<TilePlanHost> whole;
        whole.push_back(make_tile_plan(L, th->tent[op], 4, kTileSmemBudget, th->plan_ctas, &best, 0));
        for (int budget : {kTileSmemBudget * 3 / 4, kTileSmemBudget, kTileSmemBudget * 3 / 2})
            for (double cap : {1.0, 2.0, 4.0})
                whole.push_back(make_tile_plan(L, th->tent[op], 4, budget, th->plan_ctas, nullptr, 0, cap));
        // the same with the heaviest tiles split over several CTAs
        for (double split : {0.5, 1.0})
            whole.push_back(make_tile_plan(L, th->tent[op], 4, kTileSmemBudget, th->plan_ctas, &best, 0, 2.0, split));
        for (double cap : {2.0, 4.0})
            whole.push_back(make_tile_plan(L, th->tent[op], 4, kTileSmemBudget, th->plan_ctas, nullptr, 0, cap, 1.0));
        // and with super tiles (2 x 2 tiles staged together) where they fit one buffer
        for (int budget : {kTileSmemBudget, kTileSmemBudget * 3 / 2})
            whole.push_back(make_tile_plan(L, th->tent[op], 4, budget, th->plan_ctas, &best, 0, 2.0, 0.0, true));
        for (double cap : {2.0, 4.0})
            whole.push_back(make_tile_plan(L, th->tent[op], 4, kTileSmemBudget, th->plan_ctas, nullptr, 0, cap, 0.0,
                                           true));
        // and with grouped items (each input region staged once for every subband of a level)
        for (int budget : {kTileSmemBudget, kTileSmemBudget * 3 / 2})
            whole.push_back(make_tile_plan(L, th->tent[op], 4, budget, th->plan_ctas, &best, 0, 2.0, 0.0, false, true));
        for (double cap : {1.0, 2.0, 4.0})
            whole.push_back(make_tile_plan(L, th->tent[op], 4, kTileSmemBudget, th->plan_ctas, nullptr, 0, cap, 0.0,
                                           false, true));
        float best_ms = 1e30f;
        for (size_t k = 0; k < whole.size() && s == WDB_OK; ++k) {
            const float ms = time_plan(whole[k]);
            if (ms < best_ms) {
                best_ms = ms;
                th->tplan[op][0] = whole[k];
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(in);
    cudaFree(out);
    cudaFree(part);
    if (s == WDB_OK) th->tuned = 1;
    return s;
}

static wdb_status upload_plan(wdb_theta* th, const TilePlanHost& h, TileArgs& a, cudaStream_t st) {
    WDB_TRY(upload(th, h.pairs, const_cast<TilePair**>(&a.plan.pairs), st));
    WDB_TRY(upload(th, h.pair_sm, const_cast<PairSm**>(&a.plan.pair_sm), st));
    WDB_TRY(upload(th, h.subs, const_cast<TileSub**>(&a.plan.subs), st));
    WDB_TRY(upload(th, h.batches, const_cast<TileBatch**>(&a.plan.batches), st));
    WDB_TRY(upload(th, h.items, const_cast<TileItem**>(&a.plan.items), st));
    WDB_TRY(upload(th, h.tap_off, const_cast<int**>(&a.plan.tap_off), st));
    WDB_TRY(upload(th, h.tap_lin, const_cast<int**>(&a.plan.tap_lin), st));
    WDB_TRY(upload(th, h.tap_v, const_cast<float**>(&a.plan.tap_v), st));
    WDB_TRY(upload(th, h.tap_v64, const_cast<double**>(&a.plan.tap_v64), st));
    WDB_TRY(upload(th, h.tap_ov, const_cast<TapOV**>(&a.plan.tap_ov), st));
    a.plan.split_ctr = nullptr;
    a.plan.split_base = nullptr;
    a.plan.split_buf = nullptr;
    if (h.n_split > 0) {   // split tiles: zeroed arrival counters and the partial sums
        std::vector<unsigned int> zero(h.n_split, 0u);
        WDB_TRY(upload(th, zero, &a.plan.split_ctr, st));
        WDB_TRY(upload(th, h.split_base, const_cast<long long**>(&a.plan.split_base), st));
        void* b = nullptr;
        WDB_CK(cudaMalloc(&b, (size_t)h.esize * h.split_elems));
        th->allocs.push_back(b);
        a.plan.split_buf = b;
    }
    a.plan.n_items = (int)h.items.size();
    a.plan.n_sup = h.n_sup;
    a.plan.n_grp = h.n_grp;
    a.plan.buf_elems = h.buf_elems;
    a.plan.smem_bytes = h.smem_bytes;
    a.sb = th->d_sb;
    void* q = nullptr;
    WDB_CK(cudaMalloc(&q, sizeof(TileQueue)));
    th->allocs.push_back(q);
    WDB_CK(cudaMemsetAsync(q, 0, sizeof(TileQueue), st));
    a.queue = static_cast<TileQueue*>(q);
    a.grid = std::max(1, std::min(a.plan.n_items, tile_grid(h.smem_bytes)));
    return WDB_OK;
}

TileArgs tile_args(const wdb_theta* th, bool adj, bool fp64) { return th->targs[adj ? 1 : 0][fp64 ? 1 : 0]; }

// Plans for batched solves: the autotuner's tile side and thread map per output level (the
// planner's where the operator was not tuned) with a loose per-tile cap (16 per-CTA shares),
// since the tiles of many problems share the CTAs; built on first use.
wdb_status theta_batch_plans(wdb_theta* th, cudaStream_t st) {
    if (th->bplan_ok) return WDB_OK;
    for (int op = 0; op < 2; ++op) {
        const std::vector<TileTune>* tune =
            (int)th->tune_levels[op].size() == th->lay.S ? &th->tune_levels[op] : nullptr;
        // grouped items: one item per (level, tile) computes every subband of the level, so
        // the per-item set-up and staging of the many small items of a batch are shared
        th->bplan[op] = make_tile_plan(th->lay, th->tent[op], 4, kTileSmemBudget, th->plan_ctas, tune, 0, 16.0, 0.0,
                                       false, true);
        WDB_TRY(upload_plan(th, th->bplan[op], th->bargs[op], st));
    }
    th->bplan_ok = true;
    return WDB_OK;
}

// Planner plans in place of the FP32 plans (no autotuning); captured solve graphs hold the
// old plans' arguments and are dropped.
wdb_status theta_replan(wdb_theta* th, int budget, double cap_share, double split_share, int tiling,
                        cudaStream_t st) {
    for (int op = 0; op < 2; ++op) {
        th->tplan[op][0] = make_tile_plan(th->lay, th->tent[op], 4, budget, th->plan_ctas, nullptr, 0, cap_share,
                                          split_share, tiling == 1, tiling == 2);
        WDB_TRY(upload_plan(th, th->tplan[op][0], th->targs[op][0], st));
    }
    th->tuned = 0;
    for (auto& e : th->engine) e.release();
    WDB_CK(cudaStreamSynchronize(st));
    return WDB_OK;
}

// max image-space distance between the two coefficients of a kept entry (pixels)
static long long tap_reach(const wdb_theta* th) {
    const Layout& L = th->lay;
    long long D = 0;
    for (const Tap& t : th->taps) {
        const SubbandDev &sa = L.sb[t.a], &sb = L.sb[t.b];
        const SubbandDev& arr = (sa.level <= sb.level) ? sa : sb;
        long long dy = std::llabs((long long)wrap_signed(t.oy, arr.rows)) << arr.level;
        long long dx = std::llabs((long long)wrap_signed(t.ox, arr.cols)) << arr.level;
        D = std::max(D, std::max(dy, dx));
    }
    return D;
}

bool setup_fp64(const wdb_theta* th) { return th->lay.N <= (1LL << 21); }

// diag(M), diag(M^2) per phase class by comb probes
template <typename T>
static wdb_status diag_tables(wdb_theta* th, cudaStream_t st) {
    const Layout& L = th->lay;
    const long long N = L.N;
    T *v = nullptr, *u = nullptr, *w = nullptr;
    WDB_CK(cudaMalloc(&v, sizeof(T) * N));
    WDB_CK(cudaMalloc(&u, sizeof(T) * N));
    WDB_CK(cudaMalloc(&w, sizeof(T) * N));
    double* d_out = nullptr;
    WDB_CK(cudaMalloc(&d_out, sizeof(double) * 2 * L.tab_len));
    WDB_CK(cudaMemsetAsync(v, 0, sizeof(T) * N, st));
    const long long D = tap_reach(th);
    const long long P2 = 1LL << L.J;
    const long long Timg = P2 * ((4 * D + 1 + P2 - 1) / P2);
    const int ty = (int)std::max<long long>(1, L.n_rows / Timg), tx = (int)std::max<long long>(1, L.n_cols / Timg);
    const bool f64 = sizeof(T) == 8;
    TileArgs F = tile_args(th, false, f64), A = tile_args(th, true, f64);
    wdb_status s = WDB_OK;
    for (int b = 0; b < L.S && s == WDB_OK; ++b) {
        const SubbandDev& sb = L.sb[b];
        const int R = 1 << sb.lgR;
        const int step = (int)(Timg >> sb.level);
        for (int py = 0; py < R && s == WDB_OK; ++py)
            for (int px = 0; px < R && s == WDB_OK; ++px) {
                const int cls = sb.tab_off + py * R + px;
                comb_kernel<T><<<(ty * tx + 255) / 256, 256, 0, st>>>(v, sb.off, sb.cols, py, px, step, ty, tx, (T)1);
                count_launch();
                s = tile_apply<T>(F, v, u, nullptr, d_out + 2 * cls, th->d_red_part, st);
                if (s == WDB_OK) s = tile_apply<T>(A, u, w, nullptr, d_out + 2 * cls + 1, th->d_red_part, st);
                comb_kernel<T><<<(ty * tx + 255) / 256, 256, 0, st>>>(v, sb.off, sb.cols, py, px, step, ty, tx, (T)0);
                count_launch();
            }
    }
    std::vector<double> out(2 * L.tab_len);
    if (s == WDB_OK) {
        cudaError_t e = cudaMemcpyAsync(out.data(), d_out, sizeof(double) * out.size(), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_error(e, "diag tables", __FILE__, __LINE__);
    }
    cudaFree(v);
    cudaFree(u);
    cudaFree(w);
    cudaFree(d_out);
    if (s != WDB_OK) return s;
    const double teeth = (double)ty * tx;
    th->Md.resize(L.tab_len);
    th->M2d.resize(L.tab_len);
    for (int c = 0; c < L.tab_len; ++c) {
        th->Md[c] = out[2 * c] / teeth;
        th->M2d[c] = out[2 * c + 1] / teeth;
    }
    th->diag_valid = true;
    return WDB_OK;
}

// Tile plans, subband schedule, workspace for reductions, diag tables.
wdb_status theta_finalize(wdb_theta* th, cudaStream_t st) {
    const Layout& L = th->lay;
    th->K_eff = 0;
    for (const Tap& t : th->taps) {
        const SubbandDev &sa = L.sb[t.a], &sb = L.sb[t.b];
        th->K_eff += std::min((long long)sa.rows * sa.cols, (long long)sb.rows * sb.cols);
    }
    build_ops(th);
    std::vector<SubbandDev> sbv(L.sb, L.sb + L.S);
    WDB_TRY(upload(th, sbv, &th->d_sb, st));
    th->sched = make_schedule(L);
    WDB_TRY(upload(th, th->sched.vb_start, &th->d_vb_start, st));
    th->grid = std::max(1, std::min(th->sched.nvb, subband_grid_limit()));
    th->part_len = th->grid;
    if (kAutotunePlans) WDB_TRY(autotune_plans(th, st));
    for (int op = 0; op < 2; ++op)
        for (int pr = 0; pr < 2; ++pr) {
            WDB_TRY(upload_plan(th, th->tplan[op][pr], th->targs[op][pr], st));
            th->part_len = std::max(th->part_len, th->targs[op][pr].grid);
        }
    WDB_TRY(th_alloc(th, &th->d_red_part, (size_t)th->part_len * 4));
    unsigned int* cnt = nullptr;
    WDB_CK(cudaMalloc(&cnt, sizeof(unsigned int) * 4));
    th->allocs.push_back(cnt);
    WDB_CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned int) * 4, st));
    th->d_counter = cnt;
    if (setup_fp64(th)) WDB_TRY(diag_tables<double>(th, st));
    else WDB_TRY(diag_tables<float>(th, st));
    return WDB_OK;
}

// ---------------------------------------------------------------------------------------
// Algorithm 2 + Sec. 3.7 on the device
// ---------------------------------------------------------------------------------------
wdb_status theta_build_device(wdb_theta* th, const double* psf_host, int kh, int kw, long long K, int rule,
                              cudaStream_t st) {
    const Layout& L = th->lay;
    const long long N = L.N;
    const int R = L.n_rows, C = L.n_cols, C2 = C / 2 + 1;
    const long long NC = (long long)R * C2;
    // device scratch
    double *psf = nullptr, *img = nullptr, *coef = nullptr, *scr = nullptr, *probes = nullptr;
    cufftDoubleComplex *hhat = nullptr, *spec = nullptr, *prod = nullptr;
    std::vector<void*> tmp;
    auto dmalloc = [&](void** p, size_t bytes) -> wdb_status {
        WDB_CK(cudaMalloc(p, std::max<size_t>(bytes, 1)));
        tmp.push_back(*p);
        return WDB_OK;
    };
    auto cleanup = [&]() {
        for (void* p : tmp) cudaFree(p);
        tmp.clear();
    };
    cufftHandle pf = 0, pi = 0;
    bool have_pf = false, have_pi = false;
    wdb_status s = WDB_OK;
    do {
        if ((s = dmalloc((void**)&psf, sizeof(double) * kh * kw))) break;
        if ((s = dmalloc((void**)&img, sizeof(double) * N))) break;
        if ((s = dmalloc((void**)&coef, sizeof(double) * N))) break;
        if ((s = dmalloc((void**)&scr, sizeof(double) * (N / 2 + 1)))) break;
        if ((s = dmalloc((void**)&probes, sizeof(double) * N * 2 * L.S))) break;
        if ((s = dmalloc((void**)&hhat, sizeof(cufftDoubleComplex) * NC))) break;
        if ((s = dmalloc((void**)&spec, sizeof(cufftDoubleComplex) * NC))) break;
        if ((s = dmalloc((void**)&prod, sizeof(cufftDoubleComplex) * NC))) break;
        cufftResult fr = cufftPlan2d(&pf, R, C, CUFFT_D2Z);
        if (fr != CUFFT_SUCCESS) { s = cufft_error(fr, "cufftPlan2d D2Z", __FILE__, __LINE__); break; }
        have_pf = true;
        fr = cufftPlan2d(&pi, R, C, CUFFT_Z2D);
        if (fr != CUFFT_SUCCESS) { s = cufft_error(fr, "cufftPlan2d Z2D", __FILE__, __LINE__); break; }
        have_pi = true;
        cufftSetStream(pf, st);
        cufftSetStream(pi, st);
        cudaError_t ce = cudaMemcpyAsync(psf, psf_host, sizeof(double) * kh * kw, cudaMemcpyHostToDevice, st);
        if (ce != cudaSuccess) { s = cuda_error(ce, "copy psf", __FILE__, __LINE__); break; }
        if ((s = launch_pad_psf(psf, kh, kw, img, R, C, st))) break;
        fr = cufftExecD2Z(pf, img, hhat);
        if (fr != CUFFT_SUCCESS) { s = cufft_error(fr, "D2Z psf", __FILE__, __LINE__); break; }
        // probes (Algorithm 2)
        for (int b = 0; b < L.S && s == WDB_OK; ++b) {
            cudaMemsetAsync(coef, 0, sizeof(double) * N, st);
            set_value_kernel<<<1, 1, 0, st>>>(coef, L.sb[b].off, 1.0);
            count_launch();
            if ((s = idwt2<double>(coef, img, L, th->filt, scr, st))) break;
            fr = cufftExecD2Z(pf, img, spec);
            if (fr != CUFFT_SUCCESS) { s = cufft_error(fr, "D2Z probe", __FILE__, __LINE__); break; }
            for (int which = 0; which < 2 && s == WDB_OK; ++which) {   // 0: H (column), 1: H^T (row)
                if ((s = launch_cmul64(spec, hhat, prod, NC, which, 1.0 / (double)N, st))) break;
                fr = cufftExecZ2D(pi, prod, img);
                if (fr != CUFFT_SUCCESS) { s = cufft_error(fr, "Z2D probe", __FILE__, __LINE__); break; }
                double* dst = probes + (size_t)(which * L.S + b) * N;
                s = dwt2<double>(img, dst, L, th->filt, scr, st);
            }
        }
        if (s) break;
        // candidate pairs
        std::vector<CandPair> cp(L.S * L.S);
        long long base = 0;
        int maxn = 1;
        for (int a = 0; a < L.S; ++a)
            for (int b = 0; b < L.S; ++b) {
                const SubbandDev &sa = L.sb[a], &sb = L.sb[b];
                CandPair& c = cp[a * L.S + b];
                if (sa.level <= sb.level) {
                    c.src = probes + (size_t)b * N + sa.off;
                    c.rows = sa.rows;
                    c.cols = sa.cols;
                    c.mult = (unsigned long long)sb.rows * sb.cols;
                } else {
                    c.src = probes + (size_t)(L.S + a) * N + sb.off;
                    c.rows = sb.rows;
                    c.cols = sb.cols;
                    c.mult = (unsigned long long)sa.rows * sa.cols;
                }
                c.sigma = (rule == WDB_RULE_NAIVE) ? 1.0 : std::ldexp(1.0, sb.level);
                c.base = base;
                base += (long long)c.rows * c.cols;
                maxn = std::max(maxn, c.rows * c.cols);
            }
        th->n_candidates = base;
        int ibits = 8;
        while (ibits < 64 && (base >> ibits) != 0) ibits += 8;
        CandPair* d_cp = nullptr;
        SelState* d_sel = nullptr;
        if ((s = dmalloc((void**)&d_cp, sizeof(CandPair) * cp.size()))) break;
        if ((s = dmalloc((void**)&d_sel, sizeof(SelState)))) break;
        SelState h0;
        std::memset(&h0, 0, sizeof h0);
        h0.K = (unsigned long long)std::max<long long>(K, 0);
        cudaMemcpyAsync(d_cp, cp.data(), sizeof(CandPair) * cp.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_sel, &h0, sizeof h0, cudaMemcpyHostToDevice, st);
        dim3 g((unsigned)std::min(64, (maxn + 255) / 256), (unsigned)cp.size());
        vmax_kernel<<<g, 256, 0, st>>>(d_cp, d_sel);
        count_launch();
        const int passes = 8 + ibits / 8;
        for (int p = 0; p < passes; ++p) {
            sel_hist_kernel<<<g, 256, 0, st>>>(d_cp, d_sel, p, ibits);
            sel_scan_kernel<<<1, 32, 0, st>>>(d_sel, p);
            count_launch(2);
        }
        sel_emit_kernel<<<g, 256, 0, st>>>(d_cp, d_sel, nullptr, nullptr, nullptr, 0);
        count_launch();
        SelState hs;
        ce = cudaMemcpyAsync(&hs, d_sel, sizeof hs, cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce == cudaSuccess) ce = cudaGetLastError();
        if (ce != cudaSuccess) { s = cuda_error(ce, "tap selection", __FILE__, __LINE__); break; }
        std::memcpy(&th->theta_max_abs, &hs.vmax_bits, sizeof(double));
        const unsigned long long nk = hs.count;
        int *d_pair = nullptr, *d_e = nullptr;
        double* d_v = nullptr;
        if ((s = dmalloc((void**)&d_pair, sizeof(int) * nk))) break;
        if ((s = dmalloc((void**)&d_e, sizeof(int) * nk))) break;
        if ((s = dmalloc((void**)&d_v, sizeof(double) * nk))) break;
        cudaMemsetAsync(&d_sel->count, 0, sizeof(unsigned long long), st);
        sel_emit_kernel<<<g, 256, 0, st>>>(d_cp, d_sel, d_pair, d_e, d_v, nk);
        count_launch();
        std::vector<int> hp(nk), he(nk);
        std::vector<double> hv(nk);
        if (nk) {
            cudaMemcpyAsync(hp.data(), d_pair, sizeof(int) * nk, cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(he.data(), d_e, sizeof(int) * nk, cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(hv.data(), d_v, sizeof(double) * nk, cudaMemcpyDeviceToHost, st);
        }
        ce = cudaStreamSynchronize(st);
        if (ce == cudaSuccess) ce = cudaGetLastError();
        if (ce != cudaSuccess) { s = cuda_error(ce, "tap emit", __FILE__, __LINE__); break; }
        std::vector<size_t> ord(nk);
        for (size_t i = 0; i < nk; ++i) ord[i] = i;
        std::sort(ord.begin(), ord.end(), [&](size_t x, size_t y) {
            return hp[x] != hp[y] ? hp[x] < hp[y] : he[x] < he[y];
        });
        th->taps.resize(nk);
        for (size_t i = 0; i < nk; ++i) {
            const size_t k = ord[i];
            const CandPair& c = cp[hp[k]];
            Tap& t = th->taps[i];
            t.a = hp[k] / L.S;
            t.b = hp[k] % L.S;
            t.oy = he[k] / c.cols;
            t.ox = he[k] % c.cols;
            t.v = hv[k];
        }
    } while (false);
    if (have_pf) cufftDestroy(pf);
    if (have_pi) cufftDestroy(pi);
    cudaStreamSynchronize(st);
    cleanup();
    return s;
}

// ---------------------------------------------------------------------------------------
// Preconditioner tables and step (power iteration)
// ---------------------------------------------------------------------------------------
template <typename T>
static wdb_status power_iteration(wdb_theta* th, const std::vector<double>& P, cudaStream_t st, double* L_out) {
    const Layout& L = th->lay;
    const long long N = L.N;
    std::vector<double> sc(P.size());
    for (size_t i = 0; i < P.size(); ++i) sc[i] = 1.0 / std::sqrt(P[i]);
    T *v = nullptr, *t = nullptr, *u = nullptr;
    double *d_sc = nullptr, *d_out = nullptr;
    WDB_CK(cudaMalloc(&v, sizeof(T) * N));
    WDB_CK(cudaMalloc(&t, sizeof(T) * N));
    WDB_CK(cudaMalloc(&u, sizeof(T) * N));
    WDB_CK(cudaMalloc(&d_sc, sizeof(double) * sc.size()));
    WDB_CK(cudaMalloc(&d_out, sizeof(double)));
    WDB_CK(cudaMemcpyAsync(d_sc, sc.data(), sizeof(double) * sc.size(), cudaMemcpyHostToDevice, st));
    SubbandArgs F = subband_args(th);
    const bool f64 = sizeof(T) == 8;
    TileArgs TF = tile_args(th, false, f64), TA = tile_args(th, true, f64);
    wdb_status s = WDB_OK;
    double lam = 0.0, h_out = 0.0;
    RedTarget red = th_red(th, d_out);
    if (s == WDB_OK) s = launch_splitmix<T>(v, N, kPowerSeed, st);
    if (s == WDB_OK) s = launch_norm2<T>(v, N, red, th->grid, st);
    cudaMemcpyAsync(&h_out, d_out, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) s = set_error(WDB_ECUDA, "power iteration start");
    if (s == WDB_OK) s = launch_scale_const<T>(v, v, N, 1.0 / std::sqrt(h_out), st);
    for (int it = 1; it <= kPowerIters && s == WDB_OK; ++it) {
        if ((s = launch_scale<T>(F, th->grid, v, t, d_sc, st))) break;
        if ((s = tile_apply<T>(TF, t, u, nullptr, nullptr, th->d_red_part, st))) break;
        if ((s = tile_apply<T>(TA, u, t, d_sc, d_out, th->d_red_part, st))) break;
        cudaMemcpyAsync(&h_out, d_out, sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { s = cuda_error(e, "power iteration", __FILE__, __LINE__); break; }
        const double lam_new = std::sqrt(h_out);
        if (!(lam_new > 0.0) || !std::isfinite(lam_new)) { lam = lam_new; break; }
        if ((s = launch_scale_const<T>(t, v, N, 1.0 / lam_new, st))) break;
        const bool done = std::fabs(lam_new - lam) <= kPowerRtol * lam_new;
        lam = lam_new;
        if (done) break;
    }
    cudaStreamSynchronize(st);
    cudaFree(v);
    cudaFree(t);
    cudaFree(u);
    cudaFree(d_sc);
    cudaFree(d_out);
    if (s != WDB_OK) return s;
    if (!std::isfinite(lam)) return set_error(WDB_ENAN, "power iteration produced %g", lam);
    *L_out = lam;
    return WDB_OK;
}

std::vector<double> precond_table(const std::vector<double>& Md, const std::vector<double>& M2d, int kind,
                                  double eps) {
    std::vector<double> P(Md.size(), 1.0);
    if (kind == WDB_PRECOND_JACOBI) {
        double mx = 0.0;
        for (double m : Md) mx = std::max(mx, m);
        const double e = eps > 0.0 ? eps : 1e-6 * mx;
        for (size_t i = 0; i < P.size(); ++i) P[i] = std::max(Md[i], e);
        for (double& p : P)
            if (!(p > 0.0)) p = 1.0;
    } else if (kind == WDB_PRECOND_SPAI) {
        for (size_t i = 0; i < P.size(); ++i) P[i] = Md[i] > 0.0 ? M2d[i] / Md[i] : 1.0;
    }
    return P;
}

wdb_status precond_upload(wdb_theta* th, PrecondCache& pc, cudaStream_t st) {
    const int n = (int)pc.P.size();
    if (!pc.d_step) WDB_TRY(th_alloc(th, &pc.d_step, n));
    std::vector<float> stp(n);
    for (int i = 0; i < n; ++i) stp[i] = (float)(pc.tau / pc.P[i]);
    WDB_CK(cudaMemcpyAsync(pc.d_step, stp.data(), sizeof(float) * n, cudaMemcpyHostToDevice, st));
    WDB_CK(cudaStreamSynchronize(st));
    return WDB_OK;
}

wdb_status theta_precond(wdb_theta* th, int kind, double eps, cudaStream_t st) {
    if (kind < 0 || kind > 2) return set_error(WDB_EINVAL, "unknown preconditioner %d", kind);
    PrecondCache& pc = th->pc[kind];
    if (pc.valid && (pc.pinned || kind != WDB_PRECOND_JACOBI || pc.eps == eps)) return WDB_OK;
    if (!th->diag_valid) return set_error(WDB_EINVAL, "diagonal tables missing");
    pc.P = precond_table(th->Md, th->M2d, kind, eps);
    double Lh = 0.0;
    if (setup_fp64(th)) WDB_TRY(power_iteration<double>(th, pc.P, st, &Lh));
    else WDB_TRY(power_iteration<float>(th, pc.P, st, &Lh));
    pc.L_hat = Lh;
    pc.tau = Lh > 0.0 ? 1.0 / (kStepMargin * Lh) : 1.0;
    pc.eps = eps;
    WDB_TRY(precond_upload(th, pc, st));
    pc.valid = true;
    return WDB_OK;
}

}  // namespace wdb
