// Spatially varying blur (Sec. 3.1, 3.4, 3.5): Theta_K of an operator whose PSF varies
// from image row to image row, built on the device in FP64, and the FISTA iteration
// (Algorithm 3) on it.
//
// H: the input pixels of image row i spread with psfs[i] (odd kh x kw, centre at the origin)
// on the torus. Such an H commutes with horizontal translations, so Theta = Psi* H Psi is
// circulant along the column axis inside every pair of subbands: an entry is fixed by the
// output row (a, py), the input row (b, qy) and one horizontal tap offset ox, with
//   column form (s_a <= s_b, r = 2^{s_b - s_a}): px = ox + r qx (mod C_a),
//   row form    (s_a >  s_b, r = 2^{s_a - s_b}): qx = ox + r px (mod C_b).
//
//  1. probes: the wavelet of (b, qy, 0) is the outer product of two 1-D synthesis functions
//     (computed on the host); H of it (column probe, every input row of every subband) or
//     H^T of the wavelet of (a, py, 0) (row probe, every output row of a subband above level
//     1) is evaluated on the window the result can occupy, then one FP64 forward DWT. The
//     windows of the coefficients that can be nonzero (propagated level by level through
//     the analysis filters) are copied to a flat candidate array (Sec. 3.4, one probe per
//     row instead of one per column).
//  2. selection (Sec. 3.7): the weighted radix select of select.cuh over the score digits
//     finds the score of the first tap whose entries would exceed K; taps above it are kept,
//     taps at exactly that score in (a, py, b, qy, ox) order while the count stays <= K.
//  3. row plans: Theta_K and Theta_K^T as per-output-row tap lists. One CTA per output row:
//     taps whose input index moves with the output index (ci = ox + r c, or c - ox) are
//     summed in registers, outputs along the threads; taps of an input coarser than the
//     output (ci = (c - ox) / r on outputs c = ox mod r) run phase by phase, a warp's lanes
//     on consecutive inputs of one phase, into a shared-memory row accumulator. The
//     epilogues (residual, fused step / soft threshold / momentum, objective) and the
//     FP64 grid reductions are those of the circulant kernels.
//  4. preconditioner (Sec. 4.2, 4.3) on the host in FP64: diag(M) and diag(M^2) of
//     M = Theta_K^T Theta_K per class (b, qy, qx mod 2^{J - s_b}) from the tap lists; the
//     step by power iteration on the device (FP64 kernels).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>

#include "device_util.cuh"
#include "select.cuh"
#include "solve_impl.h"
#include "subband_ops.cuh"
#include "theta_impl.h"
#include "vtheta.h"

namespace wdb {

namespace {

constexpr int kVThreads = 256;
constexpr int kVMaxCols = 1024;   // outputs of one row held by one CTA (4 per thread)

enum { kVApply = 0, kVK1 = 1, kVK2 = 2, kVObj = 3 };

struct VEpi {
    const float* x0;          // K1, Obj
    float* x;                 // K2: x^(k-1) in, x^(k) out
    float* y;                 // K2: y^(k) in, y^(k+1) out
    const float* step_tab;    // K2: tau / P per class
    const float* w_sb;        // K2, Obj: weight per subband
    const float* xl1;         // Obj: the iterate whose l1 term is summed (the apply's input)
    const double* scale;      // Apply: per-class output scale (may be NULL)
    SolveState* st;
    double* part;             // grid x 3 partials
    unsigned int* counter;
    double* red_out;          // Apply (norm^2), Obj (rr, l1, support)
};

template <typename T>
__device__ __forceinline__ T tap_value(const VPlanDev& P, int i) {
    if constexpr (sizeof(T) == 8) return P.v64[i];
    else return P.v32[i];
}

// one register tap for the outputs c = lt + To e of this thread
template <typename T>
__device__ __forceinline__ void reg_tap(const VTap& tp, T v, const T* __restrict__ in, int lt, int To, int cols,
                                        T (&acc)[4]) {
    const T* __restrict__ src = in + tp.in_off;
    if (tp.mode & kVTapU) {
        // same level: ci = c - ox (mod cols)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = lt + To * e;
            if (c < cols) {
                int ci = c - tp.ox;
                if (ci < 0) ci += cols;
                acc[e] += v * src[ci];
            }
        }
    } else {
        // input finer (or same level, transposed): ci = ox + r c (mod r cols)
        const int lgr = tp.mode & 255, cin = cols << lgr;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = lt + To * e;
            if (c < cols) {
                int ci = tp.ox + (c << lgr);
                if (ci >= cin) ci -= cin;
                acc[e] += v * src[ci];
            }
        }
    }
}

template <typename T, int EPI>
__global__ void __launch_bounds__(kVThreads) vrow_kernel(VPlanDev P, const T* __restrict__ in, T* __restrict__ out,
                                                        VEpi ep) {
    __shared__ T acc_s[kVMaxCols];
    __shared__ T red[4 * kVThreads];
    if (EPI == kVK1 || EPI == kVK2) {
        if (*(volatile int*)&ep.st->stop) return;
    }
    const int t = threadIdx.x;
    const VRow R = P.rows[P.order[blockIdx.x]];
    const int cols = R.cols;
    // taps summed in registers: a thread owns the outputs c = lt + To e (e < 4), To = the
    // row's columns / 4 rounded up to a warp (32 ... 256); the G = 256 / To groups of threads
    // split the taps, two taps in flight per thread, and their sums are added in group order
    const int q = (cols + 3) >> 2;
    const int To = q <= 32 ? 32 : (q >= kVThreads ? kVThreads : ((q + 31) & ~31));
    const int G = kVThreads / To;
    const int grp = t / To, lt = t - grp * To;
    T acc[4] = {0, 0, 0, 0};
    if (grp < G) {   // (threads past the last whole group, when To does not divide 256, idle)
        int i = R.t0 + grp;
        for (; i + G < R.t1; i += 2 * G) {
            const VTap t0 = P.taps[i], t1 = P.taps[i + G];
            const T v0 = tap_value<T>(P, i), v1 = tap_value<T>(P, i + G);
            reg_tap<T>(t0, v0, in, lt, To, cols, acc);
            reg_tap<T>(t1, v1, in, lt, To, cols, acc);
        }
        if (i < R.t1) reg_tap<T>(P.taps[i], tap_value<T>(P, i), in, lt, To, cols, acc);
    }
    if (G == 1) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = lt + To * e;
            if (c < cols) acc_s[c] = acc[e];
        }
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) red[e * kVThreads + t] = acc[e];
        __syncthreads();
        if (t < To) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = t + To * e;
                if (c < cols) {
                    T s = 0;
                    for (int g = 0; g < G; ++g) s += red[e * kVThreads + g * To + t];
                    acc_s[c] = s;
                }
            }
        }
    }
    __syncthreads();
    // taps of coarser inputs, one group per input level, phase by phase
    for (int g = R.g0; g < R.g1; ++g) {
        const VGroup gr = P.groups[g];
        for (int idx = t; idx < cols; idx += kVThreads) {
            const int p = idx / gr.cin, tq = idx - p * gr.cin;
            const int c = p + (tq << gr.lgr);
            const int e0 = P.ph[gr.ph0 + p], e1 = P.ph[gr.ph0 + p + 1];
            T s = 0;
            for (int i = e0; i < e1; ++i) {
                const VTap tp = P.taps[i];
                int d = c - tp.ox;
                if (d < 0) d += cols;
                s += tap_value<T>(P, i) * in[tp.in_off + (d >> gr.lgr)];
            }
            acc_s[c] += s;
        }
        __syncthreads();
    }
    // epilogue
    double p0 = 0.0, p1 = 0.0, p2 = 0.0;
    float beta = 0.f;
    if (EPI == kVK2) {
        const int k = ep.st->k;
        beta = ep.st->ista ? 0.f : (float)(k - 1) / (float)(k + 2);
    }
    const int mR = (1 << R.lgR) - 1;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int c = t + kVThreads * e;
        if (c >= cols) break;
        const long long i = R.out_off + c;
        const T a = acc_s[c];
        if (EPI == kVApply) {
            T o = a;
            if (ep.scale) o = (T)((double)o * ep.scale[R.cls_off + (c & mR)]);
            out[i] = o;
            p0 += (double)o * (double)o;
        } else if (EPI == kVK1 || EPI == kVObj) {
            const float xv = ep.x0[i];
            const float rv = (float)a - xv;
            if (EPI == kVK1) out[i] = (T)rv;
            p0 += (double)rv * (double)rv;
            if (EPI == kVK1) p1 += (double)xv * (double)rv;
            if (EPI == kVObj) {
                const float xi = ep.xl1[i];
                p1 += (double)ep.w_sb[R.sb] * (double)fabsf(xi);
                p2 += xi != 0.f ? 1.0 : 0.0;
            }
        } else if (EPI == kVK2) {
            const float gv = (float)a;
            const float stp = ep.step_tab[R.cls_off + (c & mR)];
            const float wv = ep.w_sb[R.sb];
            const float yv = ep.y[i], xo = ep.x[i];
            const float z = yv - stp * gv;
            const float xn = copysignf(fmaxf(fabsf(z) - stp * wv, 0.f), z);
            ep.x[i] = xn;
            ep.y[i] = xn + beta * (xn - xo);
            p0 += (double)wv * (double)fabsf(yv);
            p1 = fmax(p1, (double)gw_ratio(gv, wv));
        }
    }
    double v[3] = {p0, p1, p2}, tot[3];
    if (grid_reduce<3>(v, EPI == kVK2 ? 2u : 0u, ep.part, ep.counter, tot) && t == 0) {
        if (EPI == kVK1) {
            ep.st->rr = tot[0];
            ep.st->x0r = tot[1];
        } else if (EPI == kVK2) {
            finish_iteration(ep.st, tot[0], tot[1]);
        } else if (ep.red_out) {
            ep.red_out[0] = tot[0];
            ep.red_out[1] = tot[1];
            ep.red_out[2] = tot[2];
        }
    }
}

// out[i] = in[i] * tab[class of i], one CTA per row (FP64 power iteration)
__global__ void vrow_scale_kernel(VPlanDev P, const double* __restrict__ in, double* __restrict__ out,
                                  const double* __restrict__ tab) {
    const VRow R = P.rows[blockIdx.x];
    const int mR = (1 << R.lgR) - 1;
    for (int c = threadIdx.x; c < R.cols; c += blockDim.x)
        out[R.out_off + c] = in[R.out_off + c] * tab[R.cls_off + (c & mR)];
}

// ---------------------------------------------------------------------------------------
// Construction kernels
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int vmod(long long v, int n) {
    long long m = v % n;
    return (int)(m < 0 ? m + n : m);
}

// z on the window (wy0 + [0, wh)) x (wx0 + [0, ww)) (torus): H psi (transpose = 0) or H^T psi
// (1), psi[y, x] = Fv[(y - qshift) mod R] Fh[x mod C].
__global__ void probe_blur_kernel(const double* __restrict__ psfs, int kh, int kw, int R, int C,
                                  const double* __restrict__ Fv, const double* __restrict__ Fh, int qshift,
                                  int wy0, int wh, int wx0, int ww, int transpose, double* __restrict__ z) {
    const int ch = kh / 2, cw = kw / 2;
    const long long n = (long long)wh * ww;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int yy = (int)(e / ww), xx = (int)(e - (long long)yy * ww);
        const int y = vmod((long long)wy0 + yy, R), x = vmod((long long)wx0 + xx, C);
        double s = 0.0;
        for (int a = 0; a < kh; ++a) {
            // H: the input row y - (a - ch) spreads with its own PSF; H^T: the PSF of row y
            const int ys = transpose ? vmod((long long)y + (a - ch), R) : vmod((long long)y - (a - ch), R);
            const double fv = Fv[vmod((long long)ys - qshift, R)];
            if (fv == 0.0) continue;
            const double* __restrict__ prow = psfs + ((size_t)(transpose ? y : ys) * kh + a) * kw;
            double sb = 0.0;
            for (int b = 0; b < kw; ++b) {
                const int xs = transpose ? vmod((long long)x + (b - cw), C) : vmod((long long)x - (b - cw), C);
                sb += prow[b] * Fh[xs];
            }
            s += fv * sb;
        }
        z[(size_t)y * C + x] = s;
    }
}

__global__ void extract_kernel(const double* __restrict__ coef, const VSeg* __restrict__ segs, int s0,
                               const SubbandDev* __restrict__ sb, double* __restrict__ cand) {
    const VSeg g = segs[s0 + blockIdx.y];
    const SubbandDev d = sb[g.sub];
    const long long n = (long long)g.h * g.w;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / g.w), j = (int)(e - (long long)i * g.w);
        const int row = vmod((long long)g.r0 + i, d.rows), col = vmod((long long)g.c0 + j, d.cols);
        cand[g.base + e] = coef[d.off + (long long)row * d.cols + col];
    }
}

__global__ void zero_window_kernel(double* __restrict__ z, int R, int C, int wy0, int wh, int wx0, int ww) {
    const long long n = (long long)wh * ww;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int yy = (int)(e / ww), xx = (int)(e - (long long)yy * ww);
        z[(size_t)vmod((long long)wy0 + yy, R) * C + vmod((long long)wx0 + xx, C)] = 0.0;
    }
}

// selection over segments (one CTA per segment)
__global__ void vsel_vmax_kernel(const VSeg* __restrict__ segs, const double* __restrict__ cand, SelState* sel) {
    const VSeg g = segs[blockIdx.x];
    const long long n = (long long)g.h * g.w;
    double m = 0.0;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) m = fmax(m, fabs(cand[g.base + e]));
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(&sel->vmax_bits, (unsigned long long)__double_as_longlong(m));
}

__device__ __forceinline__ unsigned long long vsel_hi(double av, double sigma) {
    return ~(unsigned long long)__double_as_longlong(av * sigma);
}

__global__ void vsel_hist_kernel(const VSeg* __restrict__ segs, const double* __restrict__ cand, SelState* sel,
                                 int pass, unsigned long long* nz_count) {
    __shared__ unsigned long long h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0ull;
    __syncthreads();
    const VSeg g = segs[blockIdx.x];
    const long long n = (long long)g.h * g.w;
    const double thr = 1e-14 * __longlong_as_double((long long)sel->vmax_bits);
    const unsigned long long phi = sel->prefix_hi;
    const bool skip = sel->keep_all != 0;
    unsigned long long nz = 0;
    if (!skip || nz_count) {
        for (long long e = threadIdx.x; e < n; e += blockDim.x) {
            const double av = fabs(cand[g.base + e]);
            if (!(av > thr)) continue;
            ++nz;
            if (skip) continue;
            const unsigned long long hi = vsel_hi(av, g.sigma);
            if (pass > 0 && (hi >> (64 - 8 * pass)) != phi) continue;
            atomicAdd(&h[(int)((hi >> (56 - 8 * pass)) & 255ull)], g.mult);
        }
    }
    if (nz_count && nz) atomicAdd(nz_count, nz);
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(&sel->hist[i], h[i]);
}

// candidates at or above the boundary score (all with keep_all): flat index and value
__global__ void vsel_emit_kernel(const VSeg* __restrict__ segs, const double* __restrict__ cand, SelState* sel,
                                 long long* out_idx, double* out_v, unsigned long long cap) {
    const VSeg g = segs[blockIdx.x];
    const long long n = (long long)g.h * g.w;
    const double thr = 1e-14 * __longlong_as_double((long long)sel->vmax_bits);
    const unsigned long long phi = sel->prefix_hi;
    const bool all = sel->keep_all != 0;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) {
        const double v = cand[g.base + e];
        const double av = fabs(v);
        if (!(av > thr)) continue;
        if (!all && vsel_hi(av, g.sigma) > phi) continue;
        const unsigned long long slot = atomicAdd(&sel->count, 1ull);
        if (out_idx && slot < cap) {
            out_idx[slot] = g.base + e;
            out_v[slot] = v;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------------------
long long floor_half(long long a) { return a >= 0 ? a / 2 : -((-a + 1) / 2); }
long long ceil_half(long long a) { return -floor_half(-a); }

struct Iv {
    long long lo, hi;   // unwrapped, hi - lo + 1 <= n
};
Iv iv_make(long long lo, long long hi, long long n) {
    if (hi - lo + 1 >= n) return {0, n - 1};
    return {lo, hi};
}
// one analysis step: out[i] reads in[(2i + k) mod n], k < L
Iv iv_down(Iv x, int L, long long n_in) {
    const long long n_out = n_in / 2;
    if (x.hi - x.lo + 1 >= n_in) return {0, n_out - 1};
    return iv_make(ceil_half(x.lo - L + 1), floor_half(x.hi), n_out);
}

// 1-D synthesis function of a unit coefficient at position 0 of level s, first filter
// `high` ? g : h, then h down to level 0 (length n, periodic): out[(2i + k) mod n] += f[k] c[i]
std::vector<double> synth_1d(const Filters& f, int n, int s, bool high) {
    std::vector<double> c(n >> s, 0.0);
    c[0] = 1.0;
    for (int l = s; l >= 1; --l) {
        const int m = n >> (l - 1);
        std::vector<double> o(m, 0.0);
        const double* fk = (l == s && high) ? f.g : f.h;
        for (int i = 0; i < (int)c.size(); ++i) {
            if (c[i] == 0.0) continue;
            for (int k = 0; k < f.L; ++k) o[(2 * i + k) % m] += fk[k] * c[i];
        }
        c.swap(o);
    }
    return c;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Handle helpers
// ---------------------------------------------------------------------------------------
template <typename T>
static wdb_status vt_alloc(wdb_vtheta* op, T** p, size_t n) {
    void* q = nullptr;
    WDB_CK(cudaMalloc(&q, std::max<size_t>(n * sizeof(T), 1)));
    op->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return WDB_OK;
}

void vtheta_release(wdb_vtheta* op) {
    if (!op) return;
    if (op->work) cudaStreamSynchronize(op->work);
    for (auto& e : op->engine) e.release();
    if (op->work) cudaStreamDestroy(op->work);
    if (op->ev_in) cudaEventDestroy(op->ev_in);
    if (op->ev_out) cudaEventDestroy(op->ev_out);
    for (void* p : op->allocs) cudaFree(p);
    if (op->h_state) cudaFreeHost(op->h_state);
    delete op;
}

static int class_period_lg(const Layout& L, int b) { return L.J - L.sb[b].level; }

wdb_status vtheta_new(int n_rows, int n_cols, const char* wavelet, int levels, wdb_vtheta** out) {
    Layout L;
    WDB_TRY(make_layout(n_rows, n_cols, levels, &L));
    if (n_cols / 2 > kVMaxCols)
        return set_error(WDB_EUNSUPPORTED, "row-varying operator: rows of at most %d coefficients (n_cols <= %d)",
                         kVMaxCols, 2 * kVMaxCols);
    Filters f;
    WDB_TRY(wavelet_filters(wavelet, &f));
    wdb_vtheta* op = new (std::nothrow) wdb_vtheta();
    if (!op) return set_error(WDB_ENOMEM, "host allocation");
    op->lay = L;
    op->filt = f;
    op->wavelet = wavelet;
    op->cls_off.assign(L.S + 1, 0);
    for (int b = 0; b < L.S; ++b)
        op->cls_off[b + 1] = op->cls_off[b] + L.sb[b].rows * (1 << class_period_lg(L, b));
    op->n_classes = op->cls_off[L.S];
    *out = op;
    return WDB_OK;
}

// ---------------------------------------------------------------------------------------
// Row plans
// ---------------------------------------------------------------------------------------
static void build_plan(const wdb_vtheta* op, bool adj, VPlanHost& P) {
    const Layout& L = op->lay;
    // rows in planar order: (subband, row)
    std::vector<int> row_base(L.S + 1, 0);
    for (int b = 0; b < L.S; ++b) row_base[b + 1] = row_base[b] + L.sb[b].rows;
    const int nrows = row_base[L.S];
    struct E1 { int row; long long in_off; int ox; int mode; double v; };
    struct E2 { int row; int lgr; int cin; int ph; long long in_off; int ox; double v; };
    std::vector<E1> e1;
    std::vector<E2> e2;
    for (const VTapH& t : op->taps) {
        const SubbandDev &sa = L.sb[t.a], &sb = L.sb[t.b];
        // forward: output (a, py), input (b, qy); transposed: output (b, qy), input (a, py)
        const int o_sub = adj ? t.b : t.a, o_row = adj ? t.qy : t.py;
        const int i_sub = adj ? t.a : t.b, i_row = adj ? t.py : t.qy;
        const SubbandDev& si = L.sb[i_sub];
        const long long in_off = si.off + (long long)i_row * si.cols;
        const int row = row_base[o_sub] + o_row;
        const bool colform = sa.level <= sb.level;
        if (!adj) {
            if (!colform) e1.push_back({row, in_off, t.ox, sa.level - sb.level, t.v});          // input finer
            else if (sa.level == sb.level) e1.push_back({row, in_off, t.ox, kVTapU, t.v});      // same level
            else {
                const int lgr = sb.level - sa.level;
                e2.push_back({row, lgr, sb.cols, t.ox & ((1 << lgr) - 1), in_off, t.ox, t.v}); // input coarser
            }
        } else {
            if (colform) e1.push_back({row, in_off, t.ox, sb.level - sa.level, t.v});           // input a finer/same
            else {
                const int lgr = sa.level - sb.level;
                e2.push_back({row, lgr, sa.cols, t.ox & ((1 << lgr) - 1), in_off, t.ox, t.v});
            }
        }
    }
    std::sort(e1.begin(), e1.end(), [](const E1& x, const E1& y) {
        return std::tie(x.row, x.in_off, x.ox) < std::tie(y.row, y.in_off, y.ox);
    });
    std::sort(e2.begin(), e2.end(), [](const E2& x, const E2& y) {
        return std::tie(x.row, x.lgr, x.ph, x.in_off, x.ox) < std::tie(y.row, y.lgr, y.ph, y.in_off, y.ox);
    });
    P = VPlanHost();
    P.rows.resize(nrows);
    std::vector<double> work(nrows, 0.0);
    size_t i1 = 0, i2 = 0;
    for (int b = 0; b < L.S; ++b) {
        const SubbandDev& s = L.sb[b];
        for (int r = 0; r < s.rows; ++r) {
            const int row = row_base[b] + r;
            VRow& R = P.rows[row];
            R.out_off = s.off + (long long)r * s.cols;
            R.cols = s.cols;
            R.sb = b;
            R.lgR = class_period_lg(L, b);
            R.cls_off = op->cls_off[b] + r * (1 << R.lgR);
            R.t0 = (int)P.taps.size();
            for (; i1 < e1.size() && e1[i1].row == row; ++i1) {
                P.taps.push_back({(int)e1[i1].in_off, e1[i1].ox, e1[i1].mode, 0});
                P.v64.push_back(e1[i1].v);
            }
            R.t1 = (int)P.taps.size();
            R.g0 = (int)P.groups.size();
            double w2 = 0.0;
            while (i2 < e2.size() && e2[i2].row == row) {
                const int lgr = e2[i2].lgr, nph = 1 << lgr;
                VGroup g{lgr, e2[i2].cin, (int)P.ph.size(), 0};
                std::vector<int> starts(nph + 1, 0);
                const int first = (int)P.taps.size();
                int cur = 0;
                for (; i2 < e2.size() && e2[i2].row == row && e2[i2].lgr == lgr; ++i2) {
                    while (cur <= e2[i2].ph) starts[cur++] = (int)P.taps.size();
                    P.taps.push_back({(int)e2[i2].in_off, e2[i2].ox, lgr, 0});
                    P.v64.push_back(e2[i2].v);
                }
                while (cur <= nph) starts[cur++] = (int)P.taps.size();
                P.ph.insert(P.ph.end(), starts.begin(), starts.end());
                w2 += (double)(P.taps.size() - first) / nph;
                P.groups.push_back(g);
            }
            R.g1 = (int)P.groups.size();
            work[row] = (double)s.cols * ((R.t1 - R.t0) + w2 + 2.0);
        }
    }
    P.v32.assign(P.v64.begin(), P.v64.end());
    P.order.resize(nrows);
    std::iota(P.order.begin(), P.order.end(), 0);
    std::stable_sort(P.order.begin(), P.order.end(), [&](int x, int y) { return work[x] > work[y]; });
}

// Host emulation of one application through the row plan, with the kernel's index arithmetic
// and a bounds check of every access (no GPU): y = Theta_K x (adj = 0) or Theta_K^T x.
wdb_status vtheta_plan_emulate(const wdb_vtheta* op, bool adj, const double* x, double* y) {
    const Layout& L = op->lay;
    VPlanHost P;
    build_plan(op, adj, P);
    const long long N = L.N;
    std::vector<int> seen(N, 0);
    if ((long long)P.order.size() != (long long)P.rows.size()) return set_error(WDB_EPLAN, "order size");
    std::vector<int> in_order(P.rows.size(), 0);
    for (int r : P.order) {
        if (r < 0 || r >= (int)P.rows.size() || in_order[r]++) return set_error(WDB_EPLAN, "order is not a permutation");
    }
    for (size_t ri = 0; ri < P.rows.size(); ++ri) {
        const VRow& R = P.rows[ri];
        const int cols = R.cols;
        if (cols < 1 || cols > kVMaxCols) return set_error(WDB_EPLAN, "row %zu: %d columns", ri, cols);
        if (R.out_off < 0 || R.out_off + cols > N) return set_error(WDB_EPLAN, "row %zu outside the vector", ri);
        if (R.cls_off < 0 || R.cls_off + (1 << R.lgR) > op->n_classes || (1 << R.lgR) > cols)
            return set_error(WDB_EPLAN, "row %zu: class range", ri);
        if (R.t0 < 0 || R.t1 < R.t0 || R.t1 > (int)P.taps.size() || R.g0 < 0 || R.g1 < R.g0 ||
            R.g1 > (int)P.groups.size())
            return set_error(WDB_EPLAN, "row %zu: tap or group range", ri);
        std::vector<double> acc(cols, 0.0);
        for (int c = 0; c < cols; ++c) {
            if (seen[R.out_off + c]++) return set_error(WDB_EPLAN, "output %lld twice", R.out_off + c);
            double a = 0.0;
            for (int i = R.t0; i < R.t1; ++i) {
                const VTap& tp = P.taps[i];
                long long ci;
                if (tp.mode & kVTapU) {
                    if (tp.ox < 0 || tp.ox >= cols) return set_error(WDB_EPLAN, "tap %d: ox", i);
                    ci = c - tp.ox;
                    if (ci < 0) ci += cols;
                    if (ci < 0 || ci >= cols) return set_error(WDB_EPLAN, "tap %d: index", i);
                } else {
                    const int lgr = tp.mode & 255;
                    const long long cin = (long long)cols << lgr;
                    if (tp.ox < 0 || tp.ox >= cin) return set_error(WDB_EPLAN, "tap %d: ox", i);
                    ci = tp.ox + ((long long)c << lgr);
                    if (ci >= cin) ci -= cin;
                    if (ci < 0 || ci >= cin) return set_error(WDB_EPLAN, "tap %d: index", i);
                }
                if (tp.in_off < 0 || tp.in_off + ci >= N) return set_error(WDB_EPLAN, "tap %d reads outside", i);
                a += P.v64[i] * x[tp.in_off + ci];
            }
            acc[c] = a;
        }
        for (int g = R.g0; g < R.g1; ++g) {
            const VGroup& gr = P.groups[g];
            const int r = 1 << gr.lgr;
            if (gr.lgr < 1 || (long long)gr.cin * r != cols) return set_error(WDB_EPLAN, "group %d: shape", g);
            if (gr.ph0 < 0 || gr.ph0 + r >= (int)P.ph.size()) return set_error(WDB_EPLAN, "group %d: phases", g);
            std::vector<int> hit(cols, 0);
            for (int idx = 0; idx < cols; ++idx) {
                const int p = idx / gr.cin, tq = idx - p * gr.cin;
                const int c = p + (tq << gr.lgr);
                if (c < 0 || c >= cols || hit[c]++) return set_error(WDB_EPLAN, "group %d: output map", g);
                const int e0 = P.ph[gr.ph0 + p], e1 = P.ph[gr.ph0 + p + 1];
                if (e0 < R.t1 || e1 < e0 || e1 > (int)P.taps.size()) return set_error(WDB_EPLAN, "group %d: phase list", g);
                double s = 0.0;
                for (int i = e0; i < e1; ++i) {
                    const VTap& tp = P.taps[i];
                    if (tp.ox < 0 || tp.ox >= cols || (tp.ox & (r - 1)) != p)
                        return set_error(WDB_EPLAN, "tap %d: phase %d", i, p);
                    int d = c - tp.ox;
                    if (d < 0) d += cols;
                    if (d < 0 || (d & (r - 1)) || (d >> gr.lgr) >= gr.cin) return set_error(WDB_EPLAN, "tap %d: index", i);
                    if (tp.in_off < 0 || tp.in_off + (d >> gr.lgr) >= N) return set_error(WDB_EPLAN, "tap %d reads outside", i);
                    s += P.v64[i] * x[tp.in_off + (d >> gr.lgr)];
                }
                acc[c] += s;
            }
        }
        for (int c = 0; c < cols; ++c) y[R.out_off + c] = acc[c];
    }
    for (long long i = 0; i < N; ++i)
        if (seen[i] != 1) return set_error(WDB_EPLAN, "output %lld not produced", i);
    return WDB_OK;
}

template <typename T>
static wdb_status upload_vec(wdb_vtheta* op, const std::vector<T>& h, const T** d, cudaStream_t st) {
    T* p = nullptr;
    WDB_TRY(vt_alloc(op, &p, h.size()));
    if (!h.empty()) WDB_CK(cudaMemcpyAsync(p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st));
    *d = p;
    return WDB_OK;
}

wdb_status vtheta_finalize(wdb_vtheta* op, cudaStream_t st) {
    const Layout& L = op->lay;
    long long keff = 0;
    for (const VTapH& t : op->taps) keff += std::min(L.sb[t.a].cols, L.sb[t.b].cols);
    op->K_eff = keff;
    for (int adj = 0; adj < 2; ++adj) {
        build_plan(op, adj != 0, op->hplan[adj]);
        const VPlanHost& H = op->hplan[adj];
        VPlanDev& D = op->plan[adj];
        WDB_TRY(upload_vec(op, H.rows, &D.rows, st));
        WDB_TRY(upload_vec(op, H.order, &D.order, st));
        WDB_TRY(upload_vec(op, H.taps, &D.taps, st));
        WDB_TRY(upload_vec(op, H.v32, &D.v32, st));
        WDB_TRY(upload_vec(op, H.v64, &D.v64, st));
        WDB_TRY(upload_vec(op, H.groups, &D.groups, st));
        WDB_TRY(upload_vec(op, H.ph, &D.ph, st));
        D.n_rows = (int)H.rows.size();
    }
    op->grid = op->plan[0].n_rows;
    WDB_TRY(vt_alloc(op, &op->d_part, (size_t)op->grid * 3));
    WDB_TRY(vt_alloc(op, &op->d_counter, 4));
    WDB_CK(cudaMemsetAsync(op->d_counter, 0, sizeof(unsigned int) * 4, st));
    WDB_TRY(vt_alloc(op, &op->d_red, 4));
    WDB_CK(cudaStreamSynchronize(st));
    return WDB_OK;
}

// ---------------------------------------------------------------------------------------
// Construction (probes + selection)
// ---------------------------------------------------------------------------------------
wdb_status vtheta_build_device(wdb_vtheta* op, const double* psfs_host, int kh, int kw, long long K, int rule,
                               cudaStream_t st) {
    const Layout& L = op->lay;
    const Filters& f = op->filt;
    const int R = L.n_rows, C = L.n_cols, J = L.J, S = L.S;
    const long long N = L.N;
    const int ch = kh / 2, cw = kw / 2;
    // 1-D synthesis functions per (level, low/high) for both axes
    std::vector<double> Fv_h, Fh_h;
    std::vector<int> fv_off(2 * (J + 1), 0), fh_off(2 * (J + 1), 0);
    for (int s = 1; s <= J; ++s)
        for (int e = 0; e < 2; ++e) {
            fv_off[2 * s + e] = (int)Fv_h.size();
            auto v = synth_1d(f, R, s, e == 1);
            Fv_h.insert(Fv_h.end(), v.begin(), v.end());
            fh_off[2 * s + e] = (int)Fh_h.size();
            auto h = synth_1d(f, C, s, e == 1);
            Fh_h.insert(Fh_h.end(), h.begin(), h.end());
        }
    // probes and their candidate windows
    struct Probe {
        int kind, sub, row;     // 0: column probe of (sub, row); 1: row probe
        Iv zy, zx;              // window of H psi / H^T psi
        int seg0, seg1;
    };
    std::vector<Probe> probes;
    std::vector<VSeg> segs;
    long long base = 0;
    auto add_probe = [&](int kind, int sub, int row) {
        const SubbandDev& sd = L.sb[sub];
        const long long step = 1LL << sd.level, span = (long long)(f.L - 1) * (step - 1);
        const Iv py = iv_make(row * step, row * step + span, R), px = iv_make(0, span, C);
        Probe p{kind, sub, row, iv_make(py.lo - ch, py.hi + ch, R), iv_make(px.lo - cw, px.hi + cw, C),
                (int)segs.size(), 0};
        Iv wy = p.zy, wx = p.zx;
        long long nr = R, nc = C;
        for (int s = 1; s <= J; ++s) {
            wy = iv_down(wy, f.L, nr);
            wx = iv_down(wx, f.L, nc);
            nr /= 2;
            nc /= 2;
            for (int o = 0; o < S; ++o) {
                const SubbandDev& so = L.sb[o];
                if (so.level != s) continue;
                // column probe of b: outputs a with s_a <= s_b; row probe of a: inputs b with s_b < s_a
                const bool use = kind == 0 ? so.level <= sd.level : so.level < sd.level;
                if (!use) continue;
                VSeg g{};
                g.base = base;
                g.sub = o;
                g.r0 = (int)(((wy.lo % so.rows) + so.rows) % so.rows);
                g.h = (int)(wy.hi - wy.lo + 1);
                g.c0 = (int)(((wx.lo % so.cols) + so.cols) % so.cols);
                g.w = (int)(wx.hi - wx.lo + 1);
                g.kind = kind;
                g.fixed_sub = sub;
                g.fixed_row = row;
                const int a = kind == 0 ? o : sub, b = kind == 0 ? sub : o;
                g.mult = (unsigned long long)std::min(L.sb[a].cols, L.sb[b].cols);
                g.sigma = rule == WDB_RULE_NAIVE ? 1.0 : std::ldexp(1.0, L.sb[b].level);
                base += (long long)g.h * g.w;
                segs.push_back(g);
            }
        }
        p.seg1 = (int)segs.size();
        probes.push_back(p);
    };
    for (int b = 0; b < S; ++b)
        for (int q = 0; q < L.sb[b].rows; ++q) add_probe(0, b, q);
    for (int a = 0; a < S; ++a)
        if (L.sb[a].level > 1)
            for (int q = 0; q < L.sb[a].rows; ++q) add_probe(1, a, q);
    op->n_probes = (int)probes.size();
    op->n_cand_slots = base;
    // device scratch
    std::vector<void*> tmp;
    auto dmalloc = [&](void** p, size_t bytes) -> wdb_status {
        WDB_CK(cudaMalloc(p, std::max<size_t>(bytes, 1)));
        tmp.push_back(*p);
        return WDB_OK;
    };
    wdb_status s = WDB_OK;
    do {
        double *d_psf = nullptr, *d_Fv = nullptr, *d_Fh = nullptr, *z = nullptr, *coef = nullptr, *scr = nullptr,
               *cand = nullptr;
        VSeg* d_seg = nullptr;
        SubbandDev* d_sb = nullptr;
        SelState* d_sel = nullptr;
        unsigned long long* d_nz = nullptr;
        if ((s = dmalloc((void**)&d_psf, sizeof(double) * (size_t)R * kh * kw))) break;
        if ((s = dmalloc((void**)&d_Fv, sizeof(double) * Fv_h.size()))) break;
        if ((s = dmalloc((void**)&d_Fh, sizeof(double) * Fh_h.size()))) break;
        if ((s = dmalloc((void**)&z, sizeof(double) * N))) break;
        if ((s = dmalloc((void**)&coef, sizeof(double) * N))) break;
        if ((s = dmalloc((void**)&scr, sizeof(double) * (N / 2 + 1)))) break;
        if ((s = dmalloc((void**)&cand, sizeof(double) * (size_t)base))) break;
        if ((s = dmalloc((void**)&d_seg, sizeof(VSeg) * segs.size()))) break;
        if ((s = dmalloc((void**)&d_sb, sizeof(SubbandDev) * S))) break;
        if ((s = dmalloc((void**)&d_sel, sizeof(SelState)))) break;
        if ((s = dmalloc((void**)&d_nz, sizeof(unsigned long long)))) break;
        cudaMemcpyAsync(d_psf, psfs_host, sizeof(double) * (size_t)R * kh * kw, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_Fv, Fv_h.data(), sizeof(double) * Fv_h.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_Fh, Fh_h.data(), sizeof(double) * Fh_h.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_seg, segs.data(), sizeof(VSeg) * segs.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_sb, L.sb, sizeof(SubbandDev) * S, cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(z, 0, sizeof(double) * N, st);
        for (const Probe& p : probes) {
            const SubbandDev& sd = L.sb[p.sub];
            const int ey = (sd.level == J && p.sub == 0) ? 0 : (p.sub - 1) % 3 == 0 ? 0 : 1;
            const int ex = (p.sub == 0) ? 0 : (p.sub - 1) % 3 == 1 ? 0 : 1;
            const int wh = (int)(p.zy.hi - p.zy.lo + 1), ww = (int)(p.zx.hi - p.zx.lo + 1);
            const int wy0 = (int)p.zy.lo, wx0 = (int)p.zx.lo;
            const long long n = (long long)wh * ww;
            const int g = (int)std::min<long long>((n + 255) / 256, 4096);
            probe_blur_kernel<<<g, 256, 0, st>>>(d_psf, kh, kw, R, C, d_Fv + fv_off[2 * sd.level + ey],
                                                 d_Fh + fh_off[2 * sd.level + ex], p.row << sd.level, wy0, wh, wx0,
                                                 ww, p.kind, z);
            count_launch();
            if ((s = dwt2<double>(z, coef, L, f, scr, st))) break;
            if (p.seg1 > p.seg0) {
                long long mx = 1;
                for (int q = p.seg0; q < p.seg1; ++q) mx = std::max(mx, (long long)segs[q].h * segs[q].w);
                dim3 eg((unsigned)std::min<long long>((mx + 255) / 256, 1024), (unsigned)(p.seg1 - p.seg0));
                extract_kernel<<<eg, 256, 0, st>>>(coef, d_seg, p.seg0, d_sb, cand);
                count_launch();
            }
            zero_window_kernel<<<g, 256, 0, st>>>(z, R, C, wy0, wh, wx0, ww);
            count_launch();
        }
        if (s) break;
        cudaError_t ce = cudaGetLastError();
        if (ce != cudaSuccess) { s = cuda_error(ce, "probes", __FILE__, __LINE__); break; }
        // selection over the score digits
        SelState h0;
        std::memset(&h0, 0, sizeof h0);
        h0.K = (unsigned long long)std::max<long long>(K, 0);
        cudaMemcpyAsync(d_sel, &h0, sizeof h0, cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(d_nz, 0, sizeof(unsigned long long), st);
        const unsigned nseg = (unsigned)segs.size();
        vsel_vmax_kernel<<<nseg, 256, 0, st>>>(d_seg, cand, d_sel);
        count_launch();
        for (int pass = 0; pass < 8; ++pass) {
            vsel_hist_kernel<<<nseg, 256, 0, st>>>(d_seg, cand, d_sel, pass, pass == 0 ? d_nz : nullptr);
            sel_scan_kernel<<<1, 32, 0, st>>>(d_sel, pass);
            count_launch(2);
        }
        vsel_emit_kernel<<<nseg, 256, 0, st>>>(d_seg, cand, d_sel, nullptr, nullptr, 0);
        count_launch();
        SelState hs;
        unsigned long long nz = 0;
        ce = cudaMemcpyAsync(&hs, d_sel, sizeof hs, cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(&nz, d_nz, sizeof nz, cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce == cudaSuccess) ce = cudaGetLastError();
        if (ce != cudaSuccess) { s = cuda_error(ce, "tap selection", __FILE__, __LINE__); break; }
        std::memcpy(&op->theta_max_abs, &hs.vmax_bits, sizeof(double));
        op->n_candidates = (long long)nz;
        const unsigned long long ne = hs.count;
        long long* d_idx = nullptr;
        double* d_v = nullptr;
        if ((s = dmalloc((void**)&d_idx, sizeof(long long) * ne))) break;
        if ((s = dmalloc((void**)&d_v, sizeof(double) * ne))) break;
        cudaMemsetAsync(&d_sel->count, 0, sizeof(unsigned long long), st);
        vsel_emit_kernel<<<nseg, 256, 0, st>>>(d_seg, cand, d_sel, d_idx, d_v, ne);
        count_launch();
        std::vector<long long> hidx(ne);
        std::vector<double> hv(ne);
        if (ne) {
            cudaMemcpyAsync(hidx.data(), d_idx, sizeof(long long) * ne, cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(hv.data(), d_v, sizeof(double) * ne, cudaMemcpyDeviceToHost, st);
        }
        ce = cudaStreamSynchronize(st);
        if (ce == cudaSuccess) ce = cudaGetLastError();
        if (ce != cudaSuccess) { s = cuda_error(ce, "tap emit", __FILE__, __LINE__); break; }
        // taps; the boundary score's ties in (a, py, b, qy, ox) order while the count fits
        std::vector<VTapH> above, ties;
        const unsigned long long bound_hi = hs.prefix_hi;
        for (unsigned long long k = 0; k < ne; ++k) {
            const long long e = hidx[k];
            const int q = (int)(std::upper_bound(segs.begin(), segs.end(), e,
                                                 [](long long x, const VSeg& g) { return x < g.base; }) -
                                segs.begin()) - 1;
            const VSeg& g = segs[q];
            const long long loc = e - g.base;
            const int i = (int)(loc / g.w), j = (int)(loc % g.w);
            const SubbandDev& so = L.sb[g.sub];
            const int orow = (g.r0 + i) % so.rows, ocol = (g.c0 + j) % so.cols;
            VTapH t;
            if (g.kind == 0) t = {g.sub, orow, g.fixed_sub, g.fixed_row, ocol, hv[k]};
            else t = {g.fixed_sub, g.fixed_row, g.sub, orow, ocol, hv[k]};
            double sc = std::fabs(hv[k]) * g.sigma;
            unsigned long long hi;
            std::memcpy(&hi, &sc, sizeof hi);
            hi = ~hi;
            if (!hs.keep_all && hi == bound_hi) ties.push_back(t);
            else above.push_back(t);
        }
        auto key = [](const VTapH& t) { return std::tie(t.a, t.py, t.b, t.qy, t.ox); };
        std::sort(ties.begin(), ties.end(), [&](const VTapH& x, const VTapH& y) { return key(x) < key(y); });
        unsigned long long cnt = hs.before;
        for (const VTapH& t : ties) {
            const unsigned long long m = (unsigned long long)std::min(L.sb[t.a].cols, L.sb[t.b].cols);
            if (cnt + m > h0.K) break;
            cnt += m;
            above.push_back(t);
        }
        std::sort(above.begin(), above.end(), [&](const VTapH& x, const VTapH& y) { return key(x) < key(y); });
        op->taps.swap(above);
    } while (false);
    cudaStreamSynchronize(st);
    for (void* p : tmp) cudaFree(p);
    return s;
}

// ---------------------------------------------------------------------------------------
// Operator applications
// ---------------------------------------------------------------------------------------
template <typename T, int EPI>
static wdb_status launch_vrow(const wdb_vtheta* op, bool adj, const T* in, T* out, const VEpi& ep, cudaStream_t st) {
    const VPlanDev& P = op->plan[adj ? 1 : 0];
    vrow_kernel<T, EPI><<<P.n_rows, kVThreads, 0, st>>>(P, in, out, ep);
    count_launch();
    WDB_CK(cudaGetLastError());
    return WDB_OK;
}

static VEpi oneoff_epi(const wdb_vtheta* op) {
    VEpi ep{};
    ep.part = op->d_part;
    ep.counter = op->d_counter;
    ep.red_out = op->d_red;
    return ep;
}

wdb_status vtheta_apply(const wdb_vtheta* op, const float* in, float* out, bool adj, cudaStream_t st) {
    return launch_vrow<float, kVApply>(op, adj, in, out, oneoff_epi(op), st);
}

// ---------------------------------------------------------------------------------------
// Preconditioner: diag(M), diag(M^2) per class on the host (FP64), step on the device
// ---------------------------------------------------------------------------------------
static void diag_tables(wdb_vtheta* op) {
    const Layout& L = op->lay;
    // forward rows (a, py) and columns (b, qy) of the tap list
    std::vector<int> row_base(L.S + 1, 0);
    for (int b = 0; b < L.S; ++b) row_base[b + 1] = row_base[b] + L.sb[b].rows;
    const int nrows = row_base[L.S];
    std::vector<std::vector<int>> by_out(nrows), by_in(nrows);
    for (int i = 0; i < (int)op->taps.size(); ++i) {
        const VTapH& t = op->taps[i];
        by_out[row_base[t.a] + t.py].push_back(i);
        by_in[row_base[t.b] + t.qy].push_back(i);
    }
    const int nc = op->n_classes;
    op->Md.assign(nc, 0.0);
    op->M2d.assign(nc, 0.0);
    // class list
    struct Cls { int b, qy, p, idx; };
    std::vector<Cls> cls;
    cls.reserve(nc);
    for (int b = 0; b < L.S; ++b) {
        const int Rb = 1 << class_period_lg(L, b);
        for (int qy = 0; qy < L.sb[b].rows; ++qy)
            for (int p = 0; p < Rb; ++p) cls.push_back({b, qy, p, op->cls_off[b] + qy * Rb + p});
    }
    auto worker = [&](int lo, int hi, std::vector<double>& acc, std::vector<long long>& touched,
                      std::vector<std::pair<long long, double>>& col) {
        for (int ci = lo; ci < hi; ++ci) {
            const Cls& c = cls[ci];
            const SubbandDev& sb = L.sb[c.b];
            const int qx = c.p;
            // column (b, qy, qx) of Theta_K
            col.clear();
            for (int i : by_in[row_base[c.b] + c.qy]) {
                const VTapH& t = op->taps[i];
                const SubbandDev& sa = L.sb[t.a];
                if (sa.level <= sb.level) {
                    const int r = 1 << (sb.level - sa.level);
                    const int px = (int)(((long long)t.ox + (long long)r * qx) % sa.cols);
                    col.push_back({sa.off + (long long)t.py * sa.cols + px, t.v});
                } else {
                    const int r = 1 << (sa.level - sb.level);
                    int d = qx - t.ox;
                    d %= sb.cols;
                    if (d < 0) d += sb.cols;
                    if (d % r) continue;
                    col.push_back({sa.off + (long long)t.py * sa.cols + d / r, t.v});
                }
            }
            double md = 0.0;
            for (auto& e : col) md += e.second * e.second;
            // M e_mu = Theta_K^T (column): rows of Theta_K at the column's outputs
            for (auto& e : col) {
                const long long lam = e.first;
                int a = 0;
                while (a + 1 < L.S && lam >= L.sb[a + 1].off) ++a;
                const SubbandDev& sa = L.sb[a];
                const int py = (int)((lam - sa.off) / sa.cols), px = (int)((lam - sa.off) % sa.cols);
                for (int i : by_out[row_base[a] + py]) {
                    const VTapH& t = op->taps[i];
                    const SubbandDev& s2 = L.sb[t.b];
                    long long mu2;
                    if (sa.level <= s2.level) {
                        const int r = 1 << (s2.level - sa.level);
                        int d = px - t.ox;
                        if (d < 0) d += sa.cols;
                        if (d % r) continue;
                        mu2 = s2.off + (long long)t.qy * s2.cols + d / r;
                    } else {
                        const int r = 1 << (sa.level - s2.level);
                        mu2 = s2.off + (long long)t.qy * s2.cols + (int)(((long long)t.ox + (long long)r * px) % s2.cols);
                    }
                    if (acc[mu2] == 0.0) touched.push_back(mu2);
                    acc[mu2] += e.second * t.v;
                }
            }
            double m2 = 0.0;
            for (long long m : touched) {
                m2 += acc[m] * acc[m];
                acc[m] = 0.0;
            }
            touched.clear();
            op->Md[c.idx] = md;
            op->M2d[c.idx] = m2;
        }
    };
    const int nt = std::max(1, std::min<int>((int)std::thread::hardware_concurrency(), 32));
    const int n = (int)cls.size();
    // classes in chunks from a shared counter (coarse subbands, first in planar order, are heavier)
    std::vector<std::thread> th;
    const int chunk = std::max(1, n / (nt * 8));
    std::atomic<int> next{0};
    for (int k = 0; k < nt; ++k)
        th.emplace_back([&]() {
            std::vector<double> acc(L.N, 0.0);
            std::vector<long long> touched;
            std::vector<std::pair<long long, double>> col;
            for (;;) {
                const int lo = next.fetch_add(chunk);
                if (lo >= n) break;
                worker(lo, std::min(n, lo + chunk), acc, touched, col);
            }
        });
    for (auto& x : th) x.join();
    op->diag_valid = true;
}

static wdb_status vt_power(wdb_vtheta* op, const std::vector<double>& P, cudaStream_t st, double* L_out) {
    const long long N = op->lay.N;
    std::vector<double> sc(P.size());
    for (size_t i = 0; i < sc.size(); ++i) sc[i] = 1.0 / std::sqrt(P[i]);
    std::vector<void*> tmp;
    auto dm = [&](void** p, size_t b) -> wdb_status {
        WDB_CK(cudaMalloc(p, std::max<size_t>(b, 1)));
        tmp.push_back(*p);
        return WDB_OK;
    };
    double *v = nullptr, *t = nullptr, *u = nullptr, *d_sc = nullptr;
    wdb_status s = WDB_OK;
    double lam = 0.0;
    do {
        if ((s = dm((void**)&v, sizeof(double) * N))) break;
        if ((s = dm((void**)&t, sizeof(double) * N))) break;
        if ((s = dm((void**)&u, sizeof(double) * N))) break;
        if ((s = dm((void**)&d_sc, sizeof(double) * sc.size()))) break;
        cudaMemcpyAsync(d_sc, sc.data(), sizeof(double) * sc.size(), cudaMemcpyHostToDevice, st);
        RedTarget red{op->d_counter + 1, op->d_part, op->d_red + 3};
        const int grid = std::min(op->grid, 1216);
        if ((s = launch_splitmix<double>(v, N, kPowerSeed, st))) break;
        if ((s = launch_norm2<double>(v, N, red, grid, st))) break;
        double h = 0.0;
        cudaMemcpyAsync(&h, op->d_red + 3, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) { s = set_error(WDB_ECUDA, "power start"); break; }
        if ((s = launch_scale_const<double>(v, v, N, 1.0 / std::sqrt(h), st))) break;
        VEpi ep = oneoff_epi(op);
        ep.red_out = nullptr;
        VEpi eps = oneoff_epi(op);
        eps.scale = d_sc;
        for (int it = 1; it <= kPowerIters; ++it) {
            vrow_scale_kernel<<<op->plan[0].n_rows, 256, 0, st>>>(op->plan[0], v, t, d_sc);
            count_launch();
            if ((s = (launch_vrow<double, kVApply>(op, false, t, u, ep, st)))) break;
            if ((s = (launch_vrow<double, kVApply>(op, true, u, t, eps, st)))) break;   // also ||t||^2
            cudaMemcpyAsync(&h, op->d_red, sizeof(double), cudaMemcpyDeviceToHost, st);
            cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) { s = cuda_error(e, "power iteration", __FILE__, __LINE__); break; }
            const double ln = std::sqrt(h);
            if (!(ln > 0.0) || !std::isfinite(ln)) { lam = ln; break; }
            if ((s = launch_scale_const<double>(t, v, N, 1.0 / ln, st))) break;
            const bool done = std::fabs(ln - lam) <= kPowerRtol * ln;
            lam = ln;
            if (done) break;
        }
    } while (false);
    cudaStreamSynchronize(st);
    for (void* p : tmp) cudaFree(p);
    if (s) return s;
    if (!std::isfinite(lam)) return set_error(WDB_ENAN, "power iteration produced %g", lam);
    *L_out = lam;
    return WDB_OK;
}

static wdb_status vt_precond_upload(wdb_vtheta* op, PrecondCache& pc) {
    if (!pc.d_step) WDB_TRY(vt_alloc(op, &pc.d_step, pc.P.size()));
    std::vector<float> stp(pc.P.size());
    for (size_t i = 0; i < stp.size(); ++i) stp[i] = (float)(pc.tau / pc.P[i]);
    WDB_CK(cudaMemcpy(pc.d_step, stp.data(), sizeof(float) * stp.size(), cudaMemcpyHostToDevice));
    return WDB_OK;
}

wdb_status vtheta_precond(wdb_vtheta* op, int kind, double eps, cudaStream_t st) {
    if (kind < 0 || kind > 2) return set_error(WDB_EINVAL, "unknown preconditioner %d", kind);
    PrecondCache& pc = op->pc[kind];
    if (pc.valid && (pc.pinned || kind != WDB_PRECOND_JACOBI || pc.eps == eps)) return WDB_OK;
    if (!op->diag_valid) diag_tables(op);
    pc.P = precond_table(op->Md, op->M2d, kind, eps);
    double Lh = 0.0;
    WDB_TRY(vt_power(op, pc.P, st, &Lh));
    pc.L_hat = Lh;
    pc.tau = Lh > 0.0 ? 1.0 / (kStepMargin * Lh) : 1.0;
    pc.eps = eps;
    WDB_TRY(vt_precond_upload(op, pc));
    pc.valid = true;
    for (auto& e : op->engine) e.release();
    return WDB_OK;
}

wdb_status vtheta_set_precond(wdb_vtheta* op, int kind, const double* P, double tau) {
    PrecondCache& pc = op->pc[kind];
    pc.P.assign(P, P + op->n_classes);
    pc.tau = tau;
    pc.L_hat = 1.0 / (kStepMargin * tau);
    WDB_TRY(vt_precond_upload(op, pc));
    pc.valid = true;
    pc.pinned = true;
    return WDB_OK;
}

// ---------------------------------------------------------------------------------------
// Solve (Algorithm 3)
// ---------------------------------------------------------------------------------------
static wdb_status vt_workspace(wdb_vtheta* op) {
    if (op->d_state) return WDB_OK;
    const long long N = op->lay.N;
    WDB_TRY(vt_alloc(op, &op->d_x0, N));
    WDB_TRY(vt_alloc(op, &op->d_y, N));
    WDB_TRY(vt_alloc(op, &op->d_r, N));
    WDB_TRY(vt_alloc(op, &op->d_xs, N));
    WDB_TRY(vt_alloc(op, &op->d_scr, N / 2 + 1));
    WDB_TRY(vt_alloc(op, &op->d_w, op->lay.S));
    SolveState* p = nullptr;
    WDB_TRY(vt_alloc(op, &p, 1));
    void* h = nullptr;
    WDB_CK(cudaMallocHost(&h, sizeof(SolveState)));
    op->h_state = static_cast<SolveState*>(h);
    op->d_state = p;
    return WDB_OK;
}

wdb_status vtheta_objective(wdb_vtheta* op, const float* x, const float* x0, const float* w_dev, cudaStream_t st,
                            double* E, long long* support) {
    VEpi ep = oneoff_epi(op);
    ep.x0 = x0;
    ep.xl1 = x;
    ep.w_sb = w_dev;
    WDB_TRY((launch_vrow<float, kVObj>(op, false, x, (float*)nullptr, ep, st)));
    double h[3];
    WDB_CK(cudaMemcpyAsync(h, op->d_red, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
    WDB_CK(cudaStreamSynchronize(st));
    *E = 0.5 * h[0] + h[1];
    if (support) *support = (long long)llround(h[2]);
    return WDB_OK;
}

wdb_status vtheta_objective_public(wdb_vtheta* op, const float* x, const float* x0, const double* w_host,
                                   cudaStream_t caller, double* E) {
    WDB_TRY(vt_workspace(op));
    WDB_TRY(work_enter(&op->work, &op->ev_in, &op->ev_out, caller));
    cudaStream_t st = op->work;
    std::vector<float> w(op->lay.S);
    for (int b = 0; b < op->lay.S; ++b) w[b] = (float)w_host[b];
    WDB_CK(cudaMemcpyAsync(op->d_w, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice, st));
    WDB_TRY(vtheta_objective(op, x, x0, op->d_w, st, E, nullptr));
    WDB_TRY(work_exit(st, op->ev_out, caller));
    WDB_CK(cudaStreamSynchronize(st));
    return WDB_OK;
}

wdb_status vtheta_solve(wdb_vtheta* op, const float* in, bool is_image, float* x_out, const wdb_solve_params* p,
                        cudaStream_t caller, wdb_solve_result* res) {
    const double t0 = solve_now_ms();
    const Layout& L = op->lay;
    WDB_TRY(solve_check_params(p, L.S));
    WDB_TRY(vt_workspace(op));
    WDB_TRY(work_enter(&op->work, &op->ev_in, &op->ev_out, caller));
    cudaStream_t st = op->work;
    WDB_TRY(vtheta_precond(op, p->precond, p->jacobi_eps, st));
    const long long N = L.N;
    const int m = p->check_every > 0 ? p->check_every : 10;
    PrecondCache& pc = op->pc[p->precond];
    if (is_image) WDB_TRY(dwt2<float>(in, op->d_x0, L, op->filt, op->d_scr, st));
    else WDB_CK(cudaMemcpyAsync(op->d_x0, in, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
    std::vector<float> w = solve_weights(p, L.S);
    WDB_CK(cudaMemcpyAsync(op->d_w, w.data(), sizeof(float) * L.S, cudaMemcpyHostToDevice, st));
    if (p->x_init_dev) {
        WDB_CK(cudaMemcpyAsync(op->d_xs, p->x_init_dev, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
        WDB_CK(cudaMemcpyAsync(op->d_y, p->x_init_dev, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
    } else {
        WDB_CK(cudaMemsetAsync(op->d_xs, 0, sizeof(float) * N, st));
        WDB_CK(cudaMemsetAsync(op->d_y, 0, sizeof(float) * N, st));
    }
    SolveState s0 = solve_init_state(p, m);
    WDB_CK(cudaMemcpyAsync(op->d_state, &s0, sizeof s0, cudaMemcpyHostToDevice, st));
    VEpi e1{}, e2{};
    e1.x0 = op->d_x0;
    e1.st = op->d_state;
    e1.part = op->d_part;
    e1.counter = &op->d_state->done[0];
    e2.x = op->d_xs;
    e2.y = op->d_y;
    e2.step_tab = pc.d_step;
    e2.w_sb = op->d_w;
    e2.st = op->d_state;
    e2.part = op->d_part;
    e2.counter = &op->d_state->done[1];
    IterEngine& E = op->engine[p->precond];
    E.d_state = op->d_state;
    E.h_state = op->h_state;
    float *y = op->d_y, *r = op->d_r;
    E.enqueue = [=](int iters) -> wdb_status {
        for (int i = 0; i < iters; ++i) {
            WDB_TRY((launch_vrow<float, kVK1>(op, false, y, r, e1, st)));
            WDB_TRY((launch_vrow<float, kVK2>(op, true, r, (float*)nullptr, e2, st)));
        }
        return WDB_OK;
    };
    E.enqueue_timed = [=](cudaEvent_t* ev) -> wdb_status {
        WDB_TRY(solve_record_ev(ev[0], st));
        WDB_TRY((launch_vrow<float, kVK1>(op, false, y, r, e1, st)));
        WDB_TRY(solve_record_ev(ev[1], st));
        WDB_TRY((launch_vrow<float, kVK2>(op, true, r, (float*)nullptr, e2, st)));
        WDB_TRY(solve_record_ev(ev[2], st));
        return WDB_OK;
    };
    WDB_TRY(solve_run_loop(E, m, !p->no_graph, p->time_kernels != 0, 2LL * m, st));
    SolveState hs = *op->h_state;
    double Eobj = 0.0;
    long long sup = 0;
    WDB_TRY(vtheta_objective(op, op->d_xs, op->d_x0, op->d_w, st, &Eobj, &sup));
    WDB_CK(cudaMemcpyAsync(x_out, op->d_xs, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
    WDB_TRY(work_exit(st, op->ev_out, caller));
    WDB_CK(cudaStreamSynchronize(st));
    res->iters = hs.iters_done;
    res->objective = Eobj;
    res->primal = hs.primal;
    res->gap = hs.gap;
    res->rel_gap = hs.rel_gap;
    res->support = sup;
    res->tau = pc.tau;
    res->L_hat = pc.L_hat;
    res->ms_k1 = E.n_timed ? E.sum_k1 / E.n_timed : 0.0;
    res->ms_k2 = E.n_timed ? E.sum_k2 / E.n_timed : 0.0;
    res->timed_chunks = E.n_timed;
    res->first_primal_below = hs.hit_k;
    res->kkt_off = res->kkt_on = res->gap64 = res->rel_gap64 = NAN;
    res->status = WDB_OK;
    if (hs.nan_flag || !std::isfinite(Eobj)) res->status = set_error(WDB_ENAN, "NaN/Inf in the objective");
    else if (hs.diverged)
        res->status = set_error(WDB_EDIVERGED, "objective %g at iteration %d, above 1e6 x its first value %g",
                                hs.primal, hs.iters_done, hs.first_primal);
    res->solve_ms = solve_now_ms() - t0;
    return res->status;
}

}  // namespace wdb
