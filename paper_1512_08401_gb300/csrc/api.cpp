// C ABI of libwdb (declared in include/wdb.h). Argument validation, handle lifetime,
// serialisation; the work is done by theta.cu, subband_ops.cu, dwt.cu and solve.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <tuple>

#include "solve_impl.h"
#include "plan_check.h"
#include "theta_impl.h"
#include "vtheta.h"
#include "wdb_internal.h"

namespace wdb {
long long launches(int reset);
const char* last_error();
}  // namespace wdb

using namespace wdb;

namespace {

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

wdb_status need_device() {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) return set_error(WDB_ECUDA, "no CUDA device available");
    return WDB_OK;
}

wdb_status check_psf(const double* psf, int kh, int kw, int n_rows, int n_cols) {
    if (!psf) return set_error(WDB_EINVAL, "psf is NULL");
    if (kh <= 0 || kw <= 0 || (kh % 2) == 0 || (kw % 2) == 0)
        return set_error(WDB_EINVAL, "PSF sides must be odd and positive (got %dx%d)", kh, kw);
    if (kh > n_rows || kw > n_cols) return set_error(WDB_EINVAL, "PSF %dx%d larger than the image", kh, kw);
    for (int i = 0; i < kh * kw; ++i)
        if (!std::isfinite(psf[i])) return set_error(WDB_EINVAL, "PSF has a non-finite value");
    return WDB_OK;
}

void theta_release(wdb_theta* th) {
    if (!th) return;
    if (th->work) cudaStreamSynchronize(th->work);
    for (auto& e : th->engine) e.release();
    if (th->work) cudaStreamDestroy(th->work);
    if (th->ev_in) cudaEventDestroy(th->ev_in);
    if (th->ev_out) cudaEventDestroy(th->ev_out);
    for (void* p : th->allocs) cudaFree(p);
    if (th->h_state) cudaFreeHost(th->h_state);
    delete th;
}

wdb_status new_theta(int n_rows, int n_cols, const char* wavelet, int levels, wdb_theta** out) {
    Layout L;
    WDB_TRY(make_layout(n_rows, n_cols, levels, &L));
    Filters f;
    WDB_TRY(wavelet_filters(wavelet, &f));
    wdb_theta* th = new (std::nothrow) wdb_theta();
    if (!th) return set_error(WDB_ENOMEM, "host allocation");
    th->lay = L;
    th->filt = f;
    th->wavelet = wavelet;
    *out = th;
    return WDB_OK;
}

constexpr char kMagic[8] = {'W', 'D', 'B', 'T', 'H', 'E', 'T', '1'};

}  // namespace

extern "C" {

wdb_status wdb_build_theta(const double* psf_host, int kh, int kw, int n_rows, int n_cols, const char* wavelet,
                           int levels, long long K, int rule, void* stream, wdb_theta** out) {
    if (!out) return set_error(WDB_EINVAL, "out is NULL");
    *out = nullptr;
    WDB_TRY(check_psf(psf_host, kh, kw, n_rows, n_cols));
    if (K < 0) return set_error(WDB_EINVAL, "K must be >= 0");
    if (rule != WDB_RULE_WEIGHTED && rule != WDB_RULE_NAIVE) return set_error(WDB_EINVAL, "unknown rule %d", rule);
    wdb_theta* th = nullptr;
    WDB_TRY(new_theta(n_rows, n_cols, wavelet, levels, &th));
    wdb_status s = need_device();
    const double t0 = now_ms();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    th->rule = rule;
    th->K_requested = K;
    if (s == WDB_OK) s = theta_build_device(th, psf_host, kh, kw, K, rule, st);
    if (s == WDB_OK) s = theta_finalize(th, st);
    if (s == WDB_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_error(e, "build", __FILE__, __LINE__);
    }
    if (s != WDB_OK) {
        theta_release(th);
        return s;
    }
    th->build_ms = now_ms() - t0;
    *out = th;
    return WDB_OK;
}

wdb_status wdb_theta_from_taps(int n_rows, int n_cols, const char* wavelet, int levels, long long n_taps,
                               const int* a, const int* b, const int* oy, const int* ox, const double* v,
                               void* stream, wdb_theta** out) {
    if (!out) return set_error(WDB_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_taps < 0) return set_error(WDB_EINVAL, "n_taps must be >= 0");
    if (n_taps > 0 && (!a || !b || !oy || !ox || !v)) return set_error(WDB_EINVAL, "tap array is NULL");
    wdb_theta* th = nullptr;
    WDB_TRY(new_theta(n_rows, n_cols, wavelet, levels, &th));
    const Layout& L = th->lay;
    th->taps.resize((size_t)n_taps);
    for (long long i = 0; i < n_taps; ++i) {
        if (a[i] < 0 || a[i] >= L.S || b[i] < 0 || b[i] >= L.S) {
            theta_release(th);
            return set_error(WDB_EINVAL, "tap %lld: subband out of range", i);
        }
        const SubbandDev &sa = L.sb[a[i]], &sb = L.sb[b[i]];
        const SubbandDev& arr = (sa.level <= sb.level) ? sa : sb;
        if (oy[i] < 0 || oy[i] >= arr.rows || ox[i] < 0 || ox[i] >= arr.cols || !std::isfinite(v[i])) {
            theta_release(th);
            return set_error(WDB_EINVAL, "tap %lld: offset out of range or value not finite", i);
        }
        th->taps[i] = Tap{a[i], b[i], oy[i], ox[i], v[i]};
    }
    std::sort(th->taps.begin(), th->taps.end(), [](const Tap& x, const Tap& y) {
        return std::tie(x.a, x.b, x.oy, x.ox) < std::tie(y.a, y.b, y.oy, y.ox);
    });
    for (size_t i = 1; i < th->taps.size(); ++i) {
        const Tap &x = th->taps[i - 1], &y = th->taps[i];
        if (x.a == y.a && x.b == y.b && x.oy == y.oy && x.ox == y.ox) {
            theta_release(th);
            return set_error(WDB_EINVAL, "duplicate tap (%d,%d,%d,%d)", x.a, x.b, x.oy, x.ox);
        }
    }
    wdb_status s = need_device();
    const double t0 = now_ms();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (s == WDB_OK) s = theta_finalize(th, st);
    if (s == WDB_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_error(e, "from_taps", __FILE__, __LINE__);
    }
    if (s != WDB_OK) {
        theta_release(th);
        return s;
    }
    th->K_requested = th->K_eff;
    th->n_candidates = -1;
    th->build_ms = now_ms() - t0;
    *out = th;
    return WDB_OK;
}

wdb_status wdb_theta_info_get(const wdb_theta* th, wdb_theta_info* info) {
    if (!th || !info) return set_error(WDB_EINVAL, "NULL argument");
    std::memset(info, 0, sizeof *info);
    info->n_rows = th->lay.n_rows;
    info->n_cols = th->lay.n_cols;
    info->levels = th->lay.J;
    info->n_subbands = th->lay.S;
    info->wavelet_taps = th->filt.L;
    info->rule = th->rule;
    info->K_requested = th->K_requested;
    info->K_eff = th->K_eff;
    info->n_taps = (long long)th->taps.size();
    info->n_candidates = th->n_candidates;
    info->theta_max_abs = th->theta_max_abs;
    info->phase_table_len = th->lay.tab_len;
    info->build_ms = th->build_ms;
    info->plan_tuned = th->tuned;
    for (int op = 0; op < 2; ++op) {
        info->plan_items[op] = (int)th->tplan[op][0].items.size();
        info->plan_split_tiles[op] = th->tplan[op][0].n_split;
        info->plan_super_subbands[op] = th->tplan[op][0].n_sup;
        info->plan_groups[op] = th->tplan[op][0].n_grp;
        info->plan_smem_bytes[op] = th->tplan[op][0].smem_bytes;
        info->plan_grid[op] = th->targs[op][0].grid;
    }
    return WDB_OK;
}

wdb_status wdb_tile_plan_check(int n_rows, int n_cols, int levels, long long n_taps, const int* a, const int* b,
                               const int* oy, const int* ox, const double* v, int transpose, int esize,
                               int smem_budget, double cap_share, double split_share, int super_tiles, int ctas,
                               wdb_plan_summary* summary) {
    if (n_taps < 0 || (n_taps > 0 && (!a || !b || !oy || !ox || !v))) return set_error(WDB_EINVAL, "bad tap arrays");
    if (esize != 4 && esize != 8) return set_error(WDB_EINVAL, "esize %d (4 or 8)", esize);
    if (smem_budget > 98304) return set_error(WDB_EINVAL, "smem_budget %d > 98304", smem_budget);
    Layout L;
    WDB_TRY(make_layout(n_rows, n_cols, levels, &L));
    std::vector<Tap> taps((size_t)n_taps);
    for (long long i = 0; i < n_taps; ++i) {
        if (a[i] < 0 || a[i] >= L.S || b[i] < 0 || b[i] >= L.S)
            return set_error(WDB_EINVAL, "tap %lld names subband (%d, %d) of %d", i, a[i], b[i], L.S);
        taps[(size_t)i] = Tap{a[i], b[i], oy[i], ox[i], v[i]};
    }
    std::vector<TileEntry> te[2];
    gather_entries(L, taps, te);
    const TilePlanHost P =
        make_tile_plan(L, te[transpose ? 1 : 0], esize, smem_budget > 0 ? smem_budget : 32768, ctas > 0 ? ctas : 456,
                       nullptr, 0, cap_share > 0.0 ? cap_share : 2.0, split_share > 0.0 ? split_share : 0.0,
                       super_tiles == 1, super_tiles == 2);
    if (summary) {
        summary->items = (int)P.items.size();
        summary->pairs = (int)P.pairs.size();
        summary->batches = (int)P.batches.size();
        summary->split_tiles = P.n_split;
        summary->super_subbands = P.n_sup;
        summary->groups = P.n_grp;
        summary->smem_bytes = P.smem_bytes;
        summary->macs = P.macs;
    }
    const std::string err = check_tile_plan(L, P);
    if (!err.empty()) return set_error(WDB_EPLAN, "%s", err.c_str());
    return WDB_OK;
}

wdb_status wdb_theta_replan(wdb_theta* th, int smem_budget, double cap_share, double split_share, int super_tiles,
                            void* stream) {
    if (!th) return set_error(WDB_EINVAL, "NULL handle");
    if (smem_budget > 98304) return set_error(WDB_EINVAL, "smem_budget %d > 98304", smem_budget);
    if (super_tiles < 0 || super_tiles > 2) return set_error(WDB_EINVAL, "tiling mode %d (0, 1 or 2)", super_tiles);
    if (super_tiles && split_share > 0.0) return set_error(WDB_EINVAL, "split tiles with super tiles or groups");
    return theta_replan(th, smem_budget > 0 ? smem_budget : 32768, cap_share > 0.0 ? cap_share : 2.0,
                        split_share > 0.0 ? split_share : 0.0, super_tiles, static_cast<cudaStream_t>(stream));
}

wdb_status wdb_theta_export_taps(const wdb_theta* th, long long cap, int* a, int* b, int* oy, int* ox, double* v) {
    if (!th) return set_error(WDB_EINVAL, "NULL handle");
    if (cap < (long long)th->taps.size()) return set_error(WDB_EINVAL, "capacity %lld < %zu taps", cap, th->taps.size());
    for (size_t i = 0; i < th->taps.size(); ++i) {
        const Tap& t = th->taps[i];
        if (a) a[i] = t.a;
        if (b) b[i] = t.b;
        if (oy) oy[i] = t.oy;
        if (ox) ox[i] = t.ox;
        if (v) v[i] = t.v;
    }
    return WDB_OK;
}

wdb_status wdb_theta_precond(wdb_theta* th, int precond, double jacobi_eps, void* stream, double* P_host,
                             double* Md_host, double* M2d_host, double* tau_host, double* L_hat_host) {
    if (!th) return set_error(WDB_EINVAL, "NULL handle");
    WDB_TRY(need_device());
    WDB_TRY(theta_precond(th, precond, jacobi_eps, static_cast<cudaStream_t>(stream)));
    const PrecondCache& pc = th->pc[precond];
    const int n = th->lay.tab_len;
    if (P_host) std::copy(pc.P.begin(), pc.P.end(), P_host);
    if (Md_host) std::copy(th->Md.begin(), th->Md.begin() + n, Md_host);
    if (M2d_host) std::copy(th->M2d.begin(), th->M2d.begin() + n, M2d_host);
    if (tau_host) *tau_host = pc.tau;
    if (L_hat_host) *L_hat_host = pc.L_hat;
    return WDB_OK;
}

wdb_status wdb_theta_set_precond(wdb_theta* th, int precond, const double* P_host, double tau) {
    if (!th || !P_host) return set_error(WDB_EINVAL, "NULL argument");
    if (precond < 0 || precond > 2) return set_error(WDB_EINVAL, "unknown preconditioner %d", precond);
    if (!(tau > 0.0) || !std::isfinite(tau)) return set_error(WDB_EINVAL, "tau must be finite and > 0");
    const int n = th->lay.tab_len;
    for (int i = 0; i < n; ++i)
        if (!(P_host[i] > 0.0) || !std::isfinite(P_host[i])) return set_error(WDB_EINVAL, "P[%d] must be > 0", i);
    PrecondCache& pc = th->pc[precond];
    pc.P.assign(P_host, P_host + n);
    pc.tau = tau;
    pc.L_hat = 1.0 / (kStepMargin * tau);
    WDB_TRY(precond_upload(th, pc, nullptr));
    pc.valid = true;
    pc.pinned = true;
    return WDB_OK;
}

wdb_status wdb_theta_save(const wdb_theta* th, const char* path) {
    if (!th || !path) return set_error(WDB_EINVAL, "NULL argument");
    FILE* f = std::fopen(path, "wb");
    if (!f) return set_error(WDB_EIO, "cannot open %s for writing", path);
    char wav[16] = {0};
    std::strncpy(wav, th->wavelet.c_str(), sizeof wav - 1);
    int hdr[4] = {th->lay.n_rows, th->lay.n_cols, th->lay.J, th->rule};
    long long k2[2] = {th->K_requested, (long long)th->taps.size()};
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(int), 4, f) == 4 &&
              std::fwrite(wav, 1, 16, f) == 16 && std::fwrite(k2, sizeof(long long), 2, f) == 2;
    for (size_t i = 0; ok && i < th->taps.size(); ++i) {
        const Tap& t = th->taps[i];
        int ij[4] = {t.a, t.b, t.oy, t.ox};
        ok = std::fwrite(ij, sizeof(int), 4, f) == 4 && std::fwrite(&t.v, sizeof(double), 1, f) == 1;
    }
    ok = (std::fclose(f) == 0) && ok;
    return ok ? WDB_OK : set_error(WDB_EIO, "write failed: %s", path);
}

wdb_status wdb_theta_load(const char* path, void* stream, wdb_theta** out) {
    if (!path || !out) return set_error(WDB_EINVAL, "NULL argument");
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) return set_error(WDB_EIO, "cannot open %s", path);
    char magic[8];
    int hdr[4];
    char wav[16];
    long long k2[2];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(hdr, sizeof(int), 4, f) == 4 && std::fread(wav, 1, 16, f) == 16 &&
              std::fread(k2, sizeof(long long), 2, f) == 2 && k2[1] >= 0 && k2[1] < (1LL << 40);
    wav[15] = 0;
    std::vector<int> A, B, OY, OX;
    std::vector<double> V;
    if (ok) {
        A.resize(k2[1]);
        B.resize(k2[1]);
        OY.resize(k2[1]);
        OX.resize(k2[1]);
        V.resize(k2[1]);
        for (long long i = 0; ok && i < k2[1]; ++i) {
            int ij[4];
            ok = std::fread(ij, sizeof(int), 4, f) == 4 && std::fread(&V[i], sizeof(double), 1, f) == 1;
            A[i] = ij[0];
            B[i] = ij[1];
            OY[i] = ij[2];
            OX[i] = ij[3];
        }
    }
    std::fclose(f);
    if (!ok) return set_error(WDB_EIO, "bad or truncated file: %s", path);
    wdb_theta* th = nullptr;
    WDB_TRY(wdb_theta_from_taps(hdr[0], hdr[1], wav, hdr[2], k2[1], A.data(), B.data(), OY.data(), OX.data(),
                                V.data(), stream, &th));
    th->rule = hdr[3];
    th->K_requested = k2[0];
    *out = th;
    return WDB_OK;
}

void wdb_theta_free(wdb_theta* th) { theta_release(th); }

wdb_status wdb_theta_apply(const wdb_theta* th, const float* in_dev, float* out_dev, int transpose, void* stream) {
    if (!th || !in_dev || !out_dev) return set_error(WDB_EINVAL, "NULL argument");
    return tile_apply<float>(tile_args(th, transpose != 0, false), in_dev, out_dev, nullptr, nullptr, th->d_red_part,
                             static_cast<cudaStream_t>(stream));
}

wdb_status wdb_solve(wdb_theta* th, const float* u_dev, float* x_dev, const wdb_solve_params* params, void* stream,
                     wdb_solve_result* result) {
    if (!th || !u_dev || !x_dev || !params || !result) return set_error(WDB_EINVAL, "NULL argument");
    std::memset(result, 0, sizeof *result);
    wdb_status s = theta_solve(th, u_dev, true, x_dev, params, static_cast<cudaStream_t>(stream), result);
    result->status = s;
    return s;
}

wdb_status wdb_solve_coeffs(wdb_theta* th, const float* x0_dev, float* x_dev, const wdb_solve_params* params,
                            void* stream, wdb_solve_result* result) {
    if (!th || !x0_dev || !x_dev || !params || !result) return set_error(WDB_EINVAL, "NULL argument");
    std::memset(result, 0, sizeof *result);
    wdb_status s = theta_solve(th, x0_dev, false, x_dev, params, static_cast<cudaStream_t>(stream), result);
    result->status = s;
    return s;
}

wdb_status wdb_solve_batch(int B, wdb_theta* const* th, const float* const* u_dev, float* const* x_dev,
                           const wdb_solve_params* params, void* stream, wdb_solve_result* results) {
    WDB_TRY(need_device());
    return solve_batch(B, th, u_dev, x_dev, params, static_cast<cudaStream_t>(stream), results);
}

wdb_status wdb_theta_objective(const wdb_theta* thc, const float* x_dev, const float* x0_dev, double lambda,
                               const double* w_subband_host, void* stream, double* E_host) {
    wdb_theta* th = const_cast<wdb_theta*>(thc);
    if (!th || !x_dev || !x0_dev || !E_host) return set_error(WDB_EINVAL, "NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    WDB_TRY(theta_workspace_public(th, st));
    std::vector<float> w(th->lay.S);
    for (int b = 0; b < th->lay.S; ++b) w[b] = (float)(w_subband_host ? w_subband_host[b] : lambda);
    WDB_CK(cudaMemcpyAsync(th->d_w, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice, st));
    return theta_objective_dev(th, x_dev, x0_dev, th->d_w, st, E_host, nullptr);
}

wdb_status wdb_theta_kkt(wdb_theta* th, const float* x_dev, const float* x0_dev, double lambda,
                         const double* w_subband_host, void* stream, wdb_kkt_result* out) {
    if (!th || !x_dev || !x0_dev || !out) return set_error(WDB_EINVAL, "NULL argument");
    if (!w_subband_host && !(lambda >= 0.0 && std::isfinite(lambda)))
        return set_error(WDB_EINVAL, "lambda must be finite and >= 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    WDB_TRY(theta_workspace_public(th, st));
    std::vector<double> w(th->lay.S);
    for (int b = 0; b < th->lay.S; ++b) w[b] = w_subband_host ? w_subband_host[b] : lambda;
    Kkt64 k{};
    WDB_TRY(theta_kkt64(th, x_dev, x0_dev, w.data(), st, &k));
    out->objective = k.objective;
    out->gap = k.gap;
    out->rel_gap = k.rel_gap;
    out->kkt_off = k.kkt_off;
    out->kkt_on = k.kkt_on;
    out->gmax = k.gmax;
    out->support = k.support;
    return WDB_OK;
}

wdb_status wdb_fftop_create(const double* psf_host, int kh, int kw, int n_rows, int n_cols, const char* wavelet,
                            int levels, void* stream, wdb_fftop** out) {
    if (!out) return set_error(WDB_EINVAL, "out is NULL");
    *out = nullptr;
    WDB_TRY(check_psf(psf_host, kh, kw, n_rows, n_cols));
    Layout L;
    WDB_TRY(make_layout(n_rows, n_cols, levels, &L));
    Filters f;
    WDB_TRY(wavelet_filters(wavelet, &f));
    WDB_TRY(need_device());
    return fftop_create(psf_host, kh, kw, L, f, wavelet, static_cast<cudaStream_t>(stream), out);
}

void wdb_fftop_free(wdb_fftop* op) { fftop_free(op); }

wdb_status wdb_fftop_objective(wdb_fftop* op, const float* u_dev, const float* x_dev, double lambda,
                               const double* w_subband_host, void* stream, double* E_host) {
    if (!op || !u_dev || !x_dev || !E_host) return set_error(WDB_EINVAL, "NULL argument");
    if (!w_subband_host && !(lambda >= 0.0 && std::isfinite(lambda)))
        return set_error(WDB_EINVAL, "lambda must be finite and >= 0");
    std::vector<double> w(op->lay.S);
    for (int b = 0; b < op->lay.S; ++b) w[b] = w_subband_host ? w_subband_host[b] : lambda;
    return fft_objective_public(op, u_dev, x_dev, w.data(), static_cast<cudaStream_t>(stream), E_host);
}

wdb_status wdb_fftop_precond(wdb_fftop* op, int precond, double jacobi_eps, void* stream, double* P_host,
                             double* tau_host, double* L_hat_host) {
    if (!op) return set_error(WDB_EINVAL, "NULL handle");
    WDB_TRY(fftop_precond(op, precond, jacobi_eps, static_cast<cudaStream_t>(stream)));
    const PrecondCache& pc = op->pc[precond];
    if (P_host)
        for (int b = 0; b < op->lay.S; ++b) P_host[b] = pc.P[op->lay.sb[b].tab_off];
    if (tau_host) *tau_host = pc.tau;
    if (L_hat_host) *L_hat_host = pc.L_hat;
    return WDB_OK;
}

wdb_status wdb_fftop_set_precond(wdb_fftop* op, int precond, const double* P_host, double tau) {
    if (!op || !P_host) return set_error(WDB_EINVAL, "NULL argument");
    if (precond < 0 || precond > 2) return set_error(WDB_EINVAL, "unknown preconditioner %d", precond);
    if (!(tau > 0.0) || !std::isfinite(tau)) return set_error(WDB_EINVAL, "tau must be finite and > 0");
    const Layout& L = op->lay;
    PrecondCache& pc = op->pc[precond];
    pc.P.assign(L.tab_len, 1.0);
    for (int b = 0; b < L.S; ++b) {
        if (!(P_host[b] > 0.0) || !std::isfinite(P_host[b])) return set_error(WDB_EINVAL, "P[%d] must be > 0", b);
        for (int i = 0; i < (1 << (2 * L.sb[b].lgR)); ++i) pc.P[L.sb[b].tab_off + i] = P_host[b];
    }
    pc.tau = tau;
    pc.L_hat = 1.0 / (kStepMargin * tau);
    if (!pc.d_step) {
        void* p = nullptr;
        WDB_CK(cudaMalloc(&p, sizeof(float) * L.tab_len));
        op->allocs.push_back(p);
        pc.d_step = static_cast<float*>(p);
    }
    std::vector<float> stp(L.tab_len);
    for (int i = 0; i < L.tab_len; ++i) stp[i] = (float)(tau / pc.P[i]);
    WDB_CK(cudaMemcpy(pc.d_step, stp.data(), sizeof(float) * stp.size(), cudaMemcpyHostToDevice));
    pc.valid = true;
    pc.pinned = true;
    return WDB_OK;
}

wdb_status wdb_solve_fft(wdb_fftop* op, const float* u_dev, float* x_dev, const wdb_solve_params* params,
                         void* stream, wdb_solve_result* result) {
    if (!op || !u_dev || !x_dev || !params || !result) return set_error(WDB_EINVAL, "NULL argument");
    std::memset(result, 0, sizeof *result);
    wdb_status s = fft_solve(op, u_dev, x_dev, params, static_cast<cudaStream_t>(stream), result);
    result->status = s;
    return s;
}

// ---- row-varying operator ----
wdb_status wdb_vtheta_build(const double* psfs_host, int kh, int kw, int n_rows, int n_cols, const char* wavelet,
                            int levels, long long K, int rule, void* stream, wdb_vtheta** out) {
    if (!out) return set_error(WDB_EINVAL, "out is NULL");
    *out = nullptr;
    if (!psfs_host) return set_error(WDB_EINVAL, "psfs is NULL");
    if (n_rows <= 0 || n_cols <= 0) return set_error(WDB_EINVAL, "bad image size %dx%d", n_rows, n_cols);
    for (int i = 0; i < n_rows; ++i)
        WDB_TRY(check_psf(psfs_host + (size_t)i * kh * kw, kh, kw, n_rows, n_cols));
    if (K < 0) return set_error(WDB_EINVAL, "K must be >= 0");
    if (rule != WDB_RULE_WEIGHTED && rule != WDB_RULE_NAIVE) return set_error(WDB_EINVAL, "unknown rule %d", rule);
    wdb_vtheta* op = nullptr;
    WDB_TRY(vtheta_new(n_rows, n_cols, wavelet, levels, &op));
    wdb_status s = need_device();
    const double t0 = now_ms();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    op->rule = rule;
    op->K_requested = K;
    if (s == WDB_OK) s = vtheta_build_device(op, psfs_host, kh, kw, K, rule, st);
    if (s == WDB_OK) s = vtheta_finalize(op, st);
    if (s != WDB_OK) {
        vtheta_release(op);
        return s;
    }
    op->build_ms = now_ms() - t0;
    *out = op;
    return WDB_OK;
}

wdb_status wdb_vtheta_from_taps(int n_rows, int n_cols, const char* wavelet, int levels, long long n_taps,
                                const int* a, const int* py, const int* b, const int* qy, const int* ox,
                                const double* v, void* stream, wdb_vtheta** out) {
    if (!out) return set_error(WDB_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_taps < 0) return set_error(WDB_EINVAL, "n_taps must be >= 0");
    if (n_taps > 0 && (!a || !py || !b || !qy || !ox || !v)) return set_error(WDB_EINVAL, "tap array is NULL");
    wdb_vtheta* op = nullptr;
    WDB_TRY(vtheta_new(n_rows, n_cols, wavelet, levels, &op));
    const Layout& L = op->lay;
    op->taps.resize((size_t)n_taps);
    for (long long i = 0; i < n_taps; ++i) {
        if (a[i] < 0 || a[i] >= L.S || b[i] < 0 || b[i] >= L.S) {
            vtheta_release(op);
            return set_error(WDB_EINVAL, "tap %lld: subband out of range", i);
        }
        const SubbandDev &sa = L.sb[a[i]], &sb = L.sb[b[i]];
        const int ocols = sa.level <= sb.level ? sa.cols : sb.cols;
        if (py[i] < 0 || py[i] >= sa.rows || qy[i] < 0 || qy[i] >= sb.rows || ox[i] < 0 || ox[i] >= ocols ||
            !std::isfinite(v[i])) {
            vtheta_release(op);
            return set_error(WDB_EINVAL, "tap %lld outside its subbands or not finite", i);
        }
        op->taps[i] = {a[i], py[i], b[i], qy[i], ox[i], v[i]};
    }
    auto key = [](const VTapH& t) { return std::tie(t.a, t.py, t.b, t.qy, t.ox); };
    std::sort(op->taps.begin(), op->taps.end(), [&](const VTapH& x, const VTapH& y) { return key(x) < key(y); });
    for (size_t i = 1; i < op->taps.size(); ++i)
        if (key(op->taps[i]) == key(op->taps[i - 1])) {
            vtheta_release(op);
            return set_error(WDB_EINVAL, "duplicate tap");
        }
    double vmax = 0.0;
    for (const VTapH& t : op->taps) vmax = std::max(vmax, std::fabs(t.v));
    op->theta_max_abs = vmax;
    op->K_requested = -1;
    wdb_status s = need_device();
    const double t0 = now_ms();
    if (s == WDB_OK) s = vtheta_finalize(op, static_cast<cudaStream_t>(stream));
    if (s != WDB_OK) {
        vtheta_release(op);
        return s;
    }
    op->K_requested = op->K_eff;
    op->build_ms = now_ms() - t0;
    *out = op;
    return WDB_OK;
}

wdb_status wdb_vtheta_info_get(const wdb_vtheta* op, wdb_vtheta_info* info) {
    if (!op || !info) return set_error(WDB_EINVAL, "NULL argument");
    std::memset(info, 0, sizeof *info);
    info->n_rows = op->lay.n_rows;
    info->n_cols = op->lay.n_cols;
    info->levels = op->lay.J;
    info->n_subbands = op->lay.S;
    info->rule = op->rule;
    info->K_requested = op->K_requested;
    info->K_eff = op->K_eff;
    info->n_taps = (long long)op->taps.size();
    info->n_candidates = op->n_candidates;
    info->candidate_slots = op->n_cand_slots;
    info->n_probes = op->n_probes;
    info->n_classes = op->n_classes;
    info->n_plan_rows = op->plan[0].n_rows;
    info->plan_taps[0] = (long long)op->hplan[0].taps.size();
    info->plan_taps[1] = (long long)op->hplan[1].taps.size();
    info->theta_max_abs = op->theta_max_abs;
    info->build_ms = op->build_ms;
    return WDB_OK;
}

wdb_status wdb_vtheta_export_taps(const wdb_vtheta* op, long long cap, int* a, int* py, int* b, int* qy, int* ox,
                                  double* v) {
    if (!op || !a || !py || !b || !qy || !ox || !v) return set_error(WDB_EINVAL, "NULL argument");
    if (cap < (long long)op->taps.size()) return set_error(WDB_EINVAL, "capacity %lld < %zu taps", cap, op->taps.size());
    for (size_t i = 0; i < op->taps.size(); ++i) {
        const VTapH& t = op->taps[i];
        a[i] = t.a;
        py[i] = t.py;
        b[i] = t.b;
        qy[i] = t.qy;
        ox[i] = t.ox;
        v[i] = t.v;
    }
    return WDB_OK;
}

wdb_status wdb_vtheta_apply(const wdb_vtheta* op, const float* in_dev, float* out_dev, int transpose, void* stream) {
    if (!op || !in_dev || !out_dev) return set_error(WDB_EINVAL, "NULL argument");
    return vtheta_apply(op, in_dev, out_dev, transpose != 0, static_cast<cudaStream_t>(stream));
}

wdb_status wdb_vtheta_precond(wdb_vtheta* op, int precond, double jacobi_eps, void* stream, double* P_host,
                              double* Md_host, double* M2d_host, double* tau_host, double* L_hat_host) {
    if (!op) return set_error(WDB_EINVAL, "NULL handle");
    WDB_TRY(need_device());
    WDB_TRY(vtheta_precond(op, precond, jacobi_eps, static_cast<cudaStream_t>(stream)));
    const PrecondCache& pc = op->pc[precond];
    if (P_host) std::copy(pc.P.begin(), pc.P.end(), P_host);
    if (Md_host) std::copy(op->Md.begin(), op->Md.end(), Md_host);
    if (M2d_host) std::copy(op->M2d.begin(), op->M2d.end(), M2d_host);
    if (tau_host) *tau_host = pc.tau;
    if (L_hat_host) *L_hat_host = pc.L_hat;
    return WDB_OK;
}

wdb_status wdb_vtheta_set_precond(wdb_vtheta* op, int precond, const double* P_host, double tau) {
    if (!op || !P_host) return set_error(WDB_EINVAL, "NULL argument");
    if (precond < 0 || precond > 2) return set_error(WDB_EINVAL, "unknown preconditioner %d", precond);
    if (!(tau > 0.0) || !std::isfinite(tau)) return set_error(WDB_EINVAL, "tau must be finite and > 0");
    for (int i = 0; i < op->n_classes; ++i)
        if (!(P_host[i] > 0.0) || !std::isfinite(P_host[i])) return set_error(WDB_EINVAL, "P[%d] must be > 0", i);
    return vtheta_set_precond(op, precond, P_host, tau);
}

wdb_status wdb_vtheta_solve(wdb_vtheta* op, const float* u_dev, float* x_dev, const wdb_solve_params* params,
                            void* stream, wdb_solve_result* result) {
    if (!op || !u_dev || !x_dev || !params || !result) return set_error(WDB_EINVAL, "NULL argument");
    std::memset(result, 0, sizeof *result);
    wdb_status s = vtheta_solve(op, u_dev, true, x_dev, params, static_cast<cudaStream_t>(stream), result);
    result->status = s;
    return s;
}

wdb_status wdb_vtheta_solve_coeffs(wdb_vtheta* op, const float* x0_dev, float* x_dev, const wdb_solve_params* params,
                                   void* stream, wdb_solve_result* result) {
    if (!op || !x0_dev || !x_dev || !params || !result) return set_error(WDB_EINVAL, "NULL argument");
    std::memset(result, 0, sizeof *result);
    wdb_status s = vtheta_solve(op, x0_dev, false, x_dev, params, static_cast<cudaStream_t>(stream), result);
    result->status = s;
    return s;
}

wdb_status wdb_vtheta_objective(wdb_vtheta* op, const float* x_dev, const float* x0_dev, double lambda,
                                const double* w_subband_host, void* stream, double* E_host) {
    if (!op || !x_dev || !x0_dev || !E_host) return set_error(WDB_EINVAL, "NULL argument");
    if (!w_subband_host && !(lambda >= 0.0 && std::isfinite(lambda)))
        return set_error(WDB_EINVAL, "lambda must be finite and >= 0");
    std::vector<double> w(op->lay.S);
    for (int b = 0; b < op->lay.S; ++b) w[b] = w_subband_host ? w_subband_host[b] : lambda;
    return vtheta_objective_public(op, x_dev, x0_dev, w.data(), static_cast<cudaStream_t>(stream), E_host);
}

void wdb_vtheta_free(wdb_vtheta* op) { vtheta_release(op); }

wdb_status wdb_vtheta_plan_check(int n_rows, int n_cols, const char* wavelet, int levels, long long n_taps,
                                 const int* a, const int* py, const int* b, const int* qy, const int* ox,
                                 const double* v, int transpose, const double* x_host, double* y_host) {
    if (!x_host || !y_host) return set_error(WDB_EINVAL, "NULL argument");
    if (n_taps < 0 || (n_taps > 0 && (!a || !py || !b || !qy || !ox || !v)))
        return set_error(WDB_EINVAL, "bad tap arrays");
    wdb_vtheta* op = nullptr;
    WDB_TRY(vtheta_new(n_rows, n_cols, wavelet, levels, &op));
    const Layout& L = op->lay;
    wdb_status s = WDB_OK;
    for (long long i = 0; i < n_taps && s == WDB_OK; ++i) {
        if (a[i] < 0 || a[i] >= L.S || b[i] < 0 || b[i] >= L.S) {
            s = set_error(WDB_EINVAL, "tap %lld: subband out of range", i);
            break;
        }
        const SubbandDev &sa = L.sb[a[i]], &sb = L.sb[b[i]];
        const int ocols = sa.level <= sb.level ? sa.cols : sb.cols;
        if (py[i] < 0 || py[i] >= sa.rows || qy[i] < 0 || qy[i] >= sb.rows || ox[i] < 0 || ox[i] >= ocols)
            s = set_error(WDB_EINVAL, "tap %lld outside its subbands", i);
        else op->taps.push_back({a[i], py[i], b[i], qy[i], ox[i], v[i]});
    }
    if (s == WDB_OK) s = vtheta_plan_emulate(op, transpose != 0, x_host, y_host);
    vtheta_release(op);
    return s;
}

wdb_status wdb_dwt(const float* img_dev, float* coef_dev, int n_rows, int n_cols, const char* wavelet, int levels,
                   void* stream) {
    if (!img_dev || !coef_dev) return set_error(WDB_EINVAL, "NULL argument");
    Layout L;
    WDB_TRY(make_layout(n_rows, n_cols, levels, &L));
    Filters f;
    WDB_TRY(wavelet_filters(wavelet, &f));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* scr = nullptr;
    WDB_CK(cudaMallocAsync(&scr, sizeof(float) * (L.N / 2 + 1), st));
    wdb_status s = dwt2<float>(img_dev, coef_dev, L, f, static_cast<float*>(scr), st);
    cudaFreeAsync(scr, st);
    return s;
}

wdb_status wdb_idwt(const float* coef_dev, float* img_dev, int n_rows, int n_cols, const char* wavelet, int levels,
                    void* stream) {
    if (!img_dev || !coef_dev) return set_error(WDB_EINVAL, "NULL argument");
    Layout L;
    WDB_TRY(make_layout(n_rows, n_cols, levels, &L));
    Filters f;
    WDB_TRY(wavelet_filters(wavelet, &f));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* scr = nullptr;
    WDB_CK(cudaMallocAsync(&scr, sizeof(float) * (L.N / 2 + 1), st));
    wdb_status s = idwt2<float>(coef_dev, img_dev, L, f, static_cast<float*>(scr), st);
    cudaFreeAsync(scr, st);
    return s;
}

wdb_status wdb_wavelet_filters(const char* wavelet, int cap, double* h, double* g, int* taps) {
    Filters f;
    WDB_TRY(wavelet_filters(wavelet, &f));
    if (taps) *taps = f.L;
    if (cap < f.L) return set_error(WDB_EINVAL, "capacity %d < %d taps", cap, f.L);
    for (int k = 0; k < f.L; ++k) {
        if (h) h[k] = f.h[k];
        if (g) g[k] = f.g[k];
    }
    return WDB_OK;
}

const char* wdb_status_str(wdb_status s) {
    switch (s) {
        case WDB_OK: return "ok";
        case WDB_EINVAL: return "invalid argument";
        case WDB_ENOMEM: return "out of memory";
        case WDB_ECUDA: return "CUDA error";
        case WDB_ENAN: return "NaN or Inf";
        case WDB_ETIMEOUT: return "timeout";
        case WDB_EDIVERGED: return "diverged";
        case WDB_EUNSUPPORTED: return "unsupported";
        case WDB_EIO: return "I/O error";
        case WDB_EPLAN: return "tile plan invariant broken";
    }
    return "unknown status";
}

const char* wdb_last_error(void) { return last_error(); }

long long wdb_kernel_launches(int reset) { return launches(reset); }

}  // extern "C"
