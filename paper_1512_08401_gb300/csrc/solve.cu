// FISTA drivers: Algorithm 3 on Theta_K (kernels 1 and 2 of subband_ops.cu) and the exact
// operator path (Algorithm 1 gradient: IDWT, R2C, spectral residual, C2R, DWT, step).
//
// The iteration runs on the device without host round trips: the step kernel's last CTA
// updates k, evaluates the duality gap of y^(k) every check_every iterations and raises a
// stop flag that turns the remaining kernels of the chunk into no-ops. The host replays a
// CUDA graph of check_every iterations and reads the 200-byte state after each replay.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "device_util.cuh"
#include "fftops.cuh"
#include "solve_impl.h"
#include "subband_ops.cuh"
#include "theta_impl.h"

namespace wdb {

namespace {

// r^ = h^ z^ - u0^ (Parseval partials over the half spectrum), z^ <- conj(h^) r^ / N
__global__ void __launch_bounds__(256) spectral_kernel(cufftComplex* __restrict__ Z, const cufftComplex* __restrict__ H,
                                                       const cufftComplex* __restrict__ U, int C2, int C, long long n,
                                                       float invN, int write_grad, double* part, unsigned int* counter,
                                                       SolveState* st, double* out_rr) {
    if (st && *(volatile int*)&st->stop) return;
    float rs = 0.f, rc = 0.f, xs = 0.f, xc = 0.f;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int kx = (int)(k % C2);
        const float wgt = (kx == 0 || (2 * kx == C)) ? 1.f : 2.f;
        const cufftComplex z = Z[k], h = H[k], u = U[k];
        const float rx = h.x * z.x - h.y * z.y - u.x;
        const float ry = h.x * z.y + h.y * z.x - u.y;
        neu_add(rs, rc, wgt * (rx * rx + ry * ry));
        neu_add(xs, xc, wgt * (u.x * rx + u.y * ry));
        if (write_grad) Z[k] = make_cuComplex((h.x * rx + h.y * ry) * invN, (h.x * ry - h.y * rx) * invN);
    }
    double v[2] = {(double)rs + (double)rc, (double)xs + (double)xc}, tot[2];
    if (grid_reduce<2>(v, 0u, part, counter, tot) && threadIdx.x == 0) {
        if (st) {
            st->rr = tot[0] * (double)invN;
            st->x0r = tot[1] * (double)invN;
        }
        if (out_rr) out_rr[0] = tot[0] * (double)invN;
    }
}

int ew_grid(long long n) {
    long long g = (n + 255) / 256;
    return (int)std::min<long long>(std::max<long long>(g, 1), 1216);
}

SolveState init_state(const wdb_solve_params* p, int m) {
    SolveState s;
    std::memset(&s, 0, sizeof s);
    s.k = 1;
    s.max_iters = p->max_iters;
    s.check_every = m;
    s.tol = p->tol;
    s.primal = s.dual = s.gap = s.rel_gap = NAN;
    s.target = p->target_objective > 0.0 ? p->target_objective : 0.0;
    s.ista = p->ista ? 1 : 0;
    return s;
}

wdb_status check_params(const wdb_solve_params* p, int S) {
    if (!p) return set_error(WDB_EINVAL, "params is NULL");
    if (p->max_iters < 1) return set_error(WDB_EINVAL, "max_iters must be >= 1");
    if (!(p->tol >= 0.0) || !std::isfinite(p->tol)) return set_error(WDB_EINVAL, "tol must be finite and >= 0");
    if (!std::isfinite(p->target_objective)) return set_error(WDB_EINVAL, "target_objective must be finite");
    if (p->precond < 0 || p->precond > 2) return set_error(WDB_EINVAL, "unknown preconditioner %d", p->precond);
    if (!p->w_subband_host && !(p->lambda >= 0.0 && std::isfinite(p->lambda)))
        return set_error(WDB_EINVAL, "lambda must be finite and >= 0");
    if (p->w_subband_host)
        for (int b = 0; b < S; ++b)
            if (!(p->w_subband_host[b] >= 0.0) || !std::isfinite(p->w_subband_host[b]))
                return set_error(WDB_EINVAL, "w_subband[%d] must be finite and >= 0", b);
    return WDB_OK;
}

std::vector<float> weights(const wdb_solve_params* p, int S) {
    std::vector<float> w(S);
    for (int b = 0; b < S; ++b) w[b] = (float)(p->w_subband_host ? p->w_subband_host[b] : p->lambda);
    return w;
}

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Shared iteration engine
// ---------------------------------------------------------------------------------------
// Runs chunks of m iterations (enqueue(m) puts m iterations on the stream) until the
// device state says stop. With graphs, the chunk is captured once per (key) and replayed.
static wdb_status run_loop(IterEngine& E, int m, bool use_graph, bool timed, long long kernels_per_chunk,
                           cudaStream_t st) {
    SolveState* hs = E.h_state;
    E.sum_k1 = E.sum_k2 = 0.0;
    E.n_timed = 0;
    if (timed && !E.ev[0])
        for (auto& e : E.ev) WDB_CK(cudaEventCreate(&e));
    auto enqueue_chunk = [&]() -> wdb_status {
        if (!timed) return E.enqueue(m);
        if (m > 1) WDB_TRY(E.enqueue(m - 1));
        return E.enqueue_timed(E.ev);
    };
    auto harvest = [&](int chunk) -> wdb_status {
        // the sample is valid only if the chunk's last iteration ran (no stop before it)
        if (timed && hs->iters_done >= chunk * m) {
            float a = 0.f, b = 0.f;
            WDB_CK(cudaEventElapsedTime(&a, E.ev[0], E.ev[1]));
            WDB_CK(cudaEventElapsedTime(&b, E.ev[1], E.ev[2]));
            E.sum_k1 += a;
            E.sum_k2 += b;
            E.n_timed++;
        }
        return WDB_OK;
    };
    if (!use_graph) {
        for (int chunk = 1;; ++chunk) {
            WDB_TRY(enqueue_chunk());
            WDB_CK(cudaMemcpyAsync(hs, E.d_state, sizeof(SolveState), cudaMemcpyDeviceToHost, st));
            WDB_CK(cudaStreamSynchronize(st));
            WDB_TRY(harvest(chunk));
            if (hs->stop) break;
        }
        return WDB_OK;
    }
    if (!E.graph_exec || E.graph_m != m || E.graph_timed != timed) {
        if (E.graph_exec) {
            cudaGraphExecDestroy(E.graph_exec);
            E.graph_exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        WDB_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        wdb_status s = enqueue_chunk();
        cudaError_t ce = cudaMemcpyAsync(hs, E.d_state, sizeof(SolveState), cudaMemcpyDeviceToHost, st);
        cudaError_t ee = cudaStreamEndCapture(st, &g);
        if (s != WDB_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (ce != cudaSuccess) return cuda_error(ce, "capture state copy", __FILE__, __LINE__);
        if (ee != cudaSuccess) return cuda_error(ee, "cudaStreamEndCapture", __FILE__, __LINE__);
        ce = cudaGraphInstantiate(&E.graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) return cuda_error(ce, "cudaGraphInstantiate", __FILE__, __LINE__);
        E.graph_m = m;
        E.graph_timed = timed;
        E.graph_kernels = kernels_per_chunk;
        count_launch(-kernels_per_chunk);   // captured, not launched
    }
    for (int chunk = 1;; ++chunk) {
        WDB_CK(cudaGraphLaunch(E.graph_exec, st));
        count_launch(E.graph_kernels);
        WDB_CK(cudaStreamSynchronize(st));
        WDB_TRY(harvest(chunk));
        if (hs->stop) break;
    }
    return WDB_OK;
}

static wdb_status record_ev(cudaEvent_t ev, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    WDB_CK(cudaStreamIsCapturing(st, &cs));
    if (cs == cudaStreamCaptureStatusActive) WDB_CK(cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal));
    else WDB_CK(cudaEventRecord(ev, st));
    return WDB_OK;
}

// The loop pieces above, for the other operator types (vtheta.cu).
SolveState solve_init_state(const wdb_solve_params* p, int m) { return init_state(p, m); }
wdb_status solve_check_params(const wdb_solve_params* p, int S) { return check_params(p, S); }
std::vector<float> solve_weights(const wdb_solve_params* p, int S) { return weights(p, S); }
double solve_now_ms() { return now_ms(); }
wdb_status solve_run_loop(IterEngine& E, int m, bool use_graph, bool timed, long long kernels_per_chunk,
                          cudaStream_t st) {
    return run_loop(E, m, use_graph, timed, kernels_per_chunk, st);
}
wdb_status solve_record_ev(cudaEvent_t ev, cudaStream_t st) { return record_ev(ev, st); }

wdb_status work_enter(cudaStream_t* work, cudaEvent_t* ev_in, cudaEvent_t* ev_out, cudaStream_t caller) {
    if (!*work) WDB_CK(cudaStreamCreateWithFlags(work, cudaStreamNonBlocking));
    if (!*ev_in) WDB_CK(cudaEventCreateWithFlags(ev_in, cudaEventDisableTiming));
    if (!*ev_out) WDB_CK(cudaEventCreateWithFlags(ev_out, cudaEventDisableTiming));
    WDB_CK(cudaEventRecord(*ev_in, caller));
    WDB_CK(cudaStreamWaitEvent(*work, *ev_in, 0));
    return WDB_OK;
}

wdb_status work_exit(cudaStream_t work, cudaEvent_t ev_out, cudaStream_t caller) {
    WDB_CK(cudaEventRecord(ev_out, work));
    WDB_CK(cudaStreamWaitEvent(caller, ev_out, 0));
    return WDB_OK;
}

void IterEngine::release() {
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    graph_exec = nullptr;
    for (auto& e : ev)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
}

// ---------------------------------------------------------------------------------------
// Theta_K path
// ---------------------------------------------------------------------------------------
wdb_status theta_workspace_public(wdb_theta* th, cudaStream_t st);
static wdb_status theta_workspace(wdb_theta* th, cudaStream_t st) { return theta_workspace_public(th, st); }
wdb_status theta_workspace_public(wdb_theta* th, cudaStream_t st) {
    if (th->ws_N == th->lay.N) return WDB_OK;
    const long long N = th->lay.N;
    WDB_TRY(th_alloc(th, &th->d_x0, N));
    WDB_TRY(th_alloc(th, &th->d_y, N));
    WDB_TRY(th_alloc(th, &th->d_r, N));
    WDB_TRY(th_alloc(th, &th->d_xs, N));
    WDB_TRY(th_alloc(th, &th->d_scr, N / 2 + 1));
    WDB_TRY(th_alloc(th, &th->d_w, th->lay.S));
    WDB_TRY(th_alloc(th, &th->d_part, (size_t)th->part_len * 4));
    void* p = nullptr;
    WDB_CK(cudaMalloc(&p, sizeof(SolveState)));
    th->allocs.push_back(p);
    th->d_state = static_cast<SolveState*>(p);
    WDB_CK(cudaMallocHost(&p, sizeof(SolveState)));
    th->h_state = static_cast<SolveState*>(p);
    th->ws_N = N;
    return WDB_OK;
}

wdb_status theta_objective_dev(wdb_theta* th, const float* x, const float* x0, const float* w_dev, cudaStream_t st,
                               double* E, long long* support) {
    SubbandArgs F = subband_args(th);
    double* d_out = reinterpret_cast<double*>(&th->d_state->scratch[0]);
    WDB_TRY(tile_resnorm(tile_args(th, false, false), x, x0, th->d_r, d_out, th->d_red_part, st));
    WDB_TRY(launch_l1_terms(F, th->grid, x, w_dev, th_red(th, d_out + 1), st));
    double h[3];
    WDB_CK(cudaMemcpyAsync(h, d_out, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
    WDB_CK(cudaStreamSynchronize(st));
    *E = 0.5 * h[0] + h[1];
    if (support) *support = (long long)llround(h[2]);
    return WDB_OK;
}

wdb_status theta_solve(wdb_theta* th, const float* in, bool is_image, float* x_out, const wdb_solve_params* p,
                       cudaStream_t caller, wdb_solve_result* res) {
    const double t0 = now_ms();
    WDB_TRY(check_params(p, th->lay.S));
    WDB_TRY(work_enter(&th->work, &th->ev_in, &th->ev_out, caller));
    cudaStream_t st = th->work;
    WDB_TRY(theta_precond(th, p->precond, p->jacobi_eps, st));
    WDB_TRY(theta_workspace(th, st));
    const Layout& L = th->lay;
    const long long N = L.N;
    const int m = p->check_every > 0 ? p->check_every : 10;
    PrecondCache& pc = th->pc[p->precond];
    // x0 = Psi* u0 (a1) or the given coefficients
    if (is_image) WDB_TRY(dwt2<float>(in, th->d_x0, L, th->filt, th->d_scr, st));
    else WDB_CK(cudaMemcpyAsync(th->d_x0, in, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
    std::vector<float> w = weights(p, L.S);
    WDB_CK(cudaMemcpyAsync(th->d_w, w.data(), sizeof(float) * L.S, cudaMemcpyHostToDevice, st));
    if (p->x_init_dev) {
        WDB_CK(cudaMemcpyAsync(th->d_xs, p->x_init_dev, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
        WDB_CK(cudaMemcpyAsync(th->d_y, p->x_init_dev, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
    } else {
        WDB_CK(cudaMemsetAsync(th->d_xs, 0, sizeof(float) * N, st));
        WDB_CK(cudaMemsetAsync(th->d_y, 0, sizeof(float) * N, st));
    }
    SolveState s0 = init_state(p, m);
    WDB_CK(cudaMemcpyAsync(th->d_state, &s0, sizeof s0, cudaMemcpyHostToDevice, st));
    const TileArgs F = tile_args(th, false, false), A = tile_args(th, true, false);
    IterEngine& E = th->engine[p->precond];
    E.d_state = th->d_state;
    E.h_state = th->h_state;
    const float* step = pc.d_step;
    const bool fused = p->fused != 0 && tile_fused_supported(F, A);
    const long long spin = p->spin_limit;
    if (fused) {
        // one cooperative launch per chunk (no graph needed)
        E.enqueue = [=](int iters) -> wdb_status {
            return tile_fused(F, A, th->d_y, th->d_x0, th->d_r, th->d_xs, step, th->d_w, th->d_part, th->d_state, iters,
                              spin, 2 * th->part_len, st);
        };
    } else {
        E.enqueue = [=](int iters) -> wdb_status {
            for (int i = 0; i < iters; ++i) {
                // each kernel after the first is a programmatic dependent of the one before it
                WDB_TRY(tile_k1(F, th->d_y, th->d_x0, th->d_r, th->d_part, th->d_state, st, i > 0));
                WDB_TRY(tile_k2(A, th->d_r, th->d_y, th->d_xs, step, th->d_w, th->d_part, th->d_state, st, true));
            }
            return WDB_OK;
        };
    }
    E.enqueue_timed = [=](cudaEvent_t* ev) -> wdb_status {
        WDB_TRY(record_ev(ev[0], st));
        WDB_TRY(tile_k1(F, th->d_y, th->d_x0, th->d_r, th->d_part, th->d_state, st));
        WDB_TRY(record_ev(ev[1], st));
        WDB_TRY(tile_k2(A, th->d_r, th->d_y, th->d_xs, step, th->d_w, th->d_part, th->d_state, st));
        WDB_TRY(record_ev(ev[2], st));
        return WDB_OK;
    };
    WDB_TRY(run_loop(E, m, !p->no_graph && !fused, p->time_kernels != 0, 2LL * m, st));
    SolveState hs = *th->h_state;
    if (hs.timeout) {
        // a pass that ran without its full grid left its work queue unreset
        WDB_CK(cudaMemsetAsync(F.queue, 0, sizeof(TileQueue), st));
        WDB_CK(cudaMemsetAsync(A.queue, 0, sizeof(TileQueue), st));
    }
    double Eobj = 0.0;
    long long sup = 0;
    WDB_TRY(theta_objective_dev(th, th->d_xs, th->d_x0, th->d_w, st, &Eobj, &sup));
    Kkt64 kk{NAN, NAN, NAN, NAN, NAN, NAN, 0};
    if (p->kkt_check) {
        std::vector<double> w64(L.S);
        for (int b = 0; b < L.S; ++b) w64[b] = p->w_subband_host ? p->w_subband_host[b] : p->lambda;
        WDB_TRY(theta_kkt64(th, th->d_xs, th->d_x0, w64.data(), st, &kk));
    }
    WDB_CK(cudaMemcpyAsync(x_out, th->d_xs, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
    WDB_TRY(work_exit(st, th->ev_out, caller));
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
    res->kkt_off = kk.kkt_off;
    res->kkt_on = kk.kkt_on;
    res->gap64 = kk.gap;
    res->rel_gap64 = kk.rel_gap;
    res->status = WDB_OK;
    if (hs.timeout)
        res->status = set_error(WDB_ETIMEOUT, "a grid barrier of the fused loop gave up after %lld polls",
                                p->spin_limit > 0 ? p->spin_limit : (1LL << 23));
    else if (hs.nan_flag || !std::isfinite(Eobj)) res->status = set_error(WDB_ENAN, "NaN/Inf in the objective");
    else if (hs.diverged)
        res->status = set_error(WDB_EDIVERGED, "objective %g at iteration %d, above 1e6 x its first value %g",
                                hs.primal, hs.iters_done, hs.first_primal);
    res->solve_ms = now_ms() - t0;
    return res->status;
}

// ---------------------------------------------------------------------------------------
// FFT path
// ---------------------------------------------------------------------------------------
static wdb_status fft_alloc(wdb_fftop* op, void** p, size_t bytes) {
    WDB_CK(cudaMalloc(p, std::max<size_t>(bytes, 1)));
    op->allocs.push_back(*p);
    return WDB_OK;
}

// diag tables of M = Psi* H^T H Psi (constant per subband) and max |h^|^2, FP64
static wdb_status fft_diagonals(wdb_fftop* op, const double* psf_dev, int kh, int kw, cudaStream_t st) {
    const Layout& L = op->lay;
    const long long N = L.N;
    const int R = L.n_rows, C = L.n_cols, C2 = C / 2 + 1;
    const long long NC = (long long)R * C2;
    double *img = nullptr, *coef = nullptr, *scr = nullptr, *d_out = nullptr;
    cufftDoubleComplex *hh = nullptr, *spec = nullptr, *prod = nullptr;
    std::vector<void*> tmp;
    auto dm = [&](void** p, size_t b) -> wdb_status {
        WDB_CK(cudaMalloc(p, std::max<size_t>(b, 1)));
        tmp.push_back(*p);
        return WDB_OK;
    };
    wdb_status s = WDB_OK;
    cufftHandle pf = 0, pi = 0;
    bool hf = false, hi = false;
    std::vector<double> out(2 * L.S + 1);
    do {
        if ((s = dm((void**)&img, sizeof(double) * N))) break;
        if ((s = dm((void**)&coef, sizeof(double) * N))) break;
        if ((s = dm((void**)&scr, sizeof(double) * (N / 2 + 1)))) break;
        if ((s = dm((void**)&d_out, sizeof(double) * (2 * L.S + 1)))) break;
        hh = op->d_hhat64;
        if ((s = dm((void**)&spec, sizeof(cufftDoubleComplex) * NC))) break;
        if ((s = dm((void**)&prod, sizeof(cufftDoubleComplex) * NC))) break;
        cufftResult fr = cufftPlan2d(&pf, R, C, CUFFT_D2Z);
        if (fr != CUFFT_SUCCESS) { s = cufft_error(fr, "plan D2Z", __FILE__, __LINE__); break; }
        hf = true;
        fr = cufftPlan2d(&pi, R, C, CUFFT_Z2D);
        if (fr != CUFFT_SUCCESS) { s = cufft_error(fr, "plan Z2D", __FILE__, __LINE__); break; }
        hi = true;
        cufftSetStream(pf, st);
        cufftSetStream(pi, st);
        if ((s = launch_pad_psf(psf_dev, kh, kw, img, R, C, st))) break;
        fr = cufftExecD2Z(pf, img, hh);
        if (fr != CUFFT_SUCCESS) { s = cufft_error(fr, "D2Z psf", __FILE__, __LINE__); break; }
        if ((s = launch_c64_to_c32(hh, op->d_hhat, NC, st))) break;
        if ((s = launch_max_abs2(hh, NC, d_out + 2 * L.S, st))) break;
        for (int b = 0; b < L.S && s == WDB_OK; ++b) {
            cudaMemsetAsync(coef, 0, sizeof(double) * N, st);
            const double one = 1.0;
            cudaMemcpyAsync(coef + L.sb[b].off, &one, sizeof(double), cudaMemcpyHostToDevice, st);
            if ((s = idwt2<double>(coef, img, L, op->filt, scr, st))) break;
            fr = cufftExecD2Z(pf, img, spec);
            if (fr != CUFFT_SUCCESS) { s = cufft_error(fr, "D2Z", __FILE__, __LINE__); break; }
            for (int which = 0; which < 2 && s == WDB_OK; ++which) {
                if (which == 0) s = launch_cmul64(spec, hh, prod, NC, 0, 1.0 / (double)N, st);
                else s = launch_cmul_abs2_64(spec, hh, prod, NC, 1.0 / (double)N, st);
                if (s) break;
                fr = cufftExecZ2D(pi, prod, img);
                if (fr != CUFFT_SUCCESS) { s = cufft_error(fr, "Z2D", __FILE__, __LINE__); break; }
                RedTarget red{op->d_counter, op->d_red_part, d_out + 2 * b + which};
                s = launch_norm2<double>(img, N, red, op->grid, st);
            }
        }
        if (s) break;
        cudaError_t ce = cudaMemcpyAsync(out.data(), d_out, sizeof(double) * out.size(), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) { s = cuda_error(ce, "fft diagonals", __FILE__, __LINE__); break; }
    } while (false);
    if (hf) cufftDestroy(pf);
    if (hi) cufftDestroy(pi);
    cudaStreamSynchronize(st);
    for (void* p : tmp) cudaFree(p);
    if (s) return s;
    op->Md_sb.resize(L.S);
    op->M2d_sb.resize(L.S);
    for (int b = 0; b < L.S; ++b) {
        op->Md_sb[b] = out[2 * b];
        op->M2d_sb[b] = out[2 * b + 1];
    }
    op->L_closed = out[2 * L.S];
    return WDB_OK;
}

wdb_status fftop_create(const double* psf_host, int kh, int kw, const Layout& L, const Filters& f,
                        const char* wavelet, cudaStream_t st, wdb_fftop** out) {
    wdb_fftop* op = new (std::nothrow) wdb_fftop();
    if (!op) return set_error(WDB_ENOMEM, "host allocation");
    op->lay = L;
    op->filt = f;
    op->wavelet = wavelet;
    const long long N = L.N;
    const int R = L.n_rows, C = L.n_cols, C2 = C / 2 + 1;
    const long long NC = (long long)R * C2;
    wdb_status s = WDB_OK;
    double* psf = nullptr;
    do {
        if ((s = fft_alloc(op, (void**)&op->d_hhat, sizeof(cufftComplex) * NC))) break;
        if ((s = fft_alloc(op, (void**)&op->d_hhat64, sizeof(cufftDoubleComplex) * NC))) break;
        if ((s = fft_alloc(op, (void**)&op->d_uhat, sizeof(cufftComplex) * NC))) break;
        if ((s = fft_alloc(op, (void**)&op->d_Z, sizeof(cufftComplex) * NC))) break;
        if ((s = fft_alloc(op, (void**)&op->d_z, sizeof(float) * N))) break;
        if ((s = fft_alloc(op, (void**)&op->d_g, sizeof(float) * N))) break;
        if ((s = fft_alloc(op, (void**)&op->d_xs, sizeof(float) * N))) break;
        if ((s = fft_alloc(op, (void**)&op->d_y, sizeof(float) * N))) break;
        if ((s = fft_alloc(op, (void**)&op->d_scr, sizeof(float) * (N / 2 + 1)))) break;
        if ((s = fft_alloc(op, (void**)&op->d_w, sizeof(float) * L.S))) break;
        std::vector<SubbandDev> sbv(L.sb, L.sb + L.S);
        if ((s = fft_alloc(op, (void**)&op->d_sb, sizeof(SubbandDev) * L.S))) break;
        cudaMemcpyAsync(op->d_sb, sbv.data(), sizeof(SubbandDev) * L.S, cudaMemcpyHostToDevice, st);
        op->sched = make_schedule(L);
        if ((s = fft_alloc(op, (void**)&op->d_vb_start, sizeof(int) * op->sched.vb_start.size()))) break;
        cudaMemcpyAsync(op->d_vb_start, op->sched.vb_start.data(), sizeof(int) * op->sched.vb_start.size(),
                        cudaMemcpyHostToDevice, st);
        op->grid = std::max(1, std::min(op->sched.nvb, subband_grid_limit()));
        if ((s = fft_alloc(op, (void**)&op->d_part, sizeof(double) * op->grid * 4))) break;
        if ((s = fft_alloc(op, (void**)&op->d_red_part, sizeof(double) * op->grid * 4))) break;
        if ((s = fft_alloc(op, (void**)&op->d_counter, sizeof(unsigned int) * 4))) break;
        cudaMemsetAsync(op->d_counter, 0, sizeof(unsigned int) * 4, st);
        if ((s = fft_alloc(op, (void**)&op->d_state, sizeof(SolveState)))) break;
        void* hp = nullptr;
        cudaError_t ce = cudaMallocHost(&hp, sizeof(SolveState));
        if (ce != cudaSuccess) { s = cuda_error(ce, "cudaMallocHost", __FILE__, __LINE__); break; }
        op->h_state = static_cast<SolveState*>(hp);
        cufftResult fr = cufftPlan2d(&op->r2c, R, C, CUFFT_R2C);
        if (fr != CUFFT_SUCCESS) { s = cufft_error(fr, "plan R2C", __FILE__, __LINE__); break; }
        op->have_r2c = true;
        fr = cufftPlan2d(&op->c2r, R, C, CUFFT_C2R);
        if (fr != CUFFT_SUCCESS) { s = cufft_error(fr, "plan C2R", __FILE__, __LINE__); break; }
        op->have_c2r = true;
        ce = cudaMalloc(&psf, sizeof(double) * kh * kw);
        if (ce != cudaSuccess) { s = cuda_error(ce, "cudaMalloc", __FILE__, __LINE__); break; }
        cudaMemcpyAsync(psf, psf_host, sizeof(double) * kh * kw, cudaMemcpyHostToDevice, st);
        s = fft_diagonals(op, psf, kh, kw, st);
    } while (false);
    if (psf) cudaFree(psf);
    if (s != WDB_OK) {
        fftop_free(op);
        return s;
    }
    *out = op;
    return WDB_OK;
}

void fftop_free(wdb_fftop* op) {
    if (!op) return;
    if (op->work) cudaStreamSynchronize(op->work);
    op->engine.release();
    if (op->work) cudaStreamDestroy(op->work);
    if (op->ev_in) cudaEventDestroy(op->ev_in);
    if (op->ev_out) cudaEventDestroy(op->ev_out);
    if (op->have_r2c) cufftDestroy(op->r2c);
    if (op->have_c2r) cufftDestroy(op->c2r);
    for (void* p : op->allocs) cudaFree(p);
    if (op->h_state) cudaFreeHost(op->h_state);
    for (auto& pc : op->pc) (void)pc;
    delete op;
}

static SubbandArgs fft_args(const wdb_fftop* op) {
    SubbandArgs A{};
    A.sb = op->d_sb;
    A.vb_start = op->d_vb_start;
    A.S = op->lay.S;
    A.nvb = op->sched.nvb;
    return A;
}

// power iteration on P^-1/2 Psi* H^T H Psi P^-1/2 in FP64
static wdb_status fft_power(wdb_fftop* op, const std::vector<double>& Ptab, cudaStream_t st, double* L_out) {
    const Layout& L = op->lay;
    const long long N = L.N;
    const int R = L.n_rows, C = L.n_cols, C2 = C / 2 + 1;
    const long long NC = (long long)R * C2;
    std::vector<double> sc(Ptab.size());
    for (size_t i = 0; i < sc.size(); ++i) sc[i] = 1.0 / std::sqrt(Ptab[i]);
    double *v = nullptr, *t = nullptr, *img = nullptr, *scr = nullptr, *d_sc = nullptr, *d_out = nullptr;
    cufftDoubleComplex *hh = nullptr, *spec = nullptr;
    std::vector<void*> tmp;
    auto dm = [&](void** p, size_t b) -> wdb_status {
        WDB_CK(cudaMalloc(p, std::max<size_t>(b, 1)));
        tmp.push_back(*p);
        return WDB_OK;
    };
    cufftHandle pf = 0, pi = 0;
    bool hf = false, hi = false;
    wdb_status s = WDB_OK;
    double lam = 0.0;
    SubbandArgs A = fft_args(op);
    do {
        if ((s = dm((void**)&v, sizeof(double) * N))) break;
        if ((s = dm((void**)&t, sizeof(double) * N))) break;
        if ((s = dm((void**)&img, sizeof(double) * N))) break;
        if ((s = dm((void**)&scr, sizeof(double) * (N / 2 + 1)))) break;
        if ((s = dm((void**)&d_sc, sizeof(double) * sc.size()))) break;
        if ((s = dm((void**)&d_out, sizeof(double)))) break;
        hh = op->d_hhat64;
        if ((s = dm((void**)&spec, sizeof(cufftDoubleComplex) * NC))) break;
        cudaMemcpyAsync(d_sc, sc.data(), sizeof(double) * sc.size(), cudaMemcpyHostToDevice, st);
        if (cufftPlan2d(&pf, R, C, CUFFT_D2Z) != CUFFT_SUCCESS) { s = set_error(WDB_ECUDA, "plan D2Z"); break; }
        hf = true;
        if (cufftPlan2d(&pi, R, C, CUFFT_Z2D) != CUFFT_SUCCESS) { s = set_error(WDB_ECUDA, "plan Z2D"); break; }
        hi = true;
        cufftSetStream(pf, st);
        cufftSetStream(pi, st);
        RedTarget red{op->d_counter, op->d_red_part, d_out};
        if ((s = launch_splitmix<double>(v, N, kPowerSeed, st))) break;
        if ((s = launch_norm2<double>(v, N, red, op->grid, st))) break;
        double h = 0.0;
        cudaMemcpyAsync(&h, d_out, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) { s = set_error(WDB_ECUDA, "power start"); break; }
        if ((s = launch_scale_const<double>(v, v, N, 1.0 / std::sqrt(h), st))) break;
        for (int it = 1; it <= kPowerIters; ++it) {
            if ((s = launch_scale<double>(A, op->grid, v, t, d_sc, st))) break;
            if ((s = idwt2<double>(t, img, L, op->filt, scr, st))) break;
            if (cufftExecD2Z(pf, img, spec) != CUFFT_SUCCESS) { s = set_error(WDB_ECUDA, "D2Z"); break; }
            if ((s = launch_cmul_abs2_64(spec, hh, spec, NC, 1.0 / (double)N, st))) break;
            if (cufftExecZ2D(pi, spec, img) != CUFFT_SUCCESS) { s = set_error(WDB_ECUDA, "Z2D"); break; }
            if ((s = dwt2<double>(img, t, L, op->filt, scr, st))) break;
            if ((s = launch_scale<double>(A, op->grid, t, t, d_sc, st))) break;
            if ((s = launch_norm2<double>(t, N, red, op->grid, st))) break;
            cudaMemcpyAsync(&h, d_out, sizeof(double), cudaMemcpyDeviceToHost, st);
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
    if (hf) cufftDestroy(pf);
    if (hi) cufftDestroy(pi);
    cudaStreamSynchronize(st);
    for (void* p : tmp) cudaFree(p);
    if (s) return s;
    if (!std::isfinite(lam)) return set_error(WDB_ENAN, "power iteration produced %g", lam);
    *L_out = lam;
    return WDB_OK;
}

std::vector<double> fft_expand(const wdb_fftop* op, const std::vector<double>& per_sb) {
    const Layout& L = op->lay;
    std::vector<double> t(L.tab_len);
    for (int b = 0; b < L.S; ++b) {
        const int n = 1 << (2 * L.sb[b].lgR);
        for (int i = 0; i < n; ++i) t[L.sb[b].tab_off + i] = per_sb[b];
    }
    return t;
}

wdb_status fftop_precond(wdb_fftop* op, int kind, double eps, cudaStream_t st) {
    if (kind < 0 || kind > 2) return set_error(WDB_EINVAL, "unknown preconditioner %d", kind);
    PrecondCache& pc = op->pc[kind];
    if (pc.valid && (pc.pinned || kind != WDB_PRECOND_JACOBI || pc.eps == eps)) return WDB_OK;
    std::vector<double> Psb = precond_table(op->Md_sb, op->M2d_sb, kind, eps);
    pc.P = fft_expand(op, Psb);
    double Lh = op->L_closed;   // Psi orthogonal: ||H Psi||^2 = max |h^|^2
    if (kind != WDB_PRECOND_NONE) WDB_TRY(fft_power(op, pc.P, st, &Lh));
    pc.L_hat = Lh;
    pc.tau = Lh > 0.0 ? 1.0 / (kStepMargin * Lh) : 1.0;
    pc.eps = eps;
    if (!pc.d_step) WDB_TRY(fft_alloc(op, (void**)&pc.d_step, sizeof(float) * pc.P.size()));
    std::vector<float> stp(pc.P.size());
    for (size_t i = 0; i < stp.size(); ++i) stp[i] = (float)(pc.tau / pc.P[i]);
    WDB_CK(cudaMemcpyAsync(pc.d_step, stp.data(), sizeof(float) * stp.size(), cudaMemcpyHostToDevice, st));
    WDB_CK(cudaStreamSynchronize(st));
    pc.valid = true;
    return WDB_OK;
}

// exact objective 1/2 ||H Psi x - u0||^2 + sum w |x| (u0^ already in d_uhat)
static wdb_status fft_objective(wdb_fftop* op, const float* x, cudaStream_t st, double* E, long long* sup) {
    const Layout& L = op->lay;
    const long long NC = (long long)L.n_rows * (L.n_cols / 2 + 1);
    WDB_TRY(idwt2<float>(x, op->d_z, L, op->filt, op->d_scr, st));
    cufftSetStream(op->r2c, st);
    WDB_CKF(cufftExecR2C(op->r2c, op->d_z, op->d_Z));
    double* d_out = reinterpret_cast<double*>(&op->d_state->scratch[0]);
    spectral_kernel<<<std::min(ew_grid(NC), op->grid), 256, 0, st>>>(op->d_Z, op->d_hhat, op->d_uhat, L.n_cols / 2 + 1, L.n_cols, NC,
                                                 1.0f / (float)L.N, 0, op->d_red_part, op->d_counter, nullptr, d_out);
    count_launch();
    WDB_CK(cudaGetLastError());
    SubbandArgs A = fft_args(op);
    WDB_TRY(launch_l1_terms(A, op->grid, x, op->d_w, RedTarget{op->d_counter, op->d_red_part, d_out + 1}, st));
    double h[3];
    WDB_CK(cudaMemcpyAsync(h, d_out, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
    WDB_CK(cudaStreamSynchronize(st));
    *E = 0.5 * h[0] + h[1];
    if (sup) *sup = (long long)llround(h[2]);
    return WDB_OK;
}

wdb_status fft_objective_public(wdb_fftop* op, const float* u, const float* x, const double* w_host,
                                cudaStream_t caller, double* E) {
    const Layout& L = op->lay;
    WDB_TRY(work_enter(&op->work, &op->ev_in, &op->ev_out, caller));
    cudaStream_t st = op->work;
    std::vector<float> w(L.S);
    for (int b = 0; b < L.S; ++b) w[b] = (float)w_host[b];
    WDB_CK(cudaMemcpyAsync(op->d_w, w.data(), sizeof(float) * L.S, cudaMemcpyHostToDevice, st));
    WDB_CK(cudaMemcpyAsync(op->d_z, u, sizeof(float) * L.N, cudaMemcpyDeviceToDevice, st));
    cufftSetStream(op->r2c, st);
    WDB_CKF(cufftExecR2C(op->r2c, op->d_z, op->d_uhat));
    WDB_TRY(fft_objective(op, x, st, E, nullptr));
    WDB_TRY(work_exit(st, op->ev_out, caller));
    WDB_CK(cudaStreamSynchronize(st));
    return WDB_OK;
}

wdb_status fft_solve(wdb_fftop* op, const float* u, float* x_out, const wdb_solve_params* p, cudaStream_t caller,
                     wdb_solve_result* res) {
    const double t0 = now_ms();
    const Layout& L = op->lay;
    WDB_TRY(check_params(p, L.S));
    WDB_TRY(work_enter(&op->work, &op->ev_in, &op->ev_out, caller));
    cudaStream_t st = op->work;
    WDB_TRY(fftop_precond(op, p->precond, p->jacobi_eps, st));
    const long long N = L.N;
    const int C2 = L.n_cols / 2 + 1;
    const long long NC = (long long)L.n_rows * C2;
    const int m = p->check_every > 0 ? p->check_every : 10;
    PrecondCache& pc = op->pc[p->precond];
    cufftSetStream(op->r2c, st);
    cufftSetStream(op->c2r, st);
    WDB_CK(cudaMemcpyAsync(op->d_z, u, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
    WDB_CKF(cufftExecR2C(op->r2c, op->d_z, op->d_uhat));
    std::vector<float> w = weights(p, L.S);
    WDB_CK(cudaMemcpyAsync(op->d_w, w.data(), sizeof(float) * L.S, cudaMemcpyHostToDevice, st));
    if (p->x_init_dev) {
        WDB_CK(cudaMemcpyAsync(op->d_xs, p->x_init_dev, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
        WDB_CK(cudaMemcpyAsync(op->d_y, p->x_init_dev, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
    } else {
        WDB_CK(cudaMemsetAsync(op->d_xs, 0, sizeof(float) * N, st));
        WDB_CK(cudaMemsetAsync(op->d_y, 0, sizeof(float) * N, st));
    }
    SolveState s0 = init_state(p, m);
    WDB_CK(cudaMemcpyAsync(op->d_state, &s0, sizeof s0, cudaMemcpyHostToDevice, st));
    SubbandArgs A = fft_args(op);
    IterEngine& E = op->engine;
    if (E.key != p->precond) E.release();
    E.key = p->precond;
    E.d_state = op->d_state;
    E.h_state = op->h_state;
    const float* step = pc.d_step;
    const float invN = 1.0f / (float)N;
    const int sgrid = std::min(ew_grid(NC), op->grid);
    E.enqueue = [=](int iters) -> wdb_status {
        for (int i = 0; i < iters; ++i) {
            WDB_TRY(idwt2<float>(op->d_y, op->d_z, L, op->filt, op->d_scr, st));
            WDB_CKF(cufftExecR2C(op->r2c, op->d_z, op->d_Z));
            spectral_kernel<<<sgrid, 256, 0, st>>>(op->d_Z, op->d_hhat, op->d_uhat, C2, L.n_cols, NC, invN, 1,
                                                         op->d_part, &op->d_state->done[0], op->d_state, nullptr);
            WDB_CK(cudaGetLastError());
            WDB_CKF(cufftExecC2R(op->c2r, op->d_Z, op->d_z));
            count_launch(1);
            WDB_TRY(dwt2<float>(op->d_z, op->d_g, L, op->filt, op->d_scr, st));
            WDB_TRY(launch_fft_step(A, op->grid, op->d_g, op->d_y, op->d_xs, step, op->d_w, op->d_part, op->d_state, st));
        }
        return WDB_OK;
    };
    E.enqueue_timed = [=](cudaEvent_t* ev) -> wdb_status {
        WDB_TRY(record_ev(ev[0], st));
        WDB_TRY(idwt2<float>(op->d_y, op->d_z, L, op->filt, op->d_scr, st));
        WDB_CKF(cufftExecR2C(op->r2c, op->d_z, op->d_Z));
        spectral_kernel<<<sgrid, 256, 0, st>>>(op->d_Z, op->d_hhat, op->d_uhat, C2, L.n_cols, NC, invN, 1,
                                               op->d_part, &op->d_state->done[0], op->d_state, nullptr);
        WDB_CK(cudaGetLastError());
        WDB_CKF(cufftExecC2R(op->c2r, op->d_Z, op->d_z));
        count_launch(1);
        WDB_TRY(dwt2<float>(op->d_z, op->d_g, L, op->filt, op->d_scr, st));
        WDB_TRY(record_ev(ev[1], st));
        WDB_TRY(launch_fft_step(A, op->grid, op->d_g, op->d_y, op->d_xs, step, op->d_w, op->d_part, op->d_state, st));
        WDB_TRY(record_ev(ev[2], st));
        return WDB_OK;
    };
    WDB_TRY(run_loop(E, m, !p->no_graph, p->time_kernels != 0, (long long)m * (2 * L.J + 2), st));
    SolveState hs = *op->h_state;
    double Eobj = 0.0;
    long long sup = 0;
    WDB_TRY(fft_objective(op, op->d_xs, st, &Eobj, &sup));
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
    res->solve_ms = now_ms() - t0;
    return res->status;
}

}  // namespace wdb
