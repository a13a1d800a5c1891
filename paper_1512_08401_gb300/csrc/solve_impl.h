// Internal interface of the solvers (solve.cu) and the FFT-path handle.
#pragma once
#include <cufft.h>

#include "subband_ops.cuh"
#include "wdb_internal.h"

struct wdb_fftop {
    wdb::Layout lay;
    wdb::Filters filt;
    std::string wavelet;
    std::vector<void*> allocs;
    cufftHandle r2c = 0, c2r = 0;
    bool have_r2c = false, have_c2r = false;
    cufftComplex *d_hhat = nullptr, *d_uhat = nullptr, *d_Z = nullptr;
    cufftDoubleComplex* d_hhat64 = nullptr;
    float *d_z = nullptr, *d_g = nullptr, *d_xs = nullptr, *d_y = nullptr, *d_scr = nullptr, *d_w = nullptr;
    double *d_part = nullptr, *d_red_part = nullptr;
    unsigned int* d_counter = nullptr;
    wdb::SolveState* d_state = nullptr;
    wdb::SolveState* h_state = nullptr;
    wdb::SubbandDev* d_sb = nullptr;
    int* d_vb_start = nullptr;
    wdb::Schedule sched;
    int grid = 0;
    std::vector<double> Md_sb, M2d_sb;   // per subband (the exact operator is fully translation invariant)
    double L_closed = 0.0;               // max |h^|^2
    wdb::PrecondCache pc[3];
    wdb::IterEngine engine;
    cudaStream_t work = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

namespace wdb {

wdb_status theta_solve(wdb_theta* th, const float* in, bool is_image, float* x_out, const wdb_solve_params* p,
                       cudaStream_t st, wdb_solve_result* res);
wdb_status theta_objective_dev(wdb_theta* th, const float* x, const float* x0, const float* w_dev, cudaStream_t st,
                               double* E, long long* support);
wdb_status theta_workspace_public(wdb_theta* th, cudaStream_t st);
struct Kkt64 {
    double objective, gap, rel_gap, kkt_off, kkt_on, gmax;
    long long support;
};
// FP64 r = Theta_K x - x0, g = Theta_K^T r, KKT residuals, objective and gap of x (kkt.cu)
// (w_host: the problem's FP64 weights per subband)
wdb_status theta_kkt64(wdb_theta* th, const float* x, const float* x0, const double* w_host, cudaStream_t st,
                       Kkt64* out);
wdb_status fftop_create(const double* psf_host, int kh, int kw, const Layout& L, const Filters& f,
                        const char* wavelet, cudaStream_t st, wdb_fftop** out);
void fftop_free(wdb_fftop* op);
wdb_status fftop_precond(wdb_fftop* op, int kind, double eps, cudaStream_t st);
wdb_status solve_batch(int B, wdb_theta* const* ths, const float* const* u, float* const* x,
                       const wdb_solve_params* params, cudaStream_t caller, wdb_solve_result* res);
wdb_status fft_objective_public(wdb_fftop* op, const float* u, const float* x, const double* w_host,
                                cudaStream_t st, double* E);
wdb_status fft_solve(wdb_fftop* op, const float* u, float* x_out, const wdb_solve_params* p, cudaStream_t st,
                     wdb_solve_result* res);

// Solve-loop pieces shared with the row-varying operator (defined in solve.cu).
SolveState solve_init_state(const wdb_solve_params* p, int m);
wdb_status solve_check_params(const wdb_solve_params* p, int S);
std::vector<float> solve_weights(const wdb_solve_params* p, int S);
double solve_now_ms();
wdb_status solve_run_loop(IterEngine& E, int m, bool use_graph, bool timed, long long kernels_per_chunk,
                          cudaStream_t st);
wdb_status solve_record_ev(cudaEvent_t ev, cudaStream_t st);

}  // namespace wdb
