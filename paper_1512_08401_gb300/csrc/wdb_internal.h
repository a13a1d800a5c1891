// Internal declarations of libwdb (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <functional>
#include <string>
#include <vector>

#include "../../include/wdb.h"
#include "layout_types.h"

namespace wdb {

// ---------------------------------------------------------------------------------------
// Daubechies filters (derived on the host by spectral factorisation)
// ---------------------------------------------------------------------------------------
struct Filters {
    int L = 0;
    double h[kMaxL], g[kMaxL];
};
wdb_status wavelet_filters(const char* name, Filters* out);

template <typename T>
struct FiltT {
    int L;
    T h[kMaxL], g[kMaxL];
};
template <typename T>
FiltT<T> filt_cast(const Filters& f) {
    FiltT<T> o;
    o.L = f.L;
    for (int k = 0; k < kMaxL; k++) {
        o.h[k] = (T)(k < f.L ? f.h[k] : 0.0);
        o.g[k] = (T)(k < f.L ? f.g[k] : 0.0);
    }
    return o;
}

// ---------------------------------------------------------------------------------------
// Wavelet transforms (dwt.cu). scratch holds >= N/2 elements.
// ---------------------------------------------------------------------------------------
template <typename T>
wdb_status dwt2(const T* img, T* coef, const Layout& L, const Filters& f, T* scratch,
                cudaStream_t st);
template <typename T>
wdb_status idwt2(const T* coef, T* img, const Layout& L, const Filters& f, T* scratch,
                 cudaStream_t st);

// Reduction slots for one-off launches (power iteration, probes, objective).
struct RedSlot {
    unsigned int done;
    unsigned int pad;
    double sum[4];
};

// Virtual-block schedule: blocks of kVB consecutive outputs that stay inside one subband.
constexpr int kVB = 256;
struct Schedule {
    int nvb = 0;                 // number of virtual blocks
    std::vector<int> vb_start;   // [S+1] first virtual block of each subband
};
Schedule make_schedule(const Layout& L);

struct Tap {
    int a, b, oy, ox;
    double v;
};

// ---------------------------------------------------------------------------------------
// Theta handle internals
// ---------------------------------------------------------------------------------------
struct PrecondCache {
    bool valid = false;
    bool pinned = false;     // set by the caller (wdb_*_set_precond): never recomputed
    double eps = 0.0;
    std::vector<double> P;   // tab_len
    double tau = 0.0, L_hat = 0.0;
    float* d_step = nullptr; // tab_len floats: tau / P (device)
    float* d_Pf = nullptr;   // tab_len floats: P
};

// A non-blocking library stream joined to the caller's stream with events on entry and
// exit, so that graph capture works whatever stream the caller uses (including the legacy
// default stream, which cannot be captured).
struct WorkStream {
    cudaStream_t* work;
    cudaEvent_t* ev_in;
    cudaEvent_t* ev_out;
};
wdb_status work_enter(cudaStream_t* work, cudaEvent_t* ev_in, cudaEvent_t* ev_out, cudaStream_t caller);
wdb_status work_exit(cudaStream_t work, cudaEvent_t ev_out, cudaStream_t caller);

// Replays chunks of iterations (as a CUDA graph when enabled) until the device state stops.
struct IterEngine {
    std::function<wdb_status(int)> enqueue;   // puts `iters` iterations on the stream
    // puts one iteration on the stream with ev[0] before, ev[1] between the residual and
    // the step part, ev[2] after (event record nodes when captured)
    std::function<wdb_status(cudaEvent_t*)> enqueue_timed;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    bool graph_timed = false;
    double sum_k1 = 0.0, sum_k2 = 0.0;
    int n_timed = 0;
    cudaGraphExec_t graph_exec = nullptr;
    int graph_m = 0;
    long long graph_kernels = 0;
    int key = -1;
    SolveState* d_state = nullptr;
    SolveState* h_state = nullptr;
    void release();
};

}  // namespace wdb

#include "tile.cuh"

struct wdb_theta {
    wdb::Layout lay;
    wdb::Filters filt;
    std::string wavelet;
    int rule = 0;
    long long K_requested = 0, K_eff = 0, n_candidates = 0;
    double theta_max_abs = 0.0, build_ms = 0.0;
    std::vector<wdb::Tap> taps;            // sorted (a, b, oy, ox)
    wdb::TilePlanHost tplan[2][2];         // [0 Theta_K, 1 Theta_K^T][0 FP32, 1 FP64]
    std::vector<wdb::TileEntry> tent[2];   // gather-form taps of Theta_K and Theta_K^T (plan input)
    int plan_ctas = 0;                     // CTAs the plans are balanced for
    int tuned = 0;                         // 1: the FP32 plans were autotuned on this GPU
    std::vector<wdb::TileTune> tune_levels[2];   // the autotuner's tile side per output subband
    wdb::TilePlanHost bplan[2];            // FP32 plans for batched solves (large tiles: the
    wdb::TileArgs bargs[2];                // batch's many problems balance the CTAs)
    bool bplan_ok = false;
    wdb::TileArgs targs[2][2];
    int part_len = 0;                      // capacity (CTAs) of the per-CTA partial buffers
    std::vector<void*> allocs;             // device buffers owned by the handle
    wdb::SubbandDev* d_sb = nullptr;
    int* d_vb_start = nullptr;
    wdb::Schedule sched;
    int grid = 0;                          // CTAs for the persistent-style loops
    unsigned int* d_counter = nullptr;     // last-CTA counter for one-off reductions
    double* d_red_part = nullptr;          // per-CTA partials for one-off reductions
    bool diag_valid = false;
    std::vector<double> Md, M2d;           // phase tables of diag(M), diag(M^2)
    wdb::PrecondCache pc[3];
    // solve workspace (allocated on first solve)
    float *d_x0 = nullptr, *d_y = nullptr, *d_r = nullptr, *d_scr = nullptr, *d_xs = nullptr;
    wdb::IterEngine engine[3];             // one captured iteration chunk per preconditioner
    cudaStream_t work = nullptr;           // library stream the solve runs (and is captured) on
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    float* d_w = nullptr;                  // per-subband weights (S floats)
    double* d_part = nullptr;              // per-CTA partials
    wdb::SolveState* d_state = nullptr;
    wdb::SolveState* h_state = nullptr;    // pinned
    long long ws_N = 0;
    double *d_x64 = nullptr, *d_r64 = nullptr;   // FP64 check workspace (wdb_theta_kkt)
    double* d_kkt_out = nullptr;
};
