// Plain data types shared by host and device code of libwdb: errors, subband layout and
// the device-resident solver state.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/wdb.h"

namespace wdb {

constexpr int kMaxS = WDB_MAX_SUBBANDS;
constexpr int kMaxL = 20;  // db10

// ---------------------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------------------
wdb_status set_error(wdb_status s, const char* fmt, ...);
wdb_status cuda_error(cudaError_t e, const char* what, const char* file, int line);

#define WDB_CK(call)                                                              \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) return ::wdb::cuda_error(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define WDB_TRY(call)                                \
    do {                                             \
        wdb_status s_ = (call);                      \
        if (s_ != WDB_OK) return s_;                 \
    } while (0)

// Count of kernels launched by the library (graph replays add their node counts).
void count_launch(long long n = 1);

// Per-device one-time set-up flags (cudaFuncSetAttribute acts on the current device only):
// bit d of *mask is set once the set-up has been done on device d (devices >= 64 always redo
// it, which is harmless).
bool done_on_device(const unsigned long long* mask);
void mark_on_device(unsigned long long* mask);

// ---------------------------------------------------------------------------------------
// Subband layout (Sec. 2): subband-planar, A_J first, then (0,1),(1,0),(1,1) for s=J..1
// ---------------------------------------------------------------------------------------
struct alignas(16) SubbandDev {   // per subband, device-resident copy (16-byte aligned: vector loads)
    long long off;       // start in the coefficient vector
    int rows, cols;
    int level;           // s (1 = finest)
    int lgR;             // log2 of the phase period R = 2^{J - s}
    int tab_off;         // start of this subband in the phase tables (4^J entries in all)
    int pad;
};

struct Layout {
    int n_rows = 0, n_cols = 0, J = 0, S = 0;
    long long N = 0;
    SubbandDev sb[kMaxS];
    int tab_len = 0;     // sum_b R_b^2 = 4^J
};
wdb_status make_layout(int n_rows, int n_cols, int J, Layout* out);

// ---------------------------------------------------------------------------------------
// Device reduction / solver state
// ---------------------------------------------------------------------------------------
struct SolveState {
    int k;                  // 1-based iteration about to run / running
    int stop;               // 1: done (converged, max_iters, or error)
    int max_iters;
    int check_every;
    double tol;
    unsigned int done[4];   // last-CTA counters
    double rr, x0r;         // from the residual kernel of the current iteration
    double wy, gmax;        // from the step kernel of the current iteration
    double primal, dual, gap, rel_gap;  // certificate of the last check
    int gap_k;              // iteration of the last check
    int iters_done;         // k of the last computed x
    int nan_flag;
    int diverged;           // primal(y^(k)) > 1e6 primal(y^(1)): the iteration is not converging
    double first_primal;
    double target;          // > 0: stop once primal(y^(k)) <= target
    int hit_k;              // first k with primal <= target
    int ista;               // 1: no momentum step (y^(k+1) = x^(k)): ISTA
    double scratch[8];      // free slots for one-off reductions
    unsigned int bar_count, bar_gen;   // grid barrier of the fused loop (arrivals, generation)
    int timeout;            // 1: a bounded wait of the fused loop gave up
};

}  // namespace wdb
