// Launch interface of the subband-walking elementwise kernels (subband_ops.cu).
#pragma once
#include "wdb_internal.h"

namespace wdb {

struct SubbandArgs {
    const SubbandDev* sb;    // device, S entries
    const int* vb_start;     // device, S+1 entries
    int S;
    int nvb;
};

struct RedTarget {
    unsigned int* counter;   // zero on entry, reset to zero by the last CTA
    double* part;            // grid x (values) scratch
    double* out;             // totals written here by the last CTA
};

int subband_grid_limit();

template <typename T>
wdb_status launch_scale(const SubbandArgs& A, int grid, const T* in, T* out, const double* scale, cudaStream_t st);
wdb_status launch_fft_step(const SubbandArgs& A, int grid, const float* g, float* y, float* x,
                           const float* step_tab, const float* w_sb, double* part, SolveState* s,
                           cudaStream_t st);
wdb_status launch_l1_terms(const SubbandArgs& A, int grid, const float* x, const float* w_sb, RedTarget red,
                           cudaStream_t st);
template <typename T>
wdb_status launch_norm2(const T* v, long long n, RedTarget red, int grid, cudaStream_t st);
template <typename T>
wdb_status launch_splitmix(T* v, long long n, unsigned long long seed, cudaStream_t st);
template <typename T>
wdb_status launch_scale_const(const T* in, T* out, long long n, double s, cudaStream_t st);

}  // namespace wdb
