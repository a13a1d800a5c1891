// Device helpers shared by the kernels of libwdb: compensated FP32 accumulation, the
// deterministic grid-wide FP64 reduction, and subband / phase-class lookups.
#pragma once
#include <cfloat>

#include "wdb_internal.h"

namespace wdb {

// Neumaier compensated summation step in FP32.
__device__ __forceinline__ void neu_add(float& s, float& c, float v) {
    float t = s + v;
    c += (fabsf(s) >= fabsf(v)) ? ((s - t) + v) : ((v - t) + s);
    s = t;
}

// Reduce NV doubles over the grid. Returns true in every thread of the last CTA to finish,
// with `tot` holding the grid totals there. Bit i of maxmask selects max instead of sum
// (values must be >= 0 for max).
template <int NV>
__device__ bool grid_reduce(double (&v)[NV], unsigned maxmask, double* part, unsigned int* counter,
                            double (&tot)[NV]) {
    __shared__ double s_w[32][NV];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        for (int off = 16; off > 0; off >>= 1) {
            double o = __shfl_down_sync(0xffffffffu, v[i], off);
            v[i] = ((maxmask >> i) & 1) ? fmax(v[i], o) : v[i] + o;
        }
        if (lane == 0) s_w[warp][i] = v[i];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double x = lane < nw ? s_w[lane][i] : 0.0;
            for (int off = 16; off > 0; off >>= 1) {
                double o = __shfl_down_sync(0xffffffffu, x, off);
                x = ((maxmask >> i) & 1) ? fmax(x, o) : x + o;
            }
            if (lane == 0) part[(size_t)blockIdx.x * NV + i] = x;
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double x = __ldcg(part + (size_t)b * NV + i);
            acc[i] = ((maxmask >> i) & 1) ? fmax(acc[i], x) : acc[i] + x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        for (int off = 16; off > 0; off >>= 1) {
            double o = __shfl_down_sync(0xffffffffu, acc[i], off);
            acc[i] = ((maxmask >> i) & 1) ? fmax(acc[i], o) : acc[i] + o;
        }
        if (lane == 0) s_w[warp][i] = acc[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double x = 0.0;
        for (int w = 0; w < nw; ++w) x = ((maxmask >> i) & 1) ? fmax(x, s_w[w][i]) : x + s_w[w][i];
        tot[i] = x;
    }
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// |g| / w, the ratio of the dual bound (infinite for g != 0 where w = 0)
__device__ __forceinline__ float gw_ratio(float g, float w) {
    const float ag = fabsf(g);
    return w > 0.f ? ag / w : (ag > 0.f ? FLT_MAX : 0.f);
}

__device__ __forceinline__ int find_subband(const int* __restrict__ vb_start, int S, int vb) {
    int o = 0;
    while (o + 1 < S && vb >= __ldg(vb_start + o + 1)) ++o;
    return o;
}

__device__ __forceinline__ int phase_class(const SubbandDev& so, int py, int px) {
    const int m = (1 << so.lgR) - 1;
    return so.tab_off + ((py & m) << so.lgR) + (px & m);
}

// ---------------------------------------------------------------------------------------
// Gap bookkeeping shared by the Theta_K and FFT paths (runs in one thread of the last CTA).
//   primal = 1/2 rr + wy; s = min(1, 1/max_i |g_i|/w_i); dual = -s x0r - s^2/2 rr
// A NaN / Inf primal or gap, or a primal above 1e6 times the first one, stops the loop.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void finish_iteration(SolveState* st, double wy, double gmax) {
    const int k = st->k;
    const double rr = st->rr, x0r = st->x0r;
    const double primal = 0.5 * rr + wy;
    const double s = gmax > 0.0 ? fmin(1.0, 1.0 / gmax) : 1.0;
    const double dual = -s * x0r - 0.5 * s * s * rr;
    const double gap = primal - dual;
    st->wy = wy;
    st->gmax = gmax;
    if (k == 1) st->first_primal = primal;
    if (!isfinite(primal) || !isfinite(gap)) {
        st->nan_flag = 1;
        st->stop = 1;
    } else if (k > 1 && primal > 1e6 * st->first_primal) {
        // a step too long for the operator makes the objective grow geometrically
        st->diverged = 1;
        st->stop = 1;
    }
    const bool check = (k % st->check_every) == 0 || k >= st->max_iters;
    if (check) {
        st->primal = primal;
        st->dual = dual;
        st->gap = gap;
        st->rel_gap = primal > 0.0 ? gap / primal : 0.0;
        st->gap_k = k;
        if (st->tol > 0.0 && (k % st->check_every) == 0 && st->rel_gap <= st->tol) st->stop = 1;
    }
    if (st->target > 0.0 && primal <= st->target) {
        if (st->hit_k == 0) st->hit_k = k;
        st->stop = 1;
    }
    st->iters_done = k;
    if (k >= st->max_iters) st->stop = 1;
    st->k = k + 1;
}

}  // namespace wdb
