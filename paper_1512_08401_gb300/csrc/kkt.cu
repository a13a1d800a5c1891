// FP64 optimality check of an iterate x of min 1/2||Theta_K x - x0||^2 + sum w|x|
// (Eq. l1problemThetaApprox): r = Theta_K x - x0 and g = Theta_K^T r with FP64 taps and FP64
// accumulation (the tile engine's FP64 instances), then, reduced in FP64,
//   * the first-order (KKT) conditions of the l1 problem, whose violation the support
//     identification discussion of Sec. 4 measures: |g_i| <= w_i everywhere, and on the
//     support g_i = -w_i sign(x_i). Reported as
//       kkt_off = max_i          (|g_i| - w_i)_+ / w_i,
//       kkt_on  = max_{x_i != 0} |g_i + w_i sign(x_i)| / w_i
//     (absolute values where w_i = 0);
//   * the objective E(x) = 1/2||r||^2 + sum w|x| and the duality gap of x with the scaled
//     residual as dual point: s = min(1, 1/max_i |g_i|/w_i), D = -s<x0, r> - s^2/2 ||r||^2.
#include <cfloat>

#include "device_util.cuh"
#include "solve_impl.h"
#include "subband_ops.cuh"
#include "theta_impl.h"

namespace wdb {

namespace {

__global__ void promote_kernel(const float* __restrict__ in, double* __restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

// r <- r - x0 in place; totals ||r||^2 and <x0, r>
__global__ void __launch_bounds__(256) resid64_kernel(double* __restrict__ r, const float* __restrict__ x0, long long n,
                                                      RedTarget red) {
    double rr = 0.0, xr = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = r[i] - (double)x0[i];
        r[i] = v;
        rr += v * v;
        xr += (double)x0[i] * v;
    }
    double v[2] = {rr, xr}, tot[2];
    if (grid_reduce<2>(v, 0u, red.part, red.counter, tot) && threadIdx.x == 0) {
        red.out[0] = tot[0];
        red.out[1] = tot[1];
    }
}

// KKT residuals, max |g|/w, sum w|x| and the support size over the coefficients, subband by
// subband, with the FP64 weights of the problem
__global__ void __launch_bounds__(kVB) kkt64_kernel(SubbandArgs A, const float* __restrict__ x,
                                                    const double* __restrict__ g, const double* __restrict__ w_sb,
                                                    RedTarget red) {
    __shared__ int s_o;
    double off = 0.0, on = 0.0, gm = 0.0, wx = 0.0, cnt = 0.0;
    for (int vb = blockIdx.x; vb < A.nvb; vb += gridDim.x) {
        if (threadIdx.x == 0) s_o = find_subband(A.vb_start, A.S, vb);
        __syncthreads();
        const int o = s_o;
        const SubbandDev so = A.sb[o];
        const int local = (vb - A.vb_start[o]) * kVB + threadIdx.x;
        if (local < so.rows * so.cols) {
            const size_t i = so.off + local;
            const double gv = g[i], wv = w_sb[o];
            const float xv = x[i];
            const double ag = fabs(gv);
            const double sc = wv > 0.0 ? 1.0 / wv : 1.0;
            off = fmax(off, fmax(ag - wv, 0.0) * sc);
            if (xv != 0.f) on = fmax(on, fabs(gv + (xv > 0.f ? wv : -wv)) * sc);
            gm = fmax(gm, wv > 0.0 ? ag / wv : (ag > 0.0 ? DBL_MAX : 0.0));
            wx += wv * fabs((double)xv);
            cnt += xv != 0.f ? 1.0 : 0.0;
        }
        __syncthreads();
    }
    double v[5] = {off, on, gm, wx, cnt}, tot[5];
    if (grid_reduce<5>(v, 7u, red.part, red.counter, tot) && threadIdx.x == 0)
        for (int q = 0; q < 5; ++q) red.out[q] = tot[q];
}

int grid_for(long long n, int cap) {
    long long g = (n + 255) / 256;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

wdb_status theta_kkt64(wdb_theta* th, const float* x, const float* x0, const double* w_host, cudaStream_t st,
                       Kkt64* out) {
    const long long N = th->lay.N;
    const int S = th->lay.S;
    if (!th->d_x64) WDB_TRY(th_alloc(th, &th->d_x64, (size_t)N));
    if (!th->d_r64) WDB_TRY(th_alloc(th, &th->d_r64, (size_t)N));
    if (!th->d_kkt_out) WDB_TRY(th_alloc(th, &th->d_kkt_out, 8 + (size_t)S));
    double* d_w64 = th->d_kkt_out + 8;
    WDB_CK(cudaMemcpyAsync(d_w64, w_host, sizeof(double) * S, cudaMemcpyHostToDevice, st));
    const TileArgs F = tile_args(th, false, true), At = tile_args(th, true, true);
    double* d_out = th->d_kkt_out;
    const int grid = grid_for(N, th->grid);
    promote_kernel<<<grid, 256, 0, st>>>(x, th->d_x64, N);
    count_launch();
    WDB_CK(cudaGetLastError());
    WDB_TRY(tile_apply<double>(F, th->d_x64, th->d_r64, nullptr, nullptr, th->d_red_part, st));
    resid64_kernel<<<grid, 256, 0, st>>>(th->d_r64, x0, N, th_red(th, d_out));
    count_launch();
    WDB_CK(cudaGetLastError());
    // g = Theta_K^T r overwrites the promoted x (no longer needed)
    double* g = th->d_x64;
    WDB_TRY(tile_apply<double>(At, th->d_r64, g, nullptr, nullptr, th->d_red_part, st));
    const SubbandArgs A = subband_args(th);
    // (the per-CTA partial buffer holds 4 values for each of part_len CTAs)
    const int kgrid = std::max(1, std::min(th->grid, th->part_len * 4 / 5));
    kkt64_kernel<<<kgrid, kVB, 0, st>>>(A, x, g, d_w64, th_red(th, d_out + 2));
    count_launch();
    WDB_CK(cudaGetLastError());
    double h[7];
    WDB_CK(cudaMemcpyAsync(h, d_out, sizeof h, cudaMemcpyDeviceToHost, st));
    WDB_CK(cudaStreamSynchronize(st));
    const double rr = h[0], x0r = h[1], gmax = h[4], wx = h[5];
    out->kkt_off = h[2];
    out->kkt_on = h[3];
    out->gmax = gmax;
    out->objective = 0.5 * rr + wx;
    const double s = gmax > 0.0 ? std::fmin(1.0, 1.0 / gmax) : 1.0;
    const double dual = -s * x0r - 0.5 * s * s * rr;
    out->gap = out->objective - dual;
    out->rel_gap = out->objective > 0.0 ? out->gap / out->objective : 0.0;
    out->support = (long long)llround(h[6]);
    return WDB_OK;
}

}  // namespace wdb
