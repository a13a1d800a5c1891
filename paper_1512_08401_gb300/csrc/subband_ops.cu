// Subband-walking elementwise kernels: the FFT path's fused FISTA step (Algorithm 3 with
// the diagonal Prox of Eq. defProxP, gradient given), the l1 terms of the objective, the
// per-phase-class diagonal scaling (Eq. defProxP's P) and the plain vector helpers of the
// power iteration (Section 4.2). The Theta_K kernels themselves are in tile.cu.
//
// Outputs are scheduled in virtual blocks of 256 consecutive coefficients of one subband; a
// CTA walks virtual blocks in a grid-stride loop so that the per-CTA partial sums of the
// reductions stay few.
//
// Reductions: each thread keeps a compensated (Neumaier) FP32 sum of its terms, the warp
// and CTA trees run in FP64, and the last CTA to finish sums the per-CTA partials in FP64
// in a fixed order (deterministic).
#include <cfloat>

#include "device_util.cuh"
#include "subband_ops.cuh"

namespace wdb {

namespace {

// elementwise out = in * scale[class]
template <typename T>
__global__ void __launch_bounds__(kVB) scale_kernel(SubbandArgs A, const T* __restrict__ in, T* __restrict__ out,
                                                    const double* __restrict__ scale) {
    __shared__ int s_o;
    for (int vb = blockIdx.x; vb < A.nvb; vb += gridDim.x) {
        if (threadIdx.x == 0) s_o = find_subband(A.vb_start, A.S, vb);
        __syncthreads();
        const int o = s_o;
        const SubbandDev so = A.sb[o];
        const int local = (vb - A.vb_start[o]) * kVB + threadIdx.x;
        if (local < so.rows * so.cols) {
            const int py = local / so.cols, px = local - py * so.cols;
            out[so.off + local] = (T)((double)in[so.off + local] * scale[phase_class(so, py, px)]);
        }
        __syncthreads();
    }
}

// |g| / w with the w = 0 convention of the dual norm (0/0 = 0, g/0 = FLT_MAX).
__device__ __forceinline__ float g_over_w(float g, float w) {
    const float ag = fabsf(g);
    return w > 0.f ? ag / w : (ag > 0.f ? FLT_MAX : 0.f);
}

// FFT path step, g given (the DWT of the image-domain gradient):
//   z = y - (tau/P) g ; x_new = soft(z, (tau/P) w) ; y_new = x_new + beta_k (x_new - x_old)
// in place on x and y; FP64 totals of sum w|y| and max |g|/w.
__global__ void __launch_bounds__(kVB) fft_step(SubbandArgs A, const float* __restrict__ g_in, float* __restrict__ y,
                                                float* __restrict__ x, const float* __restrict__ step_tab,
                                                const float* __restrict__ w_sb, double* part, SolveState* st) {
    if (*(volatile int*)&st->stop) return;
    __shared__ int s_o;
    const int k = st->k;
    const float beta = st->ista ? 0.f : (float)(k - 1) / (float)(k + 2);
    float ws = 0.f, wc = 0.f, gm = 0.f;
    for (int vb = blockIdx.x; vb < A.nvb; vb += gridDim.x) {
        if (threadIdx.x == 0) s_o = find_subband(A.vb_start, A.S, vb);
        __syncthreads();
        const int o = s_o;
        const SubbandDev so = A.sb[o];
        const int local = (vb - A.vb_start[o]) * kVB + threadIdx.x;
        if (local < so.rows * so.cols) {
            const int py = local / so.cols, px = local - py * so.cols;
            const size_t i = so.off + local;
            const float g = g_in[i];
            const float stp = step_tab[phase_class(so, py, px)];
            const float wv = w_sb[o];
            const float yv = y[i], xo = x[i];
            const float z = yv - stp * g;
            const float xn = copysignf(fmaxf(fabsf(z) - stp * wv, 0.f), z);
            x[i] = xn;
            y[i] = xn + beta * (xn - xo);
            neu_add(ws, wc, wv * fabsf(yv));
            gm = fmaxf(gm, g_over_w(g, wv));
        }
        __syncthreads();
    }
    double v[2] = {(double)ws + (double)wc, (double)gm}, tot[2];
    if (grid_reduce<2>(v, 2u, part, &st->done[1], tot) && threadIdx.x == 0) finish_iteration(st, tot[0], tot[1]);
}

// sum w|x| and the support size of x -> red.out[0], red.out[1]
__global__ void __launch_bounds__(kVB) l1_terms(SubbandArgs A, const float* __restrict__ x,
                                                const float* __restrict__ w_sb, RedTarget red) {
    __shared__ int s_o;
    float ws = 0.f, wc = 0.f;
    double cnt = 0.0;
    for (int vb = blockIdx.x; vb < A.nvb; vb += gridDim.x) {
        if (threadIdx.x == 0) s_o = find_subband(A.vb_start, A.S, vb);
        __syncthreads();
        const int o = s_o;
        const SubbandDev so = A.sb[o];
        const int local = (vb - A.vb_start[o]) * kVB + threadIdx.x;
        if (local < so.rows * so.cols) {
            const float xv = x[so.off + local];
            neu_add(ws, wc, w_sb[o] * fabsf(xv));
            cnt += (xv != 0.f) ? 1.0 : 0.0;
        }
        __syncthreads();
    }
    double v[2] = {(double)ws + (double)wc, cnt}, tot[2];
    if (grid_reduce<2>(v, 0u, red.part, red.counter, tot) && threadIdx.x == 0) {
        red.out[0] = tot[0];
        red.out[1] = tot[1];
    }
}

// splitmix64 (Steele, Lea & Flood 2014): output i of the stream seeded with s is
// mix(s + (i+1) * 0x9E3779B97F4A7C15); value in [-1, 1) = 2 (z >> 11) 2^-53 - 1.
template <typename T>
__global__ void splitmix_fill(T* __restrict__ v, long long n, unsigned long long seed) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z = z ^ (z >> 31);
        v[i] = (T)(2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0);
    }
}

template <typename T>
__global__ void scale_const_kernel(const T* __restrict__ in, T* __restrict__ out, long long n, double s) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (T)((double)in[i] * s);
}

template <typename T>
__global__ void __launch_bounds__(256) norm2_kernel(const T* __restrict__ v, long long n, RedTarget red) {
    double acc = 0.0;
    float ns = 0.f, nc = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (sizeof(T) == 8) acc += (double)v[i] * (double)v[i];
        else neu_add(ns, nc, (float)v[i] * (float)v[i]);
    }
    double a[1] = {acc + (double)ns + (double)nc}, tot[1];
    if (grid_reduce<1>(a, 0u, red.part, red.counter, tot) && threadIdx.x == 0) red.out[0] = tot[0];
}

int ew_grid(long long n) {
    long long g = (n + 255) / 256;
    return (int)(g > 2048 ? 2048 : (g < 1 ? 1 : g));
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------------------
template <typename T>
wdb_status launch_scale(const SubbandArgs& A, int grid, const T* in, T* out, const double* scale, cudaStream_t st) {
    scale_kernel<T><<<grid, kVB, 0, st>>>(A, in, out, scale);
    count_launch();
    WDB_CK(cudaGetLastError());
    return WDB_OK;
}

wdb_status launch_fft_step(const SubbandArgs& A, int grid, const float* g, float* y, float* x,
                           const float* step_tab, const float* w_sb, double* part, SolveState* s,
                           cudaStream_t st) {
    fft_step<<<grid, kVB, 0, st>>>(A, g, y, x, step_tab, w_sb, part, s);
    count_launch();
    WDB_CK(cudaGetLastError());
    return WDB_OK;
}

wdb_status launch_l1_terms(const SubbandArgs& A, int grid, const float* x, const float* w_sb, RedTarget red,
                           cudaStream_t st) {
    l1_terms<<<grid, kVB, 0, st>>>(A, x, w_sb, red);
    count_launch();
    WDB_CK(cudaGetLastError());
    return WDB_OK;
}

template <typename T>
wdb_status launch_norm2(const T* v, long long n, RedTarget red, int grid, cudaStream_t st) {
    int g = ew_grid(n);
    if (grid > 0 && g > grid) g = grid;   // the partials buffer holds `grid` CTAs
    norm2_kernel<T><<<g, 256, 0, st>>>(v, n, red);
    count_launch();
    WDB_CK(cudaGetLastError());
    return WDB_OK;
}

template <typename T>
wdb_status launch_splitmix(T* v, long long n, unsigned long long seed, cudaStream_t st) {
    splitmix_fill<T><<<ew_grid(n), 256, 0, st>>>(v, n, seed);
    count_launch();
    WDB_CK(cudaGetLastError());
    return WDB_OK;
}

template <typename T>
wdb_status launch_scale_const(const T* in, T* out, long long n, double s, cudaStream_t st) {
    scale_const_kernel<T><<<ew_grid(n), 256, 0, st>>>(in, out, n, s);
    count_launch();
    WDB_CK(cudaGetLastError());
    return WDB_OK;
}

template wdb_status launch_norm2<float>(const float*, long long, RedTarget, int, cudaStream_t);
template wdb_status launch_norm2<double>(const double*, long long, RedTarget, int, cudaStream_t);
template wdb_status launch_splitmix<float>(float*, long long, unsigned long long, cudaStream_t);
template wdb_status launch_splitmix<double>(double*, long long, unsigned long long, cudaStream_t);
template wdb_status launch_scale_const<float>(const float*, float*, long long, double, cudaStream_t);
template wdb_status launch_scale_const<double>(const double*, double*, long long, double, cudaStream_t);

int subband_grid_limit() {
    static int g = 0;
    if (g == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fft_step, kVB, 0);
        if (sms <= 0) sms = 1;
        if (per <= 0) per = 1;
        g = sms * per;
    }
    return g;
}

template wdb_status launch_scale<float>(const SubbandArgs&, int, const float*, float*, const double*, cudaStream_t);
template wdb_status launch_scale<double>(const SubbandArgs&, int, const double*, double*, const double*,
                                         cudaStream_t);

}  // namespace wdb
