// cuFFT helper kernels (FP64 setup side of the FFT-domain convolution).
#include "fftops.cuh"

namespace wdb {

wdb_status cufft_error(cufftResult r, const char* what, const char* file, int line) {
    return set_error(r == CUFFT_ALLOC_FAILED ? WDB_ENOMEM : WDB_ECUDA, "%s failed: cufftResult %d (%s:%d)", what,
                     (int)r, file, line);
}

namespace {

__global__ void pad_psf_kernel(const double* __restrict__ psf, int kh, int kw, double* __restrict__ pad, int R,
                               int C) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= kh * kw) return;
    int a = t / kw, b = t - a * kw;
    int y = (a - kh / 2) % R;
    y += y < 0 ? R : 0;
    int x = (b - kw / 2) % C;
    x += x < 0 ? C : 0;
    pad[(size_t)y * C + x] = psf[t];
}

__global__ void cmul64_kernel(const cufftDoubleComplex* __restrict__ in, const cufftDoubleComplex* __restrict__ h,
                              cufftDoubleComplex* __restrict__ out, long long n, int conj, double scale) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        cufftDoubleComplex a = in[k], b = h[k];
        double bi = conj ? -b.y : b.y;
        out[k] = make_cuDoubleComplex((a.x * b.x - a.y * bi) * scale, (a.x * bi + a.y * b.x) * scale);
    }
}

__global__ void cmul_abs2_kernel(const cufftDoubleComplex* __restrict__ in, const cufftDoubleComplex* __restrict__ h,
                                 cufftDoubleComplex* __restrict__ out, long long n, double scale) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        cufftDoubleComplex a = in[k], b = h[k];
        double m = (b.x * b.x + b.y * b.y) * scale;
        out[k] = make_cuDoubleComplex(a.x * m, a.y * m);
    }
}

__global__ void c64_to_c32_kernel(const cufftDoubleComplex* __restrict__ in, cufftComplex* __restrict__ out,
                                  long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        out[k] = make_cuComplex((float)in[k].x, (float)in[k].y);
}

__global__ void max_abs2_kernel(const cufftDoubleComplex* __restrict__ h, long long n, unsigned long long* out) {
    double m = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        m = fmax(m, h[k].x * h[k].x + h[k].y * h[k].y);
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

int grid_for(long long n) {
    long long g = (n + 255) / 256;
    return (int)(g > 4096 ? 4096 : (g < 1 ? 1 : g));
}

}  // namespace

wdb_status launch_pad_psf(const double* psf_dev, int kh, int kw, double* pad, int R, int C, cudaStream_t st) {
    WDB_CK(cudaMemsetAsync(pad, 0, sizeof(double) * (size_t)R * C, st));
    pad_psf_kernel<<<(kh * kw + 255) / 256, 256, 0, st>>>(psf_dev, kh, kw, pad, R, C);
    count_launch();
    WDB_CK(cudaGetLastError());
    return WDB_OK;
}

wdb_status launch_cmul64(const cufftDoubleComplex* in, const cufftDoubleComplex* h, cufftDoubleComplex* out,
                         long long n, int conj, double scale, cudaStream_t st) {
    cmul64_kernel<<<grid_for(n), 256, 0, st>>>(in, h, out, n, conj, scale);
    count_launch();
    WDB_CK(cudaGetLastError());
    return WDB_OK;
}

wdb_status launch_cmul_abs2_64(const cufftDoubleComplex* in, const cufftDoubleComplex* h,
                               cufftDoubleComplex* out, long long n, double scale, cudaStream_t st) {
    cmul_abs2_kernel<<<grid_for(n), 256, 0, st>>>(in, h, out, n, scale);
    count_launch();
    WDB_CK(cudaGetLastError());
    return WDB_OK;
}

wdb_status launch_c64_to_c32(const cufftDoubleComplex* in, cufftComplex* out, long long n, cudaStream_t st) {
    c64_to_c32_kernel<<<grid_for(n), 256, 0, st>>>(in, out, n);
    count_launch();
    WDB_CK(cudaGetLastError());
    return WDB_OK;
}

wdb_status launch_max_abs2(const cufftDoubleComplex* h, long long n, double* out, cudaStream_t st) {
    WDB_CK(cudaMemsetAsync(out, 0, sizeof(double), st));
    max_abs2_kernel<<<grid_for(n), 256, 0, st>>>(h, n, reinterpret_cast<unsigned long long*>(out));
    count_launch();
    WDB_CK(cudaGetLastError());
    return WDB_OK;
}

}  // namespace wdb
