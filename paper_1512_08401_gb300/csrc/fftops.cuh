// cuFFT helpers: the periodic convolution H (Sec. 3.6) in the Fourier domain.
#pragma once
#include <cufft.h>

#include "wdb_internal.h"

namespace wdb {

wdb_status cufft_error(cufftResult r, const char* what, const char* file, int line);
#define WDB_CKF(call)                                                                      \
    do {                                                                                   \
        cufftResult r_ = (call);                                                           \
        if (r_ != CUFFT_SUCCESS) return ::wdb::cufft_error(r_, #call, __FILE__, __LINE__); \
    } while (0)

// pad[(a - kh/2) mod R][(b - kw/2) mod C] = psf[a][b] on a zeroed R x C image (FP64).
wdb_status launch_pad_psf(const double* psf_dev, int kh, int kw, double* pad, int R, int C, cudaStream_t st);

// out[k] = in[k] * (conj ? conj(h[k]) : h[k]) * scale   (n complex values, FP64)
wdb_status launch_cmul64(const cufftDoubleComplex* in, const cufftDoubleComplex* h, cufftDoubleComplex* out,
                         long long n, int conj, double scale, cudaStream_t st);
// out[k] = in[k] * |h[k]|^2 * scale
wdb_status launch_cmul_abs2_64(const cufftDoubleComplex* in, const cufftDoubleComplex* h,
                               cufftDoubleComplex* out, long long n, double scale, cudaStream_t st);
// FP64 -> FP32 complex
wdb_status launch_c64_to_c32(const cufftDoubleComplex* in, cufftComplex* out, long long n, cudaStream_t st);
// max |h[k]|^2 over n values -> *out (device double; computed with an integer atomicMax)
wdb_status launch_max_abs2(const cufftDoubleComplex* h, long long n, double* out, cudaStream_t st);

// sum of squares of a real FP64 vector (grid reduction into red)
struct RedTarget;

}  // namespace wdb
