// Periodic separable 2-D DWT / IDWT (Sec. 2), FP32 and FP64.
//
// One level of analysis maps an approximation A (R x C) to A' and the three details
// (R/2 x C/2 each):  filter along x (columns) with h and g, decimate, then along y.
//   out[i] = sum_k f[k] in[(2 i + k) mod n]   (per axis)
// Orientation (e_y, e_x): (0,1) = h along y of the x-high-pass, (1,0) = g along y of the
// x-low-pass, (1,1) = g along y of the x-high-pass. Synthesis is the exact transpose.
//
// Each CTA owns an output tile; the input tile with its (L-2)-wide periodic halo is staged
// in shared memory with coalesced loads, the x pass goes to shared memory, the y pass
// writes the four outputs (coalesced). HBM-bound: each level reads its input once and
// writes its outputs once.
#include "wdb_internal.h"

namespace wdb {

namespace {

constexpr int kTile = 16;  // outputs per tile side (per subband)

// v mod n for v within a few periods of [0, n) (tile origins plus a halo): no division
__device__ __forceinline__ int wrapi(int v, int n) {
    while (v < 0) v += n;
    while (v >= n) v -= n;
    return v;
}

template <typename T>
__global__ void __launch_bounds__(256) dwt_level_kernel(const T* __restrict__ in, int R, int C,
                                                        T* __restrict__ outA, T* __restrict__ d01,
                                                        T* __restrict__ d10, T* __restrict__ d11,
                                                        FiltT<T> f) {
    extern __shared__ unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    __shared__ T sh[kMaxL], sg[kMaxL];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < kMaxL; ++k) {
            sh[k] = f.h[k];
            sg[k] = f.g[k];
        }
    }
    const int L = f.L;
    const int IY = 2 * kTile + L - 2, IX = 2 * kTile + L - 2;
    T* s_in = sm;
    T* s_lo = s_in + IY * IX;
    T* s_hi = s_lo + IY * kTile;
    const int oy0 = blockIdx.y * kTile, ox0 = blockIdx.x * kTile;
    const int R2 = R >> 1, C2 = C >> 1;
    // one warp per input row, lanes along the row (coalesced), wrap per row and per lane
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        const int gx0 = wrapi(2 * ox0 + lane, C), gx1 = wrapi(2 * ox0 + lane + 32, C);
        for (int iy = warp; iy < IY; iy += nw) {
            const T* __restrict__ row = in + (size_t)wrapi(2 * oy0 + iy, R) * C;
            if (lane < IX) s_in[iy * IX + lane] = row[gx0];
            if (lane + 32 < IX) s_in[iy * IX + lane + 32] = row[gx1];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < IY * kTile; t += blockDim.x) {
        int iy = t / kTile, jx = t - iy * kTile;
        const T* row = s_in + iy * IX + 2 * jx;
        T lo = 0, hi = 0;
        for (int k = 0; k < L; ++k) {
            T v = row[k];
            lo += sh[k] * v;
            hi += sg[k] * v;
        }
        s_lo[t] = lo;
        s_hi[t] = hi;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kTile * kTile; t += blockDim.x) {
        int i = t / kTile, j = t - i * kTile;
        int oy = oy0 + i, ox = ox0 + j;
        if (oy >= R2 || ox >= C2) continue;
        T ll = 0, lh = 0, hl = 0, hh = 0;
        for (int k = 0; k < L; ++k) {
            T lo = s_lo[(2 * i + k) * kTile + j], hi = s_hi[(2 * i + k) * kTile + j];
            ll += sh[k] * lo;
            hl += sg[k] * lo;
            lh += sh[k] * hi;
            hh += sg[k] * hi;
        }
        size_t o = (size_t)oy * C2 + ox;
        outA[o] = ll;
        d01[o] = lh;
        d10[o] = hl;
        d11[o] = hh;
    }
}

// Inverse of one level: (A', d01, d10, d11), each R2 x C2, -> A (2 R2 x 2 C2).
//   A[y] = sum_{k : (y - k) even} f[k] c[(y - k)/2]   (per axis, indices mod R2)
template <typename T>
__global__ void __launch_bounds__(256) idwt_level_kernel(const T* __restrict__ cA, const T* __restrict__ c01,
                                                         const T* __restrict__ c10, const T* __restrict__ c11,
                                                         int R2, int C2, T* __restrict__ out, FiltT<T> f) {
    extern __shared__ unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    __shared__ T sh[kMaxL], sg[kMaxL];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < kMaxL; ++k) {
            sh[k] = f.h[k];
            sg[k] = f.g[k];
        }
    }
    const int L = f.L, H2 = L / 2;
    const int CY = kTile + H2 - 1, CX = kTile + H2 - 1;
    const int OY = 2 * kTile;
    T* sLL = sm;
    T* sLH = sLL + CY * CX;   // e = (0,1)
    T* sHL = sLH + CY * CX;   // e = (1,0)
    T* sHH = sHL + CY * CX;   // e = (1,1)
    T* sLx = sHH + CY * CX;   // OY x CX
    T* sHx = sLx + OY * CX;
    const int cy0 = blockIdx.y * kTile, cx0 = blockIdx.x * kTile;
    const int by = cy0 - H2 + 1, bx = cx0 - H2 + 1;
    // one warp per coefficient row, lanes along the row (CX <= 32 + H2 - 1 < 64)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    {
        const int gx0 = wrapi(bx + lane, C2), gx1 = wrapi(bx + lane + 32, C2);
        for (int iy = warp; iy < CY; iy += nw) {
            const size_t r = (size_t)wrapi(by + iy, R2) * C2;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ix = lane + 32 * h;
                if (ix >= CX) break;
                const size_t g = r + (h ? gx1 : gx0);
                const int t = iy * CX + ix;
                sLL[t] = cA[g];
                sLH[t] = c01[g];
                sHL[t] = c10[g];
                sHH[t] = c11[g];
            }
        }
    }
    __syncthreads();
    // synthesis along y: Lx from (LL, HL), Hx from (LH, HH); t / CX through a multiply-high
    // by ceil(2^32 / CX) (exact for t < 2^16)
    const unsigned mCX = 0xffffffffu / (unsigned)CX + 1u;
    for (int t = threadIdx.x; t < OY * CX; t += blockDim.x) {
        const int yl = (int)__umulhi((unsigned)t, mCX), cx = t - yl * CX;
        T lx = 0, hx = 0;
        for (int k = (yl & 1); k < L; k += 2) {
            int ci = ((yl - k) >> 1) + H2 - 1;   // (yl - k) even
            int s = ci * CX + cx;
            lx += sh[k] * sLL[s] + sg[k] * sHL[s];
            hx += sh[k] * sLH[s] + sg[k] * sHH[s];
        }
        sLx[yl * CX + cx] = lx;
        sHx[yl * CX + cx] = hx;
    }
    __syncthreads();
    const int R = 2 * R2, C = 2 * C2;
    for (int t = threadIdx.x; t < OY * 2 * kTile; t += blockDim.x) {
        int yl = t / (2 * kTile), xl = t - yl * (2 * kTile);
        int y = 2 * cy0 + yl, x = 2 * cx0 + xl;
        if (y >= R || x >= C) continue;
        T v = 0;
        for (int k = (xl & 1); k < L; k += 2) {
            int ci = ((xl - k) >> 1) + H2 - 1;
            v += sh[k] * sLx[yl * CX + ci] + sg[k] * sHx[yl * CX + ci];
        }
        out[(size_t)y * C + x] = v;
    }
}

template <typename T>
size_t dwt_smem(int L) {
    int IY = 2 * kTile + L - 2;
    return sizeof(T) * (size_t)(IY * IY + 2 * IY * kTile);
}

template <typename T>
size_t idwt_smem(int L) {
    int C = kTile + L / 2 - 1;
    return sizeof(T) * (size_t)(4 * C * C + 2 * (2 * kTile) * C);
}

template <typename T>
wdb_status ensure_smem_attr() {
    static unsigned long long done = 0ull;
    if (!done_on_device(&done)) {
        WDB_CK(cudaFuncSetAttribute(dwt_level_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)dwt_smem<T>(kMaxL)));
        WDB_CK(cudaFuncSetAttribute(idwt_level_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)idwt_smem<T>(kMaxL)));
        mark_on_device(&done);
    }
    return WDB_OK;
}

}  // namespace

// Forward: level s reads A_{s-1} (the image for s = 1) and writes A_s and the details of
// level s. Intermediate approximations alternate between the two halves of `scratch`
// (N/4 + N/16 <= N/2 elements); A_J goes to subband 0 of coef.
template <typename T>
wdb_status dwt2(const T* img, T* coef, const Layout& Ly, const Filters& f, T* scratch,
                cudaStream_t st) {
    WDB_TRY(ensure_smem_attr<T>());
    FiltT<T> ft = filt_cast<T>(f);
    const T* src = img;
    int R = Ly.n_rows, C = Ly.n_cols;
    T* bufA = scratch;
    T* bufB = scratch + (size_t)(Ly.N / 4);
    for (int s = 1; s <= Ly.J; ++s) {
        int base = 1 + 3 * (Ly.J - s);   // subband index of (0,1) at level s
        T* dst = (s == Ly.J) ? coef + Ly.sb[0].off : ((s & 1) ? bufA : bufB);
        int R2 = R / 2, C2 = C / 2;
        dim3 grid((C2 + kTile - 1) / kTile, (R2 + kTile - 1) / kTile);
        dwt_level_kernel<T><<<grid, 256, dwt_smem<T>(f.L), st>>>(
            src, R, C, dst, coef + Ly.sb[base].off, coef + Ly.sb[base + 1].off, coef + Ly.sb[base + 2].off, ft);
        count_launch();
        WDB_CK(cudaGetLastError());
        src = dst;
        R = R2;
        C = C2;
    }
    return WDB_OK;
}

template <typename T>
wdb_status idwt2(const T* coef, T* img, const Layout& Ly, const Filters& f, T* scratch,
                 cudaStream_t st) {
    WDB_TRY(ensure_smem_attr<T>());
    FiltT<T> ft = filt_cast<T>(f);
    const T* src = coef + Ly.sb[0].off;
    T* bufA = scratch;
    T* bufB = scratch + (size_t)(Ly.N / 4);
    for (int s = Ly.J; s >= 1; --s) {
        int base = 1 + 3 * (Ly.J - s);
        int R2 = Ly.n_rows >> s, C2 = Ly.n_cols >> s;
        T* dst = (s == 1) ? img : ((s & 1) ? bufA : bufB);
        dim3 grid((C2 + kTile - 1) / kTile, (R2 + kTile - 1) / kTile);
        idwt_level_kernel<T><<<grid, 256, idwt_smem<T>(f.L), st>>>(
            src, coef + Ly.sb[base].off, coef + Ly.sb[base + 1].off, coef + Ly.sb[base + 2].off, R2, C2, dst, ft);
        count_launch();
        WDB_CK(cudaGetLastError());
        src = dst;
    }
    return WDB_OK;
}

template wdb_status dwt2<float>(const float*, float*, const Layout&, const Filters&, float*, cudaStream_t);
template wdb_status dwt2<double>(const double*, double*, const Layout&, const Filters&, double*, cudaStream_t);
template wdb_status idwt2<float>(const float*, float*, const Layout&, const Filters&, float*, cudaStream_t);
template wdb_status idwt2<double>(const double*, double*, const Layout&, const Filters&, double*, cudaStream_t);

}  // namespace wdb
