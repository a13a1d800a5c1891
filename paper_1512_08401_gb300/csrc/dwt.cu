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
#include <algorithm>
#include <cstdint>

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

// ---------------------------------------------------------------------------------------
// FP32 levels for the filter lengths of the workloads (L = 8: db4, L = 12: sym6, and every
// other even length up to 20), the filter taps compile-time constants of the unrolled loops:
// 32 x 32 outputs per subband and CTA (input halo 1.2x instead of 1.4x), input rows read
// as 8-byte column pairs split by column parity in shared memory, so that every pass reads
// consecutive words across the lanes; each thread forms two outputs from one set of loads.
// ---------------------------------------------------------------------------------------
constexpr int kFT = 32;   // outputs per tile side (per subband)

template <int L>
__global__ void __launch_bounds__(256) dwt_level_fast(const float* __restrict__ in, int R, int C,
                                                      float* __restrict__ outA, float* __restrict__ d01,
                                                      float* __restrict__ d10, float* __restrict__ d11,
                                                      FiltT<float> f) {
    // a programmatic dependent of the previous level: nothing it wrote is read before that
    // grid has completed (a no-op for ordinary launches)
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    constexpr int IY = 2 * kFT + L - 2;       // input rows of the tile (with halo)
    constexpr int PX = kFT + L / 2 - 1;       // column pairs of the tile (with halo)
    __shared__ float s_ev[IY][PX + 1], s_od[IY][PX + 1];   // even / odd input columns
    __shared__ float s_lo[IY][kFT], s_hi[IY][kFT];
    const int oy0 = blockIdx.y * kFT, ox0 = blockIdx.x * kFT;
    const int R2 = R >> 1, C2 = C >> 1;
    // load: one column pair per thread and step over the flattened (row, pair) range,
    // consecutive pairs of a row on consecutive lanes (C even: a pair never wraps); fully
    // unrolled over the thread's steps, so that all its loads are in flight together
#pragma unroll
    for (int k = 0; k < (IY * PX + 255) / 256; ++k) {
        const int q = threadIdx.x + 256 * k;
        if (q >= IY * PX) break;
        const int iy = q / PX, c = q - iy * PX;
        int gy = 2 * oy0 + iy;
        while (gy >= R) gy -= R;
        int gx = 2 * (ox0 + c);
        while (gx >= C) gx -= C;
        const float2 v = __ldg(reinterpret_cast<const float2*>(in + (size_t)gy * C + gx));
        s_ev[iy][c] = v.x;
        s_od[iy][c] = v.y;
    }
    __syncthreads();
    // along x: lo/hi[iy][j] = sum_k h/g[k] in[iy][2j + k]
    for (int t = threadIdx.x; t < IY * kFT; t += 256) {
        const int iy = t >> 5, j = t & 31;
        float lo = 0.f, hi = 0.f;
#pragma unroll
        for (int m = 0; m < L / 2; ++m) {
            const float e = s_ev[iy][j + m], o = s_od[iy][j + m];
            lo = fmaf(f.h[2 * m], e, lo);
            lo = fmaf(f.h[2 * m + 1], o, lo);
            hi = fmaf(f.g[2 * m], e, hi);
            hi = fmaf(f.g[2 * m + 1], o, hi);
        }
        s_lo[iy][j] = lo;
        s_hi[iy][j] = hi;
    }
    __syncthreads();
    // along y: output row i from rows 2i .. 2i + L - 1
    for (int t = threadIdx.x; t < kFT * kFT; t += 256) {
        const int i = t >> 5, j = t & 31;
        const int oy = oy0 + i, ox = ox0 + j;
        float ll = 0.f, lh = 0.f, hl = 0.f, hh = 0.f;
#pragma unroll
        for (int k = 0; k < L; ++k) {
            const float lo = s_lo[2 * i + k][j], hi = s_hi[2 * i + k][j];
            ll = fmaf(f.h[k], lo, ll);
            hl = fmaf(f.g[k], lo, hl);
            lh = fmaf(f.h[k], hi, lh);
            hh = fmaf(f.g[k], hi, hh);
        }
        if (oy < R2 && ox < C2) {
            const size_t o = (size_t)oy * C2 + ox;
            outA[o] = ll;
            d01[o] = lh;
            d10[o] = hl;
            d11[o] = hh;
        }
    }
}

template <int L>
__global__ void __launch_bounds__(256) idwt_level_fast(const float* __restrict__ cA, const float* __restrict__ c01,
                                                       const float* __restrict__ c10, const float* __restrict__ c11,
                                                       int R2, int C2, float* __restrict__ out, FiltT<float> f) {
    // a programmatic dependent of the previous level: nothing it wrote is read before that
    // grid has completed (a no-op for ordinary launches)
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    constexpr int H2 = L / 2;
    constexpr int CY = kFT + H2 - 1, CX = kFT + H2 - 1;   // coefficient rows / cols with halo
    __shared__ float sLL[CY][CX], sLH[CY][CX], sHL[CY][CX], sHH[CY][CX];
    __shared__ float sLx[2 * kFT][CX], sHx[2 * kFT][CX];
    const int cy0 = blockIdx.y * kFT, cx0 = blockIdx.x * kFT;
    // load: flattened (row, column) range, fully unrolled over the thread's steps
#pragma unroll
    for (int k = 0; k < (CY * CX + 255) / 256; ++k) {
        const int q = threadIdx.x + 256 * k;
        if (q >= CY * CX) break;
        const int iy = q / CX, ix = q - iy * CX;
        int gy = cy0 - H2 + 1 + iy;
        while (gy < 0) gy += R2;
        while (gy >= R2) gy -= R2;
        int gx = cx0 - H2 + 1 + ix;
        while (gx < 0) gx += C2;
        while (gx >= C2) gx -= C2;
        const size_t o = (size_t)gy * C2 + gx;
        sLL[iy][ix] = __ldg(cA + o);
        sLH[iy][ix] = __ldg(c01 + o);
        sHL[iy][ix] = __ldg(c10 + o);
        sHH[iy][ix] = __ldg(c11 + o);
    }
    __syncthreads();
    // along y: rows 2i and 2i + 1 from coefficient rows i - m, m < L/2:
    //   Lx[2i + p] = sum_m h[2m + p] LL[i - m] + g[2m + p] HL[i - m]   (Hx from LH, HH)
    for (int t = threadIdx.x; t < kFT * CX; t += 256) {
        const int i = t / CX, cx = t - i * CX;
        float l0 = 0.f, l1 = 0.f, h0 = 0.f, h1 = 0.f;
#pragma unroll
        for (int m = 0; m < H2; ++m) {
            const int ci = i - m + H2 - 1;
            const float ll = sLL[ci][cx], hl = sHL[ci][cx], lh = sLH[ci][cx], hh = sHH[ci][cx];
            l0 = fmaf(f.h[2 * m], ll, fmaf(f.g[2 * m], hl, l0));
            l1 = fmaf(f.h[2 * m + 1], ll, fmaf(f.g[2 * m + 1], hl, l1));
            h0 = fmaf(f.h[2 * m], lh, fmaf(f.g[2 * m], hh, h0));
            h1 = fmaf(f.h[2 * m + 1], lh, fmaf(f.g[2 * m + 1], hh, h1));
        }
        sLx[2 * i][cx] = l0;
        sLx[2 * i + 1][cx] = l1;
        sHx[2 * i][cx] = h0;
        sHx[2 * i + 1][cx] = h1;
    }
    __syncthreads();
    // along x: columns 2c and 2c + 1 from the same coefficient columns, one 8-byte store
    const int R = 2 * R2, C = 2 * C2;
    for (int t = threadIdx.x; t < 2 * kFT * kFT; t += 256) {
        const int yl = t >> 5, c = t & 31;
        const int y = 2 * cy0 + yl, xc = cx0 + c;
        float o0 = 0.f, o1 = 0.f;
#pragma unroll
        for (int m = 0; m < H2; ++m) {
            const float lx = sLx[yl][c - m + H2 - 1], hx = sHx[yl][c - m + H2 - 1];
            o0 = fmaf(f.h[2 * m], lx, fmaf(f.g[2 * m], hx, o0));
            o1 = fmaf(f.h[2 * m + 1], lx, fmaf(f.g[2 * m + 1], hx, o1));
        }
        if (y < R && xc < C2) *reinterpret_cast<float2*>(out + (size_t)y * C + 2 * xc) = make_float2(o0, o1);
    }
}

// Persistent, double-buffered form of dwt_level_fast for 16-byte aligned inputs whose width
// is a multiple of 4: each CTA walks tiles tile += gridDim.x and, while it filters one tile,
// cp.async brings the next tile's raw input rows (16-byte chunks; a row segment starts at a
// multiple of 64 columns, chunks past the right edge wrap to column 0) into the other buffer.
// The x pass reads the raw rows as column pairs (float2), the y pass is dwt_level_fast's.
template <int L>
struct PipeGeom {
    static constexpr int IY = 2 * kFT + L - 2;        // input rows of a tile
    static constexpr int NCH = (2 * kFT + L - 2 + 3) / 4;   // 16-byte chunks per row
    static constexpr int RP = 4 * NCH;                // row pitch (floats)
    static constexpr size_t smem = sizeof(float) * (size_t)(2 * IY * RP + 2 * IY * kFT);
};

// Launch as a programmatic dependent of the previous kernel in the stream, so that the next
// level's launch overlaps the tail of the previous one (the kernels wait for it first).
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kern)(KArgs...), dim3 grid, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, args...);   // errors surface through cudaGetLastError
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}

template <int L>
__global__ void __launch_bounds__(256) dwt_level_pipe(const float* __restrict__ in, int R, int C,
                                                      float* __restrict__ outA, float* __restrict__ d01,
                                                      float* __restrict__ d10, float* __restrict__ d11,
                                                      FiltT<float> f) {
    // a programmatic dependent of the previous level: nothing it wrote is read before that
    // grid has completed (a no-op for ordinary launches)
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    using G = PipeGeom<L>;
    extern __shared__ __align__(16) float pipe_smem[];
    float* const raw0 = pipe_smem;
    float* const raw1 = raw0 + G::IY * G::RP;
    float (*s_lo)[kFT] = reinterpret_cast<float (*)[kFT]>(raw1 + G::IY * G::RP);
    float (*s_hi)[kFT] = s_lo + G::IY;
    const int R2 = R >> 1, C2 = C >> 1;
    const int ntx = (C2 + kFT - 1) / kFT, nty = (R2 + kFT - 1) / kFT, nt = ntx * nty;
    auto stage = [&](int tile, float* buf) {
        const int oy0 = (tile / ntx) * kFT, ox0 = (tile % ntx) * kFT;
        for (int q = threadIdx.x; q < G::IY * G::NCH; q += 256) {
            const int iy = q / G::NCH, k = q - iy * G::NCH;
            int gy = 2 * oy0 + iy;
            while (gy >= R) gy -= R;
            int col = 2 * ox0 + 4 * k;
            while (col >= C) col -= C;
            cp_async16(buf + iy * G::RP + 4 * k, in + (size_t)gy * C + col);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    int tile = blockIdx.x;
    if (tile < nt) stage(tile, raw0);
    float* cur = raw0;
    float* nxt = raw1;
    for (; tile < nt; tile += gridDim.x) {
        const int next = tile + gridDim.x;
        if (next < nt) stage(next, nxt);
        else asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncthreads();
        // along x from the raw rows: column pair j + m of the tile is float2 (2(j + m), +1)
        const float2* rows2 = reinterpret_cast<const float2*>(cur);
        for (int t = threadIdx.x; t < G::IY * kFT; t += 256) {
            const int iy = t >> 5, j = t & 31;
            float lo = 0.f, hi = 0.f;
#pragma unroll
            for (int m = 0; m < L / 2; ++m) {
                const float2 v = rows2[iy * (G::RP / 2) + j + m];
                lo = fmaf(f.h[2 * m], v.x, lo);
                lo = fmaf(f.h[2 * m + 1], v.y, lo);
                hi = fmaf(f.g[2 * m], v.x, hi);
                hi = fmaf(f.g[2 * m + 1], v.y, hi);
            }
            s_lo[iy][j] = lo;
            s_hi[iy][j] = hi;
        }
        __syncthreads();
        const int oy0 = (tile / ntx) * kFT, ox0 = (tile % ntx) * kFT;
        for (int t = threadIdx.x; t < kFT * kFT; t += 256) {
            const int i = t >> 5, j = t & 31;
            const int oy = oy0 + i, ox = ox0 + j;
            float ll = 0.f, lh = 0.f, hl = 0.f, hh = 0.f;
#pragma unroll
            for (int k = 0; k < L; ++k) {
                const float lo = s_lo[2 * i + k][j], hi = s_hi[2 * i + k][j];
                ll = fmaf(f.h[k], lo, ll);
                hl = fmaf(f.g[k], lo, hl);
                lh = fmaf(f.h[k], hi, lh);
                hh = fmaf(f.g[k], hi, hh);
            }
            if (oy < R2 && ox < C2) {
                const size_t o = (size_t)oy * C2 + ox;
                outA[o] = ll;
                d01[o] = lh;
                d10[o] = hl;
                d11[o] = hh;
            }
        }
        // the next iteration writes s_lo / s_hi and stages into this iteration's buffer only
        // after its wait and barrier
        float* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Persistent, double-buffered form of idwt_level_fast for 16-byte aligned coefficient arrays
// whose width is a multiple of 4. A tile needs coefficient columns cx0 - (L/2 - 1) ... cx0 + 31;
// the staged segment starts HP >= L/2 - 1 columns before cx0 (HP a multiple of 4) so that
// every 16-byte chunk is aligned, and wraps periodically in whole chunks.
template <int L>
struct IPipeGeom {
    static constexpr int H2 = L / 2;
    static constexpr int CY = kFT + H2 - 1;            // coefficient rows of a tile
    static constexpr int CX = kFT + H2 - 1;            // coefficient columns used
    static constexpr int HP = (H2 - 1 + 3) / 4 * 4;    // staged columns left of the tile
    static constexpr int OFF = HP - (H2 - 1);          // first used column within a staged row
    static constexpr int NCH = (HP + kFT) / 4;         // 16-byte chunks per staged row
    static constexpr int RP = 4 * NCH;                 // row pitch (floats)
    static constexpr int BUF = 4 * CY * RP;            // one buffer: four subbands
    static constexpr size_t smem = sizeof(float) * (size_t)(2 * BUF + 2 * 2 * kFT * CX);
};

template <int L>
__global__ void __launch_bounds__(256) idwt_level_pipe(const float* __restrict__ cA, const float* __restrict__ c01,
                                                       const float* __restrict__ c10, const float* __restrict__ c11,
                                                       int R2, int C2, float* __restrict__ out, FiltT<float> f) {
    // a programmatic dependent of the previous level: nothing it wrote is read before that
    // grid has completed (a no-op for ordinary launches)
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    using G = IPipeGeom<L>;
    constexpr int H2 = G::H2, CX = G::CX;
    extern __shared__ __align__(16) float ipipe_smem[];
    float* const buf0 = ipipe_smem;
    float* const buf1 = buf0 + G::BUF;
    float (*sLx)[CX] = reinterpret_cast<float (*)[CX]>(buf1 + G::BUF);
    float (*sHx)[CX] = sLx + 2 * kFT;
    const int ntx = (C2 + kFT - 1) / kFT, nty = (R2 + kFT - 1) / kFT, nt = ntx * nty;
    // subband s of a buffer: rows of RP floats, s = 0..3 for cA, c01, c10, c11
    auto stage = [&](int tile, float* buf) {
        const int cy0 = (tile / ntx) * kFT, cx0 = (tile % ntx) * kFT;
        for (int q = threadIdx.x; q < 4 * G::CY * G::NCH; q += 256) {
            const int sb = q / (G::CY * G::NCH);
            const int r = q - sb * (G::CY * G::NCH);
            const int iy = r / G::NCH, k = r - iy * G::NCH;
            int gy = cy0 - H2 + 1 + iy;
            while (gy < 0) gy += R2;
            while (gy >= R2) gy -= R2;
            int col = cx0 - G::HP + 4 * k;
            while (col < 0) col += C2;
            while (col >= C2) col -= C2;
            const float* src = sb == 0 ? cA : sb == 1 ? c01 : sb == 2 ? c10 : c11;
            cp_async16(buf + (sb * G::CY + iy) * G::RP + 4 * k, src + (size_t)gy * C2 + col);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    const int R = 2 * R2, C = 2 * C2;
    int tile = blockIdx.x;
    if (tile < nt) stage(tile, buf0);
    float* cur = buf0;
    float* nxt = buf1;
    for (; tile < nt; tile += gridDim.x) {
        const int next = tile + gridDim.x;
        if (next < nt) stage(next, nxt);
        else asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncthreads();
        const float* sLL = cur;
        const float* sLH = cur + G::CY * G::RP;
        const float* sHL = cur + 2 * G::CY * G::RP;
        const float* sHH = cur + 3 * G::CY * G::RP;
        // along y, as in idwt_level_fast
        for (int t = threadIdx.x; t < kFT * CX; t += 256) {
            const int i = t / CX, cx = t - i * CX;
            float l0 = 0.f, l1 = 0.f, h0 = 0.f, h1 = 0.f;
#pragma unroll
            for (int m = 0; m < H2; ++m) {
                const int o = (i - m + H2 - 1) * G::RP + cx + G::OFF;
                const float ll = sLL[o], hl = sHL[o], lh = sLH[o], hh = sHH[o];
                l0 = fmaf(f.h[2 * m], ll, fmaf(f.g[2 * m], hl, l0));
                l1 = fmaf(f.h[2 * m + 1], ll, fmaf(f.g[2 * m + 1], hl, l1));
                h0 = fmaf(f.h[2 * m], lh, fmaf(f.g[2 * m], hh, h0));
                h1 = fmaf(f.h[2 * m + 1], lh, fmaf(f.g[2 * m + 1], hh, h1));
            }
            sLx[2 * i][cx] = l0;
            sLx[2 * i + 1][cx] = l1;
            sHx[2 * i][cx] = h0;
            sHx[2 * i + 1][cx] = h1;
        }
        __syncthreads();
        const int cy0 = (tile / ntx) * kFT, cx0 = (tile % ntx) * kFT;
        for (int t = threadIdx.x; t < 2 * kFT * kFT; t += 256) {
            const int yl = t >> 5, c = t & 31;
            const int y = 2 * cy0 + yl, xc = cx0 + c;
            float o0 = 0.f, o1 = 0.f;
#pragma unroll
            for (int m = 0; m < H2; ++m) {
                const float lx = sLx[yl][c - m + H2 - 1], hx = sHx[yl][c - m + H2 - 1];
                o0 = fmaf(f.h[2 * m], lx, fmaf(f.g[2 * m], hx, o0));
                o1 = fmaf(f.h[2 * m + 1], lx, fmaf(f.g[2 * m + 1], hx, o1));
            }
            if (y < R && xc < C2) *reinterpret_cast<float2*>(out + (size_t)y * C + 2 * xc) = make_float2(o0, o1);
        }
        // sLx / sHx are rewritten, and this buffer restaged, only after the next wait and barrier
        float* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// One tile per CTA, staged like idwt_level_pipe (16-byte cp.async chunks from 4 or 8 columns
// left of the tile) into a single buffer: for levels with many tiles, where more resident
// CTAs (38 KB of shared memory for db4) hide the staging better than a persistent pipeline.
template <int L>
__global__ void __launch_bounds__(256) idwt_level_async(const float* __restrict__ cA, const float* __restrict__ c01,
                                                        const float* __restrict__ c10, const float* __restrict__ c11,
                                                        int R2, int C2, float* __restrict__ out, FiltT<float> f) {
    // a programmatic dependent of the previous level: nothing it wrote is read before that
    // grid has completed (a no-op for ordinary launches)
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    using G = IPipeGeom<L>;
    constexpr int H2 = G::H2, CX = G::CX;
    extern __shared__ __align__(16) float iasync_smem[];
    float* const buf = iasync_smem;
    float (*sLx)[CX] = reinterpret_cast<float (*)[CX]>(buf + G::BUF);
    float (*sHx)[CX] = sLx + 2 * kFT;
    const int cy0 = blockIdx.y * kFT, cx0 = blockIdx.x * kFT;
    for (int q = threadIdx.x; q < 4 * G::CY * G::NCH; q += 256) {
        const int sb = q / (G::CY * G::NCH);
        const int r = q - sb * (G::CY * G::NCH);
        const int iy = r / G::NCH, k = r - iy * G::NCH;
        int gy = cy0 - H2 + 1 + iy;
        while (gy < 0) gy += R2;
        while (gy >= R2) gy -= R2;
        int col = cx0 - G::HP + 4 * k;
        while (col < 0) col += C2;
        while (col >= C2) col -= C2;
        const float* src = sb == 0 ? cA : sb == 1 ? c01 : sb == 2 ? c10 : c11;
        cp_async16(buf + (sb * G::CY + iy) * G::RP + 4 * k, src + (size_t)gy * C2 + col);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    const float* sLL = buf;
    const float* sLH = buf + G::CY * G::RP;
    const float* sHL = buf + 2 * G::CY * G::RP;
    const float* sHH = buf + 3 * G::CY * G::RP;
    for (int t = threadIdx.x; t < kFT * CX; t += 256) {
        const int i = t / CX, cx = t - i * CX;
        float l0 = 0.f, l1 = 0.f, h0 = 0.f, h1 = 0.f;
#pragma unroll
        for (int m = 0; m < H2; ++m) {
            const int o = (i - m + H2 - 1) * G::RP + cx + G::OFF;
            const float ll = sLL[o], hl = sHL[o], lh = sLH[o], hh = sHH[o];
            l0 = fmaf(f.h[2 * m], ll, fmaf(f.g[2 * m], hl, l0));
            l1 = fmaf(f.h[2 * m + 1], ll, fmaf(f.g[2 * m + 1], hl, l1));
            h0 = fmaf(f.h[2 * m], lh, fmaf(f.g[2 * m], hh, h0));
            h1 = fmaf(f.h[2 * m + 1], lh, fmaf(f.g[2 * m + 1], hh, h1));
        }
        sLx[2 * i][cx] = l0;
        sLx[2 * i + 1][cx] = l1;
        sHx[2 * i][cx] = h0;
        sHx[2 * i + 1][cx] = h1;
    }
    __syncthreads();
    const int R = 2 * R2, C = 2 * C2;
    for (int t = threadIdx.x; t < 2 * kFT * kFT; t += 256) {
        const int yl = t >> 5, c = t & 31;
        const int y = 2 * cy0 + yl, xc = cx0 + c;
        float o0 = 0.f, o1 = 0.f;
#pragma unroll
        for (int m = 0; m < H2; ++m) {
            const float lx = sLx[yl][c - m + H2 - 1], hx = sHx[yl][c - m + H2 - 1];
            o0 = fmaf(f.h[2 * m], lx, fmaf(f.g[2 * m], hx, o0));
            o1 = fmaf(f.h[2 * m + 1], lx, fmaf(f.g[2 * m + 1], hx, o1));
        }
        if (y < R && xc < C2) *reinterpret_cast<float2*>(out + (size_t)y * C + 2 * xc) = make_float2(o0, o1);
    }
}

template <int L>
void dwt_fast_launch(const float* src, int R, int C, float* a, float* d01, float* d10, float* d11,
                     const FiltT<float>& f, cudaStream_t st) {
    const int tiles = ((C / 2 + kFT - 1) / kFT) * ((R / 2 + kFT - 1) / kFT);
    if ((C & 3) == 0 && C >= 8 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        static unsigned long long attr = 0ull;
        static int grid_per_sm = 0;
        if (!done_on_device(&attr)) {
            cudaFuncSetAttribute(dwt_level_pipe<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)PipeGeom<L>::smem);
            int per = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, dwt_level_pipe<L>, 256, PipeGeom<L>::smem);
            grid_per_sm = per > 0 ? per : 1;
            mark_on_device(&attr);
        }
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int grid = std::max(1, std::min(tiles, std::max(sms, 1) * grid_per_sm));
        launch_pdl(dwt_level_pipe<L>, dim3(grid), PipeGeom<L>::smem, st, src, R, C, a, d01, d10, d11, f);
        return;
    }
    dim3 grid((C / 2 + kFT - 1) / kFT, (R / 2 + kFT - 1) / kFT);
    launch_pdl(dwt_level_fast<L>, grid, 0, st, src, R, C, a, d01, d10, d11, f);
}

template <int L>
void idwt_fast_launch(const float* a, const float* d01, const float* d10, const float* d11, int R2, int C2,
                      float* out, const FiltT<float>& f, cudaStream_t st) {
    // The persistent form wins while each CTA has a few tiles (4096^2 level 2: 2.2 per CTA,
    // 16.3 against 17.1 us; the coarse levels) and loses with many (level 1: 9 per CTA, 52.9
    // against 44.7 us): its three resident CTAs per SM keep fewer loads in flight than the
    // one-tile CTAs of idwt_level_fast.
    const auto aligned = [](const float* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    if ((C2 & 3) == 0 && aligned(a) && aligned(d01) && aligned(d10) && aligned(d11) && aligned(out)) {
        static unsigned long long attr = 0ull;
        static int grid_per_sm = 0;
        if (!done_on_device(&attr)) {
            cudaFuncSetAttribute(idwt_level_pipe<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)IPipeGeom<L>::smem);
            int per = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, idwt_level_pipe<L>, 256, IPipeGeom<L>::smem);
            grid_per_sm = per > 0 ? per : 1;
            mark_on_device(&attr);
        }
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int tiles = ((C2 + kFT - 1) / kFT) * ((R2 + kFT - 1) / kFT);
        const int resident = std::max(sms, 1) * grid_per_sm;
        if (tiles <= 3 * resident) {
            const int grid = std::max(1, std::min(tiles, resident));
            launch_pdl(idwt_level_pipe<L>, dim3(grid), IPipeGeom<L>::smem, st, a, d01, d10, d11, R2, C2, out, f);
            return;
        }
        constexpr size_t smem1 = sizeof(float) * (size_t)(IPipeGeom<L>::BUF + 2 * 2 * kFT * IPipeGeom<L>::CX);
        static unsigned long long attr1 = 0ull;
        if (!done_on_device(&attr1)) {
            cudaFuncSetAttribute(idwt_level_async<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
            mark_on_device(&attr1);
        }
        dim3 grid1((C2 + kFT - 1) / kFT, (R2 + kFT - 1) / kFT);
        launch_pdl(idwt_level_async<L>, grid1, smem1, st, a, d01, d10, d11, R2, C2, out, f);
        return;
    }
    dim3 grid((C2 + kFT - 1) / kFT, (R2 + kFT - 1) / kFT);
    launch_pdl(idwt_level_fast<L>, grid, 0, st, a, d01, d10, d11, R2, C2, out, f);
}

// FP32 level through the fast kernels (true) or not available for this filter length (false)
bool dwt_level_f32(const float* src, int R, int C, float* a, float* d01, float* d10, float* d11,
                   const FiltT<float>& f, cudaStream_t st) {
    // the fast kernels read the input in column pairs (8-byte loads); an input that is only
    // 4-byte aligned (a caller's view at an odd offset) takes the generic kernel
    if (reinterpret_cast<uintptr_t>(src) & 7) return false;
    switch (f.L) {
        case 2: dwt_fast_launch<2>(src, R, C, a, d01, d10, d11, f, st); return true;
        case 4: dwt_fast_launch<4>(src, R, C, a, d01, d10, d11, f, st); return true;
        case 6: dwt_fast_launch<6>(src, R, C, a, d01, d10, d11, f, st); return true;
        case 8: dwt_fast_launch<8>(src, R, C, a, d01, d10, d11, f, st); return true;
        case 10: dwt_fast_launch<10>(src, R, C, a, d01, d10, d11, f, st); return true;
        case 12: dwt_fast_launch<12>(src, R, C, a, d01, d10, d11, f, st); return true;
        default: return false;
    }
}

bool idwt_level_f32(const float* a, const float* d01, const float* d10, const float* d11, int R2, int C2,
                    float* out, const FiltT<float>& f, cudaStream_t st) {
    // the fast kernels store pixel pairs (8 bytes); an output that is only 4-byte aligned
    // takes the generic kernel
    if (reinterpret_cast<uintptr_t>(out) & 7) return false;
    switch (f.L) {
        case 2: idwt_fast_launch<2>(a, d01, d10, d11, R2, C2, out, f, st); return true;
        case 4: idwt_fast_launch<4>(a, d01, d10, d11, R2, C2, out, f, st); return true;
        case 6: idwt_fast_launch<6>(a, d01, d10, d11, R2, C2, out, f, st); return true;
        case 8: idwt_fast_launch<8>(a, d01, d10, d11, R2, C2, out, f, st); return true;
        case 10: idwt_fast_launch<10>(a, d01, d10, d11, R2, C2, out, f, st); return true;
        case 12: idwt_fast_launch<12>(a, d01, d10, d11, R2, C2, out, f, st); return true;
        default: return false;
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
        bool fast = false;
        if constexpr (sizeof(T) == 4)
            fast = dwt_level_f32(src, R, C, dst, coef + Ly.sb[base].off, coef + Ly.sb[base + 1].off,
                                 coef + Ly.sb[base + 2].off, ft, st);
        if (!fast) {
            dim3 grid((C2 + kTile - 1) / kTile, (R2 + kTile - 1) / kTile);
            dwt_level_kernel<T><<<grid, 256, dwt_smem<T>(f.L), st>>>(
                src, R, C, dst, coef + Ly.sb[base].off, coef + Ly.sb[base + 1].off, coef + Ly.sb[base + 2].off, ft);
        }
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
        bool fast = false;
        if constexpr (sizeof(T) == 4)
            fast = idwt_level_f32(src, coef + Ly.sb[base].off, coef + Ly.sb[base + 1].off, coef + Ly.sb[base + 2].off,
                                  R2, C2, dst, ft, st);
        if (!fast) {
            dim3 grid((C2 + kTile - 1) / kTile, (R2 + kTile - 1) / kTile);
            idwt_level_kernel<T><<<grid, 256, idwt_smem<T>(f.L), st>>>(
                src, coef + Ly.sb[base].off, coef + Ly.sb[base + 1].off, coef + Ly.sb[base + 2].off, R2, C2, dst, ft);
        }
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
