// Warm-start network (an addition to the paper's method): a small U-Net that maps a blurred
// image u to an image v whose wavelet coefficients start FISTA. Forward, backward and Adam
// run in the kernels below: BF16 activations and weights, FP32 accumulation, FP32 master
// weights, gradients and Adam moments.
//
// Network (levels L, channels C <= 32, periodic 3x3 convolutions, bias everywhere):
//   enc 0:   a = relu(conv(u)); e_0 = relu(conv(a))
//   enc l>0: p = avgpool2(e_{l-1}); a = relu(conv(p)); e_l = relu(conv(a))
//   dec l = L-2..0 (d_{L-1} = e_{L-1}): s = up2(d_{l+1}) + e_l; a = relu(conv(s)); d_l = relu(conv(a))
//   v = u + conv(d_0)
// Loss: mean of (v - target)^2. The flat parameter vector lists, per convolution, W
// ([C_out][C_in][3][3]) then b, in the order: in, e0, e1a, e1b, ..., d(L-2)a, d(L-2)b, ...,
// d0a, d0b, out.
//
// Convolution kernel: one CTA per 16 x 16 output tile of one image; the input tile with its
// one-pixel periodic halo and the CTA's weights are staged in shared memory; every thread
// accumulates all output channels of one pixel. The data gradient is a convolution of the
// output gradient with flipped, transposed weights: on the tensor cores (the gradient rounded
// to BF16) wherever both channel counts are 2 ... 32, else this kernel. The weight gradient is
// on the tensor cores under the same condition (wgrad_mma_kernel, the gradient rounded to
// BF16 as it is staged); the layers with one channel (input, output) use wgrad_kernel, which
// keeps a thread's 36 (c_out, c_in, tap) sums in registers and slides along image rows.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "device_util.cuh"
#include "wdb_internal.h"

namespace wdb {
namespace {

using bf16 = __nv_bfloat16;
constexpr int kT = 16;          // tile side
constexpr int kHalo = kT + 2;
constexpr int kCMax = 32;

__device__ __forceinline__ float ld(const bf16* p, size_t i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ float ld(const float* p, size_t i) { return p[i]; }

// out mode: 0 store BF16, 1 store FP32, 2 add into FP32
template <int COMAX, typename TIN>
__global__ void __launch_bounds__(256) conv3x3_kernel(const TIN* __restrict__ in, int CI, int CO, int H, int W,
                                                      const bf16* __restrict__ wt, const float* __restrict__ bias,
                                                      int out_mode, void* out, int relu,
                                                      const bf16* __restrict__ mask, const float* __restrict__ residual) {
    extern __shared__ __align__(16) float sm[];
    float* S = sm;                          // [CI][18][18]
    float* Wsm = sm + CI * kHalo * kHalo;   // [CI*9][COMAX]
    const int t = threadIdx.x;
    const int b = blockIdx.z;
    const int ty0 = blockIdx.y * kT, tx0 = blockIdx.x * kT;
    const size_t plane = (size_t)H * W;
    const int nw = CO * CI * 9;
    for (int i = t; i < CI * 9 * COMAX; i += 256) Wsm[i] = 0.f;
    __syncthreads();
    for (int i = t; i < nw; i += 256) {
        const int co = i / (CI * 9), rest = i - co * CI * 9;
        Wsm[rest * COMAX + co] = __bfloat162float(wt[i]);
    }
    const TIN* inb = in + (size_t)b * CI * plane;
    for (int i = t; i < CI * kHalo * kHalo; i += 256) {
        const int ci = i / (kHalo * kHalo), r = i - ci * kHalo * kHalo;
        const int y = r / kHalo, x = r - y * kHalo;
        int gy = (ty0 + y - 1) % H, gx = (tx0 + x - 1) % W;
        gy += gy < 0 ? H : 0;
        gx += gx < 0 ? W : 0;
        S[i] = ld(inb, (size_t)ci * plane + (size_t)gy * W + gx);
    }
    __syncthreads();
    const int py = t / kT, px = t - py * kT;
    const int oy = ty0 + py, ox = tx0 + px;
    float acc[COMAX];
#pragma unroll
    for (int co = 0; co < COMAX; ++co) acc[co] = (bias && co < CO) ? bias[co] : 0.f;
    for (int ci = 0; ci < CI; ++ci) {
        const float* s = S + ci * kHalo * kHalo + py * kHalo + px;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                const float xv = s[ky * kHalo + kx];
                const float* w = Wsm + (ci * 9 + ky * 3 + kx) * COMAX;
                if (COMAX % 4 == 0) {
#pragma unroll
                    for (int co = 0; co < COMAX; co += 4) {
                        const float4 w4 = *reinterpret_cast<const float4*>(w + co);
                        acc[co] += w4.x * xv;
                        acc[co + 1] += w4.y * xv;
                        acc[co + 2] += w4.z * xv;
                        acc[co + 3] += w4.w * xv;
                    }
                } else {
#pragma unroll
                    for (int co = 0; co < COMAX; ++co) acc[co] += w[co] * xv;
                }
            }
    }
    if (oy >= H || ox >= W) return;
    const size_t pix = (size_t)oy * W + ox;
#pragma unroll
    for (int co = 0; co < COMAX; ++co) {
        if (co >= CO) break;
        float v = acc[co];
        if (relu) v = fmaxf(v, 0.f);
        const size_t o = ((size_t)b * CO + co) * plane + pix;
        if (mask && !(__bfloat162float(mask[o]) > 0.f)) v = 0.f;
        if (residual) v += residual[(size_t)b * plane + pix];
        if (out_mode == 0) reinterpret_cast<bf16*>(out)[o] = __float2bfloat16(v);
        else if (out_mode == 1) reinterpret_cast<float*>(out)[o] = v;
        else reinterpret_cast<float*>(out)[o] += v;
    }
}

// Tensor-core 3x3 convolution of BF16 feature maps (2 <= C_in, C_out <= 32), as an implicit
// GEMM per 16 x 16 output tile: M = 256 pixels, N = C_out (padded to 32), K = 9 taps x C_in
// (padded to KCH = 16 or 32). The input tile with its periodic halo is staged channels-last
// ([18 x 18 pixels][kCP channels]) and the weights as [tap][C_out][kCP], both BF16, so that
// every A fragment (16 pixels of one tile row, 16 channels) and B fragment (8 output
// channels, 16 input channels) is one ldmatrix; mma.sync m16n8k16 (BF16 in, FP32 accumulate).
// Warp w computes tile rows 2w and 2w + 1. The FP32 results go through shared memory
// ([C_out][256 pixels]) so that the stores to the NCHW output are coalesced.
constexpr int kCP = 40;                       // channel pitch in shared memory (80 B: no ldmatrix bank conflicts)
constexpr int kMmaHalo = 18 * 18 * kCP;       // bf16 elements of the staged input tile
constexpr int kMmaW = 9 * 32 * kCP;           // bf16 elements of the staged weights
constexpr size_t kMmaSmem = sizeof(bf16) * (kMmaHalo + kMmaW);

__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                         unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

template <int KCH>
__global__ void __launch_bounds__(256) conv3x3_mma_kernel(const bf16* __restrict__ in, int CI, int CO, int H, int W,
                                                          const bf16* __restrict__ wlay, const float* __restrict__ bias,
                                                          int out_mode, void* out, int relu,
                                                          const bf16* __restrict__ mask,
                                                          const float* __restrict__ residual) {
    extern __shared__ __align__(16) unsigned char cnn_smem[];
    bf16* halo = reinterpret_cast<bf16*>(cnn_smem);   // [18*18][kCP]
    bf16* ws = halo + kMmaHalo;                        // [9][32][kCP]
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int b = blockIdx.z;
    const int ty0 = blockIdx.y * kT, tx0 = blockIdx.x * kT;
    const size_t plane = (size_t)H * W;
    // weights, already laid out as [tap][co][kCP] (zeros outside C_out x C_in): 16-byte copies
    {
        const uint4* src = reinterpret_cast<const uint4*>(wlay);
        uint4* dst = reinterpret_cast<uint4*>(ws);
        for (int i = t; i < kMmaW / 8; i += 256) dst[i] = src[i];
    }
    // input tile with its periodic halo, channels-last: one pixel per thread, channel pairs
    // packed into 32-bit words, 16-byte stores; channels CI..KCH-1 are zero
    const bf16* inb = in + (size_t)b * CI * plane;
    for (int q = t; q < kHalo * kHalo; q += 256) {
        const int y = q / kHalo, x = q - y * kHalo;
        int gy = ty0 + y - 1, gx = tx0 + x - 1;
        while (gy < 0) gy += H;
        while (gy >= H) gy -= H;
        while (gx < 0) gx += W;
        while (gx >= W) gx -= W;
        const bf16* src = inb + (size_t)gy * W + gx;
        unsigned packed[KCH / 2];
#pragma unroll
        for (int c = 0; c < KCH / 2; ++c) {
            const unsigned short lo = (2 * c < CI) ? __bfloat16_as_ushort(src[(size_t)(2 * c) * plane]) : 0;
            const unsigned short hi = (2 * c + 1 < CI) ? __bfloat16_as_ushort(src[(size_t)(2 * c + 1) * plane]) : 0;
            packed[c] = (unsigned)lo | ((unsigned)hi << 16);
        }
        uint4* dst = reinterpret_cast<uint4*>(halo + q * kCP);
#pragma unroll
        for (int c = 0; c < KCH / 8; ++c)
            dst[c] = make_uint4(packed[4 * c], packed[4 * c + 1], packed[4 * c + 2], packed[4 * c + 3]);
    }
    __syncthreads();
    float acc[2][4][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[m][nt][k] = 0.f;
    const unsigned hb = (unsigned)__cvta_generic_to_shared(halo), wb = (unsigned)__cvta_generic_to_shared(ws);
    // ldmatrix row addresses: A rows are pixels (lane % 16), k half (lane / 16);
    // B rows are output channels (lane % 8 + 8 (lane / 16)), k half ((lane / 8) % 2)
    const int a_pix = lane & 15, a_k = (lane >> 4) * 8;
    const int b_n = (lane & 7) + ((lane >> 4) << 3), b_k = ((lane >> 3) & 1) * 8;
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
        const int ky = tap / 3, kx = tap - ky * 3;
#pragma unroll
        for (int kc = 0; kc < KCH / 16; ++kc) {
            unsigned a[2][4], bf[2][4];
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int pix = (2 * warp + m + ky) * kHalo + a_pix + kx;
                ldsm_x4(hb + 2u * (unsigned)(pix * kCP + kc * 16 + a_k), a[m][0], a[m][1], a[m][2], a[m][3]);
            }
#pragma unroll
            for (int h = 0; h < 2; ++h)
                ldsm_x4(wb + 2u * (unsigned)((tap * 32 + 16 * h + b_n) * kCP + kc * 16 + b_k), bf[h][0], bf[h][1],
                        bf[h][2], bf[h][3]);
#pragma unroll
            for (int m = 0; m < 2; ++m)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
                    mma_bf16(acc[m][nt], a[m][0], a[m][1], a[m][2], a[m][3], bf[nt >> 1][(nt & 1) * 2],
                             bf[nt >> 1][(nt & 1) * 2 + 1]);
        }
    }
    __syncthreads();
    // results -> shared [co][256 pixels] (FP32), then coalesced stores
    float* res = reinterpret_cast<float*>(cnn_smem);
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int px = (lane >> 2) + ((k >> 1) << 3);
                const int co = nt * 8 + (lane & 3) * 2 + (k & 1);
                res[co * 256 + (2 * warp + m) * kT + px] = acc[m][nt][k];
            }
    __syncthreads();
    for (int i = t; i < CO * 256; i += 256) {
        const int co = i >> 8, p = i & 255;
        const int oy = ty0 + (p >> 4), ox = tx0 + (p & 15);
        if (oy >= H || ox >= W) continue;
        float v = res[i] + (bias ? bias[co] : 0.f);
        if (relu) v = fmaxf(v, 0.f);
        const size_t pix = (size_t)oy * W + ox;
        const size_t o = ((size_t)b * CO + co) * plane + pix;
        if (mask && !(__bfloat162float(mask[o]) > 0.f)) v = 0.f;
        if (residual) v += residual[(size_t)b * plane + pix];
        if (out_mode == 0) reinterpret_cast<bf16*>(out)[o] = __float2bfloat16(v);
        else if (out_mode == 1) reinterpret_cast<float*>(out)[o] = v;
        else reinterpret_cast<float*>(out)[o] += v;
    }
}

// BF16 weights [C_out][C_in][3][3] -> [tap][32][kCP] (zeros outside C_out x C_in), the layout
// conv3x3_mma_kernel stages with 16-byte copies
__global__ void relayout_weights_kernel(const bf16* __restrict__ w, bf16* __restrict__ out, int CO, int CI) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMmaW) return;
    const int tap = i / (32 * kCP), r = i - tap * 32 * kCP;
    const int co = r / kCP, ci = r - co * kCP;
    out[i] = (co < CO && ci < CI) ? w[((size_t)co * CI + ci) * 9 + tap] : __float2bfloat16(0.f);
}

// dW[co][ci][k] += sum_{b,p} dout[b][co][p] in[b][ci][p + k - 1]; db[co] += sum dout[b][co][p].
// Thread t owns c_out = t / 8 and c_in = 4 (t % 8) .. + 3, all 9 taps (36 sums).
template <typename TIN>
__global__ void __launch_bounds__(256) wgrad_kernel(const TIN* __restrict__ in, int CI, int CO, int H, int W, int B,
                                                    const float* __restrict__ dout, float* dW, float* db) {
    extern __shared__ __align__(16) float sm[];
    float* S = sm;                             // [CI][18][18]
    float* D = sm + kCMax * kHalo * kHalo;     // [CO][16][16]
    const int t = threadIdx.x;
    const int co = t >> 3, ci0 = (t & 7) * 4;
    float acc[4][9];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[c][k] = 0.f;
    float bsum = 0.f;
    const int tx = (W + kT - 1) / kT, ty = (H + kT - 1) / kT;
    const int tiles = B * tx * ty;
    const size_t plane = (size_t)H * W;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int b = tile / (tx * ty), r = tile - b * tx * ty;
        const int ty0 = (r / tx) * kT, tx0 = (r % tx) * kT;
        const TIN* inb = in + (size_t)b * CI * plane;
        for (int i = t; i < CI * kHalo * kHalo; i += 256) {
            const int c = i / (kHalo * kHalo), q = i - c * kHalo * kHalo;
            const int y = q / kHalo, x = q - y * kHalo;
            int gy = (ty0 + y - 1) % H, gx = (tx0 + x - 1) % W;
            gy += gy < 0 ? H : 0;
            gx += gx < 0 ? W : 0;
            S[i] = ld(inb, (size_t)c * plane + (size_t)gy * W + gx);
        }
        for (int i = t; i < CO * kT * kT; i += 256) {
            const int c = i / (kT * kT), q = i - c * kT * kT;
            const int y = ty0 + q / kT, x = tx0 + (q % kT);
            D[i] = (y < H && x < W) ? dout[((size_t)b * CO + c) * plane + (size_t)y * W + x] : 0.f;
        }
        __syncthreads();
        if (co < CO) {
            for (int py = 0; py < kT; ++py) {
                float d[kT];
#pragma unroll
                for (int px = 0; px < kT; ++px) d[px] = D[(co * kT + py) * kT + px];
                if ((t & 7) == 0) {
#pragma unroll
                    for (int px = 0; px < kT; ++px) bsum += d[px];
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (ci0 + c >= CI) break;
#pragma unroll
                    for (int ky = 0; ky < 3; ++ky) {
                        float row[kHalo];
                        const float* sr = S + ((ci0 + c) * kHalo + py + ky) * kHalo;
#pragma unroll
                        for (int x = 0; x < kHalo; ++x) row[x] = sr[x];
#pragma unroll
                        for (int kx = 0; kx < 3; ++kx) {
                            float a = 0.f;
#pragma unroll
                            for (int px = 0; px < kT; ++px) a += d[px] * row[px + kx];
                            acc[c][ky * 3 + kx] += a;
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    if (co < CO) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (ci0 + c >= CI) break;
#pragma unroll
            for (int k = 0; k < 9; ++k) atomicAdd(&dW[((size_t)co * CI + ci0 + c) * 9 + k], acc[c][k]);
        }
        if ((t & 7) == 0) atomicAdd(&db[co], bsum);
    }
}

// Tensor-core weight gradient (2 <= C_in, C_out <= 32): dW[co][ci][tap] += sum over pixels of
// g[co][p] x[ci][p + offset(tap)], an implicit GEMM per 16 x 16 tile with M = C_out (two
// m-tiles of 16), N = C_in per tap (four n-tiles of 8) and K = the tile's 256 pixels, one
// tile row of 16 per k-step. The FP32 output gradient is rounded to BF16 as it is staged
// ([32 c_out][kGP], pixels contiguous: A fragments by ldmatrix), the input tile with its
// periodic halo channels-last ([18 x 18][kCP]: B fragments by ldmatrix.trans). Warp w owns
// the output tile (m, n) = (w / 4, w % 4) for all nine taps, so one A fragment serves nine
// mma per k-step; the persistent CTAs accumulate over their tiles in registers and add the
// result to dW with FP32 atomics. db is summed from the FP32 gradient.
constexpr int kGP = 264;   // pixel pitch of the staged gradient tile (528-byte rows)
constexpr size_t kWgSmem = sizeof(bf16) * (kMmaHalo + 32 * kGP);

__device__ __forceinline__ void ldsm_x2_trans(unsigned addr, unsigned& r0, unsigned& r1) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}

__global__ void __launch_bounds__(256) wgrad_mma_kernel(const bf16* __restrict__ in, int CI, int CO, int H, int W,
                                                        int B, const float* __restrict__ dout, float* dW, float* db) {
    extern __shared__ __align__(16) unsigned char cnn_smem[];
    bf16* halo = reinterpret_cast<bf16*>(cnn_smem);   // [18*18][kCP]
    bf16* gs = halo + kMmaHalo;                        // [32][kGP]
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int m = warp >> 2, nt = warp & 3;
    float acc[9][4];
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[k][e] = 0.f;
    float bs[32];       // db partials: thread t sums pixel t of every tile, per c_out
#pragma unroll
    for (int j = 0; j < 32; ++j) bs[j] = 0.f;
    __shared__ float s_db[32];
    if (t < 32) s_db[t] = 0.f;
    const int tx = (W + kT - 1) / kT, ty = (H + kT - 1) / kT;
    const int tiles = B * tx * ty;
    const size_t plane = (size_t)H * W;
    const unsigned hb = (unsigned)__cvta_generic_to_shared(halo), gb = (unsigned)__cvta_generic_to_shared(gs);
    const int a_row = lane & 15, a_k = (lane >> 4) * 8;        // A: c_out rows, pixel halves
    const int b_k = (lane & 7) + ((lane >> 3) & 1) * 8;         // B (trans): pixel rows of the two 8 x 8 halves
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int b = tile / (tx * ty), r = tile - b * tx * ty;
        const int ty0 = (r / tx) * kT, tx0 = (r % tx) * kT;
        __syncthreads();   // the previous tile's fragments are read
        const bf16* inb = in + (size_t)b * CI * plane;
        for (int q = t; q < kHalo * kHalo; q += 256) {
            const int y = q / kHalo, x = q - y * kHalo;
            int gy = ty0 + y - 1, gx = tx0 + x - 1;
            while (gy < 0) gy += H;
            while (gy >= H) gy -= H;
            while (gx < 0) gx += W;
            while (gx >= W) gx -= W;
            const bf16* src = inb + (size_t)gy * W + gx;
            unsigned packed[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const unsigned short lo = (2 * c < CI) ? __bfloat16_as_ushort(src[(size_t)(2 * c) * plane]) : 0;
                const unsigned short hi = (2 * c + 1 < CI) ? __bfloat16_as_ushort(src[(size_t)(2 * c + 1) * plane]) : 0;
                packed[c] = (unsigned)lo | ((unsigned)hi << 16);
            }
            uint4* dst = reinterpret_cast<uint4*>(halo + q * kCP);
#pragma unroll
            for (int c = 0; c < 4; ++c)
                dst[c] = make_uint4(packed[4 * c], packed[4 * c + 1], packed[4 * c + 2], packed[4 * c + 3]);
        }
        const float* gbase = dout + (size_t)b * CO * plane;
        {
            const int oy = ty0 + (t >> 4), ox = tx0 + (t & 15);
            const bool inside = oy < H && ox < W;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float v = (j < CO && inside) ? gbase[(size_t)j * plane + (size_t)oy * W + ox] : 0.f;
                gs[j * kGP + t] = __float2bfloat16(v);
                bs[j] += v;
            }
        }
        __syncthreads();
#pragma unroll 1
        for (int kr = 0; kr < kT; ++kr) {
            unsigned a0, a1, a2, a3;
            ldsm_x4(gb + 2u * (unsigned)((m * 16 + a_row) * kGP + kr * 16 + a_k), a0, a1, a2, a3);
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const int ky = tap / 3, kx = tap - ky * 3;
                unsigned b0, b1;
                ldsm_x2_trans(hb + 2u * (unsigned)(((kr + ky) * kHalo + b_k + kx) * kCP + nt * 8), b0, b1);
                mma_bf16(acc[tap], a0, a1, a2, a3, b0, b1);
            }
        }
    }
    // D fragment: rows (c_out) m*16 + lane/4 (+8), columns (c_in) nt*8 + 2 (lane % 4) (+1)
#pragma unroll
    for (int tap = 0; tap < 9; ++tap)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int co = m * 16 + (lane >> 2) + ((e >> 1) << 3);
            const int ci = nt * 8 + (lane & 3) * 2 + (e & 1);
            if (co < CO && ci < CI) atomicAdd(&dW[((size_t)co * CI + ci) * 9 + tap], acc[tap][e]);
        }
    // db: per c_out, the threads' pixel sums reduced by warp, then across warps in shared memory
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        float v = bs[j];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) atomicAdd(&s_db[j], v);
    }
    __syncthreads();
    if (t < CO) atomicAdd(&db[t], s_db[t]);
}

// Wt[ci][co][8-k] = W[co][ci][k] (data gradient weights)
__global__ void flip_transpose_kernel(const bf16* __restrict__ w, bf16* __restrict__ wt, int CO, int CI) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= CO * CI * 9) return;
    const int co = i / (CI * 9), r = i - co * CI * 9, ci = r / 9, k = r - ci * 9;
    wt[((size_t)ci * CO + co) * 9 + (8 - k)] = w[i];
}

template <typename TIN>
__global__ void avgpool2_kernel(const TIN* __restrict__ in, bf16* __restrict__ out, int BC, int H, int W) {
    const size_t n = (size_t)BC * (H / 2) * (W / 2);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % (W / 2));
        const size_t q = i / (W / 2);
        const int y = (int)(q % (H / 2));
        const size_t c = q / (H / 2);
        const TIN* p = in + c * H * W + (size_t)(2 * y) * W + 2 * x;
        out[i] = __float2bfloat16(0.25f * (ld(p, 0) + ld(p, 1) + ld(p, W) + ld(p, W + 1)));
    }
}

// s = up2(d) + e  (d at half resolution)
__global__ void up2_add_kernel(const bf16* __restrict__ d, const bf16* __restrict__ e, bf16* __restrict__ s, int BC,
                               int H, int W) {
    const size_t n = (size_t)BC * H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % W);
        const size_t q = i / W;
        const int y = (int)(q % H);
        const size_t c = q / H;
        s[i] = __float2bfloat16(__bfloat162float(d[c * (H / 2) * (W / 2) + (size_t)(y / 2) * (W / 2) + x / 2]) +
                                __bfloat162float(e[i]));
    }
}

// gradient into d_{l+1}: sum over every 2 x 2 block of ds (half-resolution output, overwritten)
__global__ void up2_backward_kernel(const float* __restrict__ ds, float* __restrict__ dd, int BC, int H, int W) {
    const size_t n = (size_t)BC * (H / 2) * (W / 2);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % (W / 2));
        const size_t q = i / (W / 2);
        const int y = (int)(q % (H / 2));
        const size_t c = q / (H / 2);
        const float* p = ds + c * H * W + (size_t)(2 * y) * W + 2 * x;
        dd[i] = p[0] + p[1] + p[W] + p[W + 1];
    }
}

// gradient of avgpool2: add 1/4 of the half-resolution gradient to every pixel of its block
__global__ void avgpool2_backward_add_kernel(const float* __restrict__ dp, float* __restrict__ dx, int BC, int H, int W) {
    const size_t n = (size_t)BC * H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % W);
        const size_t q = i / W;
        const int y = (int)(q % H);
        const size_t c = q / H;
        dx[i] += 0.25f * dp[c * (H / 2) * (W / 2) + (size_t)(y / 2) * (W / 2) + x / 2];
    }
}

// g = g * (act > 0)
__global__ void relu_mask_kernel(float* __restrict__ g, const bf16* __restrict__ act, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!(__bfloat162float(act[i]) > 0.f)) g[i] = 0.f;
}

// dv = 2 (v - t) / n; loss partial sums (FP64 tree)
__global__ void __launch_bounds__(256) mse_kernel(const float* __restrict__ v, const float* __restrict__ tgt,
                                                  float* __restrict__ dv, size_t n, double* part, unsigned int* counter,
                                                  double* out) {
    float s = 0.f, c = 0.f;
    const float scale = 2.0f / (float)n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float d = v[i] - tgt[i];
        dv[i] = scale * d;
        neu_add(s, c, d * d);
    }
    double a[1] = {(double)s + (double)c}, tot[1];
    if (grid_reduce<1>(a, 0u, part, counter, tot) && threadIdx.x == 0) out[0] = tot[0] / (double)n;
}

// tot = sum v^2 (FP64 tree)
__global__ void __launch_bounds__(256) sumsq_kernel(const float* __restrict__ v, size_t n, double* part,
                                                    unsigned int* counter, double* out) {
    float s = 0.f, c = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        neu_add(s, c, v[i] * v[i]);
    double a[1] = {(double)s + (double)c}, tot[1];
    if (grid_reduce<1>(a, 0u, part, counter, tot) && threadIdx.x == 0) out[0] = tot[0];
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, bf16* __restrict__ pb, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        pb[i] = __float2bfloat16(pi);
    }
}

__global__ void to_bf16_kernel(const float* __restrict__ p, bf16* __restrict__ pb, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        pb[i] = __float2bfloat16(p[i]);
}

// splitmix64 + Box-Muller normal numbers (He initialisation of the weights)
__global__ void init_normal_kernel(float* __restrict__ p, long long n, unsigned long long seed, float std) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z[2];
        for (int k = 0; k < 2; ++k) {
            unsigned long long s = seed + (unsigned long long)(2 * i + k + 1) * 0x9E3779B97F4A7C15ull;
            s = (s ^ (s >> 30)) * 0xBF58476D1CE4E5B9ull;
            s = (s ^ (s >> 27)) * 0x94D049BB133111EBull;
            z[k] = s ^ (s >> 31);
        }
        const double u1 = ((double)(z[0] >> 11) + 1.0) * 0x1.0p-53, u2 = (double)(z[1] >> 11) * 0x1.0p-53;
        p[i] = (float)(std * sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
    }
}

int ew(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 4096)); }

}  // namespace
}  // namespace wdb

using namespace wdb;

struct ConvLayer {
    int ci, co;
    long long w_off, b_off;     // offsets in the flat parameter vector
};

struct wdb_cnn {
    int L = 4, C = 32, H = 0, W = 0, Bmax = 0;
    std::vector<ConvLayer> convs;   // order of the flat vector
    long long n_params = 0;
    long long step = 0;
    unsigned long long seed = 0;
    std::vector<void*> allocs;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;   // FP32 master, grad, Adam moments
    bf16 *pb = nullptr, *wt = nullptr;                              // BF16 weights, flipped copy
    bf16* wlay = nullptr;                                           // per layer: [tap][32][kCP] for the MMA path
    bf16* wlay_t = nullptr;                                         // flipped copy in the MMA layout (data gradient)
    bf16* gb16 = nullptr;                                           // data-gradient input rounded to BF16
    // activations (BF16) per level: inp (l > 0), a, e; decoder s, a, d
    std::vector<bf16*> e_inp, e_a, e_e, d_s, d_a, d_d;
    std::vector<float*> g_enc;          // gradient accumulators of e_l (FP32)
    float *g0 = nullptr, *g1 = nullptr, *g2 = nullptr;   // scratch gradients at full resolution
    float* dv = nullptr;
    double* part = nullptr;
    unsigned int* counter = nullptr;
    double* d_loss = nullptr;
    // batch-1 forward replayed as a CUDA graph (input copied to u1, output in g0)
    float* u1 = nullptr;
    cudaStream_t work = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t fwd1 = nullptr;
    long long fwd1_launches = 0;
};

namespace {

template <typename T>
wdb_status cnn_alloc(wdb_cnn* n, T** p, size_t count) {
    void* q = nullptr;
    WDB_CK(cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)));
    n->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return WDB_OK;
}

int lvl_h(const wdb_cnn* n, int l) { return n->H >> l; }
int lvl_w(const wdb_cnn* n, int l) { return n->W >> l; }

// conv layer index in the flat order
int idx_in() { return 0; }
int idx_e0() { return 1; }
int idx_ea(int l) { return 2 + 2 * (l - 1); }
int idx_eb(int l) { return 3 + 2 * (l - 1); }
int idx_da(const wdb_cnn* n, int l) { return 2 * n->L + 2 * (n->L - 2 - l); }
int idx_db(const wdb_cnn* n, int l) { return 2 * n->L + 2 * (n->L - 2 - l) + 1; }
int idx_out(const wdb_cnn* n) { return (int)n->convs.size() - 1; }

size_t conv_smem(int CI, int COMAX) { return sizeof(float) * (size_t)(CI * kHalo * kHalo + CI * 9 * COMAX); }

template <typename TIN>
wdb_status conv(const wdb_cnn* n, int layer, const TIN* in, int B, int l, int out_mode, void* out, int relu,
                const bf16* mask, const float* residual, bool flipped, cudaStream_t st) {
    const ConvLayer& cl = n->convs[layer];
    const int CI = flipped ? cl.co : cl.ci, CO = flipped ? cl.ci : cl.co;
    const int H = lvl_h(n, l), W = lvl_w(n, l);
    const bf16* w = n->pb + cl.w_off;
    if (flipped) {
        flip_transpose_kernel<<<(cl.co * cl.ci * 9 + 255) / 256, 256, 0, st>>>(w, n->wt, cl.co, cl.ci);
        count_launch();
        w = n->wt;
    }
    const float* bias = flipped ? nullptr : n->p + cl.b_off;
    dim3 grid((W + kT - 1) / kT, (H + kT - 1) / kT, B);
    if constexpr (std::is_same<TIN, float>::value) {
        if (flipped && CI >= 2 && CO >= 2 && CI <= kCMax && CO <= kCMax) {
            // data gradient on the tensor cores: the FP32 gradient rounded to BF16 (as the
            // feature maps are stored), the flipped weights in the MMA layout
            const long long cnt = (long long)B * CI * H * W;
            to_bf16_kernel<<<ew(cnt), 256, 0, st>>>(in, n->gb16, cnt);
            relayout_weights_kernel<<<(kMmaW + 255) / 256, 256, 0, st>>>(w, n->wlay_t, CO, CI);
            count_launch(2);
            static unsigned long long attr_t = 0ull;
            if (!done_on_device(&attr_t)) {
                WDB_CK(cudaFuncSetAttribute(conv3x3_mma_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)kMmaSmem));
                WDB_CK(cudaFuncSetAttribute(conv3x3_mma_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)kMmaSmem));
                mark_on_device(&attr_t);
            }
            if (CI <= 16)
                conv3x3_mma_kernel<16><<<grid, 256, kMmaSmem, st>>>(n->gb16, CI, CO, H, W, n->wlay_t, nullptr, out_mode,
                                                                    out, relu, mask, residual);
            else
                conv3x3_mma_kernel<32><<<grid, 256, kMmaSmem, st>>>(n->gb16, CI, CO, H, W, n->wlay_t, nullptr, out_mode,
                                                                    out, relu, mask, residual);
            count_launch();
            WDB_CK(cudaGetLastError());
            return WDB_OK;
        }
    }
    if constexpr (std::is_same<TIN, bf16>::value) {
        if (!flipped && CI >= 2 && CO >= 2 && CI <= kCMax && CO <= kCMax) {   // BF16 feature maps: tensor cores
            const bf16* wl = n->wlay + (size_t)layer * kMmaW;
            static unsigned long long attr = 0ull;
            if (!done_on_device(&attr)) {
                WDB_CK(cudaFuncSetAttribute(conv3x3_mma_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)kMmaSmem));
                WDB_CK(cudaFuncSetAttribute(conv3x3_mma_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)kMmaSmem));
                mark_on_device(&attr);
            }
            if (CI <= 16)
                conv3x3_mma_kernel<16><<<grid, 256, kMmaSmem, st>>>(in, CI, CO, H, W, wl, bias, out_mode, out, relu,
                                                                    mask, residual);
            else
                conv3x3_mma_kernel<32><<<grid, 256, kMmaSmem, st>>>(in, CI, CO, H, W, wl, bias, out_mode, out, relu,
                                                                    mask, residual);
            count_launch();
            WDB_CK(cudaGetLastError());
            return WDB_OK;
        }
    }
    if (CO <= 1) {
        conv3x3_kernel<1, TIN><<<grid, 256, conv_smem(CI, 1), st>>>(in, CI, CO, H, W, w, bias, out_mode, out, relu,
                                                                     mask, residual);
    } else {
        static unsigned long long attr = 0ull;
        if (!done_on_device(&attr)) {
            WDB_CK(cudaFuncSetAttribute(conv3x3_kernel<32, bf16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)conv_smem(32, 32)));
            WDB_CK(cudaFuncSetAttribute(conv3x3_kernel<32, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)conv_smem(32, 32)));
            mark_on_device(&attr);
        }
        conv3x3_kernel<32, TIN><<<grid, 256, conv_smem(CI, 32), st>>>(in, CI, CO, H, W, w, bias, out_mode, out, relu,
                                                                       mask, residual);
    }
    count_launch();
    WDB_CK(cudaGetLastError());
    return WDB_OK;
}

template <typename TIN>
wdb_status wgrad(const wdb_cnn* n, int layer, const TIN* in, const float* dout, int B, int l, cudaStream_t st) {
    const ConvLayer& cl = n->convs[layer];
    static unsigned long long attr = 0ull;
    const size_t smem = sizeof(float) * (size_t)(kCMax * kHalo * kHalo + kCMax * kT * kT);
    if (!done_on_device(&attr)) {
        WDB_CK(cudaFuncSetAttribute(wgrad_kernel<bf16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        WDB_CK(cudaFuncSetAttribute(wgrad_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        mark_on_device(&attr);
    }
    const int H = lvl_h(n, l), W = lvl_w(n, l);
    const int tiles = B * ((H + kT - 1) / kT) * ((W + kT - 1) / kT);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, std::min(tiles, 2 * std::max(sms, 1)));
    if constexpr (std::is_same<TIN, bf16>::value) {
        if (cl.ci >= 2 && cl.co >= 2 && cl.ci <= kCMax && cl.co <= kCMax) {   // tensor cores
            static unsigned long long attr_m = 0ull;
            if (!done_on_device(&attr_m)) {
                WDB_CK(cudaFuncSetAttribute(wgrad_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)kWgSmem));
                mark_on_device(&attr_m);
            }
            wgrad_mma_kernel<<<grid, 256, kWgSmem, st>>>(in, cl.ci, cl.co, H, W, B, dout, n->g + cl.w_off,
                                                         n->g + cl.b_off);
            count_launch();
            WDB_CK(cudaGetLastError());
            return WDB_OK;
        }
    }
    wgrad_kernel<TIN><<<grid, 256, smem, st>>>(in, cl.ci, cl.co, H, W, B, dout, n->g + cl.w_off, n->g + cl.b_off);
    count_launch();
    WDB_CK(cudaGetLastError());
    return WDB_OK;
}

wdb_status forward(wdb_cnn* n, const float* u, float* v_out, int B, cudaStream_t st) {
    const int L = n->L, C = n->C;
    for (int l = 0; l < L; ++l) {
        const int H = lvl_h(n, l), W = lvl_w(n, l);
        if (l == 0) {
            WDB_TRY(conv<float>(n, idx_in(), u, B, 0, 0, n->e_a[0], 1, nullptr, nullptr, false, st));
            WDB_TRY(conv<bf16>(n, idx_e0(), n->e_a[0], B, 0, 0, n->e_e[0], 1, nullptr, nullptr, false, st));
        } else {
            avgpool2_kernel<bf16><<<ew((long long)B * C * H * W), 256, 0, st>>>(n->e_e[l - 1], n->e_inp[l], B * C,
                                                                              2 * H, 2 * W);
            count_launch();
            WDB_TRY(conv<bf16>(n, idx_ea(l), n->e_inp[l], B, l, 0, n->e_a[l], 1, nullptr, nullptr, false, st));
            WDB_TRY(conv<bf16>(n, idx_eb(l), n->e_a[l], B, l, 0, n->e_e[l], 1, nullptr, nullptr, false, st));
        }
    }
    const bf16* d = n->e_e[L - 1];
    for (int l = L - 2; l >= 0; --l) {
        const int H = lvl_h(n, l), W = lvl_w(n, l);
        up2_add_kernel<<<ew((long long)B * C * H * W), 256, 0, st>>>(d, n->e_e[l], n->d_s[l], B * C, H, W);
        count_launch();
        WDB_TRY(conv<bf16>(n, idx_da(n, l), n->d_s[l], B, l, 0, n->d_a[l], 1, nullptr, nullptr, false, st));
        WDB_TRY(conv<bf16>(n, idx_db(n, l), n->d_a[l], B, l, 0, n->d_d[l], 1, nullptr, nullptr, false, st));
        d = n->d_d[l];
    }
    // v = u + conv(d_0)
    WDB_TRY(conv<bf16>(n, idx_out(n), d, B, 0, 1, v_out, 0, nullptr, u, false, st));
    WDB_CK(cudaGetLastError());
    return WDB_OK;
}

// d_0 of a 1-level network is e_0
const bf16* d0_of(const wdb_cnn* n) { return n->L >= 2 ? n->d_d[0] : n->e_e[0]; }

wdb_status backward(wdb_cnn* n, const float* u, int B, cudaStream_t st) {
    const int L = n->L, C = n->C;
    const long long full = (long long)B * C * n->H * n->W;
    WDB_CK(cudaMemsetAsync(n->g, 0, sizeof(float) * n->n_params, st));
    for (int l = 0; l < L; ++l)
        WDB_CK(cudaMemsetAsync(n->g_enc[l], 0, sizeof(float) * (size_t)B * C * lvl_h(n, l) * lvl_w(n, l), st));
    // output convolution
    WDB_TRY(wgrad<bf16>(n, idx_out(n), d0_of(n), n->dv, B, 0, st));
    float* dd = n->g0;   // gradient of d_0
    WDB_TRY(conv<float>(n, idx_out(n), n->dv, B, 0, 1, dd, 0, nullptr, nullptr, true, st));
    // decoder, level 0 upwards
    for (int l = 0; l < L - 1; ++l) {
        const long long cnt = (long long)B * C * lvl_h(n, l) * lvl_w(n, l);
        relu_mask_kernel<<<ew(cnt), 256, 0, st>>>(dd, n->d_d[l], cnt);
        count_launch();
        WDB_TRY(wgrad<bf16>(n, idx_db(n, l), n->d_a[l], dd, B, l, st));
        float* da = n->g1;
        WDB_TRY(conv<float>(n, idx_db(n, l), dd, B, l, 1, da, 0, n->d_a[l], nullptr, true, st));
        WDB_TRY(wgrad<bf16>(n, idx_da(n, l), n->d_s[l], da, B, l, st));
        float* ds = n->g2;
        WDB_TRY(conv<float>(n, idx_da(n, l), da, B, l, 1, ds, 0, nullptr, nullptr, true, st));
        // s = up2(d_{l+1}) + e_l
        WDB_CK(cudaMemcpyAsync(n->g_enc[l], ds, sizeof(float) * cnt, cudaMemcpyDeviceToDevice, st));
        up2_backward_kernel<<<ew(cnt / 4), 256, 0, st>>>(ds, n->g0, B * C, lvl_h(n, l), lvl_w(n, l));
        count_launch();
        dd = n->g0;
    }
    // d_{L-1} = e_{L-1}
    const long long cb = (long long)B * C * lvl_h(n, L - 1) * lvl_w(n, L - 1);
    if (L >= 2) {
        float* ge = n->g_enc[L - 1];
        WDB_CK(cudaMemcpyAsync(ge, dd, sizeof(float) * cb, cudaMemcpyDeviceToDevice, st));
    } else {
        WDB_CK(cudaMemcpyAsync(n->g_enc[0], dd, sizeof(float) * cb, cudaMemcpyDeviceToDevice, st));
    }
    // encoder, bottom level first
    for (int l = L - 1; l >= 0; --l) {
        const long long cnt = (long long)B * C * lvl_h(n, l) * lvl_w(n, l);
        float* dz = n->g_enc[l];
        relu_mask_kernel<<<ew(cnt), 256, 0, st>>>(dz, n->e_e[l], cnt);
        count_launch();
        const int la = (l == 0) ? idx_in() : idx_ea(l), lb = (l == 0) ? idx_e0() : idx_eb(l);
        WDB_TRY(wgrad<bf16>(n, lb, n->e_a[l], dz, B, l, st));
        float* da = n->g1;
        WDB_TRY(conv<float>(n, lb, dz, B, l, 1, da, 0, n->e_a[l], nullptr, true, st));
        if (l == 0) {
            WDB_TRY(wgrad<float>(n, la, u, da, B, 0, st));
        } else {
            WDB_TRY(wgrad<bf16>(n, la, n->e_inp[l], da, B, l, st));
            float* dp = n->g2;
            WDB_TRY(conv<float>(n, la, da, B, l, 1, dp, 0, nullptr, nullptr, true, st));
            avgpool2_backward_add_kernel<<<ew(cnt * 4), 256, 0, st>>>(dp, n->g_enc[l - 1], B * C, 2 * lvl_h(n, l),
                                                                      2 * lvl_w(n, l));
            count_launch();
        }
    }
    (void)full;
    WDB_CK(cudaGetLastError());
    return WDB_OK;
}

wdb_status loss(wdb_cnn* n, const float* v, const float* tgt, int B, cudaStream_t st, double* out) {
    const size_t cnt = (size_t)B * n->H * n->W;
    WDB_CK(cudaMemsetAsync(n->counter, 0, sizeof(unsigned int), st));
    mse_kernel<<<std::min(ew((long long)cnt), 1024), 256, 0, st>>>(v, tgt, n->dv, cnt, n->part, n->counter, n->d_loss);
    count_launch();
    WDB_CK(cudaGetLastError());
    WDB_CK(cudaMemcpyAsync(out, n->d_loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    WDB_CK(cudaStreamSynchronize(st));
    return WDB_OK;
}

void cnn_release(wdb_cnn* n) {
    if (!n) return;
    if (n->work) cudaStreamSynchronize(n->work);
    if (n->fwd1) cudaGraphExecDestroy(n->fwd1);
    if (n->ev_in) cudaEventDestroy(n->ev_in);
    if (n->ev_out) cudaEventDestroy(n->ev_out);
    if (n->work) cudaStreamDestroy(n->work);
    for (void* p : n->allocs) cudaFree(p);
    delete n;
}

// Forward of one image u_dev into n->g0 as one CUDA graph launch on the network's stream,
// joined to `st` by events; the graph is captured on first use (after an eager warm-up run
// that also sets the kernels' shared-memory attributes).
wdb_status forward1_graph(wdb_cnn* n, const float* u_dev, cudaStream_t st) {
    WDB_TRY(work_enter(&n->work, &n->ev_in, &n->ev_out, st));
    const size_t img = (size_t)n->H * n->W;
    WDB_CK(cudaMemcpyAsync(n->u1, u_dev, sizeof(float) * img, cudaMemcpyDeviceToDevice, n->work));
    if (!n->fwd1) {
        WDB_TRY(forward(n, n->u1, n->g0, 1, n->work));
        WDB_CK(cudaStreamSynchronize(n->work));
        const long long before = wdb_kernel_launches(0);
        cudaGraph_t g = nullptr;
        WDB_CK(cudaStreamBeginCapture(n->work, cudaStreamCaptureModeThreadLocal));
        const wdb_status s = forward(n, n->u1, n->g0, 1, n->work);
        const cudaError_t e = cudaStreamEndCapture(n->work, &g);
        if (s != WDB_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        n->fwd1_launches = wdb_kernel_launches(0) - before;
        count_launch(-n->fwd1_launches);   // captured, not run
        const cudaError_t ie = cudaGraphInstantiate(&n->fwd1, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return cuda_error(ie, "cudaGraphInstantiate", __FILE__, __LINE__);
    }
    WDB_CK(cudaGraphLaunch(n->fwd1, n->work));
    count_launch(n->fwd1_launches);
    return work_exit(n->work, n->ev_out, st);
}

// refresh the MMA-layout copy of every layer's BF16 weights (after any parameter change)
wdb_status relayout(wdb_cnn* n, cudaStream_t st) {
    for (size_t k = 0; k < n->convs.size(); ++k) {
        const ConvLayer& c = n->convs[k];
        relayout_weights_kernel<<<(kMmaW + 255) / 256, 256, 0, st>>>(n->pb + c.w_off, n->wlay + k * kMmaW, c.co, c.ci);
        count_launch();
    }
    WDB_CK(cudaGetLastError());
    return WDB_OK;
}

constexpr char kMagicCnn[8] = {'W', 'D', 'B', 'C', 'N', 'N', '0', '1'};

}  // namespace

extern "C" {

wdb_status wdb_cnn_create(int levels, int channels, int height, int width, int max_batch, unsigned long long seed,
                          void* stream, wdb_cnn** out) {
    if (!out) return set_error(WDB_EINVAL, "out is NULL");
    *out = nullptr;
    if (levels < 1 || levels > 8) return set_error(WDB_EINVAL, "levels must be in [1, 8]");
    if (channels < 1 || channels > kCMax) return set_error(WDB_EINVAL, "channels must be in [1, 32]");
    if (max_batch < 1) return set_error(WDB_EINVAL, "max_batch must be >= 1");
    if (height <= 0 || width <= 0 || (height % (1 << (levels - 1))) || (width % (1 << (levels - 1))))
        return set_error(WDB_EINVAL, "image sides must be divisible by 2^(levels-1)");
    int nd = 0;
    if (cudaGetDeviceCount(&nd) != cudaSuccess || nd == 0) return set_error(WDB_ECUDA, "no CUDA device available");
    wdb_cnn* n = new (std::nothrow) wdb_cnn();
    if (!n) return set_error(WDB_ENOMEM, "host allocation");
    n->L = levels;
    n->C = channels;
    n->H = height;
    n->W = width;
    n->Bmax = max_batch;
    n->seed = seed;
    const int C = channels;
    auto add = [&](int ci, int co) {
        ConvLayer c{ci, co, n->n_params, n->n_params + (long long)co * ci * 9};
        n->n_params += (long long)co * ci * 9 + co;
        n->convs.push_back(c);
    };
    add(1, C);
    add(C, C);
    for (int l = 1; l < levels; ++l) {
        add(C, C);
        add(C, C);
    }
    for (int l = levels - 2; l >= 0; --l) {
        add(C, C);
        add(C, C);
    }
    add(C, 1);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    wdb_status s = WDB_OK;
    auto A = [&](auto** p, size_t cnt) {
        if (s == WDB_OK) s = cnn_alloc(n, p, cnt);
    };
    A(&n->p, n->n_params);
    A(&n->g, n->n_params);
    A(&n->m, n->n_params);
    A(&n->v, n->n_params);
    A(&n->pb, n->n_params);
    A(&n->wt, (size_t)C * C * 9);
    A(&n->wlay, (size_t)kMmaW * n->convs.size());
    A(&n->wlay_t, (size_t)kMmaW);
    const size_t B = (size_t)max_batch;
    n->e_inp.assign(levels, nullptr);
    n->e_a.assign(levels, nullptr);
    n->e_e.assign(levels, nullptr);
    n->d_s.assign(levels, nullptr);
    n->d_a.assign(levels, nullptr);
    n->d_d.assign(levels, nullptr);
    n->g_enc.assign(levels, nullptr);
    for (int l = 0; l < levels; ++l) {
        const size_t cnt = B * C * (size_t)(height >> l) * (size_t)(width >> l);
        if (l > 0) A(&n->e_inp[l], cnt);
        A(&n->e_a[l], cnt);
        A(&n->e_e[l], cnt);
        if (l < levels - 1) {
            A(&n->d_s[l], cnt);
            A(&n->d_a[l], cnt);
            A(&n->d_d[l], cnt);
        }
        A(&n->g_enc[l], cnt);
    }
    const size_t full = B * C * (size_t)height * width;
    A(&n->gb16, full);
    A(&n->g0, full);
    A(&n->g1, full);
    A(&n->g2, full);
    A(&n->dv, B * (size_t)height * width);
    A(&n->u1, (size_t)height * width);
    A(&n->part, 4096 * 4);
    A(&n->counter, 4);
    A(&n->d_loss, 4);
    if (s == WDB_OK) {
        // He initialisation (weights), zero biases; the output convolution starts at 0.1 x
        cudaMemsetAsync(n->p, 0, sizeof(float) * n->n_params, st);
        for (size_t k = 0; k < n->convs.size(); ++k) {
            const ConvLayer& c = n->convs[k];
            const long long nw = (long long)c.co * c.ci * 9;
            float std = sqrtf(2.0f / (float)(c.ci * 9)) * (k + 1 == n->convs.size() ? 0.1f : 1.0f);
            init_normal_kernel<<<ew(nw), 256, 0, st>>>(n->p + c.w_off, nw, seed + 0x1000ull * (k + 1), std);
        }
        cudaMemsetAsync(n->m, 0, sizeof(float) * n->n_params, st);
        cudaMemsetAsync(n->v, 0, sizeof(float) * n->n_params, st);
        to_bf16_kernel<<<ew(n->n_params), 256, 0, st>>>(n->p, n->pb, n->n_params);
        if (relayout(n, st) != WDB_OK) s = WDB_ECUDA;
        cudaMemsetAsync(n->counter, 0, sizeof(unsigned int) * 4, st);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) s = cuda_error(e, "cnn init", __FILE__, __LINE__);
    }
    if (s != WDB_OK) {
        cnn_release(n);
        return s;
    }
    *out = n;
    return WDB_OK;
}

void wdb_cnn_free(wdb_cnn* n) { cnn_release(n); }

long long wdb_cnn_num_params(const wdb_cnn* n) { return n ? n->n_params : -1; }

wdb_status wdb_cnn_set_params(wdb_cnn* n, const float* host, long long count, void* stream) {
    if (!n || !host) return set_error(WDB_EINVAL, "NULL argument");
    if (count != n->n_params) return set_error(WDB_EINVAL, "expected %lld parameters, got %lld", n->n_params, count);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    WDB_CK(cudaMemcpyAsync(n->p, host, sizeof(float) * count, cudaMemcpyHostToDevice, st));
    WDB_CK(cudaMemsetAsync(n->m, 0, sizeof(float) * count, st));
    WDB_CK(cudaMemsetAsync(n->v, 0, sizeof(float) * count, st));
    to_bf16_kernel<<<ew(count), 256, 0, st>>>(n->p, n->pb, count);
    count_launch();
    WDB_TRY(relayout(n, st));
    n->step = 0;
    WDB_CK(cudaStreamSynchronize(st));
    return WDB_OK;
}

wdb_status wdb_cnn_get_params(const wdb_cnn* n, float* host, long long count) {
    if (!n || !host) return set_error(WDB_EINVAL, "NULL argument");
    if (count < n->n_params) return set_error(WDB_EINVAL, "capacity %lld < %lld", count, n->n_params);
    WDB_CK(cudaMemcpy(host, n->p, sizeof(float) * n->n_params, cudaMemcpyDeviceToHost));
    return WDB_OK;
}

wdb_status wdb_cnn_forward(wdb_cnn* n, const float* u_dev, float* v_dev, int B, void* stream) {
    if (!n || !u_dev || !v_dev) return set_error(WDB_EINVAL, "NULL argument");
    if (B < 1 || B > n->Bmax) return set_error(WDB_EINVAL, "batch %d outside [1, %d]", B, n->Bmax);
    return forward(n, u_dev, v_dev, B, static_cast<cudaStream_t>(stream));
}

wdb_status wdb_cnn_loss_grad(wdb_cnn* n, const float* u_dev, const float* target_dev, int B, void* stream,
                             double* loss_host, float* grad_host) {
    if (!n || !u_dev || !target_dev || !loss_host) return set_error(WDB_EINVAL, "NULL argument");
    if (B < 1 || B > n->Bmax) return set_error(WDB_EINVAL, "batch %d outside [1, %d]", B, n->Bmax);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float* vbuf = n->g2;   // the forward output is consumed by the loss before backward reuses g2
    WDB_TRY(forward(n, u_dev, vbuf, B, st));
    WDB_TRY(loss(n, vbuf, target_dev, B, st, loss_host));
    WDB_TRY(backward(n, u_dev, B, st));
    if (grad_host) {
        WDB_CK(cudaMemcpyAsync(grad_host, n->g, sizeof(float) * n->n_params, cudaMemcpyDeviceToHost, st));
        WDB_CK(cudaStreamSynchronize(st));
    }
    return WDB_OK;
}

wdb_status wdb_cnn_train_step(wdb_cnn* n, const float* u_dev, const float* target_dev, int B, double lr, void* stream,
                              double* loss_host) {
    double l = 0.0;
    WDB_TRY(wdb_cnn_loss_grad(n, u_dev, target_dev, B, stream, &l, nullptr));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    n->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)n->step), c2 = 1.f - powf(b2, (float)n->step);
    adam_kernel<<<ew(n->n_params), 256, 0, st>>>(n->p, n->g, n->m, n->v, n->pb, n->n_params, (float)lr, b1, b2, 1e-8f,
                                                 c1, c2);
    count_launch();
    WDB_TRY(relayout(n, st));
    WDB_CK(cudaGetLastError());
    if (loss_host) *loss_host = l;
    return WDB_OK;
}

wdb_status wdb_solve_warm(wdb_theta* th, wdb_cnn* n, const float* u_dev, float* x_dev, const wdb_solve_params* params,
                          void* stream, wdb_solve_result* result, int* start_used) {
    if (!th || !n || !u_dev || !x_dev || !params || !result) return set_error(WDB_EINVAL, "NULL argument");
    if (th->lay.n_rows != n->H || th->lay.n_cols != n->W)
        return set_error(WDB_EINVAL, "network is %dx%d, operator is %dx%d", n->H, n->W, th->lay.n_rows,
                         th->lay.n_cols);
    if (params->x_init_dev) return set_error(WDB_EINVAL, "x_init_dev must be NULL: the network provides the start");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long N = th->lay.N;
    float* v = n->g0;       // network output (image)
    float* xw = n->g1;      // its coefficients: the candidate start
    float* x0 = n->dv;      // coefficients of u
    float* scratch = n->g2; // N/2 floats of DWT scratch
    WDB_TRY(forward1_graph(n, u_dev, st));
    WDB_TRY(dwt2<float>(v, xw, th->lay, th->filt, scratch, st));
    WDB_TRY(dwt2<float>(u_dev, x0, th->lay, th->filt, scratch, st));
    // E(x = 0) = 1/2 ||x0||^2; the network's start is kept only when its E is lower
    WDB_CK(cudaMemsetAsync(n->counter, 0, sizeof(unsigned int), st));
    sumsq_kernel<<<std::min(ew(N), 1024), 256, 0, st>>>(x0, (size_t)N, n->part, n->counter, n->d_loss);
    count_launch();
    WDB_CK(cudaGetLastError());
    double Ec = 0.0, Ew = 0.0;
    WDB_CK(cudaMemcpyAsync(&Ec, n->d_loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    WDB_TRY(wdb_theta_objective(th, xw, x0, params->lambda, params->w_subband_host, stream, &Ew));   // synchronises
    Ec *= 0.5;
    const bool warm = std::isfinite(Ew) && Ew < Ec;
    wdb_solve_params p = *params;
    p.x_init_dev = warm ? xw : nullptr;
    if (start_used) *start_used = warm ? 1 : 0;
    return wdb_solve(th, u_dev, x_dev, &p, stream, result);
}

wdb_status wdb_cnn_save(const wdb_cnn* n, const char* path) {
    if (!n || !path) return set_error(WDB_EINVAL, "NULL argument");
    std::vector<float> p(n->n_params), m(n->n_params), v(n->n_params);
    WDB_CK(cudaMemcpy(p.data(), n->p, sizeof(float) * n->n_params, cudaMemcpyDeviceToHost));
    WDB_CK(cudaMemcpy(m.data(), n->m, sizeof(float) * n->n_params, cudaMemcpyDeviceToHost));
    WDB_CK(cudaMemcpy(v.data(), n->v, sizeof(float) * n->n_params, cudaMemcpyDeviceToHost));
    FILE* f = std::fopen(path, "wb");
    if (!f) return set_error(WDB_EIO, "cannot open %s", path);
    long long hdr[7] = {n->L, n->C, n->H, n->W, n->Bmax, n->step, (long long)n->seed};
    bool ok = std::fwrite(kMagicCnn, 1, 8, f) == 8 && std::fwrite(hdr, sizeof hdr, 1, f) == 1 &&
              std::fwrite(p.data(), sizeof(float), p.size(), f) == p.size() &&
              std::fwrite(m.data(), sizeof(float), m.size(), f) == m.size() &&
              std::fwrite(v.data(), sizeof(float), v.size(), f) == v.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? WDB_OK : set_error(WDB_EIO, "write failed: %s", path);
}

wdb_status wdb_cnn_load(const char* path, void* stream, wdb_cnn** out) {
    if (!path || !out) return set_error(WDB_EINVAL, "NULL argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return set_error(WDB_EIO, "cannot open %s", path);
    char magic[8];
    long long hdr[7];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagicCnn, 8) == 0 &&
              std::fread(hdr, sizeof hdr, 1, f) == 1;
    wdb_cnn* n = nullptr;
    if (ok) {
        wdb_status s = wdb_cnn_create((int)hdr[0], (int)hdr[1], (int)hdr[2], (int)hdr[3], (int)hdr[4],
                                      (unsigned long long)hdr[6], stream, &n);
        if (s != WDB_OK) {
            std::fclose(f);
            return s;
        }
        std::vector<float> p(n->n_params), m(n->n_params), v(n->n_params);
        ok = std::fread(p.data(), sizeof(float), p.size(), f) == p.size() &&
             std::fread(m.data(), sizeof(float), m.size(), f) == m.size() &&
             std::fread(v.data(), sizeof(float), v.size(), f) == v.size();
        if (ok) {
            cudaStream_t st = static_cast<cudaStream_t>(stream);
            cudaMemcpyAsync(n->p, p.data(), sizeof(float) * p.size(), cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(n->m, m.data(), sizeof(float) * m.size(), cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(n->v, v.data(), sizeof(float) * v.size(), cudaMemcpyHostToDevice, st);
            to_bf16_kernel<<<ew(n->n_params), 256, 0, st>>>(n->p, n->pb, n->n_params);
            relayout(n, st);
            n->step = hdr[5];
            ok = cudaStreamSynchronize(st) == cudaSuccess;
        }
    }
    std::fclose(f);
    if (!ok) {
        cnn_release(n);
        return set_error(WDB_EIO, "bad or truncated file: %s", path);
    }
    *out = n;
    return WDB_OK;
}

}  // extern "C"
