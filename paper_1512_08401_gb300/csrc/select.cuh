// Weighted radix selection of the K largest entries (Sec. 3.7 thresholding), shared by
// the circulant (theta.cu) and row-varying (vtheta.cu) constructions.
//
// Every candidate has a 128-bit key: hi = ~bits(score) (score >= 0, so a smaller hi is a
// larger score), lo = its candidate index (ties by index ascending), and a weight (the
// number of entries of Theta it stands for). Digit passes of 8 bits (8 over hi, then over
// the ibits low bits of lo) accumulate weighted histograms of the keys that share the
// prefix fixed so far; the scan keeps the digits whose total weight stays <= K. After the
// last pass, a key is kept when it sorts before the fixed prefix (the first candidate whose
// weight would exceed K), or everything is kept when the total weight never exceeds K.
#pragma once
#include "wdb_internal.h"

namespace wdb {
namespace {

struct SelState {
    unsigned long long vmax_bits;
    unsigned long long K;
    unsigned long long before;     // weight of keys strictly below the current prefix range
    unsigned long long prefix_hi, prefix_lo;
    unsigned long long count;
    int keep_all;
    int pad;
    unsigned long long hist[256];
};

__global__ void sel_scan_kernel(SelState* sel, int pass) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (!sel->keep_all) {
        unsigned long long excl = 0;
        int dsel = -1;
        for (int d = 0; d < 256; ++d) {
            const unsigned long long hd = sel->hist[d];
            if (sel->before + excl + hd > sel->K) {
                dsel = d;
                break;
            }
            excl += hd;
        }
        if (dsel < 0) {
            sel->keep_all = 1;
        } else {
            sel->before += excl;
            if (pass < 8) sel->prefix_hi = (sel->prefix_hi << 8) | (unsigned long long)dsel;
            else sel->prefix_lo = (sel->prefix_lo << 8) | (unsigned long long)dsel;
        }
    }
    for (int d = 0; d < 256; ++d) sel->hist[d] = 0ull;
}

__device__ __forceinline__ bool kept(const SelState& s, unsigned long long hi, unsigned long long lo) {
    return s.keep_all || hi < s.prefix_hi || (hi == s.prefix_hi && lo < s.prefix_lo);
}

}  // namespace
}  // namespace wdb
