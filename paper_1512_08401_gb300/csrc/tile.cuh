// Tiled gather engine for Theta_K and Theta_K^T (the hot path of Algorithm 3).
//
// A work item is a TS x TS tile of one output subband. For every input subband that feeds
// it, the CTA stages the input region of the tile (plus the tap halo) in shared memory,
// with periodic wrap, and accumulates the taps from there:
//   down pair (input finer or equal, r = 2^lg): out[p] += v_t in[r p + d_t]; the region is
//     stored as r x r polyphase planes so that neighbouring outputs read neighbouring words;
//   up pair (input coarser, r = 2^lg): out[r P + phi] += v_t in[P + d_t] over the taps of
//     phase phi, padded to the same count for every phase;
//   pairs whose region does not fit even for 1 x 1 tiles gather from global memory.
// Tiles are processed heaviest first by persistent CTAs that pull items from a device queue.
// The pairs of a tile are grouped into batches whose regions fit one buffer; each batch is
// staged with cp.async, double buffered so that the next batch's loads are in flight while
// the current batch computes.
#pragma once
#include <vector>

#include "layout_types.h"

namespace wdb {

constexpr int kTileThreads = 256;

enum TileMode { kDown = 0, kUp = 1, kDownGlobal = 2, kUpGlobal = 3 };

// The descriptors are 16-byte aligned so that a thread reads one with 128-bit loads.
struct alignas(16) TilePair {
    int in_sb;
    int soff;         // staged: element offset of this pair's region in the tile's buffer
    int mode;         // TileMode
    int lg;           // log2 of the scale ratio r
    int RR, RC;       // staged region rows / cols (input units for down, P units for up)
    int PR, PC;       // plane rows / cols (down: ceil(RR / r), ceil(RC / r) padded; up: RR, RC padded)
    int PS;           // down: element stride between polyphase planes (>= PR * PC)
    int y0, x0;       // region origin: down Y0 = (ty0 << lg) + y0; up Y0 = (ty0 >> lg) + y0
    int tap_begin;    // first tap (up: phase-interleaved, index tap_begin + j r^2 + phase)
    int ntap;         // down: taps; up: padded taps per phase
    int vec;          // 1: rows staged in 16-byte chunks from a 4-aligned column (up or r = 1 pairs)
    int tst;          // up pairs: 1 when the phase tables are staged with the batch (else read from
                      // global memory)
    int nm;           // output subbands that read this region (grouped items: up to 4; else 1)
    int mtb[4], mnt[4];   // per output subband of the group: first tap and taps (up: per phase)
};

constexpr int kMaxBatchPairs = 16;   // pairs per batch (their descriptors sit in shared memory)

struct alignas(16) TileSub {      // per output subband
    int TS;           // tile side (a power of two)
    int lgTS;
    int pair_begin, pair_end;
    int batch_begin, batch_end;   // batches of pairs whose staged regions share one buffer
    int e4;           // 1: 4 outputs per thread (TS >= 8), 0: 1 output per thread
    int sup;          // 1: work items are super tiles (2 x 2 tiles of side TS staged together)
    int grp;          // grouped items: subbands of this subband's group (the item's o is the first)
    int pad[3];
};

struct TileTune {     // autotuner's choice for one output subband (ts = 0: the planner's)
    int ts;
    int e4;
};

struct alignas(16) TileBatch {    // pairs [pair_begin, pair_end) of one subband, staged together
    int pair_begin, pair_end;
    int tap_begin, tap_end;       // taps of the staged pairs, copied to shared memory
    int tap_soff;                 // int offset of the staged taps in the buffer (FP32: TapOV
                                  // records there; FP64: the offsets, values at val_soff)
    int val_soff;                 // FP64: element offset of the tap values (FP32: = tap_soff)
    int pad[2];
};

struct alignas(16) TileItem {     // one tile (or one part of it); carries what the kernel needs
    int o;
    int ty0, tx0;
    int batch_begin, batch_end;   // batches of the subband this item accumulates
    int geo;                      // the subband's tile side and thread map:
                                  // lgTS | e4 << 8 | sup << 9 (sup: a 2 x 2 super tile)
                                  // | nm << 12 (grouped items: the tile of subbands o .. o + nm - 1)
    int split;                    // part | nparts << 16 (nparts > 1: the tile's batches are split
                                  // over nparts items)
    int sid;                      // split tiles: index of the arrival counter and partial sums
#ifdef __CUDACC__
    __host__ __device__
#endif
    int lgTS() const { return geo & 0xff; }
#ifdef __CUDACC__
    __host__ __device__
#endif
    int TS() const { return 1 << (geo & 0xff); }
#ifdef __CUDACC__
    __host__ __device__
#endif
    int e4() const { return (geo >> 8) & 1; }
#ifdef __CUDACC__
    __host__ __device__
#endif
    int sup() const { return (geo >> 9) & 1; }
#ifdef __CUDACC__
    __host__ __device__
#endif
    int nm() const { return (geo >> 12) & 7; }
#ifdef __CUDACC__
    __host__ __device__
#endif
    int part() const { return split & 0xffff; }
#ifdef __CUDACC__
    __host__ __device__
#endif
    int nparts() const { return split >> 16; }
};

// One FP32 tap as the kernel reads it: offset and value in one 8-byte load.
struct alignas(8) TapOV {
    int off;
    float v;
};

// A pair's descriptor with its input subband's geometry (the per-batch shared-memory table
// of the kernel holds these).
struct alignas(16) PairSm {
    TilePair p;
    long long in_off;
    int in_rows, in_cols;
    int shift;        // vec pairs: staged column of the region's first column (0..3), set per tile
    int yb, xb;       // staged pairs: the region's first input row and column (wrapped), set per tile
    int pad;
};

struct TilePlanDev {
    const TilePair* pairs;
    const TileSub* subs;
    const TileBatch* batches;
    const TileItem* items;
    const PairSm* pair_sm;    // pairs with their input geometry (parallel to pairs)
    const int* tap_off;       // staged: offset in shared memory; global: (dy << 16) | (dx & 0xffff)
    const int* tap_lin;       // global pairs: dy * (input columns) + dx (interior fast path)
    const float* tap_v;
    const double* tap_v64;
    const TapOV* tap_ov;      // (tap_off, tap_v) interleaved: the FP32 kernels' tap records
    int n_sup;                // subbands tiled in super tiles (0: none)
    int n_grp;                // groups of subbands worked together (0: none)
    unsigned int* split_ctr;  // per split tile: parts finished (zero between launches)
    const long long* split_base;   // per split tile: first element of its partial sums
    void* split_buf;          // per split tile: nparts x TS^2 partial sums (element type of the plan)
    int n_items;
    int buf_elems;            // elements of one staging buffer (two buffers per CTA)
    int smem_bytes;           // dynamic shared memory per CTA
};

struct TilePlanHost {
    std::vector<TilePair> pairs;
    std::vector<TileSub> subs;
    std::vector<TileBatch> batches;
    std::vector<TileItem> items;
    std::vector<PairSm> pair_sm;
    std::vector<int> tap_off;
    std::vector<int> tap_lin;
    std::vector<float> tap_v;
    std::vector<double> tap_v64;
    std::vector<TapOV> tap_ov;
    std::vector<double> item_cost;   // estimated cost of every item (items are sorted by it)
    int esize = 4;                   // element size (4: FP32, 8: FP64)
    int n_sup = 0;                   // subbands tiled in super tiles
    int n_grp = 0;                   // groups of subbands worked together (grouped items)
    int n_split = 0;                 // split tiles
    std::vector<long long> split_base;   // first partial-sum element of each split tile
    long long split_elems = 0;       // partial-sum elements of all split tiles
    int buf_elems = 0;
    int smem_bytes = 0;
    long long macs = 0;        // MACs per application (taps x outputs, padding included)
};

struct TileEntry {             // one tap of one pair, in gather form
    int out, in, up, lg, phase, dy, dx;
    double v;
};

// Build the plan of one operator for element size `esize` and a per-buffer shared-memory
// budget (a batch of staged regions shares one buffer; a CTA holds two buffers); `ctas` is
// the number of CTAs that will share the tiles (it caps the cost of one tile). split_share >
// 0: a tile of several batches whose modelled cost exceeds split_share times one CTA's share
// is split at batch boundaries into parts that different CTAs run concurrently; the last
// part to finish sums the parts' partial sums in part order and runs the epilogue.
// super_tiles: subbands of 32-tiles whose pairs all fit one buffer for a 64-tile are worked
// in items of 2 x 2 tiles staged together (no split tiles then).
// grouped: the subbands of one level (A_J with the level-J details) are worked together: an
// item is one tile of every subband of the group, each input region is staged once for all
// of them (the union of their pairs' regions) and each member keeps its own taps (no split
// or super tiles then).
TilePlanHost make_tile_plan(const Layout& L, const std::vector<TileEntry>& entries, int esize, int smem_budget,
                            int ctas = 456, const std::vector<TileTune>* tune = nullptr, int level_only = 0,
                            double cap_share = 2.0, double split_share = 0.0, bool super_tiles = false,
                            bool grouped = false);

struct TileQueue {             // device counters of one operator launch
    unsigned int next;         // next work item
    unsigned int done;         // CTAs finished
};

struct TileArgs {
    TilePlanDev plan;
    const SubbandDev* sb;
    TileQueue* queue;
    int grid;
};

// One problem of a batched solve (device-resident descriptor).
struct BatchProblem {
    TilePlanDev fwd, adj;          // the problem's plans for Theta_K and Theta_K^T
    const SubbandDev* sb;
    float *y, *x, *r;              // iterates and residual (in place)
    const float* x0;
    const float* step_tab;         // tau / P per phase class
    const float* w_sb;             // weights per subband
    SolveState* st;
    double* sums;                  // [4] accumulated by the tiles: rr, <x0,r>, sum w|y|, max |g|/w
};

struct BatchItem {                 // tile `item` of problem p's plan (the plan of the phase)
    int p, item;
};

struct BatchArgs {
    const BatchProblem* probs;
    int B;
    const BatchItem* items;        // all problems' tiles of this phase, heaviest first
    int n_items;
    const int* n_items_dev;        // if set: the item count, read on the device (the host compacts
                                   // the list to the running problems between graph chunks)
    TileQueue* queue;
    int* running;                  // written by the last CTA of the step kernel
    int* run_flags;                // per problem: 1 while running (written with `running`)
    int grid;
    int buf_elems;                 // largest staging buffer of any problem's plan
    int smem_bytes;
    int grouped;                   // some problem's plans have grouped items (kernel instance)
};

int tile_batch_grid(int smem_bytes, bool grouped);
wdb_status batch_k1(const BatchArgs& B, cudaStream_t st);
wdb_status batch_k2(const BatchArgs& B, cudaStream_t st);
// x -> sums[0] = ||Theta_K x - x0||^2, sums[1] = sum w|x| for every problem
wdb_status batch_objective(const BatchArgs& B, cudaStream_t st);

template <typename T>
wdb_status tile_apply(const TileArgs& A, const T* in, T* out, const double* scale, double* norm_out,
                      double* part, cudaStream_t st);
// pdl: launch as a programmatic dependent of the previous kernel in the stream (the FISTA
// loop's K1 / K2 alternation)
wdb_status tile_k1(const TileArgs& A, const float* y, const float* x0, float* r, double* part, SolveState* s,
                   cudaStream_t st, bool pdl = false);
wdb_status tile_k2(const TileArgs& A, const float* r, float* y, float* x, const float* step_tab,
                   const float* w_sb, double* part, SolveState* s, cudaStream_t st, bool pdl = false);
wdb_status tile_resnorm(const TileArgs& A, const float* x, const float* x0, float* r, double* out, double* part,
                        cudaStream_t st);
// Fused FISTA loop: `iters` iterations of kernel 1 (plan F) and kernel 2 (plan A) in one
// cooperative launch of the resident CTAs (at most max_ctas: `part` holds 2 doubles per CTA),
// the passes separated by grid barriers whose waits poll at most spin_limit times (<= 0:
// 2^23) before recording a timeout in the state. Stops early when the state says stop. Plans
// with split tiles are not supported (WDB_EINVAL).
bool tile_fused_supported(const TileArgs& F, const TileArgs& A);
wdb_status tile_fused(const TileArgs& F, const TileArgs& A, float* y, const float* x0, float* r, float* x,
                      const float* step_tab, const float* w_sb, double* part, SolveState* s, int iters,
                      long long spin_limit, int max_ctas, cudaStream_t st);
int tile_grid(int smem_bytes);

}  // namespace wdb
