// Tiled gather engine for Theta_K / Theta_K^T (see tile.cuh) and the fused FISTA kernels
// built on it: kernel 1 (r = Theta_K y - x0 with FP64 totals of ||r||^2 and <x0, r>) and
// kernel 2 (g = Theta_K^T r fused with the preconditioned step, soft threshold and momentum
// of Algorithm 3, with FP64 totals of sum w|y| and max |g|/w).
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <map>
#include <tuple>

#include "device_util.cuh"
#include "tile.cuh"

namespace wdb {

// ---------------------------------------------------------------------------------------
// Host: plan
// ---------------------------------------------------------------------------------------
namespace {

struct PairBuild {
    int out, in, up, lg;
    int dy0 = 1 << 30, dy1 = -(1 << 30), dx0 = 1 << 30, dx1 = -(1 << 30);
    std::vector<const TileEntry*> taps;
    int maxph = 0;     // taps applied per output: all taps (down), the fullest phase (up); grouped
                       // pairs: summed over the members
    int nm = 1;        // grouped pairs: members (output subbands of the group)
    std::vector<const TileEntry*> mtaps[4];   // grouped pairs: the taps of each member
    int mmaxph[4] = {0, 0, 0, 0};
};

// First subband of the group of subband o (grouped plans): A_J and the three details of level
// J form one group, the three details of every finer level another.
int group_first(const Layout& L, int o) { return o < 4 ? 0 : 1 + 3 * ((o - 1) / 3); }

// Cost model of one tile, in thread instructions (used to choose the tile side and, per
// pair, staging against gathering from global memory / L2).
constexpr double kCostStage = 8.0;       // per staged input element (cp.async, wrap, index)
constexpr double kCostTapStage = 6.0;    // per staged tap (offset + value)
constexpr double kCostMacGlobal = 60.0;  // per multiply-add gathered from global memory (latency bound)
constexpr double kCostItem = 20000.0;    // per tile (scheduling, descriptors, barriers, epilogue)
constexpr double kCostBatch = 6000.0;    // per batch (staging round trip, barriers)
constexpr int kUpStagedLg = 3;           // up pairs with r <= 8 always stage their phase tables

// Up pairs stage their phase tables (r^2 phases x the fullest phase's taps) with the batch when
// r <= 8, or when the table takes at most half of the staging buffer; larger tables are read
// from global memory.
bool tables_staged(int lg, int maxph, int esize, int budget) {
    return lg <= kUpStagedLg || ((long long)maxph << (2 * lg)) * (4 + esize) <= budget / 2;
}

int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

struct Geometry {
    int RR, RC, PR, PC, PS;
    long long bytes;
};

// Row pitch of a staged region. With 4 outputs per thread (TS >= 8) the threads of one warp
// read TS / 4 consecutive words in each of 128 / TS rows, so a pitch congruent to TS / 4
// modulo TS / 2 puts the rows on disjoint banks; one output per thread: an odd pitch.
int pitch(int width, int TS, bool e4) {
    if (TS < 8 || !e4) return width | 1;
    const int lanes = TS / 4;
    int p = width;
    while (p % (2 * lanes) != lanes) ++p;
    return p;
}

// Rows of an up pair or an r = 1 down pair can be staged in 16-byte chunks starting at the
// 4-aligned column at or before the region's first column (16- or 32-wide tiles with the
// 4-output map, whose pitches are multiples of 4, and inputs whose rows are 4-aligned).
bool vec_pair(const PairBuild& p, const Layout& L, int TS, bool e4, int esize) {
    const SubbandDev& si = L.sb[p.in];
    return esize == 4 && e4 && TS >= 16 && (p.up || p.lg == 0) && si.cols % 4 == 0 && si.off % 4 == 0;
}

// Region of pair p for a staged tile of side TS; the row pitch suits the thread map of tiles
// of side pts (<= 0: TS; super tiles stage 2 x 2 tiles of side pts = TS / 2 together).
Geometry geometry(const PairBuild& p, int TS, int esize, bool e4, bool vec = false, int pts = 0) {
    Geometry g;
    const int r = 1 << p.lg;
    const int PT = pts > 0 ? pts : TS;
    if (!p.up) {
        g.RR = r * (TS - 1) + (p.dy1 - p.dy0) + 1;
        g.RC = r * (TS - 1) + (p.dx1 - p.dx0) + 1;
        g.PR = (g.RR + r - 1) / r;
        g.PC = pitch(vec ? (g.RC + 6) & ~3 : (g.RC + r - 1) / r, PT, e4);
        g.PS = g.PR * g.PC;
        g.bytes = (long long)r * r * g.PS * esize;
    } else {
        const int rows = std::max(1, TS >> p.lg);
        g.RR = rows + (p.dy1 - p.dy0);
        g.RC = rows + (p.dx1 - p.dx0);
        g.PR = g.RR;
        g.PC = pitch(vec ? (g.RC + 6) & ~3 : g.RC, PT, e4);
        g.PS = g.PR * g.PC;
        g.bytes = (long long)g.PR * g.PC * esize;
    }
    return g;
}


// Modelled cost per output of subband o's tiles of side ts; glob[k] receives the cheaper
// mode of pair k (true: gather from global memory).
double subband_cost(const SubbandDev& so, const std::vector<PairBuild*>& prs, int ts, bool e4, int esize, int budget,
                    std::vector<bool>& glob) {
    const double outs = (double)std::min(ts, so.rows) * std::min(ts, so.cols);
    const double mac_smem = e4 ? 2.75 : 5.0;
    double c = kCostItem;
    glob.assign(prs.size(), false);
    for (size_t k = 0; k < prs.size(); ++k) {
        const PairBuild& pb = *prs[k];
        const Geometry g = geometry(pb, ts, esize, e4);
        const double macs = outs * pb.maxph;
        double cs = 1e300;
        if (g.bytes <= budget)
            cs = (double)g.RR * g.RC * kCostStage + macs * mac_smem +
                 kCostTapStage * (double)(!pb.up ? (int)pb.taps.size()
                                                 : (tables_staged(pb.lg, pb.maxph, esize, budget) ? pb.maxph << (2 * pb.lg) : 0));
        const double cg = macs * kCostMacGlobal;
        glob[k] = cg < cs;
        c += std::min(cs, cg);
    }
    return c / outs;
}

}  // namespace

TilePlanHost make_tile_plan(const Layout& L, const std::vector<TileEntry>& entries, int esize, int budget, int ctas,
                            const std::vector<TileTune>* tune, int level_only, double cap_share, double split_share,
                            bool super_tiles, bool grouped) {
    if (super_tiles) split_share = 0.0;   // a plan has split tiles or super tiles, not both
    if (grouped) {   // a plan has grouped items, or split or super tiles
        super_tiles = false;
        split_share = 0.0;
    }
    TilePlanHost plan;
    plan.esize = esize;
    std::map<std::pair<int, int>, PairBuild> pairs;
    for (const TileEntry& e : entries) {
        const int u = grouped ? group_first(L, e.out) : e.out;
        PairBuild& p = pairs[{u, e.in}];
        p.out = u;
        p.in = e.in;
        p.up = e.up;
        p.lg = e.lg;
        p.dy0 = std::min(p.dy0, e.dy);
        p.dy1 = std::max(p.dy1, e.dy);
        p.dx0 = std::min(p.dx0, e.dx);
        p.dx1 = std::max(p.dx1, e.dx);
        p.taps.push_back(&e);
        if (grouped) p.mtaps[e.out - u].push_back(&e);
    }
    // units of work: every subband, or (grouped) the first subband of every group
    std::vector<int> unit_nm(L.S, 0);
    for (int o = 0; o < L.S; ++o) {
        const int u = grouped ? group_first(L, o) : o;
        unit_nm[u] = std::max(unit_nm[u], o - u + 1);
    }
    std::vector<std::vector<PairBuild*>> by_out(L.S);
    for (auto& kv : pairs) by_out[kv.first.first].push_back(&kv.second);
    plan.subs.resize(L.S);
    int max_bytes = 0;
    struct ItemCost {
        TileItem it;
        double cost;
    };
    std::vector<ItemCost> items;
    std::vector<std::vector<double>> sub_bcost(L.S);
    for (int o = 0; o < L.S; ++o)
        for (PairBuild* pb : by_out[o]) {
            auto maxph_of = [&](const std::vector<const TileEntry*>& tl) {
                if (!pb->up) return (int)tl.size();
                std::vector<int> cnt(1 << (2 * pb->lg), 0);
                for (const TileEntry* e : tl) cnt[e->phase]++;
                return *std::max_element(cnt.begin(), cnt.end());
            };
            if (!grouped) {
                pb->maxph = maxph_of(pb->taps);
            } else {
                pb->nm = unit_nm[o];
                pb->maxph = 0;
                for (int k = 0; k < pb->nm; ++k) {
                    pb->mmaxph[k] = maxph_of(pb->mtaps[k]);
                    pb->maxph += pb->mmaxph[k];
                }
            }
        }
    // balance: the whole operator's modelled cost (each subband at its cheapest tile side)
    // shared by `ctas` CTAs bounds the cost of one tile, so that no tile is the critical path
    std::vector<int> ts_max(L.S);
    double total = 0.0;
    {
        std::vector<bool> tmp;
        for (int o = 0; o < L.S; ++o) {
            const SubbandDev& so = L.sb[o];
            ts_max[o] = std::min(32, next_pow2(std::max(so.rows, so.cols)));
            if (grouped && group_first(L, o) != o) continue;   // counted with the group's first
            double bc = 1e300;
            for (int ts = ts_max[o]; ts >= 1; ts >>= 1)
                bc = std::min(bc, subband_cost(so, by_out[o], ts, ts >= 8, esize, budget, tmp));
            total += bc * so.rows * so.cols;
        }
    }
    // (a tile's fixed cost makes tiles cheaper than ~16 of it wasteful, so the cap never
    // goes below that: small operators accept some imbalance)
    const double item_cap = std::max(cap_share * total / std::max(1, ctas), 16.0 * kCostItem);
    for (int o = 0; o < L.S; ++o) {
        if (grouped && group_first(L, o) != o) continue;   // worked by the group's items
        const SubbandDev& so = L.sb[o];
        // tile side and per-pair mode (staged in shared memory or gathered from global
        // memory) that minimise the modelled cost per output, among the sides whose tiles
        // stay under the balance cap (else the side with the cheapest tile); a staged region
        // must fit one buffer
        const int np = (int)by_out[o].size();
        std::vector<bool> global, trial;
        int TS = 0;
        bool e4 = false;
        double best = 1e300, best_item = 1e300;
        if (tune && (*tune)[o].ts > 0) {   // forced by the autotuner
            TS = std::min((*tune)[o].ts, ts_max[o]);
            e4 = TS == 32 || (TS >= 8 && (*tune)[o].e4);
            best = subband_cost(so, by_out[o], TS, e4, esize, budget, global);
        } else {
            for (int ts = ts_max[o]; ts >= 1; ts >>= 1) {
                const double c = subband_cost(so, by_out[o], ts, ts >= 8, esize, budget, trial);
                const double item = c * std::min(ts, so.rows) * std::min(ts, so.cols);
                const bool ok = item <= item_cap, best_ok = best_item <= item_cap;
                if (TS == 0 || (ok && (!best_ok || c < best)) || (!ok && !best_ok && item < best_item)) {
                    TS = ts;
                    best = c;
                    best_item = item;
                    global = trial;
                }
            }
            e4 = TS >= 8;
        }
        // pairs whose rows are staged in 16-byte chunks (when their wider region still fits)
        std::vector<bool> vecf(np, false);
        for (int k = 0; k < np; ++k)
            vecf[k] = !global[k] && vec_pair(*by_out[o][k], L, TS, e4, esize) &&
                      geometry(*by_out[o][k], TS, esize, e4, true).bytes <= budget;
        // super tiles: 2 x 2 tiles of side 32 staged together in one batch (every pair staged,
        // all regions in one buffer) and computed one after the other, so that the set-up of
        // a work item and of its pairs' staging serves four tiles
        int ST = TS;   // side of the staged tile
        bool sup = false;
        if (super_tiles && TS == 32 && e4 && so.rows >= 64 && so.cols >= 64 && np <= kMaxBatchPairs) {
            bool ok = true;
            long long regs = 0, ntaps = 0;
            for (int k = 0; k < np && ok; ++k) {
                const PairBuild& pb = *by_out[o][k];
                if (global[k]) ok = false;
                const Geometry g = geometry(pb, 64, esize, e4, vecf[k], 32);
                regs += (g.bytes + 15) / 16 * 16 / esize;
                ntaps += !pb.up ? (long long)pb.taps.size()
                                : (tables_staged(pb.lg, pb.maxph, esize, budget) ? (long long)pb.maxph << (2 * pb.lg) : 0);
            }
            const long long tapel = (ntaps * (4 + esize) + 15) / 16 * 16 / esize;
            if (ok && regs + tapel <= budget / esize) {
                sup = true;
                ST = 64;
            }
        }
        // staged down pairs, staged up pairs (in batches that fill a buffer), then the global
        // ones; within a batch the staged taps (down pairs only) are contiguous
        std::vector<int> order;
        for (int k = 0; k < np; ++k)
            if (!global[k] && !by_out[o][k]->up) order.push_back(k);
        auto tst = [&](int k) { return tables_staged(by_out[o][k]->lg, by_out[o][k]->maxph, esize, budget); };
        for (int k = 0; k < np; ++k)
            if (!global[k] && by_out[o][k]->up && tst(k)) order.push_back(k);
        for (int k = 0; k < np; ++k)
            if (!global[k] && by_out[o][k]->up && !tst(k)) order.push_back(k);
        for (int k = 0; k < np; ++k)
            if (global[k]) order.push_back(k);
        TileSub& sub = plan.subs[o];
        sub.TS = TS;
        sub.e4 = e4 ? 1 : 0;
        sub.pair_begin = (int)plan.pairs.size();
        sub.batch_begin = sub.batch_end = 0;
        // (batches are filled in below)
        double taps_per_out = 0.0;
        // first pass: geometry and batch membership (regions plus their taps must fit)
        const int ebudget = budget / esize;
        std::vector<int> batch_of(order.size()), pair_soff(order.size(), 0);
        std::vector<int> batch_regions(1, 0), batch_taps(1, 0), batch_count(1, 0);
        for (size_t q = 0; q < order.size(); ++q) {
            const int k = order[q];
            if (global[k]) {   // global pairs join the last batch while it has room
                if (batch_count.back() >= kMaxBatchPairs) {
                    batch_regions.push_back(0);
                    batch_taps.push_back(0);
                    batch_count.push_back(0);
                }
                batch_count.back() += 1;
                batch_of[q] = (int)batch_regions.size() - 1;
                continue;
            }
            const PairBuild& pb = *by_out[o][k];
            const Geometry g = geometry(pb, ST, esize, e4, vecf[k], TS);
            const int need = (int)((g.bytes + 15) / 16 * 16 / esize);
            // staged taps: down pairs and up pairs with r <= 8 (larger phase tables are read
            // from global memory)
            const int nt = !pb.up ? (int)pb.taps.size()
                                  : (tables_staged(pb.lg, pb.maxph, esize, budget) ? pb.maxph << (2 * pb.lg) : 0);
            // taps: one int offset + one value each, rounded to 16 bytes
            auto tap_elems = [&](int ntaps) { return (int)(((long long)ntaps * (4 + esize) + 15) / 16 * 16 / esize); };
            const bool nonempty = batch_regions.back() > 0;
            if (nonempty && (batch_regions.back() + need + tap_elems(batch_taps.back() + nt) > ebudget ||
                             batch_count.back() >= kMaxBatchPairs)) {
                batch_regions.push_back(0);
                batch_taps.push_back(0);
                batch_count.push_back(0);
            }
            batch_count.back() += 1;
            batch_of[q] = (int)batch_regions.size() - 1;
            pair_soff[q] = batch_regions.back();
            batch_regions.back() += need;
            batch_taps.back() += nt;
        }
        // modelled cost of each batch for a full tile (splitting tiles at batch boundaries)
        {
            const double outs_full = (double)std::min(TS, so.rows) * std::min(TS, so.cols);
            const double mac_smem = e4 ? 2.75 : 5.0;
            std::vector<double>& bc = sub_bcost[o];
            bc.assign(batch_regions.size(), kCostBatch);
            for (size_t q = 0; q < order.size(); ++q) {
                const PairBuild& pb = *by_out[o][order[q]];
                const double macs = outs_full * pb.maxph;
                double c = macs * kCostMacGlobal;
                if (!global[order[q]]) {
                    const Geometry g = geometry(pb, ST, esize, e4, vecf[order[q]], TS);
                    const int nt = !pb.up ? (int)pb.taps.size()
                                          : (tables_staged(pb.lg, pb.maxph, esize, budget) ? pb.maxph << (2 * pb.lg) : 0);
                    c = (double)g.RR * g.RC * kCostStage + macs * mac_smem + kCostTapStage * nt;
                }
                bc[batch_of[q]] += c;
            }
        }
        sub.batch_begin = (int)plan.batches.size();
        for (size_t bi = 0; bi < batch_regions.size(); ++bi) {
            TileBatch bt{};
            bt.pair_begin = bt.pair_end = (int)plan.pairs.size();
            plan.batches.push_back(bt);
        }
        for (size_t q = 0; q < order.size(); ++q) {
            const int k = order[q];
            const PairBuild& pb = *by_out[o][k];
            const Geometry g = geometry(pb, ST, esize, e4, vecf[k], TS);
            const int r = 1 << pb.lg, m = r - 1;
            TileBatch& bt = plan.batches[sub.batch_begin + batch_of[q]];
            if (bt.pair_end == bt.pair_begin) {
                bt.pair_begin = bt.pair_end = (int)plan.pairs.size();
                bt.tap_begin = bt.tap_end = (int)plan.tap_off.size();
            }
            TilePair tp;
            tp.in_sb = pb.in;
            tp.lg = pb.lg;
            tp.mode = pb.up ? (global[k] ? kUpGlobal : kUp) : (global[k] ? kDownGlobal : kDown);
            tp.RR = g.RR;
            tp.RC = g.RC;
            tp.PR = g.PR;
            tp.PC = g.PC;
            tp.PS = g.PS;
            tp.y0 = pb.dy0;
            tp.x0 = pb.dx0;
            tp.vec = vecf[k] ? 1 : 0;
            tp.tst = (pb.up && !global[k] && tables_staged(pb.lg, pb.maxph, esize, budget)) ? 1 : 0;
            if (global[k]) {   // bounding box of the taps (input units) for the interior test
                tp.RR = pb.dy1 - pb.dy0 + 1;
                tp.RC = pb.dx1 - pb.dx0 + 1;
                tp.PR = tp.PC = tp.PS = 0;
            }
            tp.soff = global[k] ? 0 : pair_soff[q];
            tp.tap_begin = (int)plan.tap_off.size();
            const int cin = L.sb[pb.in].cols;
            auto offset = [&](const TileEntry& e) -> int {
                if (global[k]) return (e.dy << 16) | (e.dx & 0xffff);
                if (!pb.up) {
                    const int yy = e.dy - pb.dy0, xx = e.dx - pb.dx0;
                    const int plane = ((yy & m) << pb.lg) + (xx & m);
                    return plane * g.PS + (yy >> pb.lg) * g.PC + (xx >> pb.lg) + tp.soff;
                }
                return (e.dy - pb.dy0) * g.PC + (e.dx - pb.dx0) + tp.soff;
            };
            // taps member by member (one member unless the plan is grouped): down pairs
            // their list, up pairs their phase table padded to the member's fullest phase
            tp.nm = pb.nm;
            for (int mk = 0; mk < 4; ++mk) tp.mtb[mk] = tp.mnt[mk] = 0;
            int per_out = 0;
            for (int mk = 0; mk < pb.nm; ++mk) {
                const std::vector<const TileEntry*>& tl = grouped ? pb.mtaps[mk] : pb.taps;
                tp.mtb[mk] = (int)plan.tap_off.size();
                if (!pb.up) {
                    tp.mnt[mk] = (int)tl.size();
                    for (const TileEntry* e : tl) {
                        plan.tap_off.push_back(offset(*e));
                        plan.tap_lin.push_back(global[k] ? e->dy * cin + e->dx : 0);
                        plan.tap_v.push_back((float)e->v);
                        plan.tap_v64.push_back(e->v);
                    }
                } else {
                    const int nph = r * r;
                    std::vector<std::vector<const TileEntry*>> ph(nph);
                    for (const TileEntry* e : tl) ph[e->phase].push_back(e);
                    int mx = 0;
                    for (auto& v : ph) mx = std::max(mx, (int)v.size());
                    tp.mnt[mk] = mx;
                    for (int j = 0; j < mx; ++j)
                        for (int qq = 0; qq < nph; ++qq) {
                            if (j < (int)ph[qq].size()) {
                                plan.tap_off.push_back(offset(*ph[qq][j]));
                                plan.tap_lin.push_back(global[k] ? ph[qq][j]->dy * cin + ph[qq][j]->dx : 0);
                                plan.tap_v.push_back((float)ph[qq][j]->v);
                                plan.tap_v64.push_back(ph[qq][j]->v);
                            } else {
                                // padding: value 0 at the region origin (staged) or the
                                // output's own input position (global)
                                plan.tap_off.push_back(global[k] ? 0 : tp.soff);
                                plan.tap_lin.push_back(0);
                                plan.tap_v.push_back(0.f);
                                plan.tap_v64.push_back(0.0);
                            }
                        }
                }
                per_out += tp.mnt[mk];
            }
            tp.ntap = tp.mnt[0];
            taps_per_out += per_out;
            plan.pairs.push_back(tp);
            bt.pair_end = (int)plan.pairs.size();
            if (!global[k] && (!pb.up || tp.tst)) bt.tap_end = (int)plan.tap_off.size();
        }
        // tap copies follow the regions of each batch in the buffer
        for (int bi = sub.batch_begin; bi < (int)plan.batches.size(); ++bi) {
            TileBatch& bt = plan.batches[bi];
            if (bt.tap_end < bt.tap_begin) bt.tap_end = bt.tap_begin;
            const int nt = bt.tap_end - bt.tap_begin;
            const int reg = batch_regions[bi - sub.batch_begin];
            bt.tap_soff = reg * esize / 4;   // in ints (regions are whole 16-byte chunks)
            int total;
            if (esize == 4) {                // (offset, value) records
                bt.val_soff = bt.tap_soff;
                total = bt.tap_soff * 4 + nt * (int)sizeof(TapOV);
            } else {                         // offsets, then the values
                bt.val_soff = (int)(((long long)(bt.tap_soff + nt) * 4 + esize - 1) / esize);   // in T
                total = (bt.val_soff + nt) * esize;
            }
            max_bytes = std::max(max_bytes, (total + 15) / 16 * 16);
        }
        sub.pair_end = (int)plan.pairs.size();
        sub.batch_end = (int)plan.batches.size();
        sub.sup = sup ? 1 : 0;
        sub.lgTS = 0;
        while ((1 << sub.lgTS) < TS) ++sub.lgTS;
        const int ty = (so.rows + ST - 1) / ST, tx = (so.cols + ST - 1) / ST;
        for (int a = 0; a < ty; ++a)
            for (int b = 0; b < tx; ++b) {
                const int vy = std::min(ST, so.rows - a * ST), vx = std::min(ST, so.cols - b * ST);
                const double outs = (double)vy * vx;
                // MACs per thread-slot plus staging; small tiles leave threads in groups (a super
                // tile pays the per-tile cost once for its four tiles)
                const double cost = best * outs - (sup ? 0.75 * kCostItem * outs / (TS * TS) : 0.0);
                plan.macs += (long long)(outs * taps_per_out);
                if (level_only <= 0 || so.level == level_only)
                    items.push_back({TileItem{o, a * ST, b * ST, sub.batch_begin, sub.batch_end,
                                              sub.lgTS | (sub.e4 << 8) | (sub.sup << 9) |
                                                  (grouped ? unit_nm[o] << 12 : 0),
                                              1 << 16, -1},
                                     cost});
            }
        plan.n_sup += sup ? 1 : 0;
        if (grouped) {   // the group's other subbands share its tiles, pairs and batches
            sub.grp = unit_nm[o];
            for (int k = 1; k < unit_nm[o]; ++k) plan.subs[o + k] = sub;
            plan.n_grp += 1;
        }
    }
    if (split_share > 0.0 && !items.empty()) {
        // split the tiles that would dominate one CTA's share into parts of whole batches
        double sum = 0.0;
        for (const ItemCost& ic : items) sum += ic.cost;
        const double thr = std::max(split_share * sum / std::max(1, ctas), 2.0 * kCostItem);
        std::vector<ItemCost> out;
        for (const ItemCost& ic : items) {
            const TileItem& w = ic.it;
            const int nb = w.batch_end - w.batch_begin;
            const int np = std::min(nb, (int)std::ceil(ic.cost / thr));
            if (np < 2) {
                out.push_back(ic);
                continue;
            }
            const SubbandDev& so = L.sb[w.o];
            const int TS = w.TS();
            const double f = (double)std::min(TS, so.rows - w.ty0) * std::min(TS, so.cols - w.tx0) /
                             ((double)std::min(TS, so.rows) * std::min(TS, so.cols));
            const std::vector<double>& bc = sub_bcost[w.o];
            const int b0 = w.batch_begin - plan.subs[w.o].batch_begin;
            double tot = 0.0;
            for (int b = 0; b < nb; ++b) tot += bc[b0 + b];
            // contiguous parts: cut where the running cost passes the next multiple of tot / np,
            // leaving at least one batch for every later part
            int begin = 0, part = 0;
            double run = 0.0;
            const int sid = plan.n_split++;
            plan.split_base.push_back(plan.split_elems);
            plan.split_elems += (long long)np * TS * TS;
            for (int b = 0; b < nb; ++b) {
                run += bc[b0 + b];
                const bool last = b == nb - 1;
                const bool cut = !last && part < np - 1 &&
                                 (run >= tot * (part + 1) / np || nb - (b + 1) == np - (part + 1));
                if (cut || last) {
                    double c = kCostItem;
                    for (int k = begin; k <= b; ++k) c += bc[b0 + k];
                    TileItem pw = w;
                    pw.batch_begin = w.batch_begin + begin;
                    pw.batch_end = w.batch_begin + b + 1;
                    pw.split = part | (np << 16);
                    pw.sid = sid;
                    out.push_back({pw, c * f});
                    ++part;
                    begin = b + 1;
                }
            }
        }
        items.swap(out);
    }
    std::stable_sort(items.begin(), items.end(), [](const ItemCost& x, const ItemCost& y) { return x.cost > y.cost; });
    for (auto& ic : items) {
        plan.items.push_back(ic.it);
        plan.item_cost.push_back(ic.cost);
    }
    plan.tap_ov.resize(plan.tap_off.size());
    for (size_t k = 0; k < plan.tap_off.size(); ++k) plan.tap_ov[k] = TapOV{plan.tap_off[k], plan.tap_v[k]};
    plan.pair_sm.resize(plan.pairs.size());
    for (size_t k = 0; k < plan.pairs.size(); ++k) {
        const SubbandDev& si = L.sb[plan.pairs[k].in_sb];
        plan.pair_sm[k] = PairSm{plan.pairs[k], si.off, si.rows, si.cols, 0, 0, 0, 0};
    }
    plan.buf_elems = std::max(max_bytes, 16) / esize;
    plan.smem_bytes = 2 * plan.buf_elems * esize;
    return plan;
}

// ---------------------------------------------------------------------------------------
// Device
// ---------------------------------------------------------------------------------------
namespace {

enum Epi { kApply = 0, kApplyNorm = 1, kK1 = 2, kK2 = 3, kResNorm = 4, kObj = 5 };

struct EpiArgs {
    const float* x0;          // kK1, kResNorm, kObj
    float* y;                 // kK2 (in place)
    float* x;                 // kK2 (in place)
    const float* step_tab;    // kK2: tau / P per phase class
    const float* w_sb;        // kK2, kObj: weights per subband
    const double* scale;      // kApply*: optional factor per phase class
    double* part;             // per-CTA partials
    SolveState* st;           // kK1, kK2
    double* red_out;          // kApplyNorm, kResNorm
};

template <typename T>
__device__ __forceinline__ const T* tvals(const TilePlanDev& p);
template <>
__device__ __forceinline__ const float* tvals<float>(const TilePlanDev& p) { return p.tap_v; }
template <>
__device__ __forceinline__ const double* tvals<double>(const TilePlanDev& p) { return p.tap_v64; }

// Taps of a batch as the inner loops read them: FP32 from (offset, value) records (one 8-byte
// load), FP64 from the separate offset and value arrays.
template <typename T>
struct TapSrc;
template <>
struct TapSrc<float> {
    const TapOV* ov;
    __device__ __forceinline__ void get(int j, int& o, float& v) const {
        const TapOV q = ov[j];
        o = q.off;
        v = q.v;
    }
    __device__ __forceinline__ TapSrc operator+(int k) const { return TapSrc{ov + k}; }
};
template <>
struct TapSrc<double> {
    const int* to;
    const double* tv;
    __device__ __forceinline__ void get(int j, int& o, double& v) const {
        o = to[j];
        v = tv[j];
    }
    __device__ __forceinline__ TapSrc operator+(int k) const { return TapSrc{to + k, tv + k}; }
};

// The batch's staged taps, indexed by plan tap index.
template <typename T>
__device__ __forceinline__ TapSrc<T> staged_taps(const T* S, const TileBatch& bt);
template <>
__device__ __forceinline__ TapSrc<float> staged_taps<float>(const float* S, const TileBatch& bt) {
    return TapSrc<float>{reinterpret_cast<const TapOV*>(reinterpret_cast<const int*>(S) + bt.tap_soff) - bt.tap_begin};
}
template <>
__device__ __forceinline__ TapSrc<double> staged_taps<double>(const double* S, const TileBatch& bt) {
    return TapSrc<double>{reinterpret_cast<const int*>(S) + bt.tap_soff - bt.tap_begin, S + bt.val_soff - bt.tap_begin};
}

// The plan's taps in global memory.
template <typename T>
__device__ __forceinline__ TapSrc<T> global_taps(const TilePlanDev& p);
template <>
__device__ __forceinline__ TapSrc<float> global_taps<float>(const TilePlanDev& p) {
    return TapSrc<float>{p.tap_ov};
}
template <>
__device__ __forceinline__ TapSrc<double> global_taps<double>(const TilePlanDev& p) {
    return TapSrc<double>{p.tap_off, p.tap_v64};
}

__device__ __forceinline__ int wrap1(int v, int n) {
    v += (v < 0) ? n : 0;
    return v - ((v >= n) ? n : 0);
}

// v mod n for v within a few periods of [0, n) (region origins): no integer division
__device__ __forceinline__ int pos_mod(int v, int n) {
    while (v < 0) v += n;
    while (v >= n) v -= n;
    return v;
}

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
template <int B>
__device__ __forceinline__ void cp_async_to(unsigned s, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Issue the asynchronous copies of batch `bi` of tile `w` into buffer S: every staged region
// (one warp per row, lanes along the row, periodic wrap) and the batch's taps. Lane l copies
// the row's columns xr = l + 32k; for a down pair (r = 2^lg <= 32) its polyphase destination
// is then (l & m) * plane + (l >> lg) + k * (32 >> lg): one constant per lane plus a fixed
// step, so the inner loop is one copy and three additions.
// The batch's pair table `tab` is filled first (one thread per pair, then a barrier that
// every thread of the CTA reaches).
template <typename T>
__device__ __forceinline__ void stage_batch(const TilePlanDev& plan, const T* __restrict__ in, const TileItem& w,
                                            int bi, T* S, PairSm* tab) {
    const TileBatch bt = plan.batches[bi];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = kTileThreads / 32;
    constexpr unsigned ES = sizeof(T);
    const unsigned S0 = smem_addr(S);
    const int np = bt.pair_end - bt.pair_begin;
    if ((int)threadIdx.x < np) {
        // this tile's region origin, wrapped once here for every warp that stages the pair;
        // vec pairs start at staged column (first column mod 4)
        PairSm e = plan.pair_sm[bt.pair_begin + threadIdx.x];
        const bool dn = e.p.mode == kDown || e.p.mode == kDownGlobal;
        const int Y0 = dn ? ((w.ty0 << e.p.lg) + e.p.y0) : ((w.ty0 >> e.p.lg) + e.p.y0);
        const int X0 = dn ? ((w.tx0 << e.p.lg) + e.p.x0) : ((w.tx0 >> e.p.lg) + e.p.x0);
        if (e.p.mode == kDown || e.p.mode == kUp) {
            e.yb = pos_mod(Y0, e.in_rows);
            e.xb = pos_mod(X0, e.in_cols);
            if (e.p.vec) e.shift = e.xb & 3;
        }
        tab[threadIdx.x] = e;
    }
    __syncthreads();
    // 16-byte copies need a 16-byte aligned input vector (the library's own buffers are)
    const bool in_aligned = (reinterpret_cast<unsigned long long>(in) & 15) == 0;
    for (int i = 0; i < np; ++i) {
        const TilePair P = tab[i].p;
        if (P.mode != kDown && P.mode != kUp) break;   // global pairs come last in a subband
        const SubbandDev si{tab[i].in_off, tab[i].in_rows, tab[i].in_cols, 0, 0, 0, 0};
        const T* __restrict__ src = in + si.off;
        const int lg = P.lg, m = (1 << lg) - 1;
        const bool down = P.mode == kDown;
        const int yb = tab[i].yb, xb = tab[i].xb;
        const int plane = P.PS;
        const unsigned base = S0 + (unsigned)P.soff * ES;
        if (P.vec) {
            // rows of RCv = roundup4(RC + 3) columns starting at the 4-aligned column xb & ~3;
            // input rows are 4-aligned and a chunk never straddles the periodic wrap
            const int xa = xb & ~3, RCv = (P.RC + 6) & ~3;
            for (int yr = warp; yr < P.RR; yr += NW) {
                int gy = yb + yr;
                while (gy >= si.rows) gy -= si.rows;
                const T* __restrict__ row = src + (size_t)gy * si.cols;
                const unsigned drow = base + (unsigned)(yr * P.PC) * ES;
                if (in_aligned) {
                    for (int c = lane; 4 * c < RCv; c += 32) {
                        int gx = xa + 4 * c;
                        while (gx >= si.cols) gx -= si.cols;
                        cp_async_to<16>(drow + 16u * c, row + gx);
                    }
                } else {
                    for (int xr = lane; xr < RCv; xr += 32) {
                        int gx = xa + xr;
                        while (gx >= si.cols) gx -= si.cols;
                        cp_async_to<ES>(drow + (unsigned)xr * ES, row + gx);
                    }
                }
            }
        } else if (!down || lg <= 5) {
            const int colc = down ? ((lane & m) * plane + (lane >> lg)) : lane;
            const unsigned step = (unsigned)(down ? (32 >> lg) : 32) * ES;
            for (int yr = warp; yr < P.RR; yr += NW) {
                int gy = yb + yr;
                while (gy >= si.rows) gy -= si.rows;
                const T* __restrict__ row = src + (size_t)gy * si.cols;
                const int rowoff = down ? (((yr & m) << lg) * plane + (yr >> lg) * P.PC) : yr * P.PC;
                unsigned d = base + (unsigned)(rowoff + colc) * ES;
                int gx = xb + lane;
                while (gx >= si.cols) gx -= si.cols;
                for (int xr = lane; xr < P.RC; xr += 32) {
                    cp_async_to<ES>(d, row + gx);
                    d += step;
                    gx += 32;
                    while (gx >= si.cols) gx -= si.cols;
                }
            }
        } else {
            for (int yr = warp; yr < P.RR; yr += NW) {
                int gy = yb + yr;
                while (gy >= si.rows) gy -= si.rows;
                const T* __restrict__ row = src + (size_t)gy * si.cols;
                const int rowoff = ((yr & m) << lg) * plane + (yr >> lg) * P.PC;
                int gx = xb + lane;
                while (gx >= si.cols) gx -= si.cols;
                for (int xr = lane; xr < P.RC; xr += 32) {
                    cp_async_to<ES>(base + (unsigned)(rowoff + (xr & m) * plane + (xr >> lg)) * ES, row + gx);
                    gx += 32;
                    while (gx >= si.cols) gx -= si.cols;
                }
            }
        }
    }
    const int nt = bt.tap_end - bt.tap_begin;
    const unsigned toff = S0 + (unsigned)bt.tap_soff * 4u;
    if (sizeof(T) == 4) {   // (offset, value) records, 8 bytes each
        const TapOV* __restrict__ ov = plan.tap_ov + bt.tap_begin;
        for (int j = threadIdx.x; j < nt; j += kTileThreads) cp_async_to<8>(toff + 8u * j, ov + j);
    } else {
        const unsigned tval = S0 + (unsigned)bt.val_soff * ES;
        const T* __restrict__ vals = tvals<T>(plan) + bt.tap_begin;
        const int* __restrict__ offs = plan.tap_off + bt.tap_begin;
        for (int j = threadIdx.x; j < nt; j += kTileThreads) {
            cp_async_to<4>(toff + 4u * j, offs + j);
            cp_async_to<ES>(tval + ES * j, vals + j);
        }
    }
}

// Outputs of this thread in a TS x TS tile. TS = 32, or TS = 8 / 16 with the e4 map: 4
// outputs in row ly at columns lx + sx e (sx = TS / 4, lx < sx), so the e-th output of a
// down pair is sx e words after the first in the polyphase plane (an immediate offset);
// G = 1024 / TS^2 thread groups split the taps. Otherwise 1 output per thread and
// G = 256 / TS^2 groups.
struct ThreadMap {
    int E, G, g, nout;
    int sx, lgsx;     // column stride of the 4 outputs (TS >= 8)
    int ly, lx;       // first output of this thread (row, column within the tile)
};

__device__ __forceinline__ ThreadMap thread_map(const TileItem& w) {
    ThreadMap tm;
    const int t = threadIdx.x, TS = w.TS(), lgTS = w.lgTS();
    tm.nout = TS * TS;
    if (TS == 32 || (TS >= 8 && w.e4())) {
        tm.E = 4;
        tm.lgsx = lgTS - 2;
        tm.sx = 1 << tm.lgsx;
        const int lgper = 2 * lgTS - 2;             // threads per group: TS^2 / 4
        tm.G = kTileThreads >> lgper;
        tm.g = t >> lgper;
        const int u = t & ((1 << lgper) - 1);
        tm.lx = u & (tm.sx - 1);
        tm.ly = u >> tm.lgsx;
    } else {
        tm.E = 1;
        tm.sx = tm.lgsx = 0;
        tm.G = kTileThreads >> (2 * lgTS);
        tm.g = t >> (2 * lgTS);
        const int oi = t & (tm.nout - 1);
        tm.lx = oi & (TS - 1);
        tm.ly = oi >> lgTS;
    }
    return tm;
}

// Down pair, 4 outputs SX words apart in the plane; taps j = j0, j0 + G, ...
template <int SX, typename T>
__device__ __forceinline__ void down_taps4(const TapSrc<T> ts, int j0, int n, int G, const T* __restrict__ Sb,
                                           T (&acc)[4]) {
#pragma unroll 2
    for (int j = j0; j < n; j += G) {
        int o;
        T v;
        ts.get(j, o, v);
        const T* s = Sb + o;
        acc[0] = fma(v, s[0], acc[0]);
        acc[1] = fma(v, s[SX], acc[1]);
        acc[2] = fma(v, s[2 * SX], acc[2]);
        acc[3] = fma(v, s[3 * SX], acc[3]);
    }
}

// Up pair with staged phase tables and r dividing the output stride sx: the 4 outputs of a
// thread share one phase and their coarse columns are STEP = sx / r apart; taps j0, j0 + G, ...
template <int STEP, typename T>
__device__ __forceinline__ void up_taps4(TapSrc<T> ts, int j0, int n, int G, int rr, const T* __restrict__ Sb,
                                         T (&acc)[4]) {
    ts = ts + j0 * rr;
    const int stp = G * rr;
    for (int j = j0; j < n; j += G) {
        int o;
        T v;
        ts.get(0, o, v);
        ts = ts + stp;
        const T* s = Sb + o;
        acc[0] = fma(v, s[0], acc[0]);
        acc[1] = fma(v, s[STEP], acc[1]);
        acc[2] = fma(v, s[2 * STEP], acc[2]);
        acc[3] = fma(v, s[3 * STEP], acc[3]);
    }
}

// A load of the operator's input vector in the global-gather paths: through the read-only
// cache in kernels that run one pass (the input is not written during the launch), and
// through L2 (COH) in the fused loop, where the other pass of the same launch writes it.
template <bool COH, typename T>
__device__ __forceinline__ T ld_in(const T* p) {
    if constexpr (COH) return __ldcg(p);
    else return __ldg(p);
}

// Accumulate the pairs of batch `bi` of tile `w` (staged in S) into acc.
// (oy, ox): offset of the computed tile inside the staged one (a super tile's quarter; 0, 0
// for ordinary tiles)
// M: accumulator sets (1, or 4 for grouped items, whose pairs hold one tap list per member
// output subband; the region and the per-thread set-up of a pair serve every member).
template <typename T, int M, bool COH = false>
__device__ __forceinline__ void compute_batch(const TilePlanDev& plan, const T* __restrict__ in, const TileItem& w,
                                              const SubbandDev& so, int bi, const T* __restrict__ S,
                                              const PairSm* __restrict__ tab, const ThreadMap& tm, T (&acc)[M][4],
                                              int oy = 0, int ox = 0) {
    const TileBatch bt = plan.batches[bi];
    const TapSrc<T> stap = staged_taps<T>(S, bt);
    const T* __restrict__ gvals = tvals<T>(plan);
    const int E = tm.E, G = tm.G, g = tm.g;
    const int np = bt.pair_end - bt.pair_begin;
    for (int i = 0; i < np; ++i) {
        const TilePair P = tab[i].p;
        const int sh = tab[i].shift;   // staged column of the region's first column (vec pairs)
        const int lg = P.lg, r = 1 << lg, m = r - 1;
        const int nmem = M == 1 ? 1 : P.nm;
        if (P.mode == kDown) {
            const T* __restrict__ Sb = S + (tm.ly + oy) * P.PC + tm.lx + ox + sh;
            #pragma unroll
            for (int mk = 0; mk < M; ++mk) {
                if (mk >= nmem) break;
                const TapSrc<T> ts = stap + (M == 1 ? P.tap_begin : P.mtb[mk]);
                const int ntap = M == 1 ? P.ntap : P.mnt[mk];
                T (&ac)[4] = acc[mk];
                if (E == 4) {
                    if (tm.sx == 8) down_taps4<8, T>(ts, g, ntap, G, Sb, ac);
                    else if (tm.sx == 4) down_taps4<4, T>(ts, g, ntap, G, Sb, ac);
                    else down_taps4<2, T>(ts, g, ntap, G, Sb, ac);
                } else {
                    T a0 = 0, a1 = 0;
                    int j = g;
                    for (; j + G < ntap; j += 2 * G) {
                        int o0, o1;
                        T v0, v1;
                        ts.get(j, o0, v0);
                        ts.get(j + G, o1, v1);
                        a0 = fma(v0, Sb[o0], a0);
                        a1 = fma(v1, Sb[o1], a1);
                    }
                    if (j < ntap) {
                        int o0;
                        T v0;
                        ts.get(j, o0, v0);
                        a0 = fma(v0, Sb[o0], a0);
                    }
                    ac[0] += a0 + a1;
                }
            }
        } else if (P.mode == kUp) {
            // the phase tables (r^2 interleaved phases per tap slot) are staged with the batch
            // (tst) or read from global memory, where neighbouring outputs read neighbouring
            // phases and every tile of the subband reads the same table (L1/L2 hits)
            const int rr = r * r;
            const int py = w.ty0 + oy + tm.ly, px = w.tx0 + ox + tm.lx;
            const int rowb = ((py >> lg) - (w.ty0 >> lg)) * P.PC + sh;
            const bool st = P.tst != 0;
            const TapSrc<T> gts0 = st ? stap : global_taps<T>(plan);
            if (E == 4 && st && lg <= tm.lgsx) {
                const int ph = ((py & m) << lg) + (px & m);
                const T* __restrict__ Sb = S + rowb + ((px >> lg) - (w.tx0 >> lg));
                const int stepc = tm.lgsx - lg;   // log2 of the coarse column step
                #pragma unroll
            for (int mk = 0; mk < M; ++mk) {
                if (mk >= nmem) break;
                    const TapSrc<T> gts = gts0 + ((M == 1 ? P.tap_begin : P.mtb[mk]) + ph);
                    const int ntap = M == 1 ? P.ntap : P.mnt[mk];
                    if (stepc == 2) up_taps4<4, T>(gts, g, ntap, G, rr, Sb, acc[mk]);
                    else if (stepc == 1) up_taps4<2, T>(gts, g, ntap, G, rr, Sb, acc[mk]);
                    else up_taps4<1, T>(gts, g, ntap, G, rr, Sb, acc[mk]);
                }
            } else if (E == 4) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int pxe = px + tm.sx * e;
                    const int ph = ((py & m) << lg) + (pxe & m);
                    const T* __restrict__ Sb = S + rowb + ((pxe >> lg) - (w.tx0 >> lg));
                    const int stp = G * rr;
                    #pragma unroll
            for (int mk = 0; mk < M; ++mk) {
                if (mk >= nmem) break;
                        TapSrc<T> ts = gts0 + ((M == 1 ? P.tap_begin : P.mtb[mk]) + ph + g * rr);
                        const int ntap = M == 1 ? P.ntap : P.mnt[mk];
                        T a = 0;
                        for (int j = g; j < ntap; j += G) {
                            int o;
                            T v;
                            ts.get(0, o, v);
                            a = fma(v, Sb[o], a);
                            ts = ts + stp;
                        }
                        acc[mk][e] += a;
                    }
                }
            } else {
                const int ph = ((py & m) << lg) + (px & m);
                const T* __restrict__ Sb = S + rowb + ((px >> lg) - (w.tx0 >> lg));
                const int stp = G * rr;
                #pragma unroll
            for (int mk = 0; mk < M; ++mk) {
                if (mk >= nmem) break;
                    TapSrc<T> ts = gts0 + ((M == 1 ? P.tap_begin : P.mtb[mk]) + ph + g * rr);
                    const int ntap = M == 1 ? P.ntap : P.mnt[mk];
                    T a = 0;
                    for (int j = g; j < ntap; j += G) {
                        int o;
                        T v;
                        ts.get(0, o, v);
                        a = fma(v, Sb[o], a);
                        ts = ts + stp;
                    }
                    acc[mk][0] += a;
                }
            }
        } else {
            // gather from global memory (regions larger than the shared-memory budget, or
            // too little reuse to pay for staging)
            const T* __restrict__ src = in + tab[i].in_off;
            const int R = tab[i].in_rows, C = tab[i].in_cols;
            if (P.mode == kDownGlobal && E == 4) {
                // the four outputs of the thread share the pair's taps: when all four gather
                // inside the subband (no wrap), each tap's offset and value are loaded once and
                // its four inputs are independent loads
                const int py = w.ty0 + oy + tm.ly, px0 = w.tx0 + ox + tm.lx;
                const int by = py << lg, bx0 = px0 << lg, bstep = tm.sx << lg;
                const bool rows_ok = py < so.rows && by + P.y0 >= 0 && by + P.y0 + P.RR <= R;
                const bool cols_ok = px0 + 3 * tm.sx < so.cols && bx0 + P.x0 >= 0 && bx0 + 3 * bstep + P.x0 + P.RC <= C;
                if (rows_ok && cols_ok) {
                    const T* __restrict__ bp = src + (size_t)by * C + bx0;
                    #pragma unroll
            for (int mk = 0; mk < M; ++mk) {
                if (mk >= nmem) break;
                        const int tb = M == 1 ? P.tap_begin : P.mtb[mk];
                        const int ntap = M == 1 ? P.ntap : P.mnt[mk];
                        const int* __restrict__ tl = plan.tap_lin + tb;
                        const T* __restrict__ tv = gvals + tb;
                        T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll 2
                        for (int j = g; j < ntap; j += G) {
                            const int l = __ldg(tl + j);
                            const T v = __ldg(tv + j);
                            const T* __restrict__ q = bp + l;
                            a0 = fma(v, ld_in<COH>(q), a0);
                            a1 = fma(v, ld_in<COH>(q + bstep), a1);
                            a2 = fma(v, ld_in<COH>(q + 2 * bstep), a2);
                            a3 = fma(v, ld_in<COH>(q + 3 * bstep), a3);
                        }
                        acc[mk][0] += a0;
                        acc[mk][1] += a1;
                        acc[mk][2] += a2;
                        acc[mk][3] += a3;
                    }
                    continue;
                }
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (e >= E) continue;
                const int py = w.ty0 + oy + tm.ly, px = w.tx0 + ox + tm.lx + tm.sx * e;
                if (py >= so.rows || px >= so.cols) continue;
                int by, bx, pho, step;
                if (P.mode == kDownGlobal) {
                    by = py << lg;
                    bx = px << lg;
                    pho = 0;
                    step = 1;
                } else {
                    by = py >> lg;
                    bx = px >> lg;
                    pho = ((py & m) << lg) + (px & m);
                    step = r * r;
                }
                // interior: every tap of the pair lands inside the input subband, no wrap
                const bool inside = by + P.y0 >= 0 && by + P.y0 + P.RR <= R && bx + P.x0 >= 0 && bx + P.x0 + P.RC <= C;
                #pragma unroll
            for (int mk = 0; mk < M; ++mk) {
                if (mk >= nmem) break;
                    const int tb = (M == 1 ? P.tap_begin : P.mtb[mk]) + pho;
                    const int ntap = M == 1 ? P.ntap : P.mnt[mk];
                    T a = 0;
                    if (inside) {
                        // four independent chains (offset, then input) in flight
                        const T* __restrict__ bp = src + (size_t)by * C + bx;
                        const int* __restrict__ tl = plan.tap_lin + tb;
                        const T* __restrict__ tv = gvals + tb;
                        T a1 = 0, a2 = 0, a3 = 0;
                        int j = g;
                        for (; j + 3 * G < ntap; j += 4 * G) {
                            const int l0 = __ldg(tl + j * step), l1 = __ldg(tl + (j + G) * step);
                            const int l2 = __ldg(tl + (j + 2 * G) * step), l3 = __ldg(tl + (j + 3 * G) * step);
                            const T v0 = __ldg(tv + j * step), v1 = __ldg(tv + (j + G) * step);
                            const T v2 = __ldg(tv + (j + 2 * G) * step), v3 = __ldg(tv + (j + 3 * G) * step);
                            a = fma(v0, ld_in<COH>(bp + l0), a);
                            a1 = fma(v1, ld_in<COH>(bp + l1), a1);
                            a2 = fma(v2, ld_in<COH>(bp + l2), a2);
                            a3 = fma(v3, ld_in<COH>(bp + l3), a3);
                        }
                        for (; j < ntap; j += G) a = fma(__ldg(tv + j * step), ld_in<COH>(bp + __ldg(tl + j * step)), a);
                        a += (a1 + a2) + a3;
                    } else {
                        for (int j = g; j < ntap; j += G) {
                            const int pk = __ldg(plan.tap_off + tb + j * step);
                            const int yy = wrap1(by + (pk >> 16), R), xx = wrap1(bx + (int)(short)(pk & 0xffff), C);
                            a += __ldg(gvals + tb + j * step) * src[(size_t)yy * C + xx];
                        }
                    }
                    acc[mk][e] += a;
                }
            }
        }
    }
}

// Sum the G partial accumulators of each output (groups of threads that split the taps).
template <typename T>
__device__ __forceinline__ void group_reduce(const ThreadMap& tm, T (&acc)[4], T* red_buf) {
    if (tm.G > 1) {
        const int per = kTileThreads / tm.G;   // threads per group
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (e < tm.E) red_buf[e * kTileThreads + threadIdx.x] = acc[e];
        __syncthreads();
        if (tm.g == 0)
            for (int k = 1; k < tm.G; ++k)
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (e < tm.E) acc[e] += red_buf[e * kTileThreads + threadIdx.x + k * per];
    }
}

// Split tile (w.nparts() > 1): store this part's sums (threads of group 0), count the part as
// finished, and let the last part to finish sum all parts' sums in part order (the result
// does not depend on which part finishes last). Returns true in the CTA that runs the
// epilogue; every thread of the CTA calls it.
template <typename T>
__device__ __forceinline__ bool combine_parts(const TilePlanDev& plan, const TileItem& w, const ThreadMap& tm,
                                              T (&acc)[4]) {
    __shared__ int s_last;
    T* const buf = static_cast<T*>(plan.split_buf) + plan.split_base[w.sid];
    const int nout = tm.nout, np = w.nparts();
    const int q0 = (tm.ly << w.lgTS()) + tm.lx;
    if (tm.g == 0) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (e < tm.E) buf[w.part() * nout + q0 + tm.sx * e] = acc[e];
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(plan.split_ctr + w.sid, 1u) == (unsigned)(np - 1);
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    if (tm.g == 0) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (e >= tm.E) continue;
            T a = 0;
            for (int p = 0; p < np; ++p) a += __ldcg(buf + p * nout + q0 + tm.sx * e);
            acc[e] = a;
        }
    }
    if (threadIdx.x == 0) plan.split_ctr[w.sid] = 0u;   // ready for the next launch
    return true;
}

// Per-thread partial sums of the epilogues.
struct Partials {
    float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f, mx = 0.f;
    double d0 = 0.0;
};

// Epilogue of the outputs of one tile (threads of group 0).
template <typename T, int EPI>
__device__ __forceinline__ void epilogue(const TileItem& w, const SubbandDev& so, const ThreadMap& tm, const T (&acc)[4],
                                         T* __restrict__ out, const EpiArgs& ep, float beta, Partials& pt) {
    if (tm.g != 0) return;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (e >= tm.E) continue;
        const int py = w.ty0 + tm.ly, px = w.tx0 + tm.lx + tm.sx * e;
        if (py >= so.rows || px >= so.cols) continue;
        const size_t i = so.off + (size_t)py * so.cols + px;
        const int mR = (1 << so.lgR) - 1;
        const int cls = so.tab_off + ((py & mR) << so.lgR) + (px & mR);
        if (EPI == kApply || EPI == kApplyNorm) {
            T v = acc[e];
            if (ep.scale) v = (T)((double)v * ep.scale[cls]);
            out[i] = v;
            if (EPI == kApplyNorm) {
                if (sizeof(T) == 8) pt.d0 += (double)v * (double)v;
                else neu_add(pt.s0, pt.c0, (float)v * (float)v);
            }
        } else if (EPI == kK1 || EPI == kResNorm || EPI == kObj) {
            const float xv = ep.x0[i];
            const float rv = (float)acc[e] - xv;
            if (EPI != kObj) out[i] = (T)rv;
            neu_add(pt.s0, pt.c0, rv * rv);
            if (EPI == kK1) neu_add(pt.s1, pt.c1, xv * rv);
            if (EPI == kObj) {
                // kObj applies the operator to x itself: sum w|x| over this tile's outputs
                neu_add(pt.s1, pt.c1, ep.w_sb[w.o] * fabsf(ep.x[i]));
            }
        } else if (EPI == kK2) {
            const float gv = (float)acc[e];
            const float stp = ep.step_tab[cls];
            const float wv = ep.w_sb[w.o];
            const float yv = ep.y[i], xo = ep.x[i];
            const float z = yv - stp * gv;
            const float xn = copysignf(fmaxf(fabsf(z) - stp * wv, 0.f), z);
            ep.x[i] = xn;
            ep.y[i] = xn + beta * (xn - xo);
            neu_add(pt.s0, pt.c0, wv * fabsf(yv));
            pt.mx = fmaxf(pt.mx, gw_ratio(gv, wv));
        }
    }
}

// ---------------------------------------------------------------------------------------
// Single problem: persistent CTAs, heaviest tiles first, (tile, batch) double buffering
// ---------------------------------------------------------------------------------------
// Shared memory of one pass, declared by the kernel that runs it (so that a kernel running
// two passes holds one copy).
template <typename T>
struct PassSmem {
    unsigned char* raw;                       // the two staging buffers (dynamic)
    T* red_buf;                               // 4 x kTileThreads
    PairSm (*tab_buf)[kMaxBatchPairs];        // [2][kMaxBatchPairs]
    int* s_next;
};

// One application of a plan by the persistent CTAs of the launch: items from the queue,
// (tile, batch) double buffering, the epilogue, and the grid-wide FP64 reduction whose last
// CTA finishes the pass (COH: see ld_in).
template <typename T, int EPI, bool SPLIT, bool SUP, bool GRP, bool COH>
__device__ __forceinline__ void tile_pass(const TileArgs& A, const T* __restrict__ in, T* __restrict__ out,
                                          const EpiArgs& ep, const PassSmem<T>& sm) {
    constexpr int M = GRP ? 4 : 1;
    T* const buf0 = reinterpret_cast<T*>(sm.raw);
    T* const buf1 = buf0 + A.plan.buf_elems;
    T* const red_buf = sm.red_buf;
    const TilePlanDev& plan = A.plan;
    const int t = threadIdx.x;
    Partials pt;
    float beta = 0.f;
    if (EPI == kK2) {
        const int k = ep.st->k;
        beta = ep.st->ista ? 0.f : (float)(k - 1) / (float)(k + 2);
    }
    // work items come from a queue, heaviest first
    int& s_next = *sm.s_next;
    if (t == 0) s_next = (int)atomicAdd(&A.queue->next, 1u);
    __syncthreads();
    int it = s_next;
    TileItem w = (it < plan.n_items) ? plan.items[it] : TileItem{};
    int bi = w.batch_begin;
    T* S = buf0;
    T* Snext = buf1;
    PairSm* tab = sm.tab_buf[0];
    PairSm* tab_next = sm.tab_buf[1];
    if (it < plan.n_items) stage_batch<T>(plan, in, w, bi, S, tab);
    cp_async_commit();
    T acc[M][4];
#pragma unroll
    for (int k = 0; k < M; ++k)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[k][e] = 0;
    while (it < plan.n_items) {
        int nit = it, nbi = bi + 1;
        TileItem nw = w;
        __syncthreads();
        if (nbi >= w.batch_end) {
            if (t == 0) s_next = (int)atomicAdd(&A.queue->next, 1u);
            __syncthreads();
            nit = s_next;
            if (nit < plan.n_items) {
                nw = plan.items[nit];
                nbi = nw.batch_begin;
            }
        }
        if (nit < plan.n_items) stage_batch<T>(plan, in, nw, nbi, Snext, tab_next);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const SubbandDev so = A.sb[w.o];
        const ThreadMap tm = thread_map(w);
        if (SUP && w.sup()) {
            // a super tile (one batch, 4 outputs per thread, no thread groups): its 2 x 2
            // tiles one after the other from the same staged regions
            for (int q = 0; q < 4; ++q) {
                const int oy = (q >> 1) << w.lgTS(), ox = (q & 1) << w.lgTS();
                if (w.ty0 + oy >= so.rows || w.tx0 + ox >= so.cols) continue;
                compute_batch<T, M, COH>(plan, in, w, so, bi, S, tab, tm, acc, oy, ox);
                TileItem wq = w;
                wq.ty0 += oy;
                wq.tx0 += ox;
                epilogue<T, EPI>(wq, so, tm, acc[0], out, ep, beta, pt);
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[0][e] = 0;
            }
        } else {
            compute_batch<T, M, COH>(plan, in, w, so, bi, S, tab, tm, acc);
            if (bi + 1 == w.batch_end) {
                if (!GRP) {
                    group_reduce<T>(tm, acc[0], red_buf);
                    if (!SPLIT || w.split < (2 << 16) || combine_parts<T>(plan, w, tm, acc[0]))
                        epilogue<T, EPI>(w, so, tm, acc[0], out, ep, beta, pt);
                } else {
                    // one epilogue per member subband of the group (same geometry)
                    const int nm = w.nm() > 0 ? w.nm() : 1;
                    for (int k = 0; k < M; ++k) {
                        if (k >= nm) break;
                        if (k > 0 && tm.G > 1) __syncthreads();   // red_buf reused
                        group_reduce<T>(tm, acc[k], red_buf);
                        TileItem wk = w;
                        wk.o = w.o + k;
                        epilogue<T, EPI>(wk, A.sb[wk.o], tm, acc[k], out, ep, beta, pt);
                    }
                }
#pragma unroll
                for (int k = 0; k < M; ++k)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[k][e] = 0;
            }
        }
        it = nit;
        bi = nbi;
        w = nw;
        T* tmp = S;
        S = Snext;
        Snext = tmp;
        PairSm* tt = tab;
        tab = tab_next;
        tab_next = tt;
    }
    // this CTA has no more tiles: the next kernel of the stream may start its CTAs
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    cp_async_wait<0>();
    __syncthreads();
    double v[2] = {pt.d0 + (double)pt.s0 + (double)pt.c0, EPI == kK2 ? (double)pt.mx : (double)pt.s1 + (double)pt.c1}, tot[2];
    const unsigned maxmask = (EPI == kK2) ? 2u : 0u;
    if (grid_reduce<2>(v, maxmask, ep.part, &A.queue->done, tot)) {
        if (t == 0) {
            A.queue->next = 0u;
            if (EPI == kK1) {
                ep.st->rr = tot[0];
                ep.st->x0r = tot[1];
            } else if (EPI == kK2) {
                finish_iteration(ep.st, tot[0], tot[1]);
            } else if (EPI == kApplyNorm || EPI == kResNorm) {
                ep.red_out[0] = tot[0];
            }
        }
    }
}

// SPLIT: the plan has split tiles (a separate instance, so that plans without them run code
// that carries none of the combining step)
// SUP: the plan has super tiles (likewise a separate instance)
// GRP: the plan has grouped items (the tile of up to four subbands per item; likewise)
template <typename T, int EPI, bool SPLIT, bool SUP, bool GRP>
__global__ void __launch_bounds__(kTileThreads, 3) tile_kernel(TileArgs A, const T* __restrict__ in,
                                                            T* __restrict__ out, EpiArgs ep) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T red_buf[4 * kTileThreads];
    __shared__ PairSm tab_buf[2][kMaxBatchPairs];
    __shared__ int s_next;
    // launched as a programmatic dependent of the previous FISTA kernel: nothing it wrote is
    // read before that grid has completed (a no-op for ordinary launches)
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    if (EPI == kK1 || EPI == kK2) {
        if (*(volatile int*)&ep.st->stop) return;
    }
    tile_pass<T, EPI, SPLIT, SUP, GRP, false>(A, in, out, ep, PassSmem<T>{smem_raw, red_buf, tab_buf, &s_next});
}

// ---------------------------------------------------------------------------------------
// Batch of problems: one launch covers the tiles of every running problem
// ---------------------------------------------------------------------------------------
// Block sum of the per-thread partials of one tile, added to the problem's slots.
template <int EPI>
__device__ __forceinline__ void flush_partials(Partials& pt, double* sums, double* red) {
    double a = (double)pt.s0 + (double)pt.c0;
    double b = (EPI == kK2) ? (double)pt.mx : (double)pt.s1 + (double)pt.c1;
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        const double o = __shfl_down_sync(0xffffffffu, b, off);
        b = (EPI == kK2) ? fmax(b, o) : b + o;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[2 * warp] = a;
        red[2 * warp + 1] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0, B = 0.0;
        for (int k = 0; k < kTileThreads / 32; ++k) {
            A += red[2 * k];
            B = (EPI == kK2) ? fmax(B, red[2 * k + 1]) : B + red[2 * k + 1];
        }
        if (EPI == kK1) {
            atomicAdd(&sums[0], A);
            atomicAdd(&sums[1], B);
        } else if (EPI == kK2) {
            atomicAdd(&sums[2], A);
            atomicMax(reinterpret_cast<unsigned long long*>(&sums[3]), (unsigned long long)__double_as_longlong(B));
        } else {
            atomicAdd(&sums[0], A);
            atomicAdd(&sums[1], B);
        }
    }
    pt = Partials();
}

// GRP: the plans have grouped items (one item computes the tile of every subband of a level,
// one accumulator set and one epilogue per member subband), as in tile_kernel; that instance
// runs two CTAs per SM so that its four accumulator sets stay in registers
template <int EPI, bool GRP>
__global__ void __launch_bounds__(kTileThreads, GRP ? 2 : 3) tile_batch_kernel(BatchArgs B) {
    constexpr int M = GRP ? 4 : 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* const buf0 = reinterpret_cast<float*>(smem_raw);
    float* const buf1 = buf0 + B.buf_elems;
    __shared__ float red_buf[4 * kTileThreads];
    __shared__ double red_d[2 * kTileThreads / 32];
    __shared__ int s_next;
    const int t = threadIdx.x;
    const int n_items = B.n_items_dev ? *B.n_items_dev : B.n_items;
    // next item whose problem is still running (thread 0), broadcast through shared memory
    auto fetch = [&]() {
        if (t == 0) {
            int i;
            for (;;) {
                i = (int)atomicAdd(&B.queue->next, 1u);
                if (i >= n_items) break;
                if (EPI == kObj || !*(volatile int*)&B.probs[B.items[i].p].st->stop) break;
            }
            s_next = i;
        }
        __syncthreads();
        return s_next;
    };
    auto plan_of = [&](int p) -> const TilePlanDev& { return (EPI == kK2) ? B.probs[p].adj : B.probs[p].fwd; };
    auto in_of = [&](int p) -> const float* {
        const BatchProblem& P = B.probs[p];
        return (EPI == kK1) ? P.y : (EPI == kK2) ? P.r : P.x;
    };
    int it = fetch();
    int bi = 0;
    float* S = buf0;
    float* Snext = buf1;
    __shared__ PairSm tab_buf[2][kMaxBatchPairs];
    PairSm* tab = tab_buf[0];
    PairSm* tab_next = tab_buf[1];
    if (it < n_items) {
        const BatchItem bw = B.items[it];
        const TilePlanDev& pl = plan_of(bw.p);
        bi = pl.items[bw.item].batch_begin;
        stage_batch<float>(pl, in_of(bw.p), pl.items[bw.item], bi, S, tab);
    }
    cp_async_commit();
    float acc[M][4];
#pragma unroll
    for (int k = 0; k < M; ++k)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[k][e] = 0.f;
    Partials pt;
    while (it < n_items) {
        const BatchItem bw = B.items[it];
        const BatchProblem& P = B.probs[bw.p];
        const TilePlanDev& pl = plan_of(bw.p);
        const TileItem w = pl.items[bw.item];
        int nit = it, nbi = bi + 1;
        __syncthreads();
        if (nbi >= w.batch_end) {
            nit = fetch();
            if (nit < n_items) {
                const BatchItem nb = B.items[nit];
                nbi = plan_of(nb.p).items[nb.item].batch_begin;
            }
        }
        if (nit < n_items) {
            const BatchItem nb = B.items[nit];
            const TilePlanDev& npl = plan_of(nb.p);
            stage_batch<float>(npl, in_of(nb.p), npl.items[nb.item], nbi, Snext, tab_next);
        }
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const SubbandDev so = P.sb[w.o];
        const ThreadMap tm = thread_map(w);
        compute_batch<float, M>(pl, in_of(bw.p), w, so, bi, S, tab, tm, acc);
        if (bi + 1 == w.batch_end) {
            EpiArgs ep{};
            ep.x0 = P.x0;
            ep.y = P.y;
            ep.x = P.x;
            ep.step_tab = P.step_tab;
            ep.w_sb = P.w_sb;
            float beta = 0.f;
            if (EPI == kK2) {
                const int k = P.st->k;
                beta = P.st->ista ? 0.f : (float)(k - 1) / (float)(k + 2);
            }
            if (!GRP) {
                group_reduce<float>(tm, acc[0], red_buf);
                epilogue<float, EPI>(w, so, tm, acc[0], (EPI == kK1) ? P.r : nullptr, ep, beta, pt);
            } else {
                // one epilogue per member subband of the group (same geometry)
                const int nm = w.nm() > 0 ? w.nm() : 1;
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    if (k >= nm) break;
                    if (k > 0 && tm.G > 1) __syncthreads();   // red_buf reused
                    group_reduce<float>(tm, acc[k], red_buf);
                    TileItem wk = w;
                    wk.o = w.o + k;
                    epilogue<float, EPI>(wk, P.sb[wk.o], tm, acc[k], (EPI == kK1) ? P.r : nullptr, ep, beta, pt);
                }
            }
            flush_partials<EPI>(pt, P.sums, red_d);
#pragma unroll
            for (int k = 0; k < M; ++k)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[k][e] = 0.f;
        }
        it = nit;
        bi = nbi;
        float* tmp = S;
        S = Snext;
        Snext = tmp;
        PairSm* tt = tab;
        tab = tab_next;
        tab_next = tt;
    }
    cp_async_wait<0>();
    __syncthreads();
    // the last CTA resets the queue; after the step kernel it also finishes the iteration of
    // every running problem (one thread per problem)
    __shared__ bool s_last;
    __threadfence();
    if (t == 0) s_last = (atomicAdd(&B.queue->done, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (EPI == kK2) {
        int running = 0;
        for (int p = t; p < B.B; p += kTileThreads) {
            const BatchProblem& P = B.probs[p];
            SolveState* st = P.st;
            if (!st->stop) {
                st->rr = __ldcg(&P.sums[0]);
                st->x0r = __ldcg(&P.sums[1]);
                finish_iteration(st, __ldcg(&P.sums[2]), __ldcg(&P.sums[3]));
            }
            P.sums[0] = P.sums[1] = P.sums[2] = P.sums[3] = 0.0;
            running += st->stop ? 0 : 1;
            if (B.run_flags) B.run_flags[p] = st->stop ? 0 : 1;
        }
        for (int off = 16; off > 0; off >>= 1) running += __shfl_down_sync(0xffffffffu, running, off);
        __shared__ int s_run[kTileThreads / 32];
        if ((t & 31) == 0) s_run[t >> 5] = running;
        __syncthreads();
        if (t == 0) {
            int tot = 0;
            for (int k = 0; k < kTileThreads / 32; ++k) tot += s_run[k];
            *B.running = tot;
        }
    }
    if (t == 0) {
        B.queue->next = 0u;
        B.queue->done = 0u;
    }
}

// ---------------------------------------------------------------------------------------
// Fused FISTA loop: kernel 1 and kernel 2 of several iterations in one cooperative launch
// ---------------------------------------------------------------------------------------
// Grid-wide barrier between the passes (every CTA of a cooperative launch is resident). One
// thread per CTA reads the generation, makes the CTA's writes visible and arrives; the last
// arrival resets the count and advances the generation, the others poll it at most
// spin_limit times. A poll that runs out records the timeout (and stops the solve); a poll
// that sees another CTA's timeout returns false as well, so no CTA waits unboundedly. A CTA
// released after others gave up may run one more pass alone and then leaves at the next
// barrier; that pass's queue counters stay unreset, which the host resets after a timeout
// (WDB_ETIMEOUT).
__device__ __forceinline__ bool fused_barrier(SolveState* st, long long spin_limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned int* vgen = &st->bar_gen;
        const unsigned int g = *vgen;
        __threadfence();
        if (atomicAdd(&st->bar_count, 1u) == gridDim.x - 1) {
            atomicExch(&st->bar_count, 0u);
            __threadfence();
            atomicAdd(&st->bar_gen, 1u);
        } else {
            long long n = 0;
            while (*vgen == g) {
                if (*(volatile int*)&st->timeout) {
                    ok = 0;
                    break;
                }
                if (++n > spin_limit) {
                    atomicExch(&st->timeout, 1);
                    atomicExch(&st->stop, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

struct FusedArgs {
    TileArgs A1, A2;        // plans of Theta_K (kernel 1) and Theta_K^T (kernel 2)
    const float* y;
    float* r;
    EpiArgs e1, e2;
    int iters;
    long long spin_limit;
};

// SUPn / GRPn: the pass of plan n has super tiles / grouped items (as in tile_kernel; plans
// with split tiles run the two-launch loop instead)
template <bool SUP1, bool GRP1, bool SUP2, bool GRP2>
__global__ void __launch_bounds__(kTileThreads, 3) fista_fused_kernel(FusedArgs F) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float red_buf[4 * kTileThreads];
    __shared__ PairSm tab_buf[2][kMaxBatchPairs];
    __shared__ int s_next;
    const PassSmem<float> sm{smem_raw, red_buf, tab_buf, &s_next};
    SolveState* const st = F.e1.st;
    for (int i = 0; i < F.iters; ++i) {
        // every CTA reads the flag after the same barrier, so all leave together
        if (*(volatile int*)&st->stop || *(volatile int*)&st->timeout) break;
        tile_pass<float, kK1, false, SUP1, GRP1, true>(F.A1, F.y, F.r, F.e1, sm);
        if (!fused_barrier(st, F.spin_limit)) break;
        tile_pass<float, kK2, false, SUP2, GRP2, true>(F.A2, F.r, nullptr, F.e2, sm);
        if (!fused_barrier(st, F.spin_limit)) break;
    }
}

template <bool SUP1, bool GRP1, bool SUP2, bool GRP2>
wdb_status launch_fused_as(const FusedArgs& F, int smem, int max_ctas, cudaStream_t st) {
    auto* kern = fista_fused_kernel<SUP1, GRP1, SUP2, GRP2>;
    static unsigned long long attr = 0ull;
    if (!done_on_device(&attr)) {
        WDB_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        mark_on_device(&attr);
    }
    int dev = 0, sms = 0, per = 0;
    WDB_CK(cudaGetDevice(&dev));
    WDB_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    WDB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kTileThreads, smem));
    if (per <= 0 || sms <= 0) return set_error(WDB_EINVAL, "fused loop: no resident CTA for %d bytes", smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::max(1, std::min(sms * per, max_ctas)));
    cfg.blockDim = dim3(kTileThreads);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    WDB_CK(cudaLaunchKernelEx(&cfg, kern, F));
    count_launch();
    WDB_CK(cudaGetLastError());
    return WDB_OK;
}

template <bool SUP1, bool GRP1>
wdb_status launch_fused_2(const FusedArgs& F, int mode2, int smem, int max_ctas, cudaStream_t st) {
    if (mode2 == 1) return launch_fused_as<SUP1, GRP1, true, false>(F, smem, max_ctas, st);
    if (mode2 == 2) return launch_fused_as<SUP1, GRP1, false, true>(F, smem, max_ctas, st);
    return launch_fused_as<SUP1, GRP1, false, false>(F, smem, max_ctas, st);
}

// pdl: programmatic dependent launch, so that this grid's CTAs are scheduled while the
// previous kernel of the stream drains// pdl: programmatic dependent launch, so that this grid's CTAs are scheduled while the
// previous kernel of the stream drains (the kernel waits for that grid before its work)
template <typename T, int EPI, bool SPLIT, bool SUP, bool GRP>
wdb_status launch_tile_as(const TileArgs& A, const T* in, T* out, const EpiArgs& ep, cudaStream_t st, bool pdl) {
    static unsigned long long attr = 0ull;
    if (!done_on_device(&attr)) {
        WDB_CK(cudaFuncSetAttribute(tile_kernel<T, EPI, SPLIT, SUP, GRP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    200 * 1024));
        mark_on_device(&attr);
    }
    if (pdl) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)A.grid);
        cfg.blockDim = dim3(kTileThreads);
        cfg.dynamicSmemBytes = (size_t)A.plan.smem_bytes;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        WDB_CK(cudaLaunchKernelEx(&cfg, tile_kernel<T, EPI, SPLIT, SUP, GRP>, A, in, out, ep));
    } else {
        tile_kernel<T, EPI, SPLIT, SUP, GRP><<<A.grid, kTileThreads, A.plan.smem_bytes, st>>>(A, in, out, ep);
    }
    count_launch();
    WDB_CK(cudaGetLastError());
    return WDB_OK;
}

// Plans with split tiles or super tiles (FP32 only) run the instances with those steps.
template <typename T, int EPI>
wdb_status launch_tile(const TileArgs& A, const T* in, T* out, const EpiArgs& ep, cudaStream_t st, bool pdl = false) {
    constexpr bool f32 = sizeof(T) == 4;
    if (f32 && A.plan.split_ctr) return launch_tile_as<T, EPI, f32, false, false>(A, in, out, ep, st, pdl);
    if (f32 && A.plan.n_sup > 0) return launch_tile_as<T, EPI, false, f32, false>(A, in, out, ep, st, pdl);
    if (f32 && A.plan.n_grp > 0) return launch_tile_as<T, EPI, false, false, f32>(A, in, out, ep, st, pdl);
    return launch_tile_as<T, EPI, false, false, false>(A, in, out, ep, st, pdl);
}

template <int EPI, bool GRP>
wdb_status launch_batch_as(const BatchArgs& B, cudaStream_t st) {
    static unsigned long long attr = 0ull;
    if (!done_on_device(&attr)) {
        WDB_CK(cudaFuncSetAttribute(tile_batch_kernel<EPI, GRP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    200 * 1024));
        mark_on_device(&attr);
    }
    tile_batch_kernel<EPI, GRP><<<B.grid, kTileThreads, B.smem_bytes, st>>>(B);
    count_launch();
    WDB_CK(cudaGetLastError());
    return WDB_OK;
}

template <int EPI>
wdb_status launch_batch(const BatchArgs& B, cudaStream_t st) {
    return B.grouped ? launch_batch_as<EPI, true>(B, st) : launch_batch_as<EPI, false>(B, st);
}

}  // namespace

int tile_grid(int smem_bytes) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(tile_kernel<float, kK2, false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tile_kernel<float, kK2, false, false, false>, kTileThreads,
                                                  smem_bytes);
    if (sms <= 0) sms = 1;
    if (per <= 0) per = 1;
    return sms * per;
}

int tile_batch_grid(int smem_bytes, bool grouped) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (grouped) {
        cudaFuncSetAttribute(tile_batch_kernel<kK2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tile_batch_kernel<kK2, true>, kTileThreads, smem_bytes);
    } else {
        cudaFuncSetAttribute(tile_batch_kernel<kK2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tile_batch_kernel<kK2, false>, kTileThreads, smem_bytes);
    }
    if (sms <= 0) sms = 1;
    if (per <= 0) per = 1;
    return sms * per;
}

template <typename T>
wdb_status tile_apply(const TileArgs& A, const T* in, T* out, const double* scale, double* norm_out, double* part,
                      cudaStream_t st) {
    EpiArgs ep{};
    ep.scale = scale;
    ep.part = part;
    ep.red_out = norm_out;
    if (norm_out) return launch_tile<T, kApplyNorm>(A, in, out, ep, st);
    return launch_tile<T, kApply>(A, in, out, ep, st);
}

wdb_status tile_k1(const TileArgs& A, const float* y, const float* x0, float* r, double* part, SolveState* s,
                   cudaStream_t st, bool pdl) {
    EpiArgs ep{};
    ep.x0 = x0;
    ep.part = part;
    ep.st = s;
    return launch_tile<float, kK1>(A, y, r, ep, st, pdl);
}

wdb_status tile_k2(const TileArgs& A, const float* r, float* y, float* x, const float* step_tab, const float* w_sb,
                   double* part, SolveState* s, cudaStream_t st, bool pdl) {
    EpiArgs ep{};
    ep.y = y;
    ep.x = x;
    ep.step_tab = step_tab;
    ep.w_sb = w_sb;
    ep.part = part;
    ep.st = s;
    return launch_tile<float, kK2>(A, r, nullptr, ep, st, pdl);
}

bool tile_fused_supported(const TileArgs& F, const TileArgs& A) { return !F.plan.split_ctr && !A.plan.split_ctr; }

wdb_status tile_fused(const TileArgs& F, const TileArgs& A, float* y, const float* x0, float* r, float* x,
                      const float* step_tab, const float* w_sb, double* part, SolveState* s, int iters,
                      long long spin_limit, int max_ctas, cudaStream_t st) {
    if (!tile_fused_supported(F, A)) return set_error(WDB_EINVAL, "fused loop: plans with split tiles");
    FusedArgs fa{};
    fa.A1 = F;
    fa.A2 = A;
    fa.y = y;
    fa.r = r;
    fa.e1.x0 = x0;
    fa.e1.part = part;
    fa.e1.st = s;
    fa.e2.y = y;
    fa.e2.x = x;
    fa.e2.step_tab = step_tab;
    fa.e2.w_sb = w_sb;
    fa.e2.part = part;
    fa.e2.st = s;
    fa.iters = iters;
    fa.spin_limit = spin_limit > 0 ? spin_limit : (1LL << 23);
    const int smem = std::max(F.plan.smem_bytes, A.plan.smem_bytes);
    const int mode1 = F.plan.n_sup > 0 ? 1 : F.plan.n_grp > 0 ? 2 : 0;
    const int mode2 = A.plan.n_sup > 0 ? 1 : A.plan.n_grp > 0 ? 2 : 0;
    if (mode1 == 1) return launch_fused_2<true, false>(fa, mode2, smem, max_ctas, st);
    if (mode1 == 2) return launch_fused_2<false, true>(fa, mode2, smem, max_ctas, st);
    return launch_fused_2<false, false>(fa, mode2, smem, max_ctas, st);
}

wdb_status tile_resnorm(const TileArgs& A, const float* x, const float* x0, float* r, double* out, double* part,
                        cudaStream_t st) {
    EpiArgs ep{};
    ep.x0 = x0;
    ep.part = part;
    ep.red_out = out;
    return launch_tile<float, kResNorm>(A, x, r, ep, st);
}

wdb_status batch_k1(const BatchArgs& B, cudaStream_t st) { return launch_batch<kK1>(B, st); }
wdb_status batch_k2(const BatchArgs& B, cudaStream_t st) { return launch_batch<kK2>(B, st); }
wdb_status batch_objective(const BatchArgs& B, cudaStream_t st) { return launch_batch<kObj>(B, st); }

template wdb_status tile_apply<float>(const TileArgs&, const float*, float*, const double*, double*, double*,
                                      cudaStream_t);
template wdb_status tile_apply<double>(const TileArgs&, const double*, double*, const double*, double*, double*,
                                       cudaStream_t);

}  // namespace wdb
