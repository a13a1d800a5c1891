// Host-only structural check of a tile plan (the planner is in tile.cu): every output of
// every subband is produced by exactly one item, the parts of a split tile chain its batches
// once, every staged region and tap area lies in the staging buffer, every staged read of a
// tap stays inside its pair's region (its polyphase plane for down pairs), and super tiles,
// split tiles and pairs staged in 16-byte chunks meet their conditions.
#include <algorithm>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "plan_check.h"

namespace wdb {

std::string check_tile_plan(const Layout& L, const TilePlanHost& P) {
    char msg[256];
    auto fail = [&](const char* fmt, int a, int b) {
        std::snprintf(msg, sizeof msg, fmt, a, b);
        return std::string(msg);
    };
    const int esize = P.esize;
    const long long buf_bytes = (long long)P.buf_elems * esize;
    if ((int)P.subs.size() != L.S) return fail("plan has %d subbands, layout %d", (int)P.subs.size(), L.S);
    if (P.pair_sm.size() != P.pairs.size() || P.tap_ov.size() != P.tap_off.size())
        return fail("pair table or tap records out of step (%d, %d)", (int)P.pair_sm.size(), (int)P.tap_ov.size());
    for (size_t k = 0; k < P.pairs.size(); ++k) {
        const PairSm& e = P.pair_sm[k];
        const SubbandDev& si = L.sb[P.pairs[k].in_sb];
        const TilePair& q = P.pairs[k];
        bool same = e.p.in_sb == q.in_sb && e.p.soff == q.soff && e.p.mode == q.mode && e.p.lg == q.lg &&
                          e.p.RR == q.RR && e.p.RC == q.RC && e.p.PR == q.PR && e.p.PC == q.PC && e.p.PS == q.PS &&
                          e.p.y0 == q.y0 && e.p.x0 == q.x0 && e.p.tap_begin == q.tap_begin && e.p.ntap == q.ntap &&
                          e.p.vec == q.vec && e.p.tst == q.tst && e.p.nm == q.nm;
        for (int k = 0; k < 4 && same; ++k) same = e.p.mtb[k] == q.mtb[k] && e.p.mnt[k] == q.mnt[k];
        if (!same || e.in_off != si.off || e.in_rows != si.rows || e.in_cols != si.cols)
            return fail("pair table entry %d differs from pair %d", (int)k, (int)k);
    }
    for (int o = 0; o < L.S; ++o) {
        const TileSub& sub = P.subs[o];
        const int TS = sub.TS, TSs = sub.sup ? 2 * TS : TS;
        if (sub.sup && (TS != 32 || !sub.e4 || sub.batch_end - sub.batch_begin != 1))
            return fail("subband %d: super tiles need one batch of 32-tiles with 4 outputs per thread", o, 0);
        for (int bi = sub.batch_begin; bi < sub.batch_end; ++bi) {
            const TileBatch& bt = P.batches[bi];
            const int np = bt.pair_end - bt.pair_begin, nt = bt.tap_end - bt.tap_begin;
            if (np > kMaxBatchPairs) return fail("batch %d has %d pairs", bi, np);
            if (bt.pair_begin < sub.pair_begin || bt.pair_end > sub.pair_end) return fail("batch %d pairs outside subband %d", bi, o);
            const long long tap_byte = (long long)bt.tap_soff * 4;
            if (esize == 4) {
                if (tap_byte % 8 || tap_byte + 8LL * nt > buf_bytes) return fail("batch %d tap records outside the buffer (%d taps)", bi, nt);
            } else if ((long long)bt.val_soff * esize < tap_byte + 4LL * nt || (long long)(bt.val_soff + nt) * esize > buf_bytes) {
                return fail("batch %d tap values outside the buffer (%d taps)", bi, nt);
            }
            for (int pi = bt.pair_begin; pi < bt.pair_end; ++pi) {
                const TilePair& tp = P.pairs[pi];
                const SubbandDev& si = L.sb[tp.in_sb];
                if (sub.sup && tp.mode >= kDownGlobal) return fail("super subband %d gathers pair %d from global memory", o, pi);
                if (tp.mode >= kDownGlobal) continue;
                const int r = 1 << tp.lg;
                const long long size = tp.mode == kDown ? (long long)r * r * tp.PS : (long long)tp.PR * tp.PC;
                if (tp.soff < 0 || ((long long)tp.soff + size) * esize > tap_byte)
                    return fail("pair %d region overlaps the batch's taps (batch %d)", pi, bi);
                if (tp.vec && (esize != 4 || si.cols % 4 || si.off % 4 || tp.PC % 4 || tp.soff % 4 ||
                               (tp.mode == kDown && tp.lg != 0)))
                    return fail("pair %d staged in 16-byte chunks without 4-aligned rows (batch %d)", pi, bi);
                // every staged read of every member's taps: tap offset plus the farthest output of
                // the staged tile
                const int nmem = sub.grp > 0 ? sub.grp : 1;
                if (tp.nm != nmem) return fail("pair %d has %d members, its group another count", pi, tp.nm);
                if (tp.mtb[0] != tp.tap_begin || tp.mnt[0] != tp.ntap) return fail("pair %d member 0 is not its taps", pi, 0);
                long long table = 0;
                for (int mk = 0; mk < nmem; ++mk) table += (long long)tp.mnt[mk] * r * r;
                if (tp.mode == kUp && tp.tst && table * (4 + esize) > buf_bytes / 2 && tp.lg > 3)
                    return fail("pair %d stages a phase table above half of the buffer (batch %d)", pi, bi);
                for (int mk = 0; mk < nmem; ++mk) {
                    const int tb = tp.mtb[mk];
                    const int ntab = tp.mode == kDown ? tp.mnt[mk] : tp.mnt[mk] * r * r;
                    if (tp.mode == kDown || tp.tst)
                        if (tb < bt.tap_begin || tb + ntab > bt.tap_end) return fail("pair %d taps outside batch %d", pi, bi);
                    const int far = tp.mode == kDown ? TSs - 1 : (TSs - 1) >> tp.lg;
                    for (int j = 0; j < ntab; ++j) {
                        const long long off = P.tap_off[tb + j] - tp.soff;
                        if (off < 0 || off >= size) return fail("pair %d tap %d outside its region", pi, j);
                        const long long in_plane = tp.mode == kDown ? off % tp.PS : off;
                        const long long row = in_plane / tp.PC, col = in_plane % tp.PC;
                        if (row + far >= tp.PR || col + far + (tp.vec ? 3 : 0) >= tp.PC)
                            return fail("pair %d tap %d reads past its region's rows or columns", pi, j);
                    }
                }
            }
        }
    }
    // every output of every subband exactly once; the parts of a split tile cover its batches once
    std::vector<std::vector<unsigned char>> hit(L.S);
    for (int o = 0; o < L.S; ++o) hit[o].assign((size_t)L.sb[o].rows * L.sb[o].cols, 0);
    std::vector<std::vector<std::pair<int, int>>> parts(P.n_split);
    std::vector<int> part_sub(P.n_split, -1);
    std::map<int, std::pair<int, int>> split_origin;
    for (size_t k = 0; k < P.items.size(); ++k) {
        const TileItem& w = P.items[k];
        if (w.o < 0 || w.o >= L.S) return fail("item %d names subband %d", (int)k, w.o);
        const TileSub& sub = P.subs[w.o];
        const SubbandDev& so = L.sb[w.o];
        if (w.TS() != sub.TS || w.e4() != sub.e4 || w.sup() != sub.sup)
            return fail("item %d geometry differs from subband %d", (int)k, w.o);
        if (w.batch_begin < sub.batch_begin || w.batch_end > sub.batch_end || w.batch_begin >= w.batch_end)
            return fail("item %d batches outside subband %d", (int)k, w.o);
        const int side = sub.sup ? 2 * sub.TS : sub.TS;
        if (w.ty0 % side || w.tx0 % side || w.ty0 >= so.rows || w.tx0 >= so.cols)
            return fail("item %d origin off the tile grid of subband %d", (int)k, w.o);
        if (w.nparts() > 1) {
            if (w.sid < 0 || w.sid >= P.n_split || w.part() >= w.nparts() || sub.sup)
                return fail("item %d has bad split fields (tile %d)", (int)k, w.sid);
            if ((long long)P.split_base[w.sid] + (long long)w.nparts() * sub.TS * sub.TS > P.split_elems)
                return fail("split tile %d partial sums outside the scratch (item %d)", w.sid, (int)k);
            if (P.items.size() && (split_origin.count(w.sid) && split_origin[w.sid] != std::make_pair(w.ty0, w.tx0)))
                return fail("split tile %d parts at different origins (item %d)", w.sid, (int)k);
            split_origin[w.sid] = std::make_pair(w.ty0, w.tx0);
            parts[w.sid].push_back({w.batch_begin, w.batch_end});
            if (part_sub[w.sid] >= 0 && part_sub[w.sid] != w.o) return fail("split tile %d spans subbands (item %d)", w.sid, (int)k);
            part_sub[w.sid] = w.o;
            if (w.part() != 0) continue;
        } else if (w.batch_begin != sub.batch_begin || w.batch_end != sub.batch_end) {
            return fail("item %d does not cover the batches of subband %d", (int)k, w.o);
        }
        // a grouped item covers the tile of every subband of its group (same size)
        const int nm = w.nm() > 0 ? w.nm() : 1;
        if (nm != (sub.grp > 0 ? sub.grp : 1) || w.o + nm > L.S) return fail("item %d has %d members", (int)k, nm);
        for (int mk = 0; mk < nm; ++mk) {
            const SubbandDev& sm = L.sb[w.o + mk];
            const TileSub& subm = P.subs[w.o + mk];
            if (sm.rows != so.rows || sm.cols != so.cols || subm.TS != sub.TS || subm.batch_begin != sub.batch_begin)
                return fail("item %d member %d differs from the group's first subband", (int)k, mk);
            for (int y = w.ty0; y < std::min(w.ty0 + side, so.rows); ++y)
                for (int x = w.tx0; x < std::min(w.tx0 + side, so.cols); ++x) hit[w.o + mk][(size_t)y * so.cols + x]++;
        }
    }
    for (int o = 0; o < L.S; ++o)
        for (size_t i = 0; i < hit[o].size(); ++i)
            if (hit[o][i] != 1) return fail("output %d of subband %d not produced exactly once", (int)i, o);
    for (int t = 0; t < P.n_split; ++t) {
        auto& v = parts[t];
        std::sort(v.begin(), v.end());
        if (v.size() < 2) return fail("split tile %d has %d parts", t, (int)v.size());
        const TileSub& sub = P.subs[part_sub[t]];
        if (v.front().first != sub.batch_begin || v.back().second != sub.batch_end)
            return fail("split tile %d parts do not cover the batches of subband %d", t, part_sub[t]);
        for (size_t k = 1; k < v.size(); ++k)
            if (v[k].first != v[k - 1].second) return fail("split tile %d parts do not chain at part %d", t, (int)k);
    }
    return std::string();
}

}  // namespace wdb
