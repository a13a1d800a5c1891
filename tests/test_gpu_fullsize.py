"""The benchmark's full-size workloads against the oracle.

1024^2 headline (Gaussian sigma = 3 on 31x31, db4 J = 5, lambda = 1e-3, K = 30N, SPAI), in
the launch configuration bench.py times (CUDA graphs, checks every 10 iterations): the
integer results of the tap selection (K_eff, number of taps) exactly, the step tau, the
minimum E* and the iteration count to E*(1 + 1e-4) against the record the FP64 oracle wrote
(`python -m oracle.workloads headline`, oracle/data/headline_1024_gauss_k30_spai.json).

4096^2 (Gaussian sigma = 4 on 41x41, J = 6, K = 30N): a property that holds at any size,
<Theta_K x, y> = <x, Theta_K^T y>, so the two FISTA operators are each other's transpose on
the full-size plans; and sampled taps against the oracle's single entries, the selection at
sampled neighbours of kept taps, and sampled outputs of both kernels against FP64 sums."""
import json
import os

import numpy as np
import pytest

from paper_1512_08401_gb300 import synthetic

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
RECORD = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "data",
                      "headline_1024_gauss_k30_spai.json")


@pytest.fixture(scope="module")
def wdb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_08401_gb300 import build, wdb as w
    build.build()
    w.lib()
    return w


def test_headline_1024_against_oracle_record(wdb):
    rec = json.load(open(RECORD))
    prob = synthetic.headline_problem("gaussian", 0)
    n, J = rec["n"], rec["levels"]
    th = wdb.Theta.build(prob.psf, n, n, "db4", J, K=rec["K_requested"])
    assert th.info.K_eff == rec["K_eff"] and th.info.n_taps == rec["n_taps"]
    pc = th.precond("spai")
    assert abs(pc["tau"] - rec["tau"]) <= 1e-6 * rec["tau"]
    u = torch.from_numpy(prob.u0.astype(np.float32).ravel()).cuda()
    x = torch.zeros(n * n, device="cuda")
    r = th.solve(u, x, lam=rec["lambda"], max_iters=3000, precond="spai")
    lo, hi = rec["E_star_lower"], rec["E_star_upper"]
    # FP32 iterates: the minimum within 1e-6 relative of the oracle's bracket
    assert lo * (1 - 1e-6) <= r["objective"] <= hi * (1 + 1e-6), (r["objective"], lo, hi)
    x.zero_()
    r = th.solve(u, x, lam=rec["lambda"], max_iters=500, precond="spai", target_objective=hi * (1 + 1e-4))
    assert abs(r["first_primal_below"] - rec["iters_to_rel_1e-4"]) <= 1, (r["first_primal_below"], rec)


def test_4096_operators_are_adjoint(wdb):
    prob = synthetic.large_problem()
    n = 4096
    th = wdb.Theta.build(prob.psf, n, n, "db4", 6, K=30 * n * n)
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn(n * n, device="cuda", generator=g)
    y = torch.randn(n * n, device="cuda", generator=g)
    ax = torch.empty_like(x)
    aty = torch.empty_like(y)
    th.apply(x, ax)
    th.apply(y, aty, transpose=True)
    lhs = torch.dot(ax.double(), y.double()).item()
    rhs = torch.dot(x.double(), aty.double()).item()
    scale = (torch.linalg.vector_norm(ax.double()) * torch.linalg.vector_norm(y.double())).item()
    assert abs(lhs - rhs) <= 1e-5 * scale, (lhs, rhs, scale)
    th.free()


def test_4096_sampled_taps_selection_and_outputs(wdb):
    """4096^2, J = 6, K = 30N at full size, by sampling:
    * values: kept taps against the oracle's single entries (theta.theta_entry, Eq. matrixH
      from the separable 1-D factors), to 1e-12 max|Theta| (both FP64);
    * selection (Sec. 3.7): neighbouring taps (offsets +-1, +-2) that were not kept score at
      most the smallest kept score (1e-9 slack for the two FP64 computations);
    * kernels: Theta_K x and Theta_K^T x in FP32 at sampled outputs against an FP64 sum over
      the exported taps (circulant rule of Algorithm 2)."""
    from oracle import theta as TH
    from oracle.wavelet import layout
    prob = synthetic.large_problem()
    n, J = 4096, 6
    th = wdb.Theta.build(prob.psf, n, n, "db4", J, K=30 * n * n)
    a, b, oy, ox, v = th.export_taps()
    lay = layout(n, n, J)
    lev = np.array([s.level for s in lay])
    vmax = th.info.theta_max_abs
    score = np.abs(v) * 2.0 ** lev[b]
    smin = score.min()
    kept = set(zip(a.tolist(), b.tolist(), oy.tolist(), ox.tolist()))
    rng = np.random.default_rng(13)

    def entry(ai, bi, o_y, o_x):
        sa, sb = lay[ai], lay[bi]
        if sa.level <= sb.level:   # column form: p = o + r q at q = 0
            return TH.theta_entry(prob.psf, n, n, "db4", J, ai, (o_y, o_x), bi, (0, 0))
        return TH.theta_entry(prob.psf, n, n, "db4", J, ai, (0, 0), bi, (o_y, o_x))

    pairs = sorted(set(zip(a.tolist(), b.tolist())))
    picks = [rng.choice(np.nonzero((a == pa) & (b == pb))[0]) for pa, pb in
             [pairs[i] for i in rng.choice(len(pairs), size=min(40, len(pairs)), replace=False)]]
    for t in picks:
        ref = entry(int(a[t]), int(b[t]), int(oy[t]), int(ox[t]))
        assert abs(ref - v[t]) <= 1e-12 * vmax, (t, ref, v[t])
        sa, sb = lay[a[t]], lay[b[t]]
        rows, cols = (sa.rows, sa.cols) if sa.level <= sb.level else (sb.rows, sb.cols)
        for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0), (0, 2), (2, 0)):
            cand = (int(a[t]), int(b[t]), (int(oy[t]) + dy) % rows, (int(ox[t]) + dx) % cols)
            if cand in kept:
                continue
            sc = abs(entry(*cand)) * 2.0 ** lay[cand[1]].level
            assert sc <= smin * (1 + 1e-9), (cand, sc, smin)
    # FP32 kernels at sampled outputs against FP64 sums over the exported taps
    x = np.random.default_rng(3).standard_normal(n * n).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    y = torch.empty_like(xd)
    yt = torch.empty_like(xd)
    th.apply(xd, y)
    th.apply(xd, yt, transpose=True)
    y, yt = y.cpu().numpy(), yt.cpu().numpy()
    x64 = x.astype(np.float64)
    for _ in range(12):
        o = int(rng.integers(len(lay)))
        so = lay[o]
        py, px = int(rng.integers(so.rows)), int(rng.integers(so.cols))
        ref, reft = 0.0, 0.0
        for t in range(len(v)):
            sa, sb = lay[a[t]], lay[b[t]]
            if a[t] == o:      # row of Theta_K: entries ((o, p), (b, q))
                if sa.level <= sb.level:
                    r = 1 << (sb.level - sa.level)
                    dy, dx = (py - oy[t]) % sa.rows, (px - ox[t]) % sa.cols
                    if dy % r == 0 and dx % r == 0:
                        ref += v[t] * x64[sb.offset + (dy // r) * sb.cols + dx // r]
                else:
                    r = 1 << (sa.level - sb.level)
                    qy, qx = (oy[t] + r * py) % sb.rows, (ox[t] + r * px) % sb.cols
                    ref += v[t] * x64[sb.offset + qy * sb.cols + qx]
            if b[t] == o:      # row of Theta_K^T: entries ((a, p'), (o, p))
                if sa.level <= sb.level:
                    r = 1 << (sb.level - sa.level)
                    qy, qx = (oy[t] + r * py) % sa.rows, (ox[t] + r * px) % sa.cols
                    reft += v[t] * x64[sa.offset + qy * sa.cols + qx]
                else:
                    r = 1 << (sa.level - sb.level)
                    dy, dx = (py - oy[t]) % sb.rows, (px - ox[t]) % sb.cols
                    if dy % r == 0 and dx % r == 0:
                        reft += v[t] * x64[sa.offset + (dy // r) * sa.cols + dx // r]
        i = so.offset + py * so.cols + px
        assert abs(y[i] - ref) <= 1e-5 * max(1.0, abs(ref)), (o, py, px, y[i], ref)
        assert abs(yt[i] - reft) <= 1e-5 * max(1.0, abs(reft)), (o, py, px, yt[i], reft)
    th.free()
