"""Batched solve (several problems of uneven size advanced by shared launches) against the
single-problem solves of the same operators, and so, transitively, against the oracle."""
import numpy as np
import pytest

from paper_1512_08401_gb300 import synthetic

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def wdb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_08401_gb300 import build, wdb as w
    build.build()
    w.lib()
    return w


def problems():
    rng = np.random.default_rng(31)
    specs = [(64, 64, 3, synthetic.gaussian_psf(1.5, 9), 1e-3), (128, 128, 4, synthetic.motion_line_psf(9, 0.4), 2e-3),
             (48, 80, 3, synthetic.gaussian_psf(1.2, 7), 5e-4), (128, 128, 4, synthetic.gaussian_psf(2.5, 15), 1e-3)]
    out = []
    for nr, nc, J, psf, lam in specs:
        u0 = synthetic.blur_fft(synthetic.clean_image(nr, nc, rng), psf) + 0.01 * rng.standard_normal((nr, nc))
        out.append((nr, nc, J, psf, lam, u0))
    return out


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).ravel()).cuda()


def test_batch_matches_single_solves(wdb):
    P = problems()
    th = [wdb.Theta.build(psf, nr, nc, "db4", J, K=30 * nr * nc) for nr, nc, J, psf, lam, u0 in P]
    us = [dev(u0) for *_, u0 in P]
    kw = [dict(lam=lam, max_iters=120 + 10 * i, precond="spai") for i, (*_, lam, u0) in enumerate(P)]
    singles = []
    for t, u, k in zip(th, us, kw):
        x = torch.zeros(t.N, device="cuda")
        r = t.solve(u, x, **k)
        singles.append((r, x.clone()))
    xs = [torch.zeros(t.N, device="cuda") for t in th]
    res = wdb.solve_batch(th, us, xs, kw)
    for (r1, x1), r2, x2, k in zip(singles, res, xs, kw):
        assert r2["iters"] == k["max_iters"] == r1["iters"]
        d = (x2 - x1).abs().max().item()
        assert d <= 1e-6 * x1.abs().max().item()
        assert abs(r2["objective"] - r1["objective"]) <= 1e-6 * r1["objective"]


def test_batch_per_problem_targets(wdb):
    # each problem stops on its own objective target (the paper's protocol, Sec. 5.4)
    P = problems()
    th = [wdb.Theta.build(psf, nr, nc, "db4", J, K=30 * nr * nc) for nr, nc, J, psf, lam, u0 in P]
    us = [dev(u0) for *_, u0 in P]
    kw = []
    stops = []
    for i, (t, u, (*_, lam, u0)) in enumerate(zip(th, us, P)):
        x = torch.zeros(t.N, device="cuda")
        star = t.solve(u, x, lam=lam, max_iters=2000, precond="spai")
        target = star["objective"] * (1 + 10.0 ** -(2 + i))
        r = t.solve(u, x, lam=lam, max_iters=2000, precond="spai", target_objective=target)
        kw.append(dict(lam=lam, max_iters=2000, precond="spai", target_objective=target))
        stops.append(r["first_primal_below"])
    xs = [torch.zeros(t.N, device="cuda") for t in th]
    res = wdb.solve_batch(th, us, xs, kw)
    for r, k0, k in zip(res, stops, kw):
        assert abs(r["first_primal_below"] - k0) <= 1
        assert r["objective"] <= k["target_objective"] * (1 + 1e-6)
    assert len(set(stops)) > 1   # the problems really stop at different iterations


def test_batch_rejects_shared_handle(wdb):
    nr, nc, J, psf, lam, u0 = problems()[0]
    t = wdb.Theta.build(psf, nr, nc, "db4", J, K=30 * nr * nc)
    u = dev(u0)
    with pytest.raises(wdb.WdbError):
        wdb.solve_batch([t, t], [u, u], [torch.zeros(t.N, device="cuda")] * 2, [dict(lam=lam)] * 2)
