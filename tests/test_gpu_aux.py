"""FP64 optimality check, error statuses and operator files, through the C ABI.

* wdb_theta_kkt / params.kkt_check: r = Theta_K x - x0 and g = Theta_K^T r in FP64 on the
  device from the FP32 iterate; its KKT residuals, objective and duality gap against the
  oracle's (oracle.solver.kkt_residuals, duality_gap) evaluated on the same x and x0, to
  1e-9 (both sides FP64 with the same taps: only the summation order differs).
* Errors made on the host: a NaN in the observed image gives WDB_ENAN; a step 100 times too
  long for the operator (set through wdb_theta_set_precond) makes the objective grow and
  gives WDB_EDIVERGED. No kernel faults or waits forever in either case.
* wdb_theta_save / wdb_theta_load: the same taps and the same solve.
"""
import os

import numpy as np
import pytest

from oracle import solver
from paper_1512_08401_gb300 import synthetic

from oracle_cases import build_case, fista, precond_and_step, taps_arrays

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


@pytest.fixture(scope="module")
def small():
    prob = synthetic.small_problem()
    n, J = 128, 4
    case = build_case(prob.psf, n, n, J, 30 * n * n, prob.u0)
    Ptab, P, tau, _ = precond_and_step(case, "spai")
    return prob, case, Ptab, P, tau


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).ravel()).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def gpu_op(wdb, case, Ptab, tau, n=128, J=4):
    a, b, oy, ox, v = taps_arrays(case.th)
    g = wdb.Theta.from_taps(n, n, "db4", J, a, b, oy, ox, v)
    g.set_precond("spai", Ptab, tau)
    return g


@pytest.mark.parametrize("iters", [20, 200, 3000])
def test_kkt_and_gap_fp64_against_oracle(wdb, small, iters):
    prob, case, Ptab, P, tau = small
    n, lam = 128, prob.lam
    g = gpu_op(wdb, case, Ptab, tau)
    x0f = case.x0.astype(np.float32).astype(np.float64)     # the x0 the library is given
    x = torch.zeros(n * n, device="cuda")
    r = g.solve_coeffs(dev(x0f), x, lam=lam, max_iters=iters, tol=0.0, precond="spai", kkt_check=True)
    xg = host(x)
    A, At = solver.theta_ops(case.th)
    w = np.full(n * n, lam)
    off, on = solver.kkt_residuals((A, At), xg, x0f, w)
    res = A(xg) - x0f
    pr, _, gap = solver.duality_gap(res, At(res), xg, x0f, w)
    assert abs(r["kkt_off"] - off) <= 1e-9 * max(1.0, off), (r["kkt_off"], off)
    assert abs(r["kkt_on"] - on) <= 1e-9 * max(1.0, on), (r["kkt_on"], on)
    assert abs(r["gap64"] - gap) <= 1e-9 * pr and abs(r["rel_gap64"] - gap / pr) <= 1e-9
    k = g.kkt(x, dev(x0f), lam=lam)
    for a_, b_ in ((k["kkt_off"], r["kkt_off"]), (k["kkt_on"], r["kkt_on"]), (k["gap"], r["gap64"])):
        assert abs(a_ - b_) <= 1e-12 * max(1.0, abs(b_))
    assert abs(k["objective"] - pr) <= 1e-12 * pr and k["support"] == int(np.count_nonzero(xg))
    if iters == 3000:
        # at convergence the conditions hold up to the resolution of the FP32 iteration, two
        # terms (relative to w):
        #  * the step: an iterate stops moving once (tau / P)(g + w sign x) is below half an
        #    ulp of x, so g can stay ulp(x) P / (2 tau) away; twice that is taken (FISTA's
        #    momentum does not settle exactly);
        #  * the residual: kernel 1 forms r = Theta_K x - x0 in FP32 from terms of size
        #    |x0| (cancellation), so r carries about ulp(max|x0|) per entry and the
        #    library's g differs from the FP64 g by up to ulp(max|x0|) times the largest
        #    column sum of |Theta_K|
        ulp_x = float(np.max(np.spacing(np.abs(xg).astype(np.float32))))
        ulp_x0 = float(np.spacing(np.float32(np.abs(x0f).max())))
        colsum = float(np.asarray(abs(case.th.mat).sum(axis=0)).max())
        floor = (ulp_x * float(np.max(P)) / tau + ulp_x0 * colsum) / lam
        assert off <= floor and on <= floor, (off, on, floor)
    g.free()


def test_kkt_of_oracle_solution_is_zero_on_gpu(wdb, small):
    """The oracle's own FP64 minimiser, rounded to FP32, checked by the library: residuals at
    the FP32 rounding floor, and the gap of the returned objective consistent with E*."""
    prob, case, Ptab, P, tau = small
    n, lam = 128, prob.lam
    star = fista(case, lam, P, tau, 20000, tol=1e-12, check_every=50)
    g = gpu_op(wdb, case, Ptab, tau)
    x0f = case.x0.astype(np.float32).astype(np.float64)
    k = g.kkt(dev(star.x), dev(x0f), lam=lam)
    assert k["kkt_off"] <= 2e-3 and k["kkt_on"] <= 2e-3
    assert k["gap"] >= 0.0
    g.free()


def test_nan_in_image_gives_enan(wdb, small):
    prob, case, Ptab, P, tau = small
    n = 128
    g = gpu_op(wdb, case, Ptab, tau)
    u = prob.u0.copy()
    u[17, 33] = np.nan                                      # injected on the host
    x = torch.zeros(n * n, device="cuda")
    with pytest.raises(wdb.WdbError) as e:
        g.solve(dev(u), x, lam=prob.lam, max_iters=50, precond="spai")
    assert e.value.status == 4
    # the handle stays usable
    r = g.solve(dev(prob.u0), x, lam=prob.lam, max_iters=50, precond="spai")
    assert r["iters"] == 50 and np.isfinite(r["objective"])
    g.free()


def test_step_too_long_gives_ediverged(wdb, small):
    prob, case, Ptab, P, tau = small
    n = 128
    g = gpu_op(wdb, case, Ptab, 100.0 * tau)                # injected on the host
    x = torch.zeros(n * n, device="cuda")
    with pytest.raises(wdb.WdbError) as e:
        g.solve(dev(prob.u0), x, lam=prob.lam, max_iters=500, precond="spai")
    assert e.value.status == 6
    g.set_precond("spai", Ptab, tau)
    r = g.solve(dev(prob.u0), x, lam=prob.lam, max_iters=50, precond="spai")
    assert r["iters"] == 50 and np.isfinite(r["objective"])
    g.free()


def test_theta_save_load_round_trip(wdb, tmp_path):
    prob = synthetic.small_problem()
    n, J = 128, 4
    g = wdb.Theta.build(prob.psf, n, n, "db4", J, K=30 * n * n)
    path = os.path.join(str(tmp_path), "theta.wdb")
    g.save(path)
    h = wdb.Theta.load(path)
    ta, tb = g.export_taps(), h.export_taps()
    for p, q in zip(ta, tb):
        assert np.array_equal(p, q)
    assert h.info.K_eff == g.info.K_eff and h.info.levels == J
    u = dev(prob.u0)
    x1 = torch.zeros(n * n, device="cuda")
    x2 = torch.zeros(n * n, device="cuda")
    r1 = g.solve(u, x1, lam=prob.lam, max_iters=80, precond="spai")
    r2 = h.solve(u, x2, lam=prob.lam, max_iters=80, precond="spai")
    assert r1["iters"] == r2["iters"] == 80
    assert abs(r1["tau"] - r2["tau"]) <= 1e-12 * r1["tau"]
    assert (x1 - x2).abs().max().item() <= 1e-6 * x1.abs().max().item()
    assert abs(r1["objective"] - r2["objective"]) <= 1e-6 * r1["objective"]
    with pytest.raises(wdb.WdbError) as e:
        wdb.Theta.load(os.path.join(str(tmp_path), "missing.wdb"))
    assert e.value.status == 8
    g.free()
    h.free()
