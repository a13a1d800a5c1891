"""Fused FISTA loop (one cooperative launch per chunk: kernel 1 and kernel 2 of every
iteration separated by grid barriers) against the two-launch loop and the FP64 oracle
(Algorithm 3), and its bounded barrier wait (WDB_ETIMEOUT)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import solver
from oracle_cases import build_case, fista, precond_and_step, taps_arrays
from paper_1512_08401_gb300 import synthetic

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def wdb():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1512_08401_gb300 import build, wdb as w
    build.build()
    w.lib()
    return w


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).ravel()).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def gpu_from_oracle(wdb, case, n_rows, n_cols, J):
    a, b, oy, ox, v = taps_arrays(case.th)
    return wdb.Theta.from_taps(n_rows, n_cols, "db4", J, a, b, oy, ox, v)


@pytest.mark.parametrize("kind", ["none", "spai"])
def test_fused_trajectory_parity_128(wdb, kind):
    """200 fused iterations against the oracle's Algorithm 3 on the same Theta_K, P and tau."""
    prob = synthetic.small_problem()
    n, J, lam = 128, 4, prob.lam
    case = build_case(prob.psf, n, n, J, 30 * n * n, prob.u0)
    Ptab, P, tau, _ = precond_and_step(case, kind)
    ref = fista(case, lam, P, tau, 200)
    g = gpu_from_oracle(wdb, case, n, n, J)
    g.set_precond(kind, Ptab, tau)
    x = torch.zeros(n * n, device="cuda")
    r = g.solve_coeffs(dev(case.x0), x, lam=lam, max_iters=200, tol=0.0, precond=kind, fused=True)
    xg = host(x)
    assert r["iters"] == 200
    assert np.linalg.norm(xg - ref.x) <= 1e-5 * np.linalg.norm(ref.x)
    assert abs(r["objective"] - ref.objective) <= 1e-5 * ref.objective
    A, _ = solver.theta_ops(case.th)
    E_ora_of_gpu = solver.objective(A(xg) - case.x0, xg, np.full(n * n, lam))
    assert abs(r["objective"] - E_ora_of_gpu) <= 1e-6 * E_ora_of_gpu


@pytest.mark.parametrize("mode", ["autotuned", "super", "grouped", "split"])
def test_fused_equals_two_launch_loop(wdb, mode):
    """Same iterates as the two-launch loop under every plan family (each output is summed by
    one thread in the same order whichever CTA takes its tile; split-tile plans fall back to
    two launches)."""
    prob = synthetic.small_problem()
    n, J = 128, 4
    g = wdb.Theta.build(prob.psf, n, n, "db4", J, K=30 * n * n)
    if mode == "super":
        g.replan(super_tiles=True)
    elif mode == "grouped":
        g.replan(grouped=True)
    elif mode == "split":
        g.replan(split_share=0.5)
    u = dev(prob.u0)
    x1 = torch.zeros(n * n, device="cuda")
    x2 = torch.zeros(n * n, device="cuda")
    r1 = g.solve(u, x1, lam=prob.lam, max_iters=57, check_every=10, precond="spai")
    r2 = g.solve(u, x2, lam=prob.lam, max_iters=57, check_every=10, precond="spai", fused=True)
    assert r1["iters"] == r2["iters"] == 57
    assert torch.equal(x1, x2)
    assert abs(r1["objective"] - r2["objective"]) <= 1e-12 * abs(r1["objective"])


def test_fused_headline_1024_target_stop(wdb):
    """At 1024^2 (the headline operator) the fused loop stops at the same iteration as the
    two-launch loop for an objective target and returns the same iterate."""
    prob = synthetic.headline_problem("gaussian", 0)
    n = 1024
    g = wdb.Theta.build(prob.psf, n, n, "db4", 5, K=30 * n * n)
    u = dev(prob.u0)
    x1 = torch.zeros(n * n, device="cuda")
    x2 = torch.zeros(n * n, device="cuda")
    E = g.solve(u, x1, lam=1e-3, max_iters=400, precond="spai")["objective"]
    r1 = g.solve(u, x1, lam=1e-3, max_iters=2000, precond="spai", target_objective=E * (1 + 1e-4))
    r2 = g.solve(u, x2, lam=1e-3, max_iters=2000, precond="spai", target_objective=E * (1 + 1e-4), fused=True)
    assert r1["first_primal_below"] == r2["first_primal_below"] > 0
    assert r1["iters"] == r2["iters"]
    assert torch.equal(x1, x2)


def test_fused_barrier_timeout_is_reported(wdb):
    """A barrier allowed a single poll gives up (the first CTA to arrive cannot see the last
    one within one poll): the solve returns WDB_ETIMEOUT without a fault, and the handle and
    context stay usable."""
    prob = synthetic.small_problem()
    n, J = 128, 4
    g = wdb.Theta.build(prob.psf, n, n, "db4", J, K=30 * n * n)
    u = dev(prob.u0)
    x = torch.zeros(n * n, device="cuda")
    with pytest.raises(wdb.WdbError) as err:
        g.solve(u, x, lam=prob.lam, max_iters=20, precond="spai", fused=True, spin_limit=1)
    assert err.value.status == 5
    torch.cuda.synchronize()
    x1 = torch.zeros(n * n, device="cuda")
    x2 = torch.zeros(n * n, device="cuda")
    r1 = g.solve(u, x1, lam=prob.lam, max_iters=30, precond="spai")
    r2 = g.solve(u, x2, lam=prob.lam, max_iters=30, precond="spai", fused=True)
    assert r1["iters"] == r2["iters"] == 30
    assert torch.equal(x1, x2)
