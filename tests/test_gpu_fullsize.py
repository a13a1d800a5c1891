"""The benchmark's full-size workloads against the oracle.

1024^2 headline (Gaussian sigma = 3 on 31x31, db4 J = 5, lambda = 1e-3, K = 30N, SPAI), in
the launch configuration bench.py times (CUDA graphs, checks every 10 iterations): the
integer results of the tap selection (K_eff, number of taps) exactly, the step tau, the
minimum E* and the iteration count to E*(1 + 1e-4) against the record the FP64 oracle wrote
(`python -m oracle.workloads headline`, oracle/data/headline_1024_gauss_k30_spai.json).

4096^2 (Gaussian sigma = 4 on 41x41, J = 6, K = 30N): a property that holds at any size,
<Theta_K x, y> = <x, Theta_K^T y>, so the two FISTA operators are each other's transpose on
the full-size plans."""
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
