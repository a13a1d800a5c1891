"""GPU against the FP64 oracle, element by element, on the paths the kernels take at the
benchmark's sizes.

* J = 5 and J = 6 (256^2 and 512^2, Gaussian and motion blur): up pairs with scale ratios
  r = 16 and 32 read their phase tables from global memory and down pairs with large r gather
  from global memory; each case runs under the autotuned plan (what the solver uses), a
  super-tile plan and the planner's own plan.
* 1024^2, J = 5, both headline blurs: the oracle's operator record
  (oracle/data/theta_1024_<blur>_k30.npz, written by ``python -m oracle.workloads operators``)
  loaded through wdb_theta_from_taps under the autotuned plan the benchmark runs:
  Theta_K y and Theta_K^T r element by element, a 30-iteration FISTA trajectory, and the
  GPU-built operator's taps and SPAI table against the record.
* Batched solve: every problem of a mixed batch against oracle.solver.fista directly.

Tolerances as in test_gpu_parity.py: operator applications max |err| <= 2e-6 max |ref|;
trajectories ||x_gpu - x_ora|| <= 1e-5 ||x_ora|| and |E_gpu - E_ora| <= 1e-5 E_ora.
"""
import os

import numpy as np
import pytest

from oracle import precond, solver, theta, wavelet
from paper_1512_08401_gb300 import synthetic

from oracle_cases import build_case, fista, precond_and_step, taps_arrays

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "data")


@pytest.fixture(scope="module")
def wdb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_08401_gb300 import build, wdb as w
    build.build()
    w.lib()
    return w


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).ravel()).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def rel_max(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def check_apply(wdb, g, mat, matT, N, seed):
    rng = np.random.default_rng(seed)
    y = rng.standard_normal(N)
    out = torch.zeros(N, device="cuda")
    g.apply(dev(y), out)
    e1 = rel_max(host(out), mat @ y)
    g.apply(dev(y), out, transpose=True)
    e2 = rel_max(host(out), matT @ y)
    assert e1 < 2e-6 and e2 < 2e-6, (e1, e2)


# ---------------------------------------------------------------------------------------
# J = 5 and J = 6
# ---------------------------------------------------------------------------------------

DEEP = {
    "gauss256_j5": (lambda: synthetic.gaussian_psf(2.0, 15), 256, 5, "db4"),
    "motion256_j5": (lambda: synthetic.motion_line_psf(11, 0.6), 256, 5, "db4"),
    "gauss512_j6": (lambda: synthetic.gaussian_psf(2.0, 13), 512, 6, "db4"),
    "motion512_j6": (lambda: synthetic.motion_line_psf(9, 1.1), 512, 6, "db4"),
    "skewed256_sym6_j6": (lambda: synthetic.skewed_gaussian_psf(2.5), 256, 6, "sym6"),
}
_deep_cache = {}


def deep_case(name):
    if name not in _deep_cache:
        mk, n, J, wname = DEEP[name]
        psf = mk()
        rng = np.random.default_rng(21)
        u0 = synthetic.blur_fft(synthetic.clean_image(n, n, rng), psf) + 0.01 * rng.standard_normal((n, n))
        _deep_cache[name] = (build_case(psf, n, n, J, 30 * n * n, u0, wavelet_name=wname), n, J, wname)
    return _deep_cache[name]


@pytest.mark.parametrize("name", list(DEEP))
def test_apply_parity_deep_levels_all_plans(wdb, name):
    case, n, J, wname = deep_case(name)
    a, b, oy, ox, v = taps_arrays(case.th)
    g = wdb.Theta.from_taps(n, n, wname, J, a, b, oy, ox, v)
    assert g.info.K_eff == case.th.K_eff
    assert g.info.plan_tuned == 1
    check_apply(wdb, g, case.th.mat, case.th.matT, n * n, 1)           # autotuned plan
    g.replan(32768, 2.0, 0.0, super_tiles=True)
    if name.startswith("gauss"):   # (the motion operators' wider regions may not fit a super tile)
        assert min(g.info.plan_super_subbands) > 0
    check_apply(wdb, g, case.th.mat, case.th.matT, n * n, 2)           # super tiles where they fit
    g.replan()
    check_apply(wdb, g, case.th.mat, case.th.matT, n * n, 3)           # planner plan
    g.replan(grouped=True)
    assert min(g.info.plan_groups) == J
    check_apply(wdb, g, case.th.mat, case.th.matT, n * n, 4)           # grouped items
    g.free()


@pytest.mark.parametrize("name", ["gauss512_j6", "motion256_j5", "skewed256_sym6_j6"])
def test_fista_trajectory_parity_deep_levels(wdb, name):
    case, n, J, wname = deep_case(name)
    Ptab, P, tau, _ = precond_and_step(case, "spai")
    lam = 1e-3
    ref = fista(case, lam, P, tau, 40)
    a, b, oy, ox, v = taps_arrays(case.th)
    g = wdb.Theta.from_taps(n, n, wname, J, a, b, oy, ox, v)
    g.set_precond("spai", Ptab, tau)
    x = torch.zeros(n * n, device="cuda")
    r = g.solve_coeffs(dev(case.x0), x, lam=lam, max_iters=40, tol=0.0, precond="spai")
    xg = host(x)
    assert r["iters"] == 40
    assert np.linalg.norm(xg - ref.x) <= 1e-5 * np.linalg.norm(ref.x)
    assert abs(r["objective"] - ref.objective) <= 1e-5 * ref.objective
    g.free()


# ---------------------------------------------------------------------------------------
# 1024^2 headline operators (oracle record)
# ---------------------------------------------------------------------------------------

_rec_cache = {}


def record(blur):
    if blur not in _rec_cache:
        z = np.load(os.path.join(DATA, f"theta_1024_{blur}_k30.npz"))
        rec = {k: z[k] for k in z.files}
        n, J = int(rec["n"]), int(rec["levels"])
        lay = wavelet.layout(n, n, J)
        t = theta.Taps(rec["a"], rec["b"], rec["oy"], rec["ox"], rec["v"], np.zeros(len(rec["v"]), np.int64))
        mat = theta.theta_sparse(t, lay, n * n)
        rec["mat"], rec["matT"], rec["lay"] = mat, mat.T.tocsr(), lay
        _rec_cache[blur] = rec
    return _rec_cache[blur]


@pytest.mark.parametrize("blur", ["gaussian", "motion"])
def test_headline_1024_apply_elementwise(wdb, blur):
    rec = record(blur)
    n, J = int(rec["n"]), int(rec["levels"])
    g = wdb.Theta.from_taps(n, n, "db4", J, rec["a"], rec["b"], rec["oy"], rec["ox"], rec["v"])
    assert g.info.K_eff == int(rec["K_eff"]) and g.info.plan_tuned == 1
    check_apply(wdb, g, rec["mat"], rec["matT"], n * n, 7)
    g.free()


@pytest.mark.parametrize("blur", ["gaussian", "motion"])
def test_headline_1024_trajectory_30(wdb, blur):
    rec = record(blur)
    n, J = int(rec["n"]), int(rec["levels"])
    prob = synthetic.headline_problem(blur)
    x0 = wavelet.dwt2(prob.u0, "db4", J)
    lay = rec["lay"]
    per = precond.theta_periods(lay, J)
    P = precond.expand(rec["P_spai"], lay, per)
    tau = float(rec["tau_spai"])
    w = np.full(n * n, prob.lam)
    mat, matT = rec["mat"], rec["matT"]
    ref = solver.fista(lambda v: mat @ v, lambda v: matT @ v, x0, w, P, tau, 30)
    g = wdb.Theta.from_taps(n, n, "db4", J, rec["a"], rec["b"], rec["oy"], rec["ox"], rec["v"])
    g.set_precond("spai", rec["P_spai"], tau)
    x = torch.zeros(n * n, device="cuda")
    r = g.solve(dev(prob.u0), x, lam=prob.lam, max_iters=30, tol=0.0, precond="spai")
    xg = host(x)
    assert r["iters"] == 30
    assert np.linalg.norm(xg - ref.x) <= 1e-5 * np.linalg.norm(ref.x)
    assert abs(r["objective"] - ref.objective) <= 1e-5 * ref.objective
    g.free()


@pytest.mark.parametrize("blur", ["gaussian", "motion"])
def test_headline_1024_gpu_built_operator_against_record(wdb, blur):
    """wdb_build_theta at full size: the kept taps (values within 1e-12 max |Theta|; the kept
    sets may differ only by taps whose score lies within 1e-9 of the selection boundary, the
    two sides computing the probes with different rounding), the SPAI table and the step
    against the oracle's."""
    rec = record(blur)
    n, J = int(rec["n"]), int(rec["levels"])
    prob = synthetic.headline_problem(blur)
    g = wdb.Theta.build(prob.psf, n, n, "db4", J, K=int(rec["K_requested"]))
    assert g.info.K_eff == int(rec["K_eff"]) and g.info.n_taps == len(rec["v"])
    a, b, oy, ox, v = g.export_taps()
    ko = {(int(rec["a"][i]), int(rec["b"][i]), int(rec["oy"][i]), int(rec["ox"][i])): rec["v"][i]
          for i in range(len(rec["v"]))}
    kg = {(int(a[i]), int(b[i]), int(oy[i]), int(ox[i])): v[i] for i in range(len(v))}
    vmax = np.abs(rec["v"]).max()
    common = set(ko) & set(kg)
    assert len(common) >= len(ko) - 8
    assert max(abs(kg[k] - ko[k]) for k in common) <= 1e-12 * vmax
    lev = np.array([s.level for s in rec["lay"]], dtype=float)
    boundary = min(abs(val) * 2.0 ** lev[k[1]] for k, val in ko.items())
    for k in set(ko) ^ set(kg):
        val = kg.get(k, ko.get(k))
        assert abs(abs(val) * 2.0 ** lev[k[1]] - boundary) <= 1e-9 * boundary, k
    pc = g.precond("spai")
    assert np.abs(pc["P"] - rec["P_spai"]).max() <= 1e-10 * rec["P_spai"].max()
    assert abs(pc["tau"] - float(rec["tau_spai"])) <= 1e-6 * float(rec["tau_spai"])
    g.free()


# ---------------------------------------------------------------------------------------
# Batched solve against the oracle
# ---------------------------------------------------------------------------------------

def test_batch_against_oracle(wdb):
    specs = [(64, 3, synthetic.gaussian_psf(1.5, 9), 1e-3, 60),
             (128, 4, synthetic.motion_line_psf(9, 0.4), 2e-3, 80),
             (256, 5, synthetic.gaussian_psf(2.0, 13), 5e-4, 100)]
    rng = np.random.default_rng(41)
    ths, us, kw, refs = [], [], [], []
    for n, J, psf, lam, iters in specs:
        u0 = synthetic.blur_fft(synthetic.clean_image(n, n, rng), psf) + 0.01 * rng.standard_normal((n, n))
        case = build_case(psf, n, n, J, 30 * n * n, u0)
        Ptab, P, tau, _ = precond_and_step(case, "spai")
        refs.append(fista(case, lam, P, tau, iters))
        a, b, oy, ox, v = taps_arrays(case.th)
        g = wdb.Theta.from_taps(n, n, "db4", J, a, b, oy, ox, v)
        g.set_precond("spai", Ptab, tau)
        ths.append(g)
        us.append(dev(u0))
        kw.append(dict(lam=lam, max_iters=iters, precond="spai"))
    xs = [torch.zeros(t.N, device="cuda") for t in ths]
    res = wdb.solve_batch(ths, us, xs, kw)
    for r, x, ref, k in zip(res, xs, refs, kw):
        xg = host(x)
        assert r["iters"] == k["max_iters"]
        assert np.linalg.norm(xg - ref.x) <= 1e-5 * np.linalg.norm(ref.x)
        assert abs(r["objective"] - ref.objective) <= 1e-5 * ref.objective
    for g in ths:
        g.free()
