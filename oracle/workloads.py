"""Reference optimum E* and iteration counts of the benchmark workloads, computed by the
FP64 oracle only, written to oracle/data/<name>.json.

    python -m oracle.workloads headline [--workers 8] [--iters 6000]
    python -m oracle.workloads operators [--workers 8]

Workload "headline": 1024 x 1024 synthetic image (Gaussian sigma = 3 on 31 x 31, noise 0.01),
db4, J = 5, lambda = 1e-3, Theta_K with K = 30 N (weighted rule, Sec. 3.7), SPAI
preconditioner (Sec. 4.3), FISTA (Algorithm 3) from x = 0.

Workload "operators": the Theta_K operators of the 1024 x 1024 problems (Gaussian sigma = 3 on
31 x 31 and the seeded 21 px motion line; db4, J = 5, K = 30 N, weighted rule) as the oracle
builds them, with the SPAI table (Sec. 4.3), L and tau, written to
oracle/data/theta_1024_<blur>_k30.npz; the full-size parity tests read them so that they do not
rebuild the operator in every run.

Recorded (headline): E* bracket [best dual value, best primal value] of the run, the first iteration
whose primal value at y^(k) is within 1e-4 (relative) of E*, the same for the paper's
criterion E - E* <= 1e-3 E(x^(0)) (Sec. 5.4), and the oracle's own time per iteration.

TEST INFRASTRUCTURE: a script of the oracle; it imports nothing outside oracle/ except the
shared seeded input generator.
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time
from concurrent.futures import ProcessPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import precond, solver, theta, wavelet  # noqa: E402
from paper_1512_08401_gb300 import synthetic  # noqa: E402

DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")


def headline(workers: int = 8, iters: int = 6000, kn: int = 30, kind: str = "spai") -> dict:
    prob = synthetic.headline_problem("gaussian")
    n, J, lam = 1024, 5, prob.lam
    t0 = time.time()
    ctx = mp.get_context("spawn")
    with ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as pool:
        th = theta.build_theta(prob.psf, n, n, "db4", J, kn * n * n, "weighted", pool=pool)
    t_build = time.time() - t0
    x0 = wavelet.dwt2(prob.u0, "db4", J)
    per = precond.theta_periods(th.lay, J)
    t1 = time.time()
    Md, M2d = precond.diagonal_tables(th.mat, th.matT, th.lay, per)
    Ptab = precond.preconditioner(Md, M2d, kind)
    P = precond.expand(Ptab, th.lay, per)
    A, At = solver.theta_ops(th)
    L, pit = precond.power_iteration(lambda v: At(A(v)), P)
    tau = precond.step_size(L)
    t_setup = time.time() - t1
    w = np.full(n * n, lam)
    t2 = time.time()
    res = solver.fista(A, At, x0, w, P, tau, iters, record_every=1)
    t_fista = time.time() - t2
    hist = np.array(res.history)          # (k, primal(y_k), gap(y_k))
    primal = hist[:, 1]
    dual = primal - hist[:, 2]
    E_up = float(min(primal.min(), res.objective))
    E_low = float(dual.max())
    E0 = 0.5 * float(x0 @ x0)             # E(x^(0)) with x^(0) = 0
    rel = (primal - E_up) / E_up
    n_it = int(hist[np.argmax(rel <= 1e-4), 0]) if (rel <= 1e-4).any() else -1
    paper = (primal - E_up) <= 1e-3 * E0
    n_it_paper = int(hist[np.argmax(paper), 0]) if paper.any() else -1
    out = {
        "workload": "1024x1024 gaussian sigma=3 31x31, db4 J=5, lambda=1e-3, K=%dN weighted, %s" % (kn, kind),
        "n": n, "levels": J, "lambda": lam, "K_requested": kn * n * n, "K_eff": th.K_eff,
        "n_taps": len(th.taps), "precond": kind, "L_hat": L, "power_iters": pit, "tau": tau,
        "E_star_upper": E_up, "E_star_lower": E_low, "E0": E0,
        "iters_run": int(res.iters), "iters_to_rel_1e-4": n_it, "iters_to_paper_1e-3_E0": n_it_paper,
        "oracle_ms_per_iter": 1e3 * t_fista / res.iters, "oracle_build_s": t_build, "oracle_setup_s": t_setup,
        "rel_gap_curve_every_10": [[int(k), float(r)] for k, r in zip(hist[9::10, 0], rel[9::10])],
    }
    return out


def operator_record(blur: str, workers: int = 8, kn: int = 30, kind: str = "spai") -> dict:
    """Theta_K of the 1024^2 `blur` problem with its SPAI table, L and tau (oracle only)."""
    prob = synthetic.headline_problem(blur)
    n, J = 1024, 5
    ctx = mp.get_context("spawn")
    with ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as pool:
        th = theta.build_theta(prob.psf, n, n, "db4", J, kn * n * n, "weighted", pool=pool)
    per = precond.theta_periods(th.lay, J)
    Md, M2d = precond.diagonal_tables(th.mat, th.matT, th.lay, per)
    Ptab = precond.preconditioner(Md, M2d, kind)
    P = precond.expand(Ptab, th.lay, per)
    A, At = solver.theta_ops(th)
    L, pit = precond.power_iteration(lambda v: At(A(v)), P)
    t = th.taps
    return {"a": t.a.astype(np.int32), "b": t.b.astype(np.int32), "oy": t.oy.astype(np.int32),
            "ox": t.ox.astype(np.int32), "v": t.v, "n": n, "levels": J, "K_requested": kn * n * n,
            "K_eff": th.K_eff, "Md": Md, "M2d": M2d, "P_spai": Ptab, "L_spai": L, "tau_spai": precond.step_size(L),
            "power_iters": pit}


def main():
    name = sys.argv[1] if len(sys.argv) > 1 else "headline"
    workers = int(sys.argv[sys.argv.index("--workers") + 1]) if "--workers" in sys.argv else 8
    iters = int(sys.argv[sys.argv.index("--iters") + 1]) if "--iters" in sys.argv else 6000
    if name == "operators":
        os.makedirs(DATA, exist_ok=True)
        for blur in ("gaussian", "motion"):
            rec = operator_record(blur, workers)
            path = os.path.join(DATA, f"theta_1024_{blur}_k30.npz")
            np.savez_compressed(path, **rec)
            print(path, len(rec["v"]), rec["K_eff"], rec["L_spai"], rec["tau_spai"])
        return
    if name != "headline":
        raise SystemExit(f"unknown workload {name}")
    out = headline(workers, iters)
    os.makedirs(DATA, exist_ok=True)
    path = os.path.join(DATA, "headline_1024_gauss_k30_spai.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(path, {k: v for k, v in out.items() if k != "rel_gap_curve_every_10"})


if __name__ == "__main__":
    main()
