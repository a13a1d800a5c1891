"""Oracle pipelines for the parity tests (calls only oracle/ and the shared input generator)."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from oracle import precond, solver, theta, wavelet


@dataclass
class OracleCase:
    th: theta.ThetaK
    x0: np.ndarray
    periods: list
    Md: np.ndarray
    M2d: np.ndarray


def build_case(psf, n_rows, n_cols, J, K, u0, rule="weighted", wavelet_name="db4") -> OracleCase:
    th = theta.build_theta(psf, n_rows, n_cols, wavelet_name, J, K, rule)
    x0 = wavelet.dwt2(u0, wavelet_name, J)
    per = precond.theta_periods(th.lay, J)
    Md, M2d = precond.diagonal_tables(th.mat, th.matT, th.lay, per)
    return OracleCase(th, x0, per, Md, M2d)


def precond_and_step(case: OracleCase, kind: str, jacobi_eps=None):
    Ptab = precond.preconditioner(case.Md, case.M2d, kind, jacobi_eps)
    P = precond.expand(Ptab, case.th.lay, case.periods)
    A, At = solver.theta_ops(case.th)
    L, _ = precond.power_iteration(lambda v: At(A(v)), P)
    return Ptab, P, precond.step_size(L), L


def fista(case: OracleCase, lam, P, tau, iters, tol=0.0, check_every=10, x0=None):
    A, At = solver.theta_ops(case.th)
    b = case.x0 if x0 is None else x0
    w = np.full(len(b), lam)
    return solver.fista(A, At, b, w, P, tau, iters, tol=tol, check_every=check_every)


def taps_arrays(th: theta.ThetaK):
    t = th.taps
    return (t.a.astype(np.int32), t.b.astype(np.int32), t.oy.astype(np.int32), t.ox.astype(np.int32),
            t.v.astype(np.float64))
