"""Preconditioned FISTA on the wavelet coefficients, objective, duality gap and KKT, float64.

Paper passages followed:
  * Eq. l1problem / defF / def:G (Sec. 1.1): E(x) = 1/2||A x - b||^2 + sum_i w_i |x_i|.
  * Eq. l1problemThetaApprox and Eq. gradientapprox (Sec. 1.3): A = Theta_K, b = x0 = Psi* u0,
    grad F_K(y) = Theta_K^T (Theta_K y - x0).
  * Algorithm 3 (Sec. 4): x^(0) = y^(1) = x_init; for k >= 1
        x^(k)   = Prox^P_{tau G}(y^(k) - tau P^{-1} grad F(y^(k)))
        y^(k+1) = x^(k) + (k-1)/(k+2) (x^(k) - x^(k-1)).
    The data term printed there as u0 is read as x0 (the problem being solved is
    Eq. l1problemThetaApprox).
  * Eq. defProxP with diagonal P: per-coordinate soft threshold at tau w_i / P_i.
  * Algorithm 1 with the exact gradient (Sec. 5.2: two FFTs, two wavelet transforms): the
    same iteration with A = H Psi, b = u0; here H is applied by direct convolution.

Readings taken where the paper is silent:
  * Stopping certificate (the paper's rule needs E(x*) in advance): at check iterations
    k = m, 2m, ... the duality gap of y^(k) is formed from the residual r = A y - b and
    g = A^T r already computed for the step: primal Pr = 1/2||r||^2 + sum w|y|; dual point
    theta = s r with s = min(1, min_i w_i/|g_i|); D = -s<b, r> - s^2/2 ||r||^2;
    gap = Pr - D >= 0. The loop stops when gap/Pr <= tol and returns x^(k), whose
    objective is <= that of y^(k) because a proximal gradient step with tau <= 1/L does
    not increase E.

TEST INFRASTRUCTURE: only tests, smoke() and the bench CPU baseline use this module.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .blur import conv_adjoint, conv_periodic
from .wavelet import dwt2, idwt2


def soft(z: np.ndarray, t) -> np.ndarray:
    """Soft threshold sign(z) max(|z| - t, 0) (Prox of t|.|)."""
    return np.sign(z) * np.maximum(np.abs(z) - t, 0.0)


def objective(r: np.ndarray, x: np.ndarray, w: np.ndarray) -> float:
    """E = 1/2||r||^2 + sum w|x| for a residual r = A x - b."""
    return 0.5 * float(r @ r) + float(np.sum(w * np.abs(x)))


def duality_gap(r: np.ndarray, g: np.ndarray, y: np.ndarray, b: np.ndarray, w: np.ndarray):
    """(primal, dual, gap) at y from r = A y - b and g = A^T r."""
    primal = objective(r, y, w)
    ag = np.abs(g)
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(ag > 0, w / np.where(ag > 0, ag, 1.0), np.inf)
    s = min(1.0, float(ratio.min())) if len(ratio) else 1.0
    dual = -s * float(b @ r) - 0.5 * s * s * float(r @ r)
    return primal, dual, primal - dual


@dataclass
class FistaResult:
    x: np.ndarray
    iters: int
    objective: float            # E(x) exactly
    gap: float = float("nan")   # certificate at the last check (at y)
    rel_gap: float = float("nan")
    history: list = field(default_factory=list)   # (k, primal(y_k), gap(y_k)) per check


def fista(apply_A, apply_At, b, w, P, tau, max_iters, tol=0.0, check_every=10,
          x_init=None, record_every=0, momentum=True) -> FistaResult:
    """Algorithm 3 (preconditioned accelerated proximal gradient); momentum=False drops the
    extrapolation step (y^(k+1) = x^(k)): ISTA, the baseline curve of Sec. 5.3 / Fig. 8.

    apply_A / apply_At: the operator and its adjoint; b: data (x0 or u0); w, P: N-vectors of
    weights and preconditioner; tau: step. tol > 0 enables the gap check every
    `check_every` iterations. record_every > 0 records (k, primal, gap) at y_k every that
    many iterations regardless of tol.
    """
    N = len(w)
    x_prev = np.zeros(N) if x_init is None else np.array(x_init, dtype=np.float64)
    y = x_prev.copy()
    x = x_prev
    hist = []
    gap = rel = float("nan")
    k = 0
    for k in range(1, max_iters + 1):
        r = apply_A(y) - b
        g = apply_At(r)
        check = tol > 0 and k % check_every == 0
        record = record_every > 0 and k % record_every == 0
        if check or record:
            pr, _, gp = duality_gap(r, g, y, b, w)
            gap, rel = gp, gp / pr if pr > 0 else 0.0
            hist.append((k, pr, gp))
        z = y - tau * g / P
        x = soft(z, tau * w / P)
        if check and rel <= tol:
            break
        beta = (k - 1) / (k + 2) if momentum else 0.0
        y = x + beta * (x - x_prev)
        x_prev = x
    E = objective(apply_A(x) - b, x, w)
    return FistaResult(x, k, E, gap, rel, hist)


# ---------------------------------------------------------------------------------------
# Operators
# ---------------------------------------------------------------------------------------

def theta_ops(th):
    """(A, A^T) for A = Theta_K (a scipy CSR pair)."""
    return (lambda v: th.mat @ v), (lambda v: th.matT @ v)


class ParallelCSR:
    """The same CSR products split into row blocks evaluated on a thread pool (scipy's CSR
    product releases the interpreter lock), so that timings can use every host core. The
    arithmetic of each row is unchanged."""

    def __init__(self, mat, workers: int):
        from concurrent.futures import ThreadPoolExecutor
        n = mat.shape[0]
        self.blocks = [mat[i * n // workers:(i + 1) * n // workers] for i in range(workers)]
        self.pool = ThreadPoolExecutor(max_workers=workers)

    def __call__(self, v):
        return np.concatenate(list(self.pool.map(lambda B: B @ v, self.blocks)))

    def close(self):
        self.pool.shutdown()


def theta_ops_parallel(th, workers: int):
    """(A, A^T) for A = Theta_K with the products spread over `workers` threads."""
    return ParallelCSR(th.mat, workers), ParallelCSR(th.matT, workers)


def exact_ops(psf, n_rows, n_cols, wavelet, levels):
    """(A, A^T) for A = H Psi with H by direct periodic convolution."""
    def A(x):
        return conv_periodic(idwt2(x, n_rows, n_cols, wavelet, levels), psf).ravel()

    def At(r):
        return dwt2(conv_adjoint(r.reshape(n_rows, n_cols), psf), wavelet, levels)
    return A, At


def exact_diagonal_tables(psf, n_rows, n_cols, wavelet, levels, lay):
    """Phase tables (period 1: one value per subband) of diag(M) and diag(M^2) for the exact
    operator M = Psi* H^T H Psi, whose blocks are circulant with full translation symmetry:
    M_bb = ||H psi_b||^2 and (M^2)_bb = ||Psi* H^T H psi_b||^2 = ||H^T H psi_b||^2."""
    N = n_rows * n_cols
    Md = np.zeros(len(lay))
    M2d = np.zeros(len(lay))
    for b in lay:
        e = np.zeros(N)
        e[b.offset] = 1.0
        psi = idwt2(e, n_rows, n_cols, wavelet, levels)
        hp = conv_periodic(psi, psf)
        hhp = conv_adjoint(hp, psf)
        Md[b.index] = float(np.sum(hp * hp))
        M2d[b.index] = float(np.sum(hhp * hhp))
    return Md, M2d


# ---------------------------------------------------------------------------------------
# Independent checks
# ---------------------------------------------------------------------------------------

def kkt_residuals(A_dense_or_ops, x, b, w):
    """(max_i (|g_i| - w_i)_+ / w_i, max over the support of |g_i + w_i sign x_i| / w_i)
    with g = A^T (A x - b)."""
    if callable(A_dense_or_ops[0]):
        A, At = A_dense_or_ops
        g = At(A(x) - b)
    else:
        Ad = A_dense_or_ops[0]
        g = Ad.T @ (Ad @ x - b)
    out = float(np.max(np.maximum(np.abs(g) - w, 0.0) / w))
    sup = x != 0
    on = float(np.max(np.abs(g[sup] + w[sup] * np.sign(x[sup])) / w[sup])) if sup.any() else 0.0
    return out, on


def lasso_cd(A: np.ndarray, b: np.ndarray, w: np.ndarray, tol: float = 1e-14,
             max_sweeps: int = 200000) -> np.ndarray:
    """Cyclic coordinate descent for min 1/2||Ax - b||^2 + sum w|x| on a dense A (used only
    to pin FISTA on tiny problems; not a paper algorithm)."""
    n = A.shape[1]
    x = np.zeros(n)
    r = b.copy()                  # r = b - A x
    col_sq = np.einsum("ij,ij->j", A, A)
    for _ in range(max_sweeps):
        for j in range(n):
            if col_sq[j] == 0.0:
                continue
            aj = A[:, j]
            xj = soft(x[j] + aj @ r / col_sq[j], w[j] / col_sq[j])
            if xj != x[j]:
                r -= aj * (xj - x[j])
                x[j] = xj
        res = -r
        pr, _, gp = duality_gap(res, A.T @ res, x, b, w)
        if gp <= tol * max(pr, 1e-300):
            break
    return x
