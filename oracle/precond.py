"""Diagonal preconditioners and the step size, in float64.

Paper passages followed:
  * Sec. 4.2, Eq. Jacobi_Precond: P = max(diag(Theta_K^* Theta_K), eps).
  * Sec. 4.3, Eq. opt_diag and Lemma Eq. SPAI_Precond: the diagonal P minimising
    ||Id - P^{-1} M||_F with M = Theta_K^* Theta_K is P_ii = (M^2)_ii / M_ii, and any
    positive value where M_ii = 0.
  * Algorithm 3 step size tau = 1/||Theta_K^* Theta_K P^{-1}||_2.

Readings taken where the paper is silent:
  * Theta_K keeps whole taps, so every block stays circulant (Thm 3) and Theta_K commutes
    with image translations by 2^J pixels (subband b shifts by 2^{J - s_b} positions). The
    diagonals of M and M^2 are therefore periodic on every subband b with period
    R_b = 2^{J - s_b} along both axes. (They are not constant per subband: in a block whose
    output is coarser, a column sees only the taps of its phase.) Both diagonals are
    evaluated on one coordinate per phase class (b, qy mod R_b, qx mod R_b):
    M_ii = ||Theta_K e_i||^2 and (M^2)_ii = ||Theta_K^T Theta_K e_i||^2, and stored as a
    flat table of sum_b R_b^2 = 4^J values, subband after subband, row-major in the phase.
  * SPAI with M_ii = 0 takes P_ii = 1. Jacobi eps defaults to 1e-6 * max_i M_ii (the paper
    hand-tunes it).
  * The step uses the Lipschitz constant of the gradient in the P-metric,
    L = lambda_max(P^{-1/2} M P^{-1/2}), estimated by power iteration (<= 200 iterations,
    start vector splitmix64(seed 12345) uniform in [-1,1), stop when the estimate changes
    by <= 1e-12 relative), and tau = 1/(1.01 L). The 1 % margin covers the power-iteration
    underestimate.

TEST INFRASTRUCTURE: only tests, smoke() and the bench CPU baseline use this module.
"""
from __future__ import annotations

import numpy as np

from .rng import uniform_pm1

PRECONDS = ("none", "jacobi", "spai")
POWER_SEED = 12345
POWER_ITERS = 200
POWER_RTOL = 1e-12
STEP_MARGIN = 1.01


def phase_period(b, levels: int) -> int:
    """R_b = 2^{J - s_b}: period of the diagonals of M on subband b."""
    return 1 << (levels - b.level)


def table_offsets(lay, periods) -> np.ndarray:
    """Start of every subband's block in the flat phase table."""
    sizes = np.array([periods[b.index] ** 2 for b in lay])
    return np.concatenate([[0], np.cumsum(sizes)])


def theta_periods(lay, levels: int) -> list:
    return [phase_period(b, levels) for b in lay]


def diagonal_tables(mat, matT, lay, periods) -> tuple[np.ndarray, np.ndarray]:
    """Flat tables of M_ii and (M^2)_ii, one entry per phase class, M = Theta_K^T Theta_K.

    For the class (b, py, px) the representative coordinate is position (py, px) of b."""
    csc = mat.tocsc()
    offs = table_offsets(lay, periods)
    Md = np.zeros(offs[-1])
    M2d = np.zeros(offs[-1])
    for b in lay:
        R = periods[b.index]
        for py in range(R):
            for px in range(R):
                i = b.offset + py * b.cols + px
                v = csc[:, [i]]                 # Theta_K e_i (sparse column)
                w = matT @ v                    # M e_i
                t = offs[b.index] + py * R + px
                Md[t] = float(v.multiply(v).sum())
                M2d[t] = float(w.multiply(w).sum())
    return Md, M2d


def preconditioner(Md: np.ndarray, M2d: np.ndarray, kind: str, jacobi_eps: float | None = None) -> np.ndarray:
    """Diagonal P per phase class (Eq. Jacobi_Precond / Eq. SPAI_Precond)."""
    if kind == "none":
        return np.ones_like(Md)
    if kind == "jacobi":
        eps = 1e-6 * Md.max() if jacobi_eps is None else jacobi_eps
        return np.maximum(Md, eps)
    if kind == "spai":
        P = np.ones_like(Md)
        nz = Md > 0
        P[nz] = M2d[nz] / Md[nz]
        return P
    raise ValueError(kind)


def expand(table: np.ndarray, lay, periods) -> np.ndarray:
    """Phase table -> N-vector in planar order."""
    offs = table_offsets(lay, periods)
    out = []
    for b in lay:
        R = periods[b.index]
        tab = table[offs[b.index]:offs[b.index + 1]].reshape(R, R)
        qy = np.arange(b.rows) % R
        qx = np.arange(b.cols) % R
        out.append(tab[qy[:, None], qx[None, :]].ravel())
    return np.concatenate(out)


def power_iteration(apply_M, Pvec: np.ndarray, seed: int = POWER_SEED,
                    iters: int = POWER_ITERS, rtol: float = POWER_RTOL) -> tuple[float, int]:
    """lambda_max(P^{-1/2} M P^{-1/2}) by power iteration; returns (estimate, iterations)."""
    N = len(Pvec)
    s = 1.0 / np.sqrt(Pvec)
    v = uniform_pm1(seed, N)
    v /= np.linalg.norm(v)
    lam = 0.0
    it = 0
    for it in range(1, iters + 1):
        w = s * apply_M(s * v)
        lam_new = np.linalg.norm(w)
        if lam_new == 0.0:
            return 0.0, it
        v = w / lam_new
        done = abs(lam_new - lam) <= rtol * lam_new
        lam = lam_new
        if done:
            break
    return lam, it


def step_size(L: float) -> float:
    """tau = 1/(1.01 L)."""
    return 1.0 / (STEP_MARGIN * L) if L > 0 else 1.0
