"""Orthogonal Daubechies wavelets and the periodic separable 2-D DWT, in float64.

Paper: Sec. 2 (Notation) defines the separable isotropic wavelet basis on the torus,
psi^e_{j,m} = rho^{e_1}_{j,m_1} x ... x rho^{e_d}_{j,m_d}, with a mother wavelet of M vanishing
moments, and Psi* / Psi as the decomposition / reconstruction operators. The experiments
(Sec. 5) use an orthogonal transform with periodic boundaries; here the filter is the
Daubechies filter with p vanishing moments (2p taps), derived by spectral factorisation.

Conventions fixed here (the paper leaves them open):
  * 1-D analysis, signal s of even length n:
        a[i] = sum_k h[k] s[(2i+k) mod n],   d[i] = sum_k g[k] s[(2i+k) mod n],  i < n/2,
    with g[k] = (-1)^k h[L-1-k]. Synthesis is the exact transpose of analysis.
  * A 2-D level filters along the column index (x) of every row first, then along the row
    index (y). Orientation e = (e_y, e_x): 0 = low-pass, 1 = high-pass along that axis.
  * Coefficients are stored subband-planar: A_J first, then for s = J, J-1, ..., 1 the
    detail subbands with e = (0,1), (1,0), (1,1), each row-major of shape (n_rows/2^s,
    n_cols/2^s).

TEST INFRASTRUCTURE: only tests, smoke() and the bench CPU baseline use this module.
"""
from __future__ import annotations

from dataclasses import dataclass
from math import comb, sqrt

import numpy as np


def daubechies_lowpass(p: int) -> np.ndarray:
    """Daubechies orthogonal low-pass filter with p vanishing moments (length 2p).

    Spectral factorisation of |m0(w)|^2 = cos^{2p}(w/2) * P(sin^2(w/2)),
    P(y) = sum_{k<p} C(p-1+k, k) y^k  (Daubechies, Ten Lectures, cited in Sec. 2).
    Each root y_r of P gives a reciprocal pair of roots in z through
    y = (2 - z - 1/z)/4; the minimum-phase choice keeps, for the transfer function
    H(Z) = sum_k h[k] Z^{-k}, every zero inside the unit circle. The filter is normalised
    to sum h = sqrt(2).
    """
    if p < 1:
        raise ValueError("p must be >= 1")
    # roots of P(y); np.roots expects the highest power first
    pc = [comb(p - 1 + k, k) for k in range(p)]
    yroots = np.roots(pc[::-1]) if p > 1 else np.array([])
    zeros = []
    for y in yroots:
        b = 2.0 - 4.0 * y
        disc = np.sqrt(b * b - 4.0 + 0j)
        z1, z2 = (b + disc) / 2.0, (b - disc) / 2.0
        # zeros of H(Z) inside the unit circle => minimum phase
        zeros.append(z1 if abs(z1) < 1.0 else z2)
    # H(Z) Z^{L-1} = (Z+1)^p * prod (Z - zr) as a polynomial in Z, highest power first.
    poly = np.array([1.0 + 0j])
    for _ in range(p):
        poly = np.convolve(poly, np.array([1.0, 1.0]))
    for zr in zeros:
        poly = np.convolve(poly, np.array([1.0, -zr]))
    # coefficient of Z^{L-1-k} is h[k]
    h = np.real(poly)
    h = h * (sqrt(2.0) / h.sum())
    return h


def _factor_roots(p: int):
    """Roots of P(y) = sum_{k<p} C(p-1+k, k) y^k, grouped so that a choice keeps the filter
    real: one entry per real root, one per complex-conjugate pair (the root with Im > 0)."""
    pc = [comb(p - 1 + k, k) for k in range(p)]
    yroots = np.roots(pc[::-1]) if p > 1 else np.array([])
    groups = []
    for y in yroots:
        if abs(y.imag) <= 1e-10 * max(1.0, abs(y)):
            groups.append((complex(y.real, 0.0), False))
        elif y.imag > 0:
            groups.append((complex(y), True))
    return groups


def _filter_from_zeros(p: int, zeros: list) -> np.ndarray:
    """Real filter h with H(Z) Z^{L-1} = (Z+1)^p prod (Z - z), normalised to sum h = sqrt(2)."""
    poly = np.array([1.0 + 0j])
    for _ in range(p):
        poly = np.convolve(poly, np.array([1.0, 1.0]))
    for zr in zeros:
        poly = np.convolve(poly, np.array([1.0, -zr]))
    h = np.real(poly)
    return h * (sqrt(2.0) / h.sum())


def phase_nonlinearity(zeros: list, m: int = 2048) -> float:
    """Squared deviation of the phase of H(e^{iw}) = c e^{-i(L-1)w} prod_j (e^{iw} - z_j) from
    its least-squares line, on w_k = pi (k + 1/2) / m, k < m. The phase is summed factor by
    factor (each factor's phase is continuous: no z_j lies on the unit circle except the
    zeros at -1, whose factor has phase w/2 on [0, pi)); the linear term of e^{-i(L-1)w} does
    not change the deviation."""
    w = np.pi * (np.arange(m) + 0.5) / m
    ph = np.zeros(m)
    e = np.exp(1j * w)
    for z in zeros:
        ph += np.unwrap(np.angle(e - z))
    A = np.stack([w, np.ones_like(w)], axis=1)
    coef, *_ = np.linalg.lstsq(A, ph, rcond=None)
    return float(np.sum((ph - A @ coef) ** 2))


def symlet_lowpass(p: int) -> np.ndarray:
    """Symlet with p vanishing moments (length 2p): the same |m0(w)|^2 as db<p> (Ten Lectures,
    cited in Sec. 2, the 'least asymmetric' choice), factorised with, for every root group of
    P, the zero inside or outside the unit circle, choosing the combination whose phase is
    closest to linear (phase_nonlinearity). A filter and its time reverse tie (values within
    1e-6 of each other count as a tie); the one whose energy centroid sum_k k h[k]^2 is
    smaller is taken. Reading: the paper names Symmlet 6
    (Sec. 5) without giving its coefficients or its selection rule."""
    if p < 1:
        raise ValueError("p must be >= 1")
    groups = _factor_roots(p)
    best = None
    for mask in range(1 << len(groups)):
        zeros = []
        for gi, (y, cplx) in enumerate(groups):
            b = 2.0 - 4.0 * y
            disc = np.sqrt(b * b - 4.0 + 0j)
            z1, z2 = (b + disc) / 2.0, (b - disc) / 2.0
            zin, zout = (z1, z2) if abs(z1) < 1.0 else (z2, z1)
            z = zout if (mask >> gi) & 1 else zin
            zeros.append(z)
            if cplx:
                zeros.append(np.conj(z))
        h = _filter_from_zeros(p, zeros)
        nl = phase_nonlinearity([-1.0] * p + zeros)
        cen = float(np.sum(np.arange(len(h)) * h * h))
        if best is None or nl < best[0] * (1 - 1e-6) or (abs(nl - best[0]) <= 1e-6 * best[0] and cen < best[1]):
            best = (nl, cen, h)
    return best[2]


def highpass_from_lowpass(h: np.ndarray) -> np.ndarray:
    """Quadrature mirror high-pass g[k] = (-1)^k h[L-1-k]."""
    L = len(h)
    return np.array([(-1.0) ** k * h[L - 1 - k] for k in range(L)])


def wavelet_filters(name: str) -> tuple[np.ndarray, np.ndarray]:
    """Filters for 'db<p>' (minimum phase) or 'sym<p>' (least asymmetric), p vanishing
    moments, 2p taps."""
    if name.startswith("db"):
        h = daubechies_lowpass(int(name[2:]))
    elif name.startswith("sym"):
        h = symlet_lowpass(int(name[3:]))
    else:
        raise ValueError(f"unknown wavelet {name!r}")
    return h, highpass_from_lowpass(h)


# ---------------------------------------------------------------------------------------
# 1-D periodic analysis / synthesis along an axis
# ---------------------------------------------------------------------------------------

def analysis_1d(s: np.ndarray, f: np.ndarray, axis: int) -> np.ndarray:
    """out[i] = sum_k f[k] s[(2i+k) mod n] along `axis` (periodic, decimated)."""
    s = np.moveaxis(np.asarray(s, dtype=np.float64), axis, -1)
    n = s.shape[-1]
    if n % 2:
        raise ValueError("length must be even")
    i = np.arange(n // 2)
    out = np.zeros(s.shape[:-1] + (n // 2,))
    for k in range(len(f)):
        out += f[k] * s[..., (2 * i + k) % n]
    return np.moveaxis(out, -1, axis)


def synthesis_1d(c: np.ndarray, f: np.ndarray, axis: int) -> np.ndarray:
    """Transpose of analysis_1d: s[(2i+k) mod n] += f[k] c[i]."""
    c = np.moveaxis(np.asarray(c, dtype=np.float64), axis, -1)
    half = c.shape[-1]
    n = 2 * half
    i = np.arange(half)
    out = np.zeros(c.shape[:-1] + (n,))
    for k in range(len(f)):
        # indices (2i+k) mod n are distinct for fixed k, so a fancy-index add is exact
        idx = (2 * i + k) % n
        out[..., idx] += f[k] * c
    return np.moveaxis(out, -1, axis)


# ---------------------------------------------------------------------------------------
# Subband layout
# ---------------------------------------------------------------------------------------

@dataclass(frozen=True)
class Subband:
    index: int
    level: int          # s: 1 = finest ... J = coarsest
    e: tuple            # (e_y, e_x)
    rows: int
    cols: int
    offset: int         # start in the planar coefficient vector

    @property
    def size(self) -> int:
        return self.rows * self.cols


def layout(n_rows: int, n_cols: int, levels: int) -> list[Subband]:
    """Subband-planar layout: A_J, then (0,1),(1,0),(1,1) for s = J ... 1."""
    if levels < 1:
        raise ValueError("levels must be >= 1")
    if n_rows % (1 << levels) or n_cols % (1 << levels):
        raise ValueError("image sides must be divisible by 2^J")
    out = []
    off = 0
    rJ, cJ = n_rows >> levels, n_cols >> levels
    out.append(Subband(0, levels, (0, 0), rJ, cJ, off))
    off += rJ * cJ
    idx = 1
    for s in range(levels, 0, -1):
        r, c = n_rows >> s, n_cols >> s
        for e in ((0, 1), (1, 0), (1, 1)):
            out.append(Subband(idx, s, e, r, c, off))
            off += r * c
            idx += 1
    assert off == n_rows * n_cols
    return out


# ---------------------------------------------------------------------------------------
# 2-D multi-level transforms
# ---------------------------------------------------------------------------------------

def dwt2(u: np.ndarray, wavelet: str, levels: int) -> np.ndarray:
    """Psi* u: forward periodic separable DWT, planar coefficient vector (float64)."""
    h, g = wavelet_filters(wavelet)
    u = np.asarray(u, dtype=np.float64)
    n_rows, n_cols = u.shape
    lay = layout(n_rows, n_cols, levels)
    x = np.zeros(n_rows * n_cols)
    A = u
    for s in range(1, levels + 1):
        Lx = analysis_1d(A, h, axis=1)      # low along x
        Hx = analysis_1d(A, g, axis=1)      # high along x
        sub = {
            (0, 1): analysis_1d(Hx, h, axis=0),
            (1, 0): analysis_1d(Lx, g, axis=0),
            (1, 1): analysis_1d(Hx, g, axis=0),
        }
        A = analysis_1d(Lx, h, axis=0)
        for b in lay:
            if b.level == s and b.e != (0, 0):
                x[b.offset:b.offset + b.size] = sub[b.e].ravel()
    x[lay[0].offset:lay[0].offset + lay[0].size] = A.ravel()
    return x


def idwt2(x: np.ndarray, n_rows: int, n_cols: int, wavelet: str, levels: int) -> np.ndarray:
    """Psi x: inverse transform (the exact transpose of dwt2)."""
    h, g = wavelet_filters(wavelet)
    x = np.asarray(x, dtype=np.float64)
    lay = layout(n_rows, n_cols, levels)
    a0 = lay[0]
    A = x[a0.offset:a0.offset + a0.size].reshape(a0.rows, a0.cols)
    for s in range(levels, 0, -1):
        sub = {b.e: x[b.offset:b.offset + b.size].reshape(b.rows, b.cols)
               for b in lay if b.level == s and b.e != (0, 0)}
        Lx = synthesis_1d(A, h, axis=0) + synthesis_1d(sub[(1, 0)], g, axis=0)
        Hx = synthesis_1d(sub[(0, 1)], h, axis=0) + synthesis_1d(sub[(1, 1)], g, axis=0)
        A = synthesis_1d(Lx, h, axis=1) + synthesis_1d(Hx, g, axis=1)
    return A


def dwt_matrix(n_rows: int, n_cols: int, wavelet: str, levels: int) -> np.ndarray:
    """Dense Psi* (N x N) built column by column from unit images (tiny sizes only)."""
    N = n_rows * n_cols
    D = np.zeros((N, N))
    for k in range(N):
        e = np.zeros(N)
        e[k] = 1.0
        D[:, k] = dwt2(e.reshape(n_rows, n_cols), wavelet, levels)
    return D
