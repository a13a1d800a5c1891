"""Direct periodic convolution H and its adjoint, in float64.

Paper: Sec. 1.1 (image formation u0 = Hu + b), Sec. 3.6 (H is a convolution with kernel h on
the torus; Def. "Translation operator" with circular boundary conditions).

Convention: the PSF is an odd-sized array psf[kh, kw] whose centre (kh//2, kw//2) is the
origin, so h[a, b] = psf[a + kh//2, b + kw//2] for a in [-kh//2, kh//2], and
    (H u)[i, j] = sum_{a,b} h[a, b] u[(i - a) mod n_rows, (j - b) mod n_cols].
H^T uses h[-a, -b]. Direct summation only (no FFT).

TEST INFRASTRUCTURE: only tests, smoke() and the bench CPU baseline use this module.
"""
from __future__ import annotations

import numpy as np


def conv_periodic(u: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """H u by direct periodic summation over the PSF support."""
    u = np.asarray(u, dtype=np.float64)
    psf = np.asarray(psf, dtype=np.float64)
    kh, kw = psf.shape
    if kh % 2 == 0 or kw % 2 == 0:
        raise ValueError("PSF sides must be odd")
    ch, cw = kh // 2, kw // 2
    out = np.zeros_like(u)
    for a in range(-ch, ch + 1):
        for b in range(-cw, cw + 1):
            v = psf[a + ch, b + cw]
            if v != 0.0:
                # np.roll(u, (a, b))[i, j] = u[i - a, j - b]
                out += v * np.roll(u, (a, b), axis=(0, 1))
    return out


def conv_adjoint(u: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """H^T u: convolution with the flipped kernel h[-a, -b]."""
    return conv_periodic(u, np.asarray(psf, dtype=np.float64)[::-1, ::-1])


def conv_matrix(n_rows: int, n_cols: int, psf: np.ndarray) -> np.ndarray:
    """Dense H (N x N), column k = H e_k (tiny sizes only)."""
    N = n_rows * n_cols
    Hm = np.zeros((N, N))
    for k in range(N):
        e = np.zeros(N)
        e[k] = 1.0
        Hm[:, k] = conv_periodic(e.reshape(n_rows, n_cols), psf).ravel()
    return Hm
