"""Seeded synthetic inputs: clean images, PSFs and blurred noisy observations.

This module is the one place both the FP64 oracle tests and the CUDA path draw inputs
from. It holds none of the deblurring method's arithmetic (no wavelet transform, no Theta,
no solver). It simulates the acquisition model of Sec. 1.1, u0 = H u + b with
b ~ N(0, sigma^2 I), using a numpy FFT circular convolution, which is data synthesis and is
independent of both the oracle's direct convolution and the library's cuFFT path.

Stand-ins for the paper's images (the book and confocal photographs of Sec. 5 and the
phantom of Sec. 5.6 are not available): random axis-aligned rectangles with intensities
U[0,1] painted over a linear gradient, on the torus.

Generator recipe (seeded numpy PCG64):
  1. background 0.25 + 0.5 ((i/n_rows) cos phi + (j/n_cols) sin phi)/sqrt(2), phi ~ U[0, 2pi)
  2. R = min(256, 16 * max(1, n/128)) rectangles (n = min side); corner uniform integer,
     sides uniform integers in [n/16, n/4], wrapped periodically, painted in order with an
     intensity U[0,1] (replacing what was there)
  3. blur with the periodic PSF (centre of the odd-sized array at the origin)
  4. add N(0, noise^2) noise, no clipping
PSFs:
  * gaussian(sigma, k): exp(-(a^2+b^2)/(2 sigma^2)) on a k x k support, sum 1
  * motion_line(length, angle): points t (cos a, sin a), t in [-(L-1)/2, (L-1)/2] in steps
    of 1/8 px, bilinearly splatted into an L x L grid, sum 1
  * the five families of the paper's Sec. 5 / Table 3 (paper_blur): Gaussian, skewed
    Gaussian, spline motion blur, Airy pattern, defocus disk
  * varying_gaussian(n_rows, sigma0, sigma1, k): a spatially varying blur (Sec. 3.1, 3.5):
    the input pixels of image row i spread with a Gaussian of sigma0 + (sigma1 - sigma0) i /
    n_rows on a k x k support, sum 1 per row; blur_varying applies it by direct scatter
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def rng_for(config_id: int, instance: int = 0) -> np.random.Generator:
    """PCG64 seeded with 1000 * config_id + instance."""
    return np.random.Generator(np.random.PCG64(1000 * config_id + instance))


def gaussian_psf(sigma: float, k: int) -> np.ndarray:
    if k % 2 == 0:
        raise ValueError("PSF side must be odd")
    c = k // 2
    a = np.arange(-c, c + 1, dtype=np.float64)
    h = np.exp(-(a[:, None] ** 2 + a[None, :] ** 2) / (2.0 * sigma * sigma))
    return h / h.sum()


def motion_line_psf(length: int, angle: float) -> np.ndarray:
    """Straight motion blur of `length` px at `angle` (radians), bilinear splat."""
    if length % 2 == 0:
        raise ValueError("PSF side must be odd")
    c = length // 2
    h = np.zeros((length, length))
    half = (length - 1) / 2.0
    t = np.arange(-half, half + 1e-9, 1.0 / 8.0)
    ys = c + t * np.sin(angle)
    xs = c + t * np.cos(angle)
    for y, x in zip(ys, xs):
        y0, x0 = int(np.floor(y)), int(np.floor(x))
        fy, fx = y - y0, x - x0
        for dy, wy in ((0, 1 - fy), (1, fy)):
            for dx, wx in ((0, 1 - fx), (1, fx)):
                yy, xx = y0 + dy, x0 + dx
                if 0 <= yy < length and 0 <= xx < length and wy * wx > 0:
                    h[yy, xx] += wy * wx
    return h / h.sum()


def skewed_gaussian_psf(sigma: float, k: int | None = None) -> np.ndarray:
    """The paper's anisotropic ('skewed') Gaussian (Sec. 5): exp(-t1^2/(2 s^2) - t2^2/(2 s^2))
    for t1 >= 0 and exp(-4 t1^2/(2 s^2) - t2^2/(2 s^2)) otherwise. Readings: t1 is the row
    offset and t2 the column offset, in pixels; support k = 2 ceil(3 s) + 1; sum 1."""
    k = 2 * int(np.ceil(3 * sigma)) + 1 if k is None else k
    c = k // 2
    t = np.arange(-c, c + 1, dtype=np.float64)
    t1, t2 = t[:, None], t[None, :]
    h = np.where(t1 >= 0, np.exp(-t1 ** 2 / (2 * sigma ** 2)), np.exp(-4 * t1 ** 2 / (2 * sigma ** 2)))
    h = h * np.exp(-t2 ** 2 / (2 * sigma ** 2))
    return h / h.sum()


def spline_motion_psf(rng: np.random.Generator, points: int = 5, sigma1: float = 8.0,
                      sigma2: float = 1.0) -> np.ndarray:
    """The paper's motion blur (Sec. 5): `points` points drawn from N(0, sigma1^2 I), joined by
    a cubic spline, the curve blurred by a Gaussian of standard deviation sigma2. Readings:
    the spline is the natural cubic spline through the points in drawing order, parametrised
    by the point index; the curve is sampled at 1/256 of a parameter step, each sample
    splatted bilinearly with a weight equal to its arc length; the curve is centred on its
    arc-length centroid; the support is the odd square holding the curve plus 3 sigma2."""
    pts = rng.normal(0.0, sigma1, size=(points, 2))
    t = np.arange(points, dtype=np.float64)
    # natural cubic spline, second derivatives from the tridiagonal system
    n = points - 1
    M = np.zeros((points, 2))
    if n >= 2:
        A = np.zeros((n - 1, n - 1))
        rhs = np.zeros((n - 1, 2))
        for i in range(1, n):
            A[i - 1, i - 1] = 4.0
            if i > 1:
                A[i - 1, i - 2] = 1.0
            if i < n - 1:
                A[i - 1, i] = 1.0
            rhs[i - 1] = 6.0 * (pts[i + 1] - 2 * pts[i] + pts[i - 1])
        M[1:n] = np.linalg.solve(A, rhs)
    ts = np.arange(0, n * 256 + 1) / 256.0
    seg = np.minimum(ts.astype(int), n - 1)
    u = ts - seg
    P0, P1, M0, M1 = pts[seg], pts[seg + 1], M[seg], M[seg + 1]
    u2 = u[:, None]
    curve = ((1 - u2) * P0 + u2 * P1 + ((1 - u2) ** 3 - (1 - u2)) * M0 / 6.0 + (u2 ** 3 - u2) * M1 / 6.0)
    d = np.linalg.norm(np.diff(curve, axis=0), axis=1)
    wts = np.concatenate([[d[0] / 2], (d[:-1] + d[1:]) / 2, [d[-1] / 2]])
    curve = curve - (wts[:, None] * curve).sum(0) / wts.sum()
    ext = int(np.ceil(np.abs(curve).max() + 3 * sigma2)) + 1
    k = 2 * ext + 1
    img = np.zeros((k, k))
    for (y, x), wv in zip(curve + ext, wts):
        y0, x0 = int(np.floor(y)), int(np.floor(x))
        fy, fx = y - y0, x - x0
        img[y0, x0] += wv * (1 - fy) * (1 - fx)
        img[y0 + 1, x0] += wv * fy * (1 - fx)
        img[y0, x0 + 1] += wv * (1 - fy) * fx
        img[y0 + 1, x0 + 1] += wv * fy * fx
    g = gaussian_psf(sigma2, 2 * int(np.ceil(3 * sigma2)) + 1)
    gc = g.shape[0] // 2
    out = np.zeros_like(img)
    for a in range(g.shape[0]):
        for b in range(g.shape[1]):
            sh = np.roll(np.roll(img, a - gc, axis=0), b - gc, axis=1)
            out += g[a, b] * sh
    return out / out.sum()


def airy_psf(sigma: float) -> np.ndarray:
    """Airy pattern (2 J1(x)/x)^2 (Sec. 5, Table 3), x = r / a. Reading: the width parameter
    sigma is the standard deviation of the Gaussian that best matches the central lobe
    (a = 0.7555 sigma, first dark ring at r = 2.895 sigma); support 2 ceil(3 * 2.895 sigma) + 1
    (three rings); each pixel averages 4 x 4 sub-samples; sum 1."""
    from scipy.special import j1
    a = 0.7555 * sigma
    c = int(np.ceil(3 * 2.895 * sigma))
    sub = (np.arange(4) + 0.5) / 4 - 0.5
    t = np.arange(-c, c + 1, dtype=np.float64)
    yy = (t[:, None, None, None] + sub[None, None, :, None])
    xx = (t[None, :, None, None] + sub[None, None, None, :])
    x = np.sqrt(yy ** 2 + xx ** 2) / a
    with np.errstate(invalid="ignore", divide="ignore"):
        v = np.where(x > 1e-12, (2 * j1(x) / np.where(x > 1e-12, x, 1.0)) ** 2, 1.0)
    h = v.mean(axis=(2, 3))
    return h / h.sum()


def defocus_psf(sigma: float) -> np.ndarray:
    """Defocus blur (Sec. 5, Table 3): the uniform disk of radius sigma (reading), each pixel
    weighted by the fraction of its 8 x 8 sub-samples inside the disk; sum 1."""
    c = int(np.ceil(sigma)) + 1
    sub = (np.arange(8) + 0.5) / 8 - 0.5
    t = np.arange(-c, c + 1, dtype=np.float64)
    yy = t[:, None, None, None] + sub[None, None, :, None]
    xx = t[None, :, None, None] + sub[None, None, None, :]
    h = (yy ** 2 + xx ** 2 <= sigma ** 2).mean(axis=(2, 3))
    return h / h.sum()


def paper_blur(family: str, width: float, seed: int = 0) -> np.ndarray:
    """One of the five blur families of the paper's Table 3 at width 2.5 or 5 (sigma)."""
    if family == "gaussian":
        return gaussian_psf(width, 2 * int(np.ceil(3 * width)) + 1)
    if family == "skewed":
        return skewed_gaussian_psf(width)
    if family == "motion":
        # the paper's motion blur has sigma1 = 8 at its one stated size; the two widths of
        # Table 3 scale it by width / 5 (reading)
        return spline_motion_psf(rng_for(5, seed), sigma1=8.0 * width / 5.0)
    if family == "airy":
        return airy_psf(width)
    if family == "defocus":
        return defocus_psf(width)
    raise ValueError(family)


def clean_image(n_rows: int, n_cols: int, rng: np.random.Generator) -> np.ndarray:
    i = np.arange(n_rows, dtype=np.float64)[:, None] / n_rows
    j = np.arange(n_cols, dtype=np.float64)[None, :] / n_cols
    phi = rng.uniform(0.0, 2.0 * np.pi)
    u = 0.25 + 0.5 * (i * np.cos(phi) + j * np.sin(phi)) / np.sqrt(2.0)
    u = np.broadcast_to(u, (n_rows, n_cols)).copy()
    n = min(n_rows, n_cols)
    R = min(256, 16 * max(1, n // 128))
    lo, hi = max(1, n // 16), max(1, n // 4)
    for _ in range(R):
        y0 = int(rng.integers(0, n_rows))
        x0 = int(rng.integers(0, n_cols))
        hh = int(rng.integers(lo, hi + 1))
        ww = int(rng.integers(lo, hi + 1))
        val = rng.uniform(0.0, 1.0)
        rows = (y0 + np.arange(hh)) % n_rows
        cols = (x0 + np.arange(ww)) % n_cols
        u[np.ix_(rows, cols)] = val
    return u


def blur_fft(u: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """Circular convolution by FFT (data synthesis only)."""
    n_rows, n_cols = u.shape
    kh, kw = psf.shape
    pad = np.zeros((n_rows, n_cols))
    ch, cw = kh // 2, kw // 2
    for a in range(kh):
        for b in range(kw):
            pad[(a - ch) % n_rows, (b - cw) % n_cols] += psf[a, b]
    return np.real(np.fft.ifft2(np.fft.fft2(u) * np.fft.fft2(pad)))


def varying_gaussian(n_rows: int, sigma0: float, sigma1: float, k: int) -> np.ndarray:
    """[n_rows, k, k]: the PSF with which the input pixels of each image row spread."""
    sig = sigma0 + (sigma1 - sigma0) * np.arange(n_rows, dtype=np.float64) / n_rows
    return np.stack([gaussian_psf(float(s), k) for s in sig])


def blur_varying(u: np.ndarray, psfs: np.ndarray) -> np.ndarray:
    """out[(i + a) mod R, (j + b) mod C] += psfs[i][a + kh//2, b + kw//2] u[i, j] (data
    synthesis only)."""
    n_rows, n_cols = u.shape
    _, kh, kw = psfs.shape
    out = np.zeros((n_rows, n_cols))
    for a in range(kh):
        for b in range(kw):
            out += np.roll(psfs[:, a, b][:, None] * u, (a - kh // 2, b - kw // 2), axis=(0, 1))
    return out


@dataclass
class Problem:
    u_clean: np.ndarray     # float64 (n_rows, n_cols)
    u0: np.ndarray          # float64 observation
    psf: np.ndarray         # float64 odd-sized PSF
    lam: float
    name: str


def make_problem(n: int, psf: np.ndarray, lam: float, config_id: int, instance: int = 0,
                 noise: float = 0.01, n_cols: int | None = None, name: str = "") -> Problem:
    rng = rng_for(config_id, instance)
    n_cols = n if n_cols is None else n_cols
    u = clean_image(n, n_cols, rng)
    u0 = blur_fft(u, psf) + noise * rng.standard_normal((n, n_cols))
    return Problem(u, u0, psf, lam, name)


# ---------------------------------------------------------------------------------------
# The workloads
# ---------------------------------------------------------------------------------------

def small_problem() -> Problem:
    """128 x 128, Gaussian sigma = 2 on 15 x 15, lambda = 1e-3 (db4, J = 4, K = 30 N)."""
    return make_problem(128, gaussian_psf(2.0, 15), 1e-3, config_id=0, name="128^2 gaussian s2")


def headline_problem(blur: str = "gaussian", instance: int = 0) -> Problem:
    """1024 x 1024: Gaussian sigma = 3 on 31 x 31, or a 21 px motion line at a seeded angle
    (db4, J = 5, lambda = 1e-3)."""
    if blur == "gaussian":
        psf = gaussian_psf(3.0, 31)
    elif blur == "motion":
        angle = rng_for(1, 100 + instance).uniform(0.0, np.pi)
        psf = motion_line_psf(21, angle)
    else:
        raise ValueError(blur)
    return make_problem(1024, psf, 1e-3, config_id=1, instance=instance, name=f"1024^2 {blur}")


def large_problem() -> Problem:
    """4096 x 4096, Gaussian sigma = 4 on 41 x 41 (db4, J = 6, K = 30 N)."""
    return make_problem(4096, gaussian_psf(4.0, 41), 1e-3, config_id=2, name="4096^2 gaussian s4")


def blur_pool(count: int, config_id: int):
    """`count` seeded blurs drawn like batch_mix's: a Gaussian of sigma ~ U[1, 4] on a
    (2 ceil(3 sigma)+1)^2 support or a motion line of length U{9..21} (odd) at an angle
    U[0, pi), probability 1/2 each. Returns [(psf, name)]."""
    rng = rng_for(config_id, 998)
    out = []
    for _ in range(count):
        if rng.uniform() < 0.5:
            s = rng.uniform(1.0, 4.0)
            out.append((gaussian_psf(s, 2 * int(np.ceil(3 * s)) + 1), f"gauss{s:.2f}"))
        else:
            L = int(rng.choice(np.arange(9, 22, 2)))
            out.append((motion_line_psf(L, rng.uniform(0.0, np.pi)), f"motion{L}"))
    return out


def varying_problem(n: int = 512, sigma0: float = 1.0, sigma1: float = 4.0, k: int = 25,
                    lam: float = 1e-3, instance: int = 0, noise: float = 0.01) -> Problem:
    """n x n, row-varying Gaussian (sigma from sigma0 at the top row to sigma1 at the bottom,
    k x k support), noise 0.01, lambda = 1e-3 (db4, J = 5, K = 30 N). `psf` holds the
    [n, k, k] stack of row PSFs."""
    rng = rng_for(4, instance)
    psfs = varying_gaussian(n, sigma0, sigma1, k)
    u = clean_image(n, n, rng)
    u0 = blur_varying(u, psfs) + noise * rng.standard_normal((n, n))
    return Problem(u, u0, psfs, lam, f"{n}^2 varying gaussian s{sigma0:g}-{sigma1:g}")


def batch_mix(count: int = 256, seed_config: int = 3):
    """Mixed batch: sizes from {256, 512, 1024}, Gaussian sigma ~ U[1,4] on a
    (2 ceil(3 sigma)+1)^2 support or a motion line of length U{9..21} (odd) at a random
    angle (probability 1/2 each), lambda log-uniform in [5e-4, 5e-3]."""
    rng = rng_for(seed_config, 999)
    out = []
    for i in range(count):
        n = int(rng.choice([256, 512, 1024]))
        if rng.uniform() < 0.5:
            s = rng.uniform(1.0, 4.0)
            psf = gaussian_psf(s, 2 * int(np.ceil(3 * s)) + 1)
            kind = f"gauss{s:.2f}"
        else:
            L = int(rng.choice(np.arange(9, 22, 2)))
            psf = motion_line_psf(L, rng.uniform(0.0, np.pi))
            kind = f"motion{L}"
        lam = float(np.exp(rng.uniform(np.log(5e-4), np.log(5e-3))))
        out.append(make_problem(n, psf, lam, config_id=seed_config, instance=i, name=f"{n}^2 {kind}"))
    return out
