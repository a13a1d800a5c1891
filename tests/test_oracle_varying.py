"""Pins of the spatially varying oracle (oracle.varying) to what the definitions fix.

* H against a brute-force double loop over K(x, y) (Sec. 3.1 definition) on a tiny image;
  H^T is its adjoint; every column of H sums to 1 (row PSFs of sum 1).
* One PSF for every row: H is oracle.blur's convolution and Theta_K (every K) is the
  circulant oracle's (Algorithm 2 + Sec. 3.7), both built by independent code.
* The per-row probes + horizontal tap rule reproduce Theta probed column by column
  (Sec. 3.4), square and rectangular, db and sym wavelets.
* Psi is orthogonal, so trace(Theta) = trace(H) and ||Theta||_F = ||H||_F, both in closed form
  from the row PSFs.
* Thresholding: at most K entries, the next tap would exceed K, kept scores dominate dropped
  ones, K = 0 keeps nothing; the kept entries are entries of Theta.
* The diagonals of M = Theta_K^T Theta_K and M^2 are constant on the preconditioner classes.
"""
import numpy as np
import pytest

from oracle import blur, theta as TH, varying as V
from oracle.wavelet import layout
from paper_1512_08401_gb300 import synthetic as S


def psf_stack(n, s0, s1, k):
    return S.varying_gaussian(n, s0, s1, k)


def test_apply_H_brute_force_definition():
    rng = np.random.default_rng(3)
    R, C, kh, kw = 6, 8, 3, 5
    psfs = rng.uniform(0.0, 1.0, (R, kh, kw))
    u = rng.standard_normal((R, C))
    ref = np.zeros((R, C))
    for xr in range(R):
        for xc in range(C):
            acc = 0.0
            for yr in range(R):
                for yc in range(C):
                    # K(x, y): the PSF of input row yr, evaluated at the torus offset x - y
                    for a in range(-(kh // 2), kh // 2 + 1):
                        for b in range(-(kw // 2), kw // 2 + 1):
                            if (yr + a) % R == xr and (yc + b) % C == xc:
                                acc += psfs[yr, a + kh // 2, b + kw // 2] * u[yr, yc]
            ref[xr, xc] = acc
    assert np.abs(V.apply_H(u, psfs) - ref).max() <= 1e-13
    v = rng.standard_normal((R, C))
    assert abs(np.vdot(V.apply_H(u, psfs), v) - np.vdot(u, V.apply_Ht(v, psfs))) <= 1e-12
    # sparse inputs take the same values (only nonzeros are visited)
    us = np.zeros((R, C))
    us[2, 5] = 1.5
    assert np.abs(V.apply_H(us, psfs) - (V.H_dense(psfs, R, C) @ us.ravel()).reshape(R, C)).max() <= 1e-15


def test_columns_of_H_sum_to_one_and_adjoint():
    n = 32
    ps = psf_stack(n, 1.0, 3.0, 9)
    rng = np.random.default_rng(1)
    u, v = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    assert abs(V.apply_H(u, ps).sum() - u.sum()) <= 1e-11
    assert np.abs(V.apply_Ht(np.ones((n, n)), ps) - 1.0).max() <= 1e-14
    assert abs(np.vdot(V.apply_H(u, ps), v) - np.vdot(u, V.apply_Ht(v, ps))) <= 1e-10


def test_one_psf_for_all_rows_is_the_convolution():
    n = 32
    ps = psf_stack(n, 2.0, 2.0, 7)
    u = np.random.default_rng(2).standard_normal((n, n))
    assert np.abs(V.apply_H(u, ps) - blur.conv_periodic(u, ps[0])).max() <= 1e-14
    assert np.abs(V.apply_Ht(u, ps) - blur.conv_adjoint(u, ps[0])).max() <= 1e-14
    c = TH.build_theta(ps[0], n, n, "db4", 2, K=10**12)
    t = V.build_varying_theta(ps, n, n, "db4", 2, K=10**12)
    assert abs(c.mat - t.mat).max() <= 1e-15 and c.K_eff == t.K_eff


@pytest.mark.parametrize("shape,wavelet,J", [((32, 32), "db4", 2), ((32, 64), "db2", 3), ((32, 32), "sym4", 2)])
def test_row_probes_reproduce_theta_probed_column_by_column(shape, wavelet, J):
    R, C = shape
    ps = psf_stack(R, 0.8, 2.6, 7)
    T = V.theta_columns(ps, R, C, wavelet, J)
    th = V.build_varying_theta(ps, R, C, wavelet, J, K=10**12)
    assert np.abs(th.mat.toarray() - T).max() <= 1e-14
    # closed forms (Psi orthogonal): trace and Frobenius norm of H from the row PSFs
    kh, kw = ps.shape[1:]
    assert abs(np.trace(T) - C * ps[:, kh // 2, kw // 2].sum()) <= 1e-12 * C * R
    assert abs(np.linalg.norm(T) - np.sqrt(C * (ps ** 2).sum())) <= 1e-12 * np.linalg.norm(T)
    # Theta is not symmetric for a varying PSF (the H^T reading matters)
    assert np.abs(T - T.T).max() > 1e-3


def test_thresholding_properties():
    n, J = 32, 2
    ps = psf_stack(n, 1.0, 3.0, 9)
    lay = layout(n, n, J)
    t = V.all_taps(ps, n, n, "db4", J)
    score = V.tap_scores(t, lay, "weighted")
    vmax = np.abs(t.v).max()
    nz = np.abs(t.v) > V.ZERO_REL * vmax
    T = V.theta_columns(ps, n, n, "db4", J)
    for K in (0, 1000, 8 * n * n, 30 * n * n):
        keep = V.select_taps(t, lay, K, "weighted")
        kept = int(t.m[keep].sum())
        assert kept <= K
        if K == 0:
            assert not keep.any()
        drop = nz & ~keep
        if keep.any() and drop.any():
            assert score[keep].min() >= score[drop].max()
            # the best dropped tap would overflow K
            assert kept + int(t.m[drop][np.argmax(score[drop])]) > K
        th = V.build_varying_theta(ps, n, n, "db4", J, K)
        assert th.K_eff == kept == th.mat.nnz
        r, c = th.mat.nonzero()
        assert np.abs(th.mat.toarray()[r, c] - T[r, c]).max(initial=0.0) <= 1e-14
    w = V.select_taps(t, lay, 8 * n * n, "weighted")
    nv = V.select_taps(t, lay, 8 * n * n, "naive")
    assert (w != nv).any()


def test_diagonals_are_constant_on_classes():
    n, J = 32, 3
    ps = psf_stack(n, 1.0, 3.0, 9)
    th = V.build_varying_theta(ps, n, n, "db2", J, K=8 * n * n)
    per = V.class_periods(th.lay, J)
    Md, M2d = V.diagonal_tables(th.mat, th.matT, th.lay, per)
    A = th.mat.toarray()
    M = A.T @ A
    assert np.abs(V.expand(Md, th.lay, per) - np.diag(M)).max() <= 1e-13
    assert np.abs(V.expand(M2d, th.lay, per) - np.diag(M @ M)).max() <= 1e-13
    assert len(Md) == sum(b.rows * p for b, p in zip(th.lay, per))
