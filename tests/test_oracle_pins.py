"""Pins of the FP64 oracle against facts fixed by the paper or by mathematics.

Each test names the property it checks and why a plausible mistake would fail it.
CPU only (no GPU marker).
"""
import os

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from oracle import blur, precond, solver, theta, wavelet
from oracle.rng import splitmix64, uniform_pm1
from paper_1512_08401_gb300 import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------------------
# Filters (Sec. 2: orthogonal wavelet with M vanishing moments)
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_filter_orthonormal_and_vanishing_moments(p):
    h = wavelet.daubechies_lowpass(p)
    g = wavelet.highpass_from_lowpass(h)
    L = len(h)
    assert L == 2 * p
    for m in range(p):
        s = sum(h[k] * h[k + 2 * m] for k in range(L - 2 * m))
        assert abs(s - (1.0 if m == 0 else 0.0)) < 1e-14
    assert abs(h.sum() - np.sqrt(2.0)) < 1e-14
    k = np.arange(L, dtype=np.float64)
    for m in range(p):
        scale = np.sum(np.abs(g) * k ** m)
        assert abs(np.sum(g * k ** m)) < 1e-13 * scale


def test_db2_closed_form():
    # Daubechies' closed form for 4 taps: (1+r3, 3+r3, 3-r3, 1-r3)/(4 sqrt 2)
    r3 = np.sqrt(3.0)
    ref = np.array([1 + r3, 3 + r3, 3 - r3, 1 - r3]) / (4 * np.sqrt(2.0))
    assert np.allclose(wavelet.daubechies_lowpass(2), ref, atol=1e-15)


def test_db1_is_haar():
    assert np.allclose(wavelet.daubechies_lowpass(1), [1 / np.sqrt(2), 1 / np.sqrt(2)], atol=1e-15)


def test_db4_minimum_phase():
    h = wavelet.daubechies_lowpass(4)
    zeros = np.roots(h)            # zeros of H(Z) = sum h[k] Z^-k
    nontrivial = zeros[np.abs(zeros + 1.0) > 1e-2]
    assert len(nontrivial) == 3
    assert np.all(np.abs(nontrivial) < 1.0)
    # minimum phase concentrates energy at the start
    assert np.sum(h[:4] ** 2) > 0.9


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6, 8, 10])
def test_symlet_orthonormal_same_magnitude_as_db_and_more_linear_phase(p):
    """Symmlets (the paper's Symmlet 6, Sec. 5): an orthonormal filter with p vanishing
    moments whose magnitude response equals db<p>'s (the same |m0|^2 factorised with other
    zeros), whose zeros are those of db<p> or their inverses, and whose phase is at least as
    close to linear as db<p>'s (strictly closer from p = 4 on). A wrong zero selection, a lost
    conjugate or a broken normalisation fails one of these."""
    h = wavelet.symlet_lowpass(p)
    d = wavelet.daubechies_lowpass(p)
    g = wavelet.highpass_from_lowpass(h)
    L = len(h)
    assert L == 2 * p
    for m in range(p):
        s = sum(h[k] * h[k + 2 * m] for k in range(L - 2 * m))
        assert abs(s - (1.0 if m == 0 else 0.0)) < 1e-13
    assert abs(h.sum() - np.sqrt(2.0)) < 1e-14
    k = np.arange(L, dtype=np.float64)
    for m in range(p):
        assert abs(np.sum(g * k ** m)) < 1e-12 * np.sum(np.abs(g) * k ** m)
    w = np.linspace(0, np.pi, 257)
    E = np.exp(-1j * np.outer(w, np.arange(L)))
    assert np.abs(np.abs(E @ h) - np.abs(E @ d)).max() < 1e-12
    def nontrivial_zeros(f):
        # divide the p-fold zero at -1 out of H(Z) Z^{L-1} (synthetic division), then the rest
        q = np.array(f, dtype=np.float64)
        for _ in range(p):
            q, r = np.polydiv(q, [1.0, 1.0])
            assert abs(r[-1]) < 1e-10
        return np.roots(q)
    nz = nontrivial_zeros(h)
    nd = nontrivial_zeros(d)
    assert len(nz) == len(nd) == p - 1
    for z in nz:
        assert min(np.abs(nd - z).min(), np.abs(nd - 1 / z).min()) < 1e-4 * max(1.0, abs(z))
    nl = lambda zeros: wavelet.phase_nonlinearity([-1.0] * p + list(zeros))
    assert nl(nz) <= nl(nd) * (1 + 1e-9)
    if p >= 4:
        assert nl(nz) < 0.5 * nl(nd)


def test_symlet_small_orders_are_daubechies():
    """For p <= 3 P(y) has at most one root, so the only alternative factorisation is the
    time reverse of db<p>: the Symmlet is db<p> (its reverse has the larger energy centroid)."""
    for p in (1, 2, 3):
        assert np.abs(wavelet.symlet_lowpass(p) - wavelet.daubechies_lowpass(p)).max() < 1e-14


@pytest.mark.parametrize("J", [1, 3, 5])
def test_symlet_dwt_perfect_reconstruction(J):
    rng = np.random.default_rng(3)
    u = rng.standard_normal((64, 96))
    c = wavelet.dwt2(u, "sym6", J)
    assert abs(np.linalg.norm(c) - np.linalg.norm(u)) < 1e-12 * np.linalg.norm(u)
    assert np.abs(wavelet.idwt2(c, 64, 96, "sym6", J) - u).max() < 1e-12


# ---------------------------------------------------------------------------------------
# DWT (Sec. 2)
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("shape,J", [((32, 32), 3), ((16, 48), 2), ((8, 8), 3), ((64, 32), 5)])
def test_dwt_perfect_reconstruction_and_parseval(shape, J):
    rng = np.random.default_rng(1)
    u = rng.standard_normal(shape)
    x = wavelet.dwt2(u, "db4", J)
    assert np.abs(wavelet.idwt2(x, *shape, "db4", J) - u).max() < 1e-13
    assert abs(np.linalg.norm(x) - np.linalg.norm(u)) < 1e-12 * np.linalg.norm(u)


def test_dwt_constant_image():
    c = 0.37
    J = 3
    x = wavelet.dwt2(np.full((32, 32), c), "db4", J)
    lay = wavelet.layout(32, 32, J)
    a = lay[0]
    assert np.allclose(x[a.offset:a.offset + a.size], c * 2 ** J, atol=1e-13)
    assert np.abs(x[a.size:]).max() < 1e-13


def test_haar_one_level_textbook():
    u = np.arange(16, dtype=np.float64).reshape(4, 4) ** 1.5
    x = wavelet.dwt2(u, "db1", 1)
    lay = wavelet.layout(4, 4, 1)
    blk = u.reshape(2, 2, 2, 2).transpose(0, 2, 1, 3)   # [I, J, dy, dx]
    tl, tr, bl, br = blk[..., 0, 0], blk[..., 0, 1], blk[..., 1, 0], blk[..., 1, 1]
    ref = {
        (0, 0): (tl + tr + bl + br) / 2,
        (0, 1): (tl - tr + bl - br) / 2,     # high along x
        (1, 0): (tl + tr - bl - br) / 2,     # high along y
        (1, 1): (tl - tr - bl + br) / 2,
    }
    for b in lay:
        assert np.allclose(x[b.offset:b.offset + b.size].reshape(2, 2), ref[b.e], atol=1e-13)


@pytest.mark.parametrize("n,J", [(8, 1), (16, 2)])
def test_dwt_matrix_orthogonal(n, J):
    D = wavelet.dwt_matrix(n, n, "db4", J)
    assert np.abs(D.T @ D - np.eye(n * n)).max() < 1e-14 * 10


def test_dwt_translation_covariance():
    # shifting the image by 2^J px shifts subband s by 2^{J-s} positions: the basis
    # functions are translates, which Thm 3 relies on
    J = 3
    rng = np.random.default_rng(2)
    u = rng.standard_normal((32, 32))
    x = wavelet.dwt2(u, "db4", J)
    xs = wavelet.dwt2(np.roll(u, (8, -8), axis=(0, 1)), "db4", J)
    for b in wavelet.layout(32, 32, J):
        sh = 8 >> b.level
        A = x[b.offset:b.offset + b.size].reshape(b.rows, b.cols)
        B = xs[b.offset:b.offset + b.size].reshape(b.rows, b.cols)
        assert np.abs(np.roll(A, (sh, -sh), axis=(0, 1)) - B).max() < 1e-13


# ---------------------------------------------------------------------------------------
# Convolution (Sec. 3.6)
# ---------------------------------------------------------------------------------------

def test_conv_adjoint_and_fft_agreement():
    rng = np.random.default_rng(3)
    u = rng.standard_normal((24, 40))
    v = rng.standard_normal((24, 40))
    psf = synthetic.motion_line_psf(7, 0.6)
    Hu = blur.conv_periodic(u, psf)
    assert abs(np.sum(Hu * v) - np.sum(u * blur.conv_adjoint(v, psf))) < 1e-12
    # numpy FFT circular convolution (test-only cross check)
    pad = np.zeros((24, 40))
    for a in range(7):
        for b in range(7):
            pad[(a - 3) % 24, (b - 3) % 40] = psf[a, b]
    ref = np.real(np.fft.ifft2(np.fft.fft2(u) * np.fft.fft2(pad)))
    assert np.abs(Hu - ref).max() < 1e-13


def test_conv_delta_is_identity():
    u = np.random.default_rng(4).standard_normal((16, 16))
    d = np.zeros((3, 3))
    d[1, 1] = 1.0
    assert np.array_equal(blur.conv_periodic(u, d), u)


# ---------------------------------------------------------------------------------------
# Theta (Eq. matrixH, Thm 3, Algorithm 2)
# ---------------------------------------------------------------------------------------

def test_circulant_rule_matches_paper_example():
    rows = [list(map(int, line.split())) for line in open(os.path.join(GOLDEN, "circulant_4x8.txt"))
            if line.strip() and not line.startswith("#")]
    ref = np.array(rows) - 1
    assert np.array_equal(theta.block_tap_index(4, 8), ref)
    # and the transposed case of the definition: A[:, l] = tau_{2l}(a) for 8 x 4
    assert np.array_equal(theta.block_tap_index(8, 4), ref.T)


PSFS = {
    "gauss": synthetic.gaussian_psf(1.0, 5),
    "motion": synthetic.motion_line_psf(5, 0.7),
}


@pytest.mark.parametrize("n,J", [(8, 1), (16, 2), (32, 3)])
@pytest.mark.parametrize("kind", ["gauss", "motion"])
def test_probe_theta_equals_dense_brute_force(n, J, kind):
    psf = PSFS[kind]
    dense = theta.theta_dense(n, n, psf, "db4", J)
    pr = theta.compute_probes(psf, n, n, "db4", J)
    t = theta.all_taps(pr)
    assert t.m.sum() == (n * n) ** 2
    full = theta.theta_sparse(t, pr.lay, n * n).toarray()
    assert np.abs(full - dense).max() < 1e-13


def test_dense_theta_blocks_are_circulant():
    # Thm 3 checked on the dense brute force, without the tap index rule:
    # shifting the input position by one and the output by the scale ratio (or the output
    # by one and the input by the ratio) leaves every entry unchanged.
    n, J = 16, 2
    psf = PSFS["motion"]
    dense = theta.theta_dense(n, n, psf, "db4", J)
    lay = wavelet.layout(n, n, J)
    for a in lay:
        for b in lay:
            blk = dense[a.offset:a.offset + a.size, b.offset:b.offset + b.size]
            blk = blk.reshape(a.rows, a.cols, b.rows, b.cols)
            if a.level <= b.level:
                r = 1 << (b.level - a.level)
                sh = np.roll(blk, (r, r, 1, 1), axis=(0, 1, 2, 3))
            else:
                r = 1 << (a.level - b.level)
                sh = np.roll(blk, (1, 1, r, r), axis=(0, 1, 2, 3))
            assert np.abs(sh - blk).max() < 1e-14


def test_theta_objective_identity():
    # Eq. l1problemTheta: ||Theta x - x0|| = ||H Psi x - u0|| when nothing is dropped
    n, J = 16, 2
    psf = PSFS["motion"]
    rng = np.random.default_rng(5)
    u0 = rng.standard_normal((n, n))
    x = rng.standard_normal(n * n)
    th = theta.build_theta(psf, n, n, "db4", J, K=(n * n) ** 2)
    x0 = wavelet.dwt2(u0, "db4", J)
    lhs = np.linalg.norm(th.mat @ x - x0)
    rhs = np.linalg.norm(blur.conv_periodic(wavelet.idwt2(x, n, n, "db4", J), psf) - u0)
    assert abs(lhs - rhs) < 1e-12 * rhs


def test_delta_psf_gives_identity_theta():
    d = np.zeros((3, 3))
    d[1, 1] = 1.0
    th = theta.build_theta(d, 16, 16, "db4", 2, K=10 ** 9)
    assert th.K_eff == 256
    assert np.abs(th.mat.toarray() - np.eye(256)).max() < 1e-14


# ---------------------------------------------------------------------------------------
# Thresholding (Sec. 3.7)
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("rule", ["weighted", "naive"])
def test_selection_is_topK_of_dense_entries(rule):
    # Eq. cleverthreshold / naivethresholding, checked entry by entry on the dense Theta:
    # the kept entries are the largest |sigma_mu Theta[lam, mu]|
    n, J = 16, 2
    psf = PSFS["motion"]
    dense = theta.theta_dense(n, n, psf, "db4", J)
    lay = wavelet.layout(n, n, J)
    lev = np.concatenate([np.full(b.size, b.level) for b in lay]).astype(float)
    sigma = 2.0 ** lev if rule == "weighted" else np.ones(n * n)
    score = np.abs(dense * sigma[None, :])
    for K in (0, 700, 5000, 20000, 60000):
        th = theta.build_theta(psf, n, n, "db4", J, K=K, rule=rule)
        assert th.K_eff <= K
        kept = th.mat.toarray() != 0
        assert kept.sum() == th.K_eff
        if kept.any():
            assert np.abs(th.mat.toarray()[kept] - dense[kept]).max() < 1e-13
        if 0 < th.K_eff < n ** 4:
            assert score[kept].min() >= score[~kept].max() * (1 - 1e-12)
        # greedy whole-tap prefix: the next tap in order did not fit, so fewer than its
        # multiplicity (<= N) entries of budget remain
        assert K - th.K_eff < n * n or th.K_eff == np.count_nonzero(np.abs(dense) > 1e-14 * np.abs(dense).max())


def test_weighted_rule_restores_better_than_naive_at_equal_K():
    """Sec. 5.1 (Fig. 5): at the same number of kept entries, the weighted rule (Eq.
    cleverthreshold) restores better than the naive one (Eq. naivethresholding). Two blurs x
    three seeded 64^2 problems, K = 5N, 300 iterations of Algorithm 3 with SPAI: the weighted
    operator's pSNR is higher in every case (by 0.4-3.3 dB). Weights inverted to favour finer
    inputs (sigma = 2^-level) lose in two of the six, so the direction of sigma is pinned."""
    from oracle_cases import build_case, fista, precond_and_step
    n, J = 64, 3
    for psf in (synthetic.gaussian_psf(1.5, 9), synthetic.motion_line_psf(7, 0.9)):
        for inst in range(3):
            prob = synthetic.make_problem(n, psf, 1e-3, config_id=77, instance=inst)
            snr = {}
            for rule in ("weighted", "naive"):
                case = build_case(psf, n, n, J, 5 * n * n, prob.u0, rule=rule)
                _, P, tau, _ = precond_and_step(case, "spai")
                x = fista(case, 1e-3, P, tau, 300).x
                img = wavelet.idwt2(x, n, n, "db4", J).reshape(n, n)
                snr[rule] = 10 * np.log10(1.0 / np.mean((img - prob.u_clean) ** 2))
            assert snr["weighted"] > snr["naive"], (inst, snr)


def test_selection_weighted_differs_from_naive():
    n, J = 32, 3
    psf = synthetic.gaussian_psf(1.5, 7)
    a = theta.build_theta(psf, n, n, "db4", J, K=30 * n * n, rule="weighted")
    b = theta.build_theta(psf, n, n, "db4", J, K=30 * n * n, rule="naive")
    assert (a.mat != b.mat).nnz > 0


# ---------------------------------------------------------------------------------------
# Preconditioners (Sec. 4.2, 4.3) and step size
# ---------------------------------------------------------------------------------------

def _small_thetak():
    n, J = 16, 2
    psf = PSFS["motion"]
    return theta.build_theta(psf, n, n, "db4", J, K=12000)


def _P(th, kind, **kw):
    per = precond.theta_periods(th.lay, th.levels)
    Md, M2d = precond.diagonal_tables(th.mat, th.matT, th.lay, per)
    return precond.expand(precond.preconditioner(Md, M2d, kind, **kw), th.lay, per), Md


def test_precond_diagonals_periodic_per_subband():
    # the phase tables reproduce the full diagonals of the dense M and M^2
    th = _small_thetak()
    M = (th.matT @ th.mat).toarray()
    M2 = M @ M
    per = precond.theta_periods(th.lay, th.levels)
    Md, M2d = precond.diagonal_tables(th.mat, th.matT, th.lay, per)
    assert np.allclose(precond.expand(Md, th.lay, per), np.diag(M), rtol=1e-12, atol=1e-15)
    assert np.allclose(precond.expand(M2d, th.lay, per), np.diag(M2), rtol=1e-12, atol=1e-15)
    # and with nothing dropped they are constant on every subband (full translation symmetry)
    full = theta.build_theta(PSFS["motion"], 16, 16, "db4", 2, K=10 ** 12)
    Mf = (full.matT @ full.mat).toarray()
    for b in full.lay:
        d = np.diag(Mf)[b.offset:b.offset + b.size]
        assert np.ptp(d) < 1e-13 * d.max()


def test_spai_minimises_frobenius():
    th = _small_thetak()
    M = (th.matT @ th.mat).toarray()
    P, _ = _P(th, "spai")
    # per coordinate: row i of P^{-1} M is q * M[i, :]; best q by a scalar minimiser
    for i in (0, 5, 17, 100, 200, 255):
        f = lambda q: np.sum((np.eye(len(P))[i] - q * M[i]) ** 2)
        q = minimize_scalar(f, bracket=(0.0, 2.0 / max(M[i, i], 1e-300)), tol=1e-14).x
        assert abs(1.0 / q - P[i]) < 1e-6 * P[i]
    base = np.linalg.norm(np.eye(len(P)) - M / P[:, None])
    for b in th.lay:
        for f in (0.99, 1.01):
            Pp = P.copy()
            Pp[b.offset:b.offset + b.size] *= f
            assert np.linalg.norm(np.eye(len(P)) - M / Pp[:, None]) > base


def test_jacobi_is_clamped_diagonal():
    th = _small_thetak()
    M = (th.matT @ th.mat).toarray()
    eps = 0.5 * np.diag(M).max()
    P, _ = _P(th, "jacobi", jacobi_eps=eps)
    assert np.allclose(P, np.maximum(np.diag(M), eps), rtol=1e-12)


def test_power_iteration_matches_eigvalsh():
    th = _small_thetak()
    M = (th.matT @ th.mat).toarray()
    P, _ = _P(th, "spai")
    s = 1.0 / np.sqrt(P)
    ref = np.linalg.eigvalsh(s[:, None] * M * s[None, :]).max()
    L, _ = precond.power_iteration(lambda v: th.matT @ (th.mat @ v), P, iters=5000, rtol=1e-15)
    assert abs(L - ref) < 1e-9 * ref


def test_lipschitz_closed_form_without_precond():
    # Psi orthogonal => ||H Psi||^2 = max |h_hat|^2
    n, J = 32, 3
    psf = synthetic.gaussian_psf(1.3, 7)
    th = theta.build_theta(psf, n, n, "db4", J, K=10 ** 12)
    L, _ = precond.power_iteration(lambda v: th.matT @ (th.mat @ v), np.ones(n * n))
    pad = np.zeros((n, n))
    for a in range(7):
        for b in range(7):
            pad[(a - 3) % n, (b - 3) % n] = psf[a, b]
    ref = np.max(np.abs(np.fft.fft2(pad)) ** 2)
    assert abs(L - ref) < 1e-8 * ref


def test_splitmix64_reference_values():
    # Outputs of splitmix64 seeded with 0, from the published reference implementation's
    # definition (first value is the well-known 0xE220A8397B1DCDAF)
    z = splitmix64(0, 3)
    assert int(z[0]) == 0xE220A8397B1DCDAF
    assert int(z[1]) == 0x6E789E6AA1B965F4
    assert int(z[2]) == 0x06C45D188009454F
    u = uniform_pm1(12345, 1000)
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.1


# ---------------------------------------------------------------------------------------
# FISTA (Algorithm 3), gap, KKT
# ---------------------------------------------------------------------------------------

def test_soft_threshold_closed_form():
    z = np.array([-3.0, -1.0, -0.5, 0.0, 0.5, 1.0, 3.0])
    assert np.array_equal(solver.soft(z, 1.0), [-2.0, 0.0, 0.0, 0.0, 0.0, 0.0, 2.0])
    # prox property: argmin 1/2 (x - z)^2 + t|x| by brute force on a grid
    xs = np.linspace(-4, 4, 80001)
    for zi in z:
        best = xs[np.argmin(0.5 * (xs - zi) ** 2 + 0.7 * np.abs(xs))]
        assert abs(best - solver.soft(np.array([zi]), 0.7)[0]) < 1e-4


def test_identity_operator_one_step():
    d = np.zeros((3, 3))
    d[1, 1] = 1.0
    n, J = 16, 2
    th = theta.build_theta(d, n, n, "db4", J, K=10 ** 9)
    rng = np.random.default_rng(6)
    x0 = rng.standard_normal(n * n)
    w = np.full(n * n, 0.3)
    A, At = solver.theta_ops(th)
    res = solver.fista(A, At, x0, w, np.ones(n * n), 1.0, max_iters=1)
    assert np.abs(res.x - solver.soft(x0, 0.3)).max() < 1e-15


def test_lambda_above_lambda_max_gives_zero():
    th = _small_thetak()
    rng = np.random.default_rng(7)
    x0 = rng.standard_normal(256)
    lam_max = np.abs(th.matT @ x0).max()
    A, At = solver.theta_ops(th)
    L, _ = precond.power_iteration(lambda v: At(A(v)), np.ones(256))
    res = solver.fista(A, At, x0, np.full(256, 1.0001 * lam_max), np.ones(256),
                       precond.step_size(L), max_iters=50)
    assert np.all(res.x == 0.0)


def test_theta_full_matches_exact_operator_trajectory():
    n, J = 16, 2
    psf = PSFS["motion"]
    prob_rng = np.random.default_rng(8)
    u0 = prob_rng.standard_normal((n, n))
    th = theta.build_theta(psf, n, n, "db4", J, K=10 ** 12)
    x0 = wavelet.dwt2(u0, "db4", J)
    w = np.full(n * n, 0.05)
    A, At = solver.theta_ops(th)
    Ae, Aet = solver.exact_ops(psf, n, n, "db4", J)
    L, _ = precond.power_iteration(lambda v: At(A(v)), np.ones(n * n))
    tau = precond.step_size(L)
    r1 = solver.fista(A, At, x0, w, np.ones(n * n), tau, max_iters=40)
    r2 = solver.fista(Ae, Aet, u0.ravel(), w, np.ones(n * n), tau, max_iters=40)
    assert np.abs(r1.x - r2.x).max() < 1e-12 * max(1.0, np.abs(r2.x).max())
    assert abs(r1.objective - r2.objective) < 1e-12 * r2.objective


@pytest.mark.parametrize("pc", ["none", "jacobi", "spai"])
def test_fista_converges_to_cd_solution_and_kkt(pc):
    th = _small_thetak()
    rng = np.random.default_rng(9)
    x0 = rng.standard_normal(256) * 2.0
    lam = 0.05
    w = np.full(256, lam)
    A, At = solver.theta_ops(th)
    P, _ = _P(th, pc)
    L, _ = precond.power_iteration(lambda v: At(A(v)), P)
    res = solver.fista(A, At, x0, w, P, precond.step_size(L), max_iters=200000, tol=1e-13,
                       check_every=10)
    assert res.rel_gap <= 1e-13
    for (_, pr, gp) in res.history:
        assert gp >= -1e-12 * pr
    Ad = th.mat.toarray()
    xcd = solver.lasso_cd(Ad, x0, w, tol=1e-15)
    Ecd = solver.objective(Ad @ xcd - x0, xcd, w)
    assert abs(res.objective - Ecd) <= 1e-9 * Ecd
    out, on = solver.kkt_residuals((Ad,), res.x, x0, w)
    assert out <= 1e-6 and on <= 1e-6


def test_gap_decreases_to_zero():
    th = _small_thetak()
    rng = np.random.default_rng(10)
    x0 = rng.standard_normal(256)
    A, At = solver.theta_ops(th)
    L, _ = precond.power_iteration(lambda v: At(A(v)), np.ones(256))
    res = solver.fista(A, At, x0, np.full(256, 0.02), np.ones(256), precond.step_size(L),
                       max_iters=3000, record_every=100)
    gaps = [g for (_, _, g) in res.history]
    assert all(g >= 0 for g in gaps)
    assert gaps[-1] < 1e-3 * gaps[0]


def _golden_rows(name):
    from fractions import Fraction
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            f = line.split()
            rows.append((int(f[0]), [float(Fraction(s)) for s in f[1:]]))
    return rows


def test_fista_momentum_schedule_hand_derived_trajectory():
    """Algorithm 3's momentum beta_k = (k-1)/(k+2) pinned by a trajectory derived by hand
    (tests/golden/fista_diag_momentum.txt): a diagonal A with a preconditioner, exact dyadic
    values for k = 1..6. A different momentum rule (k/(k+3), (k-1)/(k+3), Beck-Teboulle's t_k
    recursion, an index shifted by one), a dropped P, or a threshold of tau w instead of
    tau w / P changes x^(2) or x^(3)."""
    A = np.array([1.0, 0.5, 1.0])
    b = np.array([4.0, -3.0, 0.25])
    w = np.array([1.0, 0.5, 1.0])
    P = np.array([1.0, 0.25, 2.0])
    for k, xk in _golden_rows("fista_diag_momentum.txt"):
        res = solver.fista(lambda v: A * v, lambda v: A * v, b, w, P, 0.5, max_iters=k)
        assert res.iters == k
        assert np.array_equal(res.x, np.array(xk)), (k, res.x, xk)


def test_ista_hand_derived_trajectory():
    """ISTA (momentum off) on the same diagonal problem: the hand-derived contraction
    (tests/golden/ista_diag.txt). Any extrapolation left in, or a step applied to y instead
    of x, changes x^(3)."""
    A = np.array([1.0, 0.5, 1.0])
    b = np.array([4.0, -3.0, 0.25])
    w = np.array([1.0, 0.5, 1.0])
    P = np.array([1.0, 0.25, 2.0])
    for k, xk in _golden_rows("ista_diag.txt"):
        res = solver.fista(lambda v: A * v, lambda v: A * v, b, w, P, 0.5, max_iters=k, momentum=False)
        assert np.array_equal(res.x, np.array(xk)), (k, res.x, xk)


@pytest.mark.parametrize("shape,wname,J", [((16, 16), "db2", 2), ((16, 32), "db3", 2), ((32, 32), "sym4", 2)])
def test_theta_entry_equals_the_dense_definition(shape, wname, J):
    """theta.theta_entry (one entry from the separable 1-D factors, any size) against
    D H D^T built from unit vectors, on a non-symmetric PSF (a dropped transpose or a sign
    of the correlation shift changes the entries)."""
    R, C = shape
    psf = synthetic.motion_line_psf(5, 0.7)
    T = theta.theta_dense(R, C, psf, wname, J)
    lay = wavelet.layout(R, C, J)
    rng = np.random.default_rng(4)
    for _ in range(200):
        a, b = int(rng.integers(len(lay))), int(rng.integers(len(lay)))
        sa, sb = lay[a], lay[b]
        p = (int(rng.integers(sa.rows)), int(rng.integers(sa.cols)))
        q = (int(rng.integers(sb.rows)), int(rng.integers(sb.cols)))
        v = theta.theta_entry(psf, R, C, wname, J, a, p, b, q)
        ref = T[sa.offset + p[0] * sa.cols + p[1], sb.offset + q[0] * sb.cols + q[1]]
        assert abs(v - ref) <= 1e-14


def test_theta_entry_equals_the_probe_construction():
    n, J = 64, 3
    psf = synthetic.gaussian_psf(1.5, 9)
    th = theta.build_theta(psf, n, n, "db4", J, K=10**12)
    lay = th.lay
    A = th.mat.tocsr()
    rng = np.random.default_rng(5)
    for _ in range(100):
        a, b = int(rng.integers(len(lay))), int(rng.integers(len(lay)))
        sa, sb = lay[a], lay[b]
        p = (int(rng.integers(sa.rows)), int(rng.integers(sa.cols)))
        q = (int(rng.integers(sb.rows)), int(rng.integers(sb.cols)))
        ref = A[sa.offset + p[0] * sa.cols + p[1], sb.offset + q[0] * sb.cols + q[1]]
        assert abs(theta.theta_entry(psf, n, n, "db4", J, a, p, b, q) - ref) <= 1e-13


@pytest.mark.parametrize("shape,wname,J", [((16, 16), "db2", 2), ((32, 32), "db4", 3)])
def test_theta_of_the_autocorrelation_is_the_normal_operator(shape, wname, J):
    """HᵀH is the periodic convolution with the PSF's autocorrelation, so Algorithm 2 run on
    that PSF (unthresholded) must give ΘᵀΘ. Row and column taps of the probe construction
    meet in the product, so a transposed block, a flipped probe or a wrong row/column rule
    for coarser outputs breaks the identity. The PSF is a seeded random 5 x 5 array without
    point symmetry, so the self-convolution h * h (a plausible slip for h~ * h) fails too."""
    from scipy.signal import correlate2d
    R, C = shape
    psf = np.random.default_rng(8).random((5, 5))
    psf /= psf.sum()
    auto = correlate2d(psf, psf, mode="full")
    th = theta.build_theta(psf, R, C, wname, J, K=10**12)
    hess = theta.build_theta(auto, R, C, wname, J, K=10**12)
    normal = (th.matT @ th.mat).toarray()
    assert np.abs(hess.mat.toarray() - normal).max() <= 1e-13 * np.abs(normal).max()
