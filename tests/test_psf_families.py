"""The paper's blur families (Sec. 5: skewed Gaussian formula, spline motion blur; Table 3:
Gaussian, skewed, motion, Airy, defocus at widths 2.5 and 5) as the input generator makes
them: normalisation, support, and the property each family is defined by."""
import numpy as np
import pytest

from paper_1512_08401_gb300 import synthetic

FAMILIES = ["gaussian", "skewed", "motion", "airy", "defocus"]


@pytest.mark.parametrize("family", FAMILIES)
@pytest.mark.parametrize("width", [2.5, 5.0])
def test_psf_normalised_odd_nonnegative(family, width):
    h = synthetic.paper_blur(family, width)
    assert h.ndim == 2 and h.shape[0] == h.shape[1] and h.shape[0] % 2 == 1
    assert h.min() >= 0.0 and abs(h.sum() - 1.0) < 1e-12


def test_skewed_gaussian_follows_the_printed_formula():
    s = 5.0
    h = synthetic.skewed_gaussian_psf(s)
    c = h.shape[0] // 2
    t = np.arange(-c, c + 1)
    # columns: symmetric Gaussian of std s
    col = h.sum(axis=0)
    assert np.allclose(col, col[::-1], rtol=1e-12)
    # rows: std s for t1 >= 0, s/2 for t1 < 0 (the factor 4 in the exponent)
    row = h.sum(axis=1)
    assert row[c + 3] / row[c] == pytest.approx(np.exp(-9 / (2 * s * s)), rel=1e-12)
    assert row[c - 3] / row[c] == pytest.approx(np.exp(-36 / (2 * s * s)), rel=1e-12)
    assert 0.45 < row[:c].sum() / row[c + 1:].sum() < 0.55


def test_airy_first_dark_ring():
    s = 5.0
    h = synthetic.airy_psf(s)
    c = h.shape[0] // 2
    prof = h[c, c:]
    r = np.arange(len(prof))
    window = (r > 1.5 * s) & (r < 4 * s)
    r_min = r[window][np.argmin(prof[window])]
    assert abs(r_min - 2.895 * s) <= 1.0
    assert prof[r_min] < 0.02 * prof[0]


def test_defocus_is_a_disk():
    s = 5.0
    h = synthetic.defocus_psf(s)
    c = h.shape[0] // 2
    yy, xx = np.mgrid[-c:c + 1, -c:c + 1]
    r = np.sqrt(yy ** 2 + xx ** 2)
    assert np.all(h[r > s + 0.75] == 0.0)
    inner = h[r < s - 0.75]
    assert np.allclose(inner, inner.max(), rtol=1e-12)
    # pixel coverage fractions add up to the disk area (8 x 8 sub-samples per pixel)
    assert (h / h.max()).sum() == pytest.approx(np.pi * s * s, rel=0.01)


def test_spline_motion_seeded_and_centred():
    a = synthetic.spline_motion_psf(synthetic.rng_for(5, 0))
    b = synthetic.spline_motion_psf(synthetic.rng_for(5, 0))
    c = synthetic.spline_motion_psf(synthetic.rng_for(5, 1))
    assert np.array_equal(a, b) and not (a.shape == c.shape and np.array_equal(a, c))
    k = a.shape[0] // 2
    yy, xx = np.mgrid[-k:k + 1, -k:k + 1]
    assert abs((a * yy).sum()) < 0.5 and abs((a * xx).sum()) < 0.5
    # a thin curve: most pixels of the support are (numerically) empty
    assert (a > 1e-3 * a.max()).mean() < 0.5
