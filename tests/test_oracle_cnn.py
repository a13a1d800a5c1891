"""Pins of the FP64 warm-start network: central finite differences and the Parseval
identity that makes the image-domain loss equal the coefficient-domain loss."""
import numpy as np
import pytest

from oracle import cnn, wavelet


@pytest.mark.parametrize("levels,channels", [(2, 4), (3, 3)])
def test_gradients_match_central_differences(levels, channels):
    rng = np.random.default_rng(3)
    p = cnn.init_params(levels, channels, seed=4, out_scale=1.0)
    for n in p:                       # nonzero biases so that every term is exercised
        if n.endswith(".b"):
            p[n] = 0.1 * rng.standard_normal(p[n].shape)
    u = rng.standard_normal((2, 16, 16))
    tgt = rng.standard_normal((2, 16, 16))
    loss, g, _ = cnn.loss_and_grads(p, u, tgt, levels)
    h = 1e-6
    for name, shp in cnn.param_shapes(levels, channels):
        flat = p[name].ravel()
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp, _, _ = cnn.loss_and_grads(p, u, tgt, levels)
            flat[i] = old - h
            lm, _, _ = cnn.loss_and_grads(p, u, tgt, levels)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].ravel()[i]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-8, (name, i, fd, an)


def test_flatten_roundtrip_and_count():
    p = cnn.init_params(4, 32, seed=1)
    v = cnn.flatten(p, 4, 32)
    assert v.size == sum(int(np.prod(s)) for _, s in cnn.param_shapes(4, 32))
    assert 120_000 < v.size < 160_000
    q = cnn.unflatten(v, 4, 32)
    assert all(np.array_equal(p[n], q[n]) for n in p)


def test_image_loss_equals_coefficient_loss():
    # Psi orthogonal (Parseval): ||v - Psi x*||^2 = ||Psi* v - x*||^2
    rng = np.random.default_rng(5)
    v = rng.standard_normal((32, 32))
    xs = rng.standard_normal(32 * 32)
    img = np.sum((v - wavelet.idwt2(xs, 32, 32, "db4", 3)) ** 2)
    coef = np.sum((wavelet.dwt2(v, "db4", 3) - xs) ** 2)
    assert abs(img - coef) < 1e-10 * img
