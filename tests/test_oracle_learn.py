"""Pins of the oracle's learned-correction reference (no GPU)."""
from math import erf, sqrt

import numpy as np

from oracle import fmm, learn
from paper_2011_07099_gb300 import inputs


def _phi(x):
    return 0.5 * (1.0 + erf(x / sqrt(2.0)))


def test_gelu_is_z_times_normal_cdf():
    for z, want in [(0.0, 0.0), (1.0, 0.8413447460685429), (-1.0, -0.15865525393145707), (2.5, 2.5 * 0.9937903346742238)]:
        assert abs(float(learn.gelu(np.array(z))) - want) < 1e-15


def test_mlp_with_hand_set_weights():
    w = np.zeros(learn.N_PARAMS)
    W1, b1, W2, b2, W3, b3, W4, b4 = learn.unpack(w.copy())
    o = 0
    sizes = [64 * 5, 64, 64 * 64, 64, 64 * 64, 64, 64, 1]
    offs = np.cumsum([0] + sizes)
    w[offs[0] + 0 * 5 + 0] = 1.0        # W1[0][0]
    w[offs[2] + 0 * 64 + 0] = 2.0       # W2[0][0]
    w[offs[4] + 0 * 64 + 0] = 1.0       # W3[0][0]
    w[offs[6] + 0] = 3.0                # W4[0]
    w[offs[7]] = 0.5                    # b4
    x0 = 0.7
    g = lambda z: z * _phi(z)
    want = 3.0 * g(g(2.0 * g(x0))) + 0.5
    got = learn.mlp(w, np.array([[x0, 0.1, 0.2, 0.3, 1.0]]))[0]
    assert abs(got - want) < 1e-14


def test_correction_keeps_the_symmetries_of_g_s1():
    rng = np.random.default_rng(1)
    w = rng.normal(0, 0.5, learn.N_PARAMS)
    n = rng.integers(-11, 12, (40, 3))
    c = learn.table_correction(w, 4, 3, n)
    # G (field 0): even in every component and symmetric under axis permutations
    for flip in ([-1, 1, 1], [1, -1, 1], [1, 1, -1]):
        np.testing.assert_allclose(learn.table_correction(w, 4, 3, n * np.array(flip))[:, 0], c[:, 0], rtol=1e-14)
    np.testing.assert_allclose(learn.table_correction(w, 4, 3, n[:, [2, 0, 1]])[:, 0], c[:, 0], rtol=1e-14)
    # -dG/dx: odd in x, even in y and z; -dG/dy is -dG/dx with x and y swapped
    np.testing.assert_allclose(learn.table_correction(w, 4, 3, n * np.array([-1, 1, 1]))[:, 1], -c[:, 1], rtol=1e-14)
    np.testing.assert_allclose(learn.table_correction(w, 4, 3, n * np.array([1, -1, -1]))[:, 1], c[:, 1], rtol=1e-14)
    np.testing.assert_allclose(learn.table_correction(w, 4, 3, n[:, [1, 0, 2]])[:, 2], c[:, 1], rtol=1e-14)
    assert np.all(c[n[:, 0] == 0, 1] == 0.0)


def test_correction_is_periodic():
    rng = np.random.default_rng(2)
    w = rng.normal(0, 0.5, learn.N_PARAMS)
    p, level = 3, 2
    period = 2 ** level * p
    n = rng.integers(-9, 10, (30, 3))
    c = learn.table_correction(w, level, p, n)
    for e in np.eye(3, dtype=np.int64):
        np.testing.assert_allclose(learn.table_correction(w, level, p, n + period * e), c, rtol=1e-14)


def test_zero_weights_give_the_plain_fmm():
    rho = inputs.lognormal(16, sigma=0.5, seed=4)
    a = fmm.solve(rho, 3, 2)
    b = fmm.solve(rho, 3, 2, correction=learn.correction_fn(np.zeros(learn.N_PARAMS)))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
