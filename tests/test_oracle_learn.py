"""Pins of the oracle's learned-correction reference (no GPU)."""
from math import erf, sqrt

import numpy as np
import pytest

from oracle import fmm, green, learn, pm
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


def _brute_corrected(rho, w, S, entry_fn=None):
    """Direct periodic sum of the two-level tree (L = 2, p = S) with the
    corrected kernel written out per cell pair: at level 2 the gridlet points
    are the cell centres (spacing 1/N), so the interaction-zone pairs use
    G_S1 plus the table correction at n = target cell - source cell (x, y, z),
    and the 27 neighbour leaves use G_S1 alone (the near zone is exact)."""
    N = rho.shape[0]
    m = pm.masses(np.asarray(rho, np.float64)).ravel()
    idx = np.indices((N, N, N)).reshape(3, -1).T                  # (z, y, x), row-major cell order
    xyz = idx[:, ::-1]
    d = xyz[:, None, :] - xyz[None, :, :]                          # (target, source, 3) in cells
    leaf = idx // S
    near = np.all(np.isin((leaf[:, None, :] - leaf[None, :, :]) % 4, [0, 1, 3]), axis=-1)
    G = green.g_s1(d / N, self_value=green.self_term(N))
    mdG = -green.grad_g_s1(d / N)                                  # (t, s, 3)
    uniq, inv = np.unique(d.reshape(-1, 3), axis=0, return_inverse=True)
    entry_fn = entry_fn or (lambda n: learn.table_correction(w, 2, S, n))
    corr = entry_fn(uniq)[inv.ravel()].reshape(N ** 3, N ** 3, 4)
    corr[near] = 0.0
    phi = (G + corr[..., 0]) @ m
    g = np.stack([(mdG[..., c] + corr[..., 1 + c]) @ m for c in range(3)])
    return phi.reshape(N, N, N), g.reshape(3, N, N, N)


@pytest.mark.parametrize("N", [8, 12])
def test_corrected_two_level_tree_equals_the_corrected_direct_sum(N):
    # Sec. 3's exact case (two levels, gridlet = sub-grid) carried over to the
    # corrected tables: the FMM with correction_fn(w) must equal the direct
    # sum whose far-zone kernel is G_S1 + table_correction at the cell offset.
    # This pins the mapping n = o p + r - s of the correction into eq. fmm2.
    S = N // 4
    rho = inputs.plummer(N, n_clumps=3, seed=N, a_min=0.5, a_max=2.0)
    w = np.random.default_rng(N).normal(0.0, 0.5, learn.N_PARAMS)
    phi, g = fmm.solve(rho, 2, S, correction=learn.correction_fn(w))
    bphi, bg = _brute_corrected(rho, w, S)
    plain_phi, plain_g = fmm.solve(rho, 2, S)
    # the correction is not negligible at this weight scale ...
    assert np.linalg.norm(plain_phi - bphi) / np.linalg.norm(bphi) > 1e-5
    assert np.linalg.norm(plain_g - bg) / np.linalg.norm(bg) > 1e-5
    # ... and the corrected FMM reproduces the corrected direct sum exactly
    assert np.linalg.norm(phi - bphi) / np.linalg.norm(bphi) < 1e-12
    assert np.linalg.norm(g - bg) / np.linalg.norm(bg) < 1e-12


def test_planted_flip_of_r_minus_s_in_the_correction_is_caught():
    # n = o p + s - r instead of o p + r - s: the translation matrices of the
    # correction come out transposed in (r, s), and the exact case fails
    N, S = 8, 2
    rho = inputs.plummer(N, n_clumps=3, seed=N, a_min=0.5, a_max=2.0)
    w = np.random.default_rng(N).normal(0.0, 0.5, learn.N_PARAMS)
    good = learn.correction_fn(w)
    flipped = lambda level, p, off: np.swapaxes(good(level, p, off), 1, 2)
    phi, g = fmm.solve(rho, 2, S, correction=flipped)
    bphi, bg = _brute_corrected(rho, w, S)
    assert np.linalg.norm(phi - bphi) / np.linalg.norm(bphi) > 1e-5
    assert np.linalg.norm(g - bg) / np.linalg.norm(bg) > 1e-3


@pytest.mark.parametrize("N", [8, 12])
def test_grid_model_two_level_tree_equals_the_corrected_direct_sum(N):
    # the same exact case for the grid model of G_* (Sec. 4): every folded
    # table value its own parameter, added at the cell offset of each
    # interaction-zone pair
    S = N // 4
    rho = inputs.plummer(N, n_clumps=3, seed=N + 1, a_min=0.5, a_max=2.0)
    theta = np.random.default_rng(N + 1).normal(0.0, 50.0, learn.grid_size(2, S))
    phi, g = fmm.solve(rho, 2, S, correction=learn.grid_correction_fn(theta))
    bphi, bg = _brute_corrected(rho, None, S, entry_fn=lambda n: learn.grid_table_correction(theta, 2, S, n))
    plain_phi, plain_g = fmm.solve(rho, 2, S)
    assert np.linalg.norm(plain_g - bg) / np.linalg.norm(bg) > 1e-4
    assert np.linalg.norm(phi - bphi) / np.linalg.norm(bphi) < 1e-12
    assert np.linalg.norm(g - bg) / np.linalg.norm(bg) < 1e-12


def test_grid_model_keeps_parity_and_periodicity():
    rng = np.random.default_rng(7)
    p, L = 3, 4
    theta = rng.normal(0.0, 1.0, learn.grid_size(L, p))
    for level in (2, 3, 4):
        n = rng.integers(-(4 * p - 1), 4 * p, (60, 3))
        c = learn.grid_table_correction(theta, level, p, n)
        for k in range(3):
            flip = np.ones(3, dtype=np.int64)
            flip[k] = -1
            cf = learn.grid_table_correction(theta, level, p, n * flip)
            np.testing.assert_array_equal(cf[:, 0], c[:, 0])                 # G even
            np.testing.assert_array_equal(cf[:, 1 + k], -c[:, 1 + k])        # own gradient odd
            others = [f for f in (1, 2, 3) if f != 1 + k]
            np.testing.assert_array_equal(cf[:, others], c[:, others])      # the others even
        period = 2 ** level * p
        for e in np.eye(3, dtype=np.int64):
            np.testing.assert_array_equal(learn.grid_table_correction(theta, level, p, n + period * e), c)
