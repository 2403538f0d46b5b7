"""Pins of the oracle's PM / brute-force convolution machinery (no GPU)."""
import numpy as np
import pytest

from oracle import green, pm
from paper_2011_07099_gb300 import inputs


@pytest.mark.parametrize("n", [8, 16])
@pytest.mark.parametrize("kind", ["s1", "x"])
def test_fft_pm_equals_brute_force(n, kind):
    rho = inputs.lognormal(n, sigma=1.0, seed=5)
    m = pm.masses(rho)
    gf, gg = (green.g_s1, green.grad_g_s1) if kind == "s1" else (green.g_x, green.grad_g_x)
    sv = green.self_term(n)
    p1, g1 = pm.direct(m, gf, gg, sv)
    p2, g2 = pm.pm(m, gf, gg, sv)
    assert np.abs(p1 - p2).max() <= 1e-13 * np.abs(p1).max()
    assert np.abs(g1 - g2).max() <= 1e-13 * np.abs(g1).max()


def test_spectral_g_k_equals_real_space_sum():
    n = 8
    rho = inputs.plummer(n, n_clumps=3, seed=2, a_min=0.5, a_max=1.5)
    m = pm.masses(rho)
    k, gr = pm.g_k_real_space(n)
    p1, g1 = pm.direct_tabulated(m, k, gr)
    p2, g2 = pm.pm_gk(m)
    assert np.abs(p1 - p2).max() <= 1e-13 * np.abs(p1).max()
    assert np.abs(g1 - g2).max() <= 1e-13 * np.abs(g1).max()


def test_net_force_and_mean_mode_vanish():
    n = 16
    rho = inputs.lognormal(n, sigma=0.5, seed=3)
    m = pm.masses(rho)
    phi, g = pm.pm(m, green.g_s1, green.grad_g_s1, green.self_term(n))
    # G even => grad G odd => sum_i m_i g_i = 0 (zero net force)
    f = (m[None] * g).sum(axis=(1, 2, 3))
    assert np.abs(f).max() < 1e-12 * (np.abs(m)[None] * np.abs(g)).sum()
    # sum_j m_j = 0 => the k=0 mode of Phi is 0
    assert abs(phi.sum()) < 1e-12 * np.abs(phi).sum()
    assert abs(m.sum()) < 1e-15


def test_g_s1_and_g_k_solutions_agree_on_smooth_fields():
    # Both are Green's functions of the same periodic Poisson problem (Sec. 1);
    # on a smooth field they differ only at the mesh scale.
    n = 32
    x = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    rho = 1 + 0.5 * np.cos(2 * np.pi * X) * np.cos(2 * np.pi * Y)
    m = pm.masses(rho)
    p1, g1 = pm.pm(m, green.g_s1, green.grad_g_s1, green.self_term(n))
    p2, g2 = pm.pm_gk(m)
    assert np.linalg.norm(g1 - g2) / np.linalg.norm(g2) < 2e-2
