"""Pins of the oracle's Green's functions against what the paper and the
mathematics fix (no GPU)."""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import green, pm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _identities():
    rows = {}
    with open(os.path.join(GOLDEN, "xi_identities.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, order, c1, c3, c5 = line.split()
            rows[name] = (int(order), float(Fraction(c1)), float(Fraction(c3)), float(Fraction(c5)))
    return rows


def test_xi_s1_is_the_printed_identity():
    # Sec. 3: (9/8) sin t - (1/8) sin(3t)/3 = t + O(t^5); xi_s1(t) is that
    # expression with t -> pi t, divided by pi.
    order, c1, c3, c5 = _identities()["s1"]
    t = np.linspace(-2.0, 2.0, 101)
    printed = (c1 * np.sin(t) + c3 * np.sin(3 * t) / 3 + c5 * np.sin(5 * t) / 5) / np.pi
    np.testing.assert_allclose(green.xi_s1(t / np.pi), printed, rtol=0, atol=1e-15)


@pytest.mark.parametrize("name", ["s1", "s2"])
def test_printed_identities_have_the_stated_order(name):
    # The remainder of each printed combination scales as t^order.
    order, c1, c3, c5 = _identities()[name]
    f = lambda t: c1 * np.sin(t) + c3 * np.sin(3 * t) / 3 + c5 * np.sin(5 * t) / 5 - t
    r = f(2e-2) / f(1e-2)
    assert abs(np.log2(r) - order) < 0.02


def test_xi_s1_taylor_t5_coefficient():
    # xi(t) = t - (3 pi^4 / 40) t^5 + O(t^7): the t^3 term cancels (Sec. 3).
    t = 1e-2
    c5 = (green.xi_s1(t) - t) / t ** 5
    assert abs(c5 / (-3 * np.pi ** 4 / 40) - 1) < 1e-3


def test_xi_s1_odd_periodic_and_smooth_at_half_box():
    t = np.linspace(-1, 1, 41)
    np.testing.assert_allclose(green.xi_s1(t + 1), -green.xi_s1(t), atol=1e-15)
    assert abs(green.xi_s1(0.5) - 7 / (6 * np.pi)) < 1e-15
    assert abs(green.dxi_s1(0.5)) < 1e-15            # differentiable G at L/2 (Sec. 3)
    tt = np.linspace(0, 1, 10001)
    assert green.xi_s1(tt).max() <= 7 / (6 * np.pi) + 1e-15


def test_g_s1_periodic_even_and_newtonian_at_small_r():
    rng = np.random.default_rng(0)
    x = rng.uniform(-0.5, 0.5, (200, 3))
    g = green.g_s1(x)
    for e in np.eye(3):
        np.testing.assert_allclose(green.g_s1(x + e), g, rtol=1e-12)
        np.testing.assert_allclose(green.g_s1(x * (1 - 2 * e)), g, rtol=1e-13)
    d = rng.normal(size=(50, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    for r in (1e-2, 1e-3):
        rel = green.g_s1(r * d) / green.g0(r) - 1
        # |xhat|/|x| - 1 = -(3 pi^4/40) sum(x_i^6)/r^2 + ..., at most 7.31 r^4
        assert np.abs(rel).max() < 3 * np.pi ** 4 / 40 * r ** 4 * 1.01


def test_grad_g_s1_matches_finite_differences_and_vanishes_at_half_box():
    rng = np.random.default_rng(1)
    x = rng.uniform(-0.5, 0.5, (100, 3))
    x = x[np.linalg.norm(x, axis=1) > 0.05]
    h = 1e-6
    fd = np.stack([(green.g_s1(x + h * e) - green.g_s1(x - h * e)) / (2 * h) for e in np.eye(3)], -1)
    np.testing.assert_allclose(green.grad_g_s1(x), fd, rtol=1e-6, atol=1e-8)
    y = rng.uniform(-0.5, 0.5, (20, 3))
    for c in range(3):
        for s in (0.5, -0.5):
            z = y.copy()
            z[:, c] = s
            assert np.abs(green.grad_g_s1(z)[:, c]).max() < 1e-15


def test_g_x_is_not_differentiable_at_half_box():
    # Sec. 1: G_X is continuous but has a kink at |x| = L/2.
    e = np.array([[0.5 - 1e-7, 0.1, 0.0]])
    f = np.array([[0.5 + 1e-7, 0.1, 0.0]])
    assert np.sign(green.grad_g_x(e)[0, 0]) != np.sign(green.grad_g_x(f)[0, 0])
    assert abs(green.g_x(e)[0] - green.g_x(f)[0]) < 1e-6


def test_self_term_is_the_cube_mean_of_inverse_r():
    # Midpoint quadrature of 1/r over the unit cube (no node at the origin).
    k = 240
    c = (np.arange(k) + 0.5) / k - 0.5
    z, y, x = np.meshgrid(c, c, c, indexing="ij", sparse=True)
    q = np.mean(1.0 / np.sqrt(x * x + y * y + z * z))
    assert abs(q / green.CUBE_MEAN_INV_R - 1) < 2e-3
    assert abs(green.self_term(16) + green.CUBE_MEAN_INV_R * 16 / (4 * np.pi)) < 1e-12


def test_g_k_single_mode_closed_form():
    # Sec. 1 eq. gfk: for rho = cos(2 pi n.x) the solution of lap Phi = rho is
    # Phi = -rho / (4 pi^2 |n|^2); g = -grad Phi.
    n = 16
    x = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    ph = 2 * np.pi * (X + 2 * Y - 3 * Z)
    rho = 1.0 + np.cos(ph)
    phi, g = pm.pm_gk(pm.masses(rho))
    k2 = 4 * np.pi ** 2 * 14
    np.testing.assert_allclose(phi, -np.cos(ph) / k2, atol=1e-14)
    gx_exact = -(np.sin(ph) * 2 * np.pi) / k2          # -d/dx of -cos/k2
    np.testing.assert_allclose(g[0], gx_exact, atol=1e-14)
    np.testing.assert_allclose(g[2], -3 * gx_exact, atol=1e-14)
    assert abs(phi.mean()) < 1e-16


def test_ansatz_is_newtonian_at_small_scales_and_smooth_at_half_the_box():
    # Sec. 3: for any a_k, xhat -> x at small scales and xi_n is differentiable
    # (zero slope) at half the box; a_1 = -1/8 is G_S1
    rng = np.random.default_rng(3)
    t = np.array([1e-5, -2e-5])
    for a in ([-0.125], [-0.12], [0.05, -0.02], list(rng.normal(0, 0.1, 4))):
        np.testing.assert_allclose(green.xi_ansatz(t, a), t, rtol=1e-8)
        np.testing.assert_allclose(green.dxi_ansatz(np.array([0.5, -0.5]), a), 0.0, atol=1e-15)
        np.testing.assert_allclose(green.xi_ansatz(t + 1.0, a), -green.xi_ansatz(t, a), rtol=1e-6, atol=1e-15)
    x = rng.uniform(-0.5, 0.5, (50, 3))
    np.testing.assert_allclose(green.g_s(x, [-0.125]), green.g_s1(x), rtol=1e-14)
    np.testing.assert_allclose(green.grad_g_s(x, [-0.125]), green.grad_g_s1(x), rtol=1e-12, atol=1e-14)


def test_ansatz_gradient_is_the_derivative_of_the_ansatz():
    rng = np.random.default_rng(4)
    a = [-0.12, 0.03]
    x = rng.uniform(-0.45, 0.45, (20, 3))
    h = 1e-6
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        fd = (green.g_s(x + e, a) - green.g_s(x - e, a)) / (2 * h)
        np.testing.assert_allclose(green.grad_g_s(x, a)[:, i], fd, rtol=1e-6, atol=1e-9)
