"""Pins of the isolated (non-periodic) references of the Sec. 3 accuracy
experiment: brute force, the exact two-level case, the Hockney halo, the
4th-order difference, zone coverage and the eq. gerr norms (no GPU)."""
import os

import numpy as np
import pytest

from oracle import green
from oracle import nonperiodic as npo
from paper_2011_07099_gb300 import inputs


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_padded_pm_equals_the_isolated_brute_force_sum():
    rho = inputs.plummer(8, n_clumps=3, seed=1, a_min=0.5, a_max=2.0)
    m = npo.masses_isolated(rho)
    sv = green.self_term(8)
    phi_d, _ = npo.direct_isolated(m, sv)
    phi_p, _ = npo.pm_isolated(m, sv)
    assert _rel(phi_p, phi_d) < 1e-13


def test_padded_pm_is_exact_two_cells_beyond_the_faces():
    # the 4th-order difference at the box faces reads the potential at
    # t = -2, -1, N, N + 1: the padded convolution must hold it exactly there
    n = 8
    rho = inputs.plummer(n, n_clumps=3, seed=4, a_min=0.5, a_max=2.0)
    m = npo.masses_isolated(rho)
    sv = green.self_term(n)
    t = np.arange(-2, n + 2)
    tz, ty, tx = np.meshgrid(t, t, t, indexing="ij")
    T = np.stack([tx, ty, tz], -1).reshape(-1, 3).astype(float)
    r = np.arange(n)
    sz, sy, sx = np.meshgrid(r, r, r, indexing="ij")
    S = np.stack([sx, sy, sz], -1).reshape(-1, 3).astype(float)
    brute = (npo.g0_at((T[:, None, :] - S[None, :, :]) / n, sv) @ m.reshape(-1)).reshape(n + 4, n + 4, n + 4)
    _, pad = npo.pm_isolated(m, sv)
    idx = t % pad.shape[0]
    assert np.abs(pad[np.ix_(idx, idx, idx)] - brute).max() <= 1e-13 * np.abs(brute).max()


@pytest.mark.parametrize("n", [8, 16])
def test_isolated_two_level_tree_with_gridlet_equal_subgrid_is_exact(n):
    rho = inputs.plummer(n, n_clumps=4, seed=n, a_min=0.5, a_max=2.0)
    phi, g = npo.solve_isolated(rho, 2, n // 4)
    pd, gd = npo.direct_isolated(npo.masses_isolated(rho), green.self_term(n))
    assert _rel(phi, pd) < 1e-12 and _rel(g, gd) < 1e-12


def test_isolated_fmm_error_falls_with_order_and_net_force_vanishes():
    rho = inputs.plummer(16, n_clumps=4, seed=2, a_min=0.5, a_max=3.0)
    m = npo.masses_isolated(rho)
    pd, gd = npo.direct_isolated(m, green.self_term(16))
    errs = []
    for p in (1, 2, 3, 4):
        phi, g = npo.solve_isolated(rho, 3, p)
        errs.append(_rel(g, gd))
        f = (m[None] * g).sum(axis=(1, 2, 3))            # sum m g: zero by antisymmetry
        assert np.abs(f).max() < 1e-12 * (np.abs(m)[None] * np.abs(g)).sum()
    assert all(b < a for a, b in zip(errs, errs[1:])) and errs[-1] < 1e-3


@pytest.mark.parametrize("L", [3, 4])
def test_isolated_zones_cover_every_leaf_exactly_once(L):
    for leaf in [(0, 0, 0), (1, 2, 3), (2 ** L - 1, 0, 2 ** L - 1)]:
        count = {}
        for lev in range(2, L + 1):
            anc = tuple(i >> (L - lev) for i in leaf)
            for src in npo.interaction_list_np(lev, anc):
                sh = L - lev
                for dz in range(2 ** sh):
                    for dy in range(2 ** sh):
                        for dx in range(2 ** sh):
                            q = ((src[0] << sh) + dz, (src[1] << sh) + dy, (src[2] << sh) + dx)
                            count[q] = count.get(q, 0) + 1
        for q in npo.neighbours_np(L, leaf):
            count[q] = count.get(q, 0) + 1
        n = 2 ** L
        assert len(count) == n ** 3 and set(count.values()) == {1}


def test_fourth_order_difference_is_exact_for_quartics_and_converges_at_h4():
    n = 16
    x = (np.arange(n) + 0.5) / n
    # a quartic: the stencil is exact for polynomials of degree <= 4 away from the wrap
    f = np.broadcast_to((x ** 4 - 2 * x ** 3 + x)[None, None, :], (n, n, n)).copy()
    d = npo.fd4(f, 1.0 / n, 2)
    exact = 4 * x ** 3 - 6 * x ** 2 + 1
    assert np.abs(d[0, 0, 2:-2] - exact[2:-2]).max() < 1e-12
    errs = []
    for n in (16, 32, 64):
        x = (np.arange(n) + 0.5) / n
        phi = np.broadcast_to(np.sin(2 * np.pi * x)[None, None, :], (n, n, n)).copy()
        g = npo.fd4_accel_periodic(phi)
        errs.append(np.abs(g[0, 0, 0] + 2 * np.pi * np.cos(2 * np.pi * x)).max())
    assert errs[0] / errs[1] > 14 and errs[1] / errs[2] > 14          # ~2^4


def test_gerr_norms():
    rng = np.random.default_rng(0)
    a, b = rng.standard_normal((3, 4, 4, 4)), rng.standard_normal((3, 4, 4, 4))
    assert npo.gf_error(a, b, a, b) == (0.0, 0.0)
    d = np.zeros((3, 4, 4, 4))
    d[0, 1, 2, 3] = 3.0
    d[1, 1, 2, 3] = 4.0
    lmax, l2 = npo.gf_error(d, 0 * d, 0 * d, 0 * d)
    assert lmax == pytest.approx(5.0) and l2 == pytest.approx(5.0 / 8.0)


def test_padded_accelerations_equal_the_isolated_brute_force_sum():
    rho = inputs.plummer(8, n_clumps=3, seed=2, a_min=0.5, a_max=2.0)
    m = npo.masses_isolated(rho)
    _, g_d = npo.direct_isolated(m, green.self_term(8))
    assert _rel(npo.pm_isolated_accel(m), g_d) < 1e-13


def _point_source(n, c):
    rho = np.zeros((n, n, n))
    rho[c, c, c] = float(n) ** 3        # unit mass in a unit box
    return rho


def _gerr_terms(rho, L, p):
    from oracle import fmm, pm
    n = rho.shape[0]
    _, g_pm = pm.pm(pm.masses(rho), green.g_s1, green.grad_g_s1, green.self_term(n))
    g_pmn = npo.pm_isolated_accel(npo.masses_isolated(rho))
    _, g_f = fmm.solve(rho, L, p)
    _, g_fn = npo.solve_isolated(rho, L, p)
    return g_f, g_pm, g_fn, g_pmn


def test_gerr_vanishes_when_the_gridlet_is_the_sub_grid():
    # with two levels and p = S the expansions are exact (Sec. 3), so both
    # FMM solutions equal their PM solutions and eq. gerr is zero
    g_f, g_pm, g_fn, g_pmn = _gerr_terms(_point_source(16, 0), 2, 4)
    assert npo.me_error(g_fn, g_pmn)[0] < 1e-11
    assert max(npo.gf_error(g_f, g_pm, g_fn, g_pmn)) < 1e-11


def _table1_3d():
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_3d.txt")
    rows = np.loadtxt(path, comments="#")
    return {int(r[0]): (r[1], r[2]) for r in rows}


def test_gerr_of_g_s1_is_within_the_stated_accuracy_from_six_multipoles():
    # Sec. 3 (abstract, Fig. eng): from N_g = 6 the Green's-function error
    # of G_S1 is below 1e-3 in L_MAX and 1e-4 in L2; at N_g = 4 it is not.
    # Each order lands on the side of those bounds that its Table 1 row
    # does.  The unit source sits at the box centre, so that the
    # non-periodic problem has the periodic one's tree geometry around it
    # and eq. gerr subtracts the expansion error; at order 6 the expansion
    # error itself is the larger one.
    table = _table1_3d()
    rho = _point_source(32, 16)
    for p in (4, 6):
        terms = _gerr_terms(rho, 2, p)
        lmax, l2 = npo.gf_error(*terms)
        t_lmax, t_l2 = table[p]
        assert (lmax < 1e-3) == (t_lmax < 1e-3) and (l2 < 1e-4) == (t_l2 < 1e-4), (p, lmax, l2)
        if p == 6:
            assert npo.me_error(terms[2], terms[3])[0] > lmax


def test_sampled_isolated_solve_equals_the_full_one():
    # solve_isolated_at (leaves, and cells within them) must return exactly
    # what solve_isolated computes there
    N, L, p = 16, 2, 3
    rho = inputs.plummer(N, n_clumps=3, seed=12, a_min=0.5, a_max=2.0)
    phi, g = npo.solve_isolated(rho, L, p)
    leaves = np.array([[0, 0, 0], [3, 1, 2], [2, 3, 3]])
    cells = np.array([0, 5, 17, 63])
    S = N >> L
    full = np.concatenate([phi[None], g])
    want = np.stack([full[:, a * S:(a + 1) * S, b * S:(b + 1) * S, c * S:(c + 1) * S].reshape(4, -1)
                     for a, b, c in leaves])
    got = npo.solve_isolated_at(rho, L, p, leaves)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    got_c = npo.solve_isolated_at(rho, L, p, leaves, cells)
    np.testing.assert_allclose(got_c, want[:, :, cells], rtol=1e-12, atol=1e-12 * np.abs(want).max())
