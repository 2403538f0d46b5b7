"""Pins of the oracle's step-by-step FMM against exact special cases, brute
force and invariants (no GPU)."""
import numpy as np
import pytest

from oracle import fmm, green, pm
from paper_2011_07099_gb300 import inputs


def _pm_s1(rho):
    n = rho.shape[0]
    return pm.pm(pm.masses(rho), green.g_s1, green.grad_g_s1, green.self_term(n))


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("n", [8, 16])
def test_two_level_tree_with_gridlet_equal_subgrid_is_exact(n):
    # Sec. 3: with 2 levels and gridlet == sub-grid, FMM and PM coincide.
    rho = inputs.plummer(n, n_clumps=4, seed=n, a_min=0.5, a_max=2.0)
    S = n // 4
    phi, g = fmm.solve(rho, 2, S)
    p_ref, g_ref = pm.direct(pm.masses(rho), green.g_s1, green.grad_g_s1, green.self_term(n))
    assert _rel(phi, p_ref) < 1e-12
    assert _rel(g, g_ref) < 1e-12


@pytest.mark.parametrize("p", [4, 6, 8])
def test_p2m_identity_when_gridlet_is_subgrid_and_monopole_when_p_is_1(p):
    np.testing.assert_allclose(fmm.p2m_matrix(p, p), np.eye(p ** 3), atol=1e-12)
    np.testing.assert_allclose(fmm.p2m_matrix(p, 1), np.ones((1, p ** 3)), atol=1e-13)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_per_axis_solve_equals_the_three_dimensional_vandermonde_system(p):
    # Sec. 2 defines the gridlet masses by V M = Q over all multi-indices
    # n_i < p; where that 3-D system is well conditioned its direct solution
    # must equal the per-axis (tensor-product) solution the oracle uses.
    cells = fmm.tensor_points((np.arange(8) + 0.5) / 8 - 0.5)
    direct = np.linalg.solve(fmm.vandermonde(p), fmm.moment_matrix(cells, p))
    np.testing.assert_allclose(fmm.p2m_matrix(8, p), direct, atol=1e-9)
    pts = fmm.tensor_points(fmm.gridlet_offsets(p)) / 2.0 + (np.array([1, 0, 1]) - 0.5) / 2.0
    direct = np.linalg.solve(fmm.vandermonde(p), fmm.moment_matrix(pts, p))
    np.testing.assert_allclose(fmm.m2m_matrix(p, (1, 0, 1)), direct, atol=1e-9)


@pytest.mark.parametrize("p", [5, 8])
def test_gridlet_masses_are_the_lagrange_basis_at_high_order(p):
    # The 1-D Vandermonde solution is the Lagrange basis of the gridlet points
    # (closed form, no linear solve): T[s, j] = prod_{k != s} (x_j - g_k) / (g_s - g_k).
    g = fmm.gridlet_offsets(p)
    for S in (p, 2 * p, 24):
        x = (np.arange(S) + 0.5) / S - 0.5
        T1 = np.ones((p, S))
        for s_ in range(p):
            for k in range(p):
                if k != s_:
                    T1[s_] *= (x - g[k]) / (g[s_] - g[k])
        want = np.kron(T1, np.kron(T1, T1))
        np.testing.assert_allclose(fmm.p2m_matrix(S, p), want, atol=1e-11 * np.abs(want).max())
    # M2M: moments n_i < p of the child gridlet are preserved (relative to scale)
    for child in [(0, 0, 0), (1, 0, 1), (1, 1, 1)]:
        pts = fmm.tensor_points(g) / 2.0 + (np.array(child) - 0.5) / 2.0
        W_child = fmm.moment_matrix(pts, p)
        got = fmm.vandermonde(p) @ fmm.m2m_matrix(p, child)
        np.testing.assert_allclose(got, W_child, atol=1e-12 * np.abs(fmm.m2m_matrix(p, child)).max())


def test_p2m_two_points_per_dimension_closed_form():
    # 1-D check: two gridlet points at -1/4, +1/4 of the node carry mass and
    # dipole, M_pm = Q0/2 +- 2 Q1 for a cell at offset x with unit mass.
    S, p = 4, 2
    P = fmm.p2m_matrix(S, p)
    # cell (cx, 0, 0) at x = (cx + 1/2)/S - 1/2; gridlet s = (sx, 0, 0)
    for cx in range(S):
        x = (cx + 0.5) / S - 0.5
        y = z = (0.5) / S - 0.5
        col = P[:, cx]                     # cell (0,0,cx)
        wy = [0.5 - 2 * y, 0.5 + 2 * y]
        wz = [0.5 - 2 * z, 0.5 + 2 * z]
        wx = [0.5 - 2 * x, 0.5 + 2 * x]
        exp = np.array([wz[a] * wy[b] * wx[c] for a in range(2) for b in range(2) for c in range(2)])
        np.testing.assert_allclose(col, exp, atol=1e-13)


@pytest.mark.parametrize("p", [2, 3, 4, 6, 8])
def test_m2m_after_p2m_equals_p2m_to_the_parent(p):
    rho = inputs.lognormal(16, sigma=1.0, seed=7)
    m = pm.masses(rho)
    M3 = fmm.p2m(m, 3, p)
    np.testing.assert_allclose(fmm.m2m(M3, p), fmm.p2m(m, 2, p), atol=1e-14 * np.abs(M3).max())


@pytest.mark.parametrize("p", [2, 4, 6, 8])
def test_l2l_and_l2p_reproduce_polynomials_below_the_order(p):
    # eq. fmm3 with T^T interpolates the parent's local field at the child
    # points (and L2P at the cell centres): any polynomial of degree < p per
    # axis, sampled at the parent gridlet points, is reproduced exactly
    rng = np.random.default_rng(p)
    coef = rng.standard_normal((p, p, p))
    def poly(pts):        # pts (k, 3) as (x, y, z), node-size units about the parent centre
        out = np.zeros(len(pts))
        for a in range(p):
            for b in range(p):
                for c in range(p):
                    out += coef[a, b, c] * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c
        return out
    parent = fmm.tensor_points(fmm.gridlet_offsets(p))
    Fp = poly(parent)[None, :]                                       # one field
    for child in [(0, 0, 0), (1, 0, 1), (1, 1, 1)]:
        got = fmm.l2l(Fp, p, child)[0]
        pts = fmm.tensor_points(fmm.gridlet_offsets(p)) / 2.0 + (np.array(child) - 0.5) / 2.0
        np.testing.assert_allclose(got, poly(pts), atol=1e-10 * np.abs(Fp).max())
    S = 2 * p
    cells = fmm.tensor_points((np.arange(S) + 0.5) / S - 0.5)
    np.testing.assert_allclose(Fp[0] @ fmm.l2p_matrix(S, p).T, poly(cells), atol=1e-10 * np.abs(Fp).max())


def test_mean_potential_vanishes_for_a_mean_free_field():
    # the k = 0 mode is removed (Sec. 1): the FMM potential of a mean-free
    # field has (nearly) zero mean, to the truncation of the expansion
    rho = inputs.lognormal(16, sigma=0.8, seed=11)
    phi, _ = fmm.solve(rho, 2, 4)
    p_ref, _ = _pm_s1(rho)
    assert abs(phi.mean() - p_ref.mean()) < 1e-12 * np.abs(p_ref).max()
    assert abs(p_ref.mean()) < 1e-3 * np.abs(p_ref).max()


def test_interaction_zone_sizes_and_translation_invariance():
    assert len(fmm.interaction_list(2, (0, 0, 0))) == 37
    for lev in (3, 4):
        n = 2 ** lev
        for node in [(0, 0, 0), (1, 2, 3), (n - 1, n - 2, 0), (5 % n, 7 % n, 6 % n)]:
            il = fmm.interaction_list(lev, node)
            assert len(il) == 189
            c = tuple(i % 2 for i in node)
            offs = fmm.interaction_offsets(lev, c)
            want = {tuple((np.array(node) - np.array(o)) % n) for o in offs}
            assert want == il


@pytest.mark.parametrize("L", [3, 4])
def test_zones_cover_every_leaf_exactly_once(L):
    leaf = (1, 2, 3) if L == 3 else (5, 0, 15)
    count = {}
    for lev in range(2, L + 1):
        anc = tuple(i >> (L - lev) for i in leaf)
        for src in fmm.interaction_list(lev, anc):
            sh = L - lev
            for a in range(2 ** sh):
                for b in range(2 ** sh):
                    for c in range(2 ** sh):
                        k = ((src[0] << sh) + a, (src[1] << sh) + b, (src[2] << sh) + c)
                        count[k] = count.get(k, 0) + 1
    for nb in fmm.neighbours(L, leaf):
        count[nb] = count.get(nb, 0) + 1
    assert len(count) == 8 ** L and set(count.values()) == {1}


def test_error_against_pm_falls_with_order_and_net_force_vanishes():
    rho = inputs.lognormal(32, sigma=0.5, seed=11)
    ref_phi, ref_g = _pm_s1(rho)
    errs = []
    for p in (2, 3, 4):
        phi, g = fmm.solve(rho, 3, p)
        errs.append((_rel(phi, ref_phi), _rel(g, ref_g)))
        m = pm.masses(rho)
        f = (m[None] * g).sum(axis=(1, 2, 3))
        assert np.abs(f).max() < 1e-11 * (np.abs(m)[None] * np.abs(g)).sum()
    assert errs[0][0] > errs[1][0] > errs[2][0]
    assert errs[0][1] > errs[1][1] > errs[2][1]
    assert errs[2][1] < 2e-3


def test_solve_at_matches_full_solve():
    rho = inputs.plummer(32, n_clumps=8, seed=3)
    L, p = 3, 2
    phi, g = fmm.solve(rho, L, p)
    full = np.concatenate([phi[None], g])
    leaves = np.array([[0, 0, 0], [7, 3, 1], [2, 7, 7]])
    got = fmm.solve_at(rho, L, p, leaves)
    S = 32 // 2 ** L
    for i, (a, b, c) in enumerate(leaves):
        ref = full[:, a * S:(a + 1) * S, b * S:(b + 1) * S, c * S:(c + 1) * S].reshape(4, -1)
        np.testing.assert_allclose(got[i], ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_planted_mistake_in_l2l_is_caught(monkeypatch):
    # Using T instead of its transpose in eq. fmm3 breaks the exact-parent
    # property that the convergence pins rely on.
    rho = inputs.lognormal(16, sigma=0.5, seed=2)
    ref_phi, ref_g = _pm_s1(rho)
    good = _rel(fmm.solve(rho, 3, 2)[1], ref_g)
    monkeypatch.setattr(fmm, "l2l", lambda F, p, c: F @ fmm.m2m_matrix(p, c).T)
    bad = _rel(fmm.solve(rho, 3, 2)[1], ref_g)
    assert bad > 3 * good


def test_planted_sign_mistake_in_m2l_is_caught(monkeypatch):
    n = 8
    rho = inputs.plummer(n, n_clumps=2, seed=4, a_min=0.5, a_max=1.0)
    orig = fmm.m2l_kernel
    monkeypatch.setattr(fmm, "m2l_kernel", lambda lev, p, off: orig(lev, p, tuple(-o for o in off)))
    phi, g = fmm.solve(rho, 2, 2)
    p_ref, g_ref = pm.direct(pm.masses(rho), green.g_s1, green.grad_g_s1, green.self_term(n))
    assert _rel(g, g_ref) > 1e-3


def test_solve_at_cells_matches_full_solve():
    # the cell-sampled evaluation returns the full solve's values at those cells
    N, L, p = 16, 2, 3
    rho = inputs.lognormal(N, sigma=0.5, seed=31)
    phi, g = fmm.solve(rho, L, p)
    leaves = np.array([[0, 3, 1], [3, 3, 3]])
    cells = np.array([1, 9, 40, 63])
    S = N >> L
    full = np.concatenate([phi[None], g])
    want = np.stack([full[:, a * S:(a + 1) * S, b * S:(b + 1) * S, c * S:(c + 1) * S].reshape(4, -1)
                     for a, b, c in leaves])[:, :, cells]
    got = fmm.solve_at(rho, L, p, leaves, cells=cells)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
