"""Non-periodic references and the Green's-function error of eq. gerr, FP64
(test infrastructure: the reference side of the paper's accuracy experiment,
Sec. 3; no GPU counterpart yet).

The experiment of Sec. 3 separates the two errors of a periodic FMM solution
against a PM solution: the error of the multipole expansion, measured on the
same problem without periodic boundaries, and the error of the Green's
function, what is left (eq. gerr):

    Delta g = | g_FMM^P - g_PM^P - (g_FMM^NP - g_PM^NP) |,

with absolute norms L_MAX (maximum over cells) and L2 (root mean square over
cells) for a unit mass in a unit box (Sec. 3: the characteristic acceleration
is 1, so the absolute error is a relative one).

Readings (the paper is brief here):
  * the periodic PM of eq. gerr uses the same Green's function as the FMM,
    G_S1 sampled at the mesh offsets (Sec. 3 defines G_* as the function with
    which PM and FMM agree; the figures compare the two with one G);
  * the non-periodic problem has the isolated Green's function G_0 =
    -1/(4 pi r) everywhere, no mean removal (masses m = rho / N^3), and the
    same cell self term G(0) as the periodic solver;
  * the non-periodic PM is the zero-padded (Hockney) FFT convolution;
  * the non-periodic FMM keeps the tree, gridlets and operators of the
    periodic one and drops the wrap: a node's near zone is its in-box
    neighbours, its interaction zone the children of its parent's in-box
    neighbours that are not its neighbours (Sec. 2, Fig. fmm without the
    periodic translation), with G_0 in M2L and P2P;
  * accelerations: this FMM evaluates -grad G exactly at the cell offsets in
    its near zone and carries -grad G through its expansions, so the PM
    accelerations it is measured against are the convolutions with -grad G
    (`pm.pm` and `pm_isolated_accel`).  Sec. 3 takes the PM accelerations
    from the potential by a 4th-order difference, which matches an FMM whose
    near zone is a PM-like sub-grid solve; against this FMM the difference
    leaves an O(1) error at the source and, for a corner source, at its
    periodic images, which eq. gerr cannot subtract (the non-periodic problem
    has no images).  The difference is kept (`fd4*`) for that comparison.
"""
from functools import lru_cache

import numpy as np

from . import green
from . import pm as ppm
from .fmm import (FIELDS, all_nodes, gridlet_offsets, l2l, l2p_matrix, leaves_of, mesh_of, tensor_points,
                  upward)

FOUR_PI = 4.0 * np.pi


def masses_isolated(rho):
    """Mesh masses of an isolated distribution, m = rho / N^3 (no mean removal)."""
    rho = np.asarray(rho, dtype=np.float64)
    return rho / float(rho.shape[0]) ** 3


def g0_at(d, self_value):
    """G_0 at displacements d (box units, (..., 3)); `self_value` where d = 0."""
    r = np.sqrt(np.sum(np.asarray(d, dtype=np.float64) ** 2, axis=-1))
    zero = r == 0.0
    out = -1.0 / (FOUR_PI * np.where(zero, 1.0, r))
    return np.where(zero, self_value, out)


def grad_g0(d):
    """grad G_0 = x / (4 pi r^3); 0 at d = 0 (the cell self force vanishes)."""
    d = np.asarray(d, dtype=np.float64)
    r2 = np.sum(d * d, axis=-1)
    zero = r2 == 0.0
    r3 = np.where(zero, 1.0, r2 * np.sqrt(r2))
    out = d / (FOUR_PI * r3[..., None])
    out[zero] = 0.0
    return out


def direct_isolated(m, self_value):
    """Brute-force isolated sum over every pair of cells: (phi, g), g = -grad Phi.
    O(N^6): meant for N <= 16."""
    m = np.asarray(m, dtype=np.float64)
    n = m.shape[0]
    pos = ppm.offsets_grid(n).reshape(-1, 3)
    d = (pos[:, None, :] - pos[None, :, :]) / n
    mf = m.reshape(-1)
    phi = g0_at(d, self_value) @ mf
    g = -np.einsum("ijc,j->ic", grad_g0(d), mf)
    return phi.reshape(n, n, n), np.moveaxis(g, -1, 0).reshape(3, n, n, n)


def pm_isolated(m, self_value):
    """Zero-padded FFT convolution of the masses with G_0 sampled at the mesh
    offsets d/N (the Hockney method).  The padded mesh has 2N + 4 cells per
    side, so the convolution is also exact two cells beyond every box face
    (targets t in [-2, N + 1], offsets t - j within the kernel's
    [-(N + 2), N + 1]), where the 4th-order difference reads it.  Returns
    (phi on the box, phi on the padded mesh [z][y][x], box at [0, N)^3,
    t = -1, -2 at the last two indices)."""
    m = np.asarray(m, dtype=np.float64)
    n = m.shape[0]
    n2 = 2 * n + 4
    k = np.arange(n2)
    k = np.where(k < n2 // 2, k, k - n2).astype(np.float64)       # signed offsets in FFT order
    dz, dy, dx = np.meshgrid(k, k, k, indexing="ij")
    kern = g0_at(np.stack([dx, dy, dz], axis=-1) / n, self_value)
    mp = np.zeros((n2, n2, n2))
    mp[:n, :n, :n] = m
    phi_pad = np.fft.irfftn(np.fft.rfftn(mp) * np.fft.rfftn(kern), s=(n2, n2, n2), axes=(0, 1, 2))
    return phi_pad[:n, :n, :n], phi_pad


def pm_isolated_accel(m):
    """Accelerations g = -grad Phi of the isolated problem: zero-padded FFT
    convolution of the masses with -grad G_0 sampled at the mesh offsets
    (padded to 2N, offsets in [-(N - 1), N - 1]; zero at d = 0).  Returns
    (3, N, N, N), components (x, y, z)."""
    m = np.asarray(m, dtype=np.float64)
    n = m.shape[0]
    n2 = 2 * n
    k = np.arange(n2)
    k = np.where(k < n, k, k - n2).astype(np.float64)
    dz, dy, dx = np.meshgrid(k, k, k, indexing="ij")
    kern = -grad_g0(np.stack([dx, dy, dz], axis=-1) / n)
    mp = np.zeros((n2, n2, n2))
    mp[:n, :n, :n] = m
    fm = np.fft.rfftn(mp)
    g = [np.fft.irfftn(fm * np.fft.rfftn(kern[..., c]), s=(n2, n2, n2), axes=(0, 1, 2))[:n, :n, :n]
         for c in range(3)]
    return np.stack(g)


def fd4(phi, h, axis):
    """Central 4th-order difference d phi / dx along `axis` (periodic roll):
    [8 (f(+1) - f(-1)) - (f(+2) - f(-2))] / (12 h) (Sec. 3)."""
    p1, m1 = np.roll(phi, -1, axis), np.roll(phi, 1, axis)
    p2, m2 = np.roll(phi, -2, axis), np.roll(phi, 2, axis)
    return (8.0 * (p1 - m1) - (p2 - m2)) / (12.0 * h)


def fd4_accel_periodic(phi):
    """g = -grad Phi on a periodic N^3 mesh (box units), components (x, y, z)."""
    n = phi.shape[0]
    h = 1.0 / n
    return -np.stack([fd4(phi, h, 2), fd4(phi, h, 1), fd4(phi, h, 0)])


def fd4_accel_isolated(phi_pad, n):
    """g = -grad Phi on the box from `pm_isolated`'s padded potential: the
    stencil reaches two cells outside the box, where the padded convolution
    holds the potential of the same masses."""
    h = 1.0 / n
    g = -np.stack([fd4(phi_pad, h, 2), fd4(phi_pad, h, 1), fd4(phi_pad, h, 0)])
    return g[:, :n, :n, :n]


# --------------------------------------------------------- isolated FMM
def neighbours_np(level, node):
    """The node and its in-box neighbours (no wrap)."""
    n = 2 ** level
    out = set()
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            for c in (-1, 0, 1):
                q = (node[0] + a, node[1] + b, node[2] + c)
                if all(0 <= v < n for v in q):
                    out.add(q)
    return out


def interaction_list_np(level, node):
    """Children of the parent's in-box neighbours that are not neighbours of
    the node (Sec. 2, Fig. fmm, without the periodic wrap)."""
    parent = tuple(i // 2 for i in node)
    kids = set()
    for q in neighbours_np(level - 1, parent):
        for a in range(2):
            for b in range(2):
                for c in range(2):
                    kids.add((2 * q[0] + a, 2 * q[1] + b, 2 * q[2] + c))
    return kids - neighbours_np(level, node)


@lru_cache(maxsize=None)
def _m2l_kernel_g0(level, p, off_zyx):
    """(4, p^3, p^3) matrices of eq. fmm2 with G_0 for a node offset T - S."""
    H = 2.0 ** (-level)
    pts = tensor_points(gridlet_offsets(p))
    d = (np.array(off_zyx[::-1], dtype=np.float64)[None, None, :] + pts[:, None, :] - pts[None, :, :]) * H
    G = g0_at(d, 0.0)
    dG = grad_g0(d)
    return np.concatenate([G[None], -np.moveaxis(dG, -1, 0)], axis=0)


def _p2p_kernel_g0(N, S, off_zyx, targets=None):
    """Near-zone matrices (4, S^3, S^3) with G_0 between a target leaf and the
    source leaf at offset T - S; the coincident cell uses the self term.
    ``targets`` (flat cell indices in the leaf) keeps only those rows."""
    cells = tensor_points(np.arange(S, dtype=np.float64))
    tcells = cells if targets is None else cells[np.asarray(targets)]
    d = (np.array(off_zyx[::-1], dtype=np.float64)[None, None, :] * S + tcells[:, None, :] - cells[None, :, :]) / N
    G = g0_at(d, green.self_term(N))
    dG = grad_g0(d)
    return np.concatenate([G[None], -np.moveaxis(dG, -1, 0)], axis=0)


def solve_isolated(rho, L, p):
    """The FMM of `fmm.solve` without periodic boundaries (see the module
    readings).  Returns (phi (N,N,N), g (3,N,N,N))."""
    rho = np.asarray(rho, dtype=np.float64)
    N = rho.shape[0]
    n = 2 ** L
    S = N // n
    if N % n or L < 2 or S < 1:
        raise ValueError("need N divisible by 2^L and L >= 2")
    m = masses_isolated(rho)
    M = upward(m, L, p)
    P3 = p ** 3
    loc = None
    for lev in range(2, L + 1):
        nl = 2 ** lev
        F = np.zeros((nl, nl, nl, FIELDS, P3))
        for T in map(tuple, all_nodes(lev)):
            for src in interaction_list_np(lev, T):
                off = tuple(int(a - b) for a, b in zip(T, src))
                K = _m2l_kernel_g0(lev, p, off).reshape(FIELDS * P3, P3)
                F[T] += (K @ M[lev][src]).reshape(FIELDS, P3)
        if loc is not None:
            for cz in range(2):
                for cy in range(2):
                    for cx in range(2):
                        F[cz::2, cy::2, cx::2] += l2l(loc, p, (cx, cy, cz))
        loc = F
    far = loc @ l2p_matrix(S, p).T                                 # (n,n,n,4,S^3)
    near = _near_isolated(m, L, all_nodes(L)).reshape(n, n, n, FIELDS, S ** 3)
    mesh = mesh_of(np.moveaxis(far + near, 3, 0), S)
    return mesh[0], mesh[1:]


def _near_isolated(m, L, leaves, cells=None):
    """Near zone of the isolated problem for the given leaves ((k, 3),
    (z, y, x)): direct sums with G_0 over the in-box neighbour leaves, one
    offset at a time.  Returns (k, 4, S^3) or (k, 4, len(cells))."""
    N = m.shape[0]
    n = 2 ** L
    S = N // n
    ml = leaves_of(m, L)
    leaves = np.asarray(leaves, dtype=np.int64).reshape(-1, 3)
    nt = S ** 3 if cells is None else len(cells)
    out = np.zeros((leaves.shape[0], FIELDS, nt))
    for off in [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]:
        src = leaves - np.array(off)
        ok = np.all((src >= 0) & (src < n), axis=1)
        if not ok.any():
            continue
        K = _p2p_kernel_g0(N, S, off, cells).reshape(FIELDS * nt, S ** 3)
        s = src[ok]
        out[ok] += (ml[s[:, 0], s[:, 1], s[:, 2]] @ K.T).reshape(-1, FIELDS, nt)
    return out


def solve_isolated_at(rho, L, p, leaves, cells=None):
    """``solve_isolated`` evaluated only in the given leaves ((k, 3), (z, y,
    x)) and, if given, only at the flat cell indices ``cells`` of each:
    the whole upward pass, the local fields along each leaf's chain of
    ancestors (isolated interaction lists), L2P and the isolated near zone."""
    rho = np.asarray(rho, dtype=np.float64)
    N = rho.shape[0]
    S = N // 2 ** L
    m = masses_isolated(rho)
    M = upward(m, L, p)
    P3 = p ** 3
    leaves = np.asarray(leaves, dtype=np.int64).reshape(-1, 3)
    loc = None
    for lev in range(2, L + 1):
        anc = leaves >> (L - lev)
        F = np.zeros((len(leaves), FIELDS, P3))
        for i, T in enumerate(map(tuple, anc)):
            for src in interaction_list_np(lev, T):
                off = tuple(int(a - b) for a, b in zip(T, src))
                K = _m2l_kernel_g0(lev, p, off).reshape(FIELDS * P3, P3)
                F[i] += (K @ M[lev][src]).reshape(FIELDS, P3)
        if loc is not None:
            c = anc % 2
            for i in range(len(leaves)):
                F[i] += l2l(loc[i], p, (int(c[i, 2]), int(c[i, 1]), int(c[i, 0])))
        loc = F
    l2p = l2p_matrix(S, p)
    if cells is not None:
        l2p = l2p[np.asarray(cells)]
    return loc @ l2p.T + _near_isolated(m, L, leaves, cells)


# --------------------------------------------------------------- eq. gerr
def gf_error(g_fmm_p, g_pm_p, g_fmm_np, g_pm_np):
    """Eq. gerr: the per-cell magnitude of g_FMM^P - g_PM^P - (g_FMM^NP -
    g_PM^NP) (arrays (3, N, N, N)); returns (L_MAX, L2 = root mean square)."""
    d = (np.asarray(g_fmm_p) - np.asarray(g_pm_p)) - (np.asarray(g_fmm_np) - np.asarray(g_pm_np))
    mag = np.sqrt(np.sum(d * d, axis=0))
    return float(mag.max()), float(np.sqrt(np.mean(mag * mag)))


def me_error(g_fmm_np, g_pm_np):
    """The multipole-expansion error of the isolated problem (L_MAX, L2)."""
    d = np.asarray(g_fmm_np) - np.asarray(g_pm_np)
    mag = np.sqrt(np.sum(d * d, axis=0))
    return float(mag.max()), float(np.sqrt(np.mean(mag * mag)))

