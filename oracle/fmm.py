"""The natively periodic FMM-HPM solve, step by step in FP64 (test infrastructure).

Geometry (Sec. 2).  The unit box is covered by an N^3 mesh, cells at
(j + 1/2)/N.  Oct-tree level l has 2^l nodes per dimension of size H_l = 2^-l;
level L is the leaf level, each leaf covering S^3 cells, S = N / 2^L.  Node
arrays are indexed [iz][iy][ix]; flattened per-node vectors use x fastest.

Each node carries a "gridlet" of p^3 effective masses (p = N_g of the paper)
on a uniform mini-mesh covering the node (Sec. 2).  Reading: the mini-mesh is
cell-centred, points at node_lo + (s + 1/2) H_l / p, so that a gridlet with
p = S coincides with the leaf's cells (the special case of Sec. 3).

Steps, in the paper's order:
  a0  masses m = (rho - mean rho) / N^3                       (Sec. 1, eq. gfk: k=0 mode is 0)
  a3  P2M:  leaf gridlet masses whose Cartesian multipoles Q_n, n_i < p,
            equal those of the leaf's cell masses (Sec. 2, Vandermonde system)
  a4  M2M:  parent gridlet masses matching the children's multipoles,
            M_parent = sum_children T^C M_child (Sec. 3 eq. fmm1; T is the
            same Vandermonde construction applied to the child gridlet)
  a5/a6 M2L: Phi_T[r] = sum_{S in IL(T)} sum_s G(X^T_r - X^S_s) M_S[s]
            (Sec. 3 eq. fmm2) and g_T[r] = -sum grad G(...) M_S[s]; the
            interaction zone IL(T) is the children of the parent's neighbours
            that are not neighbours of T, with periodic wrap (Sec. 2, Fig. fmm)
  a7  L2L:  child local field = sum_r T^C_{r p} parent local field (Sec. 3
            eq. fmm3: the transpose of the M2M matrix)
  a8  L2P:  cell values from the leaf local field by the transpose of the P2M
            matrix (eq. fmm3 applied at the leaves)
  a9  P2P:  near zone (the 27 immediate neighbours of each leaf, periodic wrap)
            by direct summation with the same G (Sec. 2; Sec. 3: the near zone
            must use the same G as the PM solution)

G is G_S1 of eq. gfs1 everywhere (M2L at every level and P2P), with the cell
self term of ``green.self_term``.  Accelerations are carried as three extra
local fields built from grad G (Sec. 3: FMM accelerations come from the
multipole expansion).

Pins (tests/test_oracle_fmm.py):
  * special case L = 2, p = S: every operator is exact and the FMM equals the
    brute-force periodic sum (Sec. 3, two-level tree identical to PM);
  * P2M reproduces cell masses exactly when p = S; p = 1 gives the node mass;
  * M2M after P2M equals P2M straight to the parent (Lagrange identity);
  * the interaction lists have 37 / 189 members and, united over all levels
    with the leaf neighbours, cover every cell exactly once;
  * the FMM error against PM(G_S1) falls as p rises;
  * zero net force sum_i m_i g_i = 0 (antisymmetric operator).
"""
from math import factorial

import numpy as np

from . import green
from .pm import masses

FIELDS = 4          # Phi, g_x, g_y, g_z


# ---------------------------------------------------------------- geometry
def gridlet_offsets(p):
    """Gridlet point coordinates in one dimension, relative to the node centre,
    in units of the node size: (s + 1/2)/p - 1/2."""
    return (np.arange(p) + 0.5) / p - 0.5


def tensor_points(c1):
    """3-D tensor grid of 1-D coordinates c1 -> (k^3, 3) array of (x, y, z),
    flat index (iz * k + iy) * k + ix."""
    z, y, x = np.meshgrid(c1, c1, c1, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=-1)


def multi_indices(p):
    """Multi-indices n = (n_x, n_y, n_z) with n_i < p (Sec. 2 notation)."""
    return tensor_points(np.arange(p, dtype=np.float64)).astype(np.int64)


def moment_matrix(points, p):
    """W[n, j] = r_j^n / n!  (Sec. 2 multi-index notation), so that the
    Cartesian multipoles of masses w_j at points r_j are Q = W @ w."""
    nidx = multi_indices(p)
    fac = np.array([factorial(a) * factorial(b) * factorial(c) for a, b, c in nidx], dtype=np.float64)
    pw = np.prod(points[None, :, :] ** nidx[:, None, :], axis=-1)
    return pw / fac[:, None]


def vandermonde(p):
    """Vandermonde matrix of the gridlet points, V[n, q] = r_q^n / n!
    (Sec. 2); coordinates relative to the node centre in node-size units."""
    return moment_matrix(tensor_points(gridlet_offsets(p)), p)


# ------------------------------------------------------------- projections
def vandermonde_1d(points, p):
    """One axis of the moment matrix: V1[n, j] = r_j^n / n!, n < p."""
    n = np.arange(p)
    fac = np.array([factorial(k) for k in range(p)], dtype=np.float64)
    return np.asarray(points, dtype=np.float64)[None, :] ** n[:, None] / fac[:, None]


def solve_1d(points, p):
    """Per-axis solution of the Vandermonde system of Sec. 2: the (p, k) matrix
    T1 = V1(gridlet)^-1 V1(points) whose column j holds the gridlet masses
    that reproduce the 1-D moments n < p of a unit mass at points[j]."""
    return np.linalg.solve(vandermonde_1d(gridlet_offsets(p), p), vandermonde_1d(points, p))


def kron3(tz, ty, tx):
    """Tensor product for flat indices (iz * k + iy) * k + ix (x fastest)."""
    return np.kron(tz, np.kron(ty, tx))


def p2m_matrix(S, p):
    """Gridlet masses from leaf cell masses: solve V M = Q with Q the cell
    multipoles (Sec. 2).  Returned as the (p^3, S^3) matrix V^-1 W_cells.

    The multi-indices n_i < p make V and W tensor products of one 1-D
    moment matrix per axis (r^n / n! = prod_i r_i^{n_i} / n_i!), so
    V^-1 W = T1 (x) T1 (x) T1 with T1 the 1-D solution.  Solving per axis
    is the same system; the 3-D matrix itself has condition numbers of
    1e16 at p = 6 and 4e25 at p = 8, beyond FP64 (the 1-D one: 3.5e8 at
    p = 8, solved to 1e-12)."""
    cells = (np.arange(S) + 0.5) / S - 0.5
    T1 = solve_1d(cells, p)
    return kron3(T1, T1, T1)


def m2m_matrix(p, child):
    """T^C of eq. fmm1 for child C = (cx, cy, cz) in {0,1}^3: parent gridlet
    masses matching the multipoles of the child gridlet, V_parent^-1 W_child,
    solved per axis as in ``p2m_matrix``.  Child points in parent-size units
    relative to the parent centre are (c - 1/2)/2 + offset/2."""
    cx, cy, cz = child
    g = gridlet_offsets(p) / 2.0
    t = [solve_1d(g + (c - 0.5) / 2.0, p) for c in (cx, cy, cz)]
    return kron3(t[2], t[1], t[0])


def leaves_of(m, L):
    """Mesh (N,N,N) -> (n,n,n,S^3) cell values grouped by leaf, n = 2^L."""
    N = m.shape[0]
    n = 2 ** L
    S = N // n
    a = m.reshape(n, S, n, S, n, S).transpose(0, 2, 4, 1, 3, 5)
    return a.reshape(n, n, n, S ** 3)


def mesh_of(leafvals, S):
    """Inverse of ``leaves_of`` for arrays (..., n, n, n, S^3)."""
    lead = leafvals.shape[:-4]
    n = leafvals.shape[-4]
    a = leafvals.reshape(lead + (n, n, n, S, S, S))
    k = len(lead)
    a = np.moveaxis(a, [k + 3, k + 4, k + 5], [k + 1, k + 3, k + 5])
    return a.reshape(lead + (n * S,) * 3)


def p2m(m, L, p):
    """a3: leaf gridlet masses (Sec. 2).  Returns (n, n, n, p^3)."""
    N = m.shape[0]
    S = N // 2 ** L
    return leaves_of(m, L) @ p2m_matrix(S, p).T


def m2m(Mchild, p):
    """a4: eq. fmm1, M^{l-1} = sum over the 8 children of T^C M^l_C."""
    n = Mchild.shape[0] // 2
    out = np.zeros((n, n, n, p ** 3))
    for cz in range(2):
        for cy in range(2):
            for cx in range(2):
                T = m2m_matrix(p, (cx, cy, cz))
                out += Mchild[cz::2, cy::2, cx::2] @ T.T
    return out


def upward(m, L, p):
    """P2M at level L then M2M up to level 2.  Returns {level: (n,n,n,p^3)}."""
    M = {L: p2m(m, L, p)}
    for lev in range(L - 1, 1, -1):
        M[lev] = m2m(M[lev + 1], p)
    return M


# ------------------------------------------------------ interaction zones
def neighbours(level, node):
    """The node and its 26 immediate neighbours with periodic wrap, as a set of
    (iz, iy, ix) tuples (Sec. 2, Fig. fmm: no special cases under periodic
    boundary conditions)."""
    n = 2 ** level
    iz, iy, ix = node
    return {((iz + a) % n, (iy + b) % n, (ix + c) % n)
            for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)}


def interaction_list(level, node):
    """Children of the parent's neighbours that are not neighbours of the node
    (Sec. 2, Fig. fmm).  Level >= 2."""
    parent = tuple(i // 2 for i in node)
    kids = set()
    for q in neighbours(level - 1, parent):
        for a in range(2):
            for b in range(2):
                for c in range(2):
                    kids.add((2 * q[0] + a, 2 * q[1] + b, 2 * q[2] + c))
    return kids - neighbours(level, node)


def min_image(d, n):
    """Node-index difference wrapped to its nearest periodic image."""
    d = np.asarray(d)
    return d - n * np.rint(d / n).astype(d.dtype)


def interaction_offsets(level, child):
    """Offsets T - S (node units, (z, y, x), nearest image) of the interaction
    list of a node whose position in its parent is ``child`` = (cz, cy, cx).
    Under periodic wrap the list of any node is a translate of the list of the
    node with the same position in its parent (Fig. fmm caption)."""
    n = 2 ** level
    node = tuple(child)
    return sorted(tuple(int(v) for v in min_image(np.subtract(node, s), n))
                  for s in interaction_list(level, node))


# --------------------------------------------------------------- kernels
def m2l_kernel(level, p, off_zyx):
    """The (4, p^3, p^3) matrices of eq. fmm2 for a node offset T - S:
    entry [f, r, s] evaluates f = 0: G_S1, f = 1..3: -dG_S1/dx_i at
    X^T_r - X^S_s = ((T - S) + (o_r - o_s)) H_l."""
    H = 2.0 ** (-level)
    pts = tensor_points(gridlet_offsets(p))
    d = (np.array(off_zyx[::-1], dtype=np.float64)[None, None, :]
         + pts[:, None, :] - pts[None, :, :]) * H
    G = green.g_s1(d)
    dG = green.grad_g_s1(d)
    return np.concatenate([G[None], -np.moveaxis(dG, -1, 0)], axis=0)


def p2p_kernel(N, S, off_zyx, targets=None):
    """Near-zone matrices (4, S^3, S^3) between a target leaf and the source
    leaf at node offset T - S, cells at spacing 1/N; the coincident cell uses
    the self term.  ``targets`` (flat cell indices in the leaf) keeps only
    those rows."""
    cells = tensor_points(np.arange(S, dtype=np.float64))
    tcells = cells if targets is None else cells[np.asarray(targets)]
    d = (np.array(off_zyx[::-1], dtype=np.float64)[None, None, :] * S
         + tcells[:, None, :] - cells[None, :, :]) / N
    G = green.g_s1(d, self_value=green.self_term(N))
    dG = green.grad_g_s1(d)
    return np.concatenate([G[None], -np.moveaxis(dG, -1, 0)], axis=0)


# ------------------------------------------------------------- far field
def m2l(level, p, M, targets, correction=None):
    """a5/a6: eq. fmm2 for the given target nodes ((k,3) int array, (z,y,x)).
    Returns (k, 4, p^3): Phi and g = -grad Phi at the target gridlet points
    from the multipoles of the target's interaction zone.  ``correction``,
    if given, is a function (level, p, offset) -> (4, p^3, p^3) added to the
    translation matrices (the learned table correction)."""
    n = 2 ** level
    targets = np.asarray(targets, dtype=np.int64).reshape(-1, 3)
    out = np.zeros((targets.shape[0], FIELDS, p ** 3))
    ctype = targets % 2
    for cz in range(2):
        for cy in range(2):
            for cx in range(2):
                sel = np.nonzero((ctype[:, 0] == cz) & (ctype[:, 1] == cy) & (ctype[:, 2] == cx))[0]
                if sel.size == 0:
                    continue
                T = targets[sel]
                for off in interaction_offsets(level, (cz, cy, cx)):
                    K = m2l_kernel(level, p, off)
                    if correction is not None:
                        K = K + correction(level, p, off)
                    src = (T - np.array(off)) % n
                    Ms = M[src[:, 0], src[:, 1], src[:, 2]]
                    out[sel] += (Ms @ K.reshape(FIELDS * p ** 3, p ** 3).T).reshape(-1, FIELDS, p ** 3)
    return out


def l2l(Fparent, p, child):
    """a7: eq. fmm3, child local field = (T^C)^T parent local field (per field)."""
    T = m2m_matrix(p, child)
    return Fparent @ T


def all_nodes(level):
    n = 2 ** level
    g = np.indices((n, n, n)).reshape(3, -1).T
    return g


def downward(M, L, p, correction=None):
    """Local fields for every node: M2L at each level plus L2L from the parent.
    Returns {level: (n,n,n,4,p^3)}."""
    F = {}
    for lev in range(2, L + 1):
        n = 2 ** lev
        loc = m2l(lev, p, M[lev], all_nodes(lev), correction).reshape(n, n, n, FIELDS, p ** 3)
        if lev > 2:
            for cz in range(2):
                for cy in range(2):
                    for cx in range(2):
                        loc[cz::2, cy::2, cx::2] += l2l(F[lev - 1], p, (cx, cy, cz))
        F[lev] = loc
    return F


# ------------------------------------------------------------ near field
def p2p(m, L, leaves, cells=None):
    """a9: near zone by direct summation over the 27 neighbour leaves of each
    target leaf ((k,3) array) with periodic wrap.  Returns (k, 4, S^3), or
    (k, 4, len(cells)) for the given flat cell indices of each leaf."""
    N = m.shape[0]
    n = 2 ** L
    S = N // n
    ml = leaves_of(m, L)
    leaves = np.asarray(leaves, dtype=np.int64).reshape(-1, 3)
    nt = S ** 3 if cells is None else len(cells)
    out = np.zeros((leaves.shape[0], FIELDS, nt))
    offs = sorted({tuple(int(v) for v in min_image(np.subtract((0, 0, 0), s), n))
                   for s in neighbours(L, (0, 0, 0))})
    for off in offs:
        K = p2p_kernel(N, S, off, cells)
        src = (leaves - np.array(off)) % n
        ms = ml[src[:, 0], src[:, 1], src[:, 2]]
        out += (ms @ K.reshape(FIELDS * nt, S ** 3).T).reshape(-1, FIELDS, nt)
    return out


def l2p_matrix(S, p):
    """a8: the transpose of the P2M matrix, (S^3, p^3)."""
    return p2m_matrix(S, p).T


# ---------------------------------------------------------------- solve
def solve(rho, L, p, correction=None):
    """Full FMM solve.  Returns (phi (N,N,N), g (3,N,N,N)).  ``correction`` as
    in ``m2l``."""
    rho = np.asarray(rho, dtype=np.float64)
    N = rho.shape[0]
    n = 2 ** L
    S = N // n
    if N % n or L < 2 or S < 1:
        raise ValueError("need N divisible by 2^L and L >= 2")
    m = masses(rho)
    M = upward(m, L, p)
    F = downward(M, L, p, correction)
    far = F[L] @ l2p_matrix(S, p).T                            # (n,n,n,4,S^3)
    near = p2p(m, L, all_nodes(L)).reshape(n, n, n, FIELDS, S ** 3)
    tot = np.moveaxis(far + near, 3, 0)                         # (4,n,n,n,S^3)
    mesh = mesh_of(tot, S)
    return mesh[0], mesh[1:]


def solve_at(rho, L, p, leaves, correction=None, cells=None):
    """The same solve evaluated only in the given leaves ((k,3), (z,y,x)):
    the whole upward pass, then the local fields along each leaf's chain of
    ancestors, L2P and P2P in those leaves.  Returns (k, 4, S^3) with cells
    flattened x fastest within the leaf, or (k, 4, len(cells)) for the given
    flat cell indices.  ``correction`` as in ``m2l``."""
    rho = np.asarray(rho, dtype=np.float64)
    N = rho.shape[0]
    S = N // 2 ** L
    m = masses(rho)
    M = upward(m, L, p)
    leaves = np.asarray(leaves, dtype=np.int64).reshape(-1, 3)
    loc = None
    for lev in range(2, L + 1):
        anc = leaves >> (L - lev)
        F = m2l(lev, p, M[lev], anc, correction)
        if loc is not None:
            c = anc % 2
            for i in range(anc.shape[0]):
                F[i] += l2l(loc[i], p, (int(c[i, 2]), int(c[i, 1]), int(c[i, 0])))
        loc = F
    l2p = l2p_matrix(S, p)
    if cells is not None:
        l2p = l2p[np.asarray(cells)]
    far = loc @ l2p.T
    return far + p2p(m, L, leaves, cells)
