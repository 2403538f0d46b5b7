"""FP64 reference of the learned M2L table correction (test infrastructure).

The correction is a function of a table entry of eq. fmm2: offset n (integer
vector in gridlet units of level l, components x, y, z), field f
(0: G, 1..3: -dG/dx_i), level l, order p.  Following Sec. 4's proposal to
parameterise G_* beyond the analytic G_S1, a small network adds

    delta = scale(l, f) * sign * MLP(features)

to the G_S1 table value, where (keeping the symmetries of G_S1)
  f = 0:  features use the three |n_i| in ascending order, class 0, sign +1;
  f = i:  features use |n_i| then the other two |n_j| ascending, class 1,
          sign = sign(n_i) (0 when n_i = 0);
  features = (a, b, c) / (4 p), l / 8, class;
  scale = kappa (2^l p) / (4 pi) for f = 0 and kappa (2^l p)^2 / (4 pi) for
          f >= 1, kappa = 1e-3 (the expected size of G_* - G_S1 relative to G,
          from the spread of the fitted a_1 in Table 1).
MLP: 5 -> 64 -> 64 -> 64 -> 1, GELU(z) = z Phi(z) (erf form) on the hidden
layers, parameters flat in the order W1[64][5] b1 W2[64][64] b2 W3[64][64]
b3 W4[64] b4.

Pins (tests/test_oracle_learn.py): GELU against its closed form at chosen
points; the network with hand-set weights against a hand-computed value; the
corrected table keeps the parity of each field and is periodic; the loss
gradient of ``loss`` against central finite differences is what the GPU
gradient is checked against.
"""
from math import sqrt

import numpy as np
from scipy.special import erf as _erf

from . import fmm, green, pm

H = 64
N_IN = 5
N_PARAMS = H * N_IN + H + H * H + H + H * H + H + H + 1
KAPPA = 1e-3


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    assert w.size == N_PARAMS
    o = 0
    out = []
    for shape in [(H, N_IN), (H,), (H, H), (H,), (H, H), (H,), (H,), (1,)]:
        k = int(np.prod(shape))
        out.append(w[o:o + k].reshape(shape))
        o += k
    return out


def gelu(z):
    """z * Phi(z), Phi the standard normal CDF (erf form; the library erf
    evaluated element-wise)."""
    return 0.5 * z * (1.0 + _erf(np.asarray(z, dtype=np.float64) / sqrt(2.0)))


def mlp(w, x):
    """Forward pass; x (k, 5) -> (k,)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(w)
    h = gelu(x @ W1.T + b1)
    h = gelu(h @ W2.T + b2)
    h = gelu(h @ W3.T + b3)
    return h @ W4 + b4[0]


def features(n, f, level, p):
    """n: (k, 3) integer offsets (x, y, z).  Returns (x (k,5), sign (k,), scale).

    The offset is first taken to its nearest periodic image (the box spans
    2^l p gridlet spacings), so the correction is periodic like G_S1."""
    n = np.asarray(n, dtype=np.int64)
    period = 2 ** level * p
    n = np.mod(n, period)
    n = np.where(2 * n > period, n - period, n)     # to (-period/2, period/2]
    a = np.abs(n)
    if f == 0:
        srt = np.sort(a, axis=1)
        sign = np.ones(len(n))
        cls = 0.0
    else:
        i = f - 1
        others = np.sort(np.delete(a, i, axis=1), axis=1)
        srt = np.concatenate([a[:, i:i + 1], others], axis=1)
        sign = np.sign(n[:, i]).astype(np.float64)
        sign[2 * a[:, i] == period] = 0.0      # odd and periodic: zero at half the box
        cls = 1.0
    x = np.empty((len(n), N_IN))
    x[:, :3] = srt / (4.0 * p)
    x[:, 3] = level / 8.0
    x[:, 4] = cls
    base = float(2 ** level * p)
    scale = KAPPA * (base if f == 0 else base * base) / (4.0 * np.pi)
    return x, sign, scale


def table_correction(w, level, p, n):
    """(k, 4) corrections of the table entries with offsets n (k, 3)."""
    out = np.zeros((len(n), 4))
    for f in range(4):
        x, sign, scale = features(n, f, level, p)
        out[:, f] = scale * sign * mlp(w, x)
    out[np.all(np.asarray(n) == 0, axis=1)] = 0.0
    return out


def correction_fn(w):
    """The per-offset (4, p^3, p^3) correction of eq. fmm2's translation
    matrices for ``fmm.solve(..., correction=...)``: entry [f, r, s] is the
    table correction at n = o p + r - s (x, y, z components).  Every offset
    of the interaction zones has |o_i| <= 3, so every such n lies in the cube
    |n_i| <= 4p - 1: the correction is evaluated once per (level, p) on that
    cube and looked up."""
    return _matrices_from(lambda level, p, n: table_correction(w, level, p, n))


def _matrices_from(entry_fn):
    """(level, p, offset) -> (4, p^3, p^3) matrices of a per-entry table
    correction entry_fn(level, p, n (k, 3)) -> (k, 4)."""
    tables = {}

    def corr(level, p, off_zyx):
        h = 4 * p - 1
        if (level, p) not in tables:
            g = np.arange(-h, h + 1)
            nz, ny, nx = np.meshgrid(g, g, g, indexing="ij")
            cube = np.stack([nx.ravel(), ny.ravel(), nz.ravel()], axis=-1)     # x fastest
            tables[(level, p)] = entry_fn(level, p, cube).reshape(2 * h + 1, 2 * h + 1, 2 * h + 1, 4)
        tab = tables[(level, p)]
        g = np.arange(p)
        z, y, x = np.meshgrid(g, g, g, indexing="ij")
        pts = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=-1)            # (p^3, 3) x, y, z
        o = np.array(off_zyx[::-1], dtype=np.int64) * p
        nvec = o[None, None, :] + pts[:, None, :] - pts[None, :, :]           # (r, s, 3)
        assert np.abs(nvec).max() <= h
        c = tab[nvec[..., 2] + h, nvec[..., 1] + h, nvec[..., 0] + h]           # (r, s, 4)
        return np.moveaxis(c, -1, 0)

    return corr


# ------------------------------------------------------- grid model of G_*
# Sec. 4: G_* as a grid of values, each its own parameter.  Per level
# l = 2..L, theta[l - 2] has shape (4, 4p, 4p, 4p) = [f][a_z][a_y][a_x]: the
# table entry at offset n (gridlet units) gets theta[0][a] added to G and
# sign(n_i) theta[i][a] added to -dG/dx_i, with a = |n| component-wise after
# taking n to its nearest periodic image (period 2^l p), and the gradient
# sign 0 at half the period.

def grid_size(L, p):
    return (L - 1) * 4 * (4 * p) ** 3


def grid_table_correction(theta, level, p, n):
    """(k, 4) grid corrections of the table entries with offsets n (k, 3);
    theta: the flat parameters of all levels (grid_size(L, p) values)."""
    G = 4 * p
    blk = np.asarray(theta, dtype=np.float64).reshape(-1, 4, G, G, G)[level - 2]
    n = np.asarray(n, dtype=np.int64)
    period = 2 ** level * p
    wn = np.mod(n, period)
    wn = np.where(2 * wn > period, wn - period, wn)
    a = np.abs(wn)
    sg = np.sign(wn).astype(np.float64)
    sg[2 * a == period] = 0.0
    out = np.empty((len(n), 4))
    out[:, 0] = blk[0, a[:, 2], a[:, 1], a[:, 0]]
    for f in range(1, 4):
        out[:, f] = sg[:, f - 1] * blk[f, a[:, 2], a[:, 1], a[:, 0]]
    out[np.all(n == 0, axis=1)] = 0.0
    return out


def grid_correction_fn(theta):
    """The grid model as a ``correction`` for ``fmm.solve``."""
    return _matrices_from(lambda level, p, n: grid_table_correction(theta, level, p, n))


def grid_loss(theta, rho, L, p, target_phi, target_g, w_phi, w_g):
    """J of ``loss`` for the FMM with the grid-corrected tables (FP64)."""
    phi, g = fmm.solve(rho, L, p, correction=grid_correction_fn(theta))
    return float(w_phi * np.sum((phi - target_phi) ** 2) + w_g * np.sum((g - target_g) ** 2))


def loss(w, rho, L, p, target_phi, target_g, w_phi, w_g):
    """J = w_phi |Phi - Phi*|^2 + w_g |g - g*|^2 for the FMM with the
    corrected tables (FP64)."""
    phi, g = fmm.solve(rho, L, p, correction=correction_fn(w))
    return float(w_phi * np.sum((phi - target_phi) ** 2) + w_g * np.sum((g - target_g) ** 2))


def pm_target(rho):
    """PM with the same Green's function (G_S1), Sec. 3 eq. pmconv."""
    n = rho.shape[0]
    return pm.pm(pm.masses(rho), green.g_s1, green.grad_g_s1, green.self_term(n))
