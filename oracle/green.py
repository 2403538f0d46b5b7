"""Green's functions of the periodic Poisson problem, FP64 (test infrastructure).

Units follow Sec. 1: the continuous Green's function is G_0 = -1/(4 pi r), so
the potential solves  lap(Phi) = rho  with no 4 pi G factor, and the
acceleration is g = -grad(Phi).  The box is the unit box (L = 1).

Pins (tests/test_oracle_green.py):
  * xi_s1: its Taylor series is t + O(t^5) (Sec. 3, the cancelled t^3 term),
    odd-periodic xi(t+1) = -xi(t), maximum 7/(6 pi) at t = 1/2 with zero slope.
  * grad_g_s1: central finite differences of g_s1; zero at x_i = +-1/2.
  * g_s1 -> G_0 as r -> 0.
  * self_term: closed form of the mean of 1/r over a cube, checked against
    quadrature.
  * g_k_kernel: spectral -1/k^2 of Sec. 1 eq. gfk, checked by a single Fourier
    mode whose potential is known in closed form (see oracle/pm.py).
"""
import numpy as np

FOUR_PI = 4.0 * np.pi

# Mean of 1/r over the unit cube centred on the origin, in closed form:
#   int_{[-1/2,1/2]^3} dV / r = 3 ln(2 + sqrt 3) - pi/2 = 2.380077...
# (eight corner cubes of side 1/2, each the known corner potential of a unit
# cube scaled by (1/2)^2).  The paper is silent on G(0); this reading uses the
# cell-averaged 1/r.
CUBE_MEAN_INV_R = 3.0 * np.log(2.0 + np.sqrt(3.0)) - 0.5 * np.pi


def wrap(x):
    """Periodic coordinate wrap x <> L with L = 1 (Sec. 1, after eq. gfx):
    x - nint(x).  numpy's rint rounds halves to even; halves never decide a
    result here because every G used is 1-periodic."""
    return x - np.rint(x)


def xi_s1(t):
    """xi_n(t) of the Sec. 3 ansatz with n = 1 and a_1 = -1/8 (eq. gfs1):
    xi(t) = (1 - a_1) sin(pi t)/pi + a_1 sin(3 pi t)/(3 pi)."""
    a1 = -0.125
    return (1.0 - a1) * np.sin(np.pi * t) / np.pi + a1 * np.sin(3.0 * np.pi * t) / (3.0 * np.pi)


def dxi_s1(t):
    """d xi_s1 / dt = (1 - a_1) cos(pi t) + a_1 cos(3 pi t) with a_1 = -1/8."""
    a1 = -0.125
    return (1.0 - a1) * np.cos(np.pi * t) + a1 * np.cos(3.0 * np.pi * t)


def xi_ansatz(t, a):
    """xi_n(t) of the Sec. 3 ansatz with coefficients a = (a_1, ..., a_n):
    sin(pi t)/pi + sum_k a_k (sin((2k+1) pi t)/((2k+1) pi) - sin(pi t)/pi)."""
    t = np.asarray(t, dtype=np.float64)
    s1 = np.sin(np.pi * t) / np.pi
    out = s1.copy()
    for k, ak in enumerate(a, start=1):
        m = 2 * k + 1
        out += ak * (np.sin(m * np.pi * t) / (m * np.pi) - s1)
    return out


def dxi_ansatz(t, a):
    """d xi_n / dt = cos(pi t) + sum_k a_k (cos((2k+1) pi t) - cos(pi t))."""
    t = np.asarray(t, dtype=np.float64)
    c1 = np.cos(np.pi * t)
    out = c1.copy()
    for k, ak in enumerate(a, start=1):
        out += ak * (np.cos((2 * k + 1) * np.pi * t) - c1)
    return out


def g_s(x, a, self_value=None):
    """G_S(x) = -1/(4 pi |xhat|), xhat_i = xi_n(x_i) with coefficients a
    (Sec. 3 ansatz); ``self_value`` at x = 0 as in g_s1."""
    xh = xi_ansatz(np.asarray(x, dtype=np.float64), a)
    r = np.sqrt(np.sum(xh * xh, axis=-1))
    zero = r == 0.0
    if np.any(zero) and self_value is None:
        raise ValueError("G_S evaluated at 0 without a self-term value")
    out = np.empty_like(r)
    out[~zero] = -1.0 / (FOUR_PI * r[~zero])
    out[zero] = self_value if self_value is not None else 0.0
    return out


def grad_g_s(x, a):
    """grad G_S by the chain rule; 0 at x = 0."""
    x = np.asarray(x, dtype=np.float64)
    xh = xi_ansatz(x, a)
    r2 = np.sum(xh * xh, axis=-1)
    zero = r2 == 0.0
    r3 = np.where(zero, 1.0, r2 * np.sqrt(r2))
    out = xh * dxi_ansatz(x, a) / (FOUR_PI * r3[..., None])
    out[zero] = 0.0
    return out


def g_s1(x, self_value=None):
    """G_S1(x) = -1/(4 pi |xhat <> L|), xhat_i = L xi_s1(x_i/L)  (eq. gfs1, Sec. 4).

    ``x`` has shape (..., 3).  At x = 0 the function is singular; entries with
    |x| == 0 take ``self_value`` (the cell self-term reading, see self_term()),
    or raise if it is None.
    """
    x = np.asarray(x, dtype=np.float64)
    xh = wrap(xi_s1(x))          # the wrap of xhat is a no-op: |xi| <= 7/(6 pi) < 1/2
    r = np.sqrt(np.sum(xh * xh, axis=-1))
    zero = r == 0.0
    if np.any(zero) and self_value is None:
        raise ValueError("G_S1 evaluated at 0 without a self-term value")
    out = np.empty_like(r)
    out[~zero] = -1.0 / (FOUR_PI * r[~zero])
    out[zero] = self_value if self_value is not None else 0.0
    return out


def grad_g_s1(x):
    """grad G_S1 (chain rule on eq. gfs1): dG/dx_i = xhat_i xi'(x_i) / (4 pi |xhat|^3).

    Returns shape (..., 3).  At x = 0 the gradient is taken as 0 (G_S1 is even
    in every component, so the symmetric cell average of its gradient is 0).
    """
    x = np.asarray(x, dtype=np.float64)
    xh = xi_s1(x)
    r2 = np.sum(xh * xh, axis=-1)
    zero = r2 == 0.0
    r3 = np.where(zero, 1.0, r2 * np.sqrt(r2))
    out = xh * dxi_s1(x) / (FOUR_PI * r3[..., None])
    out[zero] = 0.0
    return out


def g_x(x, self_value=None):
    """Exact-in-real-space G_X(x) = -1/(4 pi |x <> L|)  (Sec. 1, eq. gfx)."""
    x = np.asarray(x, dtype=np.float64)
    xw = wrap(x)
    r = np.sqrt(np.sum(xw * xw, axis=-1))
    zero = r == 0.0
    if np.any(zero) and self_value is None:
        raise ValueError("G_X evaluated at 0 without a self-term value")
    out = np.empty_like(r)
    out[~zero] = -1.0 / (FOUR_PI * r[~zero])
    out[zero] = self_value if self_value is not None else 0.0
    return out


def grad_g_x(x):
    """grad G_X = x_w / (4 pi |x_w|^3) with x_w = x <> L; 0 at x = 0.

    G_X has a kink where a component of x_w is +-L/2 (Sec. 1); there the two
    one-sided derivatives are opposite and this function returns their mean, 0.
    """
    x = np.asarray(x, dtype=np.float64)
    xw = wrap(x)
    r2 = np.sum(xw * xw, axis=-1)
    zero = r2 == 0.0
    r3 = np.where(zero, 1.0, r2 * np.sqrt(r2))
    out = np.where(np.abs(xw) == 0.5, 0.0, xw) / (FOUR_PI * r3[..., None])
    out[zero] = 0.0
    return out


def g0(r):
    """Continuous Green's function G_0 = -1/(4 pi r)  (Sec. 1)."""
    return -1.0 / (FOUR_PI * np.asarray(r, dtype=np.float64))


def self_term(n_cells):
    """G(0) for a mesh of n_cells^3 cells of size h = 1/n_cells.

    Reading (the paper does not define the self term): the potential of a cell
    on itself is G_0 averaged over the cell, -(1/4 pi) <1/r>_cell =
    -(1/4 pi) CUBE_MEAN_INV_R / h.  The same constant is used by the oracle's
    PM, direct and FMM solutions, so it never separates them.
    """
    return -CUBE_MEAN_INV_R * float(n_cells) / FOUR_PI


def kvectors(n):
    """Integer wave numbers n_i in the FFT order of numpy, covering
    -N/2+1 .. N/2 as in Sec. 1 after eq. gfk (the Nyquist entry -N/2 of numpy's
    ordering is the same discrete mode as +N/2)."""
    return np.fft.fftfreq(n, d=1.0 / n)


def g_k_kernel(n):
    """Spectral G_K on an n^3 mesh: -1/k^2 with k = 2 pi n, and 0 at k = 0
    (Sec. 1, eq. gfk).  Shape (n, n, n) indexed [kz, ky, kx]."""
    f = kvectors(n)
    kz, ky, kx = np.meshgrid(f, f, f, indexing="ij")
    k2 = (2.0 * np.pi) ** 2 * (kx * kx + ky * ky + kz * kz)
    out = np.zeros_like(k2)
    nz = k2 != 0.0
    out[nz] = -1.0 / k2[nz]
    return out
