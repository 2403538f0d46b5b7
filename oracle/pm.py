"""Periodic convolution references, FP64 (test infrastructure).

Cells of an N^3 mesh over the unit box sit at x_j = (j + 1/2)/N, j in [0, N)^3,
arrays are indexed [z][y][x].  A mesh mass is m_j = (rho_j - mean rho) / N^3.
For any 1-periodic G the potential and acceleration on the mesh are

    Phi_i = sum_j G(x_i - x_j) m_j,      g_i = -sum_j grad G(x_i - x_j) m_j,

which is the PM convolution of Sec. 3 eq. pmconv (and the Sec. 1 PM method
when G = G_K).  ``direct`` evaluates the double sum literally; ``pm`` evaluates
the same circular convolution with numpy's FFT.  ``pm_gk`` is the spectral
solution with G_K of eq. gfk.

Pins (tests/test_oracle_pm.py): ``pm`` against ``direct`` on 8^3 and 16^3 for
G_S1 and G_X; ``pm_gk`` against a single Fourier mode whose potential is known
in closed form, and against ``direct`` with G_K evaluated in real space by an
explicit inverse-DFT sum.
"""
import numpy as np

from . import green


def masses(rho):
    """Mesh masses m = (rho - mean(rho)) / N^3 (Sec. 1: only the mean-free
    density has a periodic potential; the k = 0 mode of eq. gfk is zero)."""
    rho = np.asarray(rho, dtype=np.float64)
    n = rho.shape[0]
    return (rho - rho.mean()) / float(n) ** 3


def offsets_grid(n):
    """Integer offsets d in [0, n)^3 as an (n, n, n, 3) array with components
    ordered (x, y, z) and the grid indexed [dz][dy][dx]."""
    r = np.arange(n)
    dz, dy, dx = np.meshgrid(r, r, r, indexing="ij")
    return np.stack([dx, dy, dz], axis=-1).astype(np.float64)


def direct(m, gfun, gradfun, self_value, chunk=512):
    """Brute-force periodic sum over every pair of cells.

    ``gfun(x, self_value)`` and ``gradfun(x)`` take displacements in box units
    of shape (..., 3).  Returns (phi (n,n,n), g (3,n,n,n)) with g = -grad Phi.
    O(N^6): meant for N <= 16.
    """
    m = np.asarray(m, dtype=np.float64)
    n = m.shape[0]
    pos = offsets_grid(n).reshape(-1, 3)          # cell index (x, y, z) per flat cell
    mf = m.reshape(-1)
    phi = np.zeros(n ** 3)
    g = np.zeros((n ** 3, 3))
    for a in range(0, n ** 3, chunk):
        d = (pos[a:a + chunk, None, :] - pos[None, :, :]) / n      # x_i - x_j
        phi[a:a + chunk] = gfun(d, self_value) @ mf
        g[a:a + chunk] = -np.einsum("ijc,j->ic", gradfun(d), mf)
    return phi.reshape(n, n, n), np.moveaxis(g, -1, 0).reshape(3, n, n, n)


def pm(m, gfun, gradfun, self_value):
    """FFT circular convolution of the masses with G sampled at the mesh
    offsets d/N (Sec. 3 eq. pmconv; the PM method of Sec. 1 for a real-space G).
    Returns (phi, g) like ``direct``."""
    m = np.asarray(m, dtype=np.float64)
    n = m.shape[0]
    d = offsets_grid(n) / n
    kern = gfun(d, self_value)
    gk = gradfun(d)
    mh = np.fft.fftn(m)
    phi = np.fft.ifftn(mh * np.fft.fftn(kern)).real
    g = np.stack([-np.fft.ifftn(mh * np.fft.fftn(gk[..., c])).real for c in range(3)])
    return phi, g


def pm_gk(m):
    """Spectral PM with the exact-in-Fourier-space G_K (Sec. 1, eq. gfk).

    With x_j on the mesh, G_K(x) = sum_n Gt_K(2 pi n) exp(2 pi i n.x) and the
    discrete convolution becomes Phi_hat(n) = N^3 Gt_K(n) m_hat(n).  The
    acceleration is the spectral -grad: g_hat = -i k Phi_hat, with the Nyquist
    wave number (whose sine vanishes on the mesh) given zero derivative.
    """
    m = np.asarray(m, dtype=np.float64)
    n = m.shape[0]
    phih = np.fft.fftn(m) * (float(n) ** 3) * green.g_k_kernel(n)
    phi = np.fft.ifftn(phih).real
    f = green.kvectors(n)
    if n % 2 == 0:
        f = f.copy()
        f[n // 2] = 0.0
    kz, ky, kx = np.meshgrid(f, f, f, indexing="ij")
    g = np.stack([np.fft.ifftn(-1j * 2.0 * np.pi * k * phih).real for k in (kx, ky, kz)])
    return phi, g


def g_k_real_space(n):
    """G_K at the mesh offsets d/N by the explicit inverse-DFT sum of Sec. 1
    (below eq. gfk), without an FFT: G_K(d/N) = sum_n Gt_K(2 pi n) cos(2 pi n.d/N).
    Also returns grad G_K by the same sum with the Nyquist derivative zeroed,
    consistent with ``pm_gk``.  Cost O(N^6): for N <= 8."""
    f = green.kvectors(n)
    kz, ky, kx = np.meshgrid(f, f, f, indexing="ij")
    gt = green.g_k_kernel(n).reshape(-1)
    nvec = np.stack([kx, ky, kz], axis=-1).reshape(-1, 3)
    fd = f.copy()
    if n % 2 == 0:
        fd[n // 2] = 0.0
    kzd, kyd, kxd = np.meshgrid(fd, fd, fd, indexing="ij")
    nder = np.stack([kxd, kyd, kzd], axis=-1).reshape(-1, 3)
    d = offsets_grid(n).reshape(-1, 3)
    phase = 2.0 * np.pi * (d @ nvec.T) / n                 # (cells, modes)
    kern = np.cos(phase) @ gt
    # d/dx cos(2 pi n.x) = -2 pi n sin(2 pi n.x)
    grad = -(np.sin(phase) * gt[None, :]) @ (2.0 * np.pi * nder)
    return kern.reshape(n, n, n), grad.reshape(n, n, n, 3)


def direct_tabulated(m, kern, grad):
    """Direct periodic convolution with a kernel given at the mesh offsets
    (arrays from ``g_k_real_space``): Phi_i = sum_j K[(i - j) mod N] m_j."""
    m = np.asarray(m, dtype=np.float64)
    n = m.shape[0]
    phi = np.zeros_like(m)
    g = np.zeros((3,) + m.shape)
    idx = np.arange(n)
    for jz in range(n):
        for jy in range(n):
            for jx in range(n):
                mj = m[jz, jy, jx]
                if mj == 0.0:
                    continue
                sz = (idx - jz) % n
                sy = (idx - jy) % n
                sx = (idx - jx) % n
                k = kern[np.ix_(sz, sy, sx)]
                gr = grad[np.ix_(sz, sy, sx)]
                phi += k * mj
                g -= np.moveaxis(gr, -1, 0) * mj
    return phi, g
