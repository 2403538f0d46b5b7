"""Seeded synthetic density fields (host, numpy).

Shared by the tests, the bench and the oracle checks.  Holds none of the FMM's
arithmetic: only the recipes that make density fields of the shapes the paper
and its workloads use.  Every generator takes an explicit seed and returns a
C-contiguous float32 array indexed [z][y][x] (x fastest); the ``*_torch``
variants evaluate the same recipe on a torch device (for 512^3 fields).

Recipes
-------
lognormal   1 + amp * exp(sigma g - sigma^2/2), g a unit-variance Gaussian
            random field with power spectrum P(k) ~ k^-2 (k = 2 pi n), zero
            mean mode.
plummer     background + clumps rho_c(r) = (3 M / 4 pi a^3)(1 + r^2/a^2)^-5/2
            with minimum-image r, centres uniform, a log-uniform in
            [a_min, a_max] cells, M log-uniform over two decades, each clump
            truncated at 8 a (or half the box) and renormalised so its mesh
            sum is M; the clump masses add up to the background mass.
point       unit total mass in one cell (the paper's corner-source test,
            Sec. 3): rho = N^3 in that cell, 0 elsewhere.
"""
import numpy as np


def rng_for(config, field=0):
    """numpy PCG64 seeded with 1000 * config + field."""
    return np.random.Generator(np.random.PCG64(1000 * int(config) + int(field)))


def gaussian_field(n, rng, slope=-2.0):
    """Unit-variance Gaussian random field on an n^3 mesh with P(k) ~ k^slope."""
    white = rng.standard_normal((n, n, n))
    f = np.fft.fftfreq(n, d=1.0 / n)
    kz, ky, kx = np.meshgrid(f, f, f, indexing="ij")
    k = 2.0 * np.pi * np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(k)
    nz = k > 0
    amp[nz] = k[nz] ** (0.5 * slope)
    g = np.fft.ifftn(np.fft.fftn(white) * amp).real
    g -= g.mean()
    s = g.std()
    return g / s if s > 0 else g


def gaussian_field_torch(n, rng, device, slope=-2.0):
    """gaussian_field with the FFTs on a torch device (same white noise)."""
    import torch
    white = torch.from_numpy(rng.standard_normal((n, n, n))).to(device)
    f = torch.fft.fftfreq(n, d=1.0 / n, device=device, dtype=torch.float64)
    kz, ky, kx = torch.meshgrid(f, f, f, indexing="ij")
    k = 2.0 * np.pi * torch.sqrt(kx * kx + ky * ky + kz * kz)
    amp = torch.where(k > 0, k.clamp_min(1e-30) ** (0.5 * slope), torch.zeros_like(k))
    del kx, ky, kz, k
    g = torch.fft.ifftn(torch.fft.fftn(white) * amp).real
    g -= g.mean()
    s = g.std(unbiased=False)          # population deviation, as numpy's std
    return g / s if float(s) > 0 else g


def lognormal(n, sigma=0.5, seed=0, amp=0.5, background=1.0, device=None):
    """Density = background + amp * lognormal(sigma) field (mean of the
    exponential is 1).  With ``device`` (a torch device) the FFTs run there and
    a float32 torch tensor on that device is returned."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if device is not None:
        import torch
        g = gaussian_field_torch(n, rng, device)
        return (background + amp * torch.exp(sigma * g - 0.5 * sigma * sigma)).float().contiguous()
    g = gaussian_field(n, rng)
    rho = background + amp * np.exp(sigma * g - 0.5 * sigma * sigma)
    return np.ascontiguousarray(rho, dtype=np.float32)


def plummer(n, n_clumps=512, seed=0, a_min=0.5, a_max=8.0, decades=2.0,
            background=1.0, base=None):
    """Background (or ``base`` field) plus Plummer clumps; see module doc."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rho = (np.full((n, n, n), background, dtype=np.float64) if base is None
           else np.array(base, dtype=np.float64))
    centres = rng.random((n_clumps, 3)) * n                   # cell units, (x, y, z)
    a = np.exp(rng.uniform(np.log(a_min), np.log(a_max), n_clumps))
    lm = rng.uniform(0.0, decades * np.log(10.0), n_clumps)
    mass = np.exp(lm)
    # clump masses (in units where the box volume is n^3 cells) add up to the
    # background mass n^3 * background
    mass *= background * n ** 3 / mass.sum()
    for c, ac, mc in zip(centres, a, mass):
        w = int(min(n // 2 - 1, np.ceil(8.0 * ac)))
        lo = np.floor(c).astype(np.int64) - w
        idx = [np.arange(lo[i], lo[i] + 2 * w + 2) for i in range(3)]
        # minimum-image displacement of cell centres from the clump centre
        d = [((ix + 0.5 - c[i]) + 0.5 * n) % n - 0.5 * n for i, ix in enumerate(idx)]
        dz, dy, dx = np.meshgrid(d[2], d[1], d[0], indexing="ij")
        r2 = dx * dx + dy * dy + dz * dz
        prof = (1.0 + r2 / (ac * ac)) ** -2.5
        prof[r2 > (8.0 * ac) ** 2] = 0.0
        prof *= mc / prof.sum()
        iz, iy, ix = (idx[2] % n), (idx[1] % n), (idx[0] % n)
        np.add.at(rho, np.ix_(iz, iy, ix), prof)
    return np.ascontiguousarray(rho, dtype=np.float32)


def plummer_torch(base, n_clumps, seed, a_min=0.5, a_max=8.0, decades=2.0, background=1.0):
    """``plummer`` evaluated on a torch device: ``base`` is the (n,n,n) float
    tensor the clumps are added to (in place, returned).  Same parameter draws
    and profile as ``plummer``."""
    import torch
    dev = base.device
    n = base.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.random((n_clumps, 3)) * n
    a = np.exp(rng.uniform(np.log(a_min), np.log(a_max), n_clumps))
    lm = rng.uniform(0.0, decades * np.log(10.0), n_clumps)
    mass = np.exp(lm)
    mass *= background * n ** 3 / mass.sum()
    acc = base.double().reshape(-1)
    for c, ac, mc in zip(centres, a, mass):
        w = int(min(n // 2 - 1, np.ceil(8.0 * ac)))
        lo = np.floor(c).astype(np.int64) - w
        idx = [torch.arange(int(lo[i]), int(lo[i]) + 2 * w + 2, device=dev) for i in range(3)]
        d = [((ix.double() + 0.5 - float(c[i])) + 0.5 * n) % n - 0.5 * n for i, ix in enumerate(idx)]
        r2 = d[2][:, None, None] ** 2 + d[1][None, :, None] ** 2 + d[0][None, None, :] ** 2
        prof = (1.0 + r2 / (ac * ac)) ** -2.5
        prof = torch.where(r2 > (8.0 * ac) ** 2, torch.zeros_like(prof), prof)
        prof *= mc / prof.sum()
        iz, iy, ix = idx[2] % n, idx[1] % n, idx[0] % n
        flat = (iz[:, None, None] * n + iy[None, :, None]) * n + ix[None, None, :]
        acc.index_add_(0, flat.reshape(-1), prof.reshape(-1))
    return acc.reshape(n, n, n).float().contiguous()


def point(n, cell=(0, 0, 0)):
    """Unit mass in one cell ((z, y, x) index); rho = n^3 there."""
    rho = np.zeros((n, n, n), dtype=np.float32)
    rho[tuple(cell)] = float(n) ** 3
    return rho


def config_density(config, n=None, field=0):
    """The density recipe of each workload configuration, seeded with
    1000 * config + field.

    0: 32^3 lognormal sigma 0.5;  1: 128^3 background + 512 Plummer clumps;
    3: 64^3 lognormal sigma 0.5 (training fields) / 256^3 evaluation fields;
    4: 512^3 1 + lognormal sigma 1.5 plus 4096 Plummer clumps.
    ``n`` overrides the mesh size (for scaled-down parity cases).
    """
    seed = 1000 * int(config) + int(field)
    if config == 0:
        return lognormal(n or 32, sigma=0.5, seed=seed)
    if config == 1:
        return plummer(n or 128, n_clumps=512, seed=seed)
    if config == 3:
        return lognormal(n or 64, sigma=0.5, seed=seed)
    if config == 4:
        nn = n or 512
        base = lognormal(nn, sigma=1.5, seed=seed, amp=1.0, background=1.0)
        return plummer(nn, n_clumps=4096, seed=seed + 1, base=base)
    if config == 5:            # the 256^3 headline workload: lognormal sigma 0.5
        return lognormal(n or 256, sigma=0.5, seed=seed)
    raise ValueError(f"unknown config {config}")


def config_density_torch(config, device, n=None, field=0):
    """config_density on a torch device (float32 tensor); configs 4 and 5."""
    seed = 1000 * int(config) + int(field)
    if config == 4:
        nn = n or 512
        base = lognormal(nn, sigma=1.5, seed=seed, amp=1.0, background=1.0, device=device)
        return plummer_torch(base, 4096, seed + 1)
    if config == 5:
        return lognormal(n or 256, sigma=0.5, seed=seed, device=device)
    raise ValueError(f"no device recipe for config {config}")
