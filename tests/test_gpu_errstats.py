"""The sampled error statement (fmm_plan_error_stats) through the C-ABI.

Its reference is the PM solution with the FMM's own Green's function (Sec. 3:
G_* is defined by PM and FMM agreeing), i.e. the periodic convolution with
G_S1 sampled on the mesh plus the self term, which the FP64 oracle computes
by FFT.  Given the oracle's PM fields as the "solution", the statement must
read zero (to the FP32 storage of the fields and the kernel's FP32 pair
values); given a known perturbation it must read that perturbation; given the
FMM's result it must agree with the whole-mesh error.
"""
import numpy as np
import pytest

from oracle import green, pm
from paper_2011_07099_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_07099_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def _pm_fields(rho):
    n = rho.shape[0]
    return pm.pm(pm.masses(rho), green.g_s1, green.grad_g_s1, green.self_term(n))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _splitmix_cells(seed, samples, n3):
    """The sampled cells as the header documents them: the first `samples`
    outputs of splitmix64 (Steele, Lea and Flood 2014) seeded with `seed`,
    modulo N^3."""
    mask = (1 << 64) - 1
    out = []
    for i in range(samples):
        z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & mask
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        out.append((z ^ (z >> 31)) % n3)
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("N,L,p,samples", [
    (16, 2, 4, 1024),
    (24, 2, 3, 100),     # N^3 not a multiple of the source chunk; a partial block of targets
    (32, 3, 4, 777),
])
def test_pm_fields_read_as_zero_error(B, N, L, p, samples):
    rho = inputs.lognormal(N, sigma=0.5, seed=N + samples)
    phi, g = _pm_fields(rho)
    plan = B.Plan(N, L, p)
    e_phi, e_g = plan.error_stats(_dev(rho), _dev(phi), _dev(g), samples=samples, seed=7)
    plan.close()
    assert e_phi < 1e-6 and e_g < 1e-6, (e_phi, e_g)


@pytest.mark.parametrize("samples,seed", [(1, 1), (300, 9)])
def test_statement_reads_cellwise_perturbations_at_the_documented_cells(B, samples, seed):
    # every cell carries its own relative perturbation (magnitude 5e-4..1e-3,
    # random sign), so the statement depends on which cells were sampled;
    # seed 1 draws a cell where |Phi| and |g| are above their RMS
    N = 32
    rho = inputs.plummer(N, n_clumps=8, seed=3, a_min=0.5, a_max=4.0)
    phi, g = _pm_fields(rho)
    rng = np.random.default_rng(seed)
    eps = rng.uniform(5e-4, 1e-3, phi.shape) * rng.choice([-1.0, 1.0], phi.shape)
    dlt = rng.uniform(5e-4, 1e-3, phi.shape) * rng.choice([-1.0, 1.0], phi.shape)
    cells = _splitmix_cells(seed, samples, N ** 3)
    f, gf = phi.reshape(-1)[cells], g.reshape(3, -1)[:, cells]
    want_phi = np.sqrt(np.sum((eps.reshape(-1)[cells] * f) ** 2) / np.sum(f * f))
    want_g = np.sqrt(np.sum((dlt.reshape(-1)[cells] * gf) ** 2) / np.sum(gf * gf))
    plan = B.Plan(N, 3, 4)
    args = (_dev(rho), _dev(phi * (1 + eps)), _dev(g * (1 + dlt)))
    e_phi, e_g = plan.error_stats(*args, samples=samples, seed=seed)
    assert e_phi == pytest.approx(want_phi, rel=2e-3) and e_g == pytest.approx(want_g, rel=2e-3)
    assert plan.error_stats(*args, samples=samples, seed=seed) == (e_phi, e_g)   # deterministic
    plan.close()


def test_sample_counts_outside_the_range_are_refused(B):
    rho = inputs.lognormal(16, sigma=0.5, seed=2)
    phi, g = _pm_fields(rho)
    plan = B.Plan(16, 2, 4)
    for samples in (0, 1025):
        with pytest.raises(B.FMMError):
            plan.error_stats(_dev(rho), _dev(phi), _dev(g), samples=samples)
    plan.close()


def test_statement_of_a_solve_agrees_with_the_whole_mesh_error(B):
    # the plain FP32 result equals the oracle's FMM to 1e-6 (parity tests), so
    # the statement estimates the method's own error against PM; 1024 cells
    # of 64^3 give it to well within a factor 2
    N, L, p = 64, 3, 6
    rho = inputs.lognormal(N, sigma=0.5, seed=11)
    phi_pm, g_pm = _pm_fields(rho)
    plan = B.Plan(N, L, p)
    d = _dev(rho)
    phi, acc = plan.solve(d)
    torch.cuda.synchronize()
    full_phi, full_g = _rel(phi.cpu().numpy(), phi_pm), _rel(acc.cpu().numpy(), g_pm)
    e_phi, e_g = plan.error_stats(d, phi, acc, samples=1024, seed=5)
    plan.close()
    assert 0.5 < e_phi / full_phi < 2.0 and 0.5 < e_g / full_g < 2.0, (e_phi, full_phi, e_g, full_g)
