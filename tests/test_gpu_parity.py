"""CUDA path against the FP64 oracle, element by element, through the C-ABI.

The plain form (FMM_PREC_FP32) must match the oracle to relative L2 <= 1e-6 on
the potential and the acceleration (ratio of the 2-norm of the difference over
the whole mesh to the 2-norm of the oracle).  Stage buffers (gridlet masses and
local fields, Morton order on the GPU) are compared to the oracle's stages.
"""
import numpy as np
import pytest

from oracle import fmm as ofmm
from oracle import green, pm
from paper_2011_07099_gb300 import inputs
from parity_util import assert_close, corner_and_interior_leaves, leaf_values

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-6


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_07099_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _morton_keys(level):
    n = 2 ** level
    iz, iy, ix = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    key = np.zeros_like(ix)
    for b in range(level):
        key |= ((ix >> b) & 1) << (3 * b)
        key |= ((iy >> b) & 1) << (3 * b + 1)
        key |= ((iz >> b) & 1) << (3 * b + 2)
    return key


def _gpu_solve(B, rho, L, p, prec=0):
    plan = B.Plan(rho.shape[0], L, p)
    if prec:
        plan.set_precision(prec)
    d = torch.from_numpy(rho).cuda()
    phi, acc = plan.solve(d)
    torch.cuda.synchronize()
    return plan, phi.cpu().numpy(), acc.cpu().numpy()


CASES = [
    # (N, L, p, recipe)
    (8, 2, 2, "plummer"),      # two-level exact case, S = p = 2
    (16, 2, 4, "lognormal"),   # two-level exact case, S = p = 4
    (16, 3, 2, "lognormal"),
    (32, 3, 4, "plummer"),
    (32, 4, 2, "lognormal"),   # S = 2
    (32, 5, 2, "lognormal"),   # the 32^3 5-level p = 2 workload, S = 1
    (64, 3, 6, "lognormal"),   # S = 8, p = 6: several M2L tiles and a ragged last tile
    (64, 4, 3, "plummer"),     # S = 4, odd order
    (32, 3, 6, "lognormal"),   # S = 4 below p = 6: the shape of the batch workload's small order-6 fields
    (48, 3, 6, "plummer"),     # S = 6 = p, N = 48 (a batch size that needs S = 3 or 6)
]


def _density(n, recipe, seed):
    if recipe == "plummer":
        return inputs.plummer(n, n_clumps=max(2, n // 4), seed=seed, a_min=0.5, a_max=min(8.0, n / 4))
    return inputs.lognormal(n, sigma=0.5, seed=seed)


@pytest.mark.parametrize("N,L,p,recipe", CASES)
def test_fp32_solve_matches_oracle(B, N, L, p, recipe):
    rho = _density(N, recipe, seed=N * 10 + L)
    plan, phi, acc = _gpu_solve(B, rho, L, p)
    ophi, og = ofmm.solve(rho, L, p)
    assert_close(phi, ophi, TOL_FP32, f"phi {N}^3 L={L} p={p}")
    assert_close(acc, og, TOL_FP32, f"g {N}^3 L={L} p={p}")
    plan.close()


@pytest.mark.parametrize("N,L,p", [(32, 3, 3), (64, 4, 4)])
def test_stage_buffers_match_oracle(B, N, L, p):
    rho = inputs.lognormal(N, sigma=1.0, seed=3)
    plan, phi, acc = _gpu_solve(B, rho, L, p)
    m = pm.masses(rho.astype(np.float64))
    M = ofmm.upward(m, L, p)
    F = ofmm.downward(M, L, p)
    mean = plan.stage(B.FMM_STAGE_MEAN, 0).cpu().numpy()[0]
    assert abs(mean - rho.astype(np.float64).mean()) <= 1e-7 * abs(rho.mean())
    for lev in range(2, L + 1):
        key = _morton_keys(lev).reshape(-1)
        n = 2 ** lev
        gm = plan.stage(B.FMM_STAGE_MULTIPOLE, lev).cpu().numpy().reshape(8 ** lev, p ** 3)
        om = M[lev].reshape(n ** 3, p ** 3)
        assert_close(gm[key], om, TOL_FP32, f"multipoles level {lev}")
        gf = plan.stage(B.FMM_STAGE_LOCAL, lev).cpu().numpy().reshape(8 ** lev, 4, p ** 3)
        of = F[lev].reshape(n ** 3, 4, p ** 3)
        assert_close(gf[key], of, TOL_FP32, f"local fields level {lev}")
    plan.close()


def test_uniform_density_gives_zero_field(B):
    rho = np.full((32, 32, 32), 1.7, dtype=np.float32)
    plan, phi, acc = _gpu_solve(B, rho, 3, 4)
    assert np.all(phi == 0) and np.all(acc == 0)


def test_corner_point_source(B):
    # the paper's worst-case test source (Sec. 3): unit mass in the corner cell
    rho = inputs.point(32)
    plan, phi, acc = _gpu_solve(B, rho, 3, 4)
    ophi, og = ofmm.solve(rho, 3, 4)
    assert_close(phi, ophi, TOL_FP32, "corner source phi")
    assert_close(acc, og, TOL_FP32, "corner source g")
    # zero net force on the whole mesh (G odd gradient)
    m = pm.masses(rho.astype(np.float64))
    f = (m[None] * acc.astype(np.float64)).sum(axis=(1, 2, 3))
    assert np.abs(f).max() < 1e-6 * (np.abs(m)[None] * np.abs(acc)).sum()


def test_solve_is_deterministic_and_host_path_agrees(B):
    rho = inputs.lognormal(32, sigma=1.0, seed=9)
    plan = B.Plan(32, 3, 4)
    d = torch.from_numpy(rho).cuda()
    p1, a1 = plan.solve(d)
    p2, a2 = plan.solve(d)
    torch.cuda.synchronize()
    assert torch.equal(p1, p2) and torch.equal(a1, a2)
    hp = torch.empty((32, 32, 32), dtype=torch.float32).pin_memory()
    ha = torch.empty((3, 32, 32, 32), dtype=torch.float32).pin_memory()
    B.fmm_solve_host(plan.handle, torch.from_numpy(rho).pin_memory(), hp, ha)
    assert torch.equal(hp, p1.cpu()) and torch.equal(ha, a1.cpu())


def test_bad_pointers_are_rejected(B):
    plan = B.Plan(32, 3, 2)
    d = torch.zeros(32 ** 3 + 4, dtype=torch.float32, device="cuda")
    out = torch.zeros(4 * 32 ** 3 + 4, dtype=torch.float32, device="cuda")
    L = B.lib()
    # misaligned (4-byte offset) density
    rc = L.fmm_solve(plan.handle, d.data_ptr() + 4, out.data_ptr(), out.data_ptr() + 4 * 32 ** 3 * 4, None)
    assert rc == B.FMM_ERR_ARG
    rc = L.fmm_solve(plan.handle, None, out.data_ptr(), out.data_ptr(), None)
    assert rc == B.FMM_ERR_ARG
    with pytest.raises(B.FMMError):
        plan.stage(B.FMM_STAGE_LOCAL, 9)


FULL = [
    # (N, L, p, config): the 256^3 p = 6 headline workload and the 128^3
    # p = 4 Plummer-clump workload at full size, in the launch configuration
    # the bench times; the oracle evaluates only the sampled leaves (whole
    # upward pass, then each leaf's chain of ancestors): the 8 corner leaves,
    # where every periodic wrap is taken, and 2 interior leaves.
    (256, 5, 6, 5),
    (128, 5, 4, 1),
    # the clustered order-8 recipe (1 + lognormal sigma 1.5 + Plummer clumps)
    # at 256^3, S = p = 8: the high-order precision path (FP64 masses and
    # local fields, double-float M2L at every level above the leaves)
    (256, 5, 8, 4),
]


@pytest.mark.parametrize("N,L,p,cfg", FULL)
def test_full_size_sampled_leaves_match_oracle(B, N, L, p, cfg):
    if cfg == 4:   # the clump recipe is evaluated on the device (4096 clumps)
        rho = inputs.config_density_torch(cfg, torch.device("cuda", 0), n=N).cpu().numpy()
    else:
        rho = inputs.config_density(cfg, n=N)
    plan, phi, acc = _gpu_solve(B, rho, L, p)
    leaves = corner_and_interior_leaves(L, 2, seed=N + p)
    ref = ofmm.solve_at(rho, L, p, leaves)
    got = leaf_values(phi, acc, leaves, N >> L)
    assert_close(got[:, 0], ref[:, 0], TOL_FP32, f"phi {N}^3 p={p} sampled leaves")
    assert_close(got[:, 1:], ref[:, 1:], TOL_FP32, f"g {N}^3 p={p} sampled leaves")
    plan.close()


def test_full_scale_512_order8_sampled_leaves(B):
    # the full-scale workload exactly as bench.py --workload full512 runs it
    # (512^3, p = 8, L = 6, clustered recipe on the device), plain and mixed
    # forms against the oracle at the 8 corner leaves and 2 interior ones
    # (one oracle evaluation)
    N, L, p = 512, 6, 8
    leaves = corner_and_interior_leaves(L, 2, seed=512)
    rho_t = inputs.config_density_torch(4, torch.device("cuda", 0), n=N)
    rho = rho_t.cpu().numpy()
    ref = ofmm.solve_at(rho, L, p, leaves)
    S = N >> L
    for prec, tol in ((0, TOL_FP32), (B.FMM_PREC_BF16X3, 2e-5)):
        plan = B.Plan(N, L, p)
        if prec:
            plan.set_precision(prec)
        phi, acc = plan.solve(rho_t)
        torch.cuda.synchronize()
        got = np.stack([torch.cat([phi[a * S:(a + 1) * S, b * S:(b + 1) * S, c * S:(c + 1) * S].reshape(1, -1),
                                   acc[:, a * S:(a + 1) * S, b * S:(b + 1) * S, c * S:(c + 1) * S].reshape(3, -1)]
                                  ).cpu().numpy()
                        for a, b, c in leaves])
        plan.close()
        del phi, acc
        assert_close(got[:, 0], ref[:, 0], tol, f"512^3 p=8 precision {prec} phi")
        assert_close(got[:, 1:], ref[:, 1:], tol, f"512^3 p=8 precision {prec} g")
