"""Pluggable Green's functions on the GPU (G_X of eq. gfx, G_K of eq. gfk
through fmm_plan_set_green_mesh) and the ablation of Fig. errex, through the
C-ABI."""
import numpy as np
import pytest

from oracle import green, pm
from paper_2011_07099_gb300 import inputs
from parity_util import assert_close

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


def test_gx_tabulation_matches_oracle(B):
    N = 24
    plan = B.Plan(N, 2, 5)
    B.fmm_plan_set_green(plan.handle, B.FMM_GREEN_X)
    K = torch.empty(4 * N ** 3, dtype=torch.float64, device="cuda")
    B.fmm_plan_mesh_green(plan.handle, K)
    torch.cuda.synchronize()
    plan.close()
    K = K.cpu().numpy().reshape(4, N, N, N)
    k = np.arange(N)
    dz, dy, dx = np.meshgrid(k, k, k, indexing="ij")
    d = np.stack([dx, dy, dz], axis=-1) / N
    np.testing.assert_allclose(K[0], green.g_x(d, self_value=green.self_term(N)), rtol=1e-13)
    mdG = -np.moveaxis(green.grad_g_x(d), -1, 0)
    np.testing.assert_allclose(K[1:], mdG, rtol=1e-12, atol=1e-13 * np.abs(mdG).max())


def test_gk_mesh_plan_two_level_tree_equals_the_spectral_pm(B):
    # G_K handed over on the mesh: in the exact two-level case the FMM equals
    # the oracle's spectral PM with G_K (eq. gfk), potential up to a constant
    from paper_2011_07099_gb300 import ablation
    N, L, p = 16, 2, 4
    rho = inputs.plummer(N, n_clumps=4, seed=10, a_min=0.5, a_max=2.0)
    plan = ablation.make_plan(N, L, p, "K", torch.device("cuda", 0))
    phi, acc = plan.solve(torch.from_numpy(rho).cuda())
    torch.cuda.synchronize()
    plan.close()
    kphi, kg = pm.pm_gk(pm.masses(rho.astype(np.float64)))
    phi = phi.cpu().numpy().astype(np.float64)
    assert_close(phi - phi.mean(), kphi - kphi.mean(), 1e-6, "G_K two-level phi")
    assert_close(acc.cpu().numpy(), kg, 1e-6, "G_K two-level g")


def test_gk_mesh_requires_gridlets_on_the_mesh(B):
    plan = B.Plan(32, 3, 3)           # S = 4 is not a multiple of 3
    m = torch.zeros(4 * 32 ** 3, dtype=torch.float64, device="cuda")
    assert B.lib().fmm_plan_set_green_mesh(plan.handle, m.data_ptr(), m.numel()) == B.FMM_ERR_ARG
    plan.close()


def test_fig_errex_in_3d(B):
    # Fig. errex: with G_X the FMM and PM solutions differ grossly (aliasing
    # at half the box), with G_S1 they nearly agree; G_K, the PM's own
    # function, is not one the FMM reproduces either (Sec. 3).  Corner unit
    # source, 64^3 mesh, L = 3, N_g = S = 8 (gridlets on the mesh, as G_K needs)
    from paper_2011_07099_gb300 import ablation, accuracy
    N, L, p = 64, 3, 8
    d = torch.from_numpy(accuracy.point_sources(N, "corner")).cuda()
    r = {g: ablation.fmm_vs_pm(N, L, p, d, g) for g in ("S1", "X", "K")}
    for g, v in r.items():
        print(f"{g}: rel phi {v['rel_phi']:.3e} rel g {v['rel_g']:.3e} |dg| L_MAX {v['abs_g'][0]:.3e} L2 {v['abs_g'][1]:.3e}")
    assert r["X"]["rel_g"] > 10 * r["S1"]["rel_g"]
    assert r["K"]["rel_g"] > r["S1"]["rel_g"]
