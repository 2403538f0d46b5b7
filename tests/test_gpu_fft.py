"""The FFT (HPM) form of the interaction zone, Sec. 2, as an ablation of the
dense M2L: FMM_M2L_FFT against the FP64 oracle and against the dense FP32
form, through the C-ABI.

Tolerance: the convolution runs in FP32 through cuFFT over the whole 6x6x6
children block, and the 27 near nodes' terms, the largest of the block, are
subtracted afterwards; the FFT's rounding (relative to the block sum, ~1e-7
x log of the grid size) is amplified by the block-to-far-field ratio.
Bound 1e-5 (the dense FP32 form holds 1e-6)."""
import numpy as np
import pytest

from oracle import fmm as ofmm
from paper_2011_07099_gb300 import inputs
from parity_util import assert_close, corner_and_interior_leaves, leaf_values

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FFT = 1e-5


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_07099_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def _solve(B, rho, L, p, fft):
    plan = B.Plan(rho.shape[0], L, p)
    if fft:
        B.fmm_plan_set_m2l_algorithm(plan.handle, B.FMM_M2L_FFT)
    phi, acc = plan.solve(torch.from_numpy(rho).cuda())
    torch.cuda.synchronize()
    plan.close()
    return phi.cpu().numpy(), acc.cpu().numpy()


@pytest.mark.parametrize("N,L,p,recipe", [(64, 4, 4, "lognormal"), (64, 4, 3, "plummer"), (64, 5, 2, "lognormal")])
def test_fft_interaction_zone_matches_oracle(B, N, L, p, recipe):
    rho = (inputs.plummer(N, n_clumps=8, seed=N + p) if recipe == "plummer"
           else inputs.lognormal(N, sigma=0.5, seed=N + p))
    phi, acc = _solve(B, rho, L, p, fft=True)
    ophi, og = ofmm.solve(rho, L, p)
    assert_close(phi, ophi, TOL_FFT, f"FFT M2L phi {N}^3 L={L} p={p}")
    assert_close(acc, og, TOL_FFT, f"FFT M2L g {N}^3 L={L} p={p}")
    dphi, dacc = _solve(B, rho, L, p, fft=False)
    assert_close(phi, dphi, TOL_FFT, "FFT vs dense FP32 phi")


def test_fft_interaction_zone_at_256_sampled_leaves(B):
    N, L, p = 256, 5, 6
    rho = inputs.config_density(5, n=N)
    phi, acc = _solve(B, rho, L, p, fft=True)
    leaves = corner_and_interior_leaves(L, 2, seed=81)
    ref = ofmm.solve_at(rho, L, p, leaves)
    got = leaf_values(phi, acc, leaves, N >> L)
    assert_close(got[:, 0], ref[:, 0], TOL_FFT, "FFT M2L phi 256^3 sampled leaves")
    assert_close(got[:, 1:], ref[:, 1:], TOL_FFT, "FFT M2L g 256^3 sampled leaves")
