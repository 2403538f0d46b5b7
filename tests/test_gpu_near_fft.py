"""The near zone by FFT convolution on the doubled grid (FMM_NEAR_FFT, the
approach of Sec. 3 for a regular grid) against the FP64 oracle, through the
C-ABI: the plain FP32 form over whole meshes (periodic and isolated), and the
headline mixed form at the sampled leaves of the 256^3 tree.

Tolerance: the sum is the direct sum's, but each neighbour pair's
contribution passes through FP32 transforms of 16^3 points with 8 nonzero
inputs per axis (three forward axes, a 27-term product sum, three inverse
axes): rounding of ~1e-7 times the square root of the ~100 operations each
value accumulates, i.e. ~1e-6 of the near field's own size; where the near
and far fields cancel (mean-free masses), the relative error of the total
grows by the near-to-total ratio, a few.  Bound 5e-6 for the FP32 form (the
direct FP32 form holds 1e-6); the mixed form keeps its bf16x3 bound 2e-5."""
import numpy as np
import pytest

from oracle import fmm as ofmm
from oracle import nonperiodic as npo
from paper_2011_07099_gb300 import inputs
from parity_util import assert_close, corner_and_interior_leaves, leaf_values

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_NEAR_FFT = 5e-6
TOL_BF16X3 = 2e-5


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_07099_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def _solve(B, rho, L, p, fft, iso=False, prec=None, weights=None):
    plan = B.Plan(rho.shape[0], L, p)
    if iso:
        B.fmm_plan_set_boundary(plan.handle, B.FMM_BOUNDARY_ISOLATED)
    if prec is not None:
        plan.set_precision(prec)
    if weights is not None:
        B.fmm_plan_set_correction(plan.handle, torch.from_numpy(weights.astype(np.float32)).cuda())
    if fft:
        B.fmm_plan_set_near_algorithm(plan.handle, B.FMM_NEAR_FFT)
    phi, acc = plan.solve(torch.from_numpy(rho).cuda())
    torch.cuda.synchronize()
    assert B.lib().fmm_plan_check(plan.handle) == B.FMM_OK
    plan.close()
    return phi.cpu().numpy(), acc.cpu().numpy()


@pytest.mark.parametrize("N,L,p,recipe", [(32, 2, 4, "lognormal"), (64, 3, 6, "plummer"), (64, 3, 3, "lognormal")])
def test_near_fft_matches_oracle(B, N, L, p, recipe):
    rho = (inputs.plummer(N, n_clumps=8, seed=N + p) if recipe == "plummer"
           else inputs.lognormal(N, sigma=0.5, seed=N + p))
    phi, acc = _solve(B, rho, L, p, fft=True)
    ophi, og = ofmm.solve(rho, L, p)
    assert_close(phi, ophi, TOL_NEAR_FFT, f"near FFT phi {N}^3 L={L} p={p}")
    assert_close(acc, og, TOL_NEAR_FFT, f"near FFT g {N}^3 L={L} p={p}")
    dphi, dacc = _solve(B, rho, L, p, fft=False)
    assert_close(phi, dphi, TOL_NEAR_FFT, "near FFT vs direct phi")
    assert_close(acc, dacc, TOL_NEAR_FFT, "near FFT vs direct g")


def test_near_fft_isolated_matches_oracle(B):
    N, L, p = 32, 2, 6
    rho = inputs.plummer(N, n_clumps=4, seed=5, a_min=0.5, a_max=4.0)
    phi, acc = _solve(B, rho, L, p, fft=True, iso=True)
    ophi, og = npo.solve_isolated(rho, L, p)
    assert_close(phi, ophi, TOL_NEAR_FFT, "isolated near FFT phi")
    assert_close(acc, og, TOL_NEAR_FFT, "isolated near FFT g")


def test_near_fft_point_source_is_the_direct_sum(B):
    # one unit mass in a corner cell: every neighbour pair and every lag of the
    # kernel spectra is exercised at the leaves around the periodic corner
    N, L, p = 32, 2, 4
    rho = np.zeros((N, N, N), np.float32)
    rho[0, 0, 0] = N ** 3
    phi, acc = _solve(B, rho, L, p, fft=True)
    dphi, dacc = _solve(B, rho, L, p, fft=False)
    assert_close(phi, dphi, TOL_NEAR_FFT, "point source near FFT vs direct phi")
    assert_close(acc, dacc, TOL_NEAR_FFT, "point source near FFT vs direct g")


def test_near_fft_needs_8_cell_leaves(B):
    plan = B.Plan(32, 3, 4)              # 4-cell leaves
    with pytest.raises(B.FMMError) as e:
        B.fmm_plan_set_near_algorithm(plan.handle, B.FMM_NEAR_FFT)
    assert e.value.code == B.FMM_ERR_UNSUPPORTED
    B.fmm_plan_set_near_algorithm(plan.handle, B.FMM_NEAR_DIRECT)
    plan.close()


def test_headline_form_with_near_fft_at_sampled_leaves(B):
    # the bench's fastest form at 256^3 p = 6: bf16x3 tensor-core M2L, the
    # shipped order-6 correction (BF16 inference) and the near zone by FFT,
    # against the oracle's FMM with the same weights
    from oracle import learn as olearn
    from paper_2011_07099_gb300 import learn
    N, L, p = 256, 5, 6
    w = learn.shipped_weights(p)
    rho = inputs.config_density(5, n=N)
    phi, acc = _solve(B, rho, L, p, fft=True, prec=B.FMM_PREC_BF16X3, weights=w)
    leaves = corner_and_interior_leaves(L, 2, seed=67)
    ref = ofmm.solve_at(rho, L, p, leaves, correction=olearn.correction_fn(w.astype(np.float64)))
    got = leaf_values(phi, acc, leaves, N >> L)
    assert_close(got[:, 0], ref[:, 0], TOL_BF16X3, "headline form + near FFT phi, sampled leaves")
    assert_close(got[:, 1:], ref[:, 1:], TOL_BF16X3, "headline form + near FFT g, sampled leaves")


def test_overlapped_solve_equals_the_serial_one_bitwise(B):
    # an untimed solve of the tensor-core form runs the CUDA-core M2L levels
    # and the near zone's forward transform on the plan's own streams beside
    # the tensor-core levels; a stage-timed solve runs every stage in turn.
    # Same kernels on disjoint buffers: the results are equal bit for bit,
    # also for a second overlapped solve right after (the streams rejoin).
    N, L, p = 128, 4, 6
    rho = torch.from_numpy(inputs.lognormal(N, sigma=0.5, seed=21)).cuda()
    plan = B.Plan(N, L, p)
    plan.set_precision(B.FMM_PREC_BF16X3)
    B.fmm_plan_set_near_algorithm(plan.handle, B.FMM_NEAR_FFT)
    phi0, acc0 = plan.solve(rho)
    phi1, acc1 = plan.solve(rho)
    B.fmm_plan_set_timing(plan.handle, 1)
    phi2, acc2 = plan.solve(rho)
    torch.cuda.synchronize()
    assert B.lib().fmm_plan_check(plan.handle) == B.FMM_OK
    plan.close()
    for phi, acc in ((phi1, acc1), (phi2, acc2)):
        assert torch.equal(phi0, phi) and torch.equal(acc0, acc)
