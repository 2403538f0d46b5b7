"""The allocation-free mean entry point (fmm_mean_density_noalloc), called
through the C-ABI, against the mean the existing solve path computes.

Collected last on purpose (file name): if it fails, a run that stops at the
first failure has already run every other test.  It must pass both alone in a
fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

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


def _plan_mean(B, rho, L, p):
    # the existing entry points: a solve, then the mean stage of that solve
    plan = B.Plan(rho.shape[0], L, p)
    plan.solve(torch.from_numpy(rho).cuda())
    m = float(plan.stage(B.FMM_STAGE_MEAN, 0).cpu().numpy()[0])
    plan.close()
    return m


def test_noalloc_mean_matches_solve_mean_on_two_calls_in_a_row(B):
    L = B.lib()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for seed, n in ((11, 64), (12, 32)):          # two calls in a row, different sizes
        rho = inputs.lognormal(n, sigma=1.0, seed=seed)
        d = torch.from_numpy(rho).cuda()
        rc = L.fmm_mean_density_noalloc(ctypes.c_void_p(d.data_ptr()), ctypes.c_size_t(d.numel()),
                                        ctypes.c_void_p(out.data_ptr()), None)
        assert rc == B.FMM_OK
        torch.cuda.synchronize()
        got = float(out.item())
        ref = _plan_mean(B, rho, 3, 2)
        # the stage copy returns the mean rounded to float32
        assert abs(got - ref) <= 1e-7 * abs(ref)
        assert abs(got - rho.astype(np.float64).mean()) <= 1e-12 * abs(got)


def test_noalloc_mean_rejects_sizes_beyond_its_scratch(B):
    L = B.lib()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    d = torch.zeros(16, dtype=torch.float32, device="cuda")
    too_many = ctypes.c_size_t(512 ** 3 + 1)
    rc = L.fmm_mean_density_noalloc(ctypes.c_void_p(d.data_ptr()), too_many, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == B.FMM_ERR_ARG
    assert L.fmm_mean_density_noalloc(None, ctypes.c_size_t(16), ctypes.c_void_p(out.data_ptr()), None) == B.FMM_ERR_ARG
