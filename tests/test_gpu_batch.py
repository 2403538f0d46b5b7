"""Batches of uneven fields (one graph launch) and the tree-depth autotuner."""
import numpy as np
import pytest

from oracle import fmm as ofmm
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


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_leaf_size_six_matches_oracle(B):
    # N = 48 (S = 6), the uneven sizes of the batch workload
    N, L, p = 48, 3, 3
    rho = inputs.lognormal(N, sigma=0.8, seed=48)
    plan = B.Plan(N, L, p)
    phi, acc = plan.solve(torch.from_numpy(rho).cuda())
    ophi, og = ofmm.solve(rho, L, p)
    assert_close(phi.cpu().numpy(), ophi, 1e-6, "batch field phi")
    assert_close(acc.cpu().numpy(), og, 1e-6, "batch field g")


@pytest.mark.parametrize("prec", [0, 2])
def test_batch_equals_single_solves(B, prec):
    rng = np.random.default_rng(2)
    Ns = [32, 48, 64, 96, 32, 64, 48]
    ps = [4, 6, 4, 4, 6, 6, 4]
    Ls = [3, 3, 3, 4, 3, 3, 3]
    rhos = [inputs.lognormal(n, sigma=float(rng.uniform(0.3, 1.5)), seed=10 + i) for i, n in enumerate(Ns)]
    d = [torch.from_numpy(r).cuda() for r in rhos]
    pots = [torch.empty((n, n, n), device="cuda") for n in Ns]
    accs = [torch.empty((3, n, n, n), device="cuda") for n in Ns]
    batch = B.Batch(Ns, Ls, ps, precision=prec)
    for _ in range(2):                              # capture, then replay
        batch.solve(d, pots, accs)
    torch.cuda.synchronize()
    batch.check()
    for i in range(len(Ns)):
        plan = B.Plan(Ns[i], Ls[i], ps[i])
        if prec:
            plan.set_precision(prec)
        phi, acc = plan.solve(d[i])
        torch.cuda.synchronize()
        assert torch.equal(phi, pots[i]) and torch.equal(acc, accs[i]), i
        plan.close()
    batch.close()


def test_batch_with_near_fft_equals_single_solves(B):
    # fields with 8-cell leaves take the FFT near zone, the others keep the
    # direct sum; the captured batch equals the single solves bit for bit
    Ns = [32, 64, 48, 128, 64]
    ps = [4, 6, 6, 4, 3]
    Ls = [2, 3, 3, 4, 4]                            # S = 8, 8, 6, 8, 4
    rhos = [inputs.lognormal(n, sigma=0.7, seed=40 + i) for i, n in enumerate(Ns)]
    d = [torch.from_numpy(r).cuda() for r in rhos]
    pots = [torch.empty((n, n, n), device="cuda") for n in Ns]
    accs = [torch.empty((3, n, n, n), device="cuda") for n in Ns]
    batch = B.Batch(Ns, Ls, ps, precision=B.FMM_PREC_BF16X3)
    B.fmm_batch_set_near_algorithm(batch.handle, B.FMM_NEAR_FFT)
    for _ in range(2):                              # capture, then replay
        batch.solve(d, pots, accs)
    torch.cuda.synchronize()
    batch.check()
    for i in range(len(Ns)):
        plan = B.Plan(Ns[i], Ls[i], ps[i])
        plan.set_precision(B.FMM_PREC_BF16X3)
        if Ns[i] >> Ls[i] == 8:
            B.fmm_plan_set_near_algorithm(plan.handle, B.FMM_NEAR_FFT)
        phi, acc = plan.solve(d[i])
        torch.cuda.synchronize()
        assert torch.equal(phi, pots[i]) and torch.equal(acc, accs[i]), i
        plan.close()
    batch.close()


def test_autotuner_picks_a_valid_level_and_caches_it(B, tmp_path):
    cache = str(tmp_path / "tune.jsonl")
    L, ms = B.fmm_autotune_levels(64, 4, B.FMM_PREC_BF16X3, cache)
    assert L in (3, 4, 5) and ms > 0
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 1 and '"L": %d' % L in lines[0]
    L2, ms2 = B.fmm_autotune_levels(64, 4, B.FMM_PREC_BF16X3, cache)
    # the cache keeps the time with a few significant digits
    assert L2 == L and ms2 == pytest.approx(ms, rel=1e-3)
    assert len(open(cache).read().strip().splitlines()) == 1      # served from the cache


def test_batch_with_autotuned_levels(B, monkeypatch, tmp_path):
    monkeypatch.setenv("FMM_AUTOTUNE_CACHE", str(tmp_path / "tune.jsonl"))
    Ns, ps = [32, 48, 64], [4, 4, 6]
    batch = B.Batch(Ns, [0, 0, 0], ps)
    for n, l in zip(Ns, batch.levels):
        assert n % (1 << l) == 0 and l >= 3
    batch.close()
