"""The learned table correction on the GPU: its gradient against FP64 finite
differences of the oracle, and what training it gains."""
import numpy as np
import pytest

from oracle import fmm as ofmm
from oracle import learn as olearn
from paper_2011_07099_gb300 import inputs
from parity_util import assert_close, corner_and_interior_leaves, leaf_values

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


def _random_weights(seed):
    rng = np.random.default_rng(seed)
    w = rng.normal(0.0, 0.4, olearn.N_PARAMS)
    return w


def test_gpu_gradient_matches_oracle_finite_differences(B):
    N, L, p = 16, 3, 2
    rho = inputs.lognormal(N, sigma=0.8, seed=21)
    w = _random_weights(5).astype(np.float32).astype(np.float64)
    tphi, tg = olearn.pm_target(rho)
    w_phi, w_g = 1.0 / np.sum(tphi ** 2), 1.0 / np.sum(tg ** 2)
    # GPU: FP32 inference, FP32 solve, adjoint gradient
    plan = B.Plan(N, L, p)
    B.fmm_plan_set_correction_inference(plan.handle, B.FMM_INFER_FP32)
    wd = torch.from_numpy(w.astype(np.float32)).cuda()
    B.fmm_plan_set_correction(plan.handle, wd)
    d = torch.from_numpy(rho).cuda()
    tp = torch.from_numpy(tphi.astype(np.float32)).cuda()
    ta = torch.from_numpy(tg.astype(np.float32)).contiguous().cuda()
    grad = torch.zeros(B.FMM_MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    B.fmm_correction_grad(plan.handle, d, tp, ta, w_phi, w_g, grad, loss)
    torch.cuda.synchronize()
    g_gpu = grad.cpu().numpy().astype(np.float64)
    j_oracle = olearn.loss(w, rho, L, p, tphi, tg, w_phi, w_g)
    assert abs(float(loss.item()) - j_oracle) <= 1e-3 * j_oracle
    # FP64 central differences of the oracle loss on parameters of every layer
    idx = [3, 200, 330, 400, 2000, 4455, 4500, 6000, 8600, 8650, 8700, 8768]
    for i in idx:
        h = 1e-3 * max(1.0, abs(w[i]))
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (olearn.loss(wp, rho, L, p, tphi, tg, w_phi, w_g) - olearn.loss(wm, rho, L, p, tphi, tg, w_phi, w_g)) / (2 * h)
        scale = max(abs(fd), 1e-3 * np.abs(g_gpu).max())
        assert abs(g_gpu[i] - fd) <= 2e-2 * scale, (i, g_gpu[i], fd)
    plan.close()


def test_training_reduces_the_fmm_vs_pm_error_on_held_out_fields(B):
    from paper_2011_07099_gb300 import learn
    N, L, p = 32, 3, 4
    tr = learn.Trainer(N, L, p, seed=7, lr=2e-3)
    train = [tr.prepare(inputs.lognormal(N, sigma=0.5, seed=100 + i)) for i in range(8)]
    held = [tr.prepare(inputs.lognormal(N, sigma=0.5, seed=900 + i)) for i in range(4)]
    plain = B.Plan(N, L, p)

    def mean_err(plan):
        e = [learn.relative_errors(plan, *f[:3]) for f in held]
        return np.mean([x[0] for x in e]), np.mean([x[1] for x in e])

    before = mean_err(plain)
    losses = [tr.step(train) for _ in range(120)]
    after = mean_err(tr.plan)
    print(f"held-out relative L2 vs PM(G_S1): plain phi {before[0]:.3e} g {before[1]:.3e} | "
          f"learned phi {after[0]:.3e} g {after[1]:.3e} | loss {losses[0]:.3e} -> {losses[-1]:.3e}")
    assert losses[-1] < losses[0]
    # the learned table gains on fields it never saw (combined relative error);
    # at p = 4 the multipole-truncation part, which no table can remove,
    # dominates the error, so the gain is modest
    assert after[0] ** 2 + after[1] ** 2 < 0.99 * (before[0] ** 2 + before[1] ** 2)
    plain.close()


def test_checkpoint_resume_reproduces_uninterrupted_training(B, tmp_path):
    from paper_2011_07099_gb300 import learn
    N, L, p = 16, 3, 2
    fields_np = [inputs.lognormal(N, sigma=0.5, seed=300 + i) for i in range(2)]
    a = learn.Trainer(N, L, p, seed=1)
    fa = [a.prepare(x) for x in fields_np]
    for _ in range(4):
        a.step(fa)
    b = learn.Trainer(N, L, p, seed=1)
    fb = [b.prepare(x) for x in fields_np]
    for _ in range(2):
        b.step(fb)
    b.save(str(tmp_path / "ck.npz"))
    c = learn.Trainer(N, L, p, seed=99)
    c.load(str(tmp_path / "ck.npz"))
    fc = [c.prepare(x) for x in fields_np]
    for _ in range(2):
        c.step(fc)
    np.testing.assert_allclose(c.w.cpu().numpy(), a.w.cpu().numpy(), rtol=1e-5, atol=1e-7)


def test_bf16_inference_close_to_fp32_inference(B):
    N, L, p = 32, 3, 4
    rho = inputs.lognormal(N, sigma=0.5, seed=8)
    w = torch.from_numpy(_random_weights(9).astype(np.float32)).cuda()
    d = torch.from_numpy(rho).cuda()
    out = []
    for mode in (B.FMM_INFER_FP32, B.FMM_INFER_BF16):
        plan = B.Plan(N, L, p)
        B.fmm_plan_set_correction_inference(plan.handle, mode)
        B.fmm_plan_set_correction(plan.handle, w)
        phi, acc = plan.solve(d)
        out.append((phi.cpu().numpy(), acc.cpu().numpy()))
        plan.close()
    plain = B.Plan(N, L, p)
    phi0, acc0 = plain.solve(d)
    corr_size = np.linalg.norm(out[0][0] - phi0.cpu().numpy())
    assert corr_size > 0
    # BF16 inference perturbs the correction by ~2^-8 of its size
    assert np.linalg.norm(out[1][0] - out[0][0]) <= 2e-2 * corr_size


@pytest.mark.parametrize("N,L,p", [(32, 3, 4), (64, 3, 6), (32, 5, 2)])
def test_corrected_fp32_solve_matches_oracle_element_by_element(B, N, L, p):
    # the forward solve with a (random, non-negligible) table correction, FP32
    # inference and the plain FP32 form, against the oracle's FMM with the
    # FP64 network evaluated at every n = o p + r - s of eq. fmm2
    rho = inputs.lognormal(N, sigma=0.5, seed=40 + N + p)
    w = _random_weights(11).astype(np.float32).astype(np.float64)
    plan = B.Plan(N, L, p)
    B.fmm_plan_set_correction_inference(plan.handle, B.FMM_INFER_FP32)
    B.fmm_plan_set_correction(plan.handle, torch.from_numpy(w.astype(np.float32)).cuda())
    phi, acc = plan.solve(torch.from_numpy(rho).cuda())
    torch.cuda.synchronize()
    plan.close()
    ophi, og = ofmm.solve(rho, L, p, correction=olearn.correction_fn(w))
    plain_phi, plain_g = ofmm.solve(rho, L, p)
    # the correction moves the solution far beyond the tolerance ...
    assert np.linalg.norm(plain_phi - ophi) > 1e-4 * np.linalg.norm(ophi)
    # ... and the GPU follows the oracle element by element
    assert_close(phi.cpu().numpy(), ophi, 1e-6, f"corrected phi {N}^3 L={L} p={p}")
    assert_close(acc.cpu().numpy(), og, 1e-6, f"corrected g {N}^3 L={L} p={p}")


def test_headline_form_with_shipped_weights_matches_oracle_at_sampled_leaves(B):
    # exactly the form the bench times at 256^3 p = 6: bf16x3 tensor-core M2L,
    # the shipped order-6 correction with BF16 inference, against the oracle's
    # FMM with the same weights (FP64 network) at the 8 corner leaves and 2
    # interior ones.  Bound: the bf16x3 tolerance 2e-5; BF16 inference
    # perturbs the correction by ~2^-8 of its size, and the correction itself
    # moves these fields by well under 1e-3, so its share is below 1e-5.
    from paper_2011_07099_gb300 import learn
    N, L, p = 256, 5, 6
    w = learn.shipped_weights(p)
    assert w is not None
    rho = inputs.config_density(5, n=N)
    plan = B.Plan(N, L, p)
    plan.set_precision(B.FMM_PREC_BF16X3)
    B.fmm_plan_set_correction(plan.handle, torch.from_numpy(w.astype(np.float32)).cuda())
    phi, acc = plan.solve(torch.from_numpy(rho).cuda())
    torch.cuda.synchronize()
    assert B.lib().fmm_plan_check(plan.handle) == B.FMM_OK
    plan.close()
    leaves = corner_and_interior_leaves(L, 2, seed=66)
    ref = ofmm.solve_at(rho, L, p, leaves, correction=olearn.correction_fn(w.astype(np.float64)))
    got = leaf_values(phi.cpu().numpy(), acc.cpu().numpy(), leaves, N >> L)
    assert_close(got[:, 0], ref[:, 0], 2e-5, "headline form phi, sampled leaves")
    assert_close(got[:, 1:], ref[:, 1:], 2e-5, "headline form g, sampled leaves")


# ------------------------------------------------------- grid model of G_*
def test_grid_model_forward_matches_oracle_element_by_element(B):
    N, L, p = 32, 3, 4
    rho = inputs.lognormal(N, sigma=0.5, seed=77)
    n = olearn.grid_size(L, p)
    theta = np.random.default_rng(3).normal(0.0, 0.5, n).astype(np.float32).astype(np.float64)
    plan = B.Plan(N, L, p)
    assert B.fmm_plan_table_grid_size(plan.handle) == n
    B.fmm_plan_set_table_grid(plan.handle, torch.from_numpy(theta.astype(np.float32)).cuda())
    phi, acc = plan.solve(torch.from_numpy(rho).cuda())
    torch.cuda.synchronize()
    plan.close()
    ophi, og = ofmm.solve(rho, L, p, correction=olearn.grid_correction_fn(theta))
    plain_phi, _ = ofmm.solve(rho, L, p)
    assert np.linalg.norm(plain_phi - ophi) > 1e-4 * np.linalg.norm(ophi)
    assert_close(phi.cpu().numpy(), ophi, 1e-6, "grid model phi")
    assert_close(acc.cpu().numpy(), og, 1e-6, "grid model g")


def test_grid_model_gradient_matches_oracle_finite_differences(B):
    N, L, p = 16, 3, 2
    rho = inputs.lognormal(N, sigma=0.8, seed=22)
    n = olearn.grid_size(L, p)
    theta = np.random.default_rng(4).normal(0.0, 0.2, n).astype(np.float32).astype(np.float64)
    tphi, tg = olearn.pm_target(rho)
    w_phi, w_g = 1.0 / np.sum(tphi ** 2), 1.0 / np.sum(tg ** 2)
    plan = B.Plan(N, L, p)
    B.fmm_plan_set_table_grid(plan.handle, torch.from_numpy(theta.astype(np.float32)).cuda())
    d = torch.from_numpy(rho).cuda()
    tp = torch.from_numpy(tphi.astype(np.float32)).cuda()
    ta = torch.from_numpy(tg.astype(np.float32)).contiguous().cuda()
    grad = torch.zeros(n, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    B.fmm_table_grid_grad(plan.handle, d, tp, ta, w_phi, w_g, grad, loss)
    torch.cuda.synchronize()
    g_gpu = grad.cpu().numpy().astype(np.float64)
    plan.close()
    j = olearn.grid_loss(theta, rho, L, p, tphi, tg, w_phi, w_g)
    assert abs(float(loss.item()) - j) <= 1e-3 * j
    # entries with the largest gradients on every level and field, plus a few others
    G3 = (4 * p) ** 3
    idx = []
    for lev in range(L - 1):
        for f in range(4):
            blk = slice((lev * 4 + f) * G3, (lev * 4 + f + 1) * G3)
            idx.append(blk.start + int(np.argmax(np.abs(g_gpu[blk]))))
    idx += [5, n // 2 + 3]
    for i in idx:
        h = 1e-3
        tp_, tm_ = theta.copy(), theta.copy()
        tp_[i] += h
        tm_[i] -= h
        fd = (olearn.grid_loss(tp_, rho, L, p, tphi, tg, w_phi, w_g)
              - olearn.grid_loss(tm_, rho, L, p, tphi, tg, w_phi, w_g)) / (2 * h)
        scale = max(abs(fd), 1e-3 * np.abs(g_gpu).max())
        assert abs(g_gpu[i] - fd) <= 2e-2 * scale, (i, g_gpu[i], fd)


def test_grid_model_training_gains_on_held_out_fields(B):
    # Sec. 4's grid model trained against PM(G_S1) on seeded fields; its
    # held-out error is compared with the plain tables (and printed beside the
    # network's from the same fields and steps)
    from paper_2011_07099_gb300 import learn
    N, L, p = 32, 3, 4
    train_np = [inputs.lognormal(N, sigma=0.5, seed=100 + i) for i in range(8)]
    held_np = [inputs.lognormal(N, sigma=0.5, seed=900 + i) for i in range(4)]
    plain = B.Plan(N, L, p)
    res = {}
    for model, lr in (("grid", 2e-2), ("mlp", 2e-3)):
        tr = learn.Trainer(N, L, p, seed=7, lr=lr, model=model)
        train = [tr.prepare(x) for x in train_np]
        held = [tr.prepare(x) for x in held_np]
        before = np.mean([learn.relative_errors(plain, *f[:3]) for f in held], axis=0)
        losses = [tr.step(train) for _ in range(120)]
        after = np.mean([learn.relative_errors(tr.plan, *f[:3]) for f in held], axis=0)
        res[model] = (before, after, losses[0], losses[-1])
        print(f"{model}: held-out vs PM(G_S1) plain phi {before[0]:.3e} g {before[1]:.3e} -> "
              f"phi {after[0]:.3e} g {after[1]:.3e}; loss {losses[0]:.3e} -> {losses[-1]:.3e}")
    before, after, l0, l1 = res["grid"]
    assert l1 < l0
    assert after[0] ** 2 + after[1] ** 2 < 0.99 * (before[0] ** 2 + before[1] ** 2)
    plain.close()


def test_training_against_pm_gk_gains_on_held_out_fields(B):
    # the learned correction trained against PM with G_K (the target the
    # learned form names) on seeded fields: the held-out mismatch of Phi
    # (mean removed: PM(G_K) has no k = 0 mode) and of g falls.  The near
    # zone keeps G_S1 exactly (Sec. 3: it must match PM near the sources), so
    # the tables cannot remove the whole G_K mismatch of g.
    from paper_2011_07099_gb300 import learn
    N, L, p = 32, 3, 4
    tr = learn.Trainer(N, L, p, seed=7, lr=2e-3, model="mlp")
    train = [tr.prepare(inputs.lognormal(N, sigma=0.5, seed=100 + i), "gk") for i in range(8)]
    held = [tr.prepare(inputs.lognormal(N, sigma=0.5, seed=900 + i), "gk") for i in range(4)]
    plain = B.Plan(N, L, p)

    def errs(plan):
        out = []
        for d, tphi, tacc, _, _ in held:
            phi, acc = plan.solve(d)
            a, b = (phi - phi.mean()).double(), (tphi - tphi.mean()).double()
            out.append((float(((a - b) ** 2).sum().sqrt() / (b ** 2).sum().sqrt()),
                        float(((acc.double() - tacc.double()) ** 2).sum().sqrt() / (tacc.double() ** 2).sum().sqrt())))
        return np.mean(out, axis=0)

    before = errs(plain)
    losses = [tr.step(train) for _ in range(120)]
    after = errs(tr.plan)
    print(f"vs PM(G_K) held out: phi {before[0]:.3e} -> {after[0]:.3e}, g {before[1]:.3e} -> {after[1]:.3e}; "
          f"loss {losses[0]:.3e} -> {losses[-1]:.3e}")
    assert losses[-1] < 0.7 * losses[0]
    assert after[0] < 0.8 * before[0] and after[1] < before[1]
    plain.close()
    tr.plan.close()
