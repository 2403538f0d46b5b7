"""Training of the learned M2L table correction on the GPU.

Sec. 4 suggests going beyond the analytic G_S1 by giving the Green's function
many free parameters and fitting them so that the FMM reproduces the PM
solution; here those parameters are the weights of a small MLP that corrects
the tabulated G_S1 (see include/fmm.h, "learned table correction").  The
target of each training field is PM with G_S1 (the paper's definition of the
optimal G_*: PM and FMM agree).  Every step runs in libfmm's kernels: the
forward solve, the adjoint sweep, the table gradient, the MLP backward pass
and Adam (fmm_correction_grad, fmm_adam_step); the PM targets use libfmm's
mesh Green's function and cuFFT through torch.fft.

    python -m paper_2011_07099_gb300.learn --fields 256 --n 64 --L 3 --p 6 --steps 200 --out corr.npz
"""
import argparse
import json
import os
import time

import numpy as np

from . import binding as B
from . import inputs


DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")


def shipped_weights(p):
    """The trained correction weights shipped with the package for order p
    (float32 array of FMM_MLP_PARAMS values), or None if there are none."""
    path = os.path.join(DATA, f"correction_p{p}.npz")
    if not os.path.exists(path):
        return None
    with np.load(path) as z:
        return np.asarray(z["w"], dtype=np.float32)


def pm_target(density, N):
    """PM with G_S1 on the GPU: circular convolution of the mean-free masses
    with libfmm's mesh Green's function (FP64 FFTs).  Returns (phi, acc)."""
    import torch
    K = torch.empty(4 * N ** 3, dtype=torch.float32, device=density.device)
    B.fmm_mesh_green(N, K)
    torch.cuda.synchronize(density.device)
    m = density.double()
    m = (m - m.mean()) / float(N) ** 3
    mh = torch.fft.rfftn(m)
    outs = [torch.fft.irfftn(mh * torch.fft.rfftn(K[f * N ** 3:(f + 1) * N ** 3].view(N, N, N).double()),
                             s=(N, N, N)) for f in range(4)]
    return outs[0].float().contiguous(), torch.stack(outs[1:]).float().contiguous()


def pm_target_gk(density, N):
    """PM with the exact-in-Fourier-space G_K (Sec. 1, eq. gfk): spectral
    solve of lap Phi = m on the mesh, g = -grad Phi spectrally (the Nyquist
    derivative zeroed), FP64 FFTs.  Returns (phi, acc) like pm_target."""
    import torch
    m = density.double()
    m = (m - m.mean()) / float(N) ** 3
    f = torch.fft.fftfreq(N, d=1.0 / N, dtype=torch.float64, device=density.device)
    fz = torch.fft.rfftfreq(N, d=1.0 / N, dtype=torch.float64, device=density.device)
    kz, ky, kx = torch.meshgrid(f, f, fz, indexing="ij")
    k2 = (2 * np.pi) ** 2 * (kx * kx + ky * ky + kz * kz)
    gt = torch.where(k2 > 0, -1.0 / torch.where(k2 > 0, k2, torch.ones_like(k2)), torch.zeros_like(k2))
    phih = torch.fft.rfftn(m) * gt * float(N) ** 3
    phi = torch.fft.irfftn(phih, s=(N, N, N))
    nyq = N // 2 if N % 2 == 0 else None
    derivs = []
    for k in (kx, ky, kz):
        kk = k.clone()
        if nyq is not None:
            kk[kk.abs() == nyq] = 0.0
        derivs.append(torch.fft.irfftn(-2j * np.pi * kk * phih, s=(N, N, N)))
    return phi.float().contiguous(), torch.stack(derivs).float().contiguous()


def init_weights(seed):
    """Hidden layers ~ N(0, 1/fan_in), biases 0, output layer 0: the initial
    correction is exactly zero (the plain G_S1 table)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    H, I = 64, 5
    parts = [rng.normal(0.0, 1.0 / np.sqrt(I), (H, I)), np.zeros(H),
             rng.normal(0.0, 1.0 / np.sqrt(H), (H, H)), np.zeros(H),
             rng.normal(0.0, 1.0 / np.sqrt(H), (H, H)), np.zeros(H),
             np.zeros(H), np.zeros(1)]
    w = np.concatenate([x.ravel() for x in parts]).astype(np.float32)
    assert w.size == B.FMM_MLP_PARAMS
    return w


class Trainer:
    """Adam on the parameters of a table model; state = (params, m, v, step).

    model = "mlp": the learned correction's network weights
    (fmm_plan_set_correction / fmm_correction_grad); model = "grid": the grid
    model of G_* of Sec. 4, one value per folded table entry and field
    (fmm_plan_set_table_grid / fmm_table_grid_grad), starting at zero (the
    plain G_S1 tables)."""

    def __init__(self, N, L, p, seed=0, lr=1e-3, device="cuda", model="mlp"):
        import torch
        self.N, self.L, self.p, self.lr, self.model = N, L, p, lr, model
        self.device = torch.device(device)
        self.plan = B.Plan(N, L, p)
        if model == "mlp":
            B.fmm_plan_set_correction_inference(self.plan.handle, B.FMM_INFER_FP32)
            self.w = torch.from_numpy(init_weights(seed)).to(self.device)
        elif model == "grid":
            self.w = torch.zeros(B.fmm_plan_table_grid_size(self.plan.handle), dtype=torch.float32,
                                 device=self.device)
        else:
            raise ValueError(model)
        self.m = torch.zeros_like(self.w)
        self.v = torch.zeros_like(self.w)
        self.grad = torch.zeros_like(self.w)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.step_count = 0
        self._apply()

    def _apply(self):
        if self.model == "mlp":
            B.fmm_plan_set_correction(self.plan.handle, self.w)
        else:
            B.fmm_plan_set_table_grid(self.plan.handle, self.w)

    def prepare(self, density_np, target="gs1"):
        """Device density, PM target (PM with G_S1, or with G_K for
        target="gk") and the relative-error weights of a field."""
        import torch
        d = torch.from_numpy(np.ascontiguousarray(density_np, dtype=np.float32)).to(self.device)
        tphi, tacc = (pm_target_gk if target == "gk" else pm_target)(d, self.N)
        w_phi = 1.0 / float((tphi.double() ** 2).sum())
        w_g = 1.0 / float((tacc.double() ** 2).sum())
        return d, tphi, tacc, w_phi, w_g

    def step(self, batch):
        """One Adam step over the fields of `batch` (prepared tuples); returns
        the mean loss before the update."""
        self.grad.zero_()
        self.loss.zero_()
        grad_fn = B.fmm_correction_grad if self.model == "mlp" else B.fmm_table_grid_grad
        for d, tphi, tacc, w_phi, w_g in batch:
            grad_fn(self.plan.handle, d, tphi, tacc, w_phi, w_g, self.grad, self.loss)
        self.grad /= len(batch)
        self.step_count += 1
        B.fmm_adam_step(self.w, self.grad, self.m, self.v, self.step_count, self.lr)
        self._apply()
        return float(self.loss.item()) / len(batch)

    def state(self):
        return {"w": self.w.cpu().numpy(), "m": self.m.cpu().numpy(), "v": self.v.cpu().numpy(),
                "step": np.array(self.step_count)}

    def save(self, path):
        np.savez(path, **self.state())

    def load(self, path):
        import torch
        z = np.load(path)
        self.w.copy_(torch.from_numpy(z["w"]))
        self.m.copy_(torch.from_numpy(z["m"]))
        self.v.copy_(torch.from_numpy(z["v"]))
        self.step_count = int(z["step"])
        self._apply()


def relative_errors(plan, d, tphi, tacc):
    """(relative L2 of Phi, of g) of a solve against the target."""
    phi, acc = plan.solve(d)
    e1 = float(((phi.double() - tphi.double()) ** 2).sum().sqrt() / (tphi.double() ** 2).sum().sqrt())
    e2 = float(((acc.double() - tacc.double()) ** 2).sum().sqrt() / (tacc.double() ** 2).sum().sqrt())
    return e1, e2


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--fields", type=int, default=256)
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--L", type=int, default=3)
    ap.add_argument("--p", type=int, default=6)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=3000)
    ap.add_argument("--out", default="correction.npz")
    ap.add_argument("--resume", default=None)
    ap.add_argument("--model", choices=["mlp", "grid"], default="mlp")
    ap.add_argument("--target", choices=["gs1", "gk"], default="gs1",
                    help="PM reference of the loss: with G_S1 (the paper's G_* definition) or with G_K")
    args = ap.parse_args()
    tr = Trainer(args.n, args.L, args.p, seed=args.seed, lr=args.lr, model=args.model)
    if args.resume:
        tr.load(args.resume)
    fields = [tr.prepare(inputs.lognormal(args.n, sigma=0.5, seed=args.seed + i), args.target)
              for i in range(args.fields)]
    t0 = time.time()
    for s in range(tr.step_count, args.steps):
        i0 = (s * args.batch) % len(fields)
        batch = [fields[(i0 + k) % len(fields)] for k in range(args.batch)]
        loss = tr.step(batch)
        if s % 10 == 0:
            print(json.dumps({"step": s, "loss": loss, "elapsed_s": time.time() - t0}), flush=True)
    tr.save(args.out)


if __name__ == "__main__":
    main()
