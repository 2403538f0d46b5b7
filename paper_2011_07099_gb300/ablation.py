"""Green's-function ablation (Sec. 3, Fig. errex): the FMM against the PM
solution with the same Green's function, for G_S1, the exact-in-real-space
G_X (eq. gfx) and the exact-in-Fourier-space G_K (eq. gfk).

The optimal G_* of Sec. 3 is the function with which PM and FMM agree; G_X is
a valid periodic Green's function whose kink at half the box aliases in the
FMM's interpolation (the >100% errors of Fig. errex), G_K is the PM's own
function, and G_S1 is the paper's approximation of G_*.  G_K has no closed
real-space form: its values on the N^3 mesh (and those of -grad G_K) come
from an FP64 inverse FFT of -1/k^2 (k = 2 pi n, zero at k = 0, the Nyquist
derivative zeroed as in the spectral PM) and are handed to the plan with
fmm_plan_set_green_mesh, which needs the gridlets on the mesh (S a multiple
of p).  The PM references use the plan's own mesh function
(fmm_plan_mesh_green) with cuFFT; the solves are libfmm's.
"""
import numpy as np

from . import binding as B


def g_k_mesh(N, device):
    """(4 N^3,) float64 on `device`: G_K and -grad G_K at the offsets d/N,
    G_K(d/N) = sum_n Gt(n) exp(2 pi i n.d/N), Gt = -1/(2 pi n)^2, Gt(0) = 0."""
    import torch
    f = torch.fft.fftfreq(N, d=1.0 / N, dtype=torch.float64, device=device)
    kz, ky, kx = torch.meshgrid(f, f, f, indexing="ij")
    k2 = (2 * np.pi) ** 2 * (kx * kx + ky * ky + kz * kz)
    gt = torch.where(k2 > 0, -1.0 / torch.where(k2 > 0, k2, torch.ones_like(k2)), torch.zeros_like(k2))
    fd = f.clone()
    if N % 2 == 0:
        fd[N // 2] = 0.0
    dz, dy, dx = torch.meshgrid(fd, fd, fd, indexing="ij")
    out = [torch.fft.ifftn(gt).real * N ** 3]
    for k in (dx, dy, dz):
        # -dG/dx_i = sum Gt (-2 pi i n_i) exp(...)
        out.append(torch.fft.ifftn(gt * (-2j * np.pi) * k).real * N ** 3)
    return torch.stack(out).reshape(-1).contiguous()


def make_plan(N, L, p, green, device):
    """A periodic plan with the named Green's function ("S1", "X" or "K")."""
    plan = B.Plan(N, L, p)
    if green == "X":
        B.fmm_plan_set_green(plan.handle, B.FMM_GREEN_X)
    elif green == "K":
        B.fmm_plan_set_green_mesh(plan.handle, g_k_mesh(N, device))
    elif green != "S1":
        raise ValueError(green)
    return plan


def fmm_vs_pm(N, L, p, density, green):
    """Relative L2 (Phi, g) and absolute (L_MAX, L2) of |dg| of the FMM with
    `green` against PM with the same function."""
    import torch
    from . import accuracy
    plan = make_plan(N, L, p, green, density.device)
    phi, acc = plan.solve(density)
    torch.cuda.synchronize()
    B.fmm_plan_check(plan.handle)
    pphi, pacc = accuracy.pm_solution(plan, density, False)
    plan.close()
    dphi = phi.double() - pphi
    dphi = dphi - dphi.mean()          # Phi is defined up to a constant
    pphi0 = pphi - pphi.mean()
    dg = acc.double() - pacc
    mag = dg.pow(2).sum(dim=0).sqrt()
    return {"rel_phi": float(dphi.norm() / pphi0.norm()), "rel_g": float(dg.norm() / pacc.norm()),
            "abs_g": (float(mag.max()), float(mag.pow(2).mean().sqrt()))}


def m2l_forms(N, L, p, density, steps=5):
    """Per-solve time of the M2L stage (CUDA events, median of `steps` after
    one warm-up) for the dense FP32 form, the dense bf16x3 tensor-core form
    and the FFT form of the interaction zone (Sec. 2), with each form's
    relative L2 difference from the dense FP32 solve."""
    import statistics
    import torch
    out = {}
    ref = None
    for name, prec, alg in (("dense_fp32", B.FMM_PREC_FP32, B.FMM_M2L_DENSE),
                            ("dense_bf16x3", B.FMM_PREC_BF16X3, B.FMM_M2L_DENSE),
                            ("fft_fp32", B.FMM_PREC_FP32, B.FMM_M2L_FFT)):
        plan = B.Plan(N, L, p)
        if prec != B.FMM_PREC_FP32:
            plan.set_precision(prec)
        B.fmm_plan_set_m2l_algorithm(plan.handle, alg)
        phi, acc = plan.solve(density)
        B.fmm_plan_set_timing(plan.handle, True)
        m2l, lev = [], []
        for _ in range(steps):
            plan.solve(density, phi, acc)
            t = B.fmm_plan_stage_times(plan.handle)
            m2l.append(t[B.FMM_TIME_M2L])
            lev.append([t[B.FMM_TIME_M2L_LEVEL0 + l] for l in range(2, L + 1)])
        torch.cuda.synchronize()
        B.fmm_plan_check(plan.handle)
        if ref is None:
            ref = (phi.clone(), acc.clone())
        out[name] = {"m2l_ms": statistics.median(m2l),
                     "level_ms": [statistics.median(x[i] for x in lev) for i in range(L - 1)],
                     "rel_phi_vs_dense_fp32": float((phi - ref[0]).norm() / ref[0].norm()),
                     "rel_g_vs_dense_fp32": float((acc - ref[1]).norm() / ref[1].norm())}
        plan.close()
    return out


def main():
    import argparse
    import json
    import torch
    from . import accuracy
    ap = argparse.ArgumentParser(description="FMM vs PM with G_S1, G_X and G_K (Fig. errex)")
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--L", type=int, default=3)
    ap.add_argument("--p", type=int, default=8)
    ap.add_argument("--m2l", action="store_true", help="time the dense and FFT forms of M2L instead")
    args = ap.parse_args()
    if args.m2l:
        from . import inputs
        d = torch.from_numpy(inputs.lognormal(args.n, sigma=0.5, seed=5000)).cuda()
        print(json.dumps({"N": args.n, "L": args.L, "p": args.p, **m2l_forms(args.n, args.L, args.p, d)}), flush=True)
        return
    d = torch.from_numpy(accuracy.point_sources(args.n, "corner")).cuda()
    for g in ("S1", "X", "K"):
        print(json.dumps({"N": args.n, "L": args.L, "p": args.p, "green": g, **fmm_vs_pm(args.n, args.L, args.p, d, g)}),
              flush=True)


if __name__ == "__main__":
    main()
