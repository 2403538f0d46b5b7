"""The accuracy experiment of Sec. 3 on the GPU (eq. gerr, Table 1, Fig. eng).

The error of a periodic FMM solution against the PM solution with the same
Green's function has two parts: the multipole-expansion (ME) error and the
Green's-function (GF) error.  Sec. 3 estimates the first on the same problem
without periodic boundaries and subtracts it (eq. gerr):

    Delta g = | g_FMM^P - g_PM^P - (g_FMM^NP - g_PM^NP) |,

reported as L_MAX (maximum over cells) and L2 (root mean square over cells)
for unit total mass in the unit box, so the absolute error is a relative one.

Here the FMM solutions are libfmm solves (FMM_BOUNDARY_PERIODIC and
FMM_BOUNDARY_ISOLATED plans), and the PM solutions are FP64 FFT convolutions
(cuFFT through torch.fft) of the masses with the plan's own mesh Green's
function (fmm_plan_mesh_green): G_S1 (or G_S(a)) on the periodic N^3 mesh,
G_0 on the zero-padded (2N)^3 mesh.  Accelerations on the PM side are the
convolutions with -grad G, the limit the FMM converges to (the reading that
the 4th-order difference of Sec. 3 does not match an FMM whose near zone is
an exact direct sum).  This is the reference side of the experiment, not the
solve: the solves are the library's.
"""
import numpy as np

from . import binding as B


def point_sources(N, kind, seed=0, count=10):
    """Unit total mass: one cell (kind "corner": cell (0, 0, 0); "centre":
    cell (N/2, N/2, N/2)) or `count` cells drawn uniformly (seeded) with mass
    1/count each.  Returns rho (N, N, N) float32 with rho = N^3 x mass."""
    rho = np.zeros((N, N, N), dtype=np.float64)
    if kind == "corner":
        rho[0, 0, 0] = 1.0
    elif kind == "centre":
        rho[N // 2, N // 2, N // 2] = 1.0
    elif kind == "random":
        rng = np.random.Generator(np.random.PCG64(seed))
        cells = rng.choice(N ** 3, size=count, replace=False)
        rho.reshape(-1)[cells] += 1.0 / count
    else:
        raise ValueError(kind)
    return (rho * float(N) ** 3).astype(np.float32)


def pm_solution(plan, density, iso):
    """(phi, acc) of the PM method with the plan's Green's function, FP64."""
    import torch
    N = density.shape[0]
    M = 2 * N if iso else N
    K = torch.empty(4 * M ** 3, dtype=torch.float64, device=density.device)
    B.fmm_plan_mesh_green(plan.handle, K)
    m = density.double() / float(N) ** 3
    if not iso:
        m = m - m.mean()
    else:
        mp = torch.zeros((M, M, M), dtype=torch.float64, device=density.device)
        mp[:N, :N, :N] = m
        m = mp
    mh = torch.fft.rfftn(m)
    out = [torch.fft.irfftn(mh * torch.fft.rfftn(K[f * M ** 3:(f + 1) * M ** 3].view(M, M, M)), s=(M, M, M))
           [:N, :N, :N] for f in range(4)]
    return out[0], torch.stack(out[1:])


def _norms(d):
    mag = d.pow(2).sum(dim=0).sqrt()
    return float(mag.max()), float(mag.pow(2).mean().sqrt())


def gf_experiment(N, L, p, density, precision=B.FMM_PREC_FP32):
    """Eq. gerr for one source distribution (device density, unit mass):
    returns {"gf": (L_MAX, L2), "me": (L_MAX, L2), "p_vs_pm": (L_MAX, L2)}."""
    import torch
    g = {}
    for name, boundary in (("P", B.FMM_BOUNDARY_PERIODIC), ("NP", B.FMM_BOUNDARY_ISOLATED)):
        plan = B.Plan(N, L, p)
        B.fmm_plan_set_boundary(plan.handle, boundary)
        if precision != B.FMM_PREC_FP32:
            plan.set_precision(precision)
        _, acc = plan.solve(density)
        torch.cuda.synchronize()
        B.fmm_plan_check(plan.handle)
        _, pacc = pm_solution(plan, density, boundary == B.FMM_BOUNDARY_ISOLATED)
        g[name] = (acc.double(), pacc)
        plan.close()
    dp = g["P"][0] - g["P"][1]
    dnp = g["NP"][0] - g["NP"][1]
    return {"gf": _norms(dp - dnp), "me": _norms(dnp), "p_vs_pm": _norms(dp)}


def main():
    import argparse
    import json
    import torch
    ap = argparse.ArgumentParser(description="Sec. 3 accuracy experiment (eq. gerr) on the GPU")
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--L", type=int, default=3)
    ap.add_argument("--orders", default="4,6,8")
    args = ap.parse_args()
    dev = torch.device("cuda", 0)
    for p in [int(x) for x in args.orders.split(",")]:
        for kind in ("corner", "centre", "random"):
            d = torch.from_numpy(point_sources(args.n, kind, seed=7)).to(dev)
            r = gf_experiment(args.n, args.L, p, d)
            print(json.dumps({"N": args.n, "L": args.L, "p": p, "sources": kind, **r}), flush=True)


if __name__ == "__main__":
    main()
