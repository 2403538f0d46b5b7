"""Fit of the coefficients a_k of the G_S ansatz (Sec. 3, Table 1) with the
GPU solver as the objective.

Sec. 3 parameterises the optimal Green's function as G_S with
    xi_n(t) = sin(pi t)/pi + sum_k a_k (sin((2k+1) pi t)/((2k+1) pi) - sin(pi t)/pi)
and finds a_k by minimising a norm of the difference between the PM and the
FMM accelerations, both computed with G_S (the error of Fig. errex, right
panel), for a unit point source; L2 with a Hessian-based minimiser, L_MAX
with the downhill simplex (Nelder and Mead 1965).  Here every objective
evaluation re-tabulates a libfmm plan with FMM_GREEN_S(a) (fmm_plan_set_green),
solves on the GPU, and compares with the FP64 PM solution on the same mesh
Green's function (fmm_plan_mesh_green, cuFFT); the minimiser is the downhill
simplex written below.  Optionally the objective is eq. gerr instead (the
non-periodic expansion error subtracted, computed once since it does not
depend on a_k).
"""
import numpy as np

from . import binding as B


def nelder_mead(f, x0, step, xtol=1e-6, ftol=1e-12, max_iter=200):
    """Downhill simplex minimisation of f: R^n -> R (Nelder and Mead 1965),
    with the usual coefficients: reflection 1, expansion 2, contraction 1/2,
    shrink 1/2.  The initial simplex is x0 and x0 + step e_i.  Stops when the
    simplex's extent in x is below xtol and the spread of its values below
    ftol, or after max_iter iterations.  Returns (x_best, f_best, evaluations)."""
    x0 = np.asarray(x0, dtype=np.float64)
    n = x0.size
    pts = [x0.copy()]
    for i in range(n):
        x = x0.copy()
        x[i] += step[i] if np.ndim(step) else step
        pts.append(x)
    vals = [f(x) for x in pts]
    evals = n + 1
    for _ in range(max_iter):
        order = np.argsort(vals)
        pts = [pts[i] for i in order]
        vals = [vals[i] for i in order]
        extent = max(np.max(np.abs(p - pts[0])) for p in pts[1:])
        if extent < xtol and vals[-1] - vals[0] <= ftol:
            break
        centroid = np.mean(pts[:-1], axis=0)
        xr = centroid + (centroid - pts[-1])
        fr = f(xr)
        evals += 1
        if fr < vals[0]:
            xe = centroid + 2.0 * (centroid - pts[-1])
            fe = f(xe)
            evals += 1
            pts[-1], vals[-1] = (xe, fe) if fe < fr else (xr, fr)
        elif fr < vals[-2]:
            pts[-1], vals[-1] = xr, fr
        else:
            outside = fr < vals[-1]
            xc = centroid + 0.5 * ((xr if outside else pts[-1]) - centroid)
            fc = f(xc)
            evals += 1
            if fc < (fr if outside else vals[-1]):
                pts[-1], vals[-1] = xc, fc
            else:
                for i in range(1, n + 1):
                    pts[i] = pts[0] + 0.5 * (pts[i] - pts[0])
                    vals[i] = f(pts[i])
                    evals += 1
    i = int(np.argmin(vals))
    return pts[i], float(vals[i]), evals


class AnsatzObjective:
    """Error norm of the periodic FMM against PM, both with G_S(a), for one
    source distribution on the GPU.  norm: "l2" (root mean square of |dg|
    over cells) or "lmax"; gerr=True subtracts the non-periodic expansion
    error cell by cell first (eq. gerr)."""

    def __init__(self, N, L, p, density, norm="l2", gerr=False):
        import torch
        from . import accuracy
        self.N, self.L, self.p, self.norm = N, L, p, norm
        self.density = density
        self.plan = B.Plan(N, L, p)
        self.phi = torch.empty((N, N, N), dtype=torch.float32, device=density.device)
        self.acc = torch.empty((3, N, N, N), dtype=torch.float32, device=density.device)
        self.np_err = None
        if gerr:
            iso = B.Plan(N, L, p)
            B.fmm_plan_set_boundary(iso.handle, B.FMM_BOUNDARY_ISOLATED)
            _, acc = iso.solve(density)
            torch.cuda.synchronize()
            _, pacc = accuracy.pm_solution(iso, density, True)
            self.np_err = acc.double() - pacc
            iso.close()
        self.calls = 0

    def __call__(self, a):
        import torch
        from . import accuracy
        B.fmm_plan_set_green(self.plan.handle, B.FMM_GREEN_S, list(np.atleast_1d(a)))
        self.plan.solve(self.density, self.phi, self.acc)
        torch.cuda.synchronize()
        B.fmm_plan_check(self.plan.handle)
        _, pacc = accuracy.pm_solution(self.plan, self.density, False)
        d = self.acc.double() - pacc
        if self.np_err is not None:
            d = d - self.np_err
        mag = d.pow(2).sum(dim=0).sqrt()
        self.calls += 1
        return float(mag.max()) if self.norm == "lmax" else float(mag.pow(2).mean().sqrt())

    def close(self):
        self.plan.close()


def fit(N, L, p, density, n_terms=1, norm="l2", gerr=False, x0=None, step=0.01, xtol=1e-5, ftol=1e-9):
    """Best-fit a_1..a_n (starting at a_1 = -1/8, the G_S1 value) and the
    error norm there.  Returns {"a": [...], "norm": value, "evaluations": k,
    "at_gs1": the norm at a_1 = -1/8}."""
    obj = AnsatzObjective(N, L, p, density, norm=norm, gerr=gerr)
    start = np.array(x0 if x0 is not None else [-0.125] + [0.0] * (n_terms - 1), dtype=np.float64)
    at_gs1 = obj(np.array([-0.125] + [0.0] * (n_terms - 1)))
    x, fx, ev = nelder_mead(obj, start, step, xtol=xtol, ftol=ftol * at_gs1)
    obj.close()
    return {"a": [float(v) for v in x], "norm": fx, "evaluations": ev, "at_gs1": at_gs1}


def main():
    import argparse
    import json
    import torch
    from . import accuracy
    ap = argparse.ArgumentParser(description="Fit a_k of the G_S ansatz (Sec. 3, Table 1) on the GPU")
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--L", type=int, default=3)
    ap.add_argument("--orders", default="4,6,8")
    ap.add_argument("--terms", type=int, default=1)
    ap.add_argument("--norm", choices=["l2", "lmax"], default="l2")
    ap.add_argument("--source", choices=["corner", "centre", "random"], default="corner")
    ap.add_argument("--gerr", action="store_true", help="objective: eq. gerr instead of FMM vs PM")
    args = ap.parse_args()
    d = torch.from_numpy(accuracy.point_sources(args.n, args.source, seed=7)).cuda()
    for p in [int(x) for x in args.orders.split(",")]:
        r = fit(args.n, args.L, p, d, n_terms=args.terms, norm=args.norm, gerr=args.gerr)
        print(json.dumps({"N": args.n, "L": args.L, "p": p, "source": args.source, "norm": args.norm,
                          "gerr": args.gerr, **r}), flush=True)


if __name__ == "__main__":
    main()
