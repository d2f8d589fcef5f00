"""The numerical benchmarks of the paper (Section 5) on one GPU.

Equation "main_Solving_Equation" (unit diagonal) with the three regularised kernels of Section 5 (a =
0.001), points uniform in [-1, 1]^2, Chebyshev interpolation with 8 nodes per dimension, compression
tolerance 1e-14 (here the matrix-scale threshold eps * s_A), a known x and b = A~ x, solved once
without refinement (the paper's direct solve). For each kernel and N the module prints the paper's
columns: t_a (build), t_f (factor), t_s (solve), r_m (largest box rank) and the relative error of x.
--svd-eps > 0 adds the paper's SVD compression of the Chebyshev interpolation (svd_eps of
ifmm_params; the kept counts per level are printed as svd_ranks). A size whose factorisation fails
(a device allocation, say) prints a "failed" record and ends that kernel's sweep.

    python -m paper_1407_1572_gb300.paper_bench [--nmax 1000000] [--kernels log,r2log,inv] [--svd-eps 1e-14]
"""
from __future__ import annotations

import argparse
import json

KERNELS = {"log": 3, "r2log": 5, "inv": 4}   # the order of the paper's tables
SIZES = (1000, 2000, 5000, 10000, 20000, 50000, 100000, 200000, 500000, 1000000)


def run(nmax: int = 1000000, kernels=("log", "r2log", "inv"), a: float = 1e-3, eps: float = 1e-14,
        svd_eps: float = 0.0):
    import torch

    from . import ifmm, inputs

    st = torch.cuda.current_stream()
    out = []
    for name in kernels:
        for n in (s for s in SIZES if s <= nmax):
            pts = inputs.uniform_points(1407 + n, n, lo=-1.0, side=2.0)
            xs = torch.from_numpy(inputs.rhs(1407 + 7 * n, n, 1).T.copy()).cuda()
            prm = ifmm.default_params(depth=0, leaf_max=64, cheb_p=8, eps=eps, diag=1.0, kparam=(a,),
                                      box=(-1.0, -1.0, 2.0), tau_ref=1, svd_eps=svd_eps)
            torch.cuda.synchronize()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            e[0].record(st)
            g = ifmm.IFMM(pts, KERNELS[name], prm, st)
            e[1].record(st)
            b = torch.empty_like(xs)
            ifmm.ifmm_matvec(g.h, xs.data_ptr(), b.data_ptr(), 1, n)
            x = torch.empty_like(xs)
            torch.cuda.synchronize()
            e[2].record(st)
            try:
                ifmm.ifmm_factor(g.h, allow_overflow=True)
            except ifmm.IFMMError as err:   # e.g. out of device memory
                rec = dict(kernel=name, N=n, depth=g.stats()["depth"], failed=str(err))
                print(json.dumps(rec), flush=True)
                out.append(rec)
                g.close()
                break                       # larger N needs more
            e[3].record(st)
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(st)
            ifmm.ifmm_solve(g.h, b.data_ptr(), x.data_ptr(), 1, n)
            f1.record(st)
            torch.cuda.synchronize()
            s = g.stats()
            rec = dict(kernel=name, N=n, depth=s["depth"], t_a_s=s["t_build_ms"] / 1e3,
                       t_f_s=e[2].elapsed_time(e[3]) / 1e3, t_s_s=f0.elapsed_time(f1) / 1e3, r_m=s["max_rank"],
                       err=float((x - xs).norm() / xs.norm()))
            if svd_eps > 0:
                rec["svd_eps"] = svd_eps
                rec["svd_ranks"] = s["svd_ranks"][2:s["depth"] + 1]
            print(json.dumps(rec), flush=True)
            out.append(rec)
            g.close()
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--nmax", type=int, default=1000000)
    ap.add_argument("--kernels", default="log,r2log,inv")
    ap.add_argument("--svd-eps", type=float, default=0.0)
    args = ap.parse_args()
    run(args.nmax, tuple(k for k in args.kernels.split(",") if k), svd_eps=args.svd_eps)


if __name__ == "__main__":
    main()
