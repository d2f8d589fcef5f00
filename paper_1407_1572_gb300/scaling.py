"""Linear-scaling sweep of the IFMM on one GPU: factor + refined solve for N = 4^6 .. 4^10 points.

The paper's central claims (Section 1 and the remark in Section 5) are that the factorisation and the
solve cost O(N) and that the ranks of the compressed blocks do not grow with N. This module times
both phases at each N (uniform points in [0,1]^2, 64 points per leaf on average, 1/r + sqrt(N) I,
Chebyshev 4 x 4, eps 1e-6, 32 right-hand sides, GMRES refinement to 1e-7) in the mixed and the FP64
mode, and prints one JSON line per (N, mode): time per unknown, GMRES iterations, error to the
manufactured solution and the largest box rank.

    python -m paper_1407_1572_gb300.scaling [--nmax 1048576] [--modes mixed_solve,fp64]
"""
from __future__ import annotations

import argparse
import json
import math


def run(nmax: int = 1 << 20, modes=("mixed_solve", "fp64"), nrhs: int = 32, reps: int = 2):
    import torch

    from . import ifmm, inputs

    code = {"fp64": ifmm.IFMM_FP64, "mixed_solve": ifmm.IFMM_MIXED_SOLVE}
    st = torch.cuda.current_stream()
    out = []
    n = 4096
    while n <= nmax:
        depth = max(2, round(math.log(n / 64, 4)))
        pts = inputs.uniform_points(1407 + depth, n)
        xs = torch.from_numpy(inputs.rhs(1500 + depth, n, nrhs).T.copy()).cuda()
        for mode in modes:
            prm = ifmm.default_params(depth=depth, cheb_p=4, eps=1e-6, diag=math.sqrt(n), tau_ref=1,
                                      precision=code[mode], refine_tol=1e-7, refine_maxit=240, refine_restart=60)
            g = ifmm.IFMM(pts, ifmm.IFMM_K_INV_R, prm, st)
            b = torch.empty_like(xs)
            x = torch.empty_like(xs)
            ifmm.ifmm_matvec(g.h, xs.data_ptr(), b.data_ptr(), nrhs, n)
            for _ in range(reps):
                torch.cuda.synchronize()
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record(st)
                ifmm.ifmm_factor(g.h, allow_overflow=True)
                e1.record(st)
                ifmm.ifmm_solve(g.h, b.data_ptr(), x.data_ptr(), nrhs, n, allow_noconv=True)
                e2.record(st)
                torch.cuda.synchronize()
            s = g.stats()
            tf, ts = e0.elapsed_time(e1), e1.elapsed_time(e2)
            err = float(((x - xs).norm(dim=1) / xs.norm(dim=1)).max())
            rec = dict(N=n, depth=depth, mode=mode, t_factor_ms=tf, t_solve_ms=ts,
                       us_per_unknown=1000.0 * (tf + ts) / n, unknowns_per_s=n / ((tf + ts) / 1000.0),
                       refine_iters=s["refine_iters"], err=err, max_rank=s["max_rank"])
            print(json.dumps(rec), flush=True)
            out.append(rec)
            g.close()
        n *= 4
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--nmax", type=int, default=1 << 20)
    ap.add_argument("--modes", default="mixed_solve,fp64")
    args = ap.parse_args()
    run(args.nmax, tuple(m for m in args.modes.split(",") if m))


if __name__ == "__main__":
    main()
