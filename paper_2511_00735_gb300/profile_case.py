"""Run one phase of the 64x64, N = 16 scattering workload in isolation (for profilers).

  python -m paper_2511_00735_gb300.profile_case --phase leaf|merge|matvec|precond|solve
         [--nx 64] [--precision mixed|fp64] [--repeat R]

leaf:    R leaf builds;  merge: leaves + R merge-tree builds;  matvec: R FP64 skeleton
matvecs with 16 right-hand sides;  precond: R preconditioner applications;
solve: one full step (leaves, merges, FGMRES to 1e-10).
"""
from __future__ import annotations

import argparse
import time

import numpy as np


def main():
    import torch

    from . import hps as H
    from . import inputs

    ap = argparse.ArgumentParser()
    ap.add_argument("--phase", default="leaf", choices=["leaf", "merge", "matvec", "precond", "solve"])
    ap.add_argument("--nx", type=int, default=64)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--nrhs", type=int, default=16)
    ap.add_argument("--multi", action="store_true", help="the 128x128 kappa=200 eight-bump problem")
    a = ap.parse_args()
    prec = H.HPS_MIXED if a.precision == "mixed" else H.HPS_FP64
    kappa = 100.0 * a.nx / 64.0
    L = 2 * int(round(np.log2(a.nx)))
    if a.multi:
        prob = inputs.mixed_128x128(seed=2, nrhs=a.nrhs)
    else:
        prob = inputs.single_bump(a.nx, 16, kappa, a.nrhs, seed=1, L_exact=max(L - 2, 0))
    s = H.Solver(0)
    t = H.setup(s, prob, prec, build=False)
    td = torch.from_numpy(t).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if a.phase == "leaf":
        for _ in range(a.repeat):
            s.build_leaves(prec)
    else:
        s.build_leaves(prec)
        if a.phase == "merge":
            for _ in range(a.repeat):
                s.merge_levels(prob.L_exact)
        elif a.phase == "matvec":
            x = torch.randn((a.nrhs, s.n_skel), dtype=torch.complex128, device="cuda")
            for _ in range(a.repeat):
                s.matvec(x)
        elif a.phase == "precond":
            s.merge_levels(prob.L_exact)
            r = torch.randn((a.nrhs, s.n_skel), dtype=torch.complex128, device="cuda")
            for _ in range(a.repeat):
                s.precond_apply(r, prob.inner_iters)
        else:
            s.merge_levels(prob.L_exact)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            _, info = s.gmres_solve(td, tol=1e-10, inner_iters=prob.inner_iters)
            print("iterations", info["outer_iterations"], "residual", info["max_rel_residual"],
                  f"solve {time.perf_counter() - t1:.3f} s, bytes held {s.bytes_held() / 1e9:.1f} GB")
    torch.cuda.synchronize()
    print(f"{a.phase} x{a.repeat} on {a.nx}x{a.nx}: {time.perf_counter() - t0:.3f} s")
    s.close()


if __name__ == "__main__":
    main()
