"""The paper's experiment shape (Section 4, Tables 2 and 3, Figure 1) on
synthetic gauge fields: L dependence of block BiCGSTAB and block BiCGGR.

    python -m paper_0903_4936_gb300.experiments [--dims 16 16 16 32] [--seeds 1003 1013 1023]

For every kappa, method and block size L, the 12 point sources at the origin
are split into 12 / L blocks of L columns, each block a system of its own (the
paper solves them one after another; here they run in one batched FP64 call,
so "time" is the call's wall time for all 12 sources).  The stopping rule is
the paper's: recursive relative residual <= tol (1e-14 in the paper), after
which the true residual max_i ||A x_i - b_i|| / ||b_i|| is evaluated.  Printed
per row, averaged over the gauge seeds: iterations (mean over blocks),
time, time per source, and the max / min true residual over seeds and blocks,
as in the paper's tables; a block that does not reach tol within maxiter is
counted in the "failed" column.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def block_size_scan(dims, kappas, Ls, methods, seeds, tol=1e-14, eps=0.5, csw=1.0, maxiter=1000):
    """Rows of (kappa, method, L, mean iterations, mean seconds, seconds per
    source, max true residual, min true residual, failed blocks)."""
    import synth

    import paper_0903_4936_gb300 as bk

    B = torch.from_numpy(synth.point_sources(dims)).cuda()
    acc = {}
    for seed in seeds:
        lat = bk.Lattice(dims)
        lat.upload_gauge(synth.random_su3_field(dims, eps, seed))
        lat.build_clover(csw)
        for kappa in kappas:
            for method in methods:
                for L in Ls:
                    Ls_sys = [L] * (12 // L)
                    # warm-up of the operator's launch shapes for this column count
                    lat.block_solve_batched(B, [kappa] * len(Ls_sys), Ls_sys, method=method, prec="fp64",
                                            tol=1e-4, maxiter=50, raise_on_fail=False)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    X, infos = lat.block_solve_batched(B, [kappa] * len(Ls_sys), Ls_sys, method=method,
                                                       prec="fp64", tol=tol, maxiter=maxiter,
                                                       raise_on_fail=False)
                    torch.cuda.synchronize()
                    dt = time.perf_counter() - t0
                    a = acc.setdefault((kappa, method, L), dict(it=[], t=[], tr=[], fail=0))
                    a["it"].append(np.mean([i["iterations"] for i in infos]))
                    a["t"].append(dt)
                    a["tr"] += [i["true_res_max"] for i in infos]
                    a["fail"] += sum(1 for i in infos if not i["converged"])
    rows = []
    for (kappa, method, L), a in acc.items():
        t = float(np.mean(a["t"]))
        rows.append((kappa, method, L, float(np.mean(a["it"])), t, t / 12.0, max(a["tr"]), min(a["tr"]), a["fail"]))
    return rows


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--dims", type=int, nargs=4, default=[16, 16, 16, 32])
    ap.add_argument("--kappas", type=float, nargs="+", default=[0.120, 0.125, 0.130])
    ap.add_argument("--L", type=int, nargs="+", default=[1, 2, 4, 12])
    ap.add_argument("--methods", nargs="+", default=["bicgstab", "bicggr"])
    ap.add_argument("--seeds", type=int, nargs="+", default=[1003, 1013, 1023])
    ap.add_argument("--tol", type=float, default=1e-14)
    args = ap.parse_args(argv)
    rows = block_size_scan(tuple(args.dims), args.kappas, args.L, args.methods, args.seeds, args.tol)
    print(f"| kappa | method | L | iterations | time [s] | time/source [s] | true res max | true res min | failed |")
    print("|---|---|---|---|---|---|---|---|---|")
    for r in rows:
        print(f"| {r[0]:.3f} | {r[1]} | {r[2]} | {r[3]:.1f} | {r[4]:.3f} | {r[5]:.4f} | {r[6]:.2e} | {r[7]:.2e} | {r[8]} |",
              flush=True)


if __name__ == "__main__":
    main()
