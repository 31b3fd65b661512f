"""The paper's experiment shape (Section 4, Tables 2 and 3, Figures 1 and 2) on
synthetic gauge fields: L dependence of block BiCGSTAB and block BiCGGR.

    python -m paper_0903_4936_gb300.experiments [--dims 16 16 16 32] [--seeds 1003 1013]
        [--kappas ...] [--scan] [--json out.json] [--markdown]
    python -m paper_0903_4936_gb300.experiments --kappas 0.1425 --L 4 12 --deflate --json out.json
    python -m paper_0903_4936_gb300.experiments --from-json result.json

For every kappa, method and block size L, the 12 point sources at the origin
are split into 12 / L blocks of L columns, each block a system of its own (the
paper solves them one after another; here they run in one batched FP64 call,
so "time" is the call's wall time for all 12 sources).  The stopping rule is
the paper's: recursive relative residual <= tol (1e-14 in the paper), after
which the true residual max_i ||A x_i - b_i|| / ||b_i|| is evaluated.  Per
row, averaged over the gauge seeds: iterations (mean over blocks), time, time
per source, and the max / min true residual over seeds and blocks, as in the
paper's tables; a block that does not reach tol within maxiter is counted in
the "failed" column.

--scan first raises kappa on the first seed until the single-source solve
needs about 1000 iterations (the paper's light quarks: 1519 to 2440
iterations at kappa 0.1355 to 0.1359 on its Iwasaki configurations), and runs
the grid at three kappas approaching that point.  --json writes the scan, the
grid and the residual histories of the first seed at the lightest kappa (the
paper's Figure 2) to a file; --markdown prints the grid as a table.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _lattice(dims, eps, seed, csw):
    import synth

    import paper_0903_4936_gb300 as bk
    lat = bk.Lattice(dims)
    lat.upload_gauge(synth.random_su3_field(dims, eps, seed))
    lat.build_clover(csw)
    return lat


def kappa_scan(dims, seed, kappas, eps=0.5, csw=1.0, target=1000, maxiter=4000):
    """Iterations of the FP64 single-source solve (point source, column 0) as
    kappa rises; stops after the first kappa that needs more than `target`
    iterations or does not converge."""
    import synth
    lat = _lattice(dims, eps, seed, csw)
    B = torch.from_numpy(synth.point_sources(dims)[:1].copy()).cuda()
    out = []
    for k in kappas:
        X, info = lat.block_solve(B, k, method="bicgstab", prec="fp64", tol=1e-14, maxiter=maxiter,
                                  raise_on_fail=False)
        out.append(dict(kappa=k, iterations=info["iterations"], converged=bool(info["converged"]),
                        true_res=info["true_res_max"]))
        if info["iterations"] > target or not info["converged"]:
            break
    return out


def block_size_scan(dims, kappas, Ls, methods, seeds, tol=1e-14, eps=0.5, csw=1.0, maxiter=6000,
                    history_seed=None, history_kappa=None, deflate=False):
    """Rows of (kappa, method, L, mean iterations, mean seconds, seconds per
    source, max true residual, min true residual, failed blocks), and the
    residual histories (first block) of history_seed at history_kappa."""
    import synth

    B = torch.from_numpy(synth.point_sources(dims)).cuda()
    acc, hist = {}, {}
    for seed in seeds:
        lat = _lattice(dims, eps, seed, csw)
        for kappa in kappas:
            for method in methods:
                for L in Ls:
                    Ls_sys = [L] * (12 // L)
                    want_hist = seed == history_seed and kappa == history_kappa
                    # warm-up of the operator's launch shapes for this column count
                    lat.block_solve_batched(B, [kappa] * len(Ls_sys), Ls_sys, method=method, prec="fp64",
                                            tol=1e-4, maxiter=50, raise_on_fail=False, deflate=deflate)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    X, infos = lat.block_solve_batched(B, [kappa] * len(Ls_sys), Ls_sys, method=method,
                                                       prec="fp64", tol=tol, maxiter=maxiter,
                                                       raise_on_fail=False, history=want_hist, deflate=deflate)
                    torch.cuda.synchronize()
                    dt = time.perf_counter() - t0
                    a = acc.setdefault((kappa, method, L), dict(it=[], t=[], tr=[], fail=0))
                    a["it"].append(float(np.mean([i["iterations"] for i in infos])))
                    a["t"].append(dt)
                    a["tr"] += [i["true_res_max"] for i in infos]
                    a["fail"] += sum(1 for i in infos if not i["converged"])
                    if want_hist:
                        hist[f"{method}_L{L}"] = infos[0]["history"]
    rows = []
    for (kappa, method, L), a in acc.items():
        t = float(np.mean(a["t"]))
        rows.append(dict(kappa=kappa, method=method, L=L, iterations=float(np.mean(a["it"])), time_s=t,
                         time_per_source_s=t / 12.0, true_res_max=max(a["tr"]), true_res_min=min(a["tr"]),
                         failed=a["fail"]))
    return rows, hist


def markdown(rows):
    lines = ["| kappa | method | L | iterations | time [s] | time/source [s] | true res max | true res min | failed |",
             "|---|---|---|---|---|---|---|---|---|"]
    for r in rows:
        lines.append(f"| {r['kappa']:.4f} | {r['method']} | {r['L']} | {r['iterations']:.1f} | {r['time_s']:.3f} | "
                     f"{r['time_per_source_s']:.4f} | {r['true_res_max']:.2e} | {r['true_res_min']:.2e} | "
                     f"{r['failed']} |")
    return "\n".join(lines)


def markdown_report(result):
    """The scan and the grid of a result file as markdown (the tables of the
    design notes are generated with --from-json)."""
    out = []
    for key, title in (("scan", "kappa scan, FP64 BiCGSTAB, one point source"),
                       ("scan_fine", "refined between the last two kappas")):
        if result.get(key):
            out.append(f"{title} (seed {result['seeds'][0]}):\n")
            out.append("| kappa | iterations | converged | true residual |")
            out.append("|---|---|---|---|")
            for r in result[key]:
                out.append(f"| {r['kappa']:.5f} | {r['iterations']} | {r['converged']} | {r['true_res']:.2e} |")
            out.append("")
    out.append(markdown(result["grid"]))
    h = result.get("histories", {})
    if h.get("by_method_L"):
        out.append("")
        out.append(f"residual histories (seed {h['seed']}, kappa {h['kappa']}): iterations to 1e-4 / 1e-8 / 1e-12")
        out.append("")
        out.append("| method, L | 1e-4 | 1e-8 | 1e-12 | total |")
        out.append("|---|---|---|---|---|")
        for k, hist in h["by_method_L"].items():
            def first(t):
                return next((i for i, v in enumerate(hist) if v <= t), "-")
            out.append(f"| {k} | {first(1e-4)} | {first(1e-8)} | {first(1e-12)} | {len(hist) - 1} |")
    return "\n".join(out)


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--dims", type=int, nargs=4, default=[16, 16, 16, 32])
    ap.add_argument("--kappas", type=float, nargs="+", default=[0.120, 0.125, 0.130])
    ap.add_argument("--L", type=int, nargs="+", default=[1, 2, 4, 12])
    ap.add_argument("--methods", nargs="+", default=["bicgstab", "bicggr"])
    ap.add_argument("--seeds", type=int, nargs="+", default=[1003, 1013, 1023])
    ap.add_argument("--tol", type=float, default=1e-14)
    ap.add_argument("--scan", action="store_true")
    ap.add_argument("--json")
    ap.add_argument("--markdown", action="store_true")
    ap.add_argument("--deflate", action="store_true",
                    help="breakdown-robust form: orthonormalised sources, restarts on L x L breakdown")
    ap.add_argument("--from-json", help="print the tables of an earlier --json result and exit")
    args = ap.parse_args(argv)
    if args.from_json:
        with open(args.from_json) as f:
            print(markdown_report(json.load(f)))
        return
    dims = tuple(args.dims)
    result = dict(dims=list(dims), eps=0.5, csw=1.0, tol=args.tol, seeds=args.seeds,
                  sources="the 12 point sources at the origin, split into 12/L blocks of L columns",
                  precision="FP64 (the paper's method)")
    kappas = args.kappas
    if args.scan:
        scan = kappa_scan(dims, args.seeds[0], [round(0.130 + 0.005 * i, 4) for i in range(9)])
        result["scan"] = scan
        print(json.dumps(dict(scan=scan)), flush=True)
        # the last converged kappa below ~1000 iterations and the first beyond:
        # refine between them and take three kappas approaching the light point
        conv = [s for s in scan if s["converged"]]
        lo = conv[-1]["kappa"] if conv else 0.130
        hi = scan[-1]["kappa"] if scan and (scan[-1]["iterations"] > 1000 or not scan[-1]["converged"]) else lo
        fine = kappa_scan(dims, args.seeds[0], [round(lo + (hi - lo) * f, 5) for f in (0.25, 0.5, 0.75)]) \
            if hi > lo else []
        result["scan_fine"] = fine
        print(json.dumps(dict(scan_fine=fine)), flush=True)
        pts = [s for s in scan + fine if s["converged"]]
        pts.sort(key=lambda s: s["kappa"])
        light = [s["kappa"] for s in pts if s["iterations"] <= 3000][-3:]
        kappas = light
    rows, hist = block_size_scan(dims, kappas, args.L, args.methods, args.seeds, args.tol,
                                 history_seed=args.seeds[0], history_kappa=max(kappas), deflate=args.deflate)
    result["deflate"] = bool(args.deflate)
    result["kappas"] = kappas
    result["grid"] = rows
    result["histories"] = dict(kappa=max(kappas), seed=args.seeds[0], by_method_L=hist)
    if args.json:
        with open(args.json, "w") as f:
            json.dump(result, f, indent=1)
    if args.markdown or not args.json:
        print(markdown(rows), flush=True)


if __name__ == "__main__":
    main()
