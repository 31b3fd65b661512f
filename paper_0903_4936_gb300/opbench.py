"""Operator microbenchmark: one multi-RHS operator launch shape, timed with
CUDA events, on a seeded random SU(3) field.

    python -m paper_0903_4936_gb300.opbench --dims 16 16 16 32 --L 30 --prec fp32 fp64

Prints one JSON line per precision: microseconds per launch, algorithmic
bytes per launch (links and clover once per site, every column read once and
written once) and the resulting GB/s and flop rate (1872 flops per site and
column).  After the timed launches, one more launch per precision runs
between cudaProfilerStart/Stop, so `ncu --profile-from-start off` captures
exactly those.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FLOPS_PER_SITE_COLUMN = 1872


def operator_bytes(V: int, L: int, prec: str) -> int:
    """Algorithmic bytes of one launch over L columns."""
    real = {"fp64": 8, "df64": 8, "fp32": 4, "fp16": 4}[prec]
    spinor = {"fp64": 384, "df64": 384, "fp32": 192, "fp16": 2 * (48 + 4)}[prec]
    return V * (4 * 18 * real + 72 * real) + V * L * spinor


def main(argv=None) -> None:
    import synth

    import paper_0903_4936_gb300 as bk

    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--dims", type=int, nargs=4, default=[16, 16, 16, 32])
    ap.add_argument("--L", type=int, default=30)
    ap.add_argument("--prec", nargs="+", default=["fp32"])
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--kappa", type=float, default=0.125)
    args = ap.parse_args(argv)
    dims, L = tuple(args.dims), args.L
    lat = bk.Lattice(dims)
    lat.upload_gauge(synth.random_su3_field(dims, 0.5, 1003))
    lat.build_clover(1.0)
    X = torch.from_numpy(synth.z2_noise(dims, L, 5)).cuda()
    fields = {}
    for p in args.prec:
        sp = "fp64" if p == "df64" else p
        fields[p] = (lat.pack(X, sp), lat.empty_field(L, sp))
    del X
    for p, (F, Y) in fields.items():  # warm-up (and launch-shape tuning)
        for _ in range(3):
            lat.dslash_dev(F, L, args.kappa, p, out=Y)
    torch.cuda.synchronize()
    for p, (F, Y) in fields.items():
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.reps):
            lat.dslash_dev(F, L, args.kappa, p, out=Y)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / args.reps
        b = operator_bytes(lat.V, L, p)
        print(json.dumps({"kernel": f"k_dslash<{p.upper()}>", "dims": list(dims), "L": L, "us": ms * 1e3,
                          "alg_bytes": b, "gbs": b / ms / 1e6,
                          "tflops": FLOPS_PER_SITE_COLUMN * lat.V * L / ms / 1e9}), flush=True)
    torch.cuda.profiler.start()
    for p, (F, Y) in fields.items():
        lat.dslash_dev(F, L, args.kappa, p, out=Y)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()


if __name__ == "__main__":
    main()
