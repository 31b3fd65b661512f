#!/usr/bin/env python
"""Benchmark: right-hand sides solved per second to true relative residual 1e-10
with the mixed-precision block BiCGGR solver, on a synthetic 16^3 x 32 clover
Wilson-Dirac problem, plus the multi-RHS operator's HBM roofline.

One step = every case of the workload solved once through the C ABI (block
BiCGGR, FP16-stored / FP32-arithmetic inner iterations, FP64 reliable updates
and FP64 true residual).  Each solve must reach a FP64 true residual <= 1e-10,
else the run fails.  Prints ONE JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--workload c3|c3-12|c3-48|c2] [--no-fp64] [--no-cpu-baseline]

--impl reference times the FP64 CPU oracle (test infrastructure, written from
the paper) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RHS solved/s to rel resid 1e-10 (mixed vs FP64); multi-RHS dslash HBM GB/s"

# Workloads: (Lx, Ly, Lz, Lt), link spread eps, c_SW, cases (kappa, L, source kind).
WORKLOADS = {
    "c3": dict(dims=(16, 16, 16, 32), eps=0.5, csw=1.0, gauge_seed=1003, prec="fp32", method="bicgstab",
               block=6, delta=0.03,
               cases=[(k, L, src) for k in (0.120, 0.125, 0.130) for (L, src) in ((12, "point"), (48, "z2"))],
               desc="16^3x32 clover Wilson-Dirac, random SU(3) links eps=0.5, c_SW=1.0, kappa in "
                    "{0.120,0.125,0.130} x (L=12 point sources, L=48 complex-Z2 noise) = 180 right-hand sides; "
                    "mixed: one batched block BiCGSTAB solve over 30 systems of 6 columns, FP32 inner iterations "
                    "with per-iteration Cholesky basis of P, FP64 residual replacement (delta 0.03), FP64 true "
                    "residual <= 1e-10 for every column; FP64 comparison: the paper's plain FP64 block BiCGGR "
                    "per case (one block of L columns), same true residual"),
    "c4": dict(dims=(24, 24, 24, 48), eps=0.5, csw=1.0, gauge_seed=1004, prec="fp32", method="bicgstab",
               block=6, delta=0.03, e2e=False, distinct_sources=True,
               e2e_note="host-buffer pass not run: its staging copies of B and X (2 x 25 GB) do not fit beside "
                        "the solve's 250 GB on the device",
               cases=list(zip((0.120, 0.122, 0.124, 0.126, 0.128, 0.130), (4, 12, 12, 24, 48, 96), ["z4"] * 6)),
               desc="24^3x48 clover Wilson-Dirac, random SU(3) links eps=0.5, c_SW=1.0: 6 systems, kappa "
                    "{0.120,...,0.130} with L {4,12,12,24,48,96} Z4 noise = 196 right-hand sides; mixed: one "
                    "batched block BiCGSTAB solve over 33 systems of at most 6 columns, FP32 inner iterations, "
                    "FP64 residual replacement (delta 0.03), FP64 true residual <= 1e-10 for every column; FP64 "
                    "comparison: the paper's plain FP64 block BiCGGR per system"),
    "c3-12": dict(dims=(16, 16, 16, 32), eps=0.5, csw=1.0, gauge_seed=1003, prec="fp32", method="bicgstab",
                  cases=[(0.125, 12, "point")],
                  desc="16^3x32, eps=0.5, c_SW=1.0, kappa=0.125, L=12 point sources; block BiCGSTAB, "
                       "FP32 inner iterations, FP64 residual replacement, tol 1e-10"),
    "c3-48": dict(dims=(16, 16, 16, 32), eps=0.5, csw=1.0, gauge_seed=1003, prec="fp32", method="bicgstab",
                  cases=[(0.125, 48, "z2")],
                  desc="16^3x32, eps=0.5, c_SW=1.0, kappa=0.125, L=48 complex-Z2 noise; block BiCGSTAB, "
                       "FP32 inner iterations, FP64 residual replacement, tol 1e-10"),
    "c2": dict(dims=(8, 8, 8, 16), eps=0.5, csw=1.0, gauge_seed=1002, prec="fp32", method="bicgstab",
               cases=[(0.125, 12, "point")],
               desc="8^3x16, eps=0.5, c_SW=1.0, kappa=0.125, L=12 point sources; block BiCGSTAB FP32 inner + "
                    "FP64 residual replacement, tol 1e-10"),
}
TOL = 1e-10
MAXITER = 5000


def spinor_bytes(prec):
    # per site and column: read 24 reals, write 24 reals (+ one FP32 scale each way for FP16)
    return {"fp64": 2 * 24 * 8, "fp32": 2 * 24 * 4, "fp16": 2 * (24 * 2 + 4)}[prec]


def dslash_bytes(V, L, prec, launches=1):
    """Algorithmic bytes of `launches` multi-RHS operator launches over L
    columns in total: per launch 4 links and the 72-real clover per site once;
    every spinor column read once and written once."""
    s = 8 if prec == "fp64" else 4
    return launches * V * (4 * 18 * s + 72 * s) + V * L * spinor_bytes(prec)


def sources(dims, L, kind, seed):
    import synth
    if kind == "point":
        B = synth.point_sources(dims)
        return B[:L].copy() if L <= 12 else None
    if kind == "z2":
        return synth.z2_noise(dims, L, seed)
    if kind == "z4":
        return synth.z4_noise(dims, L, seed)
    return synth.gaussian_sources(dims, L, seed)


# sources that define the operator kernel k_dslash (its own file and the
# headers it includes)
OPERATOR_SOURCES = ["paper_0903_4936_gb300/csrc/dslash.cu", "paper_0903_4936_gb300/csrc/bk_common.cuh",
                    "paper_0903_4936_gb300/csrc/dd.cuh", "paper_0903_4936_gb300/csrc/bk_kernels.h",
                    "include/bkrylov.h"]


def source_hash():
    h = hashlib.sha256()
    for f in OPERATOR_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic(prec, alg_bytes_per_launch):
    """DRAM bytes per inner-operator launch: the measured DRAM / algorithmic
    byte ratio of the committed ncu capture of the same kernel (a smaller
    launch of the same shape), scaled to this run's average launch.  None
    unless the capture was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "dslash_traffic.json")
    if not os.path.exists(p) or alg_bytes_per_launch is None:
        return None
    d = json.load(open(p))
    if d.get("source_hash") != source_hash():
        return None
    c = d.get("captures", {}).get(prec)
    if not c:
        return None
    return c["dram_bytes"] / c["alg_bytes"] * alg_bytes_per_launch


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"bk_clocks_gpu{index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return None
        mhz = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": mhz[len(mhz) // 2] if mhz else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------ oracle baseline

ORACLE_SNIPPET = r"""
import os, sys, time, json
sys.path.insert(0, {root!r})
import numpy as np, synth
from oracle import clover, dense, dirac, solvers
dims = {dims!r}; kappa = {kappa!r}; L = {L}; kind = {kind!r}
U = synth.random_su3_field(dims, {eps!r}, {gseed!r})
B = synth.point_sources(dims)[:L].copy() if kind == "point" else synth.z2_noise(dims, L, {sseed!r})
t0 = time.perf_counter()
F = clover.field_strength(U)
A = lambda M: dense.to_columns(dirac.apply_dirac(U, dense.from_columns(M, dims), kappa, {csw!r}, F=F))
Bc = dense.to_columns(B)
t1 = time.perf_counter()
A(Bc)  # one operator application: the set-up product W_0 = A R_0 of the solve below
t2 = time.perf_counter()
X, info = solvers.block_bicggr(A, Bc, 1e-300, {iters})
t3 = time.perf_counter()
it = max(1, info["iterations"])
print(json.dumps(dict(setup_s=t1 - t0, apply_s=t2 - t1, iter_s=((t3 - t2) - (t2 - t1)) / it, iterations=it)))
"""


def run_oracle_sample(wl, case, iters=1):
    """Time `iters` iterations of the oracle's block BiCGGR (plus the initial
    operator application) on one case, single-threaded, in a fresh process."""
    kappa, L, kind = case
    code = ORACLE_SNIPPET.format(root=ROOT, dims=wl["dims"], kappa=kappa, L=L, kind=kind, eps=wl["eps"],
                                 gseed=wl["gauge_seed"], sseed=2000 + L, csw=wl["csw"], iters=iters)
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError("oracle sample failed: " + out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


# ------------------------------------------------------------------ GPU arm

def max_over_ranks(ms, world, device):
    """The slowest rank's timed milliseconds (every rank gets it)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, rhs_per_step, steps, max_ms):
    """Whole-job RHS/s: every rank (an independent replica with its own
    sources) solves rhs_per_step per step; the job takes the slowest rank's time."""
    return world * rhs_per_step * steps / (max_ms / 1e3)


def replica_seed(L, rank):
    """Source seed of a replica: each rank solves its own noise vectors."""
    return 2000 + L + 7919 * rank


def gb300_arm(args, wl, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_0903_4936_gb300 as bk
    import synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dims = wl["dims"]
    U = synth.random_su3_field(dims, wl["eps"], wl["gauge_seed"])
    lat = bk.Lattice(dims, local_rank)
    lat.upload_gauge(U)
    lat.build_clover(wl["csw"])
    V = lat.V
    del U
    with_e2e = wl.get("e2e", True)
    cases = []
    batch = None
    if wl.get("block"):
        # batched mode: all cases' sources in one device block (each case a
        # view of its columns), every case split into systems of at most
        # `block` columns, all systems solved together.  Sources go to the
        # device one case at a time, so the host holds at most one case.
        blk = wl["block"]
        Lt = sum(L for (_, L, _) in wl["cases"])
        Ball = torch.empty((Lt,) + tuple(reversed(dims)) + (4, 3), dtype=torch.complex128, device=dev)
        kap_s, L_s, owner = [], [], []
        c0 = 0
        for ci, (kappa, L, kind) in enumerate(wl["cases"]):
            seed = replica_seed(L, rank) + (100 * ci if wl.get("distinct_sources") else 0)
            Ball[c0:c0 + L].copy_(torch.from_numpy(sources(dims, L, kind, seed)))
            cases.append(dict(kappa=kappa, L=L, kind=kind, B=Ball[c0:c0 + L]))
            for j0 in range(0, L, blk):
                kap_s.append(kappa)
                L_s.append(min(blk, L - j0))
                owner.append(ci)
            c0 += L
        batch = dict(kappas=kap_s, Ls=L_s, owner=owner, B=Ball,
                     Bh=Ball.cpu().pin_memory() if with_e2e else None)
    else:
        for (kappa, L, kind) in wl["cases"]:
            B = sources(dims, L, kind, replica_seed(L, rank))
            cases.append(dict(kappa=kappa, L=L, kind=kind, B=torch.from_numpy(B).to(dev),
                              Bh=torch.from_numpy(B).pin_memory()))
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def step(record, host=False):
        tot = dict(rhs=0, launches=0, t_inner=0.0, n_inner=0, bytes_inner=0.0)
        if batch is not None:
            B = batch["Bh"] if host else batch["B"]
            X, infos = lat.block_solve_batched(B, batch["kappas"], batch["Ls"], method=wl["method"],
                                               prec=wl["prec"], tol=TOL, maxiter=MAXITER, timing=record,
                                               delta=wl.get("delta", 0.0))
            for si, info in enumerate(infos):
                if not (info["converged"] and info["true_res_max"] <= TOL):
                    raise RuntimeError(f"system {si} did not reach {TOL}: {info}")
            ltot = sum(batch["Ls"])
            info = infos[0]
            tot["rhs"] = ltot
            tot["launches"] = info["n_launches"]
            tot["t_inner"] = info["time_dslash_inner_ms"]
            tot["n_inner"] = info["n_dslash_inner"]
            tot["bytes_inner"] = dslash_bytes(V, info["cols_dslash_inner"], wl["prec"], info["n_dslash_inner"])
            for ci, c in enumerate(cases):
                mine = [infos[si] for si in range(len(infos)) if batch["owner"][si] == ci]
                c["last_info"] = dict(iterations=max(i["iterations"] for i in mine),
                                      reliable_updates=max(i["reliable_updates"] for i in mine),
                                      true_res_max=max(i["true_res_max"] for i in mine))
            return tot
        for c in cases:
            B = c["Bh"] if host else c["B"]
            X, info = lat.block_solve(B, c["kappa"], method=wl["method"], prec=wl["prec"], tol=TOL,
                                      maxiter=MAXITER, timing=record)
            if not (info["converged"] and info["true_res_max"] <= TOL):
                raise RuntimeError(f"solve did not reach {TOL}: {info}")
            tot["rhs"] += c["L"]
            tot["launches"] += info["n_launches"]
            tot["t_inner"] += info["time_dslash_inner_ms"]
            tot["n_inner"] += info["n_dslash_inner"]
            tot["bytes_inner"] += dslash_bytes(V, info["cols_dslash_inner"], wl["prec"], info["n_dslash_inner"])
            c["last_info"] = info
        return tot

    for _ in range(args.warmup):
        step(False)
        flush.fill_(1)
    torch.cuda.synchronize()

    clocks = Clocks(local_rank)
    if rank == 0:
        clocks.start()
    per_step_ms = []
    agg = dict(rhs=0, launches=0, t_inner=0.0, n_inner=0, bytes_inner=0.0)
    stream = torch.cuda.current_stream(dev)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    # marks the timed steps for a profiler started with --profile-from-start off
    torch.cuda.profiler.start()
    total_ms = 0.0
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t = step(True)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        per_step_ms.append(ms)
        total_ms += ms
        for k in agg:
            agg[k] += t[k]
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    if world > 1:
        dist.barrier()
    clk = clocks.stop() if rank == 0 else None

    # e2e: the same metric through the public API with host (pinned) buffers:
    # B copied in and X copied out inside every call.
    e2e_ms = 0.0
    h2d = d2h = 0
    n_e2e = max(1, min(args.steps, 3))
    if with_e2e:
        for _ in range(n_e2e):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            t = step(False, host=True)
            torch.cuda.synchronize()
            e2e_ms += (time.perf_counter() - t0) * 1e3
        for c in cases:
            h2d += c["B"].numel() * 16
            d2h += c["B"].numel() * 16
    else:
        e2e_ms = None
    batched = None
    if batch is not None:
        batched = dict(systems=len(batch["Ls"]), block=wl["block"], columns=sum(batch["Ls"]))

    fp64 = None
    if not args.no_fp64 and rank == 0:
        # plain FP64 block BiCGGR (the paper's method) on every case, to the same
        # FP64 true residual, timed with CUDA events outside the timed loop
        rhs, ms = 0, 0.0
        per = {}
        for c in cases:
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            X, info = lat.block_solve(c["B"], c["kappa"], method="bicggr", prec="fp64", tol=TOL, maxiter=MAXITER)
            e1.record()
            e1.synchronize()
            if info["true_res_max"] > TOL:
                raise RuntimeError(f"FP64 solve did not reach {TOL}: {info}")
            t = e0.elapsed_time(e1)
            ms += t
            rhs += c["L"]
            per[f"k{c['kappa']}_L{c['L']}"] = dict(ms=round(t, 1), iterations=info["iterations"])
        fp64 = dict(method="block BiCGGR, FP64", fp64_rhs_per_s=rhs / (ms / 1e3), cases=per)

    return dict(total_ms=total_ms, per_step_ms=per_step_ms, agg=agg, clocks=clk,
                e2e_ms=e2e_ms / n_e2e if e2e_ms is not None else None,
                h2d=h2d, d2h=d2h, fp64=fp64, V=V, batched=batched,
                iters={f"k{c['kappa']}_L{c['L']}": c["last_info"]["iterations"] for c in cases},
                true_res={f"k{c['kappa']}_L{c['L']}": c["last_info"]["true_res_max"] for c in cases},
                rel_updates={f"k{c['kappa']}_L{c['L']}": c["last_info"]["reliable_updates"] for c in cases})


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    total_rhs_per_step = sum(L for (_, L, _) in wl["cases"])

    if args.impl == "reference":
        if rank != 0:
            return
        # Reference arm: the CPU oracle as it stands, one process, one thread.
        first = wl["cases"][0]
        samples = []
        for _ in range(args.warmup + args.steps):
            samples.append(run_oracle_sample(wl, first, iters=1))
        timed = samples[args.warmup:]
        iter_s = sum(s["iter_s"] for s in timed) / len(timed)
        n_it = GPU_ITERS_HINT.get(args.workload, 100)
        value = first[1] / (iter_s * n_it)
        line = {
            "impl": "reference", "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": iter_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["desc"], "parallelism": "none (CPU oracle)"},
            "cpu_baseline": {"value": value, "unit": "RHS/s", "cores": 1, "kind": "oracle",
                             "sample": f"one block BiCGGR iteration of the FP64 numpy oracle per step on the case "
                                       f"kappa={first[0]}, L={first[1]} {first[2]}; RHS/s = L / (seconds per "
                                       f"iteration x {n_it} iterations, the GPU solver's count for this case)"},
            "e2e": {"value": value, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line))
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    # The oracle baseline runs in a spawned process before any GPU work.
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu_case = wl["cases"][0]
        cpu = run_oracle_sample(wl, cpu_case, iters=1)

    r = gb300_arm(args, wl, rank, world, local_rank)

    total_ms = max_over_ranks(r["total_ms"], world, "cuda")
    value = job_value(world, total_rhs_per_step, args.steps, total_ms)
    agg = r["agg"]
    hbm, peak_kind = measured_peaks()
    achieved = (agg["bytes_inner"] / agg["n_inner"]) / ((agg["t_inner"] / agg["n_inner"]) / 1e3) / 1e9 \
        if agg["n_inner"] else None
    traffic = ncu_traffic(wl["prec"], agg["bytes_inner"] / agg["n_inner"] if agg["n_inner"] else None)
    line = {
        "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "storage": wl["prec"], "data": "synthetic",
        "mixed_precision": "inner iterations in FP32, FP64 residual replacement and true residual",
        "config": {"workload": wl["desc"], "lattice": "x".join(map(str, wl["dims"])),
                   "rhs_per_step": total_rhs_per_step, "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "l2": "inputs larger than L2 and a 256 MB L2 flush before every timed step"},
        "roofline": {"bound": "hbm", "kernel": f"k_dslash<{wl['prec'].upper()}> (inner operator, all columns)",
                     "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": (achieved / hbm) if achieved else None, "peak_kind": peak_kind,
                     "traffic": traffic, "launches": agg["n_inner"],
                     "avg_launch_us": agg["t_inner"] / agg["n_inner"] * 1e3 if agg["n_inner"] else None},
        "e2e": ({"value": world * total_rhs_per_step / (r["e2e_ms"] / 1e3), "unit": "RHS/s",
                 "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"]} if r["e2e_ms"] is not None else
                {"value": None, "unit": "RHS/s", "skipped": wl.get("e2e_note")}),
        "gpu_launches": int(agg["launches"]),
        "clocks": r["clocks"],
        "iterations": r["iters"], "reliable_updates": r["rel_updates"], "true_res_max": r["true_res"],
        "batched": r["batched"],
    }
    if r["fp64"]:
        r["fp64"]["mixed_over_fp64"] = (value / world) / r["fp64"]["fp64_rhs_per_s"]
        line["fp64_comparison"] = r["fp64"]
    if cpu is not None:
        its = r["iters"].get(f"k{wl['cases'][0][0]}_L{wl['cases'][0][1]}", 100)
        cv = wl["cases"][0][1] / (cpu["iter_s"] * its)
        line["cpu_baseline"] = {"value": cv, "unit": "RHS/s", "cores": 1, "kind": "oracle",
                                "sample": f"one FP64 numpy-oracle block BiCGGR iteration ({cpu['iter_s']:.1f} s) on "
                                          f"kappa={wl['cases'][0][0]}, L={wl['cases'][0][1]}; RHS/s = L / (s/iter x "
                                          f"{its} iterations, the GPU solver's count for that case)"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# Iteration counts of the GPU solver per workload's first case, used to turn the
# oracle's seconds per iteration into RHS/s on the reference arm.
GPU_ITERS_HINT = {"c3": 42, "c4": 45, "c3-12": 57, "c3-48": 281, "c2": 122}

if __name__ == "__main__":
    main()
