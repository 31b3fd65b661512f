#!/usr/bin/env python
"""Benchmark: right-hand sides solved per second to FP64 true relative residual
1e-10 on a synthetic clover Wilson-Dirac problem, plus the inner operator's
HBM roofline.

Default workload (`--workload c4`): 24^3 x 48, random SU(3) links eps = 0.5,
c_SW = 1, six systems kappa in {0.120, ..., 0.130} with L = {4, 12, 12, 24, 48,
96} Z4 noise sources (196 right-hand sides).  One step = the whole workload
solved once through the C ABI as one batched solve: every system split into
block systems of at most 6 columns, block BiCGSTAB on the even-odd Schur
system (--no-eo: on the full system) with FP32 inner iterations and residual
replacement at delta 0.003 (an FP64 true residual after every 1e-4 of
reduction and for every convergence decision, FP32 updates r -= A dx between;
--anchor 0: always FP64), each column to an FP64 true residual <= 1e-10 of
the full system (the run fails otherwise).  Prints ONE JSON line
on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--workload c4|c3|c2|c3-12|c3-24] [--no-fp64] [--fp64-full] [--no-cpu-baseline]
                  [--eo | --no-eo] [--delta D] [--anchor A] [--update fp64|df64]
                  [--oracle-solve] [--cpu-procs N]   (reference arm)

Comparisons on the same GPU (after the timed steps): the plain FP64 method at
the same 6-column split and formulation (isolates precision) and, with
--fp64-full, the paper's FP64 block BiCGGR with every system as one block of
all its columns on the full system.

--impl reference times the FP64 CPU oracle (test infrastructure, written from
the paper) on bounded samples of the same workload on the host cores
(--oracle-solve: its full solve of the first block system, one core).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RHS solved/s to rel resid 1e-10 (mixed vs FP64); multi-RHS dslash HBM GB/s"

_C4_CASES = list(zip((0.120, 0.122, 0.124, 0.126, 0.128, 0.130), (4, 12, 12, 24, 48, 96), ["z4"] * 6))
_C3_CASES = [(k, L, src) for k in (0.120, 0.125, 0.130) for (L, src) in ((12, "point"), (48, "z2"))]

# Workloads: (Lx, Ly, Lz, Lt), link spread eps, c_SW, cases (kappa, L, source kind).
WORKLOADS = {
    "c4": dict(dims=(24, 24, 24, 48), eps=0.5, csw=1.0, gauge_seed=1004, prec="fp32", method="bicgstab",
               block=6, delta=0.003, anchor=1e-4, eo=True, distinct_sources=True, cases=_C4_CASES,
               desc="24^3x48 clover Wilson-Dirac, random SU(3) links eps=0.5, c_SW=1.0: 6 systems, kappa "
                    "{0.120,...,0.130} with L {4,12,12,24,48,96} Z4 noise = 196 right-hand sides; one batched "
                    "block BiCGSTAB solve over 33 block systems of at most 6 columns on the even-odd Schur "
                    "system, FP32 inner iterations, residual replacement at delta 0.003 (FP64 after every 1e-4 "
                    "of reduction, FP32 between), FP64 true residual of the full system <= 1e-10 for every "
                    "column"),
    "c3": dict(dims=(16, 16, 16, 32), eps=0.5, csw=1.0, gauge_seed=1003, prec="fp32", method="bicgstab",
               block=6, delta=0.003, anchor=1e-4, eo=True, cases=_C3_CASES,
               desc="16^3x32 clover Wilson-Dirac, random SU(3) links eps=0.5, c_SW=1.0, kappa in "
                    "{0.120,0.125,0.130} x (L=12 point sources, L=48 complex-Z2 noise) = 180 right-hand sides; "
                    "one batched block BiCGSTAB solve over 30 systems of 6 columns on the even-odd Schur system, "
                    "FP32 inner iterations, residual replacement at delta 0.003 (FP64 after every 1e-4 of "
                    "reduction, FP32 between), FP64 true residual of the full system <= 1e-10 for every column"),
    "c2": dict(dims=(8, 8, 8, 16), eps=0.5, csw=1.0, gauge_seed=1002, prec="fp32", method="bicggr",
               cases=[(0.125, 12, "point")],
               desc="8^3x16, eps=0.5, c_SW=1.0, kappa=0.125, L=12 point sources; block BiCGGR with FP32 inner "
                    "iterations (Cholesky basis of P) and FP64 residual replacement, tol 1e-10"),
    "c3-24": dict(dims=(16, 16, 16, 32), eps=0.5, csw=1.0, gauge_seed=1003, prec="fp32", method="bicgstab",
                  block=6, delta=0.003, eo=True, cases=[(0.125, 24, "z2")],
                  desc="16^3x32, eps=0.5, c_SW=1.0, kappa=0.125, 24 complex-Z2 sources as 4 systems of 6 columns "
                       "on the even-odd Schur system, FP32 inner iterations, FP64 residual replacement (delta "
                       "0.003), tol 1e-10 (the small case for ncu captures: every block above L2, a few GB)"),
    "c3-12": dict(dims=(16, 16, 16, 32), eps=0.5, csw=1.0, gauge_seed=1003, prec="fp32", method="bicgstab",
                  cases=[(0.125, 12, "point")],
                  desc="16^3x32, eps=0.5, c_SW=1.0, kappa=0.125, L=12 point sources; block BiCGSTAB, "
                       "FP32 inner iterations, FP64 residual replacement, tol 1e-10"),
}
DEFAULT_WORKLOAD = "c4"
TOL = 1e-10
MAXITER = 5000


def spinor_bytes(prec):
    # per site and column: read 24 reals, write 24 reals (+ one FP32 scale each way for FP16)
    return {"fp64": 2 * 24 * 8, "fp32": 2 * 24 * 4, "fp16": 2 * (24 * 2 + 4)}[prec]


def schur_bytes(V, L, prec, applications=1):
    """Algorithmic bytes of `applications` even-odd Schur operator
    applications over L columns in total (two half-lattice launches each):
    per application the links twice (4 per site) and the 72-real site
    inverse once per site; per column the even input read twice, the odd
    temporary written and read, the output written (5 half-lattice passes)."""
    s = 8 if prec == "fp64" else 4
    return applications * V * (2 * 4 * 18 * s + 72 * s) + (V // 2) * L * 5 * (spinor_bytes(prec) // 2)


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


def case_seed(wl, ci, L, rank):
    """Source seed of case ci: each rank (replica) solves its own noise vectors."""
    return replica_seed(L, rank) + (100 * ci if wl.get("distinct_sources") else 0)


def systems(wl):
    """The block systems of the batched solve: (kappa, columns, case index)."""
    out = []
    blk = wl.get("block")
    for ci, (kappa, L, _) in enumerate(wl["cases"]):
        step = blk or L
        for j0 in range(0, L, step):
            out.append((kappa, min(step, L - j0), ci))
    return out


# sources that define the inner operator kernel (its own file and the headers it includes)
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
#
# The FP64 numpy oracle as it stands, on the host cores.  A full oracle solve
# of the benchmark's lattice takes hours, so a sample is one oracle
# application of D_W to the first block system's columns: the oracle block
# BiCGGR spends 2 such applications per iteration (plus one at set-up and one
# for the true residual) and its block algebra on top, which the sample leaves
# out (so the CPU figure is an upper bound).  RHS/s = columns / (seconds per
# application x (2 iterations + 2)), with the iteration count of the same
# FP64 block BiCGGR on the GPU for that system (iterate for iterate the
# oracle's recursion in the parity tests).  Every host core runs its own
# sample concurrently (one process each); the figure is their sum.

def _oracle_worker(args):
    """One process: load the shared gauge field and clover field strength,
    build the system's sources, time `reps` oracle operator applications."""
    root, dims, eps, gpath, fpath, csw, kappa, L, kind, seed, reps = args
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    sys.path.insert(0, root)
    import numpy as np

    import synth  # noqa: F401
    from oracle import dense, dirac
    U = np.load(gpath, mmap_mode="r")
    F = np.load(fpath, mmap_mode="r")
    B = sources(dims, L, kind, seed)[:L]
    Bc = dense.to_columns(B)
    out = []
    for _ in range(reps):
        t0 = time.perf_counter()
        dense.to_columns(dirac.apply_dirac(U, dense.from_columns(Bc, dims), kappa, csw, F=F))
        out.append(time.perf_counter() - t0)
    return out


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _mem_available_gb():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) / 1024 / 1024
    except OSError:
        pass
    return 16.0


def oracle_samples(wl, nsamples, rank=0, max_procs=None):
    """Run nsamples timed oracle applications spread over the host cores
    (one process per core, at most max_procs, spawned, no GPU).  Returns
    (per-sample seconds, processes used, the sampled system's (kappa, L))."""
    import numpy as np

    import synth
    from oracle import clover
    dims = wl["dims"]
    kappa, L, ci = systems(wl)[0]
    kind = wl["cases"][ci][2]
    Lcase = wl["cases"][ci][1]
    seed = case_seed(wl, ci, Lcase, rank)
    tmp = tempfile.mkdtemp(prefix="bk_oracle_")
    gpath, fpath = os.path.join(tmp, "U.npy"), os.path.join(tmp, "F.npy")
    U = synth.random_su3_field(dims, wl["eps"], wl["gauge_seed"])
    np.save(gpath, U)
    np.save(fpath, clover.field_strength(U))
    del U
    V = synth.lattice_volume(dims)
    per_proc_gb = 2.5 + V * L * 12 * 16 * 8 / 2**30  # the application's temporaries
    procs = max(1, min(_host_cores(), nsamples, int(_mem_available_gb() * 0.7 / per_proc_gb)))
    if max_procs:
        procs = min(procs, max_procs)
    reps = [nsamples // procs + (1 if i < nsamples % procs else 0) for i in range(procs)]
    jobs = [(ROOT, dims, wl["eps"], gpath, fpath, wl["csw"], kappa, Lcase, kind, seed, r) for r in reps if r > 0]
    try:
        ctx = multiprocessing.get_context("spawn")
        with ctx.Pool(len(jobs)) as pool:
            res = pool.map(_oracle_worker, jobs)
    finally:
        for f in (gpath, fpath):
            try:
                os.remove(f)
            except OSError:
                pass
        os.rmdir(tmp)
    secs = [t for r in res for t in r]
    return secs, len(jobs), (kappa, L)


def _oracle_solve_worker(args):
    """One process, one core: the full FP64 oracle block BiCGGR solve of one
    block system to the benchmark's tolerance (the oracle as it stands)."""
    root, dims, eps, gauge_seed, csw, kappa, L, kind, seed = args
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    sys.path.insert(0, root)
    import synth
    from oracle import clover, dense, dirac, solvers
    U = synth.random_su3_field(dims, eps, gauge_seed)
    F = clover.field_strength(U)
    B = sources(dims, L, kind, seed)[:L]

    def A(M):
        return dense.to_columns(dirac.apply_dirac(U, dense.from_columns(M, dims), kappa, csw, F=F))

    Bc = dense.to_columns(B)
    t0 = time.perf_counter()
    X, info = solvers.block_bicggr(A, Bc, TOL, MAXITER)
    secs = time.perf_counter() - t0
    res, _ = solvers.true_residual(A, Bc, X)
    return secs, int(info["iterations"]), float(res)


def oracle_full_solve(wl, rank=0):
    """Seconds, iterations and true residual of the oracle's full solve of the
    workload's first block system (spawned, so the thread limits hold)."""
    kappa, L, ci = systems(wl)[0]
    kind = wl["cases"][ci][2]
    Lcase = wl["cases"][ci][1]
    job = (ROOT, wl["dims"], wl["eps"], wl["gauge_seed"], wl["csw"], kappa, Lcase, kind,
           case_seed(wl, ci, Lcase, rank))
    ctx = multiprocessing.get_context("spawn")
    with ctx.Pool(1) as pool:
        secs, iters, res = pool.map(_oracle_solve_worker, [job])[0]
    return secs, iters, res, (kappa, Lcase)


def oracle_rhs_per_s(secs, procs, L, iters):
    """Whole-host RHS/s: procs concurrent samples, each an L-column operator
    application, (2 iterations + 2) applications per solve."""
    mean = sum(secs) / len(secs)
    return procs * L / (mean * (2 * iters + 2)), mean


# Iteration count of the FP64 block BiCGGR on the first block system of each
# workload on the full system (the oracle's form), as measured by this
# benchmark's FP64 comparison on a GB300 (--no-eo); the reference arm, which
# has no GPU, uses it to turn the oracle's seconds per application into RHS/s.
FP64_ITERS_FIRST_SYSTEM = {"c4": 42, "c3": 45, "c2": 50, "c3-12": 54}


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
    # All cases' sources in one device block (each case a view of its columns);
    # the host copy is pinned for the end-to-end pass.
    Lt = sum(L for (_, L, _) in wl["cases"])
    Ball = torch.empty((Lt,) + tuple(reversed(dims)) + (4, 3), dtype=torch.complex128, device=dev)
    cases = []
    c0 = 0
    for ci, (kappa, L, kind) in enumerate(wl["cases"]):
        Ball[c0:c0 + L].copy_(torch.from_numpy(sources(dims, L, kind, case_seed(wl, ci, L, rank))))
        cases.append(dict(kappa=kappa, L=L, kind=kind, c0=c0))
        c0 += L
    sysl = systems(wl)
    kap_s, L_s, owner = [s[0] for s in sysl], [s[1] for s in sysl], [s[2] for s in sysl]
    update = args.update or wl.get("update", "fp64")
    eo = wl.get("eo", False) if args.eo is None else args.eo
    anchor = wl.get("anchor", 0.0) if args.anchor is None else args.anchor
    delta = args.delta if args.delta is not None else wl.get("delta", 0.0)
    Xdev = torch.empty_like(Ball)
    Bh = Ball.cpu().pin_memory()
    Xh = torch.empty_like(Bh).pin_memory()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def solve(B, X, record, prec=None, method=None):
        return lat.block_solve_batched(B, kap_s, L_s, method=method or wl["method"], prec=prec or wl["prec"],
                                       tol=TOL, maxiter=MAXITER, timing=record, delta=delta,
                                       out=X, raise_on_fail=False, update=update, eo=eo, anchor=anchor)

    def check(infos, what):
        for si, info in enumerate(infos):
            if not (info["converged"] and info["true_res_max"] <= TOL):
                raise RuntimeError(f"{what}: system {si} did not reach {TOL}: {info}")

    def step(record, host=False):
        X, infos = solve(Bh if host else Ball, Xh if host else Xdev, record)
        check(infos, "mixed solve")
        info = infos[0]
        return dict(launches=info["n_launches"], t_inner=info["time_dslash_inner_ms"],
                    n_inner=info["n_dslash_inner"],
                    bytes_inner=(schur_bytes if eo else dslash_bytes)(V, info["cols_dslash_inner"], wl["prec"],
                                                                      info["n_dslash_inner"]),
                    infos=infos)

    last = None
    for _ in range(args.warmup):
        last = step(False)
        flush.fill_(1)
    torch.cuda.synchronize()

    clocks = Clocks(local_rank)
    if rank == 0:
        clocks.start()
    per_step_ms = []
    agg = dict(launches=0, t_inner=0.0, n_inner=0, bytes_inner=0.0)
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
        last = t
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    if world > 1:
        dist.barrier()
    clk = clocks.stop() if rank == 0 else None

    # e2e: the same metric through the public API with pinned host buffers: B
    # is copied in and X copied out (through a bounded device staging buffer,
    # a chunk of columns at a time) inside every call.
    n_e2e = max(1, min(args.steps, 3))
    e2e_ms = 0.0
    for _ in range(n_e2e):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(False, host=True)
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
    h2d = d2h = Ball.numel() * 16

    infos = last["infos"]
    per_case = {}
    for ci, c in enumerate(cases):
        mine = [infos[si] for si in range(len(infos)) if owner[si] == ci]
        per_case[f"k{c['kappa']}_L{c['L']}"] = dict(
            iterations=max(i["iterations"] for i in mine), reliable_updates=max(i["reliable_updates"] for i in mine),
            true_res_max=max(i["true_res_max"] for i in mine))

    fp64 = None
    if not args.no_fp64 and rank == 0:
        fp64 = {}

        def timed(fn):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            out = fn()
            e1.record()
            e1.synchronize()
            return out, e0.elapsed_time(e1)

        # the plain FP64 block BiCGGR at the same split: precision alone.  One
        # batched solve per case (all cases at once would need seven FP64
        # blocks of every column beside the benchmark's buffers); a short
        # untimed solve first tunes the FP64 operator's launch shape.
        tot, its, first = 0.0, [], None
        for ci, c in enumerate(cases):
            idx = [si for si in range(len(L_s)) if owner[si] == ci]
            Bc = Ball[c["c0"]:c["c0"] + c["L"]]
            Xc = Xdev[c["c0"]:c["c0"] + c["L"]]
            ks, ls = [kap_s[si] for si in idx], [L_s[si] for si in idx]
            lat.block_solve_batched(Bc, ks, ls, method="bicggr", prec="fp64", tol=TOL, maxiter=1, out=Xc,
                                    raise_on_fail=False, eo=eo)
            (X, inf64), ms = timed(lambda: lat.block_solve_batched(Bc, ks, ls, method="bicggr", prec="fp64",
                                                                   tol=TOL, maxiter=MAXITER, out=Xc,
                                                                   raise_on_fail=False, eo=eo))
            check(inf64, "FP64 solve at the same split")
            tot += ms
            its += [i["iterations"] for i in inf64]
            if first is None:
                first = inf64[0]["iterations"]
        fp64["same_split"] = dict(method="block BiCGGR, FP64, the same block systems (one batched solve per case)"
                                  + (", even-odd form" if eo else ""),
                                  rhs_per_s=Lt / (tot / 1e3), ms=round(tot, 1), iterations_first_system=first,
                                  iterations_max=max(its))
        if args.fp64_full:
            # the paper's method as printed: every case one block of all its
            # columns, on the full system.  A fresh context, so that the
            # workspace of the solves above (even-odd blocks) is released.
            lat.close()
            U = synth.random_su3_field(dims, wl["eps"], wl["gauge_seed"])
            lat = bk.Lattice(dims, local_rank)
            lat.upload_gauge(U)
            lat.build_clover(wl["csw"])
            del U
            tot, per = 0.0, {}
            for c in cases:
                Bc = Ball[c["c0"]:c["c0"] + c["L"]].contiguous()
                lat.block_solve(Bc, c["kappa"], method="bicggr", prec="fp64", tol=TOL, maxiter=1,
                                raise_on_fail=False)
                (X, info), ms = timed(lambda: lat.block_solve(Bc, c["kappa"], method="bicggr", prec="fp64", tol=TOL,
                                                              maxiter=MAXITER))
                if info["true_res_max"] > TOL:
                    raise RuntimeError(f"FP64 solve did not reach {TOL}: {info}")
                tot += ms
                per[f"k{c['kappa']}_L{c['L']}"] = dict(ms=round(ms, 1), iterations=info["iterations"])
                del Bc
            fp64["full_blocks"] = dict(method="block BiCGGR, FP64, each case one block (the paper's method)",
                                       rhs_per_s=Lt / (tot / 1e3), cases=per)

    return dict(total_ms=total_ms, per_step_ms=per_step_ms, agg=agg, clocks=clk, e2e_ms=e2e_ms / n_e2e, eo=eo,
                anchor=anchor,
                h2d=h2d, d2h=d2h, fp64=fp64, V=V, per_case=per_case,
                batched=dict(systems=len(L_s), block=wl.get("block"), columns=Lt))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--fp64-full", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-solve", action="store_true",
                    help="with --impl reference: time the oracle's full solve of the first block system")
    ap.add_argument("--cpu-procs", type=int, default=None,
                    help="with --impl reference: at most this many oracle processes")
    ap.add_argument("--eo", dest="eo", action="store_true", default=None,
                    help="solve through the even-odd Schur system (default: the workload's)")
    ap.add_argument("--no-eo", dest="eo", action="store_false")
    ap.add_argument("--prec", choices=["fp32", "fp16"], default=None,
                    help="storage of the inner iterations (default: the workload's, fp32)")
    ap.add_argument("--anchor", type=float, default=None,
                    help="fp64_anchor: replacements between FP64 ones in FP32 (default: the workload's)")
    ap.add_argument("--delta", type=float, default=None,
                    help="residual-replacement threshold (default: the workload's)")
    ap.add_argument("--update", choices=["fp64", "df64"], default=None,
                    help="arithmetic of the residual replacements (default: the workload's)")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    if args.prec:
        wl = dict(wl, prec=args.prec)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    total_rhs_per_step = sum(L for (_, L, _) in wl["cases"])

    if args.impl == "reference":
        if rank != 0:
            return
        # Reference arm: the CPU oracle as it stands.  Each step is one sample
        # (an oracle operator application on the first block system); the
        # steps run concurrently, one process per host core.
        if args.oracle_solve:
            # the full oracle solve of the first block system, one core
            secs, iters, res, (kappa, L) = oracle_full_solve(wl)
            value = L / secs
            sample = (f"one full FP64 numpy-oracle block BiCGGR solve of the first block system ({L} columns, "
                      f"kappa={kappa}, R~0 = R0) to {TOL}: {iters} iterations, {secs:.1f} s, FP64 true residual "
                      f"{res:.1e}; one process, one thread")
            print(json.dumps({
                "impl": "reference", "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": args.gpus,
                "steps": 1, "warmup": 0, "ms_per_step": secs * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl["desc"], "lattice": "x".join(map(str, wl["dims"])),
                           "parallelism": "CPU oracle, 1 process"},
                "cpu_baseline": {"value": value, "unit": "RHS/s", "cores": 1, "kind": "oracle", "sample": sample},
                "e2e": {"value": value, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "host": {"nproc": _host_cores()}}))
            return
        iters = FP64_ITERS_FIRST_SYSTEM.get(args.workload)
        if iters is None:
            raise SystemExit(f"no measured FP64 iteration count for workload {args.workload}; use --oracle-solve")
        secs, procs, (kappa, L) = oracle_samples(wl, args.warmup + args.steps, max_procs=args.cpu_procs)
        timed = secs[args.warmup:] if len(secs) > args.warmup else secs
        value, mean = oracle_rhs_per_s(timed, procs, L, iters)
        sample = (f"one FP64 numpy-oracle application of D_W to the first block system's {L} columns (kappa={kappa}) "
                  f"per step ({mean:.1f} s), {procs} processes on the host cores at once; RHS/s = processes x L / "
                  f"(s x (2 x {iters} + 2)), {iters} = the FP64 block BiCGGR iteration count of that system; the "
                  f"oracle's block algebra is left out")
        line = {
            "impl": "reference", "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["desc"], "lattice": "x".join(map(str, wl["dims"])),
                       "parallelism": f"CPU oracle, {procs} processes"},
            "cpu_baseline": {"value": value, "unit": "RHS/s", "cores": procs, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "host": {"nproc": _host_cores()},
        }
        print(json.dumps(line))
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    # The oracle baseline runs in spawned processes before any GPU work.
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_samples(wl, _host_cores())

    r = gb300_arm(args, wl, rank, world, local_rank)

    total_ms = max_over_ranks(r["total_ms"], world, "cuda")
    value = job_value(world, total_rhs_per_step, args.steps, total_ms)
    agg = r["agg"]
    hbm, peak_kind = measured_peaks()
    achieved = (agg["bytes_inner"] / agg["n_inner"]) / ((agg["t_inner"] / agg["n_inner"]) / 1e3) / 1e9 \
        if agg["n_inner"] else None
    traffic = ncu_traffic(wl["prec"] + ("_eo" if r["eo"] else ""),
                          agg["bytes_inner"] / agg["n_inner"] if agg["n_inner"] else None)
    line = {
        "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "storage": wl["prec"], "data": "synthetic",
        "mixed_precision": ("inner iterations in FP32; residual replacement " +
                            (f"in FP64 after every {r['anchor']:g} of reduction and in FP32 between"
                             if r["anchor"] else "in FP64") + "; FP64 true residual"),
        "formulation": "even-odd Schur system" if r["eo"] else "full system",
        "config": {"workload": wl["desc"], "lattice": "x".join(map(str, wl["dims"])),
                   "rhs_per_step": total_rhs_per_step, "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "l2": "inputs larger than L2 and a 256 MB L2 flush before every timed step"},
        "roofline": {"bound": "hbm",
                     "kernel": (f"k_eo_pair<{wl['prec'].upper()}> (inner Schur operator, both half-lattice launches)"
                                if r["eo"] else f"k_dslash_staged / k_dslash_pair<{wl['prec'].upper()}> "
                                                "(inner operator, all columns)"),
                     "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": (achieved / hbm) if achieved else None, "peak_kind": peak_kind,
                     "traffic": traffic, "launches": agg["n_inner"],
                     "avg_launch_us": agg["t_inner"] / agg["n_inner"] * 1e3 if agg["n_inner"] else None},
        "e2e": {"value": world * total_rhs_per_step / (r["e2e_ms"] / 1e3), "unit": "RHS/s",
                "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"]},
        "gpu_launches": int(agg["launches"]),
        "clocks": r["clocks"],
        "per_case": r["per_case"],
        "batched": r["batched"],
    }
    if r["fp64"]:
        for k, v in r["fp64"].items():
            v["mixed_over_fp64"] = (value / world) / v["rhs_per_s"]
        line["fp64_comparison"] = r["fp64"]
    if cpu is not None:
        secs, procs, (kappa, L) = cpu
        # the oracle solves the full system: its iteration count, not the even-odd one
        iters = FP64_ITERS_FIRST_SYSTEM.get(args.workload) if r["eo"] else \
            ((r["fp64"] or {}).get("same_split", {}).get("iterations_first_system") or
             FP64_ITERS_FIRST_SYSTEM.get(args.workload))
        cv, mean = oracle_rhs_per_s(secs, procs, L, iters)
        line["cpu_baseline"] = {
            "value": cv, "unit": "RHS/s", "cores": procs, "kind": "oracle",
            "sample": f"one FP64 numpy-oracle application of D_W to the first block system's {L} columns "
                      f"(kappa={kappa}, {mean:.1f} s) on each of {procs} host processes at once; RHS/s = processes x "
                      f"L / (s x (2 x {iters} + 2)), {iters} = the FP64 block BiCGGR iteration count of that system "
                      f"on the full system (GB300); the oracle's block algebra is left out"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
