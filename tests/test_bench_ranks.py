"""The benchmark's multi-rank host logic on CPU (gloo, world size 2): the
timed milliseconds reduce to the slowest rank on every rank, the whole-job
value counts every replica's right-hand sides, and replicas draw different
sources."""
import importlib.util
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, local_ms, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    out[rank] = b.max_over_ranks(local_ms[rank], world, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    local_ms = [1234.5, 987.25]
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, local_ms, out), nprocs=world, join=True)
        got = dict(out)
    assert got == {0: 1234.5, 1: 1234.5}
    b = _bench()
    # 2 replicas x 180 RHS x 3 steps in the slowest rank's 1234.5 ms
    assert b.job_value(world, 180, 3, got[0]) == pytest.approx(2 * 180 * 3 / 1.2345)
    assert b.max_over_ranks(5.0, 1, "cpu") == 5.0


def test_replicas_draw_different_sources():
    import synth
    b = _bench()
    dims = (2, 2, 2, 2)
    s0 = synth.z2_noise(dims, 4, b.replica_seed(4, 0))
    s1 = synth.z2_noise(dims, 4, b.replica_seed(4, 1))
    assert not np.array_equal(s0, s1)
    assert b.replica_seed(48, 0) == 2048


def test_reference_arm_runs_on_cpu():
    """bench.py --impl reference: the FP64 oracle timed on the host, one JSON
    line with the contract's keys (8^3 x 16 workload, one short step)."""
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c2",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600, check=True)
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "RHS/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["higher_is_better"] is True


def test_roofline_traffic_scales_the_capture(tmp_path, monkeypatch):
    """roofline.traffic = captured DRAM / algorithmic bytes x this run's bytes
    per launch, and None once the operator sources differ from the capture's."""
    import json
    b = _bench()
    d = json.load(open(os.path.join(ROOT, "profiles", "dslash_traffic.json")))
    assert d["captures"]
    for kind, c in d["captures"].items():
        if d["source_hash"] == b.source_hash():
            assert b.ncu_traffic(kind, 2e9) == pytest.approx(c["dram_bytes"] / c["alg_bytes"] * 2e9)
    monkeypatch.setattr(b, "source_hash", lambda: "0000")
    for kind in d["captures"]:
        assert b.ncu_traffic(kind, 2e9) is None
    assert b.ncu_traffic("no such capture", 2e9) is None
