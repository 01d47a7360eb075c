"""The bench's host-side contract, on the CPU.

* The reference arm (the FP64 oracle on the host, run as it stands) prints
  one JSON line with the keys the bench line carries, with value =
  lattice cells x steps / time.
* Launched as two ranks, only rank 0 runs it and prints; rank 1 exits 0
  without work.
* The timing of the replicas (one simulation per GPU, no exchange between
  them): every timed region ends with a barrier and the slowest rank's
  time, so two gloo ranks with different times both report the larger.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def _run_reference(env_extra, steps=2):
    env = dict(os.environ, **env_extra)
    env.pop("CUDA_VISIBLE_DEVICES", None)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps",
                           str(steps), "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=300)


def test_reference_arm_line(oracle_mod):
    r = _run_reference({})
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert KEYS <= set(d)
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 0 and d["value"] > 0
    # value = cells x steps / time, with the time the line reports
    n = 48 ** 3
    assert abs(d["value"] - n / (d["ms_per_step"] * 1e-3) / 1e6) <= 1e-9 * d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_rank1_is_silent(oracle_mod):
    r = _run_reference({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def _ranks(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        bench.barrier(world)
        out[rank] = bench.reduce_max(1.5 + rank, world)
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank():
    mp = pytest.importorskip("torch.multiprocessing")
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_ranks, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 2.5
