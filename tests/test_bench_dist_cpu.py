"""The multi-process path of bench.py on CPU (gloo, world size 2): the
timing reduction takes the slowest rank, the barrier holds, each rank gets
its own start-block seed, and the CPU reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys
sys.path.insert(0, os.environ["BENCH_ROOT"])
import torch.distributed as dist
import bench, synth
dist.init_process_group("gloo")
r = dist.get_rank()
bench.rank_barrier(dist)
m = bench.reduce_max(dist, 10.0 + r, "cpu")
seeds = [None, None]
dist.all_gather_object(seeds, bench.instance_seed(synth.W2D_N256, r))
print("RESULT", r, m, seeds[0] != seeds[1], flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_reduction_and_seeds():
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), BENCH_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True))
    outs = [p.communicate(timeout=120)[0] for p in procs]
    for r, (p, out) in enumerate(zip(procs, outs)):
        assert p.returncode == 0, out
        line = [x for x in out.splitlines() if x.startswith("RESULT")][-1].split()
        assert int(line[1]) == r
        assert float(line[2]) == 11.0          # the slowest rank's time
        assert line[3] == "True"               # independent instances


def test_reference_arm_prints_on_rank0_only(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        gpus, steps, warmup, cpu_iters = 2, 1, 0, 1
    bench.run_reference(A())
    assert capsys.readouterr().out == ""


def test_reference_arm_json_contract(capsys, monkeypatch):
    """Rank 0 of the CPU reference arm prints exactly one JSON line with the
    keys the benchmark contract names, on the same metric, unit and workload
    as the GPU arm; one oracle iteration keeps it short."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")

    class A:
        gpus, steps, warmup, cpu_iters = 1, 1, 0, 1
    bench.run_reference(A())
    lines = [x for x in capsys.readouterr().out.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["config"]["workload"] == bench.W.name and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] > 0 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
