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
