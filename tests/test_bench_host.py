"""Host logic of bench.py on the CPU: the replicas' timing over ranks (two gloo processes, as
torchrun launches them), the whole-job throughput, the reference arm's non-zero ranks, and the
algorithmic byte count of the FGMRES vector kernels against a count by hand."""
import importlib.util
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import importlib.util, os, sys
import torch.distributed as dist
spec = importlib.util.spec_from_file_location("bench", os.path.join(sys.argv[1], "bench.py"))
b = importlib.util.module_from_spec(spec); spec.loader.exec_module(b)
rank, local_rank, world = b.dist_env()
dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
ms = b.max_over_ranks(100.0 + 25.0 * rank, dist)
dist.barrier()
print("RESULT", rank, world, ms, b.replica_throughput(world, 1_000_000, ms))
dist.destroy_process_group()
"""


def test_max_over_ranks_gloo():
    """Two ranks with step times 100 and 125 ms both report 125 ms; 2 replicas of 1M DoFs at
    125 ms are 0.016 GDoF/s."""
    pytest.importorskip("torch.distributed")
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append([line for line in out.splitlines() if line.startswith("RESULT")][0].split())
    for _, rank, world, ms, gdofs in outs:
        assert int(world) == 2
        assert float(ms) == 125.0
        assert abs(float(gdofs) - 0.016) < 1e-15


def test_max_over_ranks_single_process():
    b = load_bench()
    assert b.max_over_ranks(7.5) == 7.5
    assert abs(b.replica_throughput(1, 6_714_692, 559.0) - 6_714_692 / 0.559 / 1e9) < 1e-15


def test_reference_arm_other_ranks_exit_quietly(monkeypatch, capsys):
    """Under torchrun only rank 0 runs the oracle and prints; rank 1 returns without output."""
    b = load_bench()
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        workload, steps, warmup = "cube64", 1, 0
    b.run_reference(Args())
    assert capsys.readouterr().out == ""


def test_krylov_bytes_by_hand():
    """restart 2, 3 iterations, N = 1: cycle 1 (2 iterations) + cycle 2 (1 iteration).
    Delayed passes: |b| 1; cycle: 6 + per k (2k + 6) + (kc + 2): 6 + 8 + 10 + 4 = 28, then
    6 + 8 + 3 = 17; final residual 4: 1 + 28 + 17 + 4 = 50 vectors. Three passes add (k + 2) per
    k < m and one more vector per k: 1 + (6 + 7 + 3 + 9 + 4) + (6 + 7 + 3 + 3) + 4 = 53."""
    b = load_bench()
    assert b.krylov_alg_bytes(1, 3, 2, delayed=True) == 8 * 50
    assert b.krylov_alg_bytes(1, 3, 2, delayed=False) == 8 * 53
