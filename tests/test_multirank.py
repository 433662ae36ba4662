"""Multi-rank host logic on CPU (no GPU): the work partition of a cell batch over ranks, two gloo
ranks running the benchmark's distributed helpers and the diagnostics all-reduce, and the
benchmark's reference arm launched as two ranks.  The data path itself exchanges nothing: cells
are independent, so each rank only evaluates its own."""
import itertools
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from paper_1704_07369_gb300 import inputs, shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_partition_covers_every_cell_once_and_balances():
    Ns = inputs.ragged_sizes(4096, seed=1234)
    for world in (1, 2, 3, 8):
        parts = shard.partition(Ns, world)
        assert len(parts) == world
        assert np.array_equal(np.sort(np.concatenate(parts)), np.arange(len(Ns)))
        ld = shard.loads(Ns, parts)
        assert max(ld) <= 1.01 * sum(ld) / world
    again = shard.partition(Ns, 4)
    assert all(np.array_equal(a, b) for a, b in zip(shard.partition(Ns, 4), again))


def test_partition_within_graham_bound_of_the_optimum():
    """Longest-processing-time-first: the heaviest rank is at most 4/3 of the best split, checked
    against brute force over every assignment of a small batch."""
    Ns = np.array([48, 48, 40, 40, 32, 32, 24, 24, 24])
    c = [shard.cell_cost(int(n)) for n in Ns]
    for world in (2, 3):
        best = min(max(sum(ci for ci, r in zip(c, a) if r == k) for k in range(world))
                   for a in itertools.product(range(world), repeat=len(Ns)))
        got = max(shard.loads(Ns, shard.partition(Ns, world)))
        assert got <= 4.0 / 3.0 * best + 1e-9


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench

    class Args:
        impl = "reference"      # the gloo path of the benchmark's set-up

    w, r, _ = bench.dist_setup(Args)
    Ns = inputs.ragged_sizes(64, seed=1234)
    parts = shard.partition(Ns, w)
    mine = torch.tensor(parts[r], dtype=torch.float64)
    diag = torch.zeros(len(mine), 10, dtype=torch.float64)
    diag[:, 0] = mine + 1          # cell i carries "mass" i + 1
    diag[:, 7] = mine              # min F
    diag[:, 8] = mine              # max nu
    diag[:, 9] = -mine             # min of the output
    g = shard.allreduce_diagnostics(diag)
    bench.barrier(w)
    t = bench.max_over_ranks(w, float(r + 1))
    sizes = torch.tensor([len(p) for p in parts], dtype=torch.int64)
    every = [torch.zeros_like(sizes) for _ in range(w)]
    dist.all_gather(every, sizes)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.json" % r), "w") as f:
        json.dump({"world": w, "mass": float(g[0]), "min": float(g[7]), "max": float(g[8]), "minout": float(g[9]),
                   "t": t, "agree": all(torch.equal(e, sizes) for e in every)}, f)


def test_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        with open(tmp_path / ("rank%d.json" % r)) as f:
            d = json.load(f)
        assert d["world"] == 2 and d["agree"]
        assert d["mass"] == sum(range(1, 65))
        assert (d["min"], d["max"], d["minout"]) == (0.0, 63.0, -63.0)
        assert d["t"] == 2.0


def test_bench_reference_arm_as_two_ranks():
    """torchrun with two ranks: rank 0 alone runs the oracle and prints the one JSON line."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
