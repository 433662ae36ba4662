"""Multi-rank host logic on CPU (no GPU): the work partition of a cell batch over ranks, two gloo
ranks running the benchmark's distributed helpers and the diagnostics all-reduce, and the
benchmark's reference arm launched as two ranks.  The homogeneous data path exchanges nothing:
cells are independent, so each rank only evaluates its own.  The spatially inhomogeneous coupling
does exchange one halo cell per neighbour and step; its split over two and three gloo ranks is
checked against the oracle's global run."""
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


# ------------------------- spatially inhomogeneous coupling split over ranks (halo exchange) ----

def _halo_case():
    import oracle
    M, N, T, dx, dt, steps = 11, 8, 4.0, 0.5, 0.05, 3
    G = np.random.default_rng(7).uniform(0.1, 1.0, size=(M, N, N))
    p = oracle.Params(d=2, N=N, T=T, kernel=oracle.KERNEL_MAXWELL, R=16)
    return oracle, G, p, T, dx, dt, steps


def _halo_block(world, rank, group=None):
    """This rank's block of the global state after the split Lie steps (the oracle's transport and
    Euler step as the local operators), and the same block of the oracle's global run."""
    import torch
    oracle, G, p, T, dx, dt, steps = _halo_case()
    start, n = shard.spatial_blocks(G.shape[0], world)[rank]
    F_ext = torch.zeros((n + 2,) + G.shape[1:], dtype=torch.float64)
    F_ext[1:n + 1] = torch.from_numpy(G[start:start + n])
    S = torch.full_like(F_ext, float("nan"))

    def transport(a, b):
        b.copy_(torch.from_numpy(oracle.transport_upwind(a.numpy(), T, dx, dt)))

    def collide(v):
        v.copy_(torch.from_numpy(np.stack([oracle.euler(p, c, dt) for c in v.numpy()])))

    out = shard.lie_steps_sharded(F_ext, S, steps, transport, collide, group)
    ref = oracle.inhomogeneous_lie(p, G, dx, dt, steps=steps)[start:start + n]
    return out[1:n + 1].numpy(), ref


def test_spatial_blocks_are_contiguous_and_balanced():
    for M, world in ((11, 1), (11, 2), (11, 3), (64, 8), (8, 8)):
        b = shard.spatial_blocks(M, world)
        assert [s for s, _ in b] == list(np.cumsum([0] + [n for _, n in b])[:-1])
        assert sum(n for _, n in b) == M and max(n for _, n in b) - min(n for _, n in b) <= 1
    with pytest.raises(ValueError):
        shard.spatial_blocks(3, 4)


def test_split_lie_steps_single_rank_wraps_onto_itself():
    got, ref = _halo_block(1, 0)
    assert np.array_equal(got, ref)


def _halo_rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method="tcp://127.0.0.1:%d" % port)
    got, ref = _halo_block(world, rank)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "halo%d.json" % rank), "w") as f:
        json.dump({"equal": bool(np.array_equal(got, ref)), "n": int(got.shape[0])}, f)


@pytest.mark.parametrize("world", [2, 3])
def test_split_lie_steps_over_gloo_ranks_equal_the_global_run(tmp_path, world):
    """Blocks of an 11-cell periodic grid on two and three gloo ranks, three Lie steps with halo
    exchanges: every rank's cells equal the oracle's global run bit for bit."""
    mp = pytest.importorskip("torch.multiprocessing")
    mp.spawn(_halo_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    total = 0
    for r in range(world):
        with open(tmp_path / ("halo%d.json" % r)) as f:
            d = json.load(f)
        assert d["equal"], r
        total += d["n"]
    assert total == 11
