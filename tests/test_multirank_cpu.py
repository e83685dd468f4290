"""Multi-rank logic on CPU: world_size-2 gloo process groups.

Each rank values its shard with the FP64 oracle standing in for its GPU.  The
policy mode uses the partition and the FP64 reduction of the totals that the
benchmark's multi-GPU path runs (``PolicyPartition``); the shards put back
together must equal the single-process result, and the max-over-ranks timing
reduction the benchmark uses must pick the slowest rank.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from paper_1401_1757_gb300.shard import PolicyPartition, policy_shard, projection_steps, scenario_shard


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, mode, out):
    import torch
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_mix(60, seed=4)
    v = synth.vasicek_paths(10, 1200, seed=4)
    if mode == "scenario":
        lo, hi = scenario_shard(v.shape[0], world, rank)
        V0, tot = oracle.reserves_batch(pol, tab, v[lo:hi], nthreads=1)
        full = torch.zeros(v.shape[0], dtype=torch.float64)
        full[lo:hi] = torch.from_numpy(tot)
        dist.all_reduce(full)            # gather for the check only
    else:
        part = PolicyPartition(projection_steps(pol), world, rank)
        V0, tot = oracle.reserves_batch(part.take(pol), tab, v, nthreads=1)
        full = part.reduce_totals(torch.from_numpy(tot), dist)   # partial per-scenario sums
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((full.numpy(), float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["scenario", "policy"])
def test_two_rank_shards_reassemble(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    tab = synth.gm_monthly_survival()
    _, want = oracle.reserves_batch(synth.portfolio_mix(60, seed=4), tab, synth.vasicek_paths(10, 1200, seed=4))
    assert np.allclose(got, want, rtol=1e-13, atol=0)
    assert tmax == 2.0


def test_shard_helpers():
    for n, w in [(1000, 1), (1000, 3), (7, 4), (3, 5)]:
        parts = [scenario_shard(n, w, r) for r in range(w)]
        assert parts[0][0] == 0 and parts[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        assert max(h - l for l, h in parts) - min(h - l for l, h in parts) <= 1
    pol = synth.portfolio_mix(300, seed=4)
    S = projection_steps(pol)
    want = [oracle.steps(int(p), int(a1), int(a2), int(t), 1440)[0] for p, a1, a2, t in
            zip(pol["product"], pol["age1_m"], pol["age2_m"], pol["term_m"])]
    assert S.tolist() == want
    assert projection_steps(pol, horizon=100).max() <= 100
    steps = np.random.default_rng(0).integers(60, 1200, 1001)
    shards = policy_shard(steps, 4)
    assert sorted(np.concatenate(shards).tolist()) == list(range(1001))
    loads = [steps[s].sum() for s in shards]
    assert max(loads) - min(loads) <= steps.max()
