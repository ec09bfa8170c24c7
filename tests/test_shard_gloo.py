"""The multi-rank sampling path on CPU ranks (gloo, world size 2).

Each rank samples its contiguous share of the worlds and one sum all-reduce (plus an
all-gather of the per-world spreads) merges the shares
(``paper_2405_12871_gb300.shard``).  Because worlds are index-addressed and every count
is an integer, the merged result must equal one call over all worlds bit for bit.  The
per-rank sampler here is the oracle (the GPU library's counts equal the oracle's,
which the GPU parity tests check).
"""
import os
import socket
from datetime import timedelta

import numpy as np
import pytest

import oracle
from paper_2405_12871_gb300 import shard, synth


def test_world_range_partitions():
    for theta in (0, 1, 2, 7, 1000, 1001):
        for ws in (1, 2, 3, 8):
            parts = [shard.world_range(theta, r, ws) for r in range(ws)]
            assert sum(c for _, c in parts) == theta
            pos = 0
            for first, cnt in parts:
                assert first == pos and cnt >= 0
                pos += cnt
            assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
    with pytest.raises(ValueError):
        shard.world_range(5, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


CASES = [  # (theta, first, mode, blocked?)
    (1001, 17, 7, False),
    (600, 0, 7, True),
    (3, 5, 1, False),      # fewer worlds than ... per rank: 2 + 1
    (1, 0, 5, False),      # one rank gets no world
]


def _worker(rank, ws, port, results):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws,
                            timeout=timedelta(seconds=120))
    try:
        g, S, cfg = synth.workload_er1k()
        og = oracle.OracleGraph.from_graph(g)
        rng = np.random.default_rng(4)
        B = rng.choice(np.setdiff1d(np.arange(g.n), S), 20, replace=False)
        for ci, (theta, first, mode, blk) in enumerate(CASES):
            got = shard.sample_sharded(og.sample, S, B if blk else (), theta=theta, first=first,
                                       per_world=True, key=3, tag=2, inst=1, mode=mode)
            if rank == 0:
                want = og.sample(S, B if blk else (), theta=theta, key=3, tag=2, inst=1, first=first,
                                 mode=mode, per_world=True)
                for k in ("reach", "credit_lower", "credit_upper"):
                    assert np.array_equal(got[k], want[k]), (ci, k)
                for k in ("total_spread", "edges_scanned", "nonempty_lrr"):
                    assert got[k] == want[k], (ci, k, got[k], want[k])
                assert np.array_equal(got["world_spread"], want["world_spread"]), ci
        if rank == 0:
            results.put("ok")
    finally:
        dist.destroy_process_group()


def test_sharded_sampling_matches_one_rank():
    import torch.multiprocessing as mp
    oracle.lib()                      # build the oracle once, before the ranks start
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_worker, args=(2, _free_port(), q), nprocs=2, join=True, start_method="spawn")
    assert q.get() == "ok"


def _gpu_worker(rank, ws, port, results):
    import torch
    import torch.distributed as dist
    from gpu_common import gpu_ctx
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws,
                            timeout=timedelta(seconds=180))
    try:
        torch.cuda.set_device(0)
        c = gpu_ctx()
        g, S, cfg = synth.workload_er1k()
        G = c.load_graph(g)
        got = shard.sample_sharded(G.sample, S, (), theta=2001, first=9, per_world=True, key=5, tag=1,
                                   mode=7)
        if rank == 0:
            want = oracle.OracleGraph.from_graph(g).sample(S, (), theta=2001, key=5, tag=1, first=9, mode=7,
                                                          per_world=True)
            for k in ("reach", "credit_lower", "credit_upper"):
                assert np.array_equal(got[k], want[k]), k
            for k in ("total_spread", "edges_scanned", "nonempty_lrr"):
                assert got[k] == want[k], k
            assert np.array_equal(got["world_spread"], want["world_spread"])
            results.put("ok")
        G.free()
        c.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
def test_sharded_gpu_sampling_two_ranks_one_gpu():
    """Two ranks on one GPU, each sampling its share through the library (independent
    launches, no kernel waits on another), merged over gloo: equal to the oracle."""
    import torch.multiprocessing as mp
    oracle.lib()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_gpu_worker, args=(2, _free_port(), q), nprocs=2, join=True, start_method="spawn")
    assert q.get() == "ok"


def test_collective_buffers_follow_the_backend(monkeypatch):
    """Under NCCL the merge buffers go to the rank's CUDA device (NCCL moves device
    memory only); under gloo they stay on the host."""
    import torch
    import torch.distributed as dist
    monkeypatch.setattr(dist, "get_backend", lambda group=None: "nccl")
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 3)
    assert shard.collective_device() == torch.device("cuda", 3)
    monkeypatch.setattr(dist, "get_backend", lambda group=None: "gloo")
    assert shard.collective_device() == torch.device("cpu")


def _world_sets(seed=5, worlds=120):
    """CP sets (dominator chains, Algorithm 2) and LRR sets (Algorithm 3) of explicit
    worlds of a small graph, built from the oracle's one-world routine."""
    g = synth.erdos_renyi(300, 1500, seed=seed)
    S = synth.seeds_uniform(g.n, 4, seed=seed + 1)
    og = oracle.OracleGraph.from_graph(g)
    Vs = og.vs(S)
    cp, lrr = [], []
    for j in range(worlds):
        live = np.array([og.edge_live(e, 3, j, 1) for e in range(g.m)], np.uint8)
        t = int(Vs[oracle.target_index(3, j, 1, 0, len(Vs))])
        w = og.world_explicit(live, S, target=t)
        seeds = set(int(s) for s in S)
        for v in np.flatnonzero(w["reached"]):
            if int(v) in seeds:
                continue
            chain, cur = [], int(v)
            while cur >= 0 and cur not in seeds:
                chain.append(cur)
                cur = int(w["idom"][cur])
            cp.append(chain)
        lr = [int(x) for x in np.flatnonzero(w["lrr"])]
        if lr:
            lrr.append(lr)
    return g.n, cp, lrr


def _csr(sets):
    off = np.zeros(len(sets) + 1, np.int64)
    for i, s in enumerate(sets):
        off[i + 1] = off[i] + len(s)
    elem = np.concatenate([np.asarray(s, np.int64) for s in sets]) if sets else np.zeros(0, np.int64)
    return off, elem


def _greedy_worker(rank, ws, port, results):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws,
                            timeout=timedelta(seconds=120))
    try:
        rng = np.random.default_rng(8)
        n = 400
        rand_sets = [list(rng.choice(n, int(rng.integers(1, 12)), replace=False)) for _ in range(2000)]
        n2, cp, lrr = _world_sets()
        for ci, (nn, sets, k) in enumerate(((n, rand_sets, 25), (n2, cp, 10), (n2, lrr, 10),
                                            (n2, lrr[:3], 10))):
            # the shards: an uneven split of the sets in order (a rank's world range)
            cut = (len(sets) * 2) // 5
            mine = sets[:cut] if rank == 0 else sets[cut:]
            off, elem = _csr(mine)
            B, cov, topk = shard.max_coverage_sharded(off, elem, nn, k)
            wB, wcov, wtopk = oracle.max_coverage_sets(sets, nn, k)
            assert np.array_equal(B, wB), (ci, B, wB)
            assert np.array_equal(cov, wcov), ci
            assert np.array_equal(topk, wtopk), ci
        if rank == 0:
            results.put("ok")
    finally:
        dist.destroy_process_group()


def test_sharded_max_coverage_matches_one_rank():
    """Max-Coverage over sets split across two ranks, with one gain all-reduce per
    round, picks the same blockers with the same Cov(B_i) and top-k sums as one
    Max-Coverage over all sets (random set systems, the CP and LRR sets of explicit
    worlds, and a case that stops early at zero gain)."""
    import torch.multiprocessing as mp
    oracle.lib()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_greedy_worker, args=(2, _free_port(), q), nprocs=2, join=True, start_method="spawn")
    assert q.get() == "ok"
