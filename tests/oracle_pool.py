"""The oracle's world loop split over host processes, for full-size parity checks.

Worlds are index-addressed, so a range [first, first + theta) splits into contiguous
sub-ranges that separate processes sample independently; the integer count vectors
are summed and the per-world spreads concatenated in world order.  Each process runs
the unchanged oracle on its own copy of the graph (loaded from a memory-mapped file).
The pool is started with ``spawn``: a forked child of a process that holds a CUDA
context can hang.
"""
import multiprocessing as mp
import os
import tempfile

import numpy as np

_G = None


def _init(path, n):
    global _G
    import oracle
    from paper_2405_12871_gb300 import synth
    z = np.load(path, mmap_mode="r")
    _G = oracle.OracleGraph.from_graph(synth.Graph(n, np.array(z["row_ptr"]), np.array(z["col"]),
                                                   np.array(z["prob"])))


def _job(args):
    S, B, first, theta, kw = args
    return first, _G.sample(S, B, theta=theta, first=first, per_world=True, **kw)


def sample_parallel(g, S, blocked=(), theta=1, first=0, procs=None, chunk=None, **kw):
    """oracle.OracleGraph(g).sample(S, blocked, theta, first=first, per_world=True, **kw),
    computed over `procs` processes."""
    procs = procs or min(16, os.cpu_count() or 1)
    chunk = chunk or max(1, -(-theta // (4 * procs)))
    tmp = tempfile.mkdtemp(prefix="oracle_pool_")
    path = os.path.join(tmp, "g.npz")
    np.savez(path, row_ptr=g.row_ptr, col=g.col, prob=g.prob)
    S = np.asarray(S, np.int32)
    B = np.asarray(blocked, np.int32)
    jobs = [(S, B, first + a, min(chunk, theta - a), kw) for a in range(0, theta, chunk)]
    try:
        with mp.get_context("spawn").Pool(procs, initializer=_init, initargs=(path, g.n)) as pool:
            parts = sorted(pool.map(_job, jobs), key=lambda x: x[0])
    finally:
        os.unlink(path)
        os.rmdir(tmp)
    out = {}
    for k in ("reach", "credit_lower", "credit_upper"):
        out[k] = np.sum([p[k] for _, p in parts], axis=0, dtype=np.uint64)
    for k in ("total_spread", "edges_scanned", "nonempty_lrr"):
        out[k] = int(sum(p[k] for _, p in parts))
    out["world_spread"] = np.concatenate([p["world_spread"] for _, p in parts])
    return out
