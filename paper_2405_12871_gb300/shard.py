"""Sharding of the sampling step across ranks (one process per GPU).

Worlds are addressed by index (a world's coins depend only on the key, the stream tag
and instance, and the world index j; Sec. 2.1 live-edge worlds), so a call over worlds
[first, first + theta) splits into contiguous sub-ranges with no communication.  Each
rank samples its own range with the library; one sum all-reduce then merges:

* the per-node count vectors (reach, credit_lower, credit_upper): integers, so the sum
  does not depend on the split or on the reduction order;
* the scalar totals (total spread, edges scanned, non-empty LRR sets);
* the per-world spreads, gathered in world order.

Max-Coverage over sample stores sharded the same way exchanges one gain vector per
round (``max_coverage_sharded``).  Collective buffers live on the rank's GPU under
NCCL and on the host under gloo.  On a box with one GPU per query this runs as
independent replicas (``bench.py --gpus N``); the merge and exchange logic is
exercised with CPU ranks over the ``gloo`` backend.
"""
from __future__ import annotations

import numpy as np

COUNT_KEYS = ("reach", "credit_lower", "credit_upper")
SCALAR_KEYS = ("total_spread", "edges_scanned", "nonempty_lrr")


def world_range(theta: int, rank: int, world_size: int):
    """(first offset, count) of this rank's contiguous share of [0, theta): the first
    theta % world_size ranks take one extra world."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("bad rank / world size")
    if theta < 0:
        raise ValueError("negative theta")
    base, extra = divmod(int(theta), world_size)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def collective_device(group=None):
    """Where a collective buffer must live: the rank's current CUDA device under NCCL
    (which only moves device memory), the host under gloo."""
    import torch
    import torch.distributed as dist

    if dist.get_backend(group) == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def sample_sharded(sample, S, blocked=(), theta=1, first=0, per_world=False, group=None, **kw):
    """Run ``sample(S, blocked, theta=count, first=first + offset, per_world=..., **kw)``
    (for instance ``Graph.sample``) on this rank's share of the worlds and merge the
    results of all ranks of ``group`` (``torch.distributed``).  Every rank returns the
    merged result, equal bit for bit to one call over all ``theta`` worlds."""
    import torch
    import torch.distributed as dist

    ws = dist.get_world_size(group)
    rank = dist.get_rank(group)
    dev = collective_device(group)
    off, cnt = world_range(theta, rank, ws)
    part = sample(S, blocked, theta=cnt, first=int(first) + off, per_world=per_world, **kw)
    out = {}
    keys = [k for k in COUNT_KEYS if k in part]
    # one all-reduce: the count vectors and the scalars in one int64 buffer (every
    # count is far below 2^63)
    n = len(part[keys[0]]) if keys else 0
    buf = np.zeros(len(keys) * n + len(SCALAR_KEYS), dtype=np.int64)
    for i, k in enumerate(keys):
        buf[i * n:(i + 1) * n] = np.asarray(part[k], dtype=np.uint64).astype(np.int64)
    for i, k in enumerate(SCALAR_KEYS):
        buf[len(keys) * n + i] = int(part.get(k, 0))
    t = torch.from_numpy(buf).to(dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    buf = t.cpu().numpy()
    for i, k in enumerate(keys):
        out[k] = buf[i * n:(i + 1) * n].astype(np.uint64)
    for i, k in enumerate(SCALAR_KEYS):
        out[k] = int(buf[len(keys) * n + i])
    if per_world:
        # every rank's spreads, in world order (ranks hold consecutive ranges)
        ws_local = torch.from_numpy(np.asarray(part["world_spread"], dtype=np.int64))
        sizes = [world_range(theta, r, ws)[1] for r in range(ws)]
        pad = torch.zeros(max(sizes), dtype=torch.int64)
        pad[:cnt] = ws_local
        pad = pad.to(dev)
        gathered = [torch.zeros_like(pad) for _ in range(ws)]
        dist.all_gather(gathered, pad, group=group)
        out["world_spread"] = np.concatenate(
            [g.cpu().numpy()[:s] for g, s in zip(gathered, sizes)]).astype(np.uint32)
    return out


def max_coverage_sharded(off, elem, n, k, group=None):
    """Procedure Max-Coverage (Algorithm 4) over a collection of sets that is sharded
    across the ranks of ``group``: this rank holds sets ``elem[off[i]:off[i+1]]``
    (node ids in [0, n)), e.g. the CP or LRR sets of its own world range.

    Each round exchanges one sum all-reduce of the per-node gains (the number of this
    rank's uncovered sets that contain the node), so that every rank sees the global
    marginal coverage and picks the same node: the largest gain, ties to the smaller
    id, no pick at zero gain.  Each rank then covers its own sets that contain the
    pick and lowers its local gains.  Returns (B, cov, topk) with cov[i] = Cov(B_i)
    and topk[i] the sum of the k largest global gains in state B_i -- on every rank,
    equal to one Max-Coverage over the union of the shards."""
    import torch
    import torch.distributed as dist

    dev = collective_device(group)
    off = np.asarray(off, dtype=np.int64)
    elem = np.asarray(elem, dtype=np.int64)
    nsets = off.shape[0] - 1
    gain = np.bincount(elem, minlength=n).astype(np.int64)
    # inverted index node -> local sets
    set_of = np.repeat(np.arange(nsets, dtype=np.int64), np.diff(off))
    order = np.argsort(elem, kind="stable")
    inv_sets = set_of[order]
    inv_off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(elem, minlength=n), out=inv_off[1:])
    covered = np.zeros(max(nsets, 1), dtype=bool)
    B, cov, topk = [], [0], []
    for i in range(k + 1):
        t = torch.from_numpy(gain.copy()).to(dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        g = t.cpu().numpy()
        topk.append(int(np.sort(g)[::-1][:k].sum()))
        if i == k:
            break
        u = int(np.argmax(g))              # first index of the maximum: ties to the smaller id
        if g[u] <= 0:
            break
        B.append(u)
        cov.append(cov[-1] + int(g[u]))
        for s in inv_sets[inv_off[u]:inv_off[u + 1]]:
            if covered[s]:
                continue
            covered[s] = True
            np.subtract.at(gain, elem[off[s]:off[s + 1]], 1)
    return (np.asarray(B, dtype=np.int32), np.asarray(cov, dtype=np.uint64),
            np.asarray(topk, dtype=np.uint64))
