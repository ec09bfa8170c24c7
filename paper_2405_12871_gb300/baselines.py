"""The dominator-tree baselines the paper compares against: AdvancedGreedy (AG) and
GreedyReplace (GR) of Xie et al., as the paper describes them (Sec. 2.3, "Dominator
tree based estimation" and the AG / GR paragraph after Example 2.1).

Both rest on one estimate: with the seeds merged into a unified source s, the expected
number of nodes that blocking v protects, given blockers B, equals the expected size of
v's subtree in the dominator tree of a live-edge world of G[V \\ B].  It is estimated
as the average subtree size over theta fresh worlds, which is the per-node lower-bound
credit of ``imin_sample`` (mode ``IMIN_CREDIT_LOWER``) divided by theta.

* AG: k times, estimate with the current B and add the node of largest estimate.
* GR: first fill B from the out-neighbours of the seeds the same way, up to
  min(|ON|, k) nodes; then, in reverse insertion order, take each blocker out, put back
  the node of largest estimate over V \\ S, and stop as soon as that node is the one
  just taken out.

Every estimate draws new worlds (the baselines re-sample after each change of B):
estimate number i uses worlds [i * theta, (i + 1) * theta) of stream tag 8, which the
solve never uses.  Ties go to the smaller node id.  ``sample`` is ``Graph.sample``
of the library (or any function with its signature and results).
"""
from __future__ import annotations

import numpy as np

TAG = 8
MODE_LOWER = 2


class _Estimator:
    def __init__(self, sample, n, S, theta, key):
        self.sample, self.n, self.theta, self.key = sample, int(n), int(theta), int(key)
        self.S = np.asarray(S, dtype=np.int32)
        self.calls = 0
        self.worlds = 0

    def credits(self, B):
        """Summed subtree sizes over theta fresh worlds of G[V \\ B] (uint64[n])."""
        r = self.sample(self.S, np.asarray(sorted(B), dtype=np.int32), theta=self.theta, key=self.key,
                        tag=TAG, first=self.calls * self.theta, mode=MODE_LOWER)
        self.calls += 1
        self.worlds += self.theta
        return np.asarray(r["credit_lower"], dtype=np.uint64)

    def best(self, B, allowed=None):
        """The node of largest estimate among `allowed` (default V \\ S \\ B), smaller id
        on ties; None when every estimate is zero."""
        c = self.credits(B).astype(np.float64)
        mask = np.ones(self.n, dtype=bool)
        mask[self.S] = False
        if B:
            mask[np.asarray(sorted(B))] = False
        if allowed is not None:
            keep = np.zeros(self.n, dtype=bool)
            keep[np.asarray(allowed, dtype=np.int64)] = True
            mask &= keep
        c[~mask] = -1.0
        v = int(np.argmax(c))            # first maximum = smallest id
        return v if c[v] > 0 else None


def out_neighbours(row_ptr, col, prob, S):
    """ON: out-neighbours of the seeds over edges of nonzero probability, seeds excluded."""
    S = set(int(s) for s in S)
    on = set()
    for s in S:
        for e in range(int(row_ptr[s]), int(row_ptr[s + 1])):
            if prob[e] > 0 and int(col[e]) not in S:
                on.add(int(col[e]))
    return sorted(on)


def advanced_greedy(sample, n, S, k, theta, key=0):
    """AG: returns (blockers in selection order, number of estimates, worlds drawn)."""
    est = _Estimator(sample, n, S, theta, key)
    B = []
    for _ in range(int(k)):
        v = est.best(B)
        if v is None:
            break
        B.append(v)
    return B, est.calls, est.worlds


def greedy_replace(sample, graph, S, k, theta, key=0):
    """GR on ``graph`` (row_ptr, col, prob, n): returns (blockers in insertion order,
    number of estimates, worlds drawn)."""
    est = _Estimator(sample, graph.n, S, theta, key)
    on = out_neighbours(graph.row_ptr, graph.col, graph.prob, S)
    B = []
    target = min(len(on), int(k))
    while len(B) < target:                       # stage 1: candidates = ON
        v = est.best(B, allowed=[u for u in on if u not in B])
        if v is None:
            break
        B.append(v)
    for b in list(reversed(B)):                  # stage 2: replacement, newest first
        rest = [u for u in B if u != b]
        v = est.best(rest)
        if v is None or v == b:
            break
        B = rest + [v]
    return B, est.calls, est.worlds
