"""Reference computations on ONE explicit live-edge world, written directly
from the paper's definitions (not from its algorithms), for pinning the oracle.

* reach(S, blocked): nodes reachable from S in phi (Sec. 2.1), by BFS.
* N_phi(v): nodes active without blockers that turn inactive when only v is
  blocked (Sec. 3.2, definition of the lower bound) -- by deleting v.
* M_phi(B): nodes reachable from B inside phi^s, the live subgraph induced on
  R_phi(s) \\ S (Sec. 3.3) -- by forward BFS from B.
* L_phi(t): nodes of phi^s that reach t (Def. 4.2) -- by a forward BFS from
  every candidate (the oracle walks backwards instead).
"""
from collections import deque

import numpy as np


def live_adj(n, src, dst, live):
    adj = [[] for _ in range(n)]
    for e in np.flatnonzero(live):
        adj[int(src[e])].append(int(dst[e]))
    return adj


def reach(adj, S, blocked=()):
    blocked = set(int(b) for b in blocked)
    seen = set()
    dq = deque()
    for s in S:
        s = int(s)
        if s not in seen:
            seen.add(s)
            dq.append(s)
    while dq:
        u = dq.popleft()
        for v in adj[u]:
            if v in blocked or v in seen:
                continue
            seen.add(v)
            dq.append(v)
    return seen


def N_phi(adj, S, v):
    base = reach(adj, S)
    if v not in base or v in set(int(s) for s in S):
        return set()
    return base - reach(adj, S, blocked=[v])


def M_phi(adj, S, B):
    R = reach(adj, S)
    Sset = set(int(s) for s in S)
    inner = R - Sset
    seen = set(b for b in (int(x) for x in B) if b in inner)
    dq = deque(seen)
    while dq:
        u = dq.popleft()
        for v in adj[u]:
            if v in inner and v not in seen:
                seen.add(v)
                dq.append(v)
    return seen


def L_phi(adj, S, t):
    R = reach(adj, S)
    Sset = set(int(s) for s in S)
    inner = R - Sset
    if t not in inner:
        return set()
    out = set()
    for u in inner:
        if t in M_phi(adj, S, [u]):
            out.add(u)
    return out


def enumerate_worlds(p):
    """All 2^m live-edge worlds with their probabilities (Eq. 1).  p must be
    dyadic with few bits so that every weight and sum is exact in float64."""
    m = len(p)
    p = np.asarray(p, dtype=np.float64)
    for mask in range(1 << m):
        live = np.array([(mask >> e) & 1 for e in range(m)], dtype=np.uint8)
        wgt = float(np.prod(np.where(live == 1, p, 1.0 - p)))
        if wgt > 0.0:
            yield live, wgt


def tiny_graph(seed, n_lo=4, n_hi=8, m_max=12, probs=(0.25, 0.5, 0.75, 1.0)):
    """A small random digraph (no self-loops, no duplicates) with dyadic p."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(n_lo, n_hi + 1))
    pairs = [(u, v) for u in range(n) for v in range(n) if u != v]
    m = int(rng.integers(n, min(m_max, len(pairs)) + 1))
    pick = rng.choice(len(pairs), m, replace=False)
    src = np.array([pairs[i][0] for i in pick])
    dst = np.array([pairs[i][1] for i in pick])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    p = np.asarray(probs, dtype=np.float32)[rng.integers(0, len(probs), m)]
    return n, src, dst, p
