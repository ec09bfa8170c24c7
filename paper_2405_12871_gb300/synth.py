"""Seeded synthetic inputs: directed graphs with per-edge probabilities, and seed sets.

This module builds workloads only.  It holds none of the influence-minimisation
arithmetic (no coins, no traversal, no estimators), so that both the CUDA path
and the CPU oracle can take their inputs from it without sharing any of the
method's code.

Probability model (Section 6, parameter settings): weighted cascade,
p(u, v) = 1 / indeg(v), computed in fp32 as ``1.0f / (float) indeg(v)``; the
R-MAT workload instead draws each p uniformly from {0.1, 0.01, 0.001}
("trivalency").  The paper's SNAP graphs are not available; the generators
below stand in for them with the same probability model.

Every draw comes from numpy's Philox bit generator, keyed by an explicit
integer seed (graph seed 1, query seed 2 by convention), so the same call
gives the same bytes on every platform.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


@dataclasses.dataclass
class Graph:
    """Directed graph in CSR-by-source form.

    row_ptr: int32[n+1]; col: int32[m] (targets, ascending within a row);
    prob: float32[m] in [0, 1].
    """

    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    prob: np.ndarray
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.col.shape[0])

    def out_degree(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)

    def in_degree(self) -> np.ndarray:
        return np.bincount(self.col, minlength=self.n).astype(np.int64)

    def edges(self):
        """(src, dst) int64 arrays in CSR order."""
        src = np.repeat(np.arange(self.n, dtype=np.int64), self.out_degree())
        return src, self.col.astype(np.int64)

    def nbytes(self) -> int:
        return int(self.row_ptr.nbytes + self.col.nbytes + self.prob.nbytes)


def csr_from_edges(n: int, src, dst, prob=None, name: str = "") -> Graph:
    """Sort edges by (src, dst) and build the CSR.  Duplicates are kept."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if src.shape[0] > 1 and np.all((src[1:] > src[:-1]) | ((src[1:] == src[:-1]) & (dst[1:] >= dst[:-1]))):
        order = None                       # already in (src, dst) order: skip the sort
    else:
        order = np.lexsort((dst, src))
        src, dst = src[order], dst[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=row_ptr[1:])
    if prob is None:
        prob = np.ones(src.shape[0], dtype=np.float32)
    else:
        prob = np.asarray(prob, dtype=np.float32)
        if order is not None:
            prob = prob[order]
    return Graph(n, row_ptr.astype(np.int32), dst.astype(np.int32), prob, name)


def weighted_cascade(g: Graph) -> Graph:
    """Set p(u, v) = 1.0f / (float) indeg(v) in fp32 (correctly rounded division)."""
    indeg = g.in_degree().astype(np.float32)
    p = np.float32(1.0) / indeg[g.col]
    return Graph(g.n, g.row_ptr, g.col, p.astype(np.float32), g.name)


def _dedupe(n: int, src, dst):
    """Drop self-loops and repeated (src, dst) pairs; return sorted unique pairs."""
    keep = src != dst
    key = src[keep].astype(np.int64) * n + dst[keep].astype(np.int64)
    key.sort()                                   # sorted unique keys (as np.unique gives)
    if key.shape[0] > 1:
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    return key // n, key % n


def erdos_renyi(n: int = 1000, m: int = 5000, seed: int = 1) -> Graph:
    """m distinct directed edges with uniform endpoints and no self-loops, WC p."""
    if m > n * (n - 1):
        raise ValueError("too many edges for a simple digraph")
    rng = _rng(seed)
    keys = np.empty(0, dtype=np.int64)
    while keys.shape[0] < m:
        need = m - keys.shape[0]
        s = rng.integers(0, n, size=2 * need + 16, dtype=np.int64)
        d = rng.integers(0, n, size=2 * need + 16, dtype=np.int64)
        k = s[s != d] * n + d[s != d]
        # keep first occurrences in draw order, then the first m distinct
        allk = np.concatenate([keys, k])
        _, first = np.unique(allk, return_index=True)
        keys = allk[np.sort(first)][:m]
    g = csr_from_edges(n, keys // n, keys % n, name=f"er-{n}-{m}")
    return weighted_cascade(g)


def chung_lu(n: int = 1_000_000, avg_deg: float = 10.0, exponent: float = 2.1,
             seed: int = 1) -> Graph:
    """Directed Chung-Lu graph with power-law expected degrees, WC p.

    Expected weights w_i = (i+1)^(-1/(exponent-1)), assigned to nodes through two
    independent random permutations (one for out-weights, one for in-weights).
    round(n * avg_deg) edges are drawn with source ~ w_out and target ~ w_in;
    self-loops and duplicates are dropped.
    """
    rng = _rng(seed)
    w = np.power(np.arange(1, n + 1, dtype=np.float64), -1.0 / (exponent - 1.0))
    w_out = np.empty(n)
    w_in = np.empty(n)
    w_out[rng.permutation(n)] = w
    w_in[rng.permutation(n)] = w
    draws = int(round(n * avg_deg))
    c_out = np.cumsum(w_out)
    c_out /= c_out[-1]
    c_in = np.cumsum(w_in)
    c_in /= c_in[-1]
    src = np.searchsorted(c_out, rng.random(draws), side="right")
    dst = np.searchsorted(c_in, rng.random(draws), side="right")
    np.minimum(src, n - 1, out=src)
    np.minimum(dst, n - 1, out=dst)
    s, d = _dedupe(n, src, dst)
    g = csr_from_edges(n, s, d, name=f"cl-{n}")
    return weighted_cascade(g)


def rmat(scale: int = 22, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 1, probs=(0.1, 0.01, 0.001)) -> Graph:
    """R-MAT graph: 2^scale nodes, edge_factor * 2^scale edge draws, recursive
    quadrant choice with (a, b, c, 1-a-b-c); self-loops and duplicates dropped;
    random relabelling; p drawn uniformly from ``probs`` (trivalency)."""
    n = 1 << scale
    draws = edge_factor * n
    rng = _rng(seed)
    src = np.zeros(draws, dtype=np.int64)
    dst = np.zeros(draws, dtype=np.int64)
    t_a = np.uint32(int(a * 2**32))
    t_ab = np.uint32(int((a + b) * 2**32))
    t_abc = np.uint32(int((a + b + c) * 2**32))
    for lvl in range(scale):
        r = rng.integers(0, 2**32, size=draws, dtype=np.uint32)
        bit = np.int64(1) << (scale - 1 - lvl)
        right = ((r >= t_a) & (r < t_ab)) | (r >= t_abc)   # quadrants b, d
        down = r >= t_ab                                     # quadrants c, d
        np.add(dst, bit, out=dst, where=right)
        np.add(src, bit, out=src, where=down)
        del r, right, down
    perm = rng.permutation(n)
    src = perm[src]
    dst = perm[dst]
    s, d = _dedupe(n, src, dst)
    del src, dst
    pv = np.asarray(probs, dtype=np.float32)
    p = pv[rng.integers(0, len(pv), size=s.shape[0])]
    g = csr_from_edges(n, s, d, p, name=f"rmat-{scale}")
    return g


def seeds_uniform(n: int, k: int, seed: int = 2, exclude=None) -> np.ndarray:
    """k distinct nodes drawn uniformly (optionally avoiding ``exclude``)."""
    rng = _rng(seed)
    if exclude is None or len(exclude) == 0:
        return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int32)
    pool = np.setdiff1d(np.arange(n), np.asarray(exclude))
    return np.sort(rng.choice(pool, size=k, replace=False)).astype(np.int32)


def seeds_top_outdeg(g: Graph, k: int, frac: float = 0.01, seed: int = 2) -> np.ndarray:
    """k distinct seeds drawn uniformly from the top ``frac`` of nodes by
    out-degree (ties broken by smaller id); the pool is widened to >= 2k."""
    deg = g.out_degree()
    order = np.lexsort((np.arange(g.n), -deg))
    pool_size = max(int(round(frac * g.n)), 2 * k)
    pool = order[:pool_size]
    rng = _rng(seed)
    return np.sort(rng.choice(pool, size=k, replace=False)).astype(np.int32)


# ---------------------------------------------------------------------------
# Named workloads (sizes of the five configurations the library is measured on)
# ---------------------------------------------------------------------------

def workload_er1k():
    """ER: 1,000 nodes, 5,000 edges, WC p, |S|=10 uniform, k=5, theta=10,000."""
    g = erdos_renyi(1000, 5000, seed=1)
    S = seeds_uniform(g.n, 10, seed=2)
    return g, S, dict(k=5, theta=10_000, key=0)


def workload_cl1m(n: int = 1_000_000):
    """Chung-Lu: 1M nodes, ~10M edges, exponent 2.1, WC p, |S|=50 from the top-1%
    out-degree nodes, k=100, eps=0.1, delta=1/n."""
    g = chung_lu(n, 10.0, 2.1, seed=1)
    S = seeds_top_outdeg(g, 50, 0.01, seed=2)
    return g, S, dict(k=100, eps=0.1, delta=1.0 / g.n, key=0)


def workload_rmat4m(scale: int = 22):
    """R-MAT scale 22 (4,194,304 nodes, 2^26 edge draws), trivalency p,
    |S|=100 uniform, k=200, eps=0.1, delta=1/n."""
    g = rmat(scale, 16, seed=1)
    S = seeds_uniform(g.n, 100, seed=2)
    return g, S, dict(k=200, eps=0.1, delta=1.0 / g.n, key=0)


def chung_lu_poisson(n: int, avg_deg: float = 10.0, exponent: float = 2.1, seed: int = 1) -> Graph:
    """Directed Chung-Lu graph in the Poisson edge model, generated in O(n + m) already
    grouped by source: node u gets Poisson(avg_deg * n * w_out(u)) out-edges whose
    targets are drawn with probability proportional to w_in.  Weights follow the
    continuous power law x^(-1/(exponent-1)) on [1, n+1), under independent random
    permutations for out- and in-weights; targets are drawn by inverting its CDF.
    Multi-edges and self-loops are kept (each edge is an independent coin).  WC p."""
    rng = _rng(seed)
    a = 1.0 / (exponent - 1.0)
    x = np.arange(1, n + 1, dtype=np.float64)
    w = np.power(x, -a)
    w /= w.sum()
    perm_out = rng.permutation(n)
    perm_in = rng.permutation(n)
    deg = rng.poisson(avg_deg * n * w)                     # out-degree of rank r
    deg_node = np.empty(n, np.int64)
    deg_node[perm_out] = deg
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(deg_node, out=row_ptr[1:])
    m = int(row_ptr[-1])
    # inverse CDF of the continuous law on [1, n+1): rank = floor(x) - 1
    u = rng.random(m)
    one_m_a = 1.0 - a
    hi = np.power(float(n + 1), one_m_a) - 1.0
    r = np.floor(np.power(1.0 + u * hi, 1.0 / one_m_a)).astype(np.int64) - 1
    np.clip(r, 0, n - 1, out=r)
    col = perm_in[r].astype(np.int32)
    g = Graph(n, row_ptr.astype(np.int32), col, np.ones(m, np.float32), f"clp-{n}")
    return weighted_cascade(g)


def workload_batch(count: int = 512, seed: int = 3):
    """The batched workload: `count` independent instances on Chung-Lu graphs with
    n log-uniform in [10^3, 10^6], average degree 10, exponent 2.1, WC p; |S| uniform
    in [5, 100] from the top-1% out-degree nodes (pool widened to >= 2|S|); k uniform
    in [10, 200]; eps = 0.2, delta = 1/n.  Returns a list of (graph, S, cfg)."""
    rng = _rng(seed)
    ns = np.round(np.power(10.0, rng.uniform(3.0, 6.0, size=count))).astype(np.int64)
    nS = rng.integers(5, 101, size=count)
    ks = rng.integers(10, 201, size=count)
    out = []
    for i in range(count):
        g = chung_lu_poisson(int(ns[i]), 10.0, 2.1, seed=1000 + i)
        S = seeds_top_outdeg(g, int(nS[i]), 0.01, seed=5000 + i)
        k = int(min(ks[i], g.n - len(S) - 1))
        out.append((g, S, dict(k=k, eps=0.2, delta=1.0 / g.n, key=0, inst=i)))
    return out
