"""Pins for the oracle's per-world structures (Algorithm 2, Algorithm 3).

* Example 2.1 / 4.2 (golden): reach set, idoms, CP sets and subtree credits.
* The submodularity-ratio chain (Sec. 2.2, Eq. 2): closed forms of D, D^L, D^U.
* Random worlds: reach vs scipy BFS; idom vs networkx.immediate_dominators;
  lower credit vs |N_phi(v)| by deletion (the definition of the lower bound);
  LRR sets vs forward reachability inside phi^s (Def. 4.2).
"""
import os

import networkx as nx
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import breadth_first_order

from conftest import GOLDEN
import oracle
from paper_2405_12871_gb300 import synth
import worlds_ref as ref


def _load_ex21():
    edges, credit, idom, cps = [], {}, {}, {}
    n = seed = None
    for line in open(os.path.join(GOLDEN, "example_2_1.txt")):
        w = line.split()
        if not w or w[0].startswith("#"):
            continue
        if w[0] == "nodes":
            n = int(w[1])
        elif w[0] == "seed":
            seed = int(w[1])
        elif w[0] == "edge":
            edges.append((int(w[1]), int(w[2])))
        elif w[0] == "credit":
            credit[int(w[1])] = int(w[2])
        elif w[0] == "idom":
            idom[int(w[1])] = int(w[2])
        elif w[0] == "cpset":
            cps[int(w[1])] = set(int(x) for x in w[2:])
    return n, seed, edges, credit, idom, cps


def test_example_2_1():
    n, seed, edges, credit, idom, cps = _load_ex21()
    src = np.array([e[0] for e in edges])
    dst = np.array([e[1] for e in edges])
    g = synth.csr_from_edges(n, src, dst)
    og = oracle.OracleGraph.from_graph(g)
    w = og.world_explicit(np.ones(g.m, np.uint8), [seed])
    assert w["R"] == 6                                        # v0 plus five receivers
    assert list(np.flatnonzero(w["reached"])) == [0, 1, 2, 3, 5, 6]
    for v, c in credit.items():
        assert int(w["credit_lower"][v]) == c, v
    for v, d in idom.items():
        # the seed v0 hangs under the virtual root; its children keep v0 as idom
        assert int(w["idom"][v]) == d, v
    assert int(w["idom"][0]) == -1 and int(w["idom"][4]) == -2
    # CP sets: credit_lower(v) = number of CP sets that contain v
    counts = {v: sum(1 for s in cps.values() if v in s) for v in range(n)}
    for v in range(1, n):
        assert int(w["credit_lower"][v]) == counts[v]


@pytest.mark.parametrize("n", [6, 10, 25])
def test_chain_example_closed_forms(n):
    """v0 -> v1, v0 -> v2, v1 -> v3, v2 -> v3, v3 -> v4..v_{n-1}, all p = 1."""
    edges = [(0, 1), (0, 2), (1, 3), (2, 3)] + [(3, i) for i in range(4, n)]
    src = np.array([e[0] for e in edges])
    dst = np.array([e[1] for e in edges])
    g = synth.csr_from_edges(n, src, dst)
    og = oracle.OracleGraph.from_graph(g)
    S = [0]
    # D(B) from the oracle's own reach counts with blockers (p = 1: one world suffices)
    I0 = og.sample(S, theta=1)["total_spread"]
    assert I0 == n
    assert I0 - og.sample(S, blocked=[1, 2], theta=1)["total_spread"] == n - 1   # D({v1,v2})
    assert I0 - og.sample(S, blocked=[1], theta=1)["total_spread"] == 1          # D({v1})
    assert I0 - og.sample(S, blocked=[2], theta=1)["total_spread"] == 1          # D({v2})
    out = og.sample(S, theta=1, mode=oracle.MODE_LOWER | oracle.MODE_UPPER)
    cl = out["credit_lower"]
    # D^L({v1, v2}) = |N(v1) u N(v2)| = 2 (no CP set holds both)
    assert int(cl[1]) == 1 and int(cl[2]) == 1
    assert int(cl[3]) == n - 3
    # D^U({v1}) = |M({v1})| = n - 2, checked through LRR sets over every target
    live = np.ones(g.m, np.uint8)
    hits = sum(int(og.world_explicit(live, S, target=t)["lrr"][1]) for t in range(1, n))
    assert hits == n - 2


def _random_world_cases():
    cases = []
    for seed in range(12):
        rng = np.random.default_rng(100 + seed)
        n = int(rng.integers(8, 60))
        m = int(rng.integers(n, 4 * n))
        src = rng.integers(0, n, m)
        dst = rng.integers(0, n, m)
        keep = src != dst
        src, dst = src[keep], dst[keep]
        live = (rng.random(src.shape[0]) < 0.6).astype(np.uint8)
        nS = int(rng.integers(1, 4))
        S = rng.choice(n, nS, replace=False)
        others = np.setdiff1d(np.arange(n), S)
        B = rng.choice(others, int(rng.integers(0, 3)), replace=False) if seed % 3 == 0 else []
        cases.append((n, src, dst, live, S, B))
    return cases


@pytest.mark.parametrize("case", _random_world_cases())
def test_random_world_against_definitions(case):
    n, src, dst, live, S, B = case
    g = synth.csr_from_edges(n, src, dst)
    # csr_from_edges sorts edges: recompute the live mask in CSR order
    order = np.lexsort((dst, src))
    live_csr = live[order]
    gs, gd = g.edges()
    og = oracle.OracleGraph.from_graph(g)
    w = og.world_explicit(live_csr, S, blocked=B)
    blocked = set(int(b) for b in B)
    # --- reach vs scipy BFS (virtual root n -> seeds; blocked targets removed)
    keep = live_csr.astype(bool) & ~np.isin(gd, list(blocked) if blocked else [-1])
    s2 = np.concatenate([gs[keep], np.full(len(S), n)])
    d2 = np.concatenate([gd[keep], S])
    A = sp.csr_matrix((np.ones(s2.shape[0]), (s2, d2)), shape=(n + 1, n + 1))
    order_bfs = breadth_first_order(A, n, directed=True, return_predecessors=False)
    R = set(int(x) for x in order_bfs) - {n}
    assert set(np.flatnonzero(w["reached"]).tolist()) == R
    assert w["R"] == len(R)
    # --- idom vs networkx on the live subgraph reached from the virtual root
    G = nx.DiGraph()
    G.add_node(n)
    for u, v in zip(s2, d2):
        if int(u) in R | {n} and int(v) in R:
            G.add_edge(int(u), int(v))
    idom = nx.immediate_dominators(G, n)
    for v in R:
        want = idom[v]
        want = -1 if want == n else want
        assert int(w["idom"][v]) == want, (v, want, int(w["idom"][v]))
    # --- lower credit = |N_phi(v)| by deletion (world without blockers only)
    if not blocked:
        adj = ref.live_adj(n, gs, gd, live_csr)
        for v in range(n):
            assert int(w["credit_lower"][v]) == len(ref.N_phi(adj, S, v)), v
        # --- LRR sets vs forward reachability in phi^s
        Sset = set(int(s) for s in S)
        for t in sorted(R - Sset)[:8]:
            wt = og.world_explicit(live_csr, S, target=t)
            got = set(np.flatnonzero(wt["lrr"]).tolist())
            assert got == ref.L_phi(adj, S, t), t
