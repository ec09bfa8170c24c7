"""Exact pins by enumerating all 2^m live-edge worlds of tiny graphs (Eq. 1).

* Eq. 3 / Sec. 3: D^L(B) <= D(B) <= D^U(B) for every blocker set.
* Lemma 3.1 and Sec. 3.3: D^L and D^U are monotone and submodular.
* Eq. 2 chain: D itself is not submodular.
* Lemma 4.1 / Lemma 4.2: the oracle's per-world lower credit and LRR sets are
  unbiased for D^L({v}) and D^U({v}) -- exactly (weighted sum over all worlds)
  and within 5 sigma for its Philox-driven Monte Carlo.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2405_12871_gb300 import synth
import worlds_ref as ref


def _exact_tables(n, src, dst, p, S, maxB=3):
    Sset = set(int(s) for s in S)
    cand = [v for v in range(n) if v not in Sset]
    subsets = [frozenset(c) for r in range(maxB + 1) for c in itertools.combinations(cand, r)]
    D = dict.fromkeys(subsets, 0.0)
    DL = dict.fromkeys(subsets, 0.0)
    DU = dict.fromkeys(subsets, 0.0)
    for live, wgt in ref.enumerate_worlds(p):
        adj = ref.live_adj(n, src, dst, live)
        base = ref.reach(adj, S)
        Nv = {v: ref.N_phi(adj, S, v) for v in cand}
        for B in subsets:
            D[B] += wgt * (len(base) - len(ref.reach(adj, S, blocked=B)))
            U = set()
            for v in B:
                U |= Nv[v]
            DL[B] += wgt * len(U)
            DU[B] += wgt * len(ref.M_phi(adj, S, B))
    return cand, subsets, D, DL, DU


@pytest.mark.parametrize("seed", range(6))
def test_sandwich_monotone_submodular(seed):
    n, src, dst, p = ref.tiny_graph(seed, n_hi=7, m_max=10)
    S = [0]
    cand, subsets, D, DL, DU = _exact_tables(n, src, dst, p, S)
    eps = 1e-12
    for B in subsets:
        assert DL[B] <= D[B] + eps and D[B] <= DU[B] + eps, (B, DL[B], D[B], DU[B])
    for A in subsets:
        for x in cand:
            if x in A or len(A) + 1 > 3:
                continue
            Ax = A | {x}
            assert DL[Ax] >= DL[A] - eps and DU[Ax] >= DU[A] - eps         # monotone
            for y in cand:
                if y in Ax or len(Ax) + 1 > 3:
                    continue
                Ay, Axy = A | {y}, Ax | {y}
                # f(A+x) - f(A) >= f(A+y+x) - f(A+y)
                assert DL[Ax] - DL[A] >= DL[Axy] - DL[Ay] - eps
                assert DU[Ax] - DU[A] >= DU[Axy] - DU[Ay] - eps


def test_chain_objective_not_submodular():
    n = 8
    edges = [(0, 1), (0, 2), (1, 3), (2, 3)] + [(3, i) for i in range(4, n)]
    src = np.array([e[0] for e in edges])
    dst = np.array([e[1] for e in edges])
    p = np.ones(len(edges), np.float32)
    _, _, D, DL, DU = _exact_tables(n, src, dst, p, [0], maxB=2)
    A = frozenset()
    assert D[frozenset({1, 2})] == n - 1 and D[frozenset({1})] == 1 and D[frozenset({2})] == 1
    # D(A+v1) - D(A) = 1 < D(A+v2+v1) - D(A+v2) = n - 2: submodularity fails
    assert D[frozenset({1})] - D[A] < D[frozenset({1, 2})] - D[frozenset({2})]
    assert DL[frozenset({1, 2})] == 2 and DU[frozenset({1})] == n - 2


@pytest.mark.parametrize("seed", range(5))
def test_lemma_4_1_and_4_2_exact_and_mc(seed):
    n, src, dst, p = ref.tiny_graph(50 + seed, n_hi=7, m_max=11)
    S = [0] if seed % 2 == 0 else [0, 1]
    Sset = set(S)
    g = synth.csr_from_edges(n, src, dst, p)
    og = oracle.OracleGraph.from_graph(g)
    cand = [v for v in range(n) if v not in Sset]
    Vs = og.vs(S)
    nVs = len(Vs)
    exact_L = np.zeros(n)
    exact_U = np.zeros(n)
    exact_R = np.zeros(n)
    sec_L = np.zeros(n)
    sec_U = np.zeros(n)
    o_L = np.zeros(n)
    o_U = np.zeros(n)
    for live, wgt in ref.enumerate_worlds(p):
        adj = ref.live_adj(n, src, dst, live)
        base = ref.reach(adj, S)
        for v in base:
            exact_R[v] += wgt
        w = og.world_explicit(live, S)
        for v in cand:
            c = len(ref.N_phi(adj, S, v))
            exact_L[v] += wgt * c
            sec_L[v] += wgt * c * c
            o_L[v] += wgt * float(w["credit_lower"][v])
            exact_U[v] += wgt * len(ref.M_phi(adj, S, [v]))
        # oracle LRR sets over the uniform target t in V'_s
        for t in Vs:
            wt = og.world_explicit(live, S, target=int(t))
            for v in cand:
                hit = float(wt["lrr"][v])
                o_U[v] += wgt * hit / nVs
                sec_U[v] += wgt * hit / nVs
    # Lemma 4.1 exactly: E[credit] == D^L({v}); Lemma 4.2: |V'_s| E[1{v in L}] == D^U({v})
    for v in cand:
        assert o_L[v] == pytest.approx(exact_L[v], abs=1e-12)
        assert nVs * o_U[v] == pytest.approx(exact_U[v], abs=1e-9)
    # Monte Carlo with Philox coins (5 sigma)
    theta = 20000
    out = og.sample(S, theta=theta, key=1234 + seed, tag=1,
                    mode=oracle.MODE_REACH | oracle.MODE_LOWER | oracle.MODE_UPPER)
    for v in range(n):
        pr = exact_R[v]
        sd = np.sqrt(max(pr * (1 - pr), 0.0) / theta)
        assert abs(int(out["reach"][v]) / theta - pr) <= 5 * sd + 1e-12, v
    for v in cand:
        mean = exact_L[v]
        sd = np.sqrt(max(sec_L[v] - mean * mean, 0.0) / theta)
        assert abs(int(out["credit_lower"][v]) / theta - mean) <= 5 * sd + 1e-12, v
        q = sec_U[v]
        sd = np.sqrt(max(q * (1 - q), 0.0) / theta)
        assert abs(int(out["credit_upper"][v]) / theta - q) <= 5 * sd + 1e-12, v
