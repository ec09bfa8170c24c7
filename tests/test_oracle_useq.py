"""Pins for the oracle's LRR-sequence estimator (Sec. 4.2, "Discussion"): in every
world, the LRR set of every node of phi^s, by its own reverse traversal.

* Per explicit world, against the definitions written out in worlds_ref: the
  sequence's coverage of a set Q is |M_phi(Q)| (the nodes of phi^s reachable from Q),
  a node's sequence credit is |M_phi({u})|, and the sequence holds sum_v |L_phi(v)|
  elements.
* Exactly over all 2^m worlds: E[Cov_{L^s}(Q)] = D^U(Q) (the estimator is unbiased).
* Monte Carlo (Philox worlds): the mean coverage is within 5 sigma of D^U(Q).
"""
import itertools

import numpy as np
import pytest

import oracle
import worlds_ref as ref
from paper_2405_12871_gb300 import synth


@pytest.mark.parametrize("seed", range(5))
def test_per_world_identities_and_exact_expectation(seed):
    n, src, dst, p = ref.tiny_graph(700 + seed, n_lo=5, n_hi=7, m_max=10)
    S = [0]
    og = oracle.OracleGraph.from_graph(synth.csr_from_edges(n, src, dst, p))
    cand = list(range(1, n))
    Qs = [()] + [(v,) for v in cand] + list(itertools.combinations(cand, 2))
    DU = dict.fromkeys(Qs, 0.0)
    est = dict.fromkeys(Qs, 0.0)
    for live, wgt in ref.enumerate_worlds(p):
        adj = ref.live_adj(n, src, dst, live)
        R = ref.reach(adj, S)
        inner = R - set(S)
        elems = sum(len(ref.L_phi(adj, S, v)) for v in inner)
        for Q in Qs:
            r = og.lrr_sequence_explicit(live, S, query=Q)
            M = ref.M_phi(adj, S, Q)
            assert r["cov"] == len(M), (Q, r["cov"], M)
            assert r["elements"] == elems and r["total_spread"] == len(R)
            DU[Q] += wgt * len(M)
            est[Q] += wgt * r["cov"]
            if Q == ():
                for u in range(n):
                    want = len(ref.M_phi(adj, S, [u])) if u in inner else 0
                    assert int(r["credit_useq"][u]) == want, (u, want)
    for Q in Qs:
        assert est[Q] == pytest.approx(DU[Q], abs=1e-12)
    assert DU[()] == 0.0


def test_monte_carlo_within_five_sigma():
    n, src, dst, p = ref.tiny_graph(711, n_lo=6, n_hi=7, m_max=11)
    S = [0]
    og = oracle.OracleGraph.from_graph(synth.csr_from_edges(n, src, dst, p))
    Q = (1, 3)
    DU = 0.0
    for live, wgt in ref.enumerate_worlds(p):
        DU += wgt * len(ref.M_phi(ref.live_adj(n, src, dst, live), S, Q))
    theta = 200_000
    r = og.lrr_sequences(S, query=Q, theta=theta, key=5, tag=10)
    cw = r["cov_world"].astype(np.float64)
    assert r["cov"] == int(cw.sum())
    sd = cw.std(ddof=1) / np.sqrt(theta)
    assert abs(cw.mean() - DU) <= 5 * sd + 1e-12, (cw.mean(), DU, sd)
