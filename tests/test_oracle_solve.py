"""Pins for the stopping-rule spread estimate and the whole solve (Algorithm 1).

* Stopping rule on a deterministic graph (p = 1): every world has the same
  spread c, so N = ceil(T / c) with T = ceil(Upsilon1 * W), and I = W*Upsilon1/N.
* Stopping rule guarantee (Dagum-Karp-Luby-Ross, the (beta, delta')-estimate
  Algorithm 4 asks for): on small graphs with exactly enumerated E[I], every
  estimate over 20 keys lies within (1 +/- beta) E[I].
* Algorithm 4 lines 2-3: |ON| <= k returns ON.
* The chain of Eq. 2 with k = 1 (p = 1): LSBM picks v3 (D^L({v3}) = n-3), GSBM
  picks v1 (D^U({v1}) = D^U({v2}) = n-2, smaller id), LHGA picks v1, and the
  Sandwich keeps B_L, whose residual spread is 3.
* On tiny graphs the LSBM answer satisfies Theorem 5.4 against the brute-force
  optimum of the exactly enumerated D^L.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2405_12871_gb300 import synth
import worlds_ref as ref


def _ups1(beta, dprime):
    ups = 4 * (math.e - 2) * math.log(2 / dprime) / beta ** 2
    return 1 + (1 + beta) * ups


def test_stop_rule_deterministic():
    n = 12
    edges = [(0, i) for i in range(1, 6)] + [(6, 7)]
    g = synth.csr_from_edges(n, [e[0] for e in edges], [e[1] for e in edges])
    og = oracle.OracleGraph.from_graph(g)
    S = [0]
    c = 6                         # v0 and its five out-neighbours; W = |V'_s| + |S| = 6
    for beta, dp in ((0.1, 0.01), (0.05, 1e-6), (0.3, 0.5)):
        N, I = og.stop_rule(S, beta=beta, dprime=dp)
        u1 = _ups1(beta, dp)
        T = math.ceil(u1 * 6)
        assert N == math.ceil(T / c)
        assert I == pytest.approx(6 * u1 / N, rel=1e-15)
        assert abs(I - c) <= c / N + 1e-9


@pytest.mark.parametrize("seed", range(4))
def test_stop_rule_guarantee(seed):
    n, src, dst, p = ref.tiny_graph(200 + seed, n_lo=6, n_hi=8, m_max=12,
                                    probs=(0.25, 0.5, 0.75))
    S = [0]
    EI = 0.0
    for live, wgt in ref.enumerate_worlds(p):
        EI += wgt * len(ref.reach(ref.live_adj(n, src, dst, live), S))
    og = oracle.OracleGraph.from_graph(synth.csr_from_edges(n, src, dst, p))
    beta, dp = 0.1, 1e-4
    for key in range(20):
        _, I = og.stop_rule(S, beta=beta, dprime=dp, key=key)
        assert (1 - beta) * EI <= I <= (1 + beta) * EI, (key, I, EI)


def test_on_shortcut():
    n = 30
    rng = np.random.default_rng(5)
    src = rng.integers(0, n, 90)
    dst = rng.integers(0, n, 90)
    keep = src != dst
    g = synth.weighted_cascade(synth.csr_from_edges(n, src[keep], dst[keep]))
    og = oracle.OracleGraph.from_graph(g)
    S = [3]
    gs, gd = g.edges()
    ON = sorted(set(int(v) for v in gd[gs == 3]) - {3})
    r = og.solve(S, k=len(ON), eps=0.2, delta=0.01)
    assert list(r["blockers"]) == ON and r["n_spread"] == 0


@pytest.mark.parametrize("variant", ["sandimin", "sandimin-"])
def test_chain_solve(variant):
    n = 12
    edges = [(0, 1), (0, 2), (1, 3), (2, 3)] + [(3, i) for i in range(4, n)]
    g = synth.csr_from_edges(n, [e[0] for e in edges], [e[1] for e in edges])
    og = oracle.OracleGraph.from_graph(g)
    r = og.solve([0], k=1, eps=0.2, delta=0.05, variant=variant)
    assert list(r["B_L"]) == [3]
    assert list(r["B_R"]) == [1]
    if variant == "sandimin":
        assert list(r["B_U"]) == [1]
    assert r["chosen"] == 0 and list(r["blockers"]) == [3]
    assert abs(r["I_after"][0] - 3) <= 3 / r["n_final"][0] + 1e-9
    assert abs(r["I_hat"] - n) <= n / r["n_spread"] + 1e-9
    # every world is the same: D^L(B_L) estimates are exact
    assert r["DL_hat"] == n - 3


@pytest.mark.parametrize("seed", range(4))
def test_lsbm_theorem_5_4_on_tiny_graphs(seed):
    n, src, dst, p = ref.tiny_graph(300 + seed, n_lo=7, n_hi=8, m_max=10)
    # make sure the seed has at least three out-neighbours (so |ON| > k)
    extra = [(0, v) for v in (1, 2, 3) if not np.any((src == 0) & (dst == v))]
    src = np.r_[src, [e[0] for e in extra]].astype(int)
    dst = np.r_[dst, [e[1] for e in extra]].astype(int)
    p = np.r_[p, np.full(len(extra), 0.5, np.float32)].astype(np.float32)
    order = np.lexsort((dst, src))
    src, dst, p = src[order], dst[order], p[order]
    S = [0]
    g = synth.csr_from_edges(n, src, dst, p)
    og = oracle.OracleGraph.from_graph(g)
    k, eps, delta = 2, 0.3, 0.05
    gs, gd = g.edges()
    ON = set(int(v) for v in gd[gs == 0]) - {0}
    if len(ON) <= k:
        pytest.skip("ON shortcut case")
    r = og.solve(S, k=k, eps=eps, delta=delta, variant="lsbm")
    cand = [v for v in range(n) if v != 0]
    DL = {}
    for live, wgt in ref.enumerate_worlds(p):
        adj = ref.live_adj(n, src, dst, live)
        Nv = {v: ref.N_phi(adj, S, v) for v in cand}
        for B in itertools.combinations(cand, k):
            U = set()
            for v in B:
                U |= Nv[v]
            DL[B] = DL.get(B, 0.0) + wgt * len(U)
    best = max(DL.values())
    got = DL[tuple(sorted(int(x) for x in r["B_L"]))] if len(r["B_L"]) == k else None
    assert got is not None and got >= (1 - 1 / math.e - eps) * best
    # the reported estimate of D^L(B_L) is an unbiased average over |C2| worlds
    assert r["theta_C2"] == r["theta_C1"] and r["theta_C1"] >= 1


def test_solve_deterministic_and_keyed():
    g, S, cfg = synth.workload_er1k()
    og = oracle.OracleGraph.from_graph(g)
    a = og.solve(S, k=cfg["k"], eps=0.3, delta=0.01, fixed_theta=2000)
    b = og.solve(S, k=cfg["k"], eps=0.3, delta=0.01, fixed_theta=2000)
    assert list(a["blockers"]) == list(b["blockers"]) and a["I_after"] == b["I_after"]
    assert a["theta_C1"] == 2000 and a["theta_L1"] == 2000
    # the chosen set is the argmin of the final estimates (ties in order L, U, R)
    ia = a["I_after"]
    assert a["chosen"] == int(np.argmin(ia))
