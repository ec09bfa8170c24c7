"""AdvancedGreedy and GreedyReplace (the paper's dominator-tree baselines), run on the
oracle's sampler: the example the paper uses to motivate GR, and the number of
estimates each performs; a second hand-checked graph; and the package's selection against
the oracle's own C implementation of AG and GR."""
import numpy as np
import pytest

import oracle
from paper_2405_12871_gb300 import baselines, synth


def example_graph():
    """Seed 0 with out-neighbours 1 and 2; both lead to 3, which leads to 4, 5, 6; every
    edge has p = 1, so every world is the whole graph.  Blocking 3 protects four nodes,
    the most of any single node, but 1 and 2 together protect everything."""
    src = [0, 0, 1, 2, 3, 3, 3]
    dst = [1, 2, 3, 3, 4, 5, 6]
    return synth.csr_from_edges(7, src, dst, np.ones(7, np.float32))


def test_ag_misses_the_out_neighbours_and_gr_finds_them():
    g = example_graph()
    og = oracle.OracleGraph.from_graph(g)
    B_ag, calls_ag, _ = baselines.advanced_greedy(og.sample, g.n, [0], k=2, theta=3)
    assert B_ag == [3, 1]                 # v2 stays reachable
    B_gr, calls_gr, _ = baselines.greedy_replace(og.sample, g, [0], k=2, theta=3)
    assert sorted(B_gr) == [1, 2]         # nothing but the seed is reached
    assert calls_ag == 2
    assert calls_gr == 3                  # two stage-1 picks, one replacement check
    for B, spread in ((B_ag, 2 * 3), (B_gr, 1 * 3)):
        r = og.sample([0], B, theta=3, mode=1)
        assert r["total_spread"] == spread


def test_estimates_are_subtree_sizes():
    g = example_graph()
    og = oracle.OracleGraph.from_graph(g)
    est = baselines._Estimator(og.sample, g.n, [0], 5, 0)
    c = est.credits([])
    assert c.tolist() == [0, 5, 5, 20, 5, 5, 5]
    assert est.best([]) == 3 and est.best([3]) == 1 and est.best([1], allowed=[2]) == 2


def test_out_neighbours_skip_zero_probability_and_seeds():
    g = synth.csr_from_edges(5, [0, 0, 0, 1], [1, 2, 3, 4], np.array([0.5, 0.0, 1.0, 1.0], np.float32))
    assert baselines.out_neighbours(g.row_ptr, g.col, g.prob, [0, 1]) == [3, 4]


def second_graph():
    """p = 1.  Seed 0 -> 1, 2, 3; 1 -> 4 -> 5, 6, 7; 2 -> 8, 3 -> 8, 8 -> 9, 10.
    Subtree sizes: 1: 5, 4: 4, 8: 3 (8 is dominated by the seed alone), 2: 1, 3: 1."""
    src = [0, 0, 0, 1, 4, 4, 4, 2, 3, 8, 8]
    dst = [1, 2, 3, 4, 5, 6, 7, 8, 8, 9, 10]
    return synth.csr_from_edges(11, src, dst, np.ones(len(src), np.float32))


def test_second_graph_hand_checked():
    """AG: 1 (5 protected), then 8 (3 of what is left).  GR: stage 1 picks 1, then 2 of
    the seed's out-neighbours {2, 3} (a tie, smaller id); stage 2 takes out 2 and puts
    back 8, then takes out 1 and puts 1 back -- done, after four estimates."""
    g = second_graph()
    og = oracle.OracleGraph.from_graph(g)
    assert baselines.advanced_greedy(og.sample, g.n, [0], k=2, theta=4)[:2] == ([1, 8], 2)
    assert baselines.greedy_replace(og.sample, g, [0], k=2, theta=4)[:2] == ([1, 8], 4)
    assert og.dt_baseline("ag", [0], 2, 4) == ([1, 8], 2)
    assert og.dt_baseline("gr", [0], 2, 4) == ([1, 8], 4)
    assert og.sample([0], [1, 8], theta=2, mode=1)["total_spread"] == 2 * 3


@pytest.mark.parametrize("which", ["ag", "gr"])
@pytest.mark.parametrize("graph", ["er1k", "cl5k"])
def test_baselines_match_the_oracles_own_implementation(which, graph):
    """The package's AG / GR (numpy selection over any sampler) and the oracle's plain C
    AG / GR (its own selection over its own worlds) pick the same blockers with the same
    number of estimates."""
    if graph == "er1k":
        g, S, _ = synth.workload_er1k()
        k, theta = 5, 2000
    else:
        g = synth.chung_lu(5000, 10.0, 2.1, seed=11)
        S = synth.seeds_top_outdeg(g, 8, 0.01, seed=12)
        k, theta = 6, 500
    og = oracle.OracleGraph.from_graph(g)
    if which == "ag":
        got = baselines.advanced_greedy(og.sample, g.n, S, k=k, theta=theta, key=3)
    else:
        got = baselines.greedy_replace(og.sample, g, S, k=k, theta=theta, key=3)
    assert got[:2] == og.dt_baseline(which, S, k, theta, key=3)
