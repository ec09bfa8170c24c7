"""AdvancedGreedy and GreedyReplace (the paper's dominator-tree baselines), run on the
oracle's sampler: the example the paper uses to motivate GR, and the number of
estimates each performs."""
import numpy as np

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
