"""Pins for the controller quantities that no sampling test reaches: OPT^L (Sec. 5.1),
the LHGA order (Sec. 5.3) and the approximation-ratio lower bound (Sec. 6.4).

Each expected value below is worked out by hand from the graph in the test, not by
calling the oracle's own formulas, and each graph is chosen so that a plausible slip
gives a different answer:

* OPT^L = sum of the k largest q(v), q(v) = 1 - prod over seed in-edges (1 - p_q).
  Node 2 has two seed in-edges (p = 0.5, 0.25: q = 0.625, where 1 - sum p gives 0.25
  and max p gives 0.5), node 6 has two seed in-edges of p = 0.1 (fp32(0.1) is not a multiple of 2^-24, so the
  quantised p_q = ceil(p 2^24) / 2^24 differs from p), node 2 also has an in-edge from
  a non-seed, a seed has an edge to the other seed (seeds are not in ON), and one
  seed edge has p = 0 (not in ON).
* LHGA ranks ON by q(v) * outdeg(v), ties to the smaller id.  The graph makes the top
  two differ from the top two by q alone, by out-degree alone and by q * in-degree,
  and node 1 ties node 2 on the score while node 2 has the larger q.
* The alternative reading of Pr[s -> v] (the reach frequency over worlds of stream
  tag 6): a node reached directly and through another node, where the two readings
  give 0.5 and about 0.75.
* ratio_lb = ((1 - gamma)^2 / (1 + gamma)^2) (1 - 1/e - eps) (I_hat - I_after[U]) / D^U_hat
  on a p = 1 graph, where every LRR set contains node 1, so B_U = {1}, D^U_hat = |V'_s|
  exactly, D^L({1}) = 3 != D^U({1}) = 5, and both stopping-rule estimates have the
  closed form W Upsilon1 / ceil(ceil(Upsilon1 W) / |R|).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import pin_graphs


def _pq(p):
    """p as the coin rule realises it: ceil(fp32(p) * 2^24) / 2^24, exactly."""
    f = Fraction(float(np.float32(p))) * (1 << 24)
    return math.ceil(f) / float(1 << 24)


def _ups1(beta, dprime):
    ups = 4 * (math.e - 2) * math.log(2 / dprime) / beta ** 2
    return 1 + (1 + beta) * ups


def _det_estimate(R, W, beta, dprime):
    """Stopping-rule estimate when every world reaches exactly R nodes."""
    u1 = _ups1(beta, dprime)
    N = math.ceil(math.ceil(u1 * W) / R)
    return W * u1 / N


# ---------------------------------------------------------------- OPT^L (Sec. 5.1)

def test_opt_lower_top_k_direct_activation():
    og = oracle.OracleGraph.from_graph(pin_graphs.opt_graph())
    k = 4
    r = og.solve([0, 1], k=k, eps=0.3, delta=0.05, variant="lsbm")
    q6 = 1 - (1 - _pq(0.1)) ** 2
    assert _pq(0.1) != float(np.float32(0.1))
    q = {2: 0.625, 3: 0.75, 4: 0.5, 5: 0.125, 6: q6, 9: 0.0625}
    top = sorted(q.values(), reverse=True)[:k]
    assert top == [0.75, 0.625, 0.5, q6]
    assert r["OPT_L"] == pytest.approx(sum(top), rel=1e-13)
    # slips that must not pass: 1 - sum p, raw p for p_q, max p, counting node 7's edge
    raw6 = 1 - (1 - float(np.float32(0.1))) ** 2
    assert abs(sum(top) - (0.75 + 0.75 + 0.5 + 0.2)) > 0.1
    assert abs(sum(top) - (0.75 + 0.625 + 0.5 + raw6)) > 1e-9
    assert abs(sum(top) - (0.75 + 0.5 + 0.5 + 0.1)) > 0.01
    assert abs(sum(top) - (0.8125 + 0.75 + 0.5 + q6)) > 0.1
    # theta_max of Lemma 5.2 is taken at this OPT^L
    th = oracle.lsbm_theta_max(r["I_hat"], pin_graphs.OPT_N, 2, k, 0.3, 0.05, 0.1, sum(top))
    assert r["theta_max_L"] == pytest.approx(th, rel=1e-12)


def test_opt_lower_with_fewer_than_k_positive_scores_is_not_taken():
    # |ON| <= k: the ON shortcut returns before OPT^L is formed
    g = pin_graphs.graph(4, [(0, 1, 0.5), (0, 2, 0.5), (2, 3, 0.5)])
    r = oracle.OracleGraph.from_graph(g).solve([0], k=2, eps=0.3, delta=0.05)
    assert list(r["blockers"]) == [1, 2] and r["OPT_L"] == 0.0


# ---------------------------------------------------------------- LHGA (Sec. 5.3)

@pytest.mark.parametrize("k,expect", [(1, [1]), (2, [1, 2]), (3, [1, 2, 3])])
def test_lhga_order(k, expect):
    g, n = pin_graphs.lhga_graph()
    r = oracle.OracleGraph.from_graph(g).solve([0], k=k, eps=0.3, delta=0.05, variant="lhga")
    assert list(r["B_R"]) == expect
    assert list(r["blockers"]) == expect


def test_lhga_graph_separates_the_slips():
    g, n = pin_graphs.lhga_graph()
    src, dst = g.edges()
    outdeg = np.bincount(src, minlength=n)
    indeg = np.bincount(dst, minlength=n)
    q = {1: 0.25, 2: 0.5, 3: 0.75, 4: 0.125}
    assert [int(outdeg[v]) for v in (1, 2, 3, 4)] == [4, 2, 1, 6]
    assert [int(indeg[v]) for v in (1, 2, 3, 4)] == [1, 1, 3, 4]

    def top2(score):
        return sorted(q, key=lambda v: (-score(v), v))[:2]

    assert top2(lambda v: q[v] * outdeg[v]) == [1, 2]
    assert top2(lambda v: q[v]) == [3, 2]
    assert top2(lambda v: outdeg[v]) == [4, 1]
    assert top2(lambda v: q[v] * indeg[v]) == [3, 2]
    assert top2(lambda v: indeg[v]) == [4, 3]
    # ties broken toward the larger q, or the larger id, would put node 2 first
    assert sorted(q, key=lambda v: (-q[v] * outdeg[v], -q[v]))[0] == 2


# ---------------------------------------------------------------- ratio_lb (Sec. 6.4)

def test_ratio_lower_bound_closed_form():
    og = oracle.OracleGraph.from_graph(pin_graphs.ratio_graph())
    eps, delta, beta, gamma = 0.2, 0.05, 0.1, 0.1
    r = og.solve([0], k=1, eps=eps, delta=delta, beta=beta, gamma=gamma, variant="sandimin")
    assert list(r["B_U"]) == [1] and list(r["B_L"]) == [1] and list(r["B_R"]) == [1]
    assert r["nVs"] == 5
    assert r["DU_hat"] == 5.0            # |V'_s| * |L2| / |L2|
    assert r["DL_hat"] == 3.0            # node 1 dominates 4 and 5
    I_hat = _det_estimate(6, 6, beta, delta / 6)
    # with node 1 blocked: R = {0, 2, 3}, V'_s = {2, 3}, W = 3
    I_after = _det_estimate(3, 3, gamma, delta)
    assert r["I_hat"] == pytest.approx(I_hat, rel=1e-14)
    assert r["I_after"][1] == pytest.approx(I_after, rel=1e-14)
    gr = (1 - gamma) ** 2 / (1 + gamma) ** 2
    expect = gr * (1 - 1 / math.e - eps) * (I_hat - I_after) / 5.0
    assert r["ratio_lb"] == pytest.approx(expect, rel=1e-12)
    # the slips: D^L in place of D^U, (1-gamma)/(1+gamma) unsquared, no (1-1/e-eps)
    assert abs(expect - gr * (1 - 1 / math.e - eps) * (I_hat - I_after) / 3.0) > 0.05
    assert abs(expect - (1 - gamma) / (1 + gamma) * (1 - 1 / math.e - eps) * (I_hat - I_after) / 5.0) > 0.01
    assert abs(expect - gr * (I_hat - I_after) / 5.0) > 0.05


def test_ratio_lower_bound_absent_without_the_upper_candidate():
    og = oracle.OracleGraph.from_graph(pin_graphs.ratio_graph())
    r = og.solve([0], k=1, eps=0.2, delta=0.05, variant="sandimin-")
    assert r["ratio_lb"] == 0.0 and r["DU_hat"] == 0.0


# ------------------------------------- Pr[s -> v] as the reach frequency (Sec. 5.1)

def _two_path_graph():
    # s = 0 -> 1 (p = 0.5), 0 -> 2 (p = 0.5), 1 -> 2 (p = 1), plus node 3 reached from 2
    # (so that |ON| = 2 > k = 1 and the solve runs).  Direct activation q(2) = 0.5, but
    # Pr[s -> 2] = 1 - 0.5 * 0.5 = 0.75 (through node 1 as well).
    return pin_graphs.graph(4, [(0, 1, 0.5), (0, 2, 0.5), (1, 2, 1.0), (2, 3, 0.5)])


def test_opt_lower_with_reach_frequency():
    """With pr_worlds = theta, OPT^L (k = 1) is the reach frequency of node 2 over the
    worlds 0 .. theta - 1 of stream tag 6: near 0.75 (the two-path probability, 5 sigma),
    where the direct-activation reading gives exactly 0.5; theta OPT^L is an integer
    equal to node 2's reach count from the oracle's sampling routine on those worlds."""
    og = oracle.OracleGraph.from_graph(_two_path_graph())
    theta = 20_000
    kw = dict(k=1, eps=0.5, delta=0.1, fixed_theta=500, key=3, inst=1)
    direct = og.solve([0], **kw)
    freq = og.solve([0], pr_worlds=theta, **kw)
    assert direct["OPT_L"] == 0.5
    sigma = math.sqrt(0.75 * 0.25 / theta)
    assert abs(freq["OPT_L"] - 0.75) < 5 * sigma
    cnt = freq["OPT_L"] * theta
    assert cnt == round(cnt)
    r = og.sample([0], theta=theta, key=3, tag=6, inst=1)
    assert int(r["reach"][2]) == int(round(cnt))
    assert int(r["reach"][1]) < int(r["reach"][2])
    # LHGA (out-degree 1 for both): the direct reading ties 0.5 * 1 = 0.5 * 1 and takes
    # the smaller id; the reach frequency ranks node 2 (about 0.75) first
    assert list(direct["B_R"]) == [1]
    assert list(freq["B_R"]) == [2]


def test_reach_frequency_zero_opt_is_an_error():
    """One world where no out-neighbour of S is reached: OPT^L = 0 cannot bound theta_max."""
    g = pin_graphs.graph(4, [(0, 1, 2.0 ** -20), (0, 2, 2.0 ** -20), (2, 3, 0.5)])
    og = oracle.OracleGraph.from_graph(g)
    with pytest.raises(ValueError):
        og.solve([0], k=1, eps=0.5, delta=0.1, fixed_theta=100, pr_worlds=1)
