"""GPU parity of the LRR-sequence estimator (imin_sample_lrr_sequences; Sec. 4.2,
"Discussion"): the per-node sequence credit, the per-world coverage of a query set and
the totals equal the oracle's bit for bit -- on the ER-1K parity graph, a small Chung-
Lu graph with hubs, p = 1 graphs (large closures, multi-edges, self-loops), and the
full 1M-node Chung-Lu workload."""
import numpy as np
import pytest

import oracle
from gpu_common import gpu_ctx, random_graph
from paper_2405_12871_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gpu_ctx()
    yield c
    c.close()


def _check(G, og, S, B, Q, theta, **kw):
    got = G.lrr_sequences(S, B, Q, theta=theta, **kw)
    want = og.lrr_sequences(S, B, Q, theta=theta, **kw)
    assert np.array_equal(got["credit_useq"], want["credit_useq"])
    assert np.array_equal(got["cov_world"], want["cov_world"])
    for k in ("elements", "cov", "total_spread"):
        assert got[k] == want[k], (k, got[k], want[k])
    assert got["worlds"] == theta
    return got


def test_er1k(ctx):
    g, S, cfg = synth.workload_er1k()
    G = ctx.load_graph(g)
    og = oracle.OracleGraph.from_graph(g)
    rng = np.random.default_rng(2)
    B = rng.choice(np.setdiff1d(np.arange(g.n), S), 30, replace=False)
    Q = rng.choice(np.setdiff1d(np.arange(g.n), S), 5, replace=False)
    r = _check(G, og, S, (), Q, 700, key=0, tag=3)
    assert r["elements"] > r["total_spread"]
    _check(G, og, S, B, Q, 500, key=2, tag=4, first=123_456)
    _check(G, og, S, B, (), 1, key=9, tag=0, first=2**32 - 1)
    G.free()


def test_small_chung_lu(ctx):
    g = synth.chung_lu(20_000, 10.0, 2.1, seed=3)
    S = synth.seeds_top_outdeg(g, 10, 0.01, seed=4)
    G = ctx.load_graph(g)
    og = oracle.OracleGraph.from_graph(g)
    Q = synth.seeds_top_outdeg(g, 40, 0.05, seed=9)
    Q = np.setdiff1d(Q, S)[:20]
    _check(G, og, S, (), Q, 400, key=1, tag=3)
    G.free()


@pytest.mark.parametrize("seed", [0, 1])
def test_p_one_graphs(ctx, seed):
    g = random_graph(50 + seed, 300, 1500, probs=(1.0, 0.5))
    S = [0, 7]
    G = ctx.load_graph(g)
    og = oracle.OracleGraph.from_graph(g)
    _check(G, og, S, (), [3, 4, 5], 50, key=seed, tag=2)
    G.free()


def test_cl1m(ctx):
    g, S, cfg = synth.workload_cl1m()
    G = ctx.load_graph(g)
    og = oracle.OracleGraph.from_graph(g)
    _check(G, og, S, (), [int(v) for v in S[:3] + 1], 96, key=0, tag=3, first=1000)
    G.free()
