"""Degenerate inputs of the newer entry points, against the oracle or closed forms:
no worlds, a graph without edges, seeds that reach nothing, a candidate that blocks
every out-neighbour of the seeds, the largest k, invalid candidate counts."""
import math

import numpy as np
import pytest

import oracle
from gpu_common import gpu_ctx
from paper_2405_12871_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gpu_ctx()
    yield c
    c.close()


def test_lrr_sequences_degenerate(ctx):
    from paper_2405_12871_gb300 import _lib
    g, S, _ = synth.workload_er1k()
    G = ctx.load_graph(g)
    r = G.lrr_sequences(S, (), [1, 2], theta=0)
    assert r["elements"] == r["cov"] == r["total_spread"] == r["worlds"] == 0
    assert int(r["credit_useq"].sum()) == 0
    with pytest.raises(_lib.IminError) as e:
        G.lrr_sequences(S, (), [1, 1], theta=5)          # duplicate query node
    assert e.value.code == _lib.IMIN_EINVAL
    G.free()
    # no edges: every world reaches the seeds only
    empty = synth.csr_from_edges(50, [], [], np.zeros(0, np.float32))
    G = ctx.load_graph(empty)
    r = G.lrr_sequences([3, 9], (), [3, 4], theta=20)
    assert r["elements"] == 0 and r["cov"] == 0 and r["total_spread"] == 40
    G.free()


def test_final_estimates_when_a_candidate_blocks_every_out_neighbour(ctx):
    from paper_2405_12871_gb300 import _lib
    g, S, _ = synth.workload_er1k()
    gs, gd = g.edges()
    on = np.setdiff1d(np.unique(gd[np.isin(gs, S)]), S)
    G = ctx.load_graph(g)
    gamma, delta = 0.1, 1.0 / g.n
    I, N = G.final_estimates(S, [on, []], gamma=gamma, delta=delta, key=2)
    # every world reaches exactly the seeds; W = 0 + |S|
    ups = 4 * (math.e - 2) * math.log(2 / delta) / gamma ** 2
    u1 = 1 + (1 + gamma) * ups
    nS = len(S)
    want_N = math.ceil(math.ceil(u1 * nS) / nS)
    assert N[0] == want_N and I[0] == pytest.approx(nS * u1 / want_N, rel=1e-14)
    og = oracle.OracleGraph.from_graph(g)
    for c, B in enumerate((on, [])):
        assert (N[c], I[c]) == og.stop_rule(S, B, beta=gamma, dprime=delta, key=2, tag=5)
    for bad in ([], [on, on, on, on]):
        with pytest.raises(_lib.IminError) as e:
            G.final_estimates(S, bad)
        assert e.value.code == _lib.IMIN_EINVAL
    G.free()


def test_solve_at_the_largest_k(ctx):
    g = synth.erdos_renyi(60, 400, seed=4)
    S = synth.seeds_uniform(g.n, 3, seed=5)
    G = ctx.load_graph(g)
    og = oracle.OracleGraph.from_graph(g)
    kw = dict(k=g.n - len(S) - 1, eps=0.3, delta=0.05, fixed_theta=200)
    got, want = G.solve(S, **kw), og.solve(S, **kw)
    assert list(got["blockers"]) == list(want["blockers"]) and got["I_after"] == want["I_after"]
    G.free()
