"""AG and GR through the library's sampler: the same blockers, estimate counts and
worlds as with the oracle's sampler (every estimate is an integer credit vector, so the
choices match exactly)."""
import numpy as np
import pytest

import oracle
from gpu_common import gpu_ctx
from paper_2405_12871_gb300 import baselines, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gpu_ctx()
    yield c
    c.close()


def test_paper_example_on_gpu(ctx):
    src = [0, 0, 1, 2, 3, 3, 3]
    dst = [1, 2, 3, 3, 4, 5, 6]
    g = synth.csr_from_edges(7, src, dst, np.ones(7, np.float32))
    G = ctx.load_graph(g)
    assert baselines.advanced_greedy(G.sample, g.n, [0], k=2, theta=3)[0] == [3, 1]
    assert sorted(baselines.greedy_replace(G.sample, g, [0], k=2, theta=3)[0]) == [1, 2]
    G.free()


@pytest.mark.parametrize("algo", ["ag", "gr"])
def test_er1k_matches_oracle(ctx, algo):
    g, S, cfg = synth.workload_er1k()
    G = ctx.load_graph(g)
    og = oracle.OracleGraph.from_graph(g)
    if algo == "ag":
        got = baselines.advanced_greedy(G.sample, g.n, S, k=5, theta=2000, key=3)
        want = baselines.advanced_greedy(og.sample, g.n, S, k=5, theta=2000, key=3)
    else:
        got = baselines.greedy_replace(G.sample, g, S, k=5, theta=2000, key=3)
        want = baselines.greedy_replace(og.sample, g, S, k=5, theta=2000, key=3)
    assert got == want
    assert len(got[0]) == 5
    G.free()


@pytest.mark.parametrize("algo", ["ag", "gr"])
def test_cl5k_matches_the_oracles_own_ag_gr(ctx, algo):
    """The package's AG / GR over the library's sampler against the oracle's separate C
    implementation over its own worlds."""
    g = synth.chung_lu(5000, 10.0, 2.1, seed=11)
    S = synth.seeds_top_outdeg(g, 8, 0.01, seed=12)
    G = ctx.load_graph(g)
    og = oracle.OracleGraph.from_graph(g)
    if algo == "ag":
        got = baselines.advanced_greedy(G.sample, g.n, S, k=6, theta=500, key=3)
    else:
        got = baselines.greedy_replace(G.sample, g, S, k=6, theta=500, key=3)
    assert got[:2] == og.dt_baseline(algo, S, 6, 500, key=3)
    G.free()
