"""GPU parity of the relabelled forward index (HotView) that the fused final estimates
traverse: nodes relabelled by reach frequency, edges copied with their whole 4-edge
groups, coins drawn from each group's original index.  The estimates count nodes, so
every result must equal the one on the original labels and the oracle's."""
import numpy as np
import pytest

import oracle
from gpu_common import gpu_ctx
from paper_2405_12871_gb300 import synth
from test_gpu_solve import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gpu_ctx()
    yield c
    c.close()


@pytest.mark.parametrize("hooks", [{}, {"IMIN_STOP_CHUNK": "613"}, {"IMIN_FINAL_QCAP": "400"},
                                   {"IMIN_HOT_WORLDS": "1"}, {"IMIN_HOT_WORLDS": "6000"},
                                   {"IMIN_REACH_SMEM": "0", "IMIN_AUTOTUNE": "0"}])
def test_solve_on_view_equals_oracle(ctx, monkeypatch, hooks):
    """Final estimates on the view (forced on a 20K-node Chung-Lu graph): in several
    chunks, with queue overflows re-run one candidate at a time on the original labels,
    with degenerate (1 world: two count values) and many (6,000) count values, and
    without the autotuner; then the same solve without the view."""
    for k, v in hooks.items():
        monkeypatch.setenv(k, v)
    g = synth.chung_lu(20_000, 10.0, 2.1, seed=7)
    S = synth.seeds_top_outdeg(g, 12, 0.01, seed=8)
    kw = dict(k=15, eps=0.3, delta=1.0 / g.n, key=4)
    G = ctx.load_graph(g)
    monkeypatch.setenv("IMIN_HOT_VIEW", "2")
    on = G.solve(S, **kw)
    monkeypatch.setenv("IMIN_HOT_VIEW", "0")
    off = G.solve(S, **kw)
    G.free()
    compare(on, off)
    compare(on, oracle.OracleGraph.from_graph(g).solve(S, **kw))
    # the view was built: its reach-count worlds and construction add launches
    assert on["kernel_launches"] > off["kernel_launches"]


def test_er1k_and_zero_degree_nodes_on_view(ctx, monkeypatch):
    """ER-1K (many rows that share a 4-edge group with their neighbours) and a graph
    where half the nodes have no out-edges, on the view."""
    monkeypatch.setenv("IMIN_HOT_VIEW", "2")
    g, S, cfg = synth.workload_er1k()
    G = ctx.load_graph(g)
    kw = dict(k=cfg["k"], eps=0.2, delta=1.0 / g.n, key=1)
    compare(G.solve(S, **kw), oracle.OracleGraph.from_graph(g).solve(S, **kw))
    G.free()
    rng = np.random.default_rng(3)
    n = 4000
    src = rng.integers(0, n // 2, 30_000) * 2          # only even nodes have out-edges
    dst = rng.integers(0, n, 30_000)
    keep = src != dst
    h = synth.weighted_cascade(synth.csr_from_edges(n, *synth._dedupe(n, src[keep], dst[keep])))
    S2 = np.array([0, 2, 4, 6, 8], np.int32)
    H = ctx.load_graph(h)
    kw = dict(k=8, eps=0.3, delta=1.0 / n, key=2)
    compare(H.solve(S2, **kw), oracle.OracleGraph.from_graph(h).solve(S2, **kw))
    H.free()


def test_final_estimates_entry_point_on_view(ctx, monkeypatch):
    """imin_final_estimates builds the view too; each candidate's (N, estimate) equals
    the oracle's stopping rule on the worlds of tag 5."""
    monkeypatch.setenv("IMIN_HOT_VIEW", "2")
    g = synth.chung_lu(20_000, 10.0, 2.1, seed=7)
    S = synth.seeds_top_outdeg(g, 12, 0.01, seed=8)
    og = oracle.OracleGraph.from_graph(g)
    rng = np.random.default_rng(5)
    pool = np.setdiff1d(np.arange(g.n), S)
    cands = [np.sort(rng.choice(pool, k, replace=False)) for k in (10, 25, 3)]
    G = ctx.load_graph(g)
    I, N = G.final_estimates(S, cands, gamma=0.1, delta=1.0 / g.n, key=6, inst=2, spread_hint=50.0)
    G.free()
    for c in range(3):
        wN, wI = og.stop_rule(S, cands[c], beta=0.1, dprime=1.0 / g.n, key=6, tag=5, inst=2)
        assert (N[c], I[c]) == (wN, wI), c
