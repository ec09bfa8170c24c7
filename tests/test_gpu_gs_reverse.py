"""Global Sampling worlds traversed backwards from the target (gs_rev.cu) give the same
LRR sets as the forward traversal: whole solves with the reverse path on and off equal
each other and the oracle, including worlds whose reverse set outgrows the warp's table
(p = 1 graphs, where a target's ancestors are many) and store growth."""
import numpy as np
import pytest

import oracle
from gpu_common import gpu_ctx, random_graph
from paper_2405_12871_gb300 import synth
from test_gpu_solve import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gpu_ctx()
    yield c
    c.close()


@pytest.mark.parametrize("graph", ["cl20k", "er1k", "dense"])
def test_gsbm_reverse_equals_forward_and_oracle(ctx, monkeypatch, graph):
    if graph == "cl20k":
        g = synth.chung_lu(20_000, 10.0, 2.1, seed=13)
        S = synth.seeds_top_outdeg(g, 10, 0.01, seed=14)
        kw = dict(k=12, eps=0.3, delta=1.0 / g.n, key=5, variant="gsbm")
    elif graph == "er1k":
        g, S, cfg = synth.workload_er1k()
        kw = dict(k=5, eps=0.2, delta=1.0 / g.n, variant="gsbm", fixed_theta=3000)
    else:   # large reverse sets: many worlds go to the forward kernel
        g = random_graph(21, 400, 3000, probs=(1.0, 0.75))
        S = [0, 1, 2]
        kw = dict(k=4, eps=0.3, delta=0.05, variant="gsbm", fixed_theta=500)
    og = oracle.OracleGraph.from_graph(g)
    G = ctx.load_graph(g)
    rev = G.solve(S, **kw)
    monkeypatch.setenv("IMIN_GS_REVERSE", "0")
    fwd = G.solve(S, **kw)
    monkeypatch.delenv("IMIN_GS_REVERSE")
    monkeypatch.setenv("IMIN_STORE_TIGHT", "1")
    tight = G.solve(S, **kw)
    G.free()
    want = og.solve(S, **kw)
    for got in (rev, fwd, tight):
        compare(got, want)
