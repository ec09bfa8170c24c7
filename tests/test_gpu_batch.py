"""The batch engine (imin_solve_batch): a mixed batch -- different graphs, seed
sets, k, eps, keys, instance ids and variants, and an instance that ON answers
at once -- gives for every query exactly the result of imin_solve on that query
alone, and (for the graphs the oracle handles quickly) the oracle's result."""
import numpy as np
import pytest

import oracle
from gpu_common import gpu_ctx
from paper_2405_12871_gb300 import synth
from test_gpu_solve import FIELDS_F, FIELDS_INT, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gpu_ctx()
    yield c
    c.close()


def test_mixed_batch_equals_alone_and_oracle(ctx):
    g1, S1, cfg1 = synth.workload_er1k()
    g2 = synth.chung_lu(20_000, 10.0, 2.1, seed=3)
    S2 = synth.seeds_top_outdeg(g2, 10, 0.01, seed=4)
    g3 = synth.chung_lu(5_000, 8.0, 2.3, seed=7)
    S3 = synth.seeds_uniform(g3.n, 12, seed=8)
    n = 12
    edges = [(0, 1), (0, 2), (1, 3), (2, 3)] + [(3, i) for i in range(4, n)]
    g4 = synth.csr_from_edges(n, [e[0] for e in edges], [e[1] for e in edges])
    G1, G2, G3, G4 = (ctx.load_graph(g) for g in (g1, g2, g3, g4))
    qs = [
        (G1, S1, 5, 0.2, 1.0 / g1.n, dict(key=0, inst=0)),
        (G2, S2, 20, 0.3, 1.0 / g2.n, dict(key=3, inst=1)),
        (G1, S1, 3, 0.5, 0.01, dict(key=9, inst=2, variant="sandimin-")),
        (G3, S3, 15, 0.25, 1.0 / g3.n, dict(key=4, inst=3)),
        (G4, [0], 2, 0.2, 0.05, dict(inst=4)),                      # |ON| <= k
        (G4, [0], 1, 0.2, 0.05, dict(inst=5, variant="lsbm")),
        (G1, S1, 5, 0.2, 1.0 / g1.n, dict(key=0, inst=0, fixed_theta=3000)),
    ]
    batch = ctx.solve_batch(qs)
    assert len(batch) == len(qs)
    for (G, S, k, eps, delta, kw), got in zip(qs, batch):
        alone = G.solve(S, k, eps, delta, **kw)
        compare(got, alone)
    # oracle on the small graphs
    ogs = {id(G1): oracle.OracleGraph.from_graph(g1), id(G3): oracle.OracleGraph.from_graph(g3),
           id(G4): oracle.OracleGraph.from_graph(g4)}
    for (G, S, k, eps, delta, kw), got in zip(qs, batch):
        if id(G) in ogs:
            compare(got, ogs[id(G)].solve(S, k, eps, delta, **kw))
    for G in (G1, G2, G3, G4):
        G.free()


@pytest.mark.parametrize("window", [None, "3", "2:6"])
def test_batch_of_many_small_instances(ctx, monkeypatch, window):
    """All ten instances in flight at once, a rolling window of three admitted as
    others finish, or a window that starts at two and widens by two per step up to six:
    the results equal the one-at-a-time solves every way."""
    if window:
        monkeypatch.setenv("IMIN_BATCH_ACTIVE", window)
    gs = [synth.chung_lu(int(n), 10.0, 2.1, seed=20 + i)
          for i, n in enumerate(np.geomspace(1000, 30_000, 10).astype(int))]
    Gs = [ctx.load_graph(g) for g in gs]
    qs = []
    for i, (g, G) in enumerate(zip(gs, Gs)):
        S = synth.seeds_top_outdeg(g, 5 + 3 * i, 0.01, seed=40 + i)
        qs.append((G, S, 10 + i, 0.3, 1.0 / g.n, dict(key=i, inst=i)))
    batch = ctx.solve_batch(qs)
    for (G, S, k, eps, delta, kw), got in zip(qs, batch):
        compare(got, G.solve(S, k, eps, delta, **kw))
    for G in Gs:
        G.free()
