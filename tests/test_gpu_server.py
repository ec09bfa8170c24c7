"""The server (continuous batching): queries submitted while others are in flight
are admitted between scheduler steps and share launches with them; every result
equals imin_solve on the same query alone.  A small concurrency limit makes
later queries wait for slots; polling reports EAGAIN while a query runs."""
import time

import numpy as np
import pytest

from gpu_common import gpu_ctx
from paper_2405_12871_gb300 import _lib, synth
from test_gpu_solve import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gpu_ctx()
    yield c
    c.close()


@pytest.mark.parametrize("max_active", [2, 16])
def test_server_results_equal_alone(ctx, max_active):
    g1, S1, _ = synth.workload_er1k()
    g2 = synth.chung_lu_poisson(30_000, 10.0, 2.1, seed=11)
    G1, G2 = ctx.load_graph(g1), ctx.load_graph(g2)
    rng = np.random.default_rng(max_active)
    qs = []
    for i in range(8):
        G, g = (G1, g1) if i % 2 == 0 else (G2, g2)
        S = synth.seeds_uniform(g.n, int(rng.integers(5, 30)), seed=100 + i)
        qs.append((G, S, int(rng.integers(3, 25)), 0.3, 1.0 / g.n, dict(key=i, inst=i)))
    alone = [G.solve(S, k, eps, delta, **kw) for (G, S, k, eps, delta, kw) in qs]
    srv = _lib.Server(ctx, max_active=max_active)
    tickets = []
    for i, (G, S, k, eps, delta, kw) in enumerate(qs):
        tickets.append(srv.submit(G, S, k, eps, delta, **kw))
        if i == 3:
            time.sleep(0.05)            # later queries arrive while earlier ones run
    early = srv.poll(tickets[-1], wait_ms=0)     # usually still running: None (EAGAIN)
    results = [srv.poll(t, wait_ms=-1) for t in tickets[:-1]]
    results.append(early if early is not None else srv.poll(tickets[-1], wait_ms=-1))
    srv.stop()
    for got, want in zip(results, alone):
        compare(got, want)
        assert got["latency_ms"] > 0
    G1.free()
    G2.free()
