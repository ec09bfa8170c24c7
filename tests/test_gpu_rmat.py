"""Sampled worlds of the full-size R-MAT workload (scale 22: 4,194,304 nodes,
65,243,094 edges after deduplication, trivalency p, |S| = 100 uniform seeds) through the
C ABI, against the oracle world by world: reach counts, lower and upper credits, per-
world spreads, edges scanned.  The worlds are taken at scattered indices so that several
Philox counter ranges are covered, with and without a blocked set, under the CTA shapes
the autotuner picks on power-law graphs and under the warp-per-world kernel.
"""
import numpy as np
import pytest

import oracle
from gpu_common import assert_sample_equal, gpu_ctx
from paper_2405_12871_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rmat():
    c = gpu_ctx()
    g, S, cfg = synth.workload_rmat4m()
    G = c.load_graph(g)
    og = oracle.OracleGraph.from_graph(g)
    rng = np.random.default_rng(31)
    B = rng.choice(np.setdiff1d(np.arange(g.n), S), 200, replace=False)
    yield g, S, B, G, og
    G.free()
    c.close()


@pytest.mark.parametrize("shape", ["256x8/g", "512x4/g", "1024x1/s", "warp"])
def test_rmat4m_sampled_worlds(rmat, monkeypatch, shape):
    g, S, B, G, og = rmat
    if shape == "warp":
        for k in ("IMIN_REACH_CTA", "IMIN_UPPER_CTA", "IMIN_LOWER_CTA"):
            monkeypatch.setenv(k, "0")
    else:
        sh, where = shape.split("/")
        bd, mb = sh.split("x")
        monkeypatch.setenv("IMIN_REACH_BD", bd)
        monkeypatch.setenv("IMIN_REACH_MINB", mb)
        monkeypatch.setenv("IMIN_REACH_SMEM", "1" if where == "s" else "0")
    for blocked, first, mode in (((), 0, 1), (B, 123_457, 1), ((), 7, 2), (B, 99_991, 3), ((), 31, 4),
                                 (B, 2**30, 5)):
        got = G.sample(S, blocked, theta=5, key=0, tag=3, first=first, mode=mode, per_world=True)
        want = og.sample(S, blocked, theta=5, key=0, tag=3, first=first, mode=mode, per_world=True)
        assert_sample_equal(got, want)
