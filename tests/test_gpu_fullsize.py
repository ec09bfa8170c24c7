"""Full-size parity of the benchmark's dominant launch: one multi-world launch on the
1M-node Chung-Lu workload in the launch shape the benchmark runs (256 threads x 8
CTAs per SM, visited bitmaps in global memory), compared with the oracle element by
element -- every node's reach count and every world's spread.  The oracle's world
loop is split over the host cores (``oracle_pool``).  Also: the three final
estimates of a full-size solve, fused and one candidate at a time, agree exactly, and
the whole solve is the same with the final estimates on the relabelled forward index
and on the original one.
"""
import numpy as np
import pytest

import oracle_pool
from gpu_common import assert_sample_equal, gpu_ctx
from paper_2405_12871_gb300 import synth
from test_gpu_solve import compare

pytestmark = pytest.mark.gpu

BENCH_SHAPE = {"IMIN_REACH_BD": "256", "IMIN_REACH_MINB": "8", "IMIN_REACH_SMEM": "0",
               "IMIN_AUTOTUNE": "0"}


@pytest.fixture(scope="module")
def cl1m():
    c = gpu_ctx()
    g, S, cfg = synth.workload_cl1m()
    G = c.load_graph(g)
    yield g, S, cfg, G
    G.free()
    c.close()


@pytest.mark.parametrize("blocked,first,tag", [(False, 0, 0), (True, 40_000, 5)])
def test_cl1m_multiworld_launch_elementwise(cl1m, monkeypatch, blocked, first, tag):
    g, S, cfg, G = cl1m
    for k, v in BENCH_SHAPE.items():
        monkeypatch.setenv(k, v)
    B = ()
    if blocked:
        rng = np.random.default_rng(12)
        B = np.sort(rng.choice(np.setdiff1d(np.arange(g.n), S), 100, replace=False)).astype(np.int32)
    theta = 2048
    from paper_2405_12871_gb300 import _lib
    got = G.sample(S, B, theta=theta, first=first, key=0, tag=tag, mode=_lib.IMIN_REACH, per_world=True)
    want = oracle_pool.sample_parallel(g, S, B, theta=theta, first=first, key=0, tag=tag, mode=1)
    assert_sample_equal(got, want, keys=("reach",))
    assert np.array_equal(got["world_spread"], want["world_spread"])


def test_cl1m_solve_final_estimates_fused_equal_separate(cl1m, monkeypatch):
    g, S, cfg, G = cl1m
    kw = dict(k=cfg["k"], eps=cfg["eps"], delta=cfg["delta"], key=cfg["key"])
    fused = G.solve(S, **kw)
    monkeypatch.setenv("IMIN_FINAL_FUSED", "0")
    sep = G.solve(S, **kw)
    assert list(fused["blockers"]) == list(sep["blockers"])
    assert fused["n_final"] == sep["n_final"] and fused["I_after"] == sep["I_after"]
    assert fused["n_spread"] == sep["n_spread"] and fused["I_hat"] == sep["I_hat"]
    # the fused final estimates above ran on the relabelled forward index (on by default
    # for this graph); on the original labels every result is the same
    monkeypatch.delenv("IMIN_FINAL_FUSED")
    monkeypatch.setenv("IMIN_HOT_VIEW", "0")
    plain = G.solve(S, **kw)
    compare(fused, plain)
    assert fused["kernel_launches"] > plain["kernel_launches"]


def test_rmat4m_multiworld_launch_elementwise(monkeypatch):
    """The R-MAT-4M workload (4,194,304 nodes, 65M edges; a world reaches about half a
    million nodes over some 57M scanned edges): one multi-world launch of 128 worlds
    in the benchmark's launch shape, element by element against the split oracle."""
    for k, v in BENCH_SHAPE.items():
        monkeypatch.setenv(k, v)
    c = gpu_ctx()
    g, S, cfg = synth.workload_rmat4m()
    G = c.load_graph(g)
    from paper_2405_12871_gb300 import _lib
    got = G.sample(S, theta=128, first=1000, key=0, tag=0, mode=_lib.IMIN_REACH, per_world=True)
    G.free()
    c.close()
    want = oracle_pool.sample_parallel(g, S, theta=128, first=1000, chunk=8, key=0, tag=0, mode=1)
    assert_sample_equal(got, want, keys=("reach",))
    assert np.array_equal(got["world_spread"], want["world_spread"])
