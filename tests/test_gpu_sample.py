"""GPU parity of imin_sample (reach counts, lower credit, upper credit) against
the oracle, bit for bit, through the C ABI.

Covers: the ER 1,000-node / 5,000-edge workload (theta = 10,000, key 0) in every
mode; blocked sets; self-loops, multi-edges, p in {0, 1}; several keys, tags,
instances and first-sample offsets; theta = 0; the deferred-world path (per-warp
queue overflow re-run on large slots); a small Chung-Lu graph with hubs; input
validation; and sampled worlds of the full-size 1M-node Chung-Lu workload.
"""
import os

import numpy as np
import pytest

import oracle
from gpu_common import ALL, assert_sample_equal, gpu_ctx, random_graph
from paper_2405_12871_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gpu_ctx()
    yield c
    c.close()


@pytest.fixture(scope="module")
def er1k(ctx):
    g, S, cfg = synth.workload_er1k()
    G = ctx.load_graph(g)
    yield g, S, cfg, G, oracle.OracleGraph.from_graph(g)
    G.free()


@pytest.mark.parametrize("mode", [1, 2, 4, ALL])
def test_er1k_theta_10000(er1k, mode):
    g, S, cfg, G, og = er1k
    theta = cfg["theta"]
    got = G.sample(S, theta=theta, key=0, tag=1, mode=mode, per_world=True)
    want = og.sample(S, theta=theta, key=0, tag=1, mode=mode, per_world=True)
    assert_sample_equal(got, want)
    assert want["total_spread"] > theta * len(S)      # the workload does spread


def test_er1k_blocked_and_offsets(er1k):
    g, S, cfg, G, og = er1k
    rng = np.random.default_rng(9)
    B = rng.choice(np.setdiff1d(np.arange(g.n), S), 25, replace=False)
    for key, tag, inst, first in ((0, 0, 0, 0), (7, 3, 2, 123_456), (2**64 - 1, 6, 9, 2**31)):
        got = G.sample(S, B, theta=1500, key=key, tag=tag, inst=inst, first=first, mode=ALL,
                       per_world=True)
        want = og.sample(S, B, theta=1500, key=key, tag=tag, inst=inst, first=first, mode=ALL,
                         per_world=True)
        assert_sample_equal(got, want)
        assert all(int(got["reach"][b]) == 0 for b in B)


@pytest.mark.parametrize("seed", range(6))
def test_random_small_graphs(ctx, seed):
    probs = [(0.0, 1.0, 0.5), None, (1.0,), (0.3, 0.05), None, (0.9, 0.0)][seed]
    n = [7, 40, 25, 300, 1000, 64][seed]
    m = [20, 150, 60, 2000, 6000, 500][seed]
    g = random_graph(seed, n, m, probs)
    G = ctx.load_graph(g)
    og = oracle.OracleGraph.from_graph(g)
    rng = np.random.default_rng(seed)
    S = rng.choice(n, min(n - 1, 1 + seed % 5), replace=False)
    B = rng.choice(np.setdiff1d(np.arange(n), S), min(3, n - len(S) - 1), replace=False) \
        if seed % 2 else []
    got = G.sample(S, B, theta=2000, key=seed, tag=4, mode=ALL, per_world=True)
    want = og.sample(S, B, theta=2000, key=seed, tag=4, mode=ALL, per_world=True)
    assert_sample_equal(got, want)
    G.free()


def test_theta_zero_and_edgeless(ctx):
    g = synth.csr_from_edges(5, np.array([], int), np.array([], int))
    G = ctx.load_graph(g)
    got = G.sample([1, 3], theta=0, mode=ALL)
    assert got["total_spread"] == 0 and not got["reach"].any()
    got = G.sample([1, 3], theta=10, mode=ALL, per_world=True)
    assert got["total_spread"] == 20 and list(got["world_spread"]) == [2] * 10
    assert int(got["reach"][1]) == 10 and not got["credit_lower"].any()
    G.free()


@pytest.mark.parametrize("mode", [2, 3])
def test_lower_pairs_overflow_to_large_slots(er1k, monkeypatch, mode):
    """A 40-pair budget per CTA slot sends most lower-bound worlds to the large-slot
    pass; the counts are unchanged."""
    g, S, cfg, G, og = er1k
    monkeypatch.setenv("IMIN_SLOT_QCAP", "40")
    got = G.sample(S, theta=2000, key=6, tag=3, mode=mode, per_world=True)
    monkeypatch.delenv("IMIN_SLOT_QCAP")
    want = og.sample(S, theta=2000, key=6, tag=3, mode=mode, per_world=True)
    assert_sample_equal(got, want)


def test_deferred_worlds_match(er1k, monkeypatch):
    """A tiny per-warp queue forces most worlds through the large-slot path."""
    g, S, cfg, G, og = er1k
    monkeypatch.setenv("IMIN_SLOT_QCAP", "40")
    got = G.sample(S, theta=3000, key=5, tag=2, mode=ALL, per_world=True)
    monkeypatch.delenv("IMIN_SLOT_QCAP")
    want = og.sample(S, theta=3000, key=5, tag=2, mode=ALL, per_world=True)
    assert_sample_equal(got, want)


@pytest.fixture(scope="module")
def hubs30k():
    """A 30,000-node Chung-Lu graph with hubs (many nodes above the hub threshold of
    the CTA kernel), its seeds, 40 blocked nodes and the oracle's reach-only worlds."""
    g = synth.chung_lu(30_000, 12.0, 2.1, seed=11)
    S = synth.seeds_top_outdeg(g, 30, 0.01, seed=12)
    rng = np.random.default_rng(13)
    B = rng.choice(np.setdiff1d(np.arange(g.n), S), 40, replace=False)
    og = oracle.OracleGraph.from_graph(g)
    cases = (([], 700, 0, 1), (B, 500, 77_777, 1), ([], 600, 5, 5), (B, 400, 999, 4),
             ([], 300, 11, 3), (B, 300, 4242, 2))
    want = [og.sample(S, b, theta=t, key=3, tag=5, first=f, mode=md, per_world=True)
            for b, t, f, md in cases]
    return g, S, cases, want


REACH_CONFIGS = ["warp"] + [f"{bd}x{mb}/{w}" for bd, mb in ((256, 4), (256, 8), (512, 2), (512, 4),
                                                            (1024, 1), (1024, 2)) for w in "gs"]


@pytest.mark.parametrize("cfg", REACH_CONFIGS)
def test_reach_launch_configurations(ctx, monkeypatch, hubs30k, cfg):
    """Reach-only, lower-bound (dominator / CP) and upper-bound (LRR) worlds give the
    same bits under every launch configuration the autotuner may pick: warp-per-world,
    or a CTA per world of 256/512/1024 threads compiled for a given number of CTAs per
    SM, with the visited bitmap in global (g) or shared (s) memory."""
    g, S, cases, want = hubs30k
    if cfg == "warp":
        monkeypatch.setenv("IMIN_REACH_CTA", "0")
        monkeypatch.setenv("IMIN_UPPER_CTA", "0")
        monkeypatch.setenv("IMIN_LOWER_CTA", "0")
    else:
        shape, where = cfg.split("/")
        bd, mb = shape.split("x")
        monkeypatch.setenv("IMIN_REACH_BD", bd)
        monkeypatch.setenv("IMIN_REACH_MINB", mb)
        monkeypatch.setenv("IMIN_REACH_SMEM", "1" if where == "s" else "0")
    G = ctx.load_graph(g)
    for (blocked, theta, first, md), w in zip(cases, want):
        got = G.sample(S, blocked, theta=theta, key=3, tag=5, first=first, mode=md, per_world=True)
        assert_sample_equal(got, w)
        if md & 4:
            assert w["nonempty_lrr"] > 0
    G.free()


@pytest.mark.parametrize("cfg", ["512x4/g", "1024x1/s", "256x8/s"])
def test_reach_many_hubs_in_one_level(ctx, monkeypatch, cfg):
    """400 hubs in one BFS level: more than the CTA kernel stages for its hub pass,
    so the rest are expanded by the warp that met them."""
    rng = np.random.default_rng(21)
    nh, deg, ns = 400, 160, 8
    n = ns + nh + 30_000
    hubs = np.arange(ns, ns + nh)
    src = [np.repeat(np.arange(ns), nh), np.repeat(hubs, deg)]
    dst = [np.tile(hubs, ns), rng.integers(ns + nh, n, nh * deg)]
    src, dst = np.concatenate(src), np.concatenate(dst)
    prob = np.where(src < ns, 1.0, 0.3).astype(np.float32)
    g = synth.csr_from_edges(n, src, dst, prob)
    shape, where = cfg.split("/")
    bd, mb = shape.split("x")
    monkeypatch.setenv("IMIN_REACH_BD", bd)
    monkeypatch.setenv("IMIN_REACH_MINB", mb)
    monkeypatch.setenv("IMIN_REACH_SMEM", "1" if where == "s" else "0")
    G = ctx.load_graph(g)
    og = oracle.OracleGraph.from_graph(g)
    S = np.arange(ns)
    for mode in (1, 4):
        got = G.sample(S, theta=200, key=9, tag=2, mode=mode, per_world=True)
        want = og.sample(S, theta=200, key=9, tag=2, mode=mode, per_world=True)
        assert_sample_equal(got, want)
        assert want["total_spread"] > 200 * (ns + nh)
    G.free()


@pytest.mark.parametrize("shape", ["256x8", "512x4", "1024x2"])
def test_smem_bitmap_above_default_dynamic_limit(ctx, monkeypatch, shape):
    """A 300,000-node graph: its visited bitmap (37.5 KB) plus the kernel's static shared
    memory passes the 48 KB that a launch gets without opting in, while the bitmap alone
    does not; every mode must still launch and match the oracle."""
    g = synth.chung_lu_poisson(300_000, 10.0, 2.1, seed=8)
    S = synth.seeds_top_outdeg(g, 20, 0.01, seed=9)
    bd, mb = shape.split("x")
    monkeypatch.setenv("IMIN_REACH_BD", bd)
    monkeypatch.setenv("IMIN_REACH_MINB", mb)
    monkeypatch.setenv("IMIN_REACH_SMEM", "1")
    G = ctx.load_graph(g)
    og = oracle.OracleGraph.from_graph(g)
    for mode in (1, 2, 4):
        got = G.sample(S, theta=60, key=4, tag=6, first=1000, mode=mode, per_world=True)
        want = og.sample(S, theta=60, key=4, tag=6, first=1000, mode=mode, per_world=True)
        assert_sample_equal(got, want)
    G.free()


def test_small_chung_lu_hubs(ctx):
    g = synth.chung_lu(20_000, 10.0, 2.1, seed=3)
    S = synth.seeds_top_outdeg(g, 20, 0.01, seed=4)
    G = ctx.load_graph(g)
    og = oracle.OracleGraph.from_graph(g)
    got = G.sample(S, theta=400, key=1, tag=1, mode=ALL, per_world=True)
    want = og.sample(S, theta=400, key=1, tag=1, mode=ALL, per_world=True)
    assert_sample_equal(got, want)
    G.free()


def test_validation(ctx, er1k):
    from paper_2405_12871_gb300 import _lib
    g, S, cfg, G, og = er1k
    with pytest.raises(_lib.IminError) as e:
        G.sample([1, 1, 2], theta=5)
    assert e.value.code == _lib.IMIN_EINVAL
    with pytest.raises(_lib.IminError) as e:
        G.sample([1, 2], blocked=[2], theta=5)
    assert e.value.code == _lib.IMIN_EINVAL
    with pytest.raises(_lib.IminError) as e:
        G.sample([g.n], theta=5)
    assert e.value.code == _lib.IMIN_EINVAL
    with pytest.raises(_lib.IminError) as e:
        G.sample([1], theta=5, first=2**32 - 2)
    assert e.value.code == _lib.IMIN_ERANGE
    bad = synth.Graph(3, np.array([0, 1, 2, 2], np.int32), np.array([1, 2], np.int32),
                      np.array([0.5, np.nan], np.float32))
    with pytest.raises(_lib.IminError) as e:
        ctx.load_graph(bad)
    assert e.value.code == _lib.IMIN_EINVAL
    bad = synth.Graph(3, np.array([0, 2, 1, 2], np.int32), np.array([1, 2], np.int32),
                      np.array([0.5, 0.5], np.float32))
    with pytest.raises(_lib.IminError) as e:
        ctx.load_graph(bad)
    assert e.value.code == _lib.IMIN_EINVAL


@pytest.fixture(scope="module")
def cl1m(ctx):
    g, S, cfg = synth.workload_cl1m()
    G = ctx.load_graph(g)
    yield g, S, cfg, G
    G.free()


def test_cl1m_sampled_worlds(cl1m):
    """Full-size 1M-node Chung-Lu workload: scattered single worlds, every mode."""
    g, S, cfg, G = cl1m
    og = oracle.OracleGraph.from_graph(g)
    for j in (0, 1, 977, 50_000, 123_457, 2**31 + 5):
        for tag in (0, 1, 3):
            got = G.sample(S, theta=1, first=j, key=0, tag=tag, mode=ALL, per_world=True)
            want = og.sample(S, theta=1, first=j, key=0, tag=tag, mode=ALL, per_world=True)
            assert_sample_equal(got, want)


def test_cl1m_batch_spread_in_bench_configuration(cl1m):
    """The stopping-rule launch shape: many worlds at once; per-world spreads of a
    random sample of them equal the oracle's, and totals are consistent."""
    g, S, cfg, G = cl1m
    theta = 20_000
    got = G.sample(S, theta=theta, key=0, tag=0, mode=1, per_world=True)
    ws = got["world_spread"]
    assert int(ws.sum()) == got["total_spread"]
    assert int(got["reach"].sum()) == got["total_spread"]
    assert all(int(got["reach"][s]) == theta for s in S)
    og = oracle.OracleGraph.from_graph(g)
    rng = np.random.default_rng(0)
    for j in rng.choice(theta, 12, replace=False):
        want = og.sample(S, theta=1, first=int(j), key=0, tag=0, per_world=True)
        assert int(ws[j]) == int(want["world_spread"][0])
