"""The seeded input generators (shared by both sides, none of the method's arithmetic):
determinism, the recipe's shapes, and the sort-free fast paths giving the same graphs."""
import numpy as np

from paper_2405_12871_gb300 import synth


def _same(a, b):
    return (a.n == b.n and np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
            and np.array_equal(a.prob, b.prob))


def test_csr_from_edges_sorted_and_shuffled_inputs_agree():
    rng = np.random.default_rng(5)
    src = rng.integers(0, 300, 4000)
    dst = rng.integers(0, 300, 4000)
    p = rng.random(4000).astype(np.float32)
    g1 = synth.csr_from_edges(300, src, dst, p)
    order = np.lexsort((dst, src))
    g2 = synth.csr_from_edges(300, src[order], dst[order], p[order])   # takes the no-sort path
    assert _same(g1, g2)
    assert np.all(np.diff(g1.row_ptr) >= 0) and g1.row_ptr[-1] == 4000


def test_dedupe_drops_loops_and_repeats_in_order():
    src = np.array([3, 1, 1, 2, 2, 0, 3])
    dst = np.array([3, 2, 2, 0, 1, 1, 0])
    s, d = synth._dedupe(4, src, dst)
    assert list(zip(s.tolist(), d.tolist())) == [(0, 1), (1, 2), (2, 0), (2, 1), (3, 0)]


def test_generators_are_deterministic():
    assert _same(synth.chung_lu(5000, 8.0, 2.1, seed=3), synth.chung_lu(5000, 8.0, 2.1, seed=3))
    assert _same(synth.chung_lu_poisson(5000, 10.0, 2.1, seed=4), synth.chung_lu_poisson(5000, 10.0, 2.1, seed=4))
    assert _same(synth.rmat(12, 8, seed=2), synth.rmat(12, 8, seed=2))
    assert not _same(synth.rmat(12, 8, seed=2), synth.rmat(12, 8, seed=3))


def test_workload_shapes():
    g, S, cfg = synth.workload_er1k()
    assert g.n == 1000 and g.m == 5000 and len(S) == 10 and cfg["k"] == 5
    assert np.all(g.col != np.repeat(np.arange(g.n), np.diff(g.row_ptr)))   # no self-loops
    indeg = np.bincount(g.col, minlength=g.n)
    assert np.array_equal(g.prob, (np.float32(1.0) / indeg[g.col].astype(np.float32)).astype(np.float32))
    g = synth.rmat(14, 16, seed=1)
    assert g.n == 1 << 14 and set(np.unique(g.prob).tolist()) <= {np.float32(0.1), np.float32(0.01),
                                                                  np.float32(0.001)}
    items = synth.workload_batch(6)
    assert len(items) == 6
    for g, S, c in items:
        assert 1000 <= g.n <= 1_000_000 and 5 <= len(S) <= 100 and 1 <= c["k"] <= 200
        assert len(np.unique(S)) == len(S) and c["eps"] == 0.2
