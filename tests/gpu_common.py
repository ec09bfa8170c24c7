"""Shared helpers of the GPU parity tests (CUDA path through the C ABI vs the oracle)."""
import numpy as np
import pytest

import oracle
from paper_2405_12871_gb300 import synth


def gpu_ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_12871_gb300 import _lib
    return _lib.Context(0)


def random_graph(seed, n, m, probs=None, self_loops=True, multi=True):
    """Small random digraph with self-loops / multi-edges allowed, given p values."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m)
    dst = rng.integers(0, n, m)
    if not self_loops:
        keep = src != dst
        src, dst = src[keep], dst[keep]
    if multi and m > 4:
        src = np.r_[src, src[:4]]
        dst = np.r_[dst, dst[:4]]
    if probs is None:
        p = rng.random(src.shape[0]).astype(np.float32)
    else:
        p = np.asarray(probs, np.float32)[rng.integers(0, len(probs), src.shape[0])]
    return synth.csr_from_edges(n, src, dst, p)


def assert_sample_equal(got, want, keys=("reach", "credit_lower", "credit_upper")):
    for k in keys:
        if k in got:
            g, w = np.asarray(got[k]), np.asarray(want[k])
            if not np.array_equal(g, w):
                bad = np.flatnonzero(g != w)[:10]
                raise AssertionError(f"{k} differs at {bad.tolist()}: gpu {g[bad].tolist()} "
                                     f"oracle {w[bad].tolist()}")
    for k in ("total_spread", "edges_scanned", "nonempty_lrr"):
        assert got[k] == want[k], (k, got[k], want[k])
    if "world_spread" in got and "world_spread" in want:
        assert np.array_equal(got["world_spread"], want["world_spread"])


ALL = 1 | 2 | 4
