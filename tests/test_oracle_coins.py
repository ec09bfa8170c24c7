"""Pins for the oracle's random source: Philox4x32-10 and the edge coin.

* Philox: the published known-answer vectors (tests/golden/philox_kat.txt) and an
  independent implementation present on this machine (Triton's Philox, run by its
  CPU interpreter).
* Coin rule: live <=> (w >> 8) < T(p) must equal the real-number rule
  u * 2^-24 < p for every one of the 2^24 values u, for a sweep of fp32 p.
* Empirical rate: an edge is live in a fraction p_q = T(p)/2^24 of worlds.
* Target draw: floor(r64 * count / 2^64) is uniform over [0, count).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from conftest import GOLDEN, ROOT
import oracle


def _kat():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = oracle.philox4x32_10(ctr, key)
        assert [int(x) for x in got] == want


_TRITON_SCRIPT = r"""
import numpy as np, torch, triton, triton.language as tl, sys
@triton.jit
def k(c0p, c1p, c2p, c3p, outp, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i),
                           tl.load(c3p + i), 10)
    tl.store(outp + i * 4, a.to(tl.int32, bitcast=True))
    tl.store(outp + i * 4 + 1, b.to(tl.int32, bitcast=True))
    tl.store(outp + i * 4 + 2, c.to(tl.int32, bitcast=True))
    tl.store(outp + i * 4 + 3, d.to(tl.int32, bitcast=True))
rng = np.random.default_rng(7)
N = 64
ctr = rng.integers(0, 2**32, size=(N, 4), dtype=np.uint64).astype(np.uint32)
for key in (0, 0x0123456789ABCDEF, 2**64 - 1):
    cs = [torch.tensor(ctr[:, i].view(np.int32).copy()) for i in range(4)]
    out = torch.zeros(N * 4, dtype=torch.int32)
    s = key - 2**64 if key >= 2**63 else key
    k[(1,)](*cs, out, s, N=N)
    o = out.numpy().view(np.uint32).reshape(N, 4)
    for r in range(N):
        print(key, *[int(x) for x in ctr[r]], *[int(x) for x in o[r]])
"""


def test_philox_matches_triton_interpreter():
    pytest.importorskip("triton")
    env = dict(os.environ, TRITON_INTERPRET="1")
    try:
        out = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], env=env, capture_output=True,
                             text=True, timeout=600)
    except subprocess.TimeoutExpired:
        pytest.skip("triton interpreter too slow here")
    if out.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + out.stderr.strip().splitlines()[-1])
    n = 0
    for line in out.stdout.split("\n"):
        if not line.strip():
            continue
        v = [int(x) for x in line.split()]
        key, ctr, want = v[0], v[1:5], v[5:9]
        got = oracle.philox4x32_10(ctr, [key & 0xFFFFFFFF, key >> 32])
        assert [int(x) for x in got] == want
        n += 1
    assert n == 3 * 64


def _p_sweep():
    ps = [0.0, 1.0, 0.5, 0.1, 0.01, 0.001, 1.0 / 3.0, 1e-9, 2.0**-24, 2.0**-25,
          1.0 - 2.0**-24, np.nextafter(np.float32(1), np.float32(0))]
    rng = np.random.default_rng(3)
    ps += list(rng.random(12).astype(np.float32))
    ps += [np.float32(1.0) / np.float32(d) for d in (3, 7, 10, 97, 1000, 12345)]
    return [np.float32(p) for p in ps]


@pytest.mark.parametrize("p", _p_sweep())
def test_coin_threshold_equals_real_rule(p):
    """For every 24-bit u: (u < T(p)) == (u * 2^-24 < p), evaluated in float64 by numpy."""
    T = oracle.coin_threshold(float(p))
    u = np.arange(1 << 24, dtype=np.float64)
    real = (u * 2.0**-24) < np.float64(p)
    assert int(real.sum()) == T
    assert bool(np.all(real[:T])) and not bool(np.any(real[T:]))


def test_coin_extremes():
    assert oracle.coin_threshold(0.0) == 0
    assert oracle.coin_threshold(1.0) == 1 << 24


def test_coin_empirical_rate():
    """Edge e of a 1-edge-per-node star is live in ~p_q of worlds (5 sigma)."""
    n = 9
    p = np.array([0.5, 0.1, 0.01, 0.9, 1.0, 0.0, 0.3, 0.77], np.float32)
    # node 0 -> nodes 1..8
    row_ptr = np.array([0] + [8] * n, np.int32)
    col = np.arange(1, n, dtype=np.int32)
    g = oracle.OracleGraph(n, row_ptr, col, p)
    theta = 20000
    out = g.sample([0], theta=theta, key=11, tag=0)
    for i, pi in enumerate(p):
        pq = oracle.coin_threshold(float(pi)) / 2.0**24
        got = int(out["reach"][i + 1]) / theta
        sd = np.sqrt(max(pq * (1 - pq), 1e-12) / theta)
        if pq in (0.0, 1.0):
            assert got == pq
        else:
            assert abs(got - pq) < 5 * sd, (i, pi, got, pq)


def test_target_index_uniform_and_bounded():
    cnt = 7
    hits = np.zeros(cnt, int)
    for j in range(7000):
        t = oracle.target_index(5, j, 3, 0, cnt)
        assert 0 <= t < cnt
        hits[t] += 1
    # chi-square with 6 dof: 99.99th percentile ~ 27.9
    chi2 = ((hits - 1000) ** 2 / 1000).sum()
    assert chi2 < 27.9
    assert oracle.target_index(5, 0, 3, 0, 1) == 0
