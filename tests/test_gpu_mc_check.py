"""The final spread of the chosen blockers, re-estimated by independent Monte Carlo
(Algorithm 1 returns the candidate whose (gamma, delta)-estimate of the residual
spread is smallest, line 4): 10^6 worlds of a stream no solve draws (key 1, tag 9).

* GPU: the library's solve equals the oracle's, the library's 10^6-world count equals
  the oracle's bit for bit, and the solve's estimate of the chosen candidate lies
  within 1% of the independent mean.
* CPU (``not gpu``): the oracle alone, the same 1% check -- an independent pin of
  the oracle's final stopping-rule estimate.
"""
import numpy as np
import pytest

import oracle
from paper_2405_12871_gb300 import synth

MC_WORLDS = 1_000_000
MC_KEY, MC_TAG = 1, 9
TOL = 0.01
CASES = [(0.2, 5), (0.1, 10)]


def _mc_rel(I_after, ws):
    ws = np.asarray(ws, np.float64)
    mc = ws.mean()
    return abs(I_after - mc) / mc, ws.std(ddof=1) / np.sqrt(len(ws)) / mc


@pytest.mark.parametrize("eps,k", CASES[:1])
def test_oracle_final_estimate_against_independent_mc(eps, k):
    g, S, _ = synth.workload_er1k()
    og = oracle.OracleGraph.from_graph(g)
    r = og.solve(S, k=k, eps=eps, delta=1.0 / g.n)
    mc = og.sample(S, r["blockers"], theta=MC_WORLDS, key=MC_KEY, tag=MC_TAG, mode=oracle.MODE_REACH,
                   per_world=True)
    rel, se = _mc_rel(r["I_after"][r["chosen"]], mc["world_spread"])
    assert se < TOL / 5           # the Monte Carlo mean itself is far tighter than 1%
    assert rel <= TOL, (rel, r["I_after"], mc["total_spread"] / MC_WORLDS)


@pytest.mark.gpu
@pytest.mark.parametrize("eps,k", CASES)
def test_gpu_final_estimate_against_independent_mc(eps, k):
    from gpu_common import gpu_ctx
    from paper_2405_12871_gb300 import _lib
    ctx = gpu_ctx()
    g, S, _ = synth.workload_er1k()
    og = oracle.OracleGraph.from_graph(g)
    G = ctx.load_graph(g)
    kw = dict(k=k, eps=eps, delta=1.0 / g.n)
    r = G.solve(S, **kw)
    o = og.solve(S, **kw)
    assert list(r["blockers"]) == list(o["blockers"]) and r["I_after"] == o["I_after"]
    B = r["blockers"]
    got = G.sample(S, B, theta=MC_WORLDS, key=MC_KEY, tag=MC_TAG, mode=_lib.IMIN_REACH, per_world=True)
    want = og.sample(S, B, theta=MC_WORLDS, key=MC_KEY, tag=MC_TAG, mode=oracle.MODE_REACH,
                     per_world=True)
    assert got["total_spread"] == want["total_spread"]
    assert np.array_equal(got["world_spread"], want["world_spread"])
    assert np.array_equal(got["reach"], want["reach"])
    rel, se = _mc_rel(r["I_after"][r["chosen"]], got["world_spread"])
    assert se < TOL / 5
    assert rel <= TOL, (rel, r["I_after"], got["total_spread"] / MC_WORLDS)
    G.free()
    ctx.close()
