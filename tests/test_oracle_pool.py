"""The split oracle world loop used by the full-size parity tests equals one oracle
call over the same worlds."""
import numpy as np

import oracle
import oracle_pool
from paper_2405_12871_gb300 import synth


def test_sample_parallel_equals_one_call():
    g, S, _ = synth.workload_er1k()
    og = oracle.OracleGraph.from_graph(g)
    B = np.array([3, 77, 500], np.int32)
    for mode in (1, 7):
        want = og.sample(S, B, theta=1001, first=13, key=2, tag=4, mode=mode, per_world=True)
        got = oracle_pool.sample_parallel(g, S, B, theta=1001, first=13, procs=3, chunk=97, key=2, tag=4,
                                          mode=mode)
        for k in ("reach", "credit_lower", "credit_upper", "world_spread"):
            assert np.array_equal(got[k], want[k]), k
        for k in ("total_spread", "edges_scanned", "nonempty_lrr"):
            assert got[k] == want[k], k
