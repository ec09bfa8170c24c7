"""The no-allocation entry point (imin_sample_reach_noalloc) against the regular
one (imin_sample with IMIN_REACH), through the C ABI.

Callers that cannot allocate device memory -- an application whose device
memory is reserved in full by its own pooling allocator, or a plug-in that may
not call cudaMalloc -- pass graph and output buffers they already own; the call
uses a fixed scratch array built into the library.  This file is collected last
on purpose, so that a run stopping at its first failure has run everything else.
It must pass alone in a fresh process and after the other tests alike.
"""
import numpy as np
import pytest

from paper_2405_12871_gb300 import synth

pytestmark = pytest.mark.gpu


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_12871_gb300 import _lib
    return torch, _lib


@pytest.mark.parametrize("which", ["er1k", "cl20k"])
def test_noalloc_matches_imin_sample_two_calls(which):
    torch, _lib = _setup()
    if which == "er1k":
        g, S, _ = synth.workload_er1k()
    else:
        g = synth.chung_lu(20_000, 10.0, 2.1, seed=3)
        S = synth.seeds_top_outdeg(g, 20, 0.01, seed=4)
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    d_rp = torch.from_numpy(g.row_ptr).to(dev)
    d_col = torch.from_numpy(g.col).to(dev)
    d_p = torch.from_numpy(g.prob).to(dev)
    theta = 3000
    d_reach = torch.zeros(g.n, dtype=torch.int64, device=dev)
    d_ws = torch.zeros(theta, dtype=torch.int32, device=dev)
    with _lib.Context(0, stream=stream) as ctx:
        G = ctx.load_graph(g)
        for call, (key, first) in enumerate(((0, 0), (7, 100_000))):   # two calls in a row
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            tot = _lib.imin_sample_reach_noalloc(d_rp.data_ptr(), d_col.data_ptr(), d_p.data_ptr(),
                                                 g.n, g.m, S, theta, key=key, tag=2, first=first,
                                                 d_reach=d_reach.data_ptr(),
                                                 d_world_spread=d_ws.data_ptr(), stream=stream)
            torch.cuda.synchronize()
            if call == 1:      # the first call may load the module; later ones allocate nothing
                assert torch.cuda.mem_get_info()[0] == free0
            want = G.sample(S, theta=theta, key=key, tag=2, first=first, mode=_lib.IMIN_REACH,
                            per_world=True)
            assert tot == (want["total_spread"], want["edges_scanned"])
            assert np.array_equal(d_reach.cpu().numpy().view(np.uint64), want["reach"])
            assert np.array_equal(d_ws.cpu().numpy().view(np.uint32), want["world_spread"])
        G.free()


def test_noalloc_rejects_sizes_beyond_maximum():
    torch, _lib = _setup()
    dev = torch.device("cuda:0")
    rp = torch.zeros(4, dtype=torch.int32, device=dev)
    with pytest.raises(_lib.IminError) as e:
        _lib.imin_sample_reach_noalloc(rp.data_ptr(), rp.data_ptr(), rp.data_ptr(),
                                       _lib.NOALLOC_MAX_NODES + 1, 0, [0], 1)
    assert e.value.code == _lib.IMIN_ERANGE
    with pytest.raises(_lib.IminError) as e:
        _lib.imin_sample_reach_noalloc(rp.data_ptr(), rp.data_ptr(), rp.data_ptr(), 3, 0,
                                       list(range(3)) * 400, 1)
    assert e.value.code == _lib.IMIN_ERANGE
    # world indices past 2^32, including a first index near 2^64 (the sum would wrap)
    for first, theta in (((1 << 32) - 5, 10), ((1 << 64) - 10, 100)):
        with pytest.raises(_lib.IminError) as e:
            _lib.imin_sample_reach_noalloc(rp.data_ptr(), rp.data_ptr(), rp.data_ptr(), 3, 0, [0],
                                           theta, first=first)
        assert e.value.code == _lib.IMIN_ERANGE


def test_noalloc_no_worlds_and_no_reach_buffer():
    torch, _lib = _setup()
    g, S, _ = synth.workload_er1k()
    dev = torch.device("cuda:0")
    d_rp = torch.from_numpy(g.row_ptr).to(dev)
    d_col = torch.from_numpy(g.col).to(dev)
    d_p = torch.from_numpy(g.prob).to(dev)
    d_reach = torch.full((g.n,), 5, dtype=torch.int64, device=dev)
    # theta = 0: nothing drawn, the reach buffer is cleared, the totals are zero
    tot = _lib.imin_sample_reach_noalloc(d_rp.data_ptr(), d_col.data_ptr(), d_p.data_ptr(), g.n,
                                         g.m, S, 0, d_reach=d_reach.data_ptr())
    assert tot == (0, 0) and int(d_reach.abs().sum()) == 0
    # no reach buffer: the totals alone, equal to imin_sample's
    tot = _lib.imin_sample_reach_noalloc(d_rp.data_ptr(), d_col.data_ptr(), d_p.data_ptr(), g.n,
                                         g.m, S, 500, key=3)
    with _lib.Context(0) as ctx:
        G = ctx.load_graph(g)
        want = G.sample(S, theta=500, key=3, mode=_lib.IMIN_REACH)
        G.free()
    assert tot == (want["total_spread"], want["edges_scanned"])


def test_noalloc_reports_invalid_device_arrays():
    """Out-of-range targets, a NaN probability and a row_ptr entry past m are caught by
    the kernel's own checks (the bad value is skipped, never used as an address) and
    reported as IMIN_EINVAL; a valid call afterwards gives the regular results."""
    torch, _lib = _setup()
    g, S, _ = synth.workload_er1k()
    dev = torch.device("cuda:0")
    s0 = int(S[0])
    e0 = int(g.row_ptr[s0])
    assert g.row_ptr[s0 + 1] - e0 >= 1
    cases = []
    col = g.col.copy(); prob = g.prob.copy()
    col[e0] = g.n + 7; prob[e0] = 1.0                  # target past n, always live
    cases.append((g.row_ptr, col, prob))
    col = g.col.copy(); prob = g.prob.copy()
    col[e0] = -3; prob[e0] = 1.0                       # negative target
    cases.append((g.row_ptr, col, prob))
    prob = g.prob.copy(); prob[e0] = np.float32("nan")
    cases.append((g.row_ptr, g.col, prob))
    rp = g.row_ptr.copy(); rp[s0 + 1] = g.m + 100      # row end past m
    cases.append((rp, g.col, g.prob))
    for rp_h, col_h, p_h in cases:
        d_rp = torch.from_numpy(np.ascontiguousarray(rp_h)).to(dev)
        d_col = torch.from_numpy(np.ascontiguousarray(col_h)).to(dev)
        d_p = torch.from_numpy(np.ascontiguousarray(p_h)).to(dev)
        with pytest.raises(_lib.IminError) as e:
            _lib.imin_sample_reach_noalloc(d_rp.data_ptr(), d_col.data_ptr(), d_p.data_ptr(),
                                           g.n, g.m, S, 200)
        assert e.value.code == _lib.IMIN_EINVAL
    d_rp = torch.from_numpy(g.row_ptr).to(dev)
    d_col = torch.from_numpy(g.col).to(dev)
    d_p = torch.from_numpy(g.prob).to(dev)
    tot = _lib.imin_sample_reach_noalloc(d_rp.data_ptr(), d_col.data_ptr(), d_p.data_ptr(), g.n,
                                         g.m, S, 200, key=1)
    with _lib.Context(0) as ctx:
        G = ctx.load_graph(g)
        want = G.sample(S, theta=200, key=1, mode=_lib.IMIN_REACH)
        G.free()
    assert tot == (want["total_spread"], want["edges_scanned"])
