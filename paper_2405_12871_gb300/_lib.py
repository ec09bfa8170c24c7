"""Thin ctypes binding of the C ABI in ``include/imin.h``.

Argument marshalling only: every step of the sampling and the solve runs in
the CUDA library.  If the compiled library is missing this module raises; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

IMIN_OK, IMIN_EINVAL, IMIN_ERANGE, IMIN_ENOMEM, IMIN_EDEVICE, IMIN_ETIMEOUT, IMIN_EAGAIN = range(7)
IMIN_REACH, IMIN_CREDIT_LOWER, IMIN_CREDIT_UPPER, IMIN_OUT_DEVICE = 1, 2, 4, 0x100
VARIANTS = {"sandimin": 0, "sandimin-": 1, "lsbm": 2, "gsbm": 3, "lhga": 4}

# names the library must export (checked by the CPU tests against include/imin.h)
EXPORTS = ["imin_create", "imin_destroy", "imin_load_graph", "imin_free_graph", "imin_sample",
           "imin_solve", "imin_strerror", "imin_last_error", "imin_sample_reach_noalloc",
           "imin_sample_lrr_sequences", "imin_final_estimates", "imin_graph_autotune",
           "imin_solve_batch", "imin_server_start", "imin_server_submit", "imin_server_poll",
           "imin_server_stop", "imin_graph_tuning"]
NOALLOC_MAX_NODES = 2_000_000


class SampleOpts(C.Structure):
    _fields_ = [("key", C.c_uint64), ("tag", C.c_uint32), ("inst", C.c_uint32),
                ("first_sample", C.c_uint64), ("mode", C.c_uint32), ("reserved", C.c_uint32)]


class SampleOut(C.Structure):
    _fields_ = [("reach", C.c_void_p), ("credit_lower", C.c_void_p),
                ("credit_upper", C.c_void_p), ("world_spread", C.c_void_p),
                ("total_spread", C.c_uint64), ("edges_scanned", C.c_uint64),
                ("nonempty_lrr", C.c_uint64)]


class SolveOpts(C.Structure):
    _fields_ = [("beta", C.c_double), ("gamma", C.c_double), ("key", C.c_uint64),
                ("inst", C.c_uint32), ("variant", C.c_int32), ("fixed_theta", C.c_uint64),
                ("pr_worlds", C.c_uint64)]


class Result(C.Structure):
    _fields_ = [
        ("blockers", C.POINTER(C.c_int32)), ("B_L", C.POINTER(C.c_int32)),
        ("B_U", C.POINTER(C.c_int32)), ("B_R", C.POINTER(C.c_int32)),
        ("n_blockers", C.c_int32), ("nBL", C.c_int32), ("nBU", C.c_int32), ("nBR", C.c_int32),
        ("chosen", C.c_int32), ("iters_L", C.c_int32), ("iters_U", C.c_int32),
        ("nVs", C.c_int32),
        ("I_hat", C.c_double), ("I_after", C.c_double * 3), ("sigmaL_L", C.c_double),
        ("sigmaU_L", C.c_double), ("sigmaL_U", C.c_double), ("sigmaU_U", C.c_double),
        ("DL_hat", C.c_double), ("DU_hat", C.c_double), ("ratio_lb", C.c_double),
        ("OPT_L", C.c_double), ("theta_max_L", C.c_double), ("theta_max_U", C.c_double),
        ("n_spread", C.c_uint64), ("theta_C1", C.c_uint64), ("theta_C2", C.c_uint64),
        ("theta_L1", C.c_uint64), ("theta_L2", C.c_uint64), ("n_final", C.c_uint64 * 3),
        ("covC2", C.c_uint64), ("covL2", C.c_uint64), ("edges_scanned", C.c_uint64),
        ("worlds_sampled", C.c_uint64), ("ms_stage", C.c_double * 8),
        ("kernel_ms", C.c_double * 4), ("reach_nodes", C.c_uint64), ("reach_edges", C.c_uint64),
        ("reach_launches", C.c_uint64), ("kernel_launches", C.c_uint64),
        ("final_kernel_ms", C.c_double), ("final_entries", C.c_uint64), ("final_edges", C.c_uint64),
        ("final_launches", C.c_uint64),
    ]


class Query(C.Structure):
    _fields_ = [("g", C.c_void_p), ("S", C.POINTER(C.c_int32)), ("nS", C.c_int32),
                ("k", C.c_int32), ("eps", C.c_double), ("delta", C.c_double),
                ("opts", SolveOpts)]


class ServerOpts(C.Structure):
    _fields_ = [("max_active", C.c_int32), ("reserved", C.c_int32), ("mem_budget", C.c_uint64)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libimin.so (building it with nvcc first when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {path}")
        _build.build()
    L = C.CDLL(path)
    P = C.POINTER
    L.imin_create.argtypes = [P(C.c_void_p), C.c_int, C.c_size_t, C.c_void_p]
    L.imin_create.restype = C.c_int
    L.imin_destroy.argtypes = [C.c_void_p]
    L.imin_destroy.restype = None
    L.imin_load_graph.argtypes = [C.c_void_p, C.c_int32, C.c_int64, P(C.c_int32), P(C.c_int32),
                                  P(C.c_float), P(C.c_void_p)]
    L.imin_load_graph.restype = C.c_int
    L.imin_free_graph.argtypes = [C.c_void_p]
    L.imin_free_graph.restype = None
    L.imin_graph_autotune.argtypes = [C.c_void_p, P(C.c_int32), C.c_int32]
    L.imin_graph_autotune.restype = C.c_int
    L.imin_graph_tuning.argtypes = [C.c_void_p, C.POINTER(C.c_int32)]
    L.imin_graph_tuning.restype = C.c_int
    L.imin_sample.argtypes = [C.c_void_p, P(C.c_int32), C.c_int32, P(C.c_int32), C.c_int32,
                              C.c_uint64, P(SampleOpts), P(SampleOut)]
    L.imin_sample.restype = C.c_int
    L.imin_solve.argtypes = [C.c_void_p, P(C.c_int32), C.c_int32, C.c_int32, C.c_double,
                             C.c_double, P(SolveOpts), P(Result)]
    L.imin_solve.restype = C.c_int
    L.imin_strerror.argtypes = [C.c_int]
    L.imin_strerror.restype = C.c_char_p
    L.imin_last_error.argtypes = [C.c_void_p, C.c_char_p, C.c_size_t]
    L.imin_last_error.restype = None
    L.imin_sample_reach_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                            C.c_int64, P(C.c_int32), C.c_int32, C.c_uint64,
                                            C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64,
                                            C.c_void_p, C.c_void_p, P(C.c_uint64), C.c_void_p]
    L.imin_sample_reach_noalloc.restype = C.c_int
    L.imin_sample_lrr_sequences.argtypes = [C.c_void_p, P(C.c_int32), C.c_int32, P(C.c_int32), C.c_int32,
                                            P(C.c_int32), C.c_int32, C.c_uint64, P(SampleOpts),
                                            P(C.c_uint64), P(C.c_uint64), P(C.c_uint64)]
    L.imin_sample_lrr_sequences.restype = C.c_int
    L.imin_final_estimates.argtypes = [C.c_void_p, P(C.c_int32), C.c_int32, C.c_int32, P(P(C.c_int32)),
                                       P(C.c_int32), C.c_double, C.c_double, C.c_uint64, C.c_uint32,
                                       C.c_double, P(C.c_double), P(C.c_uint64)]
    L.imin_final_estimates.restype = C.c_int
    L.imin_solve_batch.argtypes = [C.c_void_p, C.c_int32, P(Query), P(Result)]
    L.imin_solve_batch.restype = C.c_int
    L.imin_server_start.argtypes = [C.c_void_p, P(ServerOpts), P(C.c_void_p)]
    L.imin_server_start.restype = C.c_int
    L.imin_server_submit.argtypes = [C.c_void_p, P(Query), P(C.c_uint64)]
    L.imin_server_submit.restype = C.c_int
    L.imin_server_poll.argtypes = [C.c_void_p, C.c_uint64, C.c_int32, P(Result), P(C.c_double)]
    L.imin_server_poll.restype = C.c_int
    L.imin_server_stop.argtypes = [C.c_void_p]
    L.imin_server_stop.restype = C.c_int
    _lib = L
    return L


class IminError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


def _i32p(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32)) if a is not None and a.size else None


def _as_i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


# --- the C ABI, one Python function per entry point ---------------------------------

def imin_create(device: int = 0, device_mem_budget: int = 0, stream: int = 0):
    L = load()
    h = C.c_void_p()
    rc = L.imin_create(C.byref(h), int(device), int(device_mem_budget), C.c_void_p(stream or None))
    if rc != IMIN_OK:
        raise IminError(rc, "imin_create: " + L.imin_strerror(rc).decode())
    return h


def imin_destroy(ctx):
    load().imin_destroy(ctx)


def imin_last_error(ctx) -> str:
    buf = C.create_string_buffer(1024)
    load().imin_last_error(ctx, buf, 1024)
    return buf.value.decode(errors="replace")


def _check(ctx, rc, what):
    if rc != IMIN_OK:
        raise IminError(rc, f"{what}: {load().imin_strerror(rc).decode()}: {imin_last_error(ctx)}")


def imin_load_graph(ctx, n, row_ptr, col, prob):
    L = load()
    row_ptr = _as_i32(row_ptr)
    col = _as_i32(col)
    prob = np.ascontiguousarray(np.asarray(prob, dtype=np.float32))
    g = C.c_void_p()
    rc = L.imin_load_graph(ctx, int(n), int(col.shape[0]), _i32p(row_ptr),
                           col.ctypes.data_as(C.POINTER(C.c_int32)),
                           prob.ctypes.data_as(C.POINTER(C.c_float)), C.byref(g))
    _check(ctx, rc, "imin_load_graph")
    return g


def imin_free_graph(g):
    load().imin_free_graph(g)


def imin_sample(ctx, g, n, S, blocked=(), theta=1, key=0, tag=0, inst=0, first=0,
                mode=IMIN_REACH, out=None, per_world=False):
    """Host outputs (numpy) unless ``out`` maps names to device pointers (then
    IMIN_OUT_DEVICE is set and the pointers are written in place)."""
    L = load()
    S = _as_i32(S)
    B = _as_i32(blocked)
    opts = SampleOpts(int(key), int(tag), int(inst), int(first), int(mode), 0)
    so = SampleOut()
    res = {}
    if out is None:
        for name, bit in (("reach", IMIN_REACH), ("credit_lower", IMIN_CREDIT_LOWER),
                          ("credit_upper", IMIN_CREDIT_UPPER)):
            if mode & bit:
                res[name] = np.zeros(n, np.uint64)
                setattr(so, name, res[name].ctypes.data)
        if per_world:
            res["world_spread"] = np.zeros(max(int(theta), 1), np.uint32)
            so.world_spread = res["world_spread"].ctypes.data
    else:
        opts.mode |= IMIN_OUT_DEVICE
        for name, ptr in out.items():
            setattr(so, name, int(ptr))
    rc = L.imin_sample(g, _i32p(S), len(S), _i32p(B), len(B), int(theta), C.byref(opts),
                       C.byref(so))
    _check(ctx, rc, "imin_sample")
    res.update(total_spread=int(so.total_spread), edges_scanned=int(so.edges_scanned),
               nonempty_lrr=int(so.nonempty_lrr))
    if "world_spread" in res:
        res["world_spread"] = res["world_spread"][: int(theta)]
    return res


def imin_solve(ctx, g, S, k, eps, delta, beta=0.1, gamma=0.1, key=0, inst=0,
               variant="sandimin", fixed_theta=0, pr_worlds=0):
    L = load()
    S = _as_i32(S)
    arrs = [np.zeros(max(int(k), 1), np.int32) for _ in range(4)]
    r = Result()
    r.blockers, r.B_L, r.B_U, r.B_R = [a.ctypes.data_as(C.POINTER(C.c_int32)) for a in arrs]
    opts = SolveOpts(float(beta), float(gamma), int(key), int(inst), VARIANTS[variant],
                     int(fixed_theta), int(pr_worlds))
    rc = L.imin_solve(g, _i32p(S), len(S), int(k), float(eps), float(delta), C.byref(opts),
                      C.byref(r))
    _check(ctx, rc, "imin_solve")
    d = {}
    for name, _ in Result._fields_:
        if name in ("blockers", "B_L", "B_U", "B_R"):
            continue
        v = getattr(r, name)
        d[name] = list(v) if hasattr(v, "__len__") else v
    d["blockers"] = arrs[0][: r.n_blockers].copy()
    d["B_L"] = arrs[1][: r.nBL].copy()
    d["B_U"] = arrs[2][: r.nBU].copy()
    d["B_R"] = arrs[3][: r.nBR].copy()
    return d


def _result_dict(r, arrs):
    d = {}
    for name, _ in Result._fields_:
        if name in ("blockers", "B_L", "B_U", "B_R"):
            continue
        v = getattr(r, name)
        d[name] = list(v) if hasattr(v, "__len__") else v
    d["blockers"] = arrs[0][: r.n_blockers].copy()
    d["B_L"] = arrs[1][: r.nBL].copy()
    d["B_U"] = arrs[2][: r.nBU].copy()
    d["B_R"] = arrs[3][: r.nBR].copy()
    return d


def imin_solve_batch(ctx, queries):
    """queries: list of dicts with keys g (graph handle), S, k, eps, delta and optional
    beta, gamma, key, inst, variant, fixed_theta, pr_worlds.  Returns one result dict per query."""
    L = load()
    n = len(queries)
    qs = (Query * max(n, 1))()
    rs = (Result * max(n, 1))()
    keep = []
    for i, q in enumerate(queries):
        S = _as_i32(q["S"])
        arrs = [np.zeros(max(int(q["k"]), 1), np.int32) for _ in range(4)]
        keep.append((S, arrs))
        qs[i].g = q["g"].value if isinstance(q["g"], C.c_void_p) else q["g"]
        qs[i].S = _i32p(S)
        qs[i].nS = len(S)
        qs[i].k = int(q["k"])
        qs[i].eps = float(q["eps"])
        qs[i].delta = float(q["delta"])
        qs[i].opts = SolveOpts(float(q.get("beta", 0.1)), float(q.get("gamma", 0.1)),
                               int(q.get("key", 0)), int(q.get("inst", 0)),
                               VARIANTS[q.get("variant", "sandimin")], int(q.get("fixed_theta", 0)),
                               int(q.get("pr_worlds", 0)))
        rs[i].blockers, rs[i].B_L, rs[i].B_U, rs[i].B_R = [
            a.ctypes.data_as(C.POINTER(C.c_int32)) for a in arrs]
    rc = L.imin_solve_batch(ctx, n, qs, rs)
    _check(ctx, rc, "imin_solve_batch")
    return [_result_dict(rs[i], keep[i][1]) for i in range(n)]


class Context:
    """Convenience owner of an imin_ctx (and the graphs loaded through it)."""

    def __init__(self, device=0, device_mem_budget=0, stream=0):
        self.h = imin_create(device, device_mem_budget, stream)

    def load_graph(self, g):
        return Graph(self, g)

    def solve_batch(self, queries):
        """queries: list of (Graph, S, k, eps, delta, kwargs)."""
        qs = []
        for G, S, k, eps, delta, kw in queries:
            d = dict(g=G.h, S=S, k=k, eps=eps, delta=delta)
            d.update(kw)
            qs.append(d)
        return imin_solve_batch(self.h, qs)

    def close(self):
        if self.h:
            imin_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Graph:
    def __init__(self, ctx: Context, g):
        self.ctx = ctx
        self.n = int(g.n)
        self.m = int(g.m)
        self.h = imin_load_graph(ctx.h, g.n, g.row_ptr, g.col, g.prob)

    def sample(self, S, blocked=(), theta=1, **kw):
        return imin_sample(self.ctx.h, self.h, self.n, S, blocked, theta, **kw)

    def solve(self, S, k, eps, delta, **kw):
        return imin_solve(self.ctx.h, self.h, S, k, eps, delta, **kw)

    def final_estimates(self, S, cands, gamma=0.1, delta=0.01, key=0, inst=0, spread_hint=0.0):
        """imin_final_estimates: (I_after, n_worlds) lists for 1..3 candidate blocker sets."""
        L = load()
        S = _as_i32(S)
        arrs = [_as_i32(b) for b in cands]
        ptrs = (C.POINTER(C.c_int32) * len(arrs))(*[a.ctypes.data_as(C.POINTER(C.c_int32)) for a in arrs])
        lens = (C.c_int32 * len(arrs))(*[len(a) for a in arrs])
        I = (C.c_double * len(arrs))()
        N = (C.c_uint64 * len(arrs))()
        rc = L.imin_final_estimates(self.h, _i32p(S), len(S), len(arrs), ptrs, lens, float(gamma), float(delta),
                                    int(key), int(inst), float(spread_hint), I, N)
        _check(self.ctx.h, rc, "imin_final_estimates")
        return list(I), [int(x) for x in N]

    def lrr_sequences(self, S, blocked=(), query=(), theta=1, key=0, tag=0, inst=0, first=0, credit=True,
                      per_world=True):
        """imin_sample_lrr_sequences: the LRR set of every reached node of every world."""
        L = load()
        S, B, Q = _as_i32(S), _as_i32(blocked), _as_i32(query)
        opts = SampleOpts(int(key), int(tag), int(inst), int(first), 0, 0)
        credit_a = np.zeros(self.n, np.uint64) if credit else None
        cw = np.zeros(max(int(theta), 1), np.uint64) if per_world else None
        tot = (C.c_uint64 * 5)()
        u64p = lambda a: a.ctypes.data_as(C.POINTER(C.c_uint64)) if a is not None else None
        rc = L.imin_sample_lrr_sequences(self.h, _i32p(S), len(S), _i32p(B), len(B), _i32p(Q), len(Q),
                                         int(theta), C.byref(opts), u64p(credit_a), u64p(cw), tot)
        _check(self.ctx.h, rc, "imin_sample_lrr_sequences")
        out = dict(elements=int(tot[0]), cov=int(tot[1]), total_spread=int(tot[2]), edges_scanned=int(tot[3]),
                   worlds=int(tot[4]))
        if credit:
            out["credit_useq"] = credit_a
        if per_world:
            out["cov_world"] = cw[: int(theta)]
        return out

    def autotune(self, S):
        """imin_graph_autotune: choose the reach-only launch shape now."""
        S = _as_i32(S)
        _check(self.ctx.h, load().imin_graph_autotune(self.h, _i32p(S), len(S)), "imin_graph_autotune")

    def tuning(self):
        """The autotuner's reach-only launch choice: dict(ctas, threads, minb, smem_bitmap)."""
        out = (C.c_int32 * 4)()
        rc = load().imin_graph_tuning(self.h, out)
        if rc != IMIN_OK:
            raise IminError(rc, "imin_graph_tuning: " + load().imin_strerror(rc).decode())
        return dict(ctas=out[0], threads=out[1], minb=out[2], smem_bitmap=bool(out[3]))

    def free(self):
        if self.h:
            imin_free_graph(self.h)
            self.h = None


def imin_sample_reach_noalloc(d_row_ptr, d_col, d_prob, n, m, S, theta, key=0, tag=0, inst=0,
                              first=0, d_reach=0, d_world_spread=0, stream=0):
    """Reach-only sampling into caller-owned device buffers, with no device allocation
    (pointers are integers, e.g. torch ``data_ptr()``).  Returns (total_spread, edges)."""
    L = load()
    S = _as_i32(S)
    tot = (C.c_uint64 * 2)()
    rc = L.imin_sample_reach_noalloc(C.c_void_p(d_row_ptr), C.c_void_p(d_col or None),
                                     C.c_void_p(d_prob or None), int(n), int(m), _i32p(S), len(S),
                                     int(theta), int(key), int(tag), int(inst), int(first),
                                     C.c_void_p(d_reach or None), C.c_void_p(d_world_spread or None),
                                     tot, C.c_void_p(stream or None))
    if rc != IMIN_OK:
        raise IminError(rc, "imin_sample_reach_noalloc: " + L.imin_strerror(rc).decode())
    return int(tot[0]), int(tot[1])


class Server:
    """Continuous-batching server over graphs of one Context (imin_server_*)."""

    def __init__(self, ctx: "Context", max_active: int = 64, mem_budget: int = 0):
        L = load()
        self.ctx = ctx
        self.h = C.c_void_p()
        o = ServerOpts(int(max_active), 0, int(mem_budget))
        rc = L.imin_server_start(ctx.h, C.byref(o), C.byref(self.h))
        _check(ctx.h, rc, "imin_server_start")
        self.k = {}

    def submit(self, G, S, k, eps, delta, **kw) -> int:
        L = load()
        S = _as_i32(S)
        q = Query()
        q.g = G.h.value if isinstance(G.h, C.c_void_p) else G.h
        q.S = _i32p(S)
        q.nS = len(S)
        q.k = int(k)
        q.eps = float(eps)
        q.delta = float(delta)
        q.opts = SolveOpts(float(kw.get("beta", 0.1)), float(kw.get("gamma", 0.1)),
                           int(kw.get("key", 0)), int(kw.get("inst", 0)),
                           VARIANTS[kw.get("variant", "sandimin")], int(kw.get("fixed_theta", 0)),
                           int(kw.get("pr_worlds", 0)))
        t = C.c_uint64()
        rc = L.imin_server_submit(self.h, C.byref(q), C.byref(t))
        _check(self.ctx.h, rc, "imin_server_submit")
        self.k[int(t.value)] = int(k)
        return int(t.value)

    def poll(self, ticket: int, wait_ms: int = -1):
        """Result dict (with 'latency_ms') when done, None while running."""
        L = load()
        k = self.k[ticket]
        arrs = [np.zeros(max(k, 1), np.int32) for _ in range(4)]
        r = Result()
        r.blockers, r.B_L, r.B_U, r.B_R = [a.ctypes.data_as(C.POINTER(C.c_int32)) for a in arrs]
        lat = C.c_double()
        rc = L.imin_server_poll(self.h, int(ticket), int(wait_ms), C.byref(r), C.byref(lat))
        if rc == IMIN_EAGAIN:
            return None
        del self.k[ticket]
        _check(self.ctx.h, rc, "imin_server_poll")
        d = _result_dict(r, arrs)
        d["latency_ms"] = float(lat.value)
        return d

    def stop(self):
        if self.h:
            load().imin_server_stop(self.h)
            self.h = None
