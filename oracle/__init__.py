"""CPU oracle for the SandIMIN hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it and
shares no code with it (see ``oracle.c``'s header for what it computes and which
passages of the paper each step follows).

The C source is compiled with gcc into ``oracle/_build/liboracle.so`` on first
use (or by ``build()``), and bound here with ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

VARIANT = {"sandimin": 0, "sandimin-": 1, "lsbm": 2, "gsbm": 3, "lhga": 4}
MODE_REACH, MODE_LOWER, MODE_UPPER = 1, 2, 4
TAG_SPREAD, TAG_C1, TAG_C2, TAG_L1, TAG_L2 = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no target-specific flags)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


class OResult(C.Structure):
    _fields_ = [
        ("n_blockers", C.c_int32), ("chosen", C.c_int32), ("iters_L", C.c_int32),
        ("iters_U", C.c_int32), ("nBL", C.c_int32), ("nBU", C.c_int32), ("nBR", C.c_int32),
        ("nVs", C.c_int32),
        ("I_hat", C.c_double), ("I_after", C.c_double * 3), ("sigmaL_L", C.c_double),
        ("sigmaU_L", C.c_double), ("sigmaL_U", C.c_double), ("sigmaU_U", C.c_double),
        ("DL_hat", C.c_double), ("DU_hat", C.c_double), ("ratio_lb", C.c_double),
        ("OPT_L", C.c_double), ("theta_max_L", C.c_double), ("theta_max_U", C.c_double),
        ("n_spread", C.c_uint64), ("theta_C1", C.c_uint64), ("theta_C2", C.c_uint64),
        ("theta_L1", C.c_uint64), ("theta_L2", C.c_uint64), ("n_final", C.c_uint64 * 3),
        ("covC2", C.c_uint64), ("covL2", C.c_uint64),
    ]

    def as_dict(self) -> dict:
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else v
        return d


def _P(t):
    return C.POINTER(t)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.oracle_philox4x32_10.argtypes = [_P(C.c_uint32), _P(C.c_uint32), _P(C.c_uint32)]
        L.oracle_coin_threshold.argtypes = [C.c_float]
        L.oracle_coin_threshold.restype = C.c_uint32
        L.oracle_graph_new.argtypes = [C.c_int32, C.c_int64, _P(C.c_int32), _P(C.c_int32),
                                       _P(C.c_float)]
        L.oracle_graph_new.restype = C.c_void_p
        L.oracle_graph_free.argtypes = [C.c_void_p]
        L.oracle_edge_live.argtypes = [C.c_void_p, C.c_int64, C.c_uint64, C.c_uint64, C.c_uint32,
                                       C.c_uint32]
        L.oracle_target_index.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32,
                                          C.c_uint64]
        L.oracle_target_index.restype = C.c_uint64
        L.oracle_world_explicit.argtypes = [C.c_void_p, _P(C.c_uint8), _P(C.c_int32), C.c_int32,
                                            _P(C.c_int32), C.c_int32, C.c_int32, _P(C.c_uint8),
                                            _P(C.c_int32), _P(C.c_uint64), _P(C.c_uint8)]
        L.oracle_world_explicit.restype = C.c_int32
        L.oracle_sample.argtypes = [C.c_void_p, _P(C.c_int32), C.c_int32, _P(C.c_int32),
                                    C.c_int32, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32,
                                    C.c_uint64, C.c_uint32, _P(C.c_uint64), _P(C.c_uint64),
                                    _P(C.c_uint64), _P(C.c_uint32), _P(C.c_uint64)]
        L.oracle_vs.argtypes = [C.c_void_p, _P(C.c_int32), C.c_int32, _P(C.c_int32), C.c_int32,
                                _P(C.c_int32)]
        L.oracle_vs.restype = C.c_int32
        L.oracle_max_coverage_sets.argtypes = [C.c_int64, _P(C.c_int64), _P(C.c_int32),
                                               C.c_int32, C.c_int32, _P(C.c_int32),
                                               _P(C.c_uint64), _P(C.c_uint64)]
        L.oracle_max_coverage_sets.restype = C.c_int32
        L.oracle_stop_rule.argtypes = [C.c_void_p, _P(C.c_int32), C.c_int32, _P(C.c_int32),
                                       C.c_int32, C.c_double, C.c_double, C.c_uint64, C.c_uint32,
                                       C.c_uint32, _P(C.c_double)]
        L.oracle_stop_rule.restype = C.c_uint64
        for f in ("oracle_sigma_low", "oracle_sigma_up"):
            getattr(L, f).argtypes = [C.c_double, C.c_double, C.c_double]
            getattr(L, f).restype = C.c_double
        L.oracle_lsbm_theta_max.argtypes = [C.c_double, C.c_int32, C.c_int32, C.c_int32,
                                            C.c_double, C.c_double, C.c_double, C.c_double]
        L.oracle_lsbm_theta_max.restype = C.c_double
        L.oracle_gsbm_theta_max.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_double,
                                            C.c_double, C.c_double]
        L.oracle_gsbm_theta_max.restype = C.c_double
        L.oracle_solve.argtypes = [C.c_void_p, _P(C.c_int32), C.c_int32, C.c_int32, C.c_double,
                                   C.c_double, C.c_double, C.c_double, C.c_uint64, C.c_uint32,
                                   C.c_int32, C.c_uint64, C.c_uint64, _P(C.c_int32), _P(C.c_int32),
                                   _P(C.c_int32), _P(C.c_int32), _P(OResult)]
        L.oracle_sample_useq.argtypes = [C.c_void_p, _P(C.c_int32), C.c_int32, _P(C.c_int32), C.c_int32,
                                         _P(C.c_int32), C.c_int32, C.c_uint64, C.c_uint64, C.c_uint32,
                                         C.c_uint32, C.c_uint64, _P(C.c_uint64), _P(C.c_uint64),
                                         _P(C.c_uint64)]
        L.oracle_useq_explicit.argtypes = [C.c_void_p, _P(C.c_uint8), _P(C.c_int32), C.c_int32,
                                           _P(C.c_int32), C.c_int32, _P(C.c_uint64), _P(C.c_uint64)]
        for f in ("oracle_advanced_greedy", "oracle_greedy_replace"):
            getattr(L, f).argtypes = [C.c_void_p, _P(C.c_int32), C.c_int32, C.c_int32, C.c_uint64,
                                      C.c_uint64, _P(C.c_int32), _P(C.c_int32)]
            getattr(L, f).restype = C.c_int32
        L.oracle_result_size.restype = C.c_int32
        assert L.oracle_result_size() == C.sizeof(OResult), "OResult layout mismatch"
        _lib = L
    return _lib


def _ptr(a, t):
    if a is None:
        return None
    return a.ctypes.data_as(_P(t))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def coin_threshold(p: float) -> int:
    return int(lib().oracle_coin_threshold(float(p)))


def target_index(key: int, j: int, tag: int, inst: int, count: int) -> int:
    return int(lib().oracle_target_index(key, j, tag, inst, count))


class OracleGraph:
    """The oracle's own copy of a CSR graph (it derives thresholds and in-edges itself)."""

    def __init__(self, n, row_ptr, col, prob):
        self.n = int(n)
        self.row_ptr = _i32(row_ptr)
        self.col = _i32(col)
        self.prob = np.ascontiguousarray(np.asarray(prob, dtype=np.float32))
        self.m = int(self.col.shape[0])
        self._h = lib().oracle_graph_new(self.n, self.m, _ptr(self.row_ptr, C.c_int32),
                                         _ptr(self.col, C.c_int32), _ptr(self.prob, C.c_float))
        if not self._h:
            raise MemoryError("oracle_graph_new failed")

    @classmethod
    def from_graph(cls, g):
        return cls(g.n, g.row_ptr, g.col, g.prob)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.oracle_graph_free(h)
            self._h = None

    # -- coins -----------------------------------------------------------
    def edge_live(self, e, key, j, tag, inst=0) -> bool:
        return bool(lib().oracle_edge_live(self._h, int(e), key, j, tag, inst))

    # -- one explicit world ------------------------------------------------
    def world_explicit(self, live_mask, S, blocked=(), target=-1):
        live_mask = np.ascontiguousarray(np.asarray(live_mask, dtype=np.uint8))
        assert live_mask.shape[0] == self.m
        S = _i32(S)
        B = _i32(blocked)
        reached = np.zeros(self.n, np.uint8)
        idom = np.zeros(self.n, np.int32)
        credit = np.zeros(self.n, np.uint64)
        lrr = np.zeros(self.n, np.uint8)
        R = lib().oracle_world_explicit(self._h, _ptr(live_mask, C.c_uint8), _ptr(S, C.c_int32),
                                        len(S), _ptr(B, C.c_int32), len(B), int(target),
                                        _ptr(reached, C.c_uint8), _ptr(idom, C.c_int32),
                                        _ptr(credit, C.c_uint64), _ptr(lrr, C.c_uint8))
        return dict(R=int(R), reached=reached, idom=idom, credit_lower=credit, lrr=lrr)

    # -- imin_sample counterpart -------------------------------------------
    def sample(self, S, blocked=(), theta=1, key=0, tag=0, inst=0, first=0,
               mode=MODE_REACH, per_world=False):
        S = _i32(S)
        B = _i32(blocked)
        reach = np.zeros(self.n, np.uint64)
        cl = np.zeros(self.n, np.uint64)
        cu = np.zeros(self.n, np.uint64)
        ws = np.zeros(max(int(theta), 1), np.uint32) if per_world else None
        scal = np.zeros(3, np.uint64)
        lib().oracle_sample(self._h, _ptr(S, C.c_int32), len(S), _ptr(B, C.c_int32), len(B),
                            int(theta), int(key), int(tag), int(inst), int(first), int(mode),
                            _ptr(reach, C.c_uint64), _ptr(cl, C.c_uint64), _ptr(cu, C.c_uint64),
                            _ptr(ws, C.c_uint32), _ptr(scal, C.c_uint64))
        out = dict(reach=reach, credit_lower=cl, credit_upper=cu, total_spread=int(scal[0]),
                   edges_scanned=int(scal[1]), nonempty_lrr=int(scal[2]))
        if per_world:
            out["world_spread"] = ws[: int(theta)]
        return out

    def vs(self, S, blocked=()):
        S = _i32(S)
        B = _i32(blocked)
        out = np.zeros(self.n + 1, np.int32)
        c = lib().oracle_vs(self._h, _ptr(S, C.c_int32), len(S), _ptr(B, C.c_int32), len(B),
                            _ptr(out, C.c_int32))
        return out[:c].copy()

    def stop_rule(self, S, blocked=(), beta=0.1, dprime=0.01, key=0, tag=0, inst=0):
        S = _i32(S)
        B = _i32(blocked)
        I = C.c_double(0)
        N = lib().oracle_stop_rule(self._h, _ptr(S, C.c_int32), len(S), _ptr(B, C.c_int32),
                                   len(B), beta, dprime, key, tag, inst, C.byref(I))
        return int(N), float(I.value)

    def lrr_sequences(self, S, blocked=(), query=(), theta=1, key=0, tag=0, inst=0, first=0):
        """LRR sequences of worlds [first, first + theta): per-node sequence credit
        (|M_phi({u})| summed over worlds), per-world |M_phi(query)|, and the totals
        (elements = sum of |L(v)|, cov = sum of the per-world values, nodes reached)."""
        S, B, Q = _i32(S), _i32(blocked), _i32(query)
        credit = np.zeros(self.n, np.uint64)
        cw = np.zeros(max(int(theta), 1), np.uint64)
        scal = np.zeros(3, np.uint64)
        lib().oracle_sample_useq(self._h, _ptr(S, C.c_int32), len(S), _ptr(B, C.c_int32), len(B),
                                 _ptr(Q, C.c_int32), len(Q), int(theta), int(key), int(tag), int(inst),
                                 int(first), _ptr(credit, C.c_uint64), _ptr(cw, C.c_uint64),
                                 _ptr(scal, C.c_uint64))
        return dict(credit_useq=credit, cov_world=cw[: int(theta)], elements=int(scal[0]), cov=int(scal[1]),
                    total_spread=int(scal[2]))

    def lrr_sequence_explicit(self, live_mask, S, query=()):
        live_mask = np.ascontiguousarray(np.asarray(live_mask, dtype=np.uint8))
        S, Q = _i32(S), _i32(query)
        credit = np.zeros(self.n, np.uint64)
        scal = np.zeros(3, np.uint64)
        lib().oracle_useq_explicit(self._h, _ptr(live_mask, C.c_uint8), _ptr(S, C.c_int32), len(S),
                                   _ptr(Q, C.c_int32), len(Q), _ptr(credit, C.c_uint64), _ptr(scal, C.c_uint64))
        return dict(credit_useq=credit, elements=int(scal[0]), cov=int(scal[1]), total_spread=int(scal[2]))

    def dt_baseline(self, which, S, k, theta, key=0):
        """AdvancedGreedy (``which='ag'``) or GreedyReplace (``'gr'``) of Xie et al. as
        the paper describes them: (blockers in order, number of estimates)."""
        S = _i32(S)
        B = np.zeros(max(int(k), 1), np.int32)
        calls = C.c_int32(0)
        f = lib().oracle_advanced_greedy if which == "ag" else lib().oracle_greedy_replace
        nb = f(self._h, _ptr(S, C.c_int32), len(S), int(k), int(theta), int(key), _ptr(B, C.c_int32),
               C.byref(calls))
        return [int(x) for x in B[:nb]], int(calls.value)

    def solve(self, S, k, eps, delta, beta=0.1, gamma=0.1, key=0, inst=0, variant="sandimin",
              fixed_theta=0, pr_worlds=0):
        """Algorithm 1; pr_worlds > 0 reads Pr[s -> v] (OPT^L, LHGA) as the reach
        frequency over that many worlds of stream tag 6.  Raises ValueError when that
        reading gives OPT^L = 0."""
        S = _i32(S)
        outs = [np.zeros(max(k, 1), np.int32) for _ in range(4)]
        r = OResult()
        rc = lib().oracle_solve(self._h, _ptr(S, C.c_int32), len(S), int(k), float(eps), float(delta),
                                float(beta), float(gamma), int(key), int(inst), VARIANT[variant],
                                int(fixed_theta), int(pr_worlds), *[_ptr(o, C.c_int32) for o in outs],
                                C.byref(r))
        if rc == 2:
            raise ValueError("OPT^L = 0: no top-k node of ON was reached in the pr_worlds worlds")
        d = r.as_dict()
        d["blockers"] = outs[0][: r.n_blockers].copy()
        d["B_L"] = outs[1][: r.nBL].copy()
        d["B_U"] = outs[2][: r.nBU].copy()
        d["B_R"] = outs[3][: r.nBR].copy()
        return d


def max_coverage_sets(sets, n, k):
    """Procedure Max-Coverage over explicit sets -> (B, cov[0..|B|], topk[0..|B|])."""
    off = np.zeros(len(sets) + 1, np.int64)
    for i, s in enumerate(sets):
        off[i + 1] = off[i] + len(s)
    elem = _i32(np.concatenate([np.asarray(s, np.int32) for s in sets]) if sets else [])
    if elem.size == 0:
        elem = np.zeros(1, np.int32)
    B = np.zeros(max(k, 1), np.int32)
    cov = np.zeros(k + 1, np.uint64)
    topk = np.zeros(k + 1, np.uint64)
    nb = lib().oracle_max_coverage_sets(len(sets), _ptr(off, C.c_int64), _ptr(elem, C.c_int32),
                                        n, k, _ptr(B, C.c_int32), _ptr(cov, C.c_uint64),
                                        _ptr(topk, C.c_uint64))
    return B[:nb].copy(), cov[: nb + 1].copy(), topk[: nb + 1].copy()


def sigma_low(x, a, theta):
    return float(lib().oracle_sigma_low(x, a, theta))


def sigma_up(y, a, theta):
    return float(lib().oracle_sigma_up(y, a, theta))


def lsbm_theta_max(I_hat, n, nS, k, eps, delta, beta, OPT):
    return float(lib().oracle_lsbm_theta_max(I_hat, n, nS, k, eps, delta, beta, OPT))


def gsbm_theta_max(nVs, nS, k, eps, delta, OPT):
    return float(lib().oracle_gsbm_theta_max(nVs, nS, k, eps, delta, OPT))
