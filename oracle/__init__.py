"""CPU oracle for Dupin's batch peeling -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It wraps ``dupin_oracle.c`` (plain
single-threaded C, exact __int128 arithmetic) with ctypes and shares no code
with the CUDA library.  See ``dupin_oracle.c`` for what each routine follows
in the paper (Sec. 2 Eq. 1; Algorithms 1-4; Lemma 4.1/4.2; Thm 2.1/4.3; the
clique metrics TDS and kCLiDS of Sec. 2.1).

Pinning (tests/test_oracle.py): brute-force enumeration, exact max-flow DG,
closed forms (cliques, stars, complete bipartite graphs), hand-derived
worked examples under tests/golden/, the approximation bounds and the
per-round invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liboracle.so")
SRC_PATH = os.path.join(_HERE, "dupin_oracle.c")
_lib = None

METRICS = {"dg": 0, "dw": 1, "fd": 2}
FLAG_GPO, FLAG_LPO, FLAG_RECOMPUTE_F = 1, 2, 4
ERRORS = {0: "ok", -1: "invalid argument", -2: "weight overflow", -3: "out of memory",
          -4: "trace buffer too small", -5: "no progress / round cap"}


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC_PATH):
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-o", LIB_PATH, SRC_PATH])
    return LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB_PATH)
        P, i64, i32, u32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64
        L.og_build.restype = P
        L.og_build.argtypes = [i64, i64, P, P, P, P, ctypes.c_int, P]
        L.og_free.argtypes = [P]
        L.og_peel_batch.restype = ctypes.c_int
        L.og_peel_batch.argtypes = [P, i32, i64, i64, u32, i64, P, P, P, P, P, P, P, i64, P]
        L.og_peel_serial.restype = ctypes.c_int
        L.og_peel_serial.argtypes = [P, P, P]
        L.og_brute_force.restype = ctypes.c_int
        L.og_brute_force.argtypes = [P, P]
        L.og_exact_dg.restype = ctypes.c_int
        L.og_exact_dg.argtypes = [P, P, P]
        L.og_peel_clique.restype = ctypes.c_int
        L.og_peel_clique.argtypes = [P, i32, i32, i64, i64, u32, i64, P, P, P, P, P, P, P, i64, P]
        L.og_brute_force_clique.restype = ctypes.c_int
        L.og_brute_force_clique.argtypes = [P, i32, P]
        L.og_verify_clique.restype = ctypes.c_int
        L.og_verify_clique.argtypes = [P, i32, i32, i64, i64, P, i64, P, P, P, P, i64, i64, u64, P, i64]
        L.og_verify.restype = ctypes.c_int
        L.og_verify.argtypes = [P, i32, i64, i64, P, i64, P, P, P, P, i64, i64, u64, P, i64]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def i128(hi, lo) -> int:
    return (int(hi) << 64) + int(np.uint64(lo))


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle error {code}: {ERRORS.get(code, '?')}")
        self.code = code


class Graph:
    """The oracle's own adjacency, built from an undirected edge list."""

    def __init__(self, n: int, eu, ev, c=None, a=None, metric: str = "dw"):
        L = lib()
        self.n = int(n)
        self.metric = metric
        eu = np.ascontiguousarray(eu, dtype=np.int32)
        ev = np.ascontiguousarray(ev, dtype=np.int32)
        m = eu.shape[0]
        cc = np.ascontiguousarray(c, dtype=np.int64) if c is not None else np.full(m, 1 << 32, np.int64)
        aa = np.ascontiguousarray(a, dtype=np.int64) if a is not None else None
        err = ctypes.c_int(0)
        self._h = L.og_build(self.n, m, _p(eu), _p(ev), _p(cc), _p(aa), METRICS[metric], ctypes.byref(err))
        if not self._h:
            raise OracleError(err.value)
        self.m = m

    @classmethod
    def from_synth(cls, g, metric: str):
        u, v = g.global_edges()
        return cls(g.n, u, v, g.c, g.a, metric)

    def close(self):
        if getattr(self, "_h", None):
            lib().og_free(self._h)
            self._h = None

    def __del__(self):
        self.close()


@dataclass
class PeelResult:
    peel_round: np.ndarray
    n_rounds: int
    best_round: int
    best_size: int
    best_f: int
    trace_f: list
    trace_size: np.ndarray
    trace_peeled: np.ndarray
    trace_T: np.ndarray
    trace_kind: np.ndarray
    violations: int
    n_min_rule: int
    scan_volume: int
    clique: int = 0  # q for the clique metrics (f = clique count), 0: Q32.32 weights

    @property
    def best_mask(self) -> np.ndarray:
        return (self.peel_round > self.best_round).astype(np.uint8)

    @property
    def best_density(self) -> float:
        if not self.best_size:
            return 0.0
        return self.best_f / self.best_size / (1 if self.clique else 2**32)


def peel_batch(g: Graph, k_mult: int = 1, eps=(1, 10), flags: int = 0, max_rounds: int = 0,
               trace_cap: Optional[int] = None) -> PeelResult:
    """Algorithm 2 (with Algorithm 3 / 4 by flag); eps = (N, D) means N/D."""
    L = lib()
    n = g.n
    cap = trace_cap if trace_cap is not None else n + 2
    pr = np.zeros(n, np.int32)
    fh = np.zeros(cap, np.int64)
    fl = np.zeros(cap, np.uint64)
    sz = np.zeros(cap, np.int64)
    pe = np.zeros(cap, np.int64)
    tt = np.zeros(cap, np.int64)
    kd = np.zeros(cap, np.int32)
    out = np.zeros(8, np.int64)
    rc = L.og_peel_batch(g._h, k_mult, eps[0], eps[1], flags, max_rounds, _p(pr), _p(fh), _p(fl), _p(sz),
                         _p(pe), _p(tt), _p(kd), cap, _p(out))
    if rc != 0:
        raise OracleError(rc)
    R = int(out[0])
    return PeelResult(
        peel_round=pr, n_rounds=R, best_round=int(out[1]), best_size=int(out[2]),
        best_f=i128(out[3], np.uint64(out[4])),
        trace_f=[i128(fh[i], fl[i]) for i in range(R + 1)],
        trace_size=sz[: R + 1].copy(), trace_peeled=pe[: R + 1].copy(), trace_T=tt[: R + 1].copy(),
        trace_kind=kd[: R + 1].copy(), violations=int(out[5]), n_min_rule=int(out[6]), scan_volume=int(out[7]),
    )


def peel_clique(g: Graph, q: int = 3, k_mult: int = 3, eps=(1, 10), flags: int = 0, max_rounds: int = 0,
                trace_cap: Optional[int] = None) -> PeelResult:
    """Algorithm 2 (3 / 4 by flag) for the q-clique metrics: TDS (q = 3) and
    kCLiDS (Sec. 2.1); f and the weights are clique counts, recomputed from
    scratch each round.  The paper's multiplier for these metrics is q."""
    L = lib()
    n = g.n
    cap = trace_cap if trace_cap is not None else n + 2
    pr = np.zeros(n, np.int32)
    fh = np.zeros(cap, np.int64)
    fl = np.zeros(cap, np.uint64)
    sz = np.zeros(cap, np.int64)
    pe = np.zeros(cap, np.int64)
    tt = np.zeros(cap, np.int64)
    kd = np.zeros(cap, np.int32)
    out = np.zeros(8, np.int64)
    rc = L.og_peel_clique(g._h, q, k_mult, eps[0], eps[1], flags, max_rounds, _p(pr), _p(fh), _p(fl), _p(sz),
                          _p(pe), _p(tt), _p(kd), cap, _p(out))
    if rc != 0:
        raise OracleError(rc)
    R = int(out[0])
    return PeelResult(
        peel_round=pr, n_rounds=R, best_round=int(out[1]), best_size=int(out[2]),
        best_f=i128(out[3], np.uint64(out[4])),
        trace_f=[i128(fh[i], fl[i]) for i in range(R + 1)],
        trace_size=sz[: R + 1].copy(), trace_peeled=pe[: R + 1].copy(), trace_T=tt[: R + 1].copy(),
        trace_kind=kd[: R + 1].copy(), violations=int(out[5]), n_min_rule=int(out[6]), scan_volume=int(out[7]),
        clique=q,
    )


def brute_force_clique(g: Graph, q: int = 3):
    """(best_size, cliques in the best set, mask) over all non-empty subsets (n <= 20)."""
    out = np.zeros(3, np.int64)
    rc = lib().og_brute_force_clique(g._h, q, _p(out))
    if rc != 0:
        raise OracleError(rc)
    return int(out[0]), int(out[1]), int(out[2])


def peel_serial(g: Graph):
    """Algorithm 1: (order, best_step, best_size, best_f)."""
    L = lib()
    order = np.zeros(g.n, np.int32)
    out = np.zeros(4, np.int64)
    rc = L.og_peel_serial(g._h, _p(order), _p(out))
    if rc != 0:
        raise OracleError(rc)
    return order, int(out[0]), int(out[1]), i128(out[2], np.uint64(out[3]))


def brute_force(g: Graph):
    """(best_size, best_f, mask) over all non-empty subsets (n <= 24)."""
    out = np.zeros(4, np.int64)
    rc = lib().og_brute_force(g._h, _p(out))
    if rc != 0:
        raise OracleError(rc)
    return int(out[0]), i128(out[1], np.uint64(out[2])), int(out[3])


def exact_dg(g: Graph):
    """(|E[S*]|, |S*|, mask) of a DG densest subgraph by Goldberg max-flow."""
    out = np.zeros(2, np.int64)
    mask = np.zeros(g.n, np.uint8)
    rc = lib().og_exact_dg(g._h, _p(out), _p(mask))
    if rc != 0:
        raise OracleError(rc)
    return int(out[0]), int(out[1]), mask


def verify(g: Graph, k_mult, eps, peel_round, n_rounds, trace_f_hi, trace_f_lo, trace_size, trace_peeled,
           best_round, nsample=4, seed=1):
    """Check a plain Algorithm 2 result against the definitions; returns (code, message)."""
    msg = ctypes.create_string_buffer(512)
    pr = np.ascontiguousarray(peel_round, np.int32)
    fh = np.ascontiguousarray(trace_f_hi, np.int64)
    fl = np.ascontiguousarray(trace_f_lo, np.uint64)
    sz = np.ascontiguousarray(trace_size, np.int64)
    pe = np.ascontiguousarray(trace_peeled, np.int64)
    rc = lib().og_verify(g._h, k_mult, eps[0], eps[1], _p(pr), n_rounds, _p(fh), _p(fl), _p(sz), _p(pe),
                         best_round, nsample, seed, msg, 512)
    return rc, msg.value.decode()


def verify_clique(g: Graph, q, k_mult, eps, peel_round, n_rounds, trace_f_hi, trace_f_lo, trace_size,
                  trace_peeled, best_round, nsample=4, seed=1):
    """Check a plain clique-metric Algorithm 2 result against the definitions; returns (code, message)."""
    msg = ctypes.create_string_buffer(512)
    pr = np.ascontiguousarray(peel_round, np.int32)
    fh = np.ascontiguousarray(trace_f_hi, np.int64)
    fl = np.ascontiguousarray(trace_f_lo, np.uint64)
    sz = np.ascontiguousarray(trace_size, np.int64)
    pe = np.ascontiguousarray(trace_peeled, np.int64)
    rc = lib().og_verify_clique(g._h, q, k_mult, eps[0], eps[1], _p(pr), n_rounds, _p(fh), _p(fl), _p(sz), _p(pe),
                                best_round, nsample, seed, msg, 512)
    return rc, msg.value.decode()
