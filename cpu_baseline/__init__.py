"""Multi-threaded CPU Algorithm 2 (the paper's own design, Sec. 4.1) as a timed
baseline beside the single-threaded oracle.

``dupin_cpu.c`` runs the batch peel on the host's cores with POSIX threads:
parallel select over the live list, a shared work queue over the removed
vertices' arcs with atomic int64 decrements, per-thread partial sums of f.
Exact integer arithmetic, so its rounds, trace and best prefix equal the
oracle's (checked in tests/test_cpu_baseline.py).  Not used by the GPU path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdupin_cpu.so")
SRC_PATH = os.path.join(_HERE, "dupin_cpu.c")
_lib = None
GPO, LPO = 1, 2


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC_PATH):
        subprocess.check_call(["gcc", "-O3", "-pthread", "-fPIC", "-shared", "-o", LIB_PATH, SRC_PATH])
    return LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB_PATH)
        P, i64, i32, u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
        L.cb_peel.restype = ctypes.c_int
        L.cb_peel.argtypes = [i64, P, P, P, P, i32, i64, i64, u32, i64, ctypes.c_int, P, P, P, P, P, i64, P]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


class Graph:
    """A symmetric CSR held in host memory (from a synth graph)."""

    def __init__(self, g, metric: str):
        self.n = g.n
        self.rp, self.col, w = g.symmetric_csr()
        self.cw = None if metric == "dg" else w
        self.a = None if metric == "dg" else g.a


def peel(G: Graph, k_mult: int = 1, eps=(1, 10), flags: int = 0, threads: int = 0, max_rounds: int = 0):
    """Returns (peel_round, n_rounds, best_round, best_size, best_f, trace_f, trace_size, trace_peeled, n_min_rule)."""
    threads = threads or os.cpu_count() or 1
    n = G.n
    pr = np.empty(max(n, 1), np.int32)
    cap = n + 2
    fh, fl = np.zeros(cap, np.int64), np.zeros(cap, np.uint64)
    sz, pe = np.zeros(cap, np.int64), np.zeros(cap, np.int64)
    out = np.zeros(8, np.int64)
    rc = lib().cb_peel(n, _p(G.rp), _p(G.col), _p(G.cw), _p(G.a), k_mult, eps[0], eps[1], flags, max_rounds, threads,
                       _p(pr), _p(fh), _p(fl), _p(sz), _p(pe), cap, _p(out))
    if rc != 0:
        raise RuntimeError(f"cb_peel failed: {rc}")
    R = int(out[0])
    tf = [(int(fh[i]) << 64) + int(fl[i]) for i in range(R + 1)]
    return (pr[:n], R, int(out[1]), int(out[2]), (int(out[3]) << 64) + int(np.uint64(out[4])), tf, sz[:R + 1],
            pe[:R + 1], int(out[5]))
