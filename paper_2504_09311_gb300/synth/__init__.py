"""Seeded synthetic inputs for the peeling library.

Thin ctypes layer over ``synth.c``: every graph, weight array and layout is a
pure function of its parameters and seed, bit-identical on x86-64 and AArch64.
The module produces inputs only; it holds none of the peeling arithmetic and
is the single source of inputs for both the CUDA path and the CPU oracle.

Vertex numbering: a bipartite graph has users ``[0, n_left)`` and items
``[n_left, n_left + n_right)``; a general graph has ``n_left`` vertices and
``n_right == 0``.  Weights are Q32.32 int64 (value * 2**32).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lib = None

Q_ONE = 1 << 32


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so next to it (gcc, no libm routines)."""
    import subprocess

    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(src):
        subprocess.check_call(
            ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-pthread", "-o", LIB_PATH, src, "-lm"]
        )
    return LIB_PATH


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            build()
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        u64 = ctypes.c_uint64
        d = ctypes.c_double
        L.sg_bipartite_uniform.restype = P
        L.sg_bipartite_uniform.argtypes = [i64, i64, i64, i64, i64, d, u64]
        L.sg_bipartite_zipf.restype = P
        L.sg_bipartite_zipf.argtypes = [i64, i64, i64, d, i64, i64, i64, d, i64, u64]
        L.sg_rmat.restype = P
        L.sg_rmat.argtypes = [ctypes.c_int, i64, d, d, d, u64]
        L.sg_random_general.restype = P
        L.sg_random_general.argtypes = [i64, i64, u64]
        for nm in ("sg_n_left", "sg_n_right", "sg_m"):
            getattr(L, nm).restype = i64
            getattr(L, nm).argtypes = [P]
        for nm in ("sg_eu", "sg_ev"):
            getattr(L, nm).restype = P
            getattr(L, nm).argtypes = [P]
        L.sg_free.argtypes = [P]
        L.sg_fd_weights.argtypes = [P, P]
        L.sg_uniform_edge_weights.argtypes = [P, i64, i64, u64, P]
        L.sg_uniform_vertex_weights.argtypes = [i64, i64, i64, u64, P]
        L.sg_bipartite_csr.argtypes = [P] * 8
        L.sg_symmetric_csr.argtypes = [P] * 5
        L.sg_poisson_arrivals.argtypes = [i64, d, u64, P]
        L.sg_log_uniform.argtypes = [i64, d, d, i64, u64, P]
        L.sg_uniform_ints.argtypes = [i64, i64, u64, P]
        L.sg_ln.restype = d
        L.sg_ln.argtypes = [d]
        L.sg_exp.restype = d
        L.sg_exp.argtypes = [d]
        L.sg_set_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


@dataclass
class SynthGraph:
    """An undirected simple graph as a sorted edge list plus Q32.32 weights.

    ``eu``/``ev`` hold local ids: for a bipartite graph ``ev`` indexes items
    (global id ``n_left + ev``); for a general graph ``eu < ev``.
    ``c`` (per edge) and ``a`` (per vertex) may be None: then c_e = 1 and
    a_u = 0, the DG metric's weights.
    """

    n_left: int
    n_right: int
    eu: np.ndarray
    ev: np.ndarray
    c: Optional[np.ndarray] = None
    a: Optional[np.ndarray] = None
    name: str = ""
    _handle: Optional[int] = field(default=None, repr=False)

    @property
    def n(self) -> int:
        return self.n_left + self.n_right

    @property
    def m(self) -> int:
        return int(self.eu.shape[0])

    @property
    def bipartite(self) -> bool:
        return self.n_right > 0

    def global_edges(self):
        """(u, v) int32 arrays in global vertex ids."""
        if self.bipartite:
            return self.eu, (self.ev.astype(np.int64) + self.n_left).astype(np.int32)
        return self.eu, self.ev

    def _sorted(self) -> "SynthGraph":
        """This graph with its edge list in increasing (eu, ev) order (so every
        CSR row comes out strictly increasing, as the loader requires); self
        when it already is."""
        eu, ev = np.asarray(self.eu), np.asarray(self.ev)
        if eu.size < 2:
            return self
        key = (eu.astype(np.int64) << 32) | ev.astype(np.int64)
        if np.all(key[1:] > key[:-1]):
            return self
        order = np.argsort(key, kind="stable")
        return SynthGraph(self.n_left, self.n_right, eu[order].copy(), ev[order].copy(),
                          None if self.c is None else np.asarray(self.c)[order].copy(), self.a, self.name)

    def bipartite_csr(self):
        """(csr_ptr, csr_idx, csr_w, csc_ptr, csc_idx, csc_w); weights None when c is None."""
        assert self.bipartite
        if self._sorted() is not self:
            return self._sorted().bipartite_csr()
        L = lib()
        nU, nI, m = self.n_left, self.n_right, self.m
        csr_ptr = np.empty(nU + 1, np.int64)
        csr_idx = np.empty(m, np.int32)
        csc_ptr = np.empty(nI + 1, np.int64)
        csc_idx = np.empty(m, np.int32)
        csr_w = np.empty(m, np.int64) if self.c is not None else None
        csc_w = np.empty(m, np.int64) if self.c is not None else None
        h = self._edges_handle()
        L.sg_bipartite_csr(h, _ptr(self.c), _ptr(csr_ptr), _ptr(csr_idx), _ptr(csr_w), _ptr(csc_ptr),
                           _ptr(csc_idx), _ptr(csc_w))
        self._release(h)
        return csr_ptr, csr_idx, csr_w, csc_ptr, csc_idx, csc_w

    def symmetric_csr(self):
        """(row_ptr, col_idx, w) over global ids, each edge in both rows."""
        L = lib()
        if self.bipartite:
            u, v = self.global_edges()
            g = SynthGraph(self.n, 0, u, v, self.c, self.a)
            return g.symmetric_csr()
        if self._sorted() is not self:
            return self._sorted().symmetric_csr()
        ptr = np.empty(self.n + 1, np.int64)
        idx = np.empty(2 * self.m, np.int32)
        w = np.empty(2 * self.m, np.int64) if self.c is not None else None
        h = self._edges_handle()
        L.sg_symmetric_csr(h, _ptr(self.c), _ptr(ptr), _ptr(idx), _ptr(w))
        self._release(h)
        return ptr, idx, w

    # a transient C-side edge list view over our numpy arrays
    def _edges_handle(self):
        class _E(ctypes.Structure):
            _fields_ = [("n_left", ctypes.c_int64), ("n_right", ctypes.c_int64), ("m", ctypes.c_int64),
                        ("eu", ctypes.c_void_p), ("ev", ctypes.c_void_p)]

        self._eu_c = np.ascontiguousarray(self.eu, dtype=np.int32)
        self._ev_c = np.ascontiguousarray(self.ev, dtype=np.int32)
        e = _E(self.n_left, self.n_right, self.m, self._eu_c.ctypes.data, self._ev_c.ctypes.data)
        self._e_struct = e
        return ctypes.cast(ctypes.pointer(e), ctypes.c_void_p)

    def _release(self, h):
        self._e_struct = None


def _take(h) -> SynthGraph:
    L = lib()
    if not h:
        raise MemoryError("synth generator failed")
    nl, nr, m = L.sg_n_left(h), L.sg_n_right(h), L.sg_m(h)
    eu = np.ctypeslib.as_array(ctypes.cast(L.sg_eu(h), ctypes.POINTER(ctypes.c_int32)), shape=(m,)).copy() if m else np.zeros(0, np.int32)
    ev = np.ctypeslib.as_array(ctypes.cast(L.sg_ev(h), ctypes.POINTER(ctypes.c_int32)), shape=(m,)).copy() if m else np.zeros(0, np.int32)
    L.sg_free(h)
    return SynthGraph(int(nl), int(nr), eu, ev)


def fd_weights(g: SynthGraph) -> np.ndarray:
    """Q32.32 of 1/ln(x + 5), x = object-vertex degree (item, or larger endpoint)."""
    c = np.empty(g.m, np.int64)
    h = g._edges_handle()
    lib().sg_fd_weights(h, _ptr(c))
    g._release(h)
    return c


def uniform_edge_weights(g: SynthGraph, lo: int, hi: int, seed: int) -> np.ndarray:
    c = np.empty(g.m, np.int64)
    h = g._edges_handle()
    lib().sg_uniform_edge_weights(h, lo, hi, seed, _ptr(c))
    g._release(h)
    return c


def uniform_vertex_weights(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    a = np.empty(n, np.int64)
    lib().sg_uniform_vertex_weights(n, lo, hi, seed, _ptr(a))
    return a


def det_ln(x: float) -> float:
    return lib().sg_ln(x)


# ------------------------------------------------------------- workloads


def bipartite_uniform(nU, nI, draws, bU=0, bI=0, p=0.0, seed=1) -> SynthGraph:
    g = _take(lib().sg_bipartite_uniform(nU, nI, draws, bU, bI, p, seed))
    return g


def bipartite_zipf(nU, nI, m_bg, s=1.8, nblocks=0, bU=0, bI=0, p=0.0, camo=0, seed=1) -> SynthGraph:
    return _take(lib().sg_bipartite_zipf(nU, nI, m_bg, s, nblocks, bU, bI, p, camo, seed))


def rmat(scale, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=1) -> SynthGraph:
    return _take(lib().sg_rmat(scale, edge_factor, a, b, c, seed))


def random_general(n, draws, seed=1) -> SynthGraph:
    return _take(lib().sg_random_general(n, draws, seed))


def with_weights(g: SynthGraph, metric: str, seed: int = 1, a_range=None, c_range=(1, 100)) -> SynthGraph:
    """Attach the weights a metric uses: 'dg' none, 'dw' uniform ints, 'fd' Fraudar."""
    metric = metric.lower()
    if metric == "dg":
        g.c, g.a = None, None
    elif metric == "dw":
        g.c = uniform_edge_weights(g, c_range[0], c_range[1], seed)
        g.a = uniform_vertex_weights(g.n, a_range[0], a_range[1], seed) if a_range else None
    elif metric == "fd":
        g.c = fd_weights(g)
        g.a = uniform_vertex_weights(g.n, a_range[0], a_range[1], seed) if a_range else None
    else:
        raise ValueError(metric)
    return g


def dg_planted_block(seed: int = 1, nU=10_000, nI=5_000, draws=100_000, block=200, p=0.5) -> SynthGraph:
    """10k users x 5k items, 100k uniform pairs + a 200x200 block at p=0.5 (DG)."""
    g = bipartite_uniform(nU, nI, draws, block, block, p, seed)
    g.name = f"dg_block_{nU}x{nI}_{draws}_b{block}"
    return g


def fd_camouflage(seed: int = 1, nU=2_000_000, nI=1_000_000, m_bg=40_000_000, zipf_s=1.8, nblocks=5,
                  block=500, p=0.3, camo=150) -> SynthGraph:
    """Zipf(1.8) transaction graph with camouflaged blocks and Fraudar weights."""
    g = bipartite_zipf(nU, nI, m_bg, zipf_s, nblocks, block, block, p, camo, seed)
    g.c = fd_weights(g)
    g.name = f"fd_zipf_{nU}x{nI}_{m_bg}"
    return g


def rmat_weighted(scale=24, edge_factor=16, metric="dw", seed=1) -> SynthGraph:
    """R-MAT(0.57, 0.19, 0.19) with DW weights c in 1..100, a in 0..10 (or DG / FD)."""
    g = rmat(scale, edge_factor, 0.57, 0.19, 0.19, seed)
    if metric == "dw":
        with_weights(g, "dw", seed, a_range=(0, 10), c_range=(1, 100))
    elif metric == "fd":
        with_weights(g, "fd", seed)
    g.name = f"rmat{scale}_ef{edge_factor}_{metric}"
    return g


def window_sizes(count: int, lo: float = 1_000, hi: float = 500_000, seed: int = 1) -> np.ndarray:
    """Edge counts log-uniform in [lo, hi], multiples of 1000 (batched windows)."""
    out = np.empty(count, np.int64)
    lib().sg_log_uniform(count, lo, hi, 1000, seed, _ptr(out))
    return out


def transaction_window(m: int, seed: int) -> SynthGraph:
    """One window graph: m/10 users x m/20 items, Zipf(1.8) items, FD weights."""
    nU, nI = max(m // 10, 2), max(m // 20, 2)
    g = bipartite_zipf(nU, nI, m, 1.8, 0, 0, 0, 0.0, 0, seed)
    g.c = fd_weights(g)
    g.name = f"window_{m}"
    return g


def transaction_windows(count: int, seed: int = 1, lo: float = 1_000, hi: float = 500_000, workers: int = 0):
    """The batched workload: 'count' windows with log-uniform edge counts, built in parallel
    (the C generator releases the GIL; each window is single-threaded, so the output does not
    depend on the worker count)."""
    import concurrent.futures as cf

    sizes = window_sizes(count, lo, hi, seed=seed)
    workers = workers or (os.cpu_count() or 4)
    lib().sg_set_threads(1)
    try:
        with cf.ThreadPoolExecutor(max_workers=workers) as ex:
            return list(ex.map(lambda jm: transaction_window(int(jm[1]), seed=seed * 1_000_003 + jm[0]),
                               enumerate(sizes)))
    finally:
        lib().sg_set_threads(0)


def poisson_arrivals(k: int, rate: float, seed: int) -> np.ndarray:
    t = np.empty(k, np.float64)
    lib().sg_poisson_arrivals(k, rate, seed, _ptr(t))
    return t


def uniform_ints(count: int, k: int, seed: int) -> np.ndarray:
    out = np.empty(count, np.int64)
    lib().sg_uniform_ints(count, k, seed, _ptr(out))
    return out
