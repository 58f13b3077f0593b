"""Thin ctypes binding of libdupin.so (include/dupin.h): argument marshalling only.

Every step of the peel runs in the library's CUDA kernels; this module only
packs pointers and sizes.  Device buffers are torch tensors (torch is used for
device memory and streams), host buffers are numpy arrays.  There is no CPU
fallback: if the library is missing, importing ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdupin.so")

DG, DW, FD, TDS, KCLIDS = 0, 1, 2, 3, 4
METRICS = {"dg": DG, "dw": DW, "fd": FD, "tds": TDS, "kclids": KCLIDS}
CLIQUE_MAX_Q = 8  # kCLiDS clique sizes 3 .. CLIQUE_MAX_Q
DEVICE_PTRS = 1
GPO = 1
LPO = 2  # Algorithm 4 (implies GPO)
RESULT_DEVICE = 8
TIMING = 16
TAIL_ONE_CTA = 32  # every tail on one CTA
TAIL_CLUSTER = 64  # every tail on the thread-block cluster

OK = 0
ERR_INVALID_ARG, ERR_OVERFLOW, ERR_OOM, ERR_BUFFER_TOO_SMALL = -1, -2, -3, -4
ERR_NO_PROGRESS, ERR_CUDA, ERR_TIMEOUT, ERR_NOT_FOUND = -5, -6, -7, -8


class DupinError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"dupin error {code}: {msg}")
        self.code = code


class GraphDesc(ctypes.Structure):
    _fields_ = [("n_left", ctypes.c_int64), ("n_right", ctypes.c_int64),
                ("csr_ptr", ctypes.c_void_p), ("csr_idx", ctypes.c_void_p), ("csr_w", ctypes.c_void_p),
                ("csc_ptr", ctypes.c_void_p), ("csc_idx", ctypes.c_void_p), ("csc_w", ctypes.c_void_p),
                ("vertex_w", ctypes.c_void_p), ("flags", ctypes.c_uint32)]


class Params(ctypes.Structure):
    _fields_ = [("metric", ctypes.c_int32), ("k_mult", ctypes.c_int32), ("eps_num", ctypes.c_int64),
                ("eps_den", ctypes.c_int64), ("max_rounds", ctypes.c_int64), ("flags", ctypes.c_uint32),
                ("tail_cap", ctypes.c_int32), ("tail_arc_cap", ctypes.c_int64), ("clique_q", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("best_mask", ctypes.c_void_p), ("peel_round", ctypes.c_void_p),
                ("trace_f_hi", ctypes.c_void_p), ("trace_f_lo", ctypes.c_void_p), ("trace_size", ctypes.c_void_p),
                ("trace_peeled", ctypes.c_void_p), ("trace_cap", ctypes.c_int64), ("n_rounds", ctypes.c_int64),
                ("best_round", ctypes.c_int64), ("best_size", ctypes.c_int64), ("best_f_hi", ctypes.c_int64),
                ("best_f_lo", ctypes.c_uint64), ("best_density", ctypes.c_double), ("n_min_rule", ctypes.c_int64),
                ("n_bulk_rounds", ctypes.c_int64), ("tail_arcs", ctypes.c_int64), ("phase_ms", ctypes.c_float * 4),
                ("tail_ctas", ctypes.c_int64)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("memory_budget", ctypes.c_int64), ("max_slots", ctypes.c_int32), ("device", ctypes.c_int32)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("in_flight", ctypes.c_int64), ("queued", ctypes.c_int64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("graphs_per_s", ctypes.c_double)]


# every symbol include/dupin.h declares
EXPORTS = ["dupin_graph_load", "dupin_graph_free", "dupin_graph_info", "dupin_peel", "dupin_peel_batch",
           "dupin_serve_create", "dupin_serve_submit", "dupin_serve_poll", "dupin_serve_wait", "dupin_serve_stats",
           "dupin_serve_destroy", "dupin_last_error", "dupin_version", "dupin_peel_noalloc", "dupin_struct_size",
           "dupin_trim_cache", "dupin_batch_set_threads", "dupin_batch_get_threads", "dupin_batch_tune",
           "dupin_tune_handover"]

NOALLOC_MAX_N = 8192
BATCH_CTA_MAX_N = 131072

_lib = None


def lib():
    """Load libdupin.so (built by __graft_entry__.build()); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"libdupin.so not built: {LIB_PATH} (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        L.dupin_graph_load.argtypes = [ctypes.POINTER(GraphDesc), P, ctypes.POINTER(P)]
        L.dupin_graph_free.argtypes = [P]
        L.dupin_graph_info.argtypes = [P, P, P, P, P]
        L.dupin_peel.argtypes = [P, ctypes.POINTER(Params), ctypes.POINTER(Result), P]
        L.dupin_peel_batch.argtypes = [P, P, P, i64, P]
        L.dupin_serve_create.argtypes = [ctypes.POINTER(ServeConfig), ctypes.POINTER(P)]
        L.dupin_serve_submit.argtypes = [P, P, ctypes.POINTER(Params), ctypes.POINTER(Result),
                                         ctypes.POINTER(ctypes.c_uint64)]
        L.dupin_serve_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.dupin_serve_wait.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]
        L.dupin_serve_stats.argtypes = [P, ctypes.POINTER(ServeStats)]
        L.dupin_serve_destroy.argtypes = [P]
        L.dupin_last_error.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
        L.dupin_peel_noalloc.argtypes = [i64, P, P, P, P, ctypes.POINTER(Params), P, ctypes.POINTER(Result), P]
        L.dupin_version.restype = ctypes.c_char_p
        L.dupin_struct_size.argtypes = [ctypes.c_char_p]
        L.dupin_batch_set_threads.argtypes = [ctypes.c_int]
        L.dupin_batch_get_threads.argtypes = [P]
        L.dupin_batch_tune.argtypes = [P, P, i64, P, P]
        L.dupin_tune_handover.argtypes = [P, ctypes.POINTER(Params), P, P, P]
        for nm in EXPORTS:
            if nm not in ("dupin_version", "dupin_struct_size"):
                getattr(L, nm).restype = ctypes.c_int
        L.dupin_struct_size.restype = ctypes.c_int64
        for st, nm in ((GraphDesc, b"dupin_graph_desc"), (Params, b"dupin_params"), (Result, b"dupin_result"),
                       (ServeConfig, b"dupin_serve_config"), (ServeStats, b"dupin_serve_stats_t")):
            if L.dupin_struct_size(nm) != ctypes.sizeof(st):
                raise RuntimeError(f"libdupin.so was built with another layout of {nm.decode()}: rebuild it")
        _lib = L
    return _lib


def trim_cache() -> None:
    """Free the peeling workspaces kept from freed graphs."""
    check(lib().dupin_trim_cache())


def last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    lib().dupin_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def check(rc: int):
    if rc != OK:
        raise DupinError(rc, last_error())


def _addr(x) -> Optional[int]:
    """Address of a numpy array or torch tensor (None passes through)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    return x.data_ptr()  # torch tensor


def _stream(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Graph:
    """A graph resident in device memory (dupin_graph)."""

    def __init__(self, handle: int, n: int, m: int, n_left: int, n_right: int):
        self._h = ctypes.c_void_p(handle)
        self.n, self.m, self.n_left, self.n_right = n, m, n_left, n_right

    @property
    def handle(self):
        return self._h

    @classmethod
    def load_bipartite(cls, n_left, n_right, csr_ptr, csr_idx, csr_w, csc_ptr, csc_idx, csc_w, vertex_w=None,
                       device_ptrs=False, stream=None) -> "Graph":
        keep = [csr_ptr, csr_idx, csr_w, csc_ptr, csc_idx, csc_w, vertex_w]
        d = GraphDesc(n_left, n_right, _addr(csr_ptr), _addr(csr_idx), _addr(csr_w), _addr(csc_ptr),
                      _addr(csc_idx), _addr(csc_w), _addr(vertex_w), DEVICE_PTRS if device_ptrs else 0)
        h = ctypes.c_void_p()
        check(lib().dupin_graph_load(ctypes.byref(d), _stream(stream), ctypes.byref(h)))
        del keep
        m = int(csr_ptr[-1]) if not device_ptrs else int(csr_ptr[-1].item())
        return cls(h.value, n_left + n_right, m, n_left, n_right)

    @classmethod
    def load_symmetric(cls, n, row_ptr, col_idx, w=None, vertex_w=None, device_ptrs=False, stream=None) -> "Graph":
        keep = [row_ptr, col_idx, w, vertex_w]
        d = GraphDesc(n, 0, _addr(row_ptr), _addr(col_idx), _addr(w), None, None, None, _addr(vertex_w),
                      DEVICE_PTRS if device_ptrs else 0)
        h = ctypes.c_void_p()
        check(lib().dupin_graph_load(ctypes.byref(d), _stream(stream), ctypes.byref(h)))
        del keep
        arcs = int(row_ptr[-1]) if not device_ptrs else int(row_ptr[-1].item())
        return cls(h.value, n, arcs // 2, n, 0)

    @classmethod
    def from_synth(cls, g, stream=None) -> "Graph":
        """Load a synth.SynthGraph from host arrays (bipartite as CSR + CSC)."""
        if g.bipartite:
            csr_ptr, csr_idx, csr_w, csc_ptr, csc_idx, csc_w = g.bipartite_csr()
            return cls.load_bipartite(g.n_left, g.n_right, csr_ptr, csr_idx, csr_w, csc_ptr, csc_idx, csc_w, g.a,
                                      stream=stream)
        ptr, idx, w = g.symmetric_csr()
        return cls.load_symmetric(g.n, ptr, idx, w, g.a, stream=stream)

    def info(self):
        n, m, a, b = (ctypes.c_int64() for _ in range(4))
        check(lib().dupin_graph_info(self._h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(a), ctypes.byref(b)))
        return {"n": n.value, "m": m.value, "arcs": a.value, "device_bytes": b.value}

    def free(self):
        if self._h is not None and self._h.value:
            lib().dupin_graph_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def make_params(metric="dg", k_mult=1, eps=(1, 10), max_rounds=0, flags=0, tail_cap=0, tail_arc_cap=0,
                clique_q=0) -> Params:
    m = METRICS[metric] if isinstance(metric, str) else int(metric)
    return Params(m, k_mult, eps[0], eps[1], max_rounds, flags, tail_cap, tail_arc_cap, clique_q)


@dataclass
class PeelOutput:
    n_rounds: int
    best_round: int
    best_size: int
    best_f: int
    best_density: float
    n_min_rule: int
    peel_round: Optional[object] = None
    best_mask: Optional[object] = None
    trace_f_hi: Optional[object] = None  # f of every S_i as (hi, lo) words
    trace_f_lo: Optional[object] = None
    trace_size: Optional[object] = None
    trace_peeled: Optional[object] = None
    n_bulk_rounds: int = 0
    phase_ms: Optional[list] = None
    tail_arcs: int = 0
    tail_ctas: int = 0  # 1: the one-CTA tail ran, 8 or 16: the cluster tail, 0: none

    @property
    def trace_f(self) -> Optional[list]:
        """f(S_i) for i = 0 .. n_rounds as Python ints (Q32.32), built on first use."""
        if self.trace_f_hi is None:
            return None
        if not hasattr(self, "_trace_f"):
            self._trace_f = [(int(h) << 64) + int(lo) for h, lo in zip(self.trace_f_hi.tolist(),
                                                                       self.trace_f_lo.tolist())]
        return self._trace_f


def _result_dtype() -> np.dtype:
    """numpy view of dupin_result (same offsets and size as the ctypes Result)."""
    fmt = {ctypes.c_void_p: "<u8", ctypes.c_int64: "<i8", ctypes.c_uint64: "<u8", ctypes.c_double: "<f8"}
    names, formats, offsets = [], [], []
    for name, ct in Result._fields_:
        names.append(name)
        offsets.append(getattr(Result, name).offset)
        formats.append(fmt[ct] if ct in fmt else ("<f4", (ct._length_,)))
    return np.dtype({"names": names, "formats": formats, "offsets": offsets, "itemsize": ctypes.sizeof(Result)})


RESULT_DTYPE = _result_dtype()


def _data_addr(x) -> int:
    """Address of a numpy array or torch tensor, 0 for None."""
    if x is None:
        return 0
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.__array_interface__["data"][0]
    return x.data_ptr()


def _result_array(keep) -> np.ndarray:
    """dupin_result[k] for per-graph (peel_round, best_mask, trace) buffers, filled column by column."""
    RA = np.zeros(len(keep), RESULT_DTYPE)
    RA["peel_round"] = [_data_addr(b[0]) for b in keep]
    RA["best_mask"] = [_data_addr(b[1]) for b in keep]
    if any(b[2] is not None for b in keep):
        for name, q in (("trace_f_hi", 0), ("trace_f_lo", 1), ("trace_size", 2), ("trace_peeled", 3)):
            RA[name] = [_data_addr(b[2][q]) if b[2] is not None else 0 for b in keep]
        RA["trace_cap"] = [len(b[2][0]) if b[2] is not None else 0 for b in keep]
    return RA


def _outputs(RA: np.ndarray, keep) -> list:
    """PeelOutput per graph from a filled dupin_result[k]."""
    nr, br, bs = RA["n_rounds"].tolist(), RA["best_round"].tolist(), RA["best_size"].tolist()
    fh, fl, dens = RA["best_f_hi"].tolist(), RA["best_f_lo"].tolist(), RA["best_density"].tolist()
    nmr, nb, ta, ph = RA["n_min_rule"].tolist(), RA["n_bulk_rounds"].tolist(), RA["tail_arcs"].tolist(), \
        RA["phase_ms"].tolist()
    tc = RA["tail_ctas"].tolist()
    outs = []
    for j, (pr, mk, trace) in enumerate(keep):
        o = PeelOutput(nr[j], br[j], bs[j], (fh[j] << 64) + fl[j], dens[j], nmr[j], pr, mk, n_bulk_rounds=nb[j],
                       phase_ms=ph[j], tail_arcs=ta[j], tail_ctas=tc[j])
        if trace is not None and isinstance(trace[0], np.ndarray):
            R = nr[j] + 1
            o.trace_f_hi, o.trace_f_lo, o.trace_size, o.trace_peeled = (t[:R] for t in trace)
        outs.append(o)
    return outs


def _result_struct(peel_round=None, best_mask=None, trace=None, trace_cap=0) -> Result:
    r = Result()
    r.best_mask = _addr(best_mask)
    r.peel_round = _addr(peel_round)
    if trace is not None:
        r.trace_f_hi, r.trace_f_lo, r.trace_size, r.trace_peeled = (_addr(t) for t in trace)
    r.trace_cap = trace_cap
    return r


def _output(r: Result, peel_round, best_mask, trace) -> PeelOutput:
    out = PeelOutput(r.n_rounds, r.best_round, r.best_size, (int(r.best_f_hi) << 64) + int(r.best_f_lo),
                     r.best_density, r.n_min_rule, peel_round, best_mask, n_bulk_rounds=int(r.n_bulk_rounds),
                     phase_ms=[float(x) for x in r.phase_ms], tail_arcs=int(r.tail_arcs),
                     tail_ctas=int(r.tail_ctas))
    if trace is not None:
        R = r.n_rounds + 1
        fh, fl, sz, pe = trace
        if isinstance(fh, np.ndarray):
            out.trace_f_hi, out.trace_f_lo = fh[:R], fl[:R]
            out.trace_size, out.trace_peeled = sz[:R], pe[:R]
    return out


def peel(g: Graph, metric="dg", k_mult=1, eps=(1, 10), flags=0, max_rounds=0, tail_cap=0, want_rounds=True,
         want_mask=True, want_trace=True, stream=None, tail_arc_cap=0, clique_q=0) -> PeelOutput:
    """dupin_peel with host result buffers (numpy); clique_q is kCLiDS's clique size."""
    p = make_params(metric, k_mult, eps, max_rounds, flags, tail_cap, tail_arc_cap, clique_q)
    pr = np.empty(g.n, np.int32) if want_rounds else None
    mk = np.empty(g.n, np.uint8) if want_mask else None
    trace = None
    cap = 0
    if want_trace:
        cap = g.n + 2
        trace = (np.zeros(cap, np.int64), np.zeros(cap, np.uint64), np.zeros(cap, np.int64), np.zeros(cap, np.int64))
    r = _result_struct(pr, mk, trace, cap)
    check(lib().dupin_peel(g.handle, ctypes.byref(p), ctypes.byref(r), _stream(stream)))
    return _output(r, pr, mk, trace)


def peel_device(g: Graph, params: Params, peel_round=None, best_mask=None, stream=None) -> Result:
    """dupin_peel writing peel_round / best_mask into device tensors (DUPIN_RESULT_DEVICE)."""
    p = Params.from_buffer_copy(params)
    p.flags |= RESULT_DEVICE
    r = _result_struct(peel_round, best_mask, None, 0)
    check(lib().dupin_peel(g.handle, ctypes.byref(p), ctypes.byref(r), _stream(stream)))
    return r


def peel_batch_device(graphs: Sequence[Graph], params: Sequence[Params], peel_rounds, best_masks, stream=None):
    """dupin_peel_batch writing each peel_round / best_mask into its own device tensor
    (DUPIN_RESULT_DEVICE); returns the Result array (host scalars)."""
    k = len(graphs)
    G = (ctypes.c_void_p * k)(*[g.handle.value for g in graphs])
    P = (Params * k)(*params)
    R = (Result * k)()
    for j in range(k):
        P[j].flags |= RESULT_DEVICE
        R[j] = _result_struct(peel_rounds[j], best_masks[j], None, 0)
    check(lib().dupin_peel_batch(ctypes.cast(G, ctypes.c_void_p), ctypes.cast(P, ctypes.c_void_p),
                                 ctypes.cast(R, ctypes.c_void_p), k, _stream(stream)))
    return R


def result_buffers(n: int, want_rounds=True, want_mask=False, want_trace=False, pinned=False):
    """Host result buffers (peel_round, best_mask, trace) for a graph of n vertices;
    pinned=True places them in page-locked memory (through torch), so the result
    copies run at full link speed."""
    def arr(count, dtype):
        if not pinned:
            return np.empty(count, dtype)
        import torch

        tt = {np.dtype(np.int32): torch.int32, np.dtype(np.uint8): torch.uint8, np.dtype(np.int64): torch.int64,
              np.dtype(np.uint64): torch.int64}[np.dtype(dtype)]
        return torch.empty(count, dtype=tt, pin_memory=True).numpy().view(dtype)

    pr = arr(n, np.int32) if want_rounds else None
    mk = arr(n, np.uint8) if want_mask else None
    trace = None
    if want_trace:
        cap = n + 2
        trace = (arr(cap, np.int64), arr(cap, np.uint64), arr(cap, np.int64), arr(cap, np.int64))
    return pr, mk, trace


class BatchBuffers:
    """Host result buffers for a batch, reusable across peel_batch calls: the
    per-graph (peel_round, best_mask, trace) buffers and the result array with
    their addresses filled in once."""

    def __init__(self, keep):
        self.keep = list(keep)
        self.template = _result_array(self.keep)

    @classmethod
    def for_graphs(cls, graphs, want_rounds=True, want_mask=False, want_trace=False, pinned=False):
        if not pinned or want_mask or want_trace:
            return cls([result_buffers(g.n, want_rounds, want_mask, want_trace, pinned) for g in graphs])
        # peel rounds only: one page-locked block sliced per graph
        import torch

        total = sum(g.n for g in graphs)
        block = torch.empty(max(total, 1), dtype=torch.int32, pin_memory=True).numpy()
        keep, at = [], 0
        for g in graphs:
            keep.append((block[at:at + g.n] if want_rounds else None, None, None))
            at += g.n
        bb = cls(keep)
        bb._block = block  # keeps the page-locked memory alive
        return bb


def peel_batch(graphs: Sequence[Graph], params: Sequence[Params], want_rounds=True, want_trace=False, stream=None,
               want_mask=False, buffers=None):
    """dupin_peel_batch with host result buffers; returns a list of PeelOutput.
    buffers: optional per-graph (peel_round, best_mask, trace) from result_buffers(),
    or a BatchBuffers (reusable: addresses computed once)."""
    k = len(graphs)
    G = np.fromiter((g.handle.value for g in graphs), dtype=np.uint64, count=k)
    P = (Params * k)(*params)
    if isinstance(buffers, BatchBuffers):
        keep, RA = buffers.keep, buffers.template.copy()
    else:
        keep = list(buffers) if buffers is not None else \
            [result_buffers(g.n, want_rounds, want_mask, want_trace) for g in graphs]
        RA = _result_array(keep)
    check(lib().dupin_peel_batch(G.ctypes.data, ctypes.cast(P, ctypes.c_void_p), RA.ctypes.data, k,
                                 _stream(stream)))
    return _outputs(RA, keep)


def batch_threads(threads=None) -> int:
    """Get (or, with threads = 128 / 256 / 0 for the default, set) the current
    device's launch shape of the one-CTA-per-graph batched kernel."""
    if threads is not None:
        check(lib().dupin_batch_set_threads(int(threads)))
    t = ctypes.c_int()
    check(lib().dupin_batch_get_threads(ctypes.byref(t)))
    return t.value


def batch_tune(graphs: Sequence[Graph], params: Sequence[Params], stream=None) -> int:
    """dupin_batch_tune: time each launch shape on this batch, keep the faster
    for the current device; returns its threads per CTA."""
    k = len(graphs)
    G = (ctypes.c_void_p * k)(*[g.handle.value for g in graphs])
    P = (Params * k)(*params)
    t = ctypes.c_int()
    check(lib().dupin_batch_tune(ctypes.cast(G, ctypes.c_void_p), ctypes.cast(P, ctypes.c_void_p), k,
                                 _stream(stream), ctypes.byref(t)))
    return t.value


TUNE_HANDOVER_N = 6


def tune_handover(g: Graph, metric="dg", k_mult=1, eps=(1, 10), flags=0, stream=None):
    """dupin_tune_handover: time the peel under each hand-over candidate;
    returns (the fastest tail_arc_cap, {candidate: best ms})."""
    p = make_params(metric, k_mult, eps, flags=flags)
    best = ctypes.c_int64()
    times = (ctypes.c_float * TUNE_HANDOVER_N)()
    check(lib().dupin_tune_handover(g.handle, ctypes.byref(p), _stream(stream), ctypes.byref(best), times))
    return best.value, {1 << (16 + 2 * i): float(times[i]) for i in range(TUNE_HANDOVER_N)}


def peel_noalloc(n, row_ptr, col_idx, arc_w, vertex_w, params: Params, peel_round, best_mask=None, trace=None,
                 stream=None) -> Result:
    """dupin_peel_noalloc: graph (symmetric CSR), peel_round, best_mask and trace are device tensors."""
    r = _result_struct(None, best_mask, trace, 0 if trace is None else int(trace[0].shape[0]))
    check(lib().dupin_peel_noalloc(n, _addr(row_ptr), _addr(col_idx), _addr(arc_w), _addr(vertex_w),
                                   ctypes.byref(params), _addr(peel_round), ctypes.byref(r), _stream(stream)))
    return r


class Server:
    """dupin_serve_*: continuous batching of peel requests over resident graphs."""

    def __init__(self, memory_budget: int, max_slots: int = 64, device: int = 0):
        cfg = ServeConfig(memory_budget, max_slots, device)
        h = ctypes.c_void_p()
        check(lib().dupin_serve_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._pending = {}

    def submit(self, g: Graph, params: Params, want_rounds=True, want_trace=False) -> int:
        pr = np.empty(g.n, np.int32) if want_rounds else None
        trace = None
        cap = 0
        if want_trace:
            cap = g.n + 2
            trace = (np.zeros(cap, np.int64), np.zeros(cap, np.uint64), np.zeros(cap, np.int64),
                     np.zeros(cap, np.int64))
        r = _result_struct(pr, None, trace, cap)
        p = Params.from_buffer_copy(params)
        t = ctypes.c_uint64()
        check(lib().dupin_serve_submit(self._h, g.handle, ctypes.byref(p), ctypes.byref(r), ctypes.byref(t)))
        self._pending[t.value] = (r, p, pr, trace)
        return t.value

    def poll(self, ticket: int):
        done, st = ctypes.c_int(), ctypes.c_int()
        check(lib().dupin_serve_poll(self._h, ticket, ctypes.byref(done), ctypes.byref(st)))
        return bool(done.value), st.value

    def wait(self, ticket: int) -> PeelOutput:
        st = ctypes.c_int()
        check(lib().dupin_serve_wait(self._h, ticket, ctypes.byref(st)))
        r, p, pr, trace = self._pending.pop(ticket)
        if st.value != OK:
            raise DupinError(st.value, f"request {ticket} failed")
        return _output(r, pr, None, trace)

    def stats(self) -> dict:
        s = ServeStats()
        check(lib().dupin_serve_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in ServeStats._fields_}

    def close(self):
        if self._h is not None and self._h.value:
            check(lib().dupin_serve_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
