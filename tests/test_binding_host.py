"""Host-side marshalling of the batched binding (CPU, no library call).

peel_batch fills dupin_result[k] column by column through a numpy view of
the struct; the bytes must equal the ctypes structs built one by one, and
the outputs read back must equal the per-struct reader's.
"""
import ctypes

import numpy as np

from paper_2504_09311_gb300 import dupin


def _keep(seed):
    rng = np.random.default_rng(seed)
    keep = []
    for j in range(9):
        n = int(rng.integers(1, 50))
        pr = np.empty(n, np.int32) if j % 3 != 1 else None
        mk = np.empty(n, np.uint8) if j % 2 == 0 else None
        tr = None
        if j % 4 == 3:
            cap = n + 2
            tr = (np.zeros(cap, np.int64), np.zeros(cap, np.uint64), np.zeros(cap, np.int64), np.zeros(cap, np.int64))
        keep.append((pr, mk, tr))
    return keep


def test_result_dtype_matches_struct():
    assert dupin.RESULT_DTYPE.itemsize == ctypes.sizeof(dupin.Result)
    for name, _ in dupin.Result._fields_:
        assert dupin.RESULT_DTYPE.fields[name][1] == getattr(dupin.Result, name).offset


def test_result_array_equals_structs():
    for seed in range(3):
        keep = _keep(seed)
        RA = dupin._result_array(keep)
        R = (dupin.Result * len(keep))()
        for j, (pr, mk, tr) in enumerate(keep):
            R[j] = dupin._result_struct(pr, mk, tr, len(tr[0]) if tr is not None else 0)
        assert bytes(R) == RA.tobytes()
        bb = dupin.BatchBuffers(keep)
        assert bb.template.tobytes() == RA.tobytes()


def test_outputs_equal_struct_reader():
    keep = _keep(7)
    k = len(keep)
    rng = np.random.default_rng(3)
    RA = dupin._result_array(keep)
    RA["n_rounds"] = rng.integers(0, 40, k)
    RA["best_round"] = rng.integers(0, 40, k)
    RA["best_size"] = rng.integers(1, 1 << 40, k)
    RA["best_f_hi"] = rng.integers(-5, 1 << 30, k)
    RA["best_f_lo"] = rng.integers(0, 1 << 63, k, dtype=np.uint64) * 2 + 1
    RA["best_density"] = rng.random(k)
    RA["n_min_rule"] = rng.integers(0, 9, k)
    RA["n_bulk_rounds"] = rng.integers(0, 9, k)
    RA["tail_arcs"] = rng.integers(0, 1 << 30, k)
    RA["phase_ms"] = rng.random((k, 4)).astype(np.float32)
    for j, (pr, mk, tr) in enumerate(keep):
        if tr is not None:
            RA["n_rounds"][j] = min(int(RA["n_rounds"][j]), len(tr[0]) - 1)
    R = (dupin.Result * k).from_buffer_copy(RA.tobytes())
    new = dupin._outputs(RA, keep)
    for j in range(k):
        old = dupin._output(R[j], *keep[j])
        for f in ("n_rounds", "best_round", "best_size", "best_f", "best_density", "n_min_rule", "n_bulk_rounds",
                  "phase_ms", "tail_arcs"):
            assert getattr(new[j], f) == getattr(old, f), (j, f)
        assert new[j].peel_round is old.peel_round and new[j].best_mask is old.best_mask
        if keep[j][2] is not None:
            for f in ("trace_f_hi", "trace_f_lo", "trace_size", "trace_peeled"):
                assert np.array_equal(getattr(new[j], f), getattr(old, f))
