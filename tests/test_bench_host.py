"""Host logic of bench.py's batched leg with the library replaced by a fake (CPU).

The fake returns the same result for the batched and the one-launch-per-graph
calls, so the leg must report identical results, the autotuner's choice and
consistent timings; this guards the JSON keys the bench line carries without
a GPU.
"""
import os
import sys
import types

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


class _Out:
    def __init__(self, n):
        self.peel_round = np.arange(n, dtype=np.int32)
        self.best_round = 1
        self.best_f = 7


class _Graph:
    freed = 0

    def __init__(self, n):
        self.n = n

    @classmethod
    def from_synth(cls, g):
        return cls(g.n)

    def free(self):
        _Graph.freed += 1


def _fake_dupin():
    d = types.SimpleNamespace()
    d.Graph = _Graph
    d.BATCH_CTA_MAX_N = 131072
    d.calls = {"tune": 0, "batch": 0, "single": 0}
    d.make_params = lambda metric, k, eps, **kw: (metric, k, eps)

    def batch_tune(graphs, params, stream=None):
        d.calls["tune"] += 1
        return 128

    def peel_batch(graphs, params, want_rounds=True, stream=None, **kw):
        d.calls["batch"] += 1
        return [_Out(g.n) for g in graphs]

    def peel(g, metric, k, eps, **kw):
        d.calls["single"] += 1
        return _Out(g.n)

    d.batch_tune, d.peel_batch, d.peel = batch_tune, peel_batch, peel
    d.BatchBuffers = types.SimpleNamespace(for_graphs=lambda graphs, **kw: None)
    return d


def test_batched_leg_keys(monkeypatch):
    import torch

    import bench

    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    d = _fake_dupin()
    args = types.SimpleNamespace(windows=6)
    _Graph.freed = 0
    r = bench.bench_batched(d, None, args)
    assert r["identical_to_single"] is True
    assert r["cta_threads"] == 128 and r["one_cta_max_vertices"] == 131072
    assert r["calls"] == 3 and 0 < r["ms_best"] <= r["ms"]
    assert abs(r["graphs_per_s"] - 6 / (r["ms"] / 1e3)) < 1e-6 * r["graphs_per_s"]
    assert d.calls == {"tune": 1, "batch": 5, "single": 6}
    assert _Graph.freed == 6


def test_round_latency_reading():
    import bench

    r = bench.round_latency(6.8, 3208.0, 2070.0)
    assert r["us_per_round"] == round(6.8e3 / 3208, 3)
    assert r["floor_us"] == round((bench.L2_HIT_CYCLES + bench.SMEM_ATOMIC64_CYCLES) / 2070.0, 3)
    assert 0 < r["frac"] < 1
    assert bench.round_latency(0.0, 10, 2070.0) is None and bench.round_latency(1.0, 0, 2070.0) is None


def test_cluster_round_latency_reading():
    """The cluster tail's time per round against its floor: one L2 hit, one
    dependent shared atomic and the result exchange, in cycles at the SM clock."""
    import bench

    r = bench.cluster_round_latency(72.4, 16616.0, 2070.0)
    assert abs(r["us_per_round"] - 72.4e3 / 16616) < 1e-3
    floor = (bench.L2_HIT_CYCLES + bench.SMEM_ATOMIC64_CYCLES + bench.CLUSTER_EXCHANGE_CYCLES) / 2070.0
    assert abs(r["floor_us"] - floor) < 1e-3 and abs(r["frac"] - floor / r["us_per_round"]) < 2e-3
    assert bench.cluster_round_latency(0.0, 10, 2070.0) is None and bench.cluster_round_latency(1.0, 0, 2070.0) is None
