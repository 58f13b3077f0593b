"""The cluster tail (a thread-block cluster of 8 or 16 CTAs holding the live
sub-graph's vertex state in distributed shared memory) against the CPU oracle,
element by element, through the C ABI.

DUPIN_TAIL_CLUSTER forces every tail onto the cluster and DUPIN_TAIL_ONE_CTA
onto one CTA; tail_cap moves the hand-over from the grid-wide rounds.  Cases
cover graphs with fewer vertices than the cluster has CTAs, rounds whose
frontier in one CTA exceeds the expand window (512 entries), hubs, every
metric, k = 1 (minimum rule) and k = 2, Algorithms 3 and 4, and the hand-written
worked examples.
"""
import glob
import json
import os

import numpy as np
import pytest

import oracle
from paper_2504_09311_gb300 import synth

pytestmark = pytest.mark.gpu

Q = 1 << 32
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def dupin():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2504_09311_gb300 import dupin as d

    d.lib()
    return d


def assert_same(out, ref, ctx=""):
    assert out.n_rounds == ref.n_rounds, ctx
    assert np.array_equal(out.peel_round, ref.peel_round), ctx
    assert out.trace_f == ref.trace_f, ctx
    assert np.array_equal(np.asarray(out.trace_size), ref.trace_size), ctx
    assert np.array_equal(np.asarray(out.trace_peeled), ref.trace_peeled), ctx
    assert (out.best_round, out.best_size, out.best_f) == (ref.best_round, ref.best_size, ref.best_f), ctx
    assert out.n_min_rule == ref.n_min_rule, ctx
    assert np.array_equal(out.best_mask, ref.best_mask), ctx


def run_both(dupin, g, metric, k, eps, flags=0, tail_cap=0, tail_arc_cap=0):
    og = oracle.Graph.from_synth(g, metric)
    dg = dupin.Graph.from_synth(g)
    ref = oracle.peel_batch(og, k, eps, flags=flags & (oracle.FLAG_GPO | oracle.FLAG_LPO))
    out = dupin.peel(dg, metric, k, eps, flags=flags, tail_cap=tail_cap, tail_arc_cap=tail_arc_cap)
    dg.free()
    og.close()
    return out, ref


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "peel_*.json"))), ids=os.path.basename)
def test_golden_examples_cluster(dupin, path):
    G = json.load(open(path))
    eu = np.array([e[0] for e in G["edges"]], np.int32)
    ev = np.array([e[1] for e in G["edges"]], np.int32)
    g = synth.SynthGraph(G["n"], 0, eu, ev, np.array([e[2] * Q for e in G["edges"]], np.int64),
                         np.array([x * Q for x in G["a"]], np.int64))
    dg = dupin.Graph.from_synth(g)
    for case in G["cases"]:
        flags = {"": 0, "gpo": dupin.GPO, "lpo": dupin.LPO}[case.get("flags", "")] | dupin.TAIL_CLUSTER
        out = dupin.peel(dg, G["metric"], case["k"], tuple(case["eps"]), flags=flags)
        assert out.tail_ctas in (8, 16)
        assert list(out.peel_round) == case["peel_round"]
        assert out.trace_f == [x * Q for x in case["trace_f"]]
        assert list(out.trace_size) == case["trace_size"]
        assert list(out.trace_peeled) == case["trace_peeled"]
        assert (out.best_round, out.best_size, out.best_f) == (case["best_round"], case["best_size"], case["best_f"] * Q)
        assert out.n_min_rule == case["n_min_rule"]
    dg.free()


@pytest.mark.parametrize("metric", ["dg", "dw", "fd"])
@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("tail_cap", [0, 300])
def test_random_general_cluster(dupin, metric, k, tail_cap):
    for seed in range(2):
        g = synth.random_general(2000 + 37 * seed, 12000, seed=seed + 1)
        synth.with_weights(g, metric, seed=seed, a_range=(0, 7) if metric != "dg" else None)
        for eps in ((1, 10), (0, 1)):
            out, ref = run_both(dupin, g, metric, k, eps, flags=dupin.TAIL_CLUSTER, tail_cap=tail_cap)
            assert_same(out, ref, (metric, k, tail_cap, seed, eps))
            assert out.tail_ctas in (8, 16) or out.n_bulk_rounds == out.n_rounds


@pytest.mark.parametrize("flags", ["gpo", "lpo"])
@pytest.mark.parametrize("tail_cap", [0, 500])
def test_gpo_lpo_cluster(dupin, flags, tail_cap):
    fd = synth.bipartite_zipf(3000, 1500, 20000, 1.6, 1, 30, 30, 0.5, 12, seed=4)
    fd.c = synth.fd_weights(fd)
    cases = [(synth.rmat_weighted(13, 16, "dw", seed=3), "dw"), (fd, "fd"),
             (synth.dg_planted_block(seed=2, nU=3000, nI=1500, draws=20000, block=60, p=0.5), "dg")]
    f = dupin.GPO if flags == "gpo" else dupin.LPO
    for g, metric in cases:
        for k in (1, 2):
            for eps in ((0, 1), (1, 10)):
                out, ref = run_both(dupin, g, metric, k, eps, flags=f | dupin.TAIL_CLUSTER, tail_cap=tail_cap)
                assert_same(out, ref, (metric, k, eps, tail_cap, flags))


def test_tiny_graphs_fewer_vertices_than_ctas(dupin):
    """n < CTAs per cluster: some CTAs own no vertex; edgeless, single edge, a triangle, a star."""
    cases = [
        synth.SynthGraph(1, 0, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64), None),
        synth.SynthGraph(2, 0, np.array([0], np.int32), np.array([1], np.int32), np.array([5 * Q], np.int64), None),
        synth.SynthGraph(3, 0, np.array([0, 0, 1], np.int32), np.array([1, 2, 2], np.int32),
                         np.array([1 * Q, 2 * Q, 3 * Q], np.int64), np.array([0, Q, 2 * Q], np.int64)),
        synth.SynthGraph(7, 0, np.zeros(6, np.int32), np.arange(1, 7, dtype=np.int32), np.full(6, Q, np.int64), None),
        synth.SynthGraph(20, 0, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64),
                         synth.uniform_vertex_weights(20, 0, 9, 2)),
    ]
    for g in cases:
        for k in (1, 2):
            for flags in (0, 2):
                f = (dupin.LPO if flags else 0) | dupin.TAIL_CLUSTER
                out, ref = run_both(dupin, g, "dw", k, (1, 10), flags=f)
                assert_same(out, ref, (g.n, k, flags))


def test_large_frontier_windows(dupin):
    """A first tail round that selects thousands of vertices per CTA (more than
    one 512-entry expand window), with k = 2 on a sparse graph handed to the
    cluster at once (n <= tail_cap, few arcs)."""
    g = synth.random_general(60000, 90000, seed=9)
    synth.with_weights(g, "dw", seed=9, a_range=(0, 3))
    for k in (1, 2):
        out, ref = run_both(dupin, g, "dw", k, (1, 10), flags=dupin.TAIL_CLUSTER, tail_cap=100000,
                            tail_arc_cap=1 << 30)
        assert out.n_bulk_rounds == 0 and out.tail_ctas in (8, 16)
        assert max(ref.trace_peeled) > 16 * 512
        assert_same(out, ref, k)


@pytest.mark.parametrize("k", [1, 2])
def test_skewed_bipartite_cluster(dupin, k):
    """Zipf items (hubs with thousands of arcs) and camouflaged blocks, FD weights."""
    g = synth.bipartite_zipf(20000, 10000, 150000, 1.8, 2, 60, 60, 0.4, 20, seed=5)
    g.c = synth.fd_weights(g)
    g.a = synth.uniform_vertex_weights(g.n, 0, 2, seed=5)
    for tail_cap in (0, 1000, 30000):
        for eps in ((1, 20), (0, 1)):
            out, ref = run_both(dupin, g, "fd", k, eps, flags=dupin.TAIL_CLUSTER, tail_cap=tail_cap)
            assert_same(out, ref, (k, tail_cap, eps))


def test_rmat16_default_and_forced(dupin):
    """R-MAT scale 16 (65k vertices, more than one CTA holds): the automatic
    choice, the forced cluster and the forced one-CTA tail give the oracle's peel."""
    g = synth.rmat_weighted(16, 16, "fd", seed=2)
    for metric in ("dg", "fd"):
        for flags in (0, "cluster", "one"):
            f = {0: 0, "cluster": dupin.TAIL_CLUSTER, "one": dupin.TAIL_ONE_CTA}[flags]
            out, ref = run_both(dupin, g, metric, 1, (1, 10), flags=f)
            assert_same(out, ref, (metric, flags))
            if flags == "one":
                assert out.tail_ctas in (0, 1)
            if flags == "cluster":
                assert out.tail_ctas in (0, 8, 16)


def test_flags_exclude_each_other(dupin):
    g = synth.random_general(100, 300, seed=1)
    dg = dupin.Graph.from_synth(g)
    with pytest.raises(dupin.DupinError) as e:
        dupin.peel(dg, "dg", 1, (1, 10), flags=dupin.TAIL_CLUSTER | dupin.TAIL_ONE_CTA)
    assert e.value.code == dupin.ERR_INVALID_ARG
    dg.free()


def test_repeated_goldens_no_race(dupin):
    """Every worked example 25 times on the cluster: a remote update that a
    round's barrier failed to order would show up as a run that differs."""
    for path in sorted(glob.glob(os.path.join(GOLDEN, "peel_*.json"))):
        G = json.load(open(path))
        eu = np.array([e[0] for e in G["edges"]], np.int32)
        ev = np.array([e[1] for e in G["edges"]], np.int32)
        g = synth.SynthGraph(G["n"], 0, eu, ev, np.array([e[2] * Q for e in G["edges"]], np.int64),
                             np.array([x * Q for x in G["a"]], np.int64))
        dg = dupin.Graph.from_synth(g)
        for case in G["cases"]:
            flags = {"": 0, "gpo": dupin.GPO, "lpo": dupin.LPO}[case.get("flags", "")] | dupin.TAIL_CLUSTER
            for rep in range(25):
                out = dupin.peel(dg, G["metric"], case["k"], tuple(case["eps"]), flags=flags, want_trace=False)
                assert list(out.peel_round) == case["peel_round"], (path, case.get("flags"), rep)
        dg.free()
