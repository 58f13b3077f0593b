"""The q-clique density metric kCLiDS (Sec. 2.1) on the GPU against the CPU
oracle's clique peel, element by element, through the C ABI.

f(S) is the number of q-cliques of G[S] and w_u(S) those through u (plain
counts); the rounds are Algorithm 2 with the paper's k = q and with k = 1
(the minimum rule), and Algorithms 3 and 4 by flag.  The device lists the
cliques through each removed vertex by a depth-first walk over its sorted
row, for every q from 3 to DUPIN_CLIQUE_MAX_Q.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2504_09311_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def dupin():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2504_09311_gb300 import dupin as d

    d.lib()
    return d


def compare(dupin, g, q, k, eps, flags=0, ctx=""):
    og = oracle.Graph.from_synth(g, "dg")
    of = (oracle.FLAG_GPO if flags & dupin.GPO else 0) | (oracle.FLAG_LPO if flags & dupin.LPO else 0)
    ref = oracle.peel_clique(og, q, k, eps, flags=of)
    og.close()
    dg = dupin.Graph.from_synth(g)
    out = dupin.peel(dg, "kclids", k, eps, flags=flags, clique_q=q)
    dg.free()
    assert out.n_rounds == ref.n_rounds, ctx
    assert np.array_equal(out.peel_round, ref.peel_round), ctx
    assert out.trace_f == ref.trace_f, ctx
    assert np.array_equal(np.asarray(out.trace_size), ref.trace_size), ctx
    assert np.array_equal(np.asarray(out.trace_peeled), ref.trace_peeled), ctx
    assert (out.best_round, out.best_size, out.best_f) == (ref.best_round, ref.best_size, ref.best_f), ctx
    assert out.n_min_rule == ref.n_min_rule, ctx
    assert np.array_equal(out.best_mask, ref.best_mask), ctx
    return out


def with_clique(base, members):
    """base plus every pair of 'members' (a planted clique)."""
    m = np.asarray(members)
    iu, iv = np.triu_indices(len(m), 1)
    pairs = set(zip(base.eu.tolist(), base.ev.tolist()))
    for a, b in zip(m[iu].tolist(), m[iv].tolist()):
        pairs.add((min(a, b), max(a, b)))
    e = np.array(sorted(pairs), np.int32)
    return synth.SynthGraph(base.n_left, 0, e[:, 0].copy(), e[:, 1].copy())


def test_golden_k4_triangle(dupin):
    """The hand-derived example (a K4 with a triangle attached) for q = 3 and q = 4."""
    G = json.load(open(os.path.join(GOLDEN, "clique_k4_triangle.json")))
    eu = np.array([e[0] for e in G["edges"]], np.int32)
    ev = np.array([e[1] for e in G["edges"]], np.int32)
    g = synth.SynthGraph(G["n"], 0, eu, ev)
    dg = dupin.Graph.from_synth(g)
    for case in G["cases"]:
        out = dupin.peel(dg, "kclids", case["k"], tuple(case["eps"]), clique_q=case["q"])
        assert list(out.peel_round) == case["peel_round"], case["q"]
        assert out.trace_f == case["trace_f"]
        assert list(out.trace_size) == case["trace_size"]
        assert list(out.trace_peeled) == case["trace_peeled"]
        assert (out.best_round, out.best_size, out.best_f) == (case["best_round"], case["best_size"], case["best_f"])
        assert out.n_min_rule == case["n_min_rule"]
    dg.free()


def test_complete_graph_closed_form(dupin):
    """K_n has C(n, q) q-cliques, each vertex in C(n-1, q-1): every weight
    equals q f / n, so the first round removes every vertex."""
    from math import comb

    n = 11
    iu, iv = np.triu_indices(n, 1)
    g = synth.SynthGraph(n, 0, iu.astype(np.int32), iv.astype(np.int32))
    dg = dupin.Graph.from_synth(g)
    for q in range(3, 9):
        out = dupin.peel(dg, "kclids", q, (0, 1), clique_q=q)
        assert out.trace_f == [comb(n, q), 0], q
        assert out.n_rounds == 1 and out.best_size == n and out.best_f == comb(n, q)
    dg.free()


@pytest.mark.parametrize("q", [4, 5])
@pytest.mark.parametrize("flags", ["", "gpo", "lpo"])
def test_dense_random_graphs(dupin, q, flags):
    f = {"": 0, "gpo": dupin.GPO, "lpo": dupin.LPO}[flags]
    for seed, (n, m) in enumerate(((120, 2800), (140, 3400))):  # edge density about 0.4
        g = synth.random_general(n, m, seed=seed + 50)
        for k in (1, q):
            for eps in ((1, 10), (0, 1)):
                compare(dupin, g, q, k, eps, f, (q, k, flags, seed, eps))


def test_three_matches_tds(dupin):
    """kCLiDS with q = 3 (the walk) and TDS (the triangle merge) give the same peel."""
    g = synth.random_general(500, 7000, seed=61)
    dg = dupin.Graph.from_synth(g)
    for k, flags in ((1, 0), (3, 0), (3, dupin.LPO)):
        a = dupin.peel(dg, "kclids", k, (1, 10), flags=flags, clique_q=3)
        b = dupin.peel(dg, "tds", k, (1, 10), flags=flags)
        assert np.array_equal(a.peel_round, b.peel_round)
        assert a.trace_f == b.trace_f and (a.best_round, a.best_f) == (b.best_round, b.best_f)
    dg.free()
    compare(dupin, g, 3, 3, (1, 10), 0)


@pytest.mark.parametrize("q", [6, 7, 8])
def test_planted_clique_large_q(dupin, q):
    """A 16-clique and a 12-clique planted in a sparse random graph: the
    densest prefix holds the 16-clique; exact against the oracle."""
    base = synth.random_general(600, 1800, seed=70 + q)
    g = with_clique(with_clique(base, range(100, 116)), range(300, 312))
    for k, flags in ((1, 0), (q, 0), (q, dupin.LPO)):
        out = compare(dupin, g, q, k, (1, 10), flags, (q, k, flags))
    assert set(range(100, 116)) <= set(np.nonzero(out.best_mask)[0].tolist())


def test_rmat_with_hubs(dupin):
    """R-MAT scale 13 (rows of degree up to 1,520, hub rows re-coded on the
    device; skewed clique counts), q = 4."""
    g = synth.rmat(13, 8, seed=9)
    for k, flags in ((1, 0), (4, 0), (4, dupin.LPO)):
        compare(dupin, g, 4, k, (1, 10), flags, (k, flags))


def test_clique_free_and_tiny(dupin):
    # a triangle-free graph has no q-cliques: f = 0 and every vertex leaves in round 1
    b = synth.bipartite_uniform(200, 100, 1500, seed=4)
    out = compare(dupin, b, 4, 4, (1, 10))
    assert out.n_rounds == 1 and out.best_f == 0
    cases = [
        synth.SynthGraph(1, 0, np.zeros(0, np.int32), np.zeros(0, np.int32)),
        synth.SynthGraph(3, 0, np.array([0, 0, 1], np.int32), np.array([1, 2, 2], np.int32)),
        synth.SynthGraph(4, 0, np.array([0, 0, 0, 1, 1, 2], np.int32), np.array([1, 2, 3, 2, 3, 3], np.int32)),
    ]
    for g in cases:
        for q in (3, 4, 5):
            for k in (1, q):
                compare(dupin, g, q, k, (1, 10), 0, (g.n, q, k))


def test_clique_size_out_of_range_and_dupin_peel_only(dupin):
    g = synth.random_general(100, 600, seed=1)
    dg = dupin.Graph.from_synth(g)
    for q in (0, 2, dupin.CLIQUE_MAX_Q + 1):
        with pytest.raises(dupin.DupinError) as e:
            dupin.peel(dg, "kclids", 3, (1, 10), clique_q=q)
        assert e.value.code == dupin.ERR_INVALID_ARG, q
    with pytest.raises(dupin.DupinError) as e:
        dupin.peel_batch([dg], [dupin.make_params("kclids", 4, (1, 10), clique_q=4)])
    assert e.value.code == dupin.ERR_INVALID_ARG
    with pytest.raises(dupin.DupinError) as e:
        dupin.tune_handover(dg, "kclids", 4, (1, 10))
    assert e.value.code == dupin.ERR_INVALID_ARG
    dg.free()
