"""The triangle-density metric TDS (Sec. 2.1) on the GPU against the CPU
oracle's clique peel (q = 3), element by element, through the C ABI.

f(S) is the number of triangles of G[S] and w_u(S) those through u (plain
counts); the rounds are Algorithm 2 with the paper's k = 3 and with k = 1
(the minimum rule), and Algorithms 3 and 4 by flag.
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


def compare(dupin, g, k, eps, flags=0, ctx=""):
    og = oracle.Graph.from_synth(g, "dg")
    of = (oracle.FLAG_GPO if flags & dupin.GPO else 0) | (oracle.FLAG_LPO if flags & dupin.LPO else 0)
    ref = oracle.peel_clique(og, 3, k, eps, flags=of)
    og.close()
    dg = dupin.Graph.from_synth(g)
    out = dupin.peel(dg, "tds", k, eps, flags=flags)
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


def test_golden_k4_triangle(dupin):
    G = json.load(open(os.path.join(GOLDEN, "clique_k4_triangle.json")))
    eu = np.array([e[0] for e in G["edges"]], np.int32)
    ev = np.array([e[1] for e in G["edges"]], np.int32)
    g = synth.SynthGraph(G["n"], 0, eu, ev)
    dg = dupin.Graph.from_synth(g)
    for case in G["cases"]:
        if case["q"] != 3:
            continue
        out = dupin.peel(dg, "tds", case["k"], tuple(case["eps"]))
        assert list(out.peel_round) == case["peel_round"]
        assert out.trace_f == case["trace_f"]
        assert list(out.trace_size) == case["trace_size"]
        assert list(out.trace_peeled) == case["trace_peeled"]
        assert (out.best_round, out.best_size, out.best_f) == (case["best_round"], case["best_size"], case["best_f"])
        assert out.n_min_rule == case["n_min_rule"]
        assert out.best_density == pytest.approx(case["best_f"] / case["best_size"])
    dg.free()


@pytest.mark.parametrize("k", [1, 3])
@pytest.mark.parametrize("flags", ["", "gpo", "lpo"])
def test_random_graphs(dupin, k, flags):
    f = {"": 0, "gpo": dupin.GPO, "lpo": dupin.LPO}[flags]
    for seed in range(3):
        g = synth.random_general(400 + 97 * seed, 6000, seed=seed + 30)
        for eps in ((1, 10), (0, 1)):
            compare(dupin, g, k, eps, f, (k, flags, seed, eps))


@pytest.mark.parametrize("k", [1, 3])
def test_rmat_with_hubs(dupin, k):
    """R-MAT scale 12 (hub rows re-coded on the device, skewed triangle counts)."""
    g = synth.rmat(12, 8, seed=5)
    for flags in (0, dupin.LPO):
        compare(dupin, g, k, (1, 10), flags, (k, flags))


def test_planted_clique_is_found(dupin):
    """A 40-clique in a sparse random graph: the densest prefix is the clique."""
    base = synth.random_general(2000, 5000, seed=8)
    q = 40
    iu, iv = np.triu_indices(q, 1)
    pairs = set(zip(base.eu.tolist(), base.ev.tolist())) | set(zip(iu.tolist(), iv.tolist()))
    eu = np.array(sorted(pairs), np.int32)
    g = synth.SynthGraph(2000, 0, eu[:, 0].copy(), eu[:, 1].copy())
    out = compare(dupin, g, 3, (1, 10), 0)
    assert out.best_size >= q and out.best_f >= q * (q - 1) * (q - 2) // 6


def test_triangle_free_and_tiny(dupin):
    # a bipartite graph has no triangles: f = 0 and every vertex leaves in round 1
    b = synth.bipartite_uniform(300, 200, 2000, seed=3)
    out = compare(dupin, b, 3, (1, 10))
    assert out.n_rounds == 1 and out.best_f == 0
    cases = [
        synth.SynthGraph(1, 0, np.zeros(0, np.int32), np.zeros(0, np.int32)),
        synth.SynthGraph(3, 0, np.array([0, 0, 1], np.int32), np.array([1, 2, 2], np.int32)),
        synth.SynthGraph(5, 0, np.array([0, 1, 2, 3], np.int32), np.array([1, 2, 3, 4], np.int32)),
    ]
    for g in cases:
        for k in (1, 3):
            compare(dupin, g, k, (1, 10), 0, (g.n, k))


def test_tds_is_dupin_peel_only(dupin):
    g = synth.random_general(100, 600, seed=1)
    dg = dupin.Graph.from_synth(g)
    with pytest.raises(dupin.DupinError) as e:
        dupin.peel_batch([dg], [dupin.make_params("tds", 3, (1, 10))])
    assert e.value.code == dupin.ERR_INVALID_ARG
    dg.free()
