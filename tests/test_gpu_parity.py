"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Results are exact integers (Q32.32 weights, 128-bit f), so the bar is bit
equality of every vertex's peel round, the whole density trace (f_i, |S_i|,
|U_i|) and the best prefix.  Cases cover the tail-only path (n <= tail_cap),
the persistent bulk kernel (tail_cap forced small), both thresholds (k = 1
with the minimum rule, k = 2, k = 3), GPO, several eps, every metric, skewed
and ragged graphs, and the degenerate ones (empty, edgeless, one vertex).
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
@pytest.mark.parametrize("tail_cap", [0, 1])
def test_golden_examples(dupin, path, tail_cap):
    G = json.load(open(path))
    eu = np.array([e[0] for e in G["edges"]], np.int32)
    ev = np.array([e[1] for e in G["edges"]], np.int32)
    g = synth.SynthGraph(G["n"], 0, eu, ev, np.array([e[2] * Q for e in G["edges"]], np.int64),
                         np.array([x * Q for x in G["a"]], np.int64))
    dg = dupin.Graph.from_synth(g)
    for case in G["cases"]:
        flags = {"": 0, "gpo": dupin.GPO, "lpo": dupin.LPO}[case.get("flags", "")]
        out = dupin.peel(dg, G["metric"], case["k"], tuple(case["eps"]), flags=flags, tail_cap=tail_cap)
        assert list(out.peel_round) == case["peel_round"]
        assert out.trace_f == [x * Q for x in case["trace_f"]]
        assert list(out.trace_size) == case["trace_size"]
        assert list(out.trace_peeled) == case["trace_peeled"]
        assert (out.best_round, out.best_size, out.best_f) == (case["best_round"], case["best_size"], case["best_f"] * Q)
        assert out.n_min_rule == case["n_min_rule"]
    dg.free()


@pytest.mark.parametrize("metric", ["dg", "dw", "fd"])
@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("tail_cap", [0, 1, 300])
def test_random_general(dupin, metric, k, tail_cap):
    for seed in range(3):
        g = synth.random_general(2000 + 37 * seed, 12000, seed=seed + 1)
        synth.with_weights(g, metric, seed=seed, a_range=(0, 7) if metric != "dg" else None)
        for eps in ((1, 10), (0, 1), (3, 4)):
            out, ref = run_both(dupin, g, metric, k, eps, tail_cap=tail_cap)
            assert_same(out, ref, (metric, k, tail_cap, seed, eps))


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("tail_cap", [0, 1, 1000])
def test_skewed_bipartite_fd(dupin, k, tail_cap):
    g = synth.bipartite_zipf(20000, 10000, 150000, 1.8, 2, 60, 60, 0.4, 20, seed=5)
    g.c = synth.fd_weights(g)
    g.a = synth.uniform_vertex_weights(g.n, 0, 2, seed=5)
    for eps in ((1, 20), (0, 1), (1, 5)):
        out, ref = run_both(dupin, g, "fd", k, eps, tail_cap=tail_cap)
        assert_same(out, ref, (k, tail_cap, eps))


@pytest.mark.parametrize("tail_cap", [0, 1, 5000])
def test_rmat_dw_gpo(dupin, tail_cap):
    g = synth.rmat_weighted(14, 16, "dw", seed=3)
    for k in (1, 2):
        for flags in (0, 1):
            out, ref = run_both(dupin, g, "dw", k, (1, 10), flags=flags, tail_cap=tail_cap)
            assert_same(out, ref, (k, flags, tail_cap))


def live_arcs_after(g, peel_round, r):
    """2 |E(S_r)|: arcs whose both ends are still live after round r."""
    u, v = g.global_edges()
    return 2 * int(np.count_nonzero(np.minimum(peel_round[u], peel_round[v]) > r))


def small_round(g, ref, r):
    """Round r removed at most 64 vertices or expanded at most 2^18 arcs (the
    removed vertices' degrees in the whole graph)."""
    if ref.trace_peeled[r] <= 64:
        return True
    ptr, _, _ = g.symmetric_csr()
    deg = np.diff(ptr)
    return int(deg[np.asarray(ref.peel_round) == r].sum()) <= (1 << 18)


@pytest.mark.parametrize("tail_arc_cap", [1, 700, 20000])
def test_tail_waits_for_few_arcs(dupin, tail_arc_cap):
    """The tail starts once S fits it and either 2|E(S)| <= tail_arc_cap or the
    last grid-wide round removed at most 64 vertices; the grid-wide rounds
    track |E(S)| exactly (the arcs the tail was built from match the oracle's
    rounds), and the peel is unchanged."""
    graphs = [(synth.rmat_weighted(14, 16, "dw", seed=3), "dw"),
              (synth.bipartite_zipf(3000, 1500, 20000, 1.6, 1, 30, 30, 0.5, 12, seed=4), "fd")]
    graphs[1][0].c = synth.fd_weights(graphs[1][0])
    for g, metric in graphs:
        for k in (1, 2):
            for tail_cap in (2000, 300):
                out, ref = run_both(dupin, g, metric, k, (1, 10), tail_cap=tail_cap, tail_arc_cap=tail_arc_cap)
                ctx = (metric, k, tail_cap, tail_arc_cap)
                assert_same(out, ref, ctx)
                nb = out.n_bulk_rounds
                exact = live_arcs_after(g, ref.peel_round, nb)
                assert out.tail_arcs == exact, ctx
                # the tail starts once S fits and either its arcs are few or the
                # last grid-wide round was small (<= 64 vertices or <= 2^18 arcs) ...
                if out.tail_arcs > 0:
                    assert ref.trace_size[nb] <= tail_cap, ctx
                    assert out.tail_arcs <= tail_arc_cap or (nb > 0 and small_round(g, ref, nb)), ctx
                # ... and not later
                if nb > 0:
                    r = nb - 1
                    small = r > 0 and small_round(g, ref, r)
                    assert ref.trace_size[r] > tail_cap or (live_arcs_after(g, ref.peel_round, r) > tail_arc_cap
                                                            and not small), ctx


@pytest.mark.parametrize("tail_cap", [0, 1, 500])
def test_lpo(dupin, tail_cap):
    """Algorithm 4: trim rounds (w < max(tau_max, g)) after every round, in the
    one-CTA tail (tail_cap 0), the grid-wide kernel (tail_cap 1) and across the
    hand-over (500): bit-exact against the oracle's replay."""
    fd = synth.bipartite_zipf(3000, 1500, 20000, 1.6, 1, 30, 30, 0.5, 12, seed=4)
    fd.c = synth.fd_weights(fd)
    cases = [(synth.rmat_weighted(13, 16, "dw", seed=3), "dw"), (fd, "fd"),
             (synth.dg_planted_block(seed=2, nU=3000, nI=1500, draws=20000, block=60, p=0.5), "dg")]
    for g, metric in cases:
        for k in (1, 2):
            for eps in ((0, 1), (1, 10)):
                out, ref = run_both(dupin, g, metric, k, eps, flags=dupin.LPO, tail_cap=tail_cap)
                assert_same(out, ref, (metric, k, eps, tail_cap))


def test_planted_block_config(dupin):
    """10k x 5k bipartite DG with the 200x200 block (the small workload), every path."""
    g = synth.dg_planted_block(seed=1)
    for k in (1, 2):
        for tail_cap in (0, 1, 2048):
            out, ref = run_both(dupin, g, "dg", k, (1, 10), tail_cap=tail_cap)
            assert_same(out, ref, (k, tail_cap))
            assert 300 <= out.best_size <= 450


def test_degenerate_graphs(dupin):
    # edgeless with vertex weights; one vertex; a single edge; a clique; a star
    cases = [
        synth.SynthGraph(50, 0, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64),
                         synth.uniform_vertex_weights(50, 0, 9, 2)),
        synth.SynthGraph(1, 0, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64), None),
        synth.SynthGraph(2, 0, np.array([0], np.int32), np.array([1], np.int32), np.array([5 * Q], np.int64), None),
    ]
    q = 40
    iu, iv = np.triu_indices(q, 1)
    cases.append(synth.SynthGraph(q, 0, iu.astype(np.int32), iv.astype(np.int32), np.full(iu.size, Q, np.int64), None))
    cases.append(synth.SynthGraph(q + 1, 0, np.zeros(q, np.int32), np.arange(1, q + 1, dtype=np.int32),
                                  np.full(q, Q, np.int64), None))
    for g in cases:
        for k in (1, 2):
            for tail_cap in (0, 1):
                out, ref = run_both(dupin, g, "dw", k, (1, 10), tail_cap=tail_cap)
                assert_same(out, ref, (g.n, k, tail_cap))


def test_empty_graph(dupin):
    g = synth.SynthGraph(0, 0, np.zeros(0, np.int32), np.zeros(0, np.int32), None, None)
    dg = dupin.Graph.load_symmetric(0, np.zeros(1, np.int64), np.zeros(0, np.int32))
    out = dupin.peel(dg, "dg", 1, (1, 10))
    assert out.n_rounds == 0 and out.best_size == 0
    dg.free()
    del g


def test_repeatable(dupin):
    g = synth.rmat_weighted(13, 16, "fd", seed=9)
    dg = dupin.Graph.from_synth(g)
    outs = [dupin.peel(dg, "fd", 1, (1, 10), tail_cap=tc) for tc in (0, 0, 1, 1)]
    for o in outs[1:]:
        assert np.array_equal(o.peel_round, outs[0].peel_round) and o.trace_f == outs[0].trace_f
    dg.free()


def test_errors(dupin):
    # neighbour id out of range
    with pytest.raises(dupin.DupinError) as e:
        dupin.Graph.load_symmetric(3, np.array([0, 1, 2, 2], np.int64), np.array([1, 7], np.int32))
    assert e.value.code == dupin.ERR_INVALID_ARG
    # self-loop
    with pytest.raises(dupin.DupinError) as e:
        dupin.Graph.load_symmetric(2, np.array([0, 1, 2], np.int64), np.array([0, 1], np.int32))
    assert e.value.code == dupin.ERR_INVALID_ARG
    # negative weight (Property 3.1)
    with pytest.raises(dupin.DupinError) as e:
        dupin.Graph.load_symmetric(2, np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32),
                                   np.array([-Q, -Q], np.int64))
    assert e.value.code == dupin.ERR_INVALID_ARG
    # initial peeling weight >= 2^63
    with pytest.raises(dupin.DupinError) as e:
        dupin.Graph.load_symmetric(3, np.array([0, 2, 3, 4], np.int64), np.array([1, 2, 0, 0], np.int32),
                                   np.array([2**62, 2**62, 2**62, 2**62], np.int64))
    assert e.value.code == dupin.ERR_OVERFLOW
    # round cap and a short trace buffer
    g = synth.random_general(500, 3000, seed=2)
    synth.with_weights(g, "dw", seed=2)
    dg = dupin.Graph.from_synth(g)
    with pytest.raises(dupin.DupinError) as e:
        dupin.peel(dg, "dw", 1, (0, 1), max_rounds=3)
    assert e.value.code == dupin.ERR_NO_PROGRESS
    with pytest.raises(dupin.DupinError) as e:
        dupin.peel(dg, "dw", 1, (1, 10), k_mult=0) if False else dupin.peel(dg, "dw", 0, (1, 10))
    assert e.value.code == dupin.ERR_INVALID_ARG
    import ctypes

    p = dupin.make_params("dw", 1, (1, 10))
    fh, fl, sz, pe = (np.zeros(2, np.int64), np.zeros(2, np.uint64), np.zeros(2, np.int64), np.zeros(2, np.int64))
    r = dupin._result_struct(None, None, (fh, fl, sz, pe), 2)
    rc = dupin.lib().dupin_peel(dg.handle, ctypes.byref(p), ctypes.byref(r), None)
    assert rc == dupin.ERR_BUFFER_TOO_SMALL and r.n_rounds > 1
    # DW without weights loaded
    gu = synth.random_general(100, 300, seed=3)
    dgu = dupin.Graph.from_synth(gu)
    with pytest.raises(dupin.DupinError):
        dupin.peel(dgu, "dw", 1, (1, 10))
    dgu.free()
    dg.free()


def test_loader_rejects_malformed_adjacency(dupin):
    """dupin_graph_load: unsorted rows, a repeated pair, a missing or
    re-weighted reverse arc, and a CSC that does not hold the CSR's edges are
    INVALID_ARG; the well-formed versions load."""
    sym = lambda n, rp, col, w=None: dupin.Graph.load_symmetric(n, np.array(rp, np.int64), np.array(col, np.int32),
                                                                None if w is None else np.array(w, np.int64))
    # path 0-1-2 loads
    sym(3, [0, 1, 3, 4], [1, 0, 2, 1]).free()
    cases = [
        ("unsorted row", (3, [0, 1, 3, 4], [1, 2, 0, 1])),
        ("repeated pair", (2, [0, 2, 4], [1, 1, 0, 0])),
        ("missing reverse arc", (3, [0, 1, 2, 4], [1, 2, 0, 1])),
        ("re-weighted reverse arc", (3, [0, 1, 3, 4], [1, 0, 2, 1], [Q, Q, 2 * Q, 3 * Q])),
    ]
    for name, args in cases:
        with pytest.raises(dupin.DupinError) as e:
            sym(*args)
        assert e.value.code == dupin.ERR_INVALID_ARG, name
    # bipartite: 2 users x 2 items, edges (0,0), (1,1)
    cp, ci, cw = np.array([0, 1, 2], np.int64), np.array([0, 1], np.int32), np.array([Q, 2 * Q], np.int64)
    dupin.Graph.load_bipartite(2, 2, cp, ci, cw, np.array([0, 1, 2], np.int64), np.array([0, 1], np.int32),
                               np.array([Q, 2 * Q], np.int64)).free()
    bad_cscs = [("CSC names another user", np.array([1, 1], np.int32), np.array([Q, 2 * Q], np.int64)),
                ("CSC weight differs", np.array([0, 1], np.int32), np.array([Q, 3 * Q], np.int64))]
    for name, idx, w in bad_cscs:
        with pytest.raises(dupin.DupinError) as e:
            dupin.Graph.load_bipartite(2, 2, cp, ci, cw, np.array([0, 1, 2], np.int64), idx, w)
        assert e.value.code == dupin.ERR_INVALID_ARG, name
    # a large synthetic graph with one reverse arc re-weighted
    g = synth.random_general(5000, 40000, seed=4)
    synth.with_weights(g, "dw", seed=4)
    ptr, idx, w = g.symmetric_csr()
    dupin.Graph.load_symmetric(g.n, ptr, idx, w).free()
    w2 = w.copy()
    w2[len(w2) // 2] += Q
    with pytest.raises(dupin.DupinError) as e:
        dupin.Graph.load_symmetric(g.n, ptr, idx, w2)
    assert e.value.code == dupin.ERR_INVALID_ARG


def test_device_results(dupin):
    import torch

    g = synth.rmat_weighted(12, 8, "dw", seed=4)
    dg = dupin.Graph.from_synth(g)
    ref = dupin.peel(dg, "dw", 1, (1, 10))
    pr = torch.empty(g.n, dtype=torch.int32, device="cuda")
    mk = torch.empty(g.n, dtype=torch.uint8, device="cuda")
    r = dupin.peel_device(dg, dupin.make_params("dw", 1, (1, 10)), pr, mk)
    torch.cuda.synchronize()
    assert np.array_equal(pr.cpu().numpy(), ref.peel_round)
    assert np.array_equal(mk.cpu().numpy(), ref.best_mask)
    assert r.best_round == ref.best_round
    dg.free()


def test_device_pointer_load(dupin):
    import torch

    g = synth.bipartite_zipf(3000, 1500, 20000, 1.8, 0, 0, 0, 0.0, 0, seed=8)
    g.c = synth.fd_weights(g)
    parts = [torch.from_numpy(x).cuda() for x in g.bipartite_csr()]
    dgd = dupin.Graph.load_bipartite(g.n_left, g.n_right, *parts, device_ptrs=True)
    dgh = dupin.Graph.from_synth(g)
    a = dupin.peel(dgd, "fd", 1, (1, 10))
    b = dupin.peel(dgh, "fd", 1, (1, 10))
    assert np.array_equal(a.peel_round, b.peel_round) and a.trace_f == b.trace_f
    dgd.free()
    dgh.free()


def test_handover_autotuner(dupin):
    """dupin_tune_handover times the peel under each hand-over candidate and
    returns one of them; the peel under the winner equals the default peel and
    the oracle (the hand-over point never changes a result)."""
    g = synth.rmat_weighted(16, 16, "fd", seed=3)
    dg = dupin.Graph.from_synth(g)
    best, times = dupin.tune_handover(dg, "fd", 1, (1, 10))
    assert best in times and len(times) == dupin.TUNE_HANDOVER_N
    assert all(t > 0 for t in times.values()) and times[best] == min(times.values())
    ref = dupin.peel(dg, "fd", 1, (1, 10))
    out = dupin.peel(dg, "fd", 1, (1, 10), tail_arc_cap=best)
    assert np.array_equal(out.peel_round, ref.peel_round) and out.trace_f == ref.trace_f
    og = oracle.Graph.from_synth(g, "fd")
    orc = oracle.peel_batch(og, 1, (1, 10))
    og.close()
    assert np.array_equal(out.peel_round, orc.peel_round) and out.trace_f == orc.trace_f
    with pytest.raises(dupin.DupinError) as e:
        dupin.tune_handover(dg, "tds", 3, (1, 10))
    assert e.value.code == dupin.ERR_INVALID_ARG
    dg.free()
