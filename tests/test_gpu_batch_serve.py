"""Batched and served peels equal single-graph peels exactly (GPU).

dupin_peel_batch runs window-sized graphs one CTA each in one persistent
launch and larger graphs through the single-graph path; the serving layer
admits requests into slots under a device-memory budget and runs them
concurrently.  The arithmetic is the same exact integer peel, so every
result (peel rounds, density trace, best prefix) must be bit-identical to
dupin_peel on the same graph, alone or in a mix.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2504_09311_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dupin():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2504_09311_gb300 import dupin as d

    d.lib()
    return d


def same(a, b, ctx=""):
    assert a.n_rounds == b.n_rounds, ctx
    assert np.array_equal(a.peel_round, b.peel_round), ctx
    assert (a.best_round, a.best_size, a.best_f) == (b.best_round, b.best_size, b.best_f), ctx
    assert a.n_min_rule == b.n_min_rule, ctx
    if a.trace_f is not None and b.trace_f is not None:
        assert a.trace_f == b.trace_f, ctx
        assert np.array_equal(np.asarray(a.trace_size), np.asarray(b.trace_size)), ctx


def window_graphs(count, seed, lo=1000, hi=60000):
    sizes = synth.window_sizes(count, lo, hi, seed=seed)
    return [synth.transaction_window(int(m), seed=seed * 1000 + j) for j, m in enumerate(sizes)]


def test_batch_equals_single(dupin):
    gs = window_graphs(24, seed=3)
    # one graph beyond the one-CTA limit takes the single-graph path
    big = synth.bipartite_zipf(200_000, 100_000, 900_000, 1.8, 1, 50, 50, 0.4, 10, seed=9)
    big.c = synth.fd_weights(big)
    gs.insert(5, big)
    # and a DW graph with vertex weights, and a DG graph
    dw = synth.random_general(5000, 40000, seed=2)
    synth.with_weights(dw, "dw", seed=2, a_range=(0, 4))
    gs.append(dw)
    gs.append(synth.dg_planted_block(seed=2, nU=3000, nI=1500, draws=20000, block=60, p=0.5))
    metrics = ["fd"] * 25 + ["dw", "dg"]
    dgs = [dupin.Graph.from_synth(g) for g in gs]
    params = []
    for j, g in enumerate(gs):
        k = 1 + (j % 2)
        eps = [(1, 10), (0, 1), (1, 5)][j % 3]
        flags = dupin.GPO if j % 5 == 4 else (dupin.LPO if j % 7 == 3 else 0)
        params.append(dupin.make_params(metrics[j], k, eps, flags=flags))
    outs = dupin.peel_batch(dgs, params, want_rounds=True, want_trace=True)
    for j, (g, dg, p) in enumerate(zip(gs, dgs, params)):
        ref = dupin.peel(dg, p.metric, p.k_mult, (p.eps_num, p.eps_den), flags=p.flags)
        same(outs[j], ref, j)
    # the small case against the oracle as well
    og = oracle.Graph.from_synth(gs[0], "fd")
    r = oracle.peel_batch(og, params[0].k_mult, (params[0].eps_num, params[0].eps_den))
    assert np.array_equal(outs[0].peel_round, r.peel_round) and outs[0].trace_f == r.trace_f
    for dg in dgs:
        dg.free()


def test_batch_shapes_and_tune(dupin):
    """Both launch shapes of the one-CTA kernel give the same results, the
    graphs on either side of the one-CTA limit included; the autotuner keeps
    one of the two shapes."""
    lim = dupin.BATCH_CTA_MAX_N
    gs = window_graphs(12, seed=5)
    for n in (lim, lim + 1):  # the largest one-CTA graph, the smallest that is not
        g = synth.random_general(n, 4 * n, seed=n)
        synth.with_weights(g, "fd", seed=1)
        gs.append(g)
    assert gs[-2].n == lim and gs[-1].n == lim + 1
    dgs = [dupin.Graph.from_synth(g) for g in gs]
    params = [dupin.make_params("fd", 1 + j % 2, (1, 10), flags=dupin.LPO if j % 4 == 1 else 0)
              for j in range(len(gs))]
    keep = dupin.batch_threads()
    try:
        outs = {}
        for t in (128, 256):
            assert dupin.batch_threads(t) == t
            outs[t] = dupin.peel_batch(dgs, params, want_rounds=True, want_trace=True)
        for j in range(len(gs)):
            same(outs[128][j], outs[256][j], j)
        for j in (0, len(gs) - 2, len(gs) - 1):
            p = params[j]
            r = oracle.peel_batch(oracle.Graph.from_synth(gs[j], "fd"), p.k_mult, (p.eps_num, p.eps_den),
                                  flags=oracle.FLAG_LPO if p.flags & dupin.LPO else 0)
            assert np.array_equal(outs[128][j].peel_round, r.peel_round), j
            assert outs[128][j].trace_f == r.trace_f, j
        dupin.batch_threads(0)  # the default rule: this small launch takes 256 threads
        for j, o in enumerate(dupin.peel_batch(dgs, params, want_rounds=True, want_trace=True)):
            same(o, outs[256][j], j)
        t = dupin.batch_tune(dgs, params)
        assert t in (128, 256) and dupin.batch_threads() == t
        with pytest.raises(dupin.DupinError):
            dupin.batch_tune(dgs[-1:], params[-1:])  # nothing small enough to time
        assert dupin.batch_threads() == t
        with pytest.raises(dupin.DupinError):
            dupin.batch_threads(64)
    finally:
        dupin.batch_threads(keep)
        for dg in dgs:
            dg.free()


def test_batch_large_concurrent(dupin):
    """Several large peels in one call -- one graph under three eps, another
    under two settings, with a small graph mixed in -- run their grid-wide
    stages in turn and their tails side by side; every result equals its own
    dupin_peel (host results, then device results)."""
    import torch

    big1 = synth.bipartite_zipf(200_000, 100_000, 900_000, 1.8, 2, 60, 60, 0.4, 10, seed=11)
    big1.c = synth.fd_weights(big1)
    big2 = synth.rmat_weighted(19, 8, "dw", seed=5)
    small = synth.transaction_window(30000, seed=12)
    gs = [big1, big1, big2, small, big1, big2]
    dg1, dg2, dgs_ = dupin.Graph.from_synth(big1), dupin.Graph.from_synth(big2), dupin.Graph.from_synth(small)
    dgs = [dg1, dg1, dg2, dgs_, dg1, dg2]
    ps = [dupin.make_params("fd", 1, (0, 1)), dupin.make_params("fd", 1, (1, 20)),
          dupin.make_params("dw", 1, (1, 10)), dupin.make_params("fd", 1, (1, 10)),
          dupin.make_params("fd", 1, (1, 5)), dupin.make_params("dw", 2, (1, 10), flags=dupin.GPO)]
    outs = dupin.peel_batch(dgs, ps, want_rounds=True, want_trace=True)
    refs = [dupin.peel(dg, p.metric, p.k_mult, (p.eps_num, p.eps_den), flags=p.flags) for dg, p in zip(dgs, ps)]
    for j in range(len(gs)):
        same(outs[j], refs[j], j)
    # device-resident results through the same path
    k = len(gs)
    prs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in gs]
    mks = [torch.empty(g.n, dtype=torch.uint8, device="cuda") for g in gs]
    P = (dupin.Params * k)()
    R = (dupin.Result * k)()
    G = (ctypes.c_void_p * k)(*[dg.handle.value for dg in dgs])
    for j in range(k):
        P[j] = ps[j]
        P[j].flags |= dupin.RESULT_DEVICE
        R[j].peel_round = prs[j].data_ptr()
        R[j].best_mask = mks[j].data_ptr()
    dupin.check(dupin.lib().dupin_peel_batch(ctypes.cast(G, ctypes.c_void_p), ctypes.cast(P, ctypes.c_void_p),
                                             ctypes.cast(R, ctypes.c_void_p), k, None))
    torch.cuda.synchronize()
    for j in range(k):
        assert np.array_equal(prs[j].cpu().numpy(), refs[j].peel_round), j
        assert np.array_equal(mks[j].cpu().numpy(), refs[j].best_mask), j
        assert R[j].best_round == refs[j].best_round and R[j].n_rounds == refs[j].n_rounds, j
    for dg in (dg1, dg2, dgs_):
        dg.free()


def test_batch_repeated_graph_and_device_results(dupin):
    import torch

    g = synth.transaction_window(20000, seed=77)
    dg = dupin.Graph.from_synth(g)
    ps = [dupin.make_params("fd", 1, e) for e in ((1, 10), (1, 20), (0, 1))] * 2
    outs = dupin.peel_batch([dg] * len(ps), ps, want_rounds=True, want_trace=True)
    for o, p in zip(outs, ps):
        same(o, dupin.peel(dg, "fd", 1, (p.eps_num, p.eps_den)))
    # device-resident results
    k = 3
    prs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in range(k)]
    mks = [torch.empty(g.n, dtype=torch.uint8, device="cuda") for _ in range(k)]
    P = (dupin.Params * k)()
    R = (dupin.Result * k)()
    G = (ctypes.c_void_p * k)(*[dg.handle.value] * k)
    for j in range(k):
        P[j] = dupin.make_params("fd", 1, ((1, 10), (1, 20), (0, 1))[j], flags=dupin.RESULT_DEVICE)
        R[j].peel_round = prs[j].data_ptr()
        R[j].best_mask = mks[j].data_ptr()
    dupin.check(dupin.lib().dupin_peel_batch(ctypes.cast(G, ctypes.c_void_p), ctypes.cast(P, ctypes.c_void_p),
                                             ctypes.cast(R, ctypes.c_void_p), k, None))
    torch.cuda.synchronize()
    for j in range(k):
        ref = dupin.peel(dg, "fd", 1, ((1, 10), (1, 20), (0, 1))[j])
        assert np.array_equal(prs[j].cpu().numpy(), ref.peel_round)
        assert np.array_equal(mks[j].cpu().numpy(), ref.best_mask)
        assert R[j].best_round == ref.best_round
    dg.free()


def test_workspace_cache_across_graphs(dupin):
    """A freed graph's workspaces serve later graphs they fit (a larger graph's
    for a smaller one, DW-sized for DG); results do not change."""
    small = synth.rmat_weighted(14, 8, "dw", seed=21)
    big = synth.bipartite_zipf(200_000, 100_000, 900_000, 1.8, 1, 50, 50, 0.4, 10, seed=22)
    big.c = synth.fd_weights(big)
    dg_s = dupin.Graph.from_synth(small)
    ref = [dupin.peel(dg_s, "dw", 1, (1, 10), tail_cap=tc) for tc in (0, 1)]
    dg_s.free()
    dupin.trim_cache()
    for rep in range(2):
        dg_b = dupin.Graph.from_synth(big)
        outs = dupin.peel_batch([dg_b] * 2, [dupin.make_params("fd", 1, e) for e in ((1, 10), (1, 5))])
        assert all(o.n_rounds > 0 for o in outs)
        dg_b.free()  # its workspaces go to the cache
        dg_s = dupin.Graph.from_synth(small)
        for tc, r in zip((0, 1), ref):
            same(dupin.peel(dg_s, "dw", 1, (1, 10), tail_cap=tc), r, (rep, tc))
        dg_s.free()
    dupin.trim_cache()


def test_serving_alone_and_in_a_mix(dupin):
    gs = window_graphs(16, seed=5, lo=1000, hi=40000)
    big = synth.bipartite_zipf(40_000, 20_000, 200_000, 1.8, 1, 40, 40, 0.4, 10, seed=4)
    big.c = synth.fd_weights(big)
    gs.append(big)
    dgs = [dupin.Graph.from_synth(g) for g in gs]
    refs = [dupin.peel(dg, "fd", 1, (1, 10)) for dg in dgs]
    srv = dupin.Server(memory_budget=2 << 30, max_slots=8)
    p = dupin.make_params("fd", 1, (1, 10))
    # alone: one request at a time
    for j in (0, len(dgs) - 1):
        t = srv.submit(dgs[j], p, want_trace=True)
        same(srv.wait(t), refs[j], ("alone", j))
    # in a mix: everything at once, several times over, waited in reverse order
    tickets = [(j, srv.submit(dgs[j], p, want_trace=True)) for _ in range(3) for j in range(len(dgs))]
    for j, t in reversed(tickets):
        same(srv.wait(t), refs[j], ("mix", j))
    st = srv.stats()
    assert st["completed"] == st["submitted"] == 2 + 3 * len(dgs)
    assert st["p99_ms"] >= st["p50_ms"] > 0 and st["graphs_per_s"] > 0
    srv.close()
    for dg in dgs:
        dg.free()


def test_serving_budget(dupin):
    g = synth.transaction_window(50000, seed=8)
    dg = dupin.Graph.from_synth(g)
    srv = dupin.Server(memory_budget=1 << 16, max_slots=2)  # far below one request's state
    with pytest.raises(dupin.DupinError) as e:
        srv.submit(dg, dupin.make_params("fd", 1, (1, 10)))
    assert e.value.code == dupin.ERR_OOM
    assert srv.stats()["rejected"] == 1
    srv.close()
    dg.free()
