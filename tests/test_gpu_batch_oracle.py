"""Batched and served peels against the CPU oracle, graph by graph.

Hundreds of transaction-window graphs (edge counts log-uniform, Zipf items)
go through one dupin_peel_batch call with every metric, k_mult 1 and 2, and
Algorithms 2, 3 and 4 mixed; a serving mix adds graphs too large for one
CTA.  Each result is compared element by element with the single-threaded
oracle's peel of the same graph and parameters (not with another CUDA path).
"""
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


def assert_oracle(out, g, metric, k, eps, flags, dupin, ctx):
    of = (oracle.FLAG_GPO if flags & dupin.GPO else 0) | (oracle.FLAG_LPO if flags & dupin.LPO else 0)
    og = oracle.Graph.from_synth(g, metric)
    ref = oracle.peel_batch(og, k, eps, flags=of)
    og.close()
    assert out.n_rounds == ref.n_rounds, ctx
    assert np.array_equal(out.peel_round, ref.peel_round), ctx
    assert (out.best_round, out.best_size, out.best_f) == (ref.best_round, ref.best_size, ref.best_f), ctx
    assert out.n_min_rule == ref.n_min_rule, ctx
    if out.trace_f is not None:
        assert out.trace_f == ref.trace_f, ctx
        assert np.array_equal(np.asarray(out.trace_size), ref.trace_size), ctx
        assert np.array_equal(np.asarray(out.trace_peeled), ref.trace_peeled), ctx


def mixed_case(j, dupin):
    metric = ("dg", "dw", "fd")[j % 3]
    k = 1 + (j // 3) % 2
    eps = ((1, 10), (0, 1), (1, 5), (1, 20))[j % 4]
    flags = (0, dupin.GPO, dupin.LPO)[(j // 6) % 3]
    return metric, k, eps, flags


def weighted(g, metric, seed):
    if metric == "dw":
        h = synth.SynthGraph(g.n_left, g.n_right, g.eu, g.ev)
        return synth.with_weights(h, "dw", seed=seed, a_range=(0, 5), c_range=(1, 50))
    return g


def test_batched_windows_match_oracle(dupin):
    count = 300
    sizes = synth.window_sizes(count, 1000, 30000, seed=12)
    graphs, params, cases = [], [], []
    for j, m in enumerate(sizes):
        metric, k, eps, flags = mixed_case(j, dupin)
        g = weighted(synth.transaction_window(int(m), seed=12000 + j), metric, j)
        graphs.append(g)
        params.append(dupin.make_params(metric, k, eps, flags=flags))
        cases.append((metric, k, eps, flags))
    dgs = [dupin.Graph.from_synth(g) for g in graphs]
    outs = dupin.peel_batch(dgs, params, want_rounds=True, want_trace=True)
    for j, (g, o, c) in enumerate(zip(graphs, outs, cases)):
        assert_oracle(o, g, *c, dupin, (j, c))
    for dg in dgs:
        dg.free()


def test_serving_mix_matches_oracle(dupin):
    """A continuous-batching server under a small slot count: window requests
    and requests on graphs too large for one CTA, each result against the oracle."""
    pool = [synth.transaction_window(int(m), seed=500 + j)
            for j, m in enumerate(synth.window_sizes(24, 1000, 20000, seed=5))]
    big = synth.rmat_weighted(18, 4, "fd", seed=4)  # 262,144 vertices: above the one-CTA-per-graph limit
    big2 = synth.bipartite_zipf(150_000, 75_000, 600_000, 1.8, 1, 40, 40, 0.4, 10, seed=6)
    big2.c = synth.fd_weights(big2)
    graphs = pool + [big, big2]
    dgs = [dupin.Graph.from_synth(g) for g in graphs]
    srv = dupin.Server(memory_budget=4 << 30, max_slots=6)
    tickets = []
    for j in range(90):
        gi = j % len(graphs) if j % 15 else len(graphs) - 1 - (j // 15) % 2
        metric, k, eps, flags = mixed_case(j, dupin)
        if metric == "dw":
            metric = "fd"  # the pool carries FD weights only
        p = dupin.make_params(metric, k, eps, flags=flags)
        tickets.append((gi, (metric, k, eps, flags), srv.submit(dgs[gi], p, want_rounds=True)))
    outs = [(gi, c, srv.wait(t)) for gi, c, t in tickets]
    srv.close()
    for j, (gi, c, o) in enumerate(outs):
        assert_oracle(o, graphs[gi], *c, dupin, (j, gi, c))
    for dg in dgs:
        dg.free()
