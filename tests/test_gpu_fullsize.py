"""Full-size workloads on the GPU, checked against the oracle.

* R-MAT scale 24 (16.8M vertices, 260M edges, c in 1..100): the benchmark
  graph.  DG, FD and DW (a in 0..10) each at k = 1 and k = 2, eps = 1/10,
  bit-exact against the oracle's full replay of Algorithm 2: every vertex's
  peel round, the whole density trace, the per-round sizes, the minimum-rule
  count and the best prefix.  k = 1 peels run 3k to 13k rounds, nearly all of
  them through the cluster tail.
* FD transaction graph, 2M users x 1M items, 40.7M edges: bit-exact against
  the full replay for eps = 0, 1/20 and 1/5.
* R-MAT scale 18 (DW): bit-exact against the full replay, k = 1 and k = 2.
* R-MAT scale 22 (FD weights): the benchmark step's batched call (FD then DG)
  against the oracle's replay of each peel.
* R-MAT scale 22 (DW): the verifier checks every vertex's round against the
  definitions (its peeling weight at the start of its round is at most the
  threshold recomputed from the trace, or equals the minimum), recomputes the
  whole density trace from the peel rounds, checks the best round, and checks
  every survivor at sampled rounds.
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


def verify(og, out, k, eps, nsample=3):
    fh = np.array([x >> 64 for x in out.trace_f], np.int64)
    fl = np.array([x & ((1 << 64) - 1) for x in out.trace_f], np.uint64)
    return oracle.verify(og, k, eps, out.peel_round, out.n_rounds, fh, fl, out.trace_size, out.trace_peeled,
                         out.best_round, nsample=nsample)


def test_fd_config_full_size(dupin):
    g = synth.fd_camouflage(seed=1)
    dg = dupin.Graph.from_synth(g)
    og = oracle.Graph.from_synth(g, "fd")
    for eps in ((0, 1), (1, 20), (1, 5)):
        out = dupin.peel(dg, "fd", 1, eps)
        ref = oracle.peel_batch(og, 1, eps)
        assert np.array_equal(out.peel_round, ref.peel_round), eps
        assert out.trace_f == ref.trace_f, eps
        assert (out.best_round, out.best_size, out.best_f) == (ref.best_round, ref.best_size, ref.best_f), eps
    dg.free()
    og.close()


def test_rmat18_exact(dupin):
    g = synth.rmat_weighted(18, 16, "dw", seed=2)
    dg = dupin.Graph.from_synth(g)
    og = oracle.Graph.from_synth(g, "dw")
    for k in (1, 2):
        out = dupin.peel(dg, "dw", k, (1, 10))
        ref = oracle.peel_batch(og, k, (1, 10))
        assert np.array_equal(out.peel_round, ref.peel_round)
        assert out.trace_f == ref.trace_f
        assert (out.best_round, out.best_size, out.best_f) == (ref.best_round, ref.best_size, ref.best_f)
    dg.free()
    og.close()


def test_rmat22_verified(dupin):
    g = synth.rmat_weighted(22, 16, "dw", seed=1)
    dg = dupin.Graph.from_synth(g)
    og = oracle.Graph.from_synth(g, "dw")
    for k in (1, 2):
        out = dupin.peel(dg, "dw", k, (1, 10))
        assert verify(og, out, k, (1, 10)) == (0, "")
        assert out.trace_size[-1] == 0 and out.trace_f[-1] == 0
    dg.free()
    og.close()


@pytest.fixture(scope="module")
def rmat24():
    return synth.rmat_weighted(24, 16, "fd", seed=1)


@pytest.mark.parametrize("metric", ["dg", "fd", "dw"])
def test_rmat24_exact(dupin, rmat24, metric):
    g = rmat24
    if metric == "dw":  # same topology, DW weights
        g = synth.SynthGraph(rmat24.n_left, rmat24.n_right, rmat24.eu, rmat24.ev)
        synth.with_weights(g, "dw", 1, a_range=(0, 10), c_range=(1, 100))
    dg = dupin.Graph.from_synth(g)
    og = oracle.Graph.from_synth(g, metric)
    for k in (1, 2):
        out = dupin.peel(dg, metric, k, (1, 10), want_mask=False)
        ref = oracle.peel_batch(og, k, (1, 10))
        assert ref.violations == 0
        assert out.n_rounds == ref.n_rounds, (metric, k)
        assert np.array_equal(out.peel_round, ref.peel_round), (metric, k)
        assert out.trace_f == ref.trace_f, (metric, k)
        assert np.array_equal(out.trace_size, ref.trace_size) and np.array_equal(out.trace_peeled, ref.trace_peeled)
        assert (out.best_round, out.best_size, out.best_f) == (ref.best_round, ref.best_size, ref.best_f)
        assert out.n_min_rule == ref.n_min_rule
        if k == 1:
            assert out.tail_ctas > 1  # the rounds after the bulk phase ran in the cluster tail
    dg.free()
    og.close()


def test_rmat22_batched_step_matches_oracle(dupin):
    """The benchmark step's own path at scale 22: FD then DG (eps = 1/10,
    k = 1) in one batched call -- the grid-wide stages in turn, the DG stage
    narrowed beside the FD cluster tail, the two cluster tails side by side --
    equals the oracle's replay of each peel."""
    import torch

    g = synth.rmat_weighted(22, 16, "fd", seed=1)
    dg = dupin.Graph.from_synth(g)
    params = [dupin.make_params(m, 1, (1, 10)) for m in ("fd", "dg")]
    prs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in params]
    mks = [torch.empty(g.n, dtype=torch.uint8, device="cuda") for _ in params]
    R = dupin.peel_batch_device([dg] * 2, params, prs, mks)
    torch.cuda.synchronize()
    for j, metric in enumerate(("fd", "dg")):
        og = oracle.Graph.from_synth(g, metric)
        ref = oracle.peel_batch(og, 1, (1, 10))
        og.close()
        assert R[j].tail_ctas > 1, metric  # the cluster tail ran
        assert np.array_equal(prs[j].cpu().numpy(), ref.peel_round), metric
        assert np.array_equal(mks[j].cpu().numpy(), ref.best_mask), metric
        assert (R[j].n_rounds, R[j].best_round, R[j].best_size) == (ref.n_rounds, ref.best_round, ref.best_size)
    dg.free()
