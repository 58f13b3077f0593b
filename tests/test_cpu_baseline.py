"""The multi-threaded CPU Algorithm 2 baseline equals the oracle bit for bit.

Several thread counts, every metric, k = 1 and 2, GPO and LPO, skewed and
small graphs: peel rounds, density trace, best prefix and the count of
minimum-rule rounds must all match.
"""
import numpy as np
import pytest

import cpu_baseline
import oracle
from paper_2504_09311_gb300 import synth


def graphs():
    fd = synth.bipartite_zipf(3000, 1500, 20000, 1.6, 1, 30, 30, 0.5, 12, seed=4)
    fd.c = synth.fd_weights(fd)
    dw = synth.random_general(2000, 12000, seed=5)
    synth.with_weights(dw, "dw", seed=5, a_range=(0, 5))
    return [(synth.rmat_weighted(12, 16, "dw", seed=3), "dw"), (fd, "fd"), (dw, "dw"),
            (synth.dg_planted_block(seed=2, nU=3000, nI=1500, draws=20000, block=60, p=0.5), "dg")]


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_matches_oracle(threads):
    for g, metric in graphs():
        og = oracle.Graph.from_synth(g, metric)
        cg = cpu_baseline.Graph(g, metric)
        for k in (1, 2):
            for eps in ((0, 1), (1, 10)):
                for flags in (0, oracle.FLAG_GPO, oracle.FLAG_LPO):
                    ref = oracle.peel_batch(og, k, eps, flags=flags)
                    pr, R, br, bs, bf, tf, ts, tp, nmin = cpu_baseline.peel(cg, k, eps, flags, threads)
                    ctx = (metric, k, eps, flags, threads)
                    assert R == ref.n_rounds, ctx
                    assert np.array_equal(pr, ref.peel_round), ctx
                    assert tf == ref.trace_f, ctx
                    assert np.array_equal(ts, ref.trace_size) and np.array_equal(tp, ref.trace_peeled), ctx
                    assert (br, bs, bf) == (ref.best_round, ref.best_size, ref.best_f), ctx
                    assert nmin == ref.n_min_rule, ctx
        og.close()
