"""The seeded input generator: determinism, shapes and the FD weight formula."""
import math

import numpy as np

from paper_2504_09311_gb300 import synth

Q = 1 << 32


def test_deterministic_and_seed_dependent():
    a = synth.dg_planted_block(seed=3)
    b = synth.dg_planted_block(seed=3)
    c = synth.dg_planted_block(seed=4)
    assert np.array_equal(a.eu, b.eu) and np.array_equal(a.ev, b.ev)
    assert not (a.m == c.m and np.array_equal(a.eu, c.eu) and np.array_equal(a.ev, c.ev))


def test_thread_count_does_not_change_output():
    synth.lib().sg_set_threads(1)
    a = synth.bipartite_zipf(3000, 1500, 30000, 1.8, 1, 50, 50, 0.3, 10, seed=5)
    synth.lib().sg_set_threads(7)
    b = synth.bipartite_zipf(3000, 1500, 30000, 1.8, 1, 50, 50, 0.3, 10, seed=5)
    synth.lib().sg_set_threads(0)
    assert np.array_equal(a.eu, b.eu) and np.array_equal(a.ev, b.ev)
    r1 = synth.rmat(12, 8, seed=2)
    synth.lib().sg_set_threads(3)
    r2 = synth.rmat(12, 8, seed=2)
    synth.lib().sg_set_threads(0)
    assert np.array_equal(r1.eu, r2.eu) and np.array_equal(r1.ev, r2.ev)


def test_edge_lists_are_simple_and_sorted():
    for g in (synth.dg_planted_block(seed=1), synth.rmat(12, 8, seed=1), synth.random_general(500, 3000, seed=1)):
        key = g.eu.astype(np.int64) * (1 << 32) + g.ev.astype(np.int64)
        assert np.all(np.diff(key) > 0)  # sorted, no repeats
        if not g.bipartite:
            assert np.all(g.eu < g.ev)  # no self-loops, u < v
        else:
            assert g.eu.max() < g.n_left and g.ev.max() < g.n_right


def test_zipf_graph_has_exact_background_size_and_skew():
    g = synth.bipartite_zipf(20000, 10000, 150000, 1.8, 0, 0, 0, 0.0, 0, seed=2)
    assert g.m == 150000
    deg = np.bincount(g.ev, minlength=g.n_right)
    # Zipf(1.8): the most popular item is hit by about half of all draws and
    # saturates at every user
    assert deg.max() == 20000
    assert np.median(deg) < 20


def test_rmat_shape():
    g = synth.rmat(14, 16, seed=1)
    assert g.n == 1 << 14
    assert 0.6 * 16 * g.n < g.m < 16 * g.n  # self-loops and repeats removed
    deg = np.bincount(np.concatenate([g.eu, g.ev]), minlength=g.n)
    assert deg.max() > 50 * deg.mean()  # heavy tail


def test_fd_weights_match_formula():
    """c_e = round(2^32 / ln(x + 5)), x = item degree (Sec. 2.1 Fraudar, Listing 1)."""
    g = synth.bipartite_zipf(2000, 1000, 20000, 1.8, 0, 0, 0, 0.0, 0, seed=9)
    c = synth.fd_weights(g)
    deg = np.bincount(g.ev, minlength=g.n_right)
    expect = np.array([round(Q / math.log(deg[i] + 5.0)) for i in g.ev], np.int64)
    assert np.max(np.abs(c - expect)) <= 1
    # general graphs: the larger endpoint is the object vertex
    r = synth.random_general(300, 2000, seed=4)
    cr = synth.fd_weights(r)
    d = np.bincount(np.concatenate([r.eu, r.ev]), minlength=r.n)
    expect = np.array([round(Q / math.log(d[v] + 5.0)) for v in r.ev], np.int64)
    assert np.max(np.abs(cr - expect)) <= 1


def test_det_ln_accuracy():
    for x in [1.0, 2.0, 5.0, 6.0, 7.5, 1e3, 2e6 + 5, 123456.789, 0.3]:
        assert abs(synth.det_ln(x) - math.log(x)) <= 4e-16 * max(1.0, abs(math.log(x)))


def test_layouts():
    g = synth.dg_planted_block(seed=2, nU=300, nI=200, draws=2000, block=20, p=0.5)
    synth.with_weights(g, "dw", seed=1, a_range=(0, 10))
    csr_ptr, csr_idx, csr_w, csc_ptr, csc_idx, csc_w = g.bipartite_csr()
    assert csr_ptr[-1] == g.m and csc_ptr[-1] == g.m
    # same edge multiset with the same weights in both layouts
    e1 = sorted((u, int(csr_idx[p]), int(csr_w[p])) for u in range(g.n_left) for p in range(csr_ptr[u], csr_ptr[u + 1]))
    e2 = sorted((int(csc_idx[p]), i, int(csc_w[p])) for i in range(g.n_right) for p in range(csc_ptr[i], csc_ptr[i + 1]))
    assert e1 == e2
    ptr, idx, w = g.symmetric_csr()
    assert ptr[-1] == 2 * g.m
    for u in range(0, g.n, 37):
        row = idx[ptr[u]:ptr[u + 1]]
        assert np.all(np.diff(row) > 0)
    gu, gv = g.global_edges()
    s = set(zip(gu.tolist(), gv.tolist()))
    for u in range(0, g.n, 13):
        for p in range(ptr[u], ptr[u + 1]):
            v = int(idx[p])
            assert (min(u, v), max(u, v)) in s


def _rows_sorted_and_symmetric(ptr, idx, w):
    n = len(ptr) - 1
    row = np.repeat(np.arange(n, dtype=np.int64), np.diff(ptr))
    # strictly increasing within each row
    same_row = row[1:] == row[:-1]
    assert np.all(idx[1:][same_row] > idx[:-1][same_row])
    # the arc multiset equals its reverse, weights included
    fwd = np.lexsort((idx, row))
    rev = np.lexsort((row, idx.astype(np.int64)))
    assert np.array_equal(row[fwd], idx[rev]) and np.array_equal(idx[fwd], row[rev])
    if w is not None:
        assert np.array_equal(w[fwd], w[rev])


def test_csrs_meet_the_loader_preconditions():
    """The loader rejects rows that are not strictly increasing and asymmetric
    adjacencies; every CSR the generator hands it satisfies both."""
    g = synth.rmat_weighted(12, 16, "dw", seed=2)
    _rows_sorted_and_symmetric(*g.symmetric_csr())
    b = synth.bipartite_zipf(3000, 1500, 30000, 1.8, 1, 50, 50, 0.3, 10, seed=5)
    b.c = synth.fd_weights(b)
    _rows_sorted_and_symmetric(*b.symmetric_csr())
    cp, ci, cw, kp, ki, kw = b.bipartite_csr()
    for ptr, idx in ((cp, ci), (kp, ki)):
        r = np.repeat(np.arange(len(ptr) - 1), np.diff(ptr))
        same = r[1:] == r[:-1]
        assert np.all(idx[1:][same] > idx[:-1][same])
    # CSR and CSC hold the same (user, item, weight) triples
    u1 = np.repeat(np.arange(len(cp) - 1), np.diff(cp))
    i2 = np.repeat(np.arange(len(kp) - 1), np.diff(kp))
    a = sorted(zip(u1.tolist(), ci.tolist(), cw.tolist()))
    bb = sorted(zip(ki.tolist(), i2.tolist(), kw.tolist()))
    assert a == bb
