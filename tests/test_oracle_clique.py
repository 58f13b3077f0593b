"""Pins of the oracle's clique-metric peel (TDS, kCLiDS; Sec. 2.1) -- CPU only.

The clique metrics take f(S) = number of q-cliques of G[S] (q = 3 for TDS)
and the peeling weight w_u(S) = q-cliques of G[S] through u.  What fixes the
oracle independently of itself:
  * a hand-derived worked example (tests/golden/clique_*.json);
  * q = 2 is DG: the same peel as the Q32.32 DG peel, round for round;
  * closed forms: a clique K_p (every vertex in C(p-1, q-1) cliques; one
    round), triangle-free graphs (f = 0);
  * every round's f recounted in Python with itertools over the surviving
    set, and the per-vertex weights recounted the same way;
  * the approximation bound g(S^p) >= g* / (max(k, q)(1 + eps)) against a
    brute-force optimum (the paper's bound for multiplier q, Sec. 4.3; the
    minimum rule keeps it for smaller k because min w <= q g);
  * Lemma 4.1's shrink |S_i| < |S_{i-1}| / (1 + eps) for k = q and eps > 0,
    and Lemma 4.2 (no empty round).
The verifier for large results (og_verify_clique) accepts the oracle's runs
and rejects planted mistakes.
"""
import itertools
import json
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
Q = 1 << 32


def graph(n, edges):
    return oracle.Graph(n, [a for a, b in edges], [b for a, b in edges], metric="dg")


def random_edges(n, p, seed):
    rng = random.Random(seed)
    return [(u, v) for u in range(n) for v in range(u + 1, n) if rng.random() < p]


def cliques_in(S, q, adj):
    return sum(1 for c in itertools.combinations(sorted(S), q)
               if all(b in adj[a] for a, b in itertools.combinations(c, 2)))


def adjacency(n, edges):
    adj = [set() for _ in range(n)]
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    return adj


def test_golden_clique_peel():
    G = json.load(open(os.path.join(GOLDEN, "clique_k4_triangle.json")))
    g = graph(G["n"], G["edges"])
    for case in G["cases"]:
        r = oracle.peel_clique(g, case["q"], case["k"], tuple(case["eps"]))
        assert r.violations == 0
        assert list(r.peel_round) == case["peel_round"], case
        assert r.trace_f == case["trace_f"]
        assert list(r.trace_size) == case["trace_size"]
        assert list(r.trace_peeled) == case["trace_peeled"]
        assert list(r.trace_T) == case["trace_T"]
        assert (r.best_round, r.best_size, r.best_f) == (case["best_round"], case["best_size"], case["best_f"])
        assert r.n_min_rule == case["n_min_rule"]
    for b in G["brute_force"]:
        assert oracle.brute_force_clique(g, b["q"]) == (b["size"], b["cliques"], b["mask"])


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("k,eps", [(1, (1, 10)), (2, (0, 1)), (2, (1, 5)), (3, (1, 2))])
def test_q2_is_dg(seed, k, eps):
    n = 40
    edges = random_edges(n, 0.15, seed)
    g = graph(n, edges)
    a = oracle.peel_clique(g, 2, k, eps)
    b = oracle.peel_batch(g, k, eps)
    assert a.violations == 0 and b.violations == 0
    assert np.array_equal(a.peel_round, b.peel_round)
    assert (a.n_rounds, a.best_round, a.best_size) == (b.n_rounds, b.best_round, b.best_size)
    assert [x * Q for x in a.trace_f] == b.trace_f
    assert a.best_f * Q == b.best_f
    assert a.n_min_rule == b.n_min_rule


@pytest.mark.parametrize("p,q", [(3, 3), (5, 3), (6, 4), (7, 5), (5, 5), (9, 6), (10, 7), (11, 8)])
def test_clique_closed_form(p, q):
    edges = [(u, v) for u in range(p) for v in range(u + 1, p)]
    g = graph(p, edges)
    r = oracle.peel_clique(g, q, q, (1, 10))
    assert r.n_rounds == 1 and list(r.peel_round) == [1] * p
    assert (r.best_round, r.best_size, r.best_f) == (0, p, math.comb(p, q))
    assert r.trace_T[1] == (q * 11 * math.comb(p, q)) // (10 * p)
    assert r.trace_T[1] >= math.comb(p - 1, q - 1)  # every vertex's weight
    # multiplier 1: the threshold (1+eps) C(p-1,q-1)/q selects nobody, the minimum rule takes all
    r1 = oracle.peel_clique(g, q, 1, (1, 10))
    assert r1.n_rounds == 1 and r1.n_min_rule == 1


@pytest.mark.parametrize("seed", range(4))
def test_triangle_free(seed):
    rng = random.Random(seed)
    nl, nr = 12, 9
    edges = [(u, nl + v) for u in range(nl) for v in range(nr) if rng.random() < 0.4]
    g = graph(nl + nr, edges)
    r = oracle.peel_clique(g, 3, 3, (1, 10))
    assert r.trace_f == [0, 0] and r.n_rounds == 1
    assert (r.best_round, r.best_size, r.best_f) == (0, nl + nr, 0)


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("q", [3, 4, 5, 6])
def test_rounds_recounted(seed, q):
    n = 14
    edges = random_edges(n, 0.55 if q <= 4 else 0.75, seed)  # denser for q >= 5: some cliques exist
    adj = adjacency(n, edges)
    g = graph(n, edges)
    for k, eps in [(q, (1, 10)), (1, (0, 1))]:
        r = oracle.peel_clique(g, q, k, eps)
        assert r.violations == 0
        assert all(x > 0 for x in r.trace_peeled[1:])  # Lemma 4.2
        for i in range(r.n_rounds + 1):
            S = [u for u in range(n) if r.peel_round[u] > i]
            assert r.trace_f[i] == cliques_in(S, q, adj)
            assert r.trace_size[i] == len(S)
        # every vertex peeled in round i had at most T_i cliques through it in S_{i-1};
        # a survivor had more (threshold rounds) or more than the minimum (minimum rule)
        for i in range(1, r.n_rounds + 1):
            S = [u for u in range(n) if r.peel_round[u] >= i]
            w = {u: sum(1 for c in itertools.combinations([x for x in S if x != u], q - 1)
                        if all(b in adj[a] for a, b in itertools.combinations(c, 2))
                        and all(x in adj[u] for x in c)) for u in S}
            T = r.trace_T[i]
            for u in S:
                if r.peel_round[u] == i:
                    assert w[u] <= T
                else:
                    assert w[u] > T


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("q,k,eps", [(3, 3, (1, 10)), (3, 1, (1, 10)), (3, 3, (0, 1)), (4, 4, (1, 5)), (4, 2, (1, 2))])
def test_approximation_bound(seed, q, k, eps):
    n = 13
    edges = random_edges(n, 0.5, 100 + seed)
    g = graph(n, edges)
    size, cl, mask = oracle.brute_force_clique(g, q)
    gstar = Fraction(cl, size)
    r = oracle.peel_clique(g, q, k, eps)
    gp = Fraction(r.best_f, r.best_size)
    assert gp <= gstar
    assert gp * max(k, q) * (1 + Fraction(*eps)) >= gstar
    for flags in (oracle.FLAG_GPO, oracle.FLAG_LPO):
        rf = oracle.peel_clique(g, q, k, eps, flags=flags)
        assert rf.violations == 0
        assert Fraction(rf.best_f, rf.best_size) * max(k, q) * (1 + Fraction(*eps)) >= gstar


@pytest.mark.parametrize("seed", range(4))
def test_lemma_4_1_shrink(seed):
    n = 60
    edges = random_edges(n, 0.3, 7 + seed)
    g = graph(n, edges)
    eps = Fraction(1, 4)
    r = oracle.peel_clique(g, 3, 3, (1, 4))
    assert r.n_min_rule == 0
    for i in range(1, r.n_rounds + 1):
        assert r.trace_size[i] * (1 + eps) < r.trace_size[i - 1] or r.trace_size[i] == 0
    assert r.n_rounds <= math.log(n) / math.log(1.25) + 1


def test_brute_force_clique_matches_python():
    n = 11
    edges = random_edges(n, 0.6, 3)
    adj = adjacency(n, edges)
    g = graph(n, edges)
    for q in (3, 4):
        best = None
        for mask in range(1, 1 << n):
            S = [u for u in range(n) if mask >> u & 1]
            d = Fraction(cliques_in(S, q, adj), len(S))
            if best is None or d > best[0]:
                best = (d, len(S), mask)
        size, cl, mask = oracle.brute_force_clique(g, q)
        assert Fraction(cl, size) == best[0] and mask == best[2]


def test_clique_errors():
    g = graph(3, [(0, 1), (1, 2)])
    with pytest.raises(oracle.OracleError):
        oracle.peel_clique(g, 1, 1, (1, 10))
    with pytest.raises(oracle.OracleError):
        oracle.peel_clique(g, 3, 0, (1, 10))
    with pytest.raises(oracle.OracleError):
        oracle.brute_force_clique(graph(21, []), 3)


def _vc(g, q, k, eps, r, pr=None, fh=None, best=None, nsample=64):
    fh_arr = np.array([x >> 64 for x in r.trace_f], np.int64) if fh is None else fh
    fl_arr = np.array([x & ((1 << 64) - 1) for x in r.trace_f], np.uint64)
    return oracle.verify_clique(g, q, k, eps, r.peel_round if pr is None else pr, r.n_rounds, fh_arr, fl_arr,
                                r.trace_size, r.trace_peeled, r.best_round if best is None else best, nsample=nsample)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("q,k,eps", [(3, 3, (1, 10)), (3, 1, (0, 1)), (4, 4, (1, 5))])
def test_clique_verifier_accepts_and_rejects(seed, q, k, eps):
    n = 30
    g = graph(n, random_edges(n, 0.35, 50 + seed))
    r = oracle.peel_clique(g, q, k, eps)
    assert _vc(g, q, k, eps, r) == (0, "")
    if r.n_rounds >= 2:
        # a vertex moved to the next round
        pr = r.peel_round.copy()
        u = int(np.flatnonzero(pr == 1)[0])
        pr[u] = 2
        assert _vc(g, q, k, eps, r, pr=pr)[0] != 0
        # a wrong best round
        assert _vc(g, q, k, eps, r, best=(r.best_round + 1) % r.n_rounds)[0] != 0
    # a wrong f in the trace (high word)
    fh = np.array([x >> 64 for x in r.trace_f], np.int64)
    fh[0] += 1
    assert _vc(g, q, k, eps, r, fh=fh)[0] != 0
