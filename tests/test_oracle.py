"""Pins for the CPU oracle (no GPU needed).

The oracle is checked against things other than itself:
  * hand-derived worked examples (tests/golden/*.json, derivations inside);
  * brute-force enumeration of all subsets (n <= 16) and exact DG densest
    subgraphs by Goldberg's max-flow construction, which must agree;
  * closed forms: cliques, stars, complete bipartite graphs, disjoint unions;
  * the approximation theorems (Thm 2.1 for Algorithm 1, Thm 4.3 for
    Algorithm 2), Lemma 4.1's round bound and Lemma 4.2's non-empty rounds;
  * per-round invariants (2 f(S) = sum_{u in S} (w_u + a_u), f maintained by
    deltas equals f recomputed from scratch, w maintained equals w recomputed);
  * the verifier accepts the oracle's runs and rejects planted mistakes.
"""
import glob
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2504_09311_gb300 import synth

Q = 1 << 32
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def graph_from_lists(n, edges, a=None, metric="dw"):
    eu = np.array([e[0] for e in edges], np.int32)
    ev = np.array([e[1] for e in edges], np.int32)
    c = np.array([e[2] * Q for e in edges], np.int64) if edges and len(edges[0]) > 2 else None
    aa = np.array([x * Q for x in a], np.int64) if a is not None else None
    return oracle.Graph(n, eu, ev, c, aa, metric)


def random_small(n, p, seed, weighted=True, with_a=True):
    rng = np.random.default_rng(seed)
    edges = []
    for u in range(n):
        for v in range(u + 1, n):
            if rng.random() < p:
                edges.append((u, v, int(rng.integers(1, 9)) if weighted else 1))
    a = [int(x) for x in rng.integers(0, 4, n)] if with_a else None
    return edges, a


def density(f, s):
    return Fraction(f, s)


# ---------------------------------------------------------------- goldens


def case_flags(case) -> int:
    """A golden case's variant: "" Algorithm 2, "gpo" Algorithm 3, "lpo" Algorithm 4."""
    return {"": 0, "gpo": oracle.FLAG_GPO, "lpo": oracle.FLAG_LPO}[case.get("flags", "")]


def golden_files():
    return sorted(glob.glob(os.path.join(GOLDEN, "peel_*.json")))


@pytest.mark.parametrize("path", golden_files(), ids=lambda p: os.path.basename(p))
def test_golden_batch_peel(path):
    G = json.load(open(path))
    g = graph_from_lists(G["n"], G["edges"], G["a"], G["metric"])
    for case in G["cases"]:
        r = oracle.peel_batch(g, case["k"], tuple(case["eps"]), flags=case_flags(case) | oracle.FLAG_RECOMPUTE_F)
        assert r.violations == 0
        assert list(r.peel_round) == case["peel_round"], case
        assert r.trace_f == [x * Q for x in case["trace_f"]]
        assert list(r.trace_size) == case["trace_size"]
        assert list(r.trace_peeled) == case["trace_peeled"]
        assert r.best_round == case["best_round"]
        assert r.best_size == case["best_size"]
        assert r.best_f == case["best_f"] * Q
        assert r.n_min_rule == case["n_min_rule"]
        if "trace_T" in case:  # the integer threshold and the kind of every round
            assert [int(x) for x in r.trace_T] == case["trace_T"], case
            assert list(r.trace_kind) == case["trace_kind"], case
    if "serial" in G:
        order, step, size, f = oracle.peel_serial(g)
        assert list(order) == G["serial"]["order"]
        assert (step, size, f) == (G["serial"]["best_step"], G["serial"]["best_size"], G["serial"]["best_f"] * Q)


# ------------------------------------------------ brute force and max-flow


def test_brute_force_handmade():
    # triangle plus a pendant: triangle (3/3) ties V (4/4); the first mask wins
    g = graph_from_lists(4, [(0, 1, 1), (1, 2, 1), (0, 2, 1), (0, 3, 1)], metric="dg")
    size, f, mask = oracle.brute_force(g)
    assert (size, f, mask) == (3, 3 * Q, 0b0111)
    # K4: 6 edges / 4 vertices
    k4 = [(u, v, 1) for u in range(4) for v in range(u + 1, 4)]
    size, f, _ = oracle.brute_force(graph_from_lists(4, k4, metric="dg"))
    assert density(f, size * Q) == Fraction(3, 2)
    # weighted path 0-1-2 with c = 1, 3: {1,2} has 3/2 > 4/3
    size, f, mask = oracle.brute_force(graph_from_lists(3, [(0, 1, 1), (1, 2, 3)], metric="dw"))
    assert (size, f, mask) == (2, 3 * Q, 0b110)
    # vertex weights count once: a lone heavy vertex beats a light edge
    size, f, mask = oracle.brute_force(graph_from_lists(3, [(0, 1, 1)], a=[0, 0, 5], metric="dw"))
    assert (size, f, mask) == (1, 5 * Q, 0b100)


@pytest.mark.parametrize("seed", range(12))
def test_exact_flow_equals_brute_force(seed):
    n = 8 + seed % 7
    edges, _ = random_small(n, 0.35, seed, weighted=False, with_a=False)
    if not edges:
        edges = [(0, 1, 1)]
    g = graph_from_lists(n, edges, metric="dg")
    size, f, _ = oracle.brute_force(g)
    ec, sz, mask = oracle.exact_dg(g)
    assert Fraction(ec, sz) == Fraction(f, size * Q)
    # the returned set really has that density
    inside = set(np.nonzero(mask)[0].tolist())
    assert len(inside) == sz
    assert sum(1 for (u, v, _) in edges if u in inside and v in inside) == ec


@pytest.mark.parametrize("q", [3, 5, 9, 16])
def test_exact_flow_closed_forms(q):
    # clique K_q: (q-1)/2
    kq = [(u, v, 1) for u in range(q) for v in range(u + 1, q)]
    ec, sz, _ = oracle.exact_dg(graph_from_lists(q, kq, metric="dg"))
    assert Fraction(ec, sz) == Fraction(q - 1, 2)
    # complete bipartite K_{p,q}: pq/(p+q)
    p = q + 2
    kpq = [(u, p + v, 1) for u in range(p) for v in range(q)]
    ec, sz, _ = oracle.exact_dg(graph_from_lists(p + q, kpq, metric="dg"))
    assert Fraction(ec, sz) == Fraction(p * q, p + q)
    # K_q next to a long path: the clique alone is densest (q >= 5)
    if q >= 5:
        path = [(q + i, q + i + 1, 1) for i in range(30)]
        ec, sz, mask = oracle.exact_dg(graph_from_lists(q + 31, kq + path, metric="dg"))
        assert Fraction(ec, sz) == Fraction(q - 1, 2)
        assert sz == q and mask[:q].all()


# ------------------------------------------------ approximation theorems


@pytest.mark.parametrize("seed", range(10))
def test_serial_peel_two_approximation(seed):
    """Thm 2.1: Algorithm 1 returns g(S) >= g*/2 (DG, DW, FD-type weights)."""
    n = 10 + seed % 6
    edges, a = random_small(n, 0.4, 100 + seed)
    if not edges:
        return
    g = graph_from_lists(n, edges, a, metric="dw")
    bsize, bf, _ = oracle.brute_force(g)
    _, _, size, f = oracle.peel_serial(g)
    assert 2 * density(f, size) >= density(bf, bsize)


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("eps", [(0, 1), (1, 10), (1, 2)])
def test_batch_peel_approximation(seed, k, eps):
    """Thm 4.3: g(S^p) >= g*/(k'(1+eps)) with k' = max(k, 2) (k = 1 via the minimum rule)."""
    n = 10 + seed % 6
    edges, a = random_small(n, 0.45, 200 + seed, with_a=seed % 2 == 0)
    if not edges:
        return
    g = graph_from_lists(n, edges, a, metric="dw")
    bsize, bf, _ = oracle.brute_force(g)
    r = oracle.peel_batch(g, k, eps, flags=oracle.FLAG_RECOMPUTE_F)
    assert r.violations == 0
    kk = max(k, 2)
    bound = density(bf, bsize) / (kk * (1 + Fraction(eps[0], eps[1])))
    assert density(r.best_f, r.best_size) >= bound
    # Lemma 4.2: every round removes at least one vertex; rounds partition V
    assert all(x >= 1 for x in r.trace_peeled[1:])
    assert sum(r.trace_peeled) == n
    assert r.trace_size[-1] == 0 and r.trace_f[-1] == 0
    if k >= 2:
        assert r.n_min_rule == 0  # min w <= avg w <= 2g <= k(1+eps)g


@pytest.mark.parametrize("flags", [oracle.FLAG_GPO, oracle.FLAG_LPO])
@pytest.mark.parametrize("seed", range(6))
def test_gpo_lpo_keep_bound(flags, seed):
    """Algorithms 3 and 4 keep the approximation (Lemma 5.1, Lemma 5.3)."""
    n = 12 + seed % 4
    edges, a = random_small(n, 0.4, 300 + seed)
    if not edges:
        return
    g = graph_from_lists(n, edges, a, metric="dw")
    bsize, bf, _ = oracle.brute_force(g)
    for k in (1, 2):
        r = oracle.peel_batch(g, k, (1, 10), flags=flags | oracle.FLAG_RECOMPUTE_F)
        assert r.violations == 0
        assert density(r.best_f, r.best_size) >= density(bf, bsize) / (2 * Fraction(11, 10))
        assert sum(r.trace_peeled) == n


def test_lpo_trims_below_density():
    """Algorithm 4: after any round, no survivor keeps w_u(S_i) < g(S_i)."""
    # a 6-clique with a pendant path: trims remove the path once the clique dominates
    kq = [(u, v, 1) for u in range(6) for v in range(u + 1, 6)]
    path = [(5, 6, 1), (6, 7, 1), (7, 8, 1)]
    g = graph_from_lists(9, kq + path, metric="dg")
    r = oracle.peel_batch(g, 2, (1, 10), flags=oracle.FLAG_LPO | oracle.FLAG_RECOMPUTE_F)
    assert r.violations == 0
    assert r.best_size == 6 and r.best_f == 15 * Q


@pytest.mark.parametrize("n", [200, 1000, 5000])
def test_lemma_4_1_round_bound(n):
    """k=2, eps>0: |S_i| < |S_{i-1}|/(1+eps), hence R < log_{1+eps}|V| + 1."""
    g0 = synth.random_general(n, 6 * n, seed=n)
    synth.with_weights(g0, "dw", seed=3, a_range=(0, 5))
    g = oracle.Graph.from_synth(g0, "dw")
    for eps in ((1, 10), (1, 2), (1, 1)):
        r = oracle.peel_batch(g, 2, eps)
        e = eps[0] / eps[1]
        assert r.n_rounds < math.log(n) / math.log(1 + e) + 1
        for i in range(1, r.n_rounds + 1):
            assert r.trace_size[i] * (eps[1] + eps[0]) < r.trace_size[i - 1] * eps[1]


# ------------------------------------------------------------ closed forms


@pytest.mark.parametrize("q", [4, 7, 12])
@pytest.mark.parametrize("k", [1, 2])
def test_clique_peels_in_one_round(q, k):
    kq = [(u, v) for u in range(q) for v in range(u + 1, q)]
    g = oracle.Graph(q, [e[0] for e in kq], [e[1] for e in kq], None, None, "dg")
    r = oracle.peel_batch(g, k, (1, 10))
    assert r.n_rounds == 1 and r.best_round == 0 and r.best_size == q
    assert r.best_f == q * (q - 1) // 2 * Q
    assert r.n_min_rule == (1 if k == 1 else 0)  # w = q-1 = 2g > 1.1 g


def test_star_leaves_first():
    q = 10
    g = oracle.Graph(q + 1, [0] * q, list(range(1, q + 1)), None, None, "dg")
    r = oracle.peel_batch(g, 1, (1, 10))
    # g = q/(q+1); T = floor(1.1 q/(q+1)) = 1 >= leaf weight 1 < centre weight q
    assert list(r.peel_round) == [2] + [1] * q
    assert r.best_round == 0
    assert r.trace_size.tolist() == [q + 1, 1, 0]


def test_planted_block_recovered():
    """Config-1 shape: the 200x200 block at p=0.5 (density ~50) stands out of a
    background of density ~8; Algorithm 2 must return about its 400 vertices."""
    g0 = synth.dg_planted_block(seed=1)
    g = oracle.Graph.from_synth(g0, "dg")
    for k in (1, 2):
        r = oracle.peel_batch(g, k, (1, 10))
        assert 300 <= r.best_size <= 450
        assert r.best_density > 40.0


# ------------------------------------------------------------ error paths


def test_errors():
    with pytest.raises(oracle.OracleError) as e:
        oracle.Graph(3, [0], [0], None, None, "dg")  # self-loop
    assert e.value.code == -1
    with pytest.raises(oracle.OracleError):
        oracle.Graph(3, [0, 1], [1, 0], None, None, "dg")  # repeated pair
    with pytest.raises(oracle.OracleError) as e:
        oracle.Graph(3, [0], [1], [-5], None, "dw")  # negative weight (Property 3.1)
    with pytest.raises(oracle.OracleError) as e:
        oracle.Graph(3, [0, 0], [1, 2], [2**62, 2**62], None, "dw")  # w_0 = 2^63
    assert e.value.code == -2
    g = graph_from_lists(6, [(0, 1, 1), (1, 2, 3), (2, 3, 2), (2, 4, 2), (3, 4, 2), (4, 5, 1)])
    with pytest.raises(oracle.OracleError) as e:
        oracle.peel_batch(g, 1, (0, 1), max_rounds=2)
    assert e.value.code == -5


# ------------------------------------------------------------ the verifier


def _verify(g, r, k, eps):
    fh = np.array([x >> 64 for x in r.trace_f], np.int64)
    fl = np.array([x & ((1 << 64) - 1) for x in r.trace_f], np.uint64)
    return oracle.verify(g, k, eps, r.peel_round, r.n_rounds, fh, fl, r.trace_size, r.trace_peeled, r.best_round,
                         nsample=8)


@pytest.mark.parametrize("k", [1, 2])
def test_verifier_accepts_and_rejects(k):
    g0 = synth.random_general(300, 1500, seed=7)
    synth.with_weights(g0, "dw", seed=7, a_range=(0, 3))
    g = oracle.Graph.from_synth(g0, "dw")
    eps = (1, 10)
    r = oracle.peel_batch(g, k, eps)
    assert _verify(g, r, k, eps) == (0, "")
    # planted mistakes: a vertex moved to a later round
    bad = r.peel_round.copy()
    v = int(np.argmin(bad))
    bad[v] = min(bad[v] + 1, r.n_rounds)
    if bad[v] != r.peel_round[v]:
        rb = oracle.PeelResult(**{**r.__dict__, "peel_round": bad})
        assert _verify(g, rb, k, eps)[0] != 0
    # a wrong density in the trace
    tf = list(r.trace_f)
    tf[1] += 1
    assert _verify(g, oracle.PeelResult(**{**r.__dict__, "trace_f": tf}), k, eps)[0] != 0
    # a wrong best round
    rb = oracle.PeelResult(**{**r.__dict__, "best_round": (r.best_round + 1) % max(r.n_rounds, 1)})
    if rb.best_round != r.best_round:
        assert _verify(g, rb, k, eps)[0] != 0
    # a different eps (the run does not follow its threshold)
    assert _verify(g, r, k, (1, 1))[0] != 0 or _verify(g, r, k, (0, 1))[0] != 0
