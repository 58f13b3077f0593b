/*
 * dupin_oracle.c -- the CPU oracle for Dupin's batch peeling.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no code, header, table or
 * helper with the CUDA library: it builds its own adjacency from a plain
 * undirected edge list and runs every step with plain single-threaded loops.
 *
 * What it computes (paper "Dupin", arXiv 2504.09311):
 *   - density g(S) = f(S)/|S| with f(S) = sum_{u in S} a_u + sum_{e in E[S]} c_e
 *     (Sec. 2.1, Eq. 1); metrics DG (a=0, c=1), DW and FD (a, c supplied);
 *   - the peeling weight w_u(S) = decrease of f when u leaves S (Sec. 2.2),
 *     i.e. a_u + sum of c_uv over neighbours v still in S;
 *   - Algorithm 1 (sequential peeling, one argmin vertex per step);
 *   - Algorithm 2 (parallel batch peeling: every live u with
 *     w_u(S_{i-1}) <= k(1+eps) g(S_{i-1}) leaves in round i; the densest S_i
 *     is returned);
 *   - Algorithm 3 (global threshold tau_max) and Algorithm 4 (local trims);
 *   - the same peel for the clique metrics TDS and kCLiDS (Sec. 2.1): f(S)
 *     = number of q-cliques of G[S], w_u(S) = those through u, recomputed
 *     from scratch every round, and their brute-force optimum;
 *   - brute-force densest subgraph (n <= 24) and exact DG densest subgraph
 *     by Goldberg's max-flow construction (cited in Sec. 2.3), the two
 *     independent pins for the approximation theorems (Thm 2.1, Thm 4.3);
 *   - a verifier that checks a peel result (per-vertex rounds, trace, best
 *     prefix) against the definitions in O(|V|+|E|) plus sampled rounds.
 *
 * Weights are Q32.32 int64 (value * 2^32); f, products and comparisons are in
 * __int128 so every comparison is exact.  Readings of points the paper leaves
 * open (listed with the design notes):
 *   - threshold: w <= k(1+eps) f/|S| with eps = N/D rational and w an integer
 *     is w <= floor(k (D+N) f / (D |S|)); saturated to INT64_MAX;
 *   - empty removal set (possible for k = 1): peel every live vertex whose
 *     weight equals the minimum live weight;
 *   - best prefix: candidates S_0 .. S_{R-1}, strict ">" so the earliest round
 *     wins ties (Algorithm 1's update rule);
 *   - Algorithm 4's trims are sub-rounds: each trim step gets its own round
 *     number, trace entry and best-prefix candidacy.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>

typedef __int128 i128;

#define OG_OK 0
#define OG_ERR_ARG -1
#define OG_ERR_OVERFLOW -2
#define OG_ERR_NO_PROGRESS -5
#define OG_ERR_BUFFER -4
#define OG_ERR_OOM -3

#define OG_METRIC_DG 0
#define OG_METRIC_DW 1
#define OG_METRIC_FD 2

#define OG_FLAG_GPO 1u
#define OG_FLAG_LPO 2u
#define OG_FLAG_RECOMPUTE_F 4u /* recompute f(S_i) from scratch every round */

#define Q_ONE ((int64_t)1 << 32)

/* ------------------------------------------------------------------ graph */

typedef struct {
    int64_t n, m;
    int64_t *off; /* n+1 */
    int32_t *nbr; /* 2m  */
    int64_t *cw;  /* 2m  */
    int64_t *a;   /* n   */
} og_graph;

void og_free(og_graph *g) {
    if (!g) return;
    free(g->off);
    free(g->nbr);
    free(g->cw);
    free(g->a);
    free(g);
}

/*
 * Build the oracle's adjacency from an undirected edge list.  Each edge
 * (eu[j], ev[j]) appears in both endpoints' lists with weight c[j].  For DG the
 * supplied weights are ignored (a_u = 0, c_e = 1, Sec. 2.1 "DG").
 * Self-loops and repeated pairs are rejected: E is a set (Sec. 2.1).
 */
og_graph *og_build(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                   const int64_t *c, const int64_t *a, int metric, int *err) {
    *err = OG_OK;
    if (n < 0 || m < 0) { *err = OG_ERR_ARG; return NULL; }
    og_graph *g = (og_graph *)calloc(1, sizeof(og_graph));
    g->n = n;
    g->m = m;
    g->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    g->cw = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * m + 1));
    g->a = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!g->off || !g->nbr || !g->cw || !g->a) { og_free(g); *err = OG_ERR_OOM; return NULL; }
    for (int64_t j = 0; j < m; j++) {
        int64_t u = eu[j], v = ev[j];
        if (u < 0 || u >= n || v < 0 || v >= n || u == v) { og_free(g); *err = OG_ERR_ARG; return NULL; }
        if (metric != OG_METRIC_DG && c[j] < 0) { og_free(g); *err = OG_ERR_ARG; return NULL; }
        g->off[u + 1]++;
        g->off[v + 1]++;
    }
    for (int64_t u = 0; u < n; u++) g->off[u + 1] += g->off[u];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    memcpy(fill, g->off, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t j = 0; j < m; j++) {
        int64_t u = eu[j], v = ev[j];
        int64_t cj = (metric == OG_METRIC_DG) ? Q_ONE : c[j];
        g->nbr[fill[u]] = (int32_t)v; g->cw[fill[u]] = cj; fill[u]++;
        g->nbr[fill[v]] = (int32_t)u; g->cw[fill[v]] = cj; fill[v]++;
    }
    free(fill);
    /* repeated pairs: sort-free check with a marker array */
    int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t u = 0; u < n; u++) mark[u] = -1;
    for (int64_t u = 0; u < n; u++) {
        for (int64_t p = g->off[u]; p < g->off[u + 1]; p++) {
            int32_t v = g->nbr[p];
            if (mark[v] == u) { free(mark); og_free(g); *err = OG_ERR_ARG; return NULL; }
            mark[v] = u;
        }
    }
    free(mark);
    for (int64_t u = 0; u < n; u++) {
        int64_t au = (metric == OG_METRIC_DG || a == NULL) ? 0 : a[u];
        if (au < 0) { og_free(g); *err = OG_ERR_ARG; return NULL; }
        g->a[u] = au;
    }
    /* every initial peeling weight must fit in int64 */
    for (int64_t u = 0; u < n; u++) {
        i128 w = g->a[u];
        for (int64_t p = g->off[u]; p < g->off[u + 1]; p++) w += g->cw[p];
        if (w > (i128)INT64_MAX) { og_free(g); *err = OG_ERR_OVERFLOW; return NULL; }
    }
    return g;
}

int64_t og_n(const og_graph *g) { return g->n; }
int64_t og_m(const og_graph *g) { return g->m; }

/* f(S) from scratch: Eq. 1, each edge of E[S] once (u < v) */
static i128 f_of_set(const og_graph *g, const uint8_t *in) {
    i128 f = 0;
    for (int64_t u = 0; u < g->n; u++) {
        if (!in[u]) continue;
        f += g->a[u];
        for (int64_t p = g->off[u]; p < g->off[u + 1]; p++) {
            int32_t v = g->nbr[p];
            if (v > u && in[v]) f += g->cw[p];
        }
    }
    return f;
}

/* w_u(S) from scratch: a_u + sum of c_uv, v in N(u) and in S (Sec. 2.2) */
static int64_t w_of(const og_graph *g, const uint8_t *in, int64_t u) {
    i128 w = g->a[u];
    for (int64_t p = g->off[u]; p < g->off[u + 1]; p++)
        if (in[g->nbr[p]]) w += g->cw[p];
    return (int64_t)w;
}

/* floor(x / y), x >= 0, y > 0, saturated to INT64_MAX */
static int64_t floor_div_sat(i128 x, i128 y) {
    i128 q = x / y;
    if (q > (i128)INT64_MAX) return INT64_MAX;
    return (int64_t)q;
}

/* largest integer strictly below x / y (x >= 0, y > 0): ceil(x/y) - 1 */
static int64_t below_div_sat(i128 x, i128 y) {
    i128 q = x / y;
    if (q * y == x) q -= 1;
    if (q > (i128)INT64_MAX) return INT64_MAX;
    return (int64_t)q;
}

/* a/b > c/d for non-negative numerators, positive denominators */
static int frac_gt(i128 a, i128 b, i128 c, i128 d) { return a * d > c * b; }

/* --------------------------------------------------------- Algorithm 2 */

/*
 * out[0] = R (rounds, i.e. non-empty removal sets, trims included)
 * out[1] = best round b (S_b = {u : peel_round[u] > b})
 * out[2] = |S_b|
 * out[3], out[4] = f(S_b) high / low 64-bit words
 * out[5] = number of invariant violations seen (must be 0)
 * out[6] = number of rounds where the removal set was empty at the
 *          k(1+eps)g threshold and the minimum-weight rule was used
 * out[7] = sum over rounds of |S_{i-1}| (the live-scan volume)
 *
 * trace arrays (length >= R+1, entry 0 = S_0): f hi/lo, |S_i|, |U_i| (0 for
 * entry 0), the integer threshold used in round i (entry 0 unused), and the
 * kind of round i (0 = k(1+eps)g rule, 1 = minimum rule, 2 = local trim).
 */
int og_peel_batch(const og_graph *g, int32_t k_mult, int64_t eps_num, int64_t eps_den,
                  uint32_t flags, int64_t max_rounds, int32_t *peel_round,
                  int64_t *tr_f_hi, uint64_t *tr_f_lo, int64_t *tr_size, int64_t *tr_peeled,
                  int64_t *tr_T, int32_t *tr_kind, int64_t tr_cap, int64_t *out) {
    const int64_t n = g->n;
    if (k_mult < 1 || eps_num < 0 || eps_den < 1) return OG_ERR_ARG;
    if (max_rounds <= 0) max_rounds = n + 1;
    for (int i = 0; i < 8; i++) out[i] = 0;
    /* Algorithm 4 carries Algorithm 3's global threshold in its first step */
    if (flags & OG_FLAG_LPO) flags |= OG_FLAG_GPO;

    int64_t *w = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    uint8_t *in = (uint8_t *)malloc((size_t)n + 1);     /* u in current S */
    uint8_t *rem = (uint8_t *)calloc((size_t)n + 1, 1); /* u in removal set U */
    int32_t *ulist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    /* the members of the current S as a list: every loop "for u in S_{i-1}"
       of Algorithms 2-4 walks it; it is filtered after each removal */
    int32_t *slist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    if (!w || !in || !rem || !ulist || !slist) {
        free(w); free(in); free(rem); free(ulist); free(slist);
        return OG_ERR_OOM;
    }

    /* S_0 = V; initial peeling weights and f(S_0) */
    for (int64_t u = 0; u < n; u++) { in[u] = 1; peel_round[u] = INT32_MAX; slist[u] = (int32_t)u; }
    int64_t ns = n; /* |S| as the list's length */
    for (int64_t u = 0; u < n; u++) w[u] = w_of(g, in, u);
    i128 f = f_of_set(g, in);
    int64_t size = n;
    int64_t viol = 0, nfallback = 0, scan = 0;

    /* sum over S of (w_u + a_u) = 2 f(S): each edge twice, each a_u twice */
    {
        i128 s = 0;
        for (int64_t u = 0; u < n; u++) s += (i128)w[u] + g->a[u];
        if (s != 2 * f) viol++;
    }

    int64_t R = 0;
    int64_t best_round = 0, best_size = n;
    i128 best_f = f;
    if (tr_cap < 1) { free(w); free(in); free(rem); free(ulist); free(slist); return OG_ERR_BUFFER; }
    tr_f_hi[0] = (int64_t)(f >> 64);
    tr_f_lo[0] = (uint64_t)f;
    tr_size[0] = n;
    tr_peeled[0] = 0;
    tr_T[0] = 0;
    tr_kind[0] = 0;

    /* Algorithm 3's running maximum of g/(k(1+eps)), kept as the two integer
       forms a test needs: floor (for "w <= tau_max") and ceil-1 (for
       "w < tau_max"). Starts at 0 (Algorithm 3 initialises tau_max = 0). */
    int64_t gpo_le = 0, gpo_lt = -1;
    const i128 kD = (i128)k_mult * (eps_den + eps_num); /* k (D+N) */
    int status = OG_OK;
    int overflow_trace = 0;

    while (size > 0) {
        /* ---- one round of Algorithm 2 / 3 ---- */
        if (R + 1 > max_rounds) { status = OG_ERR_NO_PROGRESS; break; }
        scan += size;
        int64_t T = floor_div_sat(kD * f, (i128)eps_den * size);
        if (flags & OG_FLAG_GPO) {
            int64_t le = floor_div_sat((i128)eps_den * f, kD * size);
            int64_t lt = below_div_sat((i128)eps_den * f, kD * size);
            if (le > gpo_le) gpo_le = le;
            if (lt > gpo_lt) gpo_lt = lt;
            if (gpo_le > T) T = gpo_le;
        }
        int64_t nU = 0;
        for (int64_t j = 0; j < ns; j++)
            if (w[slist[j]] <= T) ulist[nU++] = slist[j];
        int kind = 0;
        if (nU == 0) {
            /* minimum-weight rule when the threshold selects nobody */
            int64_t mn = INT64_MAX;
            for (int64_t j = 0; j < ns; j++)
                if (w[slist[j]] < mn) mn = w[slist[j]];
            T = mn;
            for (int64_t j = 0; j < ns; j++)
                if (w[slist[j]] <= T) ulist[nU++] = slist[j];
            kind = 1;
            nfallback++;
        }
        if (nU == 0) { viol++; status = OG_ERR_NO_PROGRESS; break; } /* Lemma 4.2 */

        /* remove U: S_i = S_{i-1} \ U, then neighbour weight updates */
        R++;
        for (int64_t j = 0; j < nU; j++) { rem[ulist[j]] = 1; peel_round[ulist[j]] = (int32_t)R; }
        i128 df = 0;
        for (int64_t j = 0; j < nU; j++) {
            int32_t u = ulist[j];
            df += g->a[u];
            for (int64_t p = g->off[u]; p < g->off[u + 1]; p++) {
                int32_t v = g->nbr[p];
                if (!in[v]) continue;          /* peeled in an earlier round */
                if (rem[v]) {                  /* edge inside U: count once */
                    if (v > u) df += g->cw[p];
                } else {                       /* edge to a survivor */
                    df += g->cw[p];
                    w[v] -= g->cw[p];
                }
            }
        }
        for (int64_t j = 0; j < nU; j++) { in[ulist[j]] = 0; rem[ulist[j]] = 0; }
        {
            int64_t k2 = 0;
            for (int64_t j = 0; j < ns; j++)
                if (in[slist[j]]) slist[k2++] = slist[j];
            ns = k2;
        }
        f -= df;
        size -= nU;
        if (ns != size) viol++;
        if (flags & OG_FLAG_RECOMPUTE_F) {
            i128 f2 = f_of_set(g, in);
            if (f2 != f) viol++;
            i128 s = 0;
            for (int64_t u = 0; u < n; u++)
                if (in[u]) {
                    s += (i128)w[u] + g->a[u];
                    if (w[u] != w_of(g, in, u)) viol++;
                }
            if (s != 2 * f) viol++;
        }
        if (R < tr_cap) {
            tr_f_hi[R] = (int64_t)(f >> 64);
            tr_f_lo[R] = (uint64_t)f;
            tr_size[R] = size;
            tr_peeled[R] = nU;
            tr_T[R] = T;
            tr_kind[R] = kind;
        } else {
            overflow_trace = 1;
        }
        if (size > 0 && frac_gt(f, size, best_f, best_size)) {
            best_f = f; best_size = size; best_round = R;
        }

        /* ---- Algorithm 4: trim while some w_u(S_i) < g(S_i) ---- */
        if (flags & OG_FLAG_LPO) {
            while (size > 0) {
                int64_t below_g = below_div_sat(f, size); /* w < g  <=>  w <= this */
                int any = 0;
                for (int64_t j = 0; j < ns && !any; j++)
                    if (w[slist[j]] <= below_g) any = 1;
                if (!any) break;
                if (R + 1 > max_rounds) { status = OG_ERR_NO_PROGRESS; break; }
                int64_t L = below_g;
                if (gpo_lt > L) L = gpo_lt; /* tau_2 = max(tau_max, g) */
                scan += size;
                nU = 0;
                for (int64_t j = 0; j < ns; j++)
                    if (w[slist[j]] <= L) ulist[nU++] = slist[j];
                R++;
                for (int64_t j = 0; j < nU; j++) { rem[ulist[j]] = 1; peel_round[ulist[j]] = (int32_t)R; }
                df = 0;
                for (int64_t j = 0; j < nU; j++) {
                    int32_t u = ulist[j];
                    df += g->a[u];
                    for (int64_t p = g->off[u]; p < g->off[u + 1]; p++) {
                        int32_t v = g->nbr[p];
                        if (!in[v]) continue;
                        if (rem[v]) {
                            if (v > u) df += g->cw[p];
                        } else {
                            df += g->cw[p];
                            w[v] -= g->cw[p];
                        }
                    }
                }
                for (int64_t j = 0; j < nU; j++) { in[ulist[j]] = 0; rem[ulist[j]] = 0; }
                {
                    int64_t k2 = 0;
                    for (int64_t j = 0; j < ns; j++)
                        if (in[slist[j]]) slist[k2++] = slist[j];
                    ns = k2;
                }
                f -= df;
                size -= nU;
                if (ns != size) viol++;
                if (flags & OG_FLAG_RECOMPUTE_F) {
                    if (f_of_set(g, in) != f) viol++;
                }
                if (R < tr_cap) {
                    tr_f_hi[R] = (int64_t)(f >> 64);
                    tr_f_lo[R] = (uint64_t)f;
                    tr_size[R] = size;
                    tr_peeled[R] = nU;
                    tr_T[R] = L;
                    tr_kind[R] = 2;
                } else {
                    overflow_trace = 1;
                }
                if (size > 0 && frac_gt(f, size, best_f, best_size)) {
                    best_f = f; best_size = size; best_round = R;
                }
            }
            if (status != OG_OK) break;
        }
    }
    if (status == OG_OK && f != 0) viol++; /* f(empty set) = 0 */

    out[0] = R;
    out[1] = best_round;
    out[2] = best_size;
    out[3] = (int64_t)(best_f >> 64);
    out[4] = (int64_t)(uint64_t)best_f;
    out[5] = viol;
    out[6] = nfallback;
    out[7] = scan;
    free(w); free(in); free(rem); free(ulist); free(slist);
    if (status == OG_OK && overflow_trace) return OG_ERR_BUFFER;
    return status;
}

/* ------------------------------------------ clique metrics (TDS, kCLiDS) */

/*
 * TDS and kCLiDS (Sec. 2.1): f(S) is the number of q-cliques of G[S] (q = 3
 * for TDS), which Eq. 1 expresses with c = 0 and a_u = (q-cliques through
 * u)/q.  The peeling weight w_u(S) is the number of q-cliques of G[S] that
 * contain u -- the decrease of f when u leaves S -- so the weights of S sum
 * to q f(S).  Weights and f are plain clique counts here: every test the
 * peel makes compares ratios of integers, which a common scale does not
 * change.  Algorithm 2 recomputes the weights of the remaining set every
 * round (Sec. 4.1); so does this routine, by listing the cliques of G[S]
 * from scratch, which is slow and plainly follows the definition.
 */

/* each vertex's neighbours in increasing order (a copy of g->nbr) */
static int32_t *sorted_nbrs(const og_graph *g) {
    int32_t *s = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * g->m + 1));
    if (!s) return NULL;
    for (int64_t u = 0; u < g->n; u++) {
        int64_t b = g->off[u], e = g->off[u + 1];
        for (int64_t p = b; p < e; p++) s[p] = g->nbr[p];
        for (int64_t p = b + 1; p < e; p++) { /* insertion sort: lists are short in tests */
            int32_t x = s[p];
            int64_t q = p - 1;
            while (q >= b && s[q] > x) { s[q + 1] = s[q]; q--; }
            s[q + 1] = x;
        }
    }
    return s;
}

/* is v a neighbour of u (binary search in u's sorted list) */
static int adjacent(const og_graph *g, const int32_t *srt, int32_t u, int32_t v) {
    int64_t lo = g->off[u], hi = g->off[u + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (srt[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo < g->off[u + 1] && srt[lo] == v;
}

typedef struct {
    const og_graph *g;
    const int32_t *srt;
    int q;
    int32_t *chosen;  /* q vertices, increasing */
    int32_t **level;  /* candidate lists per depth, each maxdeg long */
    int64_t *w;       /* cliques through each vertex */
    i128 count;       /* cliques listed */
} clique_walk;

/* extend the chosen vertices chosen[0..depth) by every candidate in turn;
   cand holds the vertices after chosen[depth-1] that are adjacent to all of
   them and in S, in increasing order */
static void clique_extend(clique_walk *c, int depth, const int32_t *cand, int64_t nc) {
    if (depth == c->q) {
        c->count++;
        for (int j = 0; j < c->q; j++) c->w[c->chosen[j]]++;
        return;
    }
    int32_t *next = c->level[depth];
    for (int64_t i = 0; i < nc; i++) {
        int32_t v = cand[i];
        c->chosen[depth] = v;
        int64_t nn = 0;
        if (depth + 1 < c->q)
            for (int64_t j = i + 1; j < nc; j++)
                if (adjacent(c->g, c->srt, v, cand[j])) next[nn++] = cand[j];
        clique_extend(c, depth + 1, next, nn);
    }
}

/* w_u(S) for every u (0 outside S) and f(S), by listing the q-cliques of G[S] */
static i128 clique_weights(const og_graph *g, const int32_t *srt, const uint8_t *in, int q, int64_t *w,
                           int32_t *chosen, int32_t **level) {
    clique_walk c = {g, srt, q, chosen, level, w, 0};
    for (int64_t u = 0; u < g->n; u++) w[u] = 0;
    for (int64_t u = 0; u < g->n; u++) {
        if (!in[u]) continue;
        int64_t nc = 0;
        for (int64_t p = g->off[u]; p < g->off[u + 1]; p++)
            if (srt[p] > u && in[srt[p]]) level[0][nc++] = srt[p];
        chosen[0] = (int32_t)u;
        clique_extend(&c, 1, level[0], nc);
    }
    return c.count;
}

/*
 * Algorithm 2 (and 3 / 4 by flag, as og_peel_batch) for the q-clique
 * metrics, q >= 2 (q = 2 is DG with unscaled counts).  Same outputs as
 * og_peel_batch; trace f is the clique count; out[5] counts rounds where
 * the weights did not sum to q f.
 */
int og_peel_clique(const og_graph *g, int32_t q, int32_t k_mult, int64_t eps_num, int64_t eps_den,
                   uint32_t flags, int64_t max_rounds, int32_t *peel_round,
                   int64_t *tr_f_hi, uint64_t *tr_f_lo, int64_t *tr_size, int64_t *tr_peeled,
                   int64_t *tr_T, int32_t *tr_kind, int64_t tr_cap, int64_t *out) {
    const int64_t n = g->n;
    if (q < 2 || q > 16 || k_mult < 1 || eps_num < 0 || eps_den < 1) return OG_ERR_ARG;
    if (max_rounds <= 0) max_rounds = n + 1;
    for (int i = 0; i < 8; i++) out[i] = 0;
    if (flags & OG_FLAG_LPO) flags |= OG_FLAG_GPO;
    if (tr_cap < 1) return OG_ERR_BUFFER;

    int64_t maxdeg = 1;
    for (int64_t u = 0; u < n; u++)
        if (g->off[u + 1] - g->off[u] > maxdeg) maxdeg = g->off[u + 1] - g->off[u];
    int64_t *w = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    uint8_t *in = (uint8_t *)malloc((size_t)n + 1);
    int32_t *ulist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t *chosen = (int32_t *)malloc(sizeof(int32_t) * (size_t)q);
    int32_t **level = (int32_t **)calloc((size_t)q, sizeof(int32_t *));
    int32_t *srt = sorted_nbrs(g);
    int ok = w && in && ulist && chosen && level && srt;
    for (int d = 0; ok && d < q; d++) ok = (level[d] = (int32_t *)malloc(sizeof(int32_t) * (size_t)maxdeg)) != NULL;
    if (!ok) {
        if (level) for (int d = 0; d < q; d++) free(level[d]);
        free(w); free(in); free(ulist); free(chosen); free(level); free(srt);
        return OG_ERR_OOM;
    }

    for (int64_t u = 0; u < n; u++) { in[u] = 1; peel_round[u] = INT32_MAX; }
    i128 f = clique_weights(g, srt, in, q, w, chosen, level);
    int64_t size = n, viol = 0, nfallback = 0, scan = 0, R = 0;
    int64_t best_round = 0, best_size = n;
    i128 best_f = f;
    tr_f_hi[0] = (int64_t)(f >> 64);
    tr_f_lo[0] = (uint64_t)f;
    tr_size[0] = n;
    tr_peeled[0] = 0;
    tr_T[0] = 0;
    tr_kind[0] = 0;
    int64_t gpo_le = 0, gpo_lt = -1;
    const i128 kD = (i128)k_mult * (eps_den + eps_num);
    int status = OG_OK, overflow_trace = 0;

    /* remove ulist[0..nU) as round R+1 of the given kind, then recompute the
       weights and f of the remaining set from scratch */
#define CLIQUE_ROUND(TVAL, KIND)                                                       \
    do {                                                                               \
        R++;                                                                           \
        for (int64_t j = 0; j < nU; j++) { in[ulist[j]] = 0; peel_round[ulist[j]] = (int32_t)R; } \
        size -= nU;                                                                    \
        f = clique_weights(g, srt, in, q, w, chosen, level);                           \
        i128 s_ = 0;                                                                   \
        for (int64_t u = 0; u < n; u++) if (in[u]) s_ += w[u];                         \
        if (s_ != (i128)q * f) viol++;                                                 \
        if (R < tr_cap) {                                                              \
            tr_f_hi[R] = (int64_t)(f >> 64); tr_f_lo[R] = (uint64_t)f;                 \
            tr_size[R] = size; tr_peeled[R] = nU; tr_T[R] = (TVAL); tr_kind[R] = (KIND); \
        } else {                                                                       \
            overflow_trace = 1;                                                        \
        }                                                                              \
        if (size > 0 && frac_gt(f, size, best_f, best_size)) {                         \
            best_f = f; best_size = size; best_round = R;                              \
        }                                                                              \
    } while (0)

    {
        i128 s = 0;
        for (int64_t u = 0; u < n; u++) s += w[u];
        if (s != (i128)q * f) viol++;
    }
    while (size > 0) {
        if (R + 1 > max_rounds) { status = OG_ERR_NO_PROGRESS; break; }
        scan += size;
        int64_t T = floor_div_sat(kD * f, (i128)eps_den * size);
        if (flags & OG_FLAG_GPO) {
            int64_t le = floor_div_sat((i128)eps_den * f, kD * size);
            int64_t lt = below_div_sat((i128)eps_den * f, kD * size);
            if (le > gpo_le) gpo_le = le;
            if (lt > gpo_lt) gpo_lt = lt;
            if (gpo_le > T) T = gpo_le;
        }
        int64_t nU = 0;
        for (int64_t u = 0; u < n; u++)
            if (in[u] && w[u] <= T) ulist[nU++] = (int32_t)u;
        int kind = 0;
        if (nU == 0) { /* minimum-weight rule, as for the other metrics */
            int64_t mn = INT64_MAX;
            for (int64_t u = 0; u < n; u++)
                if (in[u] && w[u] < mn) mn = w[u];
            T = mn;
            for (int64_t u = 0; u < n; u++)
                if (in[u] && w[u] <= T) ulist[nU++] = (int32_t)u;
            kind = 1;
            nfallback++;
        }
        if (nU == 0) { viol++; status = OG_ERR_NO_PROGRESS; break; }
        CLIQUE_ROUND(T, kind);
        if (flags & OG_FLAG_LPO) {
            while (size > 0) {
                int64_t below_g = below_div_sat(f, size);
                int any = 0;
                for (int64_t u = 0; u < n && !any; u++)
                    if (in[u] && w[u] <= below_g) any = 1;
                if (!any) break;
                if (R + 1 > max_rounds) { status = OG_ERR_NO_PROGRESS; break; }
                int64_t L = below_g > gpo_lt ? below_g : gpo_lt;
                scan += size;
                nU = 0;
                for (int64_t u = 0; u < n; u++)
                    if (in[u] && w[u] <= L) ulist[nU++] = (int32_t)u;
                CLIQUE_ROUND(L, 2);
            }
            if (status != OG_OK) break;
        }
    }
#undef CLIQUE_ROUND
    if (status == OG_OK && f != 0) viol++;
    out[0] = R;
    out[1] = best_round;
    out[2] = best_size;
    out[3] = (int64_t)(best_f >> 64);
    out[4] = (int64_t)(uint64_t)best_f;
    out[5] = viol;
    out[6] = nfallback;
    out[7] = scan;
    for (int d = 0; d < q; d++) free(level[d]);
    free(w); free(in); free(ulist); free(chosen); free(level); free(srt);
    if (status == OG_OK && overflow_trace) return OG_ERR_BUFFER;
    return status;
}

/*
 * max over non-empty S of (q-cliques of G[S]) / |S| by enumerating all
 * 2^n - 1 subsets (n <= 20): the graph's cliques are listed once as vertex
 * masks, and a subset counts those inside it.  Ties keep the first mask.
 * out[0] = |S*|, out[1] = cliques in S*, out[2] = the mask of S*.
 */
int og_brute_force_clique(const og_graph *g, int32_t q, int64_t *out) {
    const int64_t n = g->n;
    if (n < 1 || n > 20 || q < 2 || q > 16) return OG_ERR_ARG;
    /* list the cliques: choose q vertices in increasing order, all pairs adjacent */
    int64_t cap = 1024, nk = 0;
    uint32_t *km = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)cap);
    int32_t *srt = sorted_nbrs(g);
    if (!km || !srt) { free(km); free(srt); return OG_ERR_OOM; }
    for (uint32_t mask = 1; mask < (1u << n); mask++) {
        if (__builtin_popcount(mask) != q) continue;
        int clique = 1;
        for (int64_t u = 0; u < n && clique; u++) {
            if (!((mask >> u) & 1)) continue;
            for (int64_t v = u + 1; v < n && clique; v++)
                if (((mask >> v) & 1) && !adjacent(g, srt, (int32_t)u, (int32_t)v)) clique = 0;
        }
        if (!clique) continue;
        if (nk == cap) {
            cap *= 2;
            uint32_t *t = (uint32_t *)realloc(km, sizeof(uint32_t) * (size_t)cap);
            if (!t) { free(km); free(srt); return OG_ERR_OOM; }
            km = t;
        }
        km[nk++] = mask;
    }
    int64_t bc = -1, bs = 1, bm = 0;
    for (uint32_t mask = 1; mask < (1u << n); mask++) {
        int64_t c = 0;
        for (int64_t j = 0; j < nk; j++) c += (km[j] & mask) == km[j];
        int64_t s = __builtin_popcount(mask);
        if (bc < 0 || frac_gt(c, s, bc, bs)) { bc = c; bs = s; bm = mask; }
    }
    out[0] = bs;
    out[1] = bc;
    out[2] = bm;
    free(km);
    free(srt);
    return OG_OK;
}

/* --------------------------------------------------------- Algorithm 1 */

/* binary min-heap of (w, id) pairs; stale entries are skipped on pop */
typedef struct { int64_t w; int32_t id; } hent;

static int hless(hent x, hent y) { return x.w < y.w || (x.w == y.w && x.id < y.id); }

static void hpush(hent *h, int64_t *sz, hent e) {
    int64_t i = (*sz)++;
    h[i] = e;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!hless(h[i], h[p])) break;
        hent t = h[i]; h[i] = h[p]; h[p] = t;
        i = p;
    }
}

static hent hpop(hent *h, int64_t *sz) {
    hent top = h[0];
    h[0] = h[--(*sz)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < *sz && hless(h[l], h[s])) s = l;
        if (r < *sz && hless(h[r], h[s])) s = r;
        if (s == i) break;
        hent t = h[i]; h[i] = h[s]; h[s] = t;
        i = s;
    }
    return top;
}

/*
 * Algorithm 1: repeatedly peel the live vertex of minimum peeling weight
 * (smallest id on ties), keep the densest prefix (strict ">", S_0 first).
 * order[i] = the vertex peeled in step i+1.
 * out[0] = best step b (S_b = V minus order[0..b-1]), out[1] = |S_b|,
 * out[2], out[3] = f(S_b) high/low words.
 */
int og_peel_serial(const og_graph *g, int32_t *order, int64_t *out) {
    const int64_t n = g->n;
    int64_t *w = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    uint8_t *in = (uint8_t *)malloc((size_t)n + 1);
    int64_t cap = n + 2 * g->m + 1, hs = 0;
    hent *h = (hent *)malloc(sizeof(hent) * (size_t)cap);
    if (!w || !in || !h) { free(w); free(in); free(h); return OG_ERR_OOM; }
    for (int64_t u = 0; u < n; u++) in[u] = 1;
    for (int64_t u = 0; u < n; u++) { w[u] = w_of(g, in, u); hpush(h, &hs, (hent){w[u], (int32_t)u}); }
    i128 f = f_of_set(g, in);
    int64_t size = n, best_step = 0, best_size = n;
    i128 best_f = f;
    for (int64_t step = 1; step <= n; step++) {
        hent e;
        do { e = hpop(h, &hs); } while (!in[e.id] || e.w != w[e.id]);
        int32_t u = e.id;
        order[step - 1] = u;
        in[u] = 0;
        f -= w[u]; /* w_u(S) is exactly the decrease of f */
        size--;
        for (int64_t p = g->off[u]; p < g->off[u + 1]; p++) {
            int32_t v = g->nbr[p];
            if (!in[v]) continue;
            w[v] -= g->cw[p];
            hpush(h, &hs, (hent){w[v], v});
        }
        if (size > 0 && frac_gt(f, size, best_f, best_size)) {
            best_f = f; best_size = size; best_step = step;
        }
    }
    out[0] = best_step;
    out[1] = best_size;
    out[2] = (int64_t)(best_f >> 64);
    out[3] = (int64_t)(uint64_t)best_f;
    free(w); free(in); free(h);
    return OG_OK;
}

/* ------------------------------------------------ brute force (n <= 24) */

/*
 * max over non-empty S of f(S)/|S| by enumerating all 2^n - 1 subsets; ties
 * keep the first mask in increasing order.  out[0] = |S*|, out[1], out[2] =
 * f(S*) high/low words, out[3] = the mask of S*.
 */
int og_brute_force(const og_graph *g, int64_t *out) {
    const int64_t n = g->n;
    if (n < 1 || n > 24) return OG_ERR_ARG;
    i128 bf = -1;
    int64_t bs = 1, bm = 0;
    for (int64_t mask = 1; mask < ((int64_t)1 << n); mask++) {
        i128 f = 0;
        int64_t s = 0;
        for (int64_t u = 0; u < n; u++) {
            if (!((mask >> u) & 1)) continue;
            s++;
            f += g->a[u];
            for (int64_t p = g->off[u]; p < g->off[u + 1]; p++) {
                int32_t v = g->nbr[p];
                if (v > u && ((mask >> v) & 1)) f += g->cw[p];
            }
        }
        if (bf < 0 || frac_gt(f, s, bf, bs)) { bf = f; bs = s; bm = mask; }
    }
    out[0] = bs;
    out[1] = (int64_t)(bf >> 64);
    out[2] = (int64_t)(uint64_t)bf;
    out[3] = bm;
    return OG_OK;
}

/* --------------------------------- exact DG densest subgraph by max flow */

typedef struct { int32_t to; int64_t cap; } farc;

typedef struct {
    int32_t nv;
    int64_t na, cap_arcs;
    int64_t *head; /* nv+1 offsets into arcs, filled after building */
    farc *arcs;
    int64_t *rev;
    int32_t *from;
} fnet;

/* Dinic's algorithm on a static arc list (arcs stored in pairs a, a^1) */
static int64_t dinic(int32_t nv, int64_t na, const int32_t *afrom, int32_t *ato, int64_t *acap,
                     int32_t s, int32_t t) {
    /* bucket arcs by tail */
    int64_t *first = (int64_t *)calloc((size_t)nv + 1, sizeof(int64_t));
    int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)na);
    for (int64_t a = 0; a < na; a++) first[afrom[a] + 1]++;
    for (int32_t v = 0; v < nv; v++) first[v + 1] += first[v];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv);
    for (int32_t v = 0; v < nv; v++) fill[v] = first[v];
    for (int64_t a = 0; a < na; a++) ord[fill[afrom[a]]++] = a;
    int32_t *level = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
    int64_t *it = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv);
    int32_t *stk = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
    int64_t *stkarc = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv);
    int64_t flow = 0;
    for (;;) {
        for (int32_t v = 0; v < nv; v++) level[v] = -1;
        int32_t qh = 0, qt = 0;
        queue[qt++] = s;
        level[s] = 0;
        while (qh < qt) {
            int32_t v = queue[qh++];
            for (int64_t k = first[v]; k < first[v + 1]; k++) {
                int64_t a = ord[k];
                if (acap[a] > 0 && level[ato[a]] < 0) {
                    level[ato[a]] = level[v] + 1;
                    queue[qt++] = ato[a];
                }
            }
        }
        if (level[t] < 0) break;
        for (int32_t v = 0; v < nv; v++) it[v] = first[v];
        /* iterative DFS for blocking flow */
        for (;;) {
            int32_t depth = 0;
            stk[0] = s;
            int found = 0;
            while (depth >= 0) {
                int32_t v = stk[depth];
                if (v == t) { found = 1; break; }
                int advanced = 0;
                while (it[v] < first[v + 1]) {
                    int64_t a = ord[it[v]];
                    int32_t x = ato[a];
                    if (acap[a] > 0 && level[x] == level[v] + 1) {
                        stkarc[depth] = a;
                        stk[++depth] = x;
                        advanced = 1;
                        break;
                    }
                    it[v]++;
                }
                if (!advanced) {
                    level[v] = -1; /* dead end */
                    depth--;
                    if (depth >= 0) it[stk[depth]]++;
                }
            }
            if (!found) break;
            int64_t push = INT64_MAX;
            for (int32_t d = 0; d < depth; d++)
                if (acap[stkarc[d]] < push) push = acap[stkarc[d]];
            for (int32_t d = 0; d < depth; d++) {
                acap[stkarc[d]] -= push;
                acap[stkarc[d] ^ 1] += push;
            }
            flow += push;
        }
    }
    free(first); free(ord); free(fill); free(level); free(queue); free(it); free(stk); free(stkarc);
    return flow;
}

/*
 * Goldberg's construction for guess g = p/q (DG): source -> v cap q*m,
 * v -> sink cap q*m + 2p - q*deg(v), each edge both ways cap q.  The min cut
 * equals q*m*n + 2 * min_S (p|S| - q|E[S]|); the source side of a min cut
 * is a minimiser S.  Returns min_S (p|S| - q|E[S]|) and that S in 'side'.
 */
static i128 goldberg_cut(const og_graph *g, int64_t p, int64_t q, uint8_t *side) {
    const int64_t n = g->n, m = g->m;
    int32_t nv = (int32_t)(n + 2), s = (int32_t)n, t = (int32_t)(n + 1);
    int64_t na = 2 * (2 * n + 2 * m);
    int32_t *afrom = (int32_t *)malloc(sizeof(int32_t) * (size_t)na);
    int32_t *ato = (int32_t *)malloc(sizeof(int32_t) * (size_t)na);
    int64_t *acap = (int64_t *)malloc(sizeof(int64_t) * (size_t)na);
    int64_t k = 0;
#define ADD_ARC(x, y, cp) do { afrom[k] = (x); ato[k] = (y); acap[k] = (cp); k++; \
                               afrom[k] = (y); ato[k] = (x); acap[k] = 0; k++; } while (0)
    for (int64_t v = 0; v < n; v++) {
        int64_t deg = g->off[v + 1] - g->off[v];
        ADD_ARC(s, (int32_t)v, q * m);
        ADD_ARC((int32_t)v, t, q * m + 2 * p - q * deg);
    }
    for (int64_t u = 0; u < n; u++)
        for (int64_t pp = g->off[u]; pp < g->off[u + 1]; pp++) {
            int32_t v = g->nbr[pp];
            if (v > u) {
                /* undirected unit edge: one arc each way, each with capacity q */
                afrom[k] = (int32_t)u; ato[k] = v; acap[k] = q; k++;
                afrom[k] = v; ato[k] = (int32_t)u; acap[k] = q; k++;
            }
        }
#undef ADD_ARC
    int64_t flow = dinic(nv, k, afrom, ato, acap, s, t);
    /* residual reachability from s gives the source side */
    int64_t *first = (int64_t *)calloc((size_t)nv + 1, sizeof(int64_t));
    int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    for (int64_t a = 0; a < k; a++) first[afrom[a] + 1]++;
    for (int32_t v = 0; v < nv; v++) first[v + 1] += first[v];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv);
    for (int32_t v = 0; v < nv; v++) fill[v] = first[v];
    for (int64_t a = 0; a < k; a++) ord[fill[afrom[a]]++] = a;
    uint8_t *seen = (uint8_t *)calloc((size_t)nv, 1);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
    int32_t qh = 0, qt = 0;
    queue[qt++] = s;
    seen[s] = 1;
    while (qh < qt) {
        int32_t v = queue[qh++];
        for (int64_t j = first[v]; j < first[v + 1]; j++) {
            int64_t a = ord[j];
            if (acap[a] > 0 && !seen[ato[a]]) { seen[ato[a]] = 1; queue[qt++] = ato[a]; }
        }
    }
    for (int64_t v = 0; v < n; v++) side[v] = seen[v];
    free(first); free(ord); free(fill); free(seen); free(queue);
    free(afrom); free(ato); free(acap);
    /* flow = min cut = q m n + 2 min_S(...) */
    i128 val = ((i128)flow - (i128)q * m * n);
    return val / 2;
}

/*
 * Exact DG densest subgraph (max |E[S]|/|S|): start from g = density(V) and
 * repeatedly replace g by the density of the minimiser S of p|S| - q|E[S]|
 * while that minimum is negative (each step strictly increases g).
 * out[0] = |E[S*]|, out[1] = |S*|; mask[v] = 1 for v in S*.
 */
int og_exact_dg(const og_graph *g, int64_t *out, uint8_t *mask) {
    const int64_t n = g->n, m = g->m;
    if (n < 1) return OG_ERR_ARG;
    int64_t p = m, q = n; /* density of V */
    for (int64_t v = 0; v < n; v++) mask[v] = 1;
    uint8_t *side = (uint8_t *)malloc((size_t)n);
    for (int iter = 0; iter < 10000; iter++) {
        i128 mn = goldberg_cut(g, p, q, side);
        if (mn >= 0) break;
        int64_t sz = 0, ec = 0;
        for (int64_t u = 0; u < n; u++) {
            if (!side[u]) continue;
            sz++;
            for (int64_t pp = g->off[u]; pp < g->off[u + 1]; pp++)
                if (g->nbr[pp] > u && side[g->nbr[pp]]) ec++;
        }
        if (sz == 0) break;
        p = ec;
        q = sz;
        for (int64_t v = 0; v < n; v++) mask[v] = side[v];
    }
    free(side);
    out[0] = p;
    out[1] = q;
    return OG_OK;
}

/* ------------------------------------------------------------ verifier */

/* small deterministic generator for picking sample rounds (splitmix64) */
static uint64_t v_mix(uint64_t *s) {
    uint64_t z = (*s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

/*
 * Check a plain Algorithm 2 result (no GPO/LPO) against the definitions
 * without replaying the whole run:
 *   (1) every vertex has a round in [1, R] and every round is non-empty;
 *   (2) f(S_i), |S_i| and |U_i| recomputed from peel_round equal the trace;
 *   (3) each u peeled in round i had w_u(S_{i-1}) <= T_i, where T_i is
 *       recomputed from the trace (k(1+eps)g rule) or equals the minimum
 *       live weight (minimum rule; then every vertex at the minimum left);
 *   (4) at 'nsample' sampled rounds plus the first and the last two, every
 *       survivor had w_u(S_{i-1}) > T_i (and, for the minimum rule, no live
 *       vertex was below the minimum);
 *   (5) the reported best round is the earliest argmax of f_i/|S_i|.
 * Returns 0 when every check holds, else a positive code; msg explains.
 */
int og_verify(const og_graph *g, int32_t k_mult, int64_t eps_num, int64_t eps_den,
              const int32_t *peel_round, int64_t R, const int64_t *tr_f_hi, const uint64_t *tr_f_lo,
              const int64_t *tr_size, const int64_t *tr_peeled, int64_t best_round, int64_t nsample,
              uint64_t seed, char *msg, int64_t msg_cap) {
    const int64_t n = g->n;
#define FAIL(code, ...) do { if (msg && msg_cap > 0) snprintf(msg, (size_t)msg_cap, __VA_ARGS__); rc = (code); goto done; } while (0)
    int rc = 0;
    i128 *fdel = (i128 *)calloc((size_t)R + 2, sizeof(i128));
    int64_t *cnt = (int64_t *)calloc((size_t)R + 2, sizeof(int64_t));
    i128 *fr = (i128 *)calloc((size_t)R + 2, sizeof(i128));
    int64_t *T = (int64_t *)calloc((size_t)R + 2, sizeof(int64_t));
    uint8_t *ismin = (uint8_t *)calloc((size_t)R + 2, 1);
    int64_t *minw = (int64_t *)malloc(sizeof(int64_t) * (size_t)(R + 2));
    for (int64_t i = 0; i <= R + 1; i++) minw[i] = INT64_MAX;
    uint8_t *in = NULL;
    const i128 kD = (i128)k_mult * (eps_den + eps_num);
    i128 f0 = 0;
    for (int64_t u = 0; u < n; u++) {
        int32_t r = peel_round[u];
        if (r < 1 || r > R) FAIL(1, "vertex %lld has round %d outside [1,%lld]", (long long)u, r, (long long)R);
        cnt[r]++;
        fdel[r] += g->a[u];
        f0 += g->a[u];
        for (int64_t p = g->off[u]; p < g->off[u + 1]; p++) {
            int32_t v = g->nbr[p];
            if (v <= u) continue;
            int32_t r2 = peel_round[v] < r ? peel_round[v] : r;
            if (r2 >= 1 && r2 <= R) fdel[r2] += g->cw[p];
            f0 += g->cw[p];
        }
    }
    fr[0] = f0;
    {
        int64_t sz = n;
        for (int64_t i = 1; i <= R; i++) {
            if (cnt[i] == 0) FAIL(2, "round %lld is empty", (long long)i);
            fr[i] = fr[i - 1] - fdel[i];
            sz -= cnt[i];
            i128 ft = ((i128)tr_f_hi[i] << 64) | (i128)tr_f_lo[i];
            if (ft != fr[i]) FAIL(3, "f trace mismatch at round %lld", (long long)i);
            if (tr_size[i] != sz) FAIL(4, "size trace mismatch at round %lld", (long long)i);
            if (tr_peeled[i] != cnt[i]) FAIL(5, "peeled-count mismatch at round %lld", (long long)i);
        }
        i128 ft0 = ((i128)tr_f_hi[0] << 64) | (i128)tr_f_lo[0];
        if (ft0 != fr[0] || tr_size[0] != n) FAIL(3, "trace entry 0 mismatch");
    }
    for (int64_t i = 1; i <= R; i++) {
        int64_t szp = tr_size[i - 1];
        T[i] = floor_div_sat(kD * fr[i - 1], (i128)eps_den * szp);
    }
    /* (3): peeled vertices' weights at the start of their round */
    for (int64_t u = 0; u < n; u++) {
        int32_t r = peel_round[u];
        i128 w = g->a[u];
        for (int64_t p = g->off[u]; p < g->off[u + 1]; p++)
            if (peel_round[g->nbr[p]] >= r) w += g->cw[p];
        if (w > T[r]) {
            ismin[r] = 1; /* only legal under the minimum rule */
        }
        if ((int64_t)w < minw[r]) minw[r] = (int64_t)w;
    }
    for (int64_t u = 0; u < n; u++) {
        int32_t r = peel_round[u];
        if (!ismin[r]) continue;
        i128 w = g->a[u];
        for (int64_t p = g->off[u]; p < g->off[u + 1]; p++)
            if (peel_round[g->nbr[p]] >= r) w += g->cw[p];
        if ((int64_t)w != minw[r])
            FAIL(6, "round %d: vertex %lld above threshold and not at the round's minimum", r, (long long)u);
    }
    /* (4): sampled rounds, full survivor check */
    in = (uint8_t *)malloc((size_t)n + 1);
    {
        uint64_t st = seed;
        int64_t ns = nsample + 3;
        for (int64_t s = 0; s < ns; s++) {
            int64_t i;
            if (s == 0) i = 1;
            else if (s == 1) i = R;
            else if (s == 2) i = R > 1 ? R - 1 : 1;
            else i = 1 + (int64_t)(v_mix(&st) % (uint64_t)R);
            for (int64_t u = 0; u < n; u++) in[u] = peel_round[u] >= i;
            int64_t live_min = INT64_MAX;
            for (int64_t u = 0; u < n; u++) {
                if (!in[u]) continue;
                int64_t w = w_of(g, in, u);
                if (w < live_min) live_min = w;
                if (peel_round[u] > i) {
                    if (!ismin[i] && w <= T[i])
                        FAIL(7, "round %lld: survivor %lld has w <= T", (long long)i, (long long)u);
                    if (ismin[i] && w <= minw[i])
                        FAIL(8, "round %lld: survivor %lld at or below the minimum", (long long)i, (long long)u);
                }
            }
            if (ismin[i] && live_min != minw[i])
                FAIL(9, "round %lld: minimum rule did not take the minimum", (long long)i);
            if (ismin[i] && live_min <= T[i])
                FAIL(10, "round %lld: minimum rule used though the threshold selects", (long long)i);
        }
    }
    /* (5): best round */
    {
        int64_t b = 0;
        for (int64_t i = 1; i < R; i++)
            if (frac_gt(fr[i], tr_size[i], fr[b], tr_size[b])) b = i;
        if (b != best_round) FAIL(11, "best round %lld, expected %lld", (long long)best_round, (long long)b);
    }
done:
    free(fdel); free(cnt); free(fr); free(T); free(ismin); free(minw); free(in);
    return rc;
#undef FAIL
}

/*
 * Check a plain Algorithm 2 result for the q-clique metrics (no GPO/LPO)
 * against the definitions, for graphs too large to replay:
 *   (1) every vertex has a round in [1, R], every round is non-empty, and
 *       |S_i|, |U_i| from peel_round equal the trace;
 *   (2) at 'nsample' sampled rounds plus the first and the last two, the
 *       q-cliques of G[S_{i-1}] are listed afresh: f(S_{i-1}) equals the
 *       trace, every vertex peeled in round i had w_u(S_{i-1}) <= T_i and
 *       every survivor more (T_i from the trace by the k(1+eps)g rule, or
 *       the minimum live weight when the rule selects nobody);
 *   (3) the reported best round is the earliest argmax of f_i/|S_i| over
 *       the trace.
 * Returns 0 when every check holds, else a positive code; msg explains.
 */
int og_verify_clique(const og_graph *g, int32_t q, int32_t k_mult, int64_t eps_num, int64_t eps_den,
                     const int32_t *peel_round, int64_t R, const int64_t *tr_f_hi, const uint64_t *tr_f_lo,
                     const int64_t *tr_size, const int64_t *tr_peeled, int64_t best_round, int64_t nsample,
                     uint64_t seed, char *msg, int64_t msg_cap) {
    const int64_t n = g->n;
#define FAILC(code, ...) do { if (msg && msg_cap > 0) snprintf(msg, (size_t)msg_cap, __VA_ARGS__); rc = (code); goto done; } while (0)
    int rc = 0;
    if (q < 2 || q > 16 || R < 0) return 100;
    int64_t maxdeg = 1;
    for (int64_t u = 0; u < n; u++)
        if (g->off[u + 1] - g->off[u] > maxdeg) maxdeg = g->off[u + 1] - g->off[u];
    int64_t *cnt = (int64_t *)calloc((size_t)R + 2, sizeof(int64_t));
    int64_t *w = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    uint8_t *in = (uint8_t *)malloc((size_t)n + 1);
    int32_t *chosen = (int32_t *)malloc(sizeof(int32_t) * (size_t)q);
    int32_t **level = (int32_t **)calloc((size_t)q, sizeof(int32_t *));
    int32_t *srt = sorted_nbrs(g);
    const i128 kD = (i128)k_mult * (eps_den + eps_num);
    if (!cnt || !w || !in || !chosen || !level || !srt) FAILC(101, "out of memory");
    for (int d = 0; d < q; d++)
        if (!(level[d] = (int32_t *)malloc(sizeof(int32_t) * (size_t)maxdeg))) FAILC(101, "out of memory");
    /* (1) */
    for (int64_t u = 0; u < n; u++) {
        int32_t r = peel_round[u];
        if (r < 1 || r > R) FAILC(1, "vertex %lld has round %d outside [1,%lld]", (long long)u, r, (long long)R);
        cnt[r]++;
    }
    {
        int64_t sz = n;
        if (tr_size[0] != n) FAILC(4, "trace entry 0 size mismatch");
        for (int64_t i = 1; i <= R; i++) {
            if (cnt[i] == 0) FAILC(2, "round %lld is empty", (long long)i);
            sz -= cnt[i];
            if (tr_size[i] != sz) FAILC(4, "size trace mismatch at round %lld", (long long)i);
            if (tr_peeled[i] != cnt[i]) FAILC(5, "peeled-count mismatch at round %lld", (long long)i);
        }
    }
    /* (2) */
    {
        uint64_t st = seed;
        for (int64_t s = 0; s < nsample + 3 && R > 0; s++) {
            int64_t i;
            if (s == 0) i = 1;
            else if (s == 1) i = R;
            else if (s == 2) i = R > 1 ? R - 1 : 1;
            else i = 1 + (int64_t)(v_mix(&st) % (uint64_t)R);
            for (int64_t u = 0; u < n; u++) in[u] = peel_round[u] >= i;
            const i128 f = clique_weights(g, srt, in, q, w, chosen, level);
            const i128 ft = ((i128)tr_f_hi[i - 1] << 64) | (i128)tr_f_lo[i - 1];
            if (f != ft) FAILC(3, "f trace mismatch at round %lld", (long long)(i - 1));
            int64_t T = floor_div_sat(kD * f, (i128)eps_den * tr_size[i - 1]);
            int64_t mn = INT64_MAX;
            int any_le = 0;
            for (int64_t u = 0; u < n; u++) {
                if (!in[u]) continue;
                if (w[u] < mn) mn = w[u];
                if (w[u] <= T) any_le = 1;
            }
            if (!any_le) T = mn; /* the minimum rule */
            for (int64_t u = 0; u < n; u++) {
                if (!in[u]) continue;
                if (peel_round[u] == i && w[u] > T)
                    FAILC(6, "round %lld: vertex %lld peeled above the threshold", (long long)i, (long long)u);
                if (peel_round[u] > i && w[u] <= T)
                    FAILC(7, "round %lld: survivor %lld at or below the threshold", (long long)i, (long long)u);
            }
        }
    }
    /* (3) */
    {
        int64_t b = 0;
        for (int64_t i = 1; i < R; i++) {
            const i128 fi = ((i128)tr_f_hi[i] << 64) | (i128)tr_f_lo[i];
            const i128 fb = ((i128)tr_f_hi[b] << 64) | (i128)tr_f_lo[b];
            if (frac_gt(fi, tr_size[i], fb, tr_size[b])) b = i;
        }
        if (b != best_round) FAILC(11, "best round %lld, expected %lld", (long long)best_round, (long long)b);
    }
done:
    if (level) for (int d = 0; d < q; d++) free(level[d]);
    free(cnt); free(w); free(in); free(chosen); free(level); free(srt);
    return rc;
#undef FAILC
}
