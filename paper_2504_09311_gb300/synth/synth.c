/*
 * synth.c -- seeded synthetic graph inputs for the peeling library.
 *
 * This module only produces inputs: edge lists, Q32.32 weights and CSR/CSC
 * layouts.  It holds none of the peeling method's arithmetic and is the one
 * module that both the CUDA path's tests and the CPU oracle draw inputs from.
 *
 * Everything is a pure function of (parameters, seed) and bit-identical on
 * x86-64 and AArch64: random numbers come from a counter-based splitmix64
 * (Steele, Lea & Flood, 2014) indexed by (stream, counter); the only floating
 * point is IEEE add/sub/mul/div (compiled with -ffp-contract=off) and this
 * file's own series for ln and exp, so no libm routine can differ between
 * machines.  Threads split index ranges; results do not depend on the split.
 *
 * Workload shapes (the paper's transaction graphs and skewed social graphs):
 *   - bipartite users x items, uniform pairs plus a planted dense block;
 *   - bipartite users x items with Zipf item popularity, camouflaged dense
 *     blocks (Fraudar's setting);
 *   - R-MAT (Chakrabarti, Zhan & Faloutsos, 2004) undirected graphs;
 *   - plain uniform random graphs for small tests.
 * Weights: FD edge weight 1/ln(x + 5) with x the object vertex's degree
 * (Sec. 2.1, Fraudar), uniform integer edge/vertex weights for DW; all Q32.32.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------ randomness */

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

/* the i-th value of stream 'stream' under 'seed' */
static inline uint64_t rnd(uint64_t seed, uint64_t stream, uint64_t i) {
    uint64_t base = mix64(seed * 0x9e3779b97f4a7c15ull + mix64(stream + 0x632be59bd9b4e019ull));
    return mix64(base + (i + 1) * 0x9e3779b97f4a7c15ull);
}

/* uniform double in [0, 1) with 53 random bits */
static inline double unif(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [0, k) (k < 2^32) by multiply-shift on 32 random bits */
static inline uint64_t below(uint64_t r, uint64_t k) { return ((r >> 32) * k) >> 32; }

/* uniform integer in [0, k) for any k < 2^63, by 128-bit multiply-shift */
static inline uint64_t below64(uint64_t r, uint64_t k) {
    return (uint64_t)(((unsigned __int128)r * k) >> 64);
}

/* ----------------------------------------------- deterministic ln / exp */

static const double LN2 = 0.6931471805599453094;

/* ln x for finite x > 0: x = m 2^e with m in [sqrt(1/2), sqrt(2)),
   ln m = 2 atanh((m-1)/(m+1)) summed as an odd power series. */
double sg_ln(double x) {
    int e;
    double m = frexp(x, &e);
    if (m < 0.70710678118654752440) { m *= 2.0; e -= 1; }
    double s = (m - 1.0) / (m + 1.0);
    double s2 = s * s;
    double terms[16];
    double t = s;
    for (int k = 0; k < 16; k++) { terms[k] = t / (double)(2 * k + 1); t *= s2; }
    double sum = 0.0;
    for (int k = 15; k >= 0; k--) sum += terms[k]; /* smallest first */
    return 2.0 * sum + (double)e * LN2;
}

/* e^y for |y| < 700: y = k ln2 + r, |r| <= ln2/2, Taylor series for e^r */
double sg_exp(double y) {
    double kf = y / LN2;
    long k = (long)(kf < 0 ? kf - 0.5 : kf + 0.5);
    double r = y - (double)k * LN2;
    double term = 1.0, sum = 1.0;
    for (int j = 1; j < 24; j++) { term = term * r / (double)j; sum += term; }
    return ldexp(sum, (int)k);
}

/* Q32.32 of a non-negative double: round(v * 2^32), halves away from zero */
static inline int64_t q32(double v) { return llround(ldexp(v, 32)); }

/* --------------------------------------------------------------- threads */

typedef struct {
    void (*fn)(void *ctx, int64_t lo, int64_t hi, int tid);
    void *ctx;
    int64_t lo, hi;
    int tid;
} pf_job;

static void *pf_run(void *p) {
    pf_job *j = (pf_job *)p;
    j->fn(j->ctx, j->lo, j->hi, j->tid);
    return NULL;
}

static int g_threads = 0;

static int nthreads(void) {
    if (g_threads > 0) return g_threads;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    if (c < 1) c = 1;
    if (c > 32) c = 32;
    return (int)c;
}

void sg_set_threads(int t) { g_threads = t; }

/* run fn over [0, n) split into nt contiguous chunks */
static void parallel_for(int64_t n, int nt, void (*fn)(void *, int64_t, int64_t, int), void *ctx) {
    if (nt < 1) nt = 1;
    if (n < 4096 || nt == 1) { fn(ctx, 0, n, 0); return; }
    pthread_t th[64];
    pf_job jobs[64];
    for (int t = 0; t < nt; t++) {
        jobs[t].fn = fn;
        jobs[t].ctx = ctx;
        jobs[t].lo = n * t / nt;
        jobs[t].hi = n * (t + 1) / nt;
        jobs[t].tid = t;
        pthread_create(&th[t], NULL, pf_run, &jobs[t]);
    }
    for (int t = 0; t < nt; t++) pthread_join(th[t], NULL);
}

/* ------------------------------------------- LSD radix sort (key, value) */

typedef struct {
    const uint64_t *kin;
    uint64_t *kout;
    const uint32_t *vin;
    uint32_t *vout;
    int64_t n;
    int shift;
    int nt;
    int64_t *hist; /* nt * 65536 */
} rs_ctx;

static void rs_hist(void *p, int64_t lo, int64_t hi, int tid) {
    rs_ctx *c = (rs_ctx *)p;
    int64_t *h = c->hist + (int64_t)tid * 65536;
    memset(h, 0, sizeof(int64_t) * 65536);
    for (int64_t i = lo; i < hi; i++) h[(c->kin[i] >> c->shift) & 0xffff]++;
}

static void rs_scatter(void *p, int64_t lo, int64_t hi, int tid) {
    rs_ctx *c = (rs_ctx *)p;
    int64_t *h = c->hist + (int64_t)tid * 65536;
    for (int64_t i = lo; i < hi; i++) {
        uint64_t k = c->kin[i];
        int64_t pos = h[(k >> c->shift) & 0xffff]++;
        c->kout[pos] = k;
        if (c->vin) c->vout[pos] = c->vin[i];
    }
}

/* stable sort of keys (and optional 32-bit values) on the low 'bits' bits */
static void radix_sort(uint64_t *keys, uint32_t *vals, int64_t n, int bits) {
    if (n <= 1) return;
    int nt = nthreads();
    if (n < 65536) nt = 1;
    uint64_t *k2 = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    uint32_t *v2 = vals ? (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n) : NULL;
    int64_t *hist = (int64_t *)malloc(sizeof(int64_t) * 65536 * (size_t)nt);
    uint64_t *src = keys, *dst = k2;
    uint32_t *vs = vals, *vd = v2;
    int passes = (bits + 15) / 16;
    for (int pass = 0; pass < passes; pass++) {
        rs_ctx c = {src, dst, vs, vd, n, pass * 16, nt, hist};
        parallel_for(n, nt, rs_hist, &c);
        /* exclusive prefix in (digit, thread) order keeps the sort stable */
        int64_t run = 0;
        for (int d = 0; d < 65536; d++)
            for (int t = 0; t < nt; t++) {
                int64_t x = hist[(int64_t)t * 65536 + d];
                hist[(int64_t)t * 65536 + d] = run;
                run += x;
            }
        parallel_for(n, nt, rs_scatter, &c);
        uint64_t *tk = src; src = dst; dst = tk;
        uint32_t *tv = vs; vs = vd; vd = tv;
    }
    if (src != keys) {
        memcpy(keys, src, sizeof(uint64_t) * (size_t)n);
        if (vals) memcpy(vals, vs, sizeof(uint32_t) * (size_t)n);
    }
    free(k2);
    free(v2);
    free(hist);
}

/* ------------------------------------------------------------ edge lists */

typedef struct {
    int64_t n_left, n_right, m;
    int32_t *eu, *ev;
} sg_edges;

int64_t sg_n_left(const sg_edges *e) { return e->n_left; }
int64_t sg_n_right(const sg_edges *e) { return e->n_right; }
int64_t sg_m(const sg_edges *e) { return e->m; }
const int32_t *sg_eu(const sg_edges *e) { return e->eu; }
const int32_t *sg_ev(const sg_edges *e) { return e->ev; }

void sg_free(sg_edges *e) {
    if (!e) return;
    free(e->eu);
    free(e->ev);
    free(e);
}

/* sorted unique keys (hi 32 bits = u, lo 32 bits = v) -> edge list */
static sg_edges *edges_from_keys(uint64_t *keys, int64_t n, int64_t nl, int64_t nr) {
    radix_sort(keys, NULL, n, 64);
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++)
        if (i == 0 || keys[i] != keys[i - 1]) keys[m++] = keys[i];
    sg_edges *e = (sg_edges *)calloc(1, sizeof(sg_edges));
    e->n_left = nl;
    e->n_right = nr;
    e->m = m;
    e->eu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    e->ev = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    for (int64_t i = 0; i < m; i++) {
        e->eu[i] = (int32_t)(keys[i] >> 32);
        e->ev[i] = (int32_t)(keys[i] & 0xffffffffu);
    }
    return e;
}

/* seeded permutation of [0, k) by Fisher-Yates */
static int32_t *perm(int64_t k, uint64_t seed, uint64_t stream) {
    int32_t *p = (int32_t *)malloc(sizeof(int32_t) * (size_t)(k + 1));
    for (int64_t i = 0; i < k; i++) p[i] = (int32_t)i;
    for (int64_t i = k - 1; i > 0; i--) {
        int64_t j = (int64_t)below64(rnd(seed, stream, (uint64_t)i), (uint64_t)(i + 1));
        int32_t t = p[i]; p[i] = p[j]; p[j] = t;
    }
    return p;
}

/*
 * Config-1 shape: 'draws' uniform (user, item) pairs, plus a bU x bI block
 * on seeded random users and items with each pair present with probability
 * p; duplicates merged.  Edge (u, i) is stored with u in [0, nU), i in
 * [0, nI).
 */
sg_edges *sg_bipartite_uniform(int64_t nU, int64_t nI, int64_t draws, int64_t bU, int64_t bI,
                               double p, uint64_t seed) {
    int64_t cap = draws + bU * bI;
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(cap + 1));
    int64_t k = 0;
    for (int64_t j = 0; j < draws; j++) {
        uint64_t r = rnd(seed, 1, (uint64_t)j);
        uint64_t u = below(r, (uint64_t)nU);
        uint64_t i = below(r << 32, (uint64_t)nI);
        keys[k++] = (u << 32) | i;
    }
    if (bU > 0 && bI > 0) {
        int32_t *pu = perm(nU, seed, 2), *pi = perm(nI, seed, 3);
        for (int64_t x = 0; x < bU; x++)
            for (int64_t y = 0; y < bI; y++)
                if (unif(rnd(seed, 4, (uint64_t)(x * bI + y))) < p)
                    keys[k++] = ((uint64_t)pu[x] << 32) | (uint64_t)pi[y];
        free(pu);
        free(pi);
    }
    sg_edges *e = edges_from_keys(keys, k, nU, nI);
    free(keys);
    return e;
}

/* ---------------------------------------------------------- Zipf graphs */

typedef struct {
    uint64_t seed, stream;
    int64_t nU, nI;
    const double *cdf;
    const int32_t *rank2item;
    uint64_t *keys;
    uint32_t *idx;
    int64_t base;
} zd_ctx;

/* rank r (0-based) with P(r) proportional to (r+1)^-s, by binary search */
static inline int64_t zipf_rank(const double *cdf, int64_t nI, double u) {
    int64_t lo = 0, hi = nI - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (cdf[mid] > u) hi = mid; else lo = mid + 1;
    }
    return lo;
}

static void zd_fill(void *p, int64_t lo, int64_t hi, int tid) {
    (void)tid;
    zd_ctx *c = (zd_ctx *)p;
    for (int64_t j = lo; j < hi; j++) {
        uint64_t t = (uint64_t)(c->base + j);
        uint64_t r1 = rnd(c->seed, c->stream, 2 * t), r2 = rnd(c->seed, c->stream, 2 * t + 1);
        uint64_t u = below64(r1, (uint64_t)c->nU);
        int64_t rk = zipf_rank(c->cdf, c->nI, unif(r2));
        c->keys[j] = (u << 32) | (uint64_t)(uint32_t)c->rank2item[rk];
        c->idx[j] = (uint32_t)j;
    }
}

/*
 * The first m distinct (user, item) pairs of the draw sequence
 * (user uniform, item of Zipf rank with exponent s over a seeded
 * permutation of items), as a sorted key array.
 */
static uint64_t *zipf_pairs(int64_t nU, int64_t nI, int64_t m, double s, uint64_t seed,
                            uint64_t stream, int64_t *out_m) {
    double *cdf = (double *)malloc(sizeof(double) * (size_t)nI);
    double acc = 0.0;
    for (int64_t r = 0; r < nI; r++) { acc += sg_exp(-s * sg_ln((double)(r + 1))); cdf[r] = acc; }
    for (int64_t r = 0; r < nI; r++) cdf[r] /= acc;
    cdf[nI - 1] = 1.0;
    int32_t *r2i = perm(nI, seed, stream + 1000);
    int64_t maxpairs = nU * nI;
    if (m > maxpairs) m = maxpairs;
    int64_t draws = m + m / 2 + 1024;
    uint64_t *res = NULL;
    for (;;) {
        uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)draws);
        uint32_t *idx = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)draws);
        zd_ctx c = {seed, stream, nU, nI, cdf, r2i, keys, idx, 0};
        parallel_for(draws, nthreads(), zd_fill, &c);
        radix_sort(keys, idx, draws, 64);
        /* first occurrence of each pair = smallest draw index (stable sort) */
        uint8_t *first = (uint8_t *)calloc((size_t)draws, 1);
        int64_t distinct = 0;
        for (int64_t j = 0; j < draws; j++)
            if (j == 0 || keys[j] != keys[j - 1]) { first[idx[j]] = 1; distinct++; }
        if (distinct >= m) {
            int64_t cnt = 0, cut = draws;
            for (int64_t j = 0; j < draws; j++)
                if (first[j] && ++cnt == m) { cut = j; break; }
            res = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m + 1));
            int64_t k = 0;
            for (int64_t j = 0; j < draws; j++)
                if ((j == 0 || keys[j] != keys[j - 1]) && idx[j] <= (uint32_t)cut) res[k++] = keys[j];
            *out_m = k;
            free(keys); free(idx); free(first);
            break;
        }
        free(keys); free(idx); free(first);
        /* grow the draw budget; the sequence is the same, only longer */
        draws = draws * 2;
        if (draws > ((int64_t)1 << 32) - 1) { *out_m = 0; break; }
    }
    free(cdf);
    free(r2i);
    return res;
}

/*
 * Config-2 / config-4 shape: m_bg distinct Zipf(s) pairs, plus 'nblocks'
 * blocks of bU users x bI items (seeded, disjoint user sets), each pair
 * present with probability p, and 'camo' camouflage draws per block user to
 * uniform random items; duplicates merged.
 */
sg_edges *sg_bipartite_zipf(int64_t nU, int64_t nI, int64_t m_bg, double s, int64_t nblocks,
                            int64_t bU, int64_t bI, double p, int64_t camo, uint64_t seed) {
    int64_t mb = 0;
    uint64_t *bg = zipf_pairs(nU, nI, m_bg, s, seed, 10, &mb);
    if (!bg) return NULL;
    if (bU > nU) bU = nU;
    if (bI > nI) bI = nI;
    int64_t extra = nblocks * (bU * bI + bU * camo);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(mb + extra + 1));
    memcpy(keys, bg, sizeof(uint64_t) * (size_t)mb);
    free(bg);
    int64_t k = mb;
    if (nblocks > 0 && bU > 0 && bI > 0) {
        int32_t *pu = perm(nU, seed, 20);
        for (int64_t b = 0; b < nblocks; b++) {
            int32_t *pi = perm(nI, seed, (uint64_t)(30 + b));
            for (int64_t x = 0; x < bU; x++) {
                int64_t user = pu[(b * bU + x) % nU];
                for (int64_t y = 0; y < bI; y++)
                    if (unif(rnd(seed, (uint64_t)(100 + b), (uint64_t)(x * bI + y))) < p)
                        keys[k++] = ((uint64_t)user << 32) | (uint64_t)pi[y];
                for (int64_t z = 0; z < camo; z++) {
                    uint64_t it = below64(rnd(seed, (uint64_t)(200 + b), (uint64_t)(x * camo + z)), (uint64_t)nI);
                    keys[k++] = ((uint64_t)user << 32) | it;
                }
            }
            free(pi);
        }
        free(pu);
    }
    sg_edges *e = edges_from_keys(keys, k, nU, nI);
    free(keys);
    return e;
}

/* ------------------------------------------------------------------ R-MAT */

typedef struct {
    uint64_t seed;
    int scale;
    uint32_t t0, t1, t2;
    const int32_t *relabel;
    uint64_t *keys;
} rm_ctx;

static void rm_fill(void *p, int64_t lo, int64_t hi, int tid) {
    (void)tid;
    rm_ctx *c = (rm_ctx *)p;
    for (int64_t j = lo; j < hi; j++) {
        uint64_t x = 0, y = 0, r = 0;
        for (int l = 0; l < c->scale; l++) {
            if ((l & 1) == 0) r = rnd(c->seed, 50, (uint64_t)j * 16 + (uint64_t)(l >> 1));
            uint32_t u = (uint32_t)(((l & 1) == 0) ? (r >> 32) : (r & 0xffffffffu));
            uint64_t bx, by;
            if (u < c->t0) { bx = 0; by = 0; }
            else if (u < c->t1) { bx = 0; by = 1; }
            else if (u < c->t2) { bx = 1; by = 0; }
            else { bx = 1; by = 1; }
            x = (x << 1) | bx;
            y = (y << 1) | by;
        }
        uint64_t a = (uint64_t)c->relabel[x], b = (uint64_t)c->relabel[y];
        if (a == b) { c->keys[j] = UINT64_MAX; continue; } /* self-loop: dropped */
        if (a > b) { uint64_t t = a; a = b; b = t; }
        c->keys[j] = (a << 32) | b;
    }
}

/*
 * Undirected R-MAT: 2^scale vertices, edge_factor * 2^scale generated edges
 * with quadrant probabilities (a, b, c, 1-a-b-c), seeded vertex relabelling,
 * self-loops dropped and repeated pairs merged.  Edges are stored u < v.
 */
sg_edges *sg_rmat(int scale, int64_t edge_factor, double a, double b, double c, uint64_t seed) {
    int64_t n = (int64_t)1 << scale;
    int64_t draws = edge_factor * n;
    double two32 = 4294967296.0;
    rm_ctx ctx;
    ctx.seed = seed;
    ctx.scale = scale;
    ctx.t0 = (uint32_t)(a * two32);
    ctx.t1 = (uint32_t)((a + b) * two32);
    ctx.t2 = (uint32_t)((a + b + c) * two32);
    int32_t *rl = perm(n, seed, 51);
    ctx.relabel = rl;
    ctx.keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)draws);
    parallel_for(draws, nthreads(), rm_fill, &ctx);
    free(rl);
    int64_t k = 0;
    for (int64_t j = 0; j < draws; j++)
        if (ctx.keys[j] != UINT64_MAX) ctx.keys[k++] = ctx.keys[j];
    sg_edges *e = edges_from_keys(ctx.keys, k, n, 0);
    free(ctx.keys);
    return e;
}

/* n vertices, 'draws' uniform pairs (self-loops dropped, merged), u < v */
sg_edges *sg_random_general(int64_t n, int64_t draws, uint64_t seed) {
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(draws + 1));
    int64_t k = 0;
    for (int64_t j = 0; j < draws; j++) {
        uint64_t r = rnd(seed, 60, (uint64_t)j);
        uint64_t a = below(r, (uint64_t)n), b = below(r << 32, (uint64_t)n);
        if (a == b) continue;
        if (a > b) { uint64_t t = a; a = b; b = t; }
        keys[k++] = (a << 32) | b;
    }
    sg_edges *e = edges_from_keys(keys, k, n, 0);
    free(keys);
    return e;
}

/* ---------------------------------------------------------------- weights */

/*
 * Fraudar edge weights c_e = 1/ln(x + 5) in Q32.32, x = degree of the
 * object vertex of e: the item for bipartite lists, the larger-id endpoint
 * for general lists.  Degrees are taken in the input graph.
 */
void sg_fd_weights(const sg_edges *e, int64_t *c_out) {
    int64_t nobj = e->n_right > 0 ? e->n_right : e->n_left;
    int64_t *deg = (int64_t *)calloc((size_t)nobj + 1, sizeof(int64_t));
    if (e->n_right > 0) {
        for (int64_t j = 0; j < e->m; j++) deg[e->ev[j]]++;
    } else {
        for (int64_t j = 0; j < e->m; j++) { deg[e->eu[j]]++; deg[e->ev[j]]++; }
    }
    /* one table entry per distinct degree value would do; the direct form
       keeps the definition visible */
    for (int64_t j = 0; j < e->m; j++) {
        int64_t x = deg[e->ev[j]]; /* ev is the item, or the larger endpoint */
        c_out[j] = q32(1.0 / sg_ln((double)x + 5.0));
    }
    free(deg);
}

/* edge weights (lo + hash(seed, u, v) mod (hi - lo + 1)) << 32 */
void sg_uniform_edge_weights(const sg_edges *e, int64_t lo, int64_t hi, uint64_t seed, int64_t *c_out) {
    uint64_t span = (uint64_t)(hi - lo + 1);
    for (int64_t j = 0; j < e->m; j++) {
        uint64_t key = ((uint64_t)(uint32_t)e->eu[j] << 32) | (uint64_t)(uint32_t)e->ev[j];
        uint64_t r = rnd(seed, 70, key);
        c_out[j] = (int64_t)((uint64_t)lo + below64(r, span)) << 32;
    }
}

/* vertex weights (lo + uniform mod (hi - lo + 1)) << 32 */
void sg_uniform_vertex_weights(int64_t n, int64_t lo, int64_t hi, uint64_t seed, int64_t *a_out) {
    uint64_t span = (uint64_t)(hi - lo + 1);
    for (int64_t u = 0; u < n; u++)
        a_out[u] = (int64_t)((uint64_t)lo + below64(rnd(seed, 71, (uint64_t)u), span)) << 32;
}

/* ------------------------------------------------------------ CSR layouts */

/*
 * Bipartite layouts: CSR rows = users (columns = item ids), CSC rows = items
 * (columns = user ids), both rows sorted, weights carried along.  'c' may be
 * NULL (then csr_w / csc_w are left untouched).
 */
void sg_bipartite_csr(const sg_edges *e, const int64_t *c, int64_t *csr_ptr, int32_t *csr_idx,
                      int64_t *csr_w, int64_t *csc_ptr, int32_t *csc_idx, int64_t *csc_w) {
    int64_t nU = e->n_left, nI = e->n_right, m = e->m;
    memset(csr_ptr, 0, sizeof(int64_t) * (size_t)(nU + 1));
    memset(csc_ptr, 0, sizeof(int64_t) * (size_t)(nI + 1));
    for (int64_t j = 0; j < m; j++) { csr_ptr[e->eu[j] + 1]++; csc_ptr[e->ev[j] + 1]++; }
    for (int64_t u = 0; u < nU; u++) csr_ptr[u + 1] += csr_ptr[u];
    for (int64_t i = 0; i < nI; i++) csc_ptr[i + 1] += csc_ptr[i];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nI + 1));
    memcpy(fill, csc_ptr, sizeof(int64_t) * (size_t)(nI + 1));
    for (int64_t j = 0; j < m; j++) { /* edges are sorted by (u, i) */
        csr_idx[j] = e->ev[j];
        if (c) csr_w[j] = c[j];
        int64_t q = fill[e->ev[j]]++;
        csc_idx[q] = e->eu[j];
        if (c) csc_w[q] = c[j];
    }
    free(fill);
}

/*
 * Symmetric CSR of a general list (u < v): each edge in both rows, rows
 * sorted.  'c' may be NULL.
 */
void sg_symmetric_csr(const sg_edges *e, const int64_t *c, int64_t *ptr, int32_t *idx, int64_t *w) {
    int64_t n = e->n_left, m = e->m;
    memset(ptr, 0, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t j = 0; j < m; j++) { ptr[e->eu[j] + 1]++; ptr[e->ev[j] + 1]++; }
    for (int64_t u = 0; u < n; u++) ptr[u + 1] += ptr[u];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    memcpy(fill, ptr, sizeof(int64_t) * (size_t)(n + 1));
    /* in (u, v) order, row u receives its larger neighbours ascending and
       row v its smaller ones ascending, smaller ones first */
    for (int64_t j = 0; j < m; j++) {
        int64_t u = e->eu[j], v = e->ev[j];
        int64_t p = fill[u]++, q = fill[v]++;
        idx[p] = (int32_t)v;
        idx[q] = (int32_t)u;
        if (c) { w[p] = c[j]; w[q] = c[j]; }
    }
    free(fill);
}

/* exponential gaps (mean 1/rate) for a Poisson arrival stream, in seconds */
void sg_poisson_arrivals(int64_t k, double rate, uint64_t seed, double *t_out) {
    double t = 0.0;
    for (int64_t j = 0; j < k; j++) {
        double u = unif(rnd(seed, 80, (uint64_t)j));
        t += -sg_ln(1.0 - u) / rate;
        t_out[j] = t;
    }
}

/* log-uniform integers in [lo, hi], rounded to multiples of 'unit' */
void sg_log_uniform(int64_t k, double lo, double hi, int64_t unit, uint64_t seed, int64_t *out) {
    double a = sg_ln(lo), b = sg_ln(hi);
    for (int64_t j = 0; j < k; j++) {
        double u = unif(rnd(seed, 81, (uint64_t)j));
        double x = sg_exp(a + u * (b - a)) / (double)unit;
        int64_t r = (int64_t)(x + 0.5);
        if (r < 1) r = 1;
        out[j] = r * unit;
    }
}

/* uniform integers in [0, k) (k < 2^63), one per index, stream 82 */
void sg_uniform_ints(int64_t count, int64_t k, uint64_t seed, int64_t *out) {
    for (int64_t j = 0; j < count; j++) out[j] = (int64_t)below64(rnd(seed, 82, (uint64_t)j), (uint64_t)k);
}
