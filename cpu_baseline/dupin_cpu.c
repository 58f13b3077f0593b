/*
 * dupin_cpu.c -- Algorithm 2 of Dupin (Sec. 4.1) on the host's cores: the
 * paper's own multi-core design (parallel_for over the live vertices and the
 * removed vertices' arcs, parallel_sum of f), with Algorithms 3 and 4 by flag
 * (Sec. 5.1, 5.2).  A timed CPU baseline beside the single-threaded oracle;
 * not part of the GPU path and not the oracle.
 *
 * Exact integer arithmetic as in the GPU library: Q32.32 int64 peeling
 * weights, __int128 f, thresholds as exact floors (w <= floor(k(D+N) f /
 * (D |S|)), minimum rule when that selects nobody), so a peel's rounds,
 * trace and best prefix equal the oracle's bit for bit.  Neighbour weights
 * drop by atomic fetch-and-subtract (each arc touched once per run).
 *
 * Threads: one pool per call; the rounds advance in lock step on a
 * sense-reversing spin-then-yield barrier.
 */
#include <pthread.h>
#include <sched.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

#define CB_GPO 1u
#define CB_LPO 2u

typedef struct {
    volatile int count, sense;
    int n;
} cbar;

static void cbar_wait(cbar *b, int *local_sense) {
    *local_sense = !*local_sense;
    if (__atomic_add_fetch(&b->count, 1, __ATOMIC_ACQ_REL) == b->n) {
        __atomic_store_n(&b->count, 0, __ATOMIC_RELAXED);
        __atomic_store_n(&b->sense, *local_sense, __ATOMIC_RELEASE);
    } else {
        int spins = 0;
        while (__atomic_load_n(&b->sense, __ATOMIC_ACQUIRE) != *local_sense)
            if (++spins > 1024) sched_yield();
    }
}

static int64_t floor_div_sat(i128 x, i128 y) {
    i128 q = x / y;
    return q > (i128)INT64_MAX ? INT64_MAX : (int64_t)q;
}

static int64_t below_div_sat(i128 x, i128 y) { /* ceil(x / y) - 1 */
    if (x <= 0) return -1;
    return floor_div_sat(x - 1, y);
}

typedef struct {
    /* graph (symmetric CSR) */
    int64_t n;
    const int64_t *rp;
    const int32_t *col;
    const int64_t *cw; /* NULL: every arc weighs 1.0 */
    const int64_t *a;  /* NULL: 0 */
    /* parameters */
    int64_t kD, D;
    int use_min, gpo, lpo;
    int64_t max_rounds;
    int T;
    /* state */
    int64_t *w;
    uint8_t *in, *rem;
    int32_t *live, *live2;
    int64_t live_len;
    int32_t *sel;      /* per thread: the vertices it selected (slice-sized region) */
    int64_t *sel_cnt;  /* per thread */
    int64_t *tmin;     /* per thread: minimum live weight seen */
    i128 *tdf;         /* per thread: f decrement */
    int64_t next;      /* expand work queue over the selected vertices */
    int64_t *sel_off;  /* prefix of sel_cnt */
    /* round state, written by thread 0 between barriers */
    i128 f;
    int64_t size, R, thr, U, best_round, best_size, gpo_le, gpo_lt, n_min_rule;
    i128 best_f;
    int kind;          /* 0 threshold, 1 minimum rule, 2 trim */
    int stop, status;
    /* outputs */
    int32_t *peel_round;
    int64_t *tr_f_hi;
    uint64_t *tr_f_lo;
    int64_t *tr_size, *tr_peeled, tr_cap;
    cbar bar;
} cpu_peel_t;

typedef struct {
    cpu_peel_t *P;
    int t;
} targ;

static int64_t w_init(const cpu_peel_t *P, int64_t u) {
    int64_t s = P->a ? P->a[u] : 0;
    for (int64_t p = P->rp[u]; p < P->rp[u + 1]; p++) s += P->cw ? P->cw[p] : ((int64_t)1 << 32);
    return s;
}

static int frac_gt(i128 a, i128 b, i128 c, i128 d) { return a * d > c * b; }

/* select the live vertices of this thread's slice with w <= thr (or == thr
   for the minimum rule); also the slice's minimum live weight */
static void select_slice(cpu_peel_t *P, int t, int64_t thr, int exact) {
    const int64_t L = P->live_len, j0 = L * t / P->T, j1 = L * (t + 1) / P->T;
    int32_t *out = P->sel + j0; /* this thread's region: at most j1 - j0 vertices */
    int64_t cnt = 0, mn = INT64_MAX;
    for (int64_t j = j0; j < j1; j++) {
        const int32_t u = P->live[j];
        if (u < 0 || !P->in[u]) continue;
        const int64_t wu = P->w[u];
        if (wu < mn) mn = wu;
        if (exact ? wu == thr : wu <= thr) out[cnt++] = u;
    }
    P->sel_cnt[t] = cnt;
    P->tmin[t] = mn;
}

static void *worker(void *arg) {
    cpu_peel_t *P = ((targ *)arg)->P;
    const int t = ((targ *)arg)->t, T = P->T;
    int sense = 0;
    for (;;) {
        /* thread 0 planned the round (or set stop) before this barrier */
        cbar_wait(&P->bar, &sense);
        if (P->stop) break;
        select_slice(P, t, P->thr, 0);
        cbar_wait(&P->bar, &sense);
        if (t == 0) {
            int64_t U = 0, mn = INT64_MAX;
            for (int q = 0; q < T; q++) {
                U += P->sel_cnt[q];
                if (P->tmin[q] < mn) mn = P->tmin[q];
            }
            P->U = U;
            if (U == 0 && P->kind == 0 && P->use_min && mn != INT64_MAX) {
                P->kind = 1; /* minimum rule: every live vertex of minimum weight */
                P->thr = mn;
            }
        }
        cbar_wait(&P->bar, &sense);
        if (P->kind == 1 && P->U == 0) {
            select_slice(P, t, P->thr, 1);
            cbar_wait(&P->bar, &sense);
            if (t == 0) {
                int64_t U = 0;
                for (int q = 0; q < T; q++) U += P->sel_cnt[q];
                P->U = U;
            }
            cbar_wait(&P->bar, &sense);
        }
        if (P->U == 0) { /* cannot happen (Lemma 4.2 / minimum rule) */
            if (t == 0) { P->status = -5; P->stop = 1; }
            cbar_wait(&P->bar, &sense);
            break;
        }
        /* mark U_i */
        {
            const int64_t L = P->live_len, j0 = L * t / T;
            for (int64_t c = 0; c < P->sel_cnt[t]; c++) {
                const int32_t u = P->sel[j0 + c];
                P->rem[u] = 1;
                P->peel_round[u] = (int32_t)(P->R + 1);
            }
            if (t == 0) {
                int64_t o = 0;
                for (int q = 0; q < T; q++) { P->sel_off[q] = o; o += P->sel_cnt[q]; }
                P->sel_off[T] = o;
                P->next = 0;
            }
        }
        cbar_wait(&P->bar, &sense);
        /* expand: chunks of the selected vertices from a shared counter */
        {
            i128 df = 0;
            const int64_t L = P->live_len;
            for (;;) {
                const int64_t c0 = __atomic_fetch_add(&P->next, 64, __ATOMIC_RELAXED);
                if (c0 >= P->U) break;
                const int64_t c1 = c0 + 64 < P->U ? c0 + 64 : P->U;
                int q = 0;
                for (int64_t c = c0; c < c1; c++) {
                    while (P->sel_off[q + 1] <= c) q++;
                    const int32_t u = P->sel[L * q / T + (c - P->sel_off[q])];
                    if (P->a) df += P->a[u];
                    for (int64_t p = P->rp[u]; p < P->rp[u + 1]; p++) {
                        const int32_t v = P->col[p];
                        if (!P->in[v]) continue;
                        const int64_t cv = P->cw ? P->cw[p] : ((int64_t)1 << 32);
                        if (P->rem[v]) {
                            if (v > u) df += cv;
                        } else {
                            df += cv;
                            __atomic_fetch_sub(&P->w[v], cv, __ATOMIC_RELAXED);
                        }
                    }
                }
            }
            P->tdf[t] = df;
        }
        cbar_wait(&P->bar, &sense);
        /* leave S */
        {
            const int64_t j0 = P->live_len * t / T;
            for (int64_t c = 0; c < P->sel_cnt[t]; c++) {
                const int32_t u = P->sel[j0 + c];
                P->in[u] = 0;
                P->rem[u] = 0;
            }
        }
        cbar_wait(&P->bar, &sense);
        if (t == 0) {
            /* close the round, compact the live list when it halved, plan the next */
            i128 df = 0;
            for (int q = 0; q < T; q++) df += P->tdf[q];
            P->f -= df;
            P->size -= P->U;
            P->R++;
            if (P->kind == 1) P->n_min_rule++;
            if (P->R < P->tr_cap) {
                P->tr_f_hi[P->R] = (int64_t)(P->f >> 64);
                P->tr_f_lo[P->R] = (uint64_t)P->f;
                P->tr_size[P->R] = P->size;
                P->tr_peeled[P->R] = P->U;
            }
            if (P->size > 0 && frac_gt(P->f, P->size, P->best_f, P->best_size)) {
                P->best_f = P->f;
                P->best_size = P->size;
                P->best_round = P->R;
            }
            if (2 * P->size <= P->live_len) {
                int64_t o = 0;
                for (int64_t j = 0; j < P->live_len; j++) {
                    const int32_t u = P->live[j];
                    if (u >= 0 && P->in[u]) P->live2[o++] = u;
                }
                int32_t *tmp = P->live; P->live = P->live2; P->live2 = tmp;
                P->live_len = o;
            }
        }
        /* Algorithm 4: is some live w < g(S)?  (a parallel minimum) */
        if (P->lpo) {
            cbar_wait(&P->bar, &sense);
            const int64_t L = P->live_len, j0 = L * t / T, j1 = L * (t + 1) / T;
            int64_t mn = INT64_MAX;
            for (int64_t j = j0; j < j1; j++) {
                const int32_t u = P->live[j];
                if (u >= 0 && P->in[u] && P->w[u] < mn) mn = P->w[u];
            }
            P->tmin[t] = mn;
            cbar_wait(&P->bar, &sense);
        }
        if (t == 0) {
            P->stop = 0;
            if (P->size == 0) P->stop = 1;
            else if (P->R >= P->max_rounds) { P->status = -5; P->stop = 1; }
            else {
                int trim = 0;
                if (P->lpo) {
                    int64_t mn = INT64_MAX;
                    for (int q = 0; q < T; q++) if (P->tmin[q] < mn) mn = P->tmin[q];
                    const int64_t bg = below_div_sat(P->f, P->size);
                    if (mn <= bg) {
                        trim = 1;
                        P->kind = 2;
                        P->thr = bg > P->gpo_lt ? bg : P->gpo_lt;
                    }
                }
                if (!trim) {
                    P->kind = 0;
                    int64_t thr = floor_div_sat((i128)P->kD * P->f, (i128)P->D * P->size);
                    if (P->gpo) {
                        const int64_t le = floor_div_sat((i128)P->D * P->f, (i128)P->kD * P->size);
                        const int64_t lt = below_div_sat((i128)P->D * P->f, (i128)P->kD * P->size);
                        if (le > P->gpo_le) P->gpo_le = le;
                        if (lt > P->gpo_lt) P->gpo_lt = lt;
                        if (P->gpo_le > thr) thr = P->gpo_le;
                    }
                    P->thr = thr;
                }
            }
        }
    }
    return NULL;
}

/*
 * out[0..5]: rounds, best round, best size, best f hi, best f lo, rounds of the
 * minimum rule.  Returns 0, -1 (arguments), -3 (memory), -4 (trace too
 * short), -5 (max_rounds).
 */
int cb_peel(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *cw, const int64_t *a, int32_t k_mult,
            int64_t eps_num, int64_t eps_den, uint32_t flags, int64_t max_rounds, int threads, int32_t *peel_round,
            int64_t *tr_f_hi, uint64_t *tr_f_lo, int64_t *tr_size, int64_t *tr_peeled, int64_t tr_cap, int64_t *out) {
    if (n < 0 || k_mult < 1 || eps_num < 0 || eps_den < 1 || threads < 1 || tr_cap < 1) return -1;
    cpu_peel_t P;
    memset(&P, 0, sizeof(P));
    P.n = n; P.rp = rp; P.col = col; P.cw = cw; P.a = a;
    P.kD = (int64_t)k_mult * (eps_den + eps_num);
    P.D = eps_den;
    P.use_min = P.kD < 2 * P.D;
    P.lpo = (flags & CB_LPO) != 0;
    P.gpo = (flags & (CB_GPO | CB_LPO)) != 0;
    P.max_rounds = max_rounds > 0 ? max_rounds : n + 1;
    P.T = threads;
    P.peel_round = peel_round;
    P.tr_f_hi = tr_f_hi; P.tr_f_lo = tr_f_lo; P.tr_size = tr_size; P.tr_peeled = tr_peeled; P.tr_cap = tr_cap;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    P.w = (int64_t *)malloc(8 * nn);
    P.in = (uint8_t *)malloc(nn);
    P.rem = (uint8_t *)calloc(nn, 1);
    P.live = (int32_t *)malloc(4 * nn);
    P.live2 = (int32_t *)malloc(4 * nn);
    P.sel = (int32_t *)malloc(4 * nn);
    P.sel_cnt = (int64_t *)calloc((size_t)threads, 8);
    P.tmin = (int64_t *)calloc((size_t)threads, 8);
    P.tdf = (i128 *)calloc((size_t)threads, sizeof(i128));
    P.sel_off = (int64_t *)calloc((size_t)threads + 1, 8);
    pthread_t *th = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    targ *ta = (targ *)calloc((size_t)threads, sizeof(targ));
    int rc = 0;
    if (!P.w || !P.in || !P.rem || !P.live || !P.live2 || !P.sel || !P.sel_cnt || !P.tmin || !P.tdf || !P.sel_off ||
        !th || !ta) rc = -3;
    if (!rc) {
        i128 s = 0;
        for (int64_t u = 0; u < n; u++) {
            P.w[u] = w_init(&P, u);
            P.in[u] = 1;
            P.live[u] = (int32_t)u;
            peel_round[u] = INT32_MAX;
            s += (i128)P.w[u] + (a ? a[u] : 0);
        }
        P.f = s / 2;
        P.size = n;
        P.live_len = n;
        P.best_f = P.f;
        P.best_size = n;
        P.gpo_lt = -1;
        tr_f_hi[0] = (int64_t)(P.f >> 64);
        tr_f_lo[0] = (uint64_t)P.f;
        tr_size[0] = n;
        tr_peeled[0] = 0;
        /* plan round 1 */
        if (n == 0) P.stop = 1;
        else {
            int64_t thr = floor_div_sat((i128)P.kD * P.f, (i128)P.D * P.size);
            if (P.gpo) {
                P.gpo_le = floor_div_sat((i128)P.D * P.f, (i128)P.kD * P.size);
                P.gpo_lt = below_div_sat((i128)P.D * P.f, (i128)P.kD * P.size);
                if (P.gpo_le > thr) thr = P.gpo_le;
            }
            P.thr = thr;
        }
        P.bar.n = threads;
        int started = 0;
        for (int t = 0; t < threads; t++) {
            ta[t].P = &P;
            ta[t].t = t;
            if (pthread_create(&th[t], NULL, worker, &ta[t]) != 0) break;
            started++;
        }
        if (started < threads) {
            /* stop at once: arrive at the first barrier for each thread that
               did not start, so the started ones pass it and leave */
            P.stop = 1;
            for (int t = started; t < threads; t++) {
                int sense = 0;
                cbar_wait(&P.bar, &sense);
            }
            rc = -3;
        }
        for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
        if (!rc) rc = P.status;
        if (!rc && P.R + 1 > tr_cap) rc = -4;
    }
    out[0] = P.R;
    out[1] = P.best_round;
    out[2] = P.best_size;
    out[3] = (int64_t)(P.best_f >> 64);
    out[4] = (int64_t)(uint64_t)P.best_f;
    out[5] = P.n_min_rule;
    free(P.w); free(P.in); free(P.rem); free(P.live); free(P.live2); free(P.sel);
    free(P.sel_cnt); free(P.tmin); free(P.tdf); free(P.sel_off); free(th); free(ta);
    return rc;
}
