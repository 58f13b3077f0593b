// tds.cu -- batch peeling under the clique metrics of Sec. 2.1: TDS
// (triangle density) and kCLiDS (q-clique density).  f(S) = number of
// q-cliques of G[S] (q = 3 for TDS), w_u(S) = the q-cliques of G[S] through
// u, so that removing u lowers f by w_u.  The rounds are Algorithm 2 (Sec.
// 4.1; the paper's k for these metrics is q) with Algorithm 3's tau_max and
// Algorithm 4's trims by flag, exactly as for the other metrics but on plain
// counts (no Q32.32 scale): every comparison is between ratios of integers.
//
// Device state lives in one control block; a round is five launches --
//   min     the minimum live weight (the minimum rule and the trim test);
//   plan    one thread: a trim round if some live w < g(S) (Algorithm 4),
//           else a main round (w <= max(tau_max, k(1+eps) g)), or the
//           minimum rule if that threshold selects nobody;
//   select  every live u with w_u <= T leaves: its round is recorded and it
//           joins the round's list;
//   expand  one warp per removed vertex u, one lane per arc u -> v with v in
//           S_{i-1}: the cliques of G[S_{i-1}] through u whose smallest
//           member besides u is v (for TDS a merge of the two sorted rows,
//           the common neighbours x > v, each triangle counted by its
//           smallest member in U_i; for kCLiDS a depth-first walk over u's
//           row after v, each candidate kept when it is in the rows of every
//           member chosen so far and, if it leaves in this round too,
//           outranks u in (degree, id), so that only the removed member of
//           lowest rank lists the clique); each clique that dies lowers f by
//           one and each member outside U_i by one;
//   close   one thread: f, |S|, the trace, the best prefix.
// The host launches rounds in groups and reads the control block between
// groups; launches after the peel ends return at once.  The initial counts
// list every clique once: TDS from its smallest vertex, kCLiDS from its
// member of lowest degree (the same walks, keeping only members that outrank
// u).  Rows are sorted (the loader checks it).
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "dupin_internal.h"

namespace {

struct TdsCtl {
    long long round, size, best_round, best_size, n_min_rule;
    long long f, bf;           // triangle counts
    long long gpo_le, gpo_lt;  // tau_max's integer forms (Algorithm 3)
    long long T;               // this round removes live w <= T
    long long kind;            // 0 main round, 1 minimum rule, 2 trim round
    long long minw;            // minimum live weight before the round
    long long ucnt;            // |U_i|
    long long df;              // triangles that die in the round
    int status;                // 0 running, 1 done
    int error;
};

struct TdsArgs {
    long long n;
    const long long *rp;
    const int *col;
    const int *hubs;
    long long *w;
    int *pr;
    int *front;
    TdsCtl *ctl;
    long long *tr_f, *tr_size, *tr_peeled;
    long long tr_cap;
    long long kD, D;
    int gpo, lpo;
    int q;  // clique size (3 for TDS)
    long long max_rounds;
};

__device__ __forceinline__ int head(const TdsArgs &A, long long p) { return arc_head(A.col[p], A.hubs); }

// first position in v's row whose neighbour id exceeds x
__device__ __forceinline__ long long row_after(const TdsArgs &A, int v, int x) {
    long long lo = A.rp[v], hi = A.rp[v + 1];
    while (lo < hi) {
        const long long mid = lo + ((hi - lo) >> 1);
        if (head(A, mid) <= x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_tds_reset(TdsArgs A) {
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < A.n; u += (long long)gridDim.x * blockDim.x) {
        A.w[u] = 0;
        A.pr[u] = DUPIN_LIVE;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        TdsCtl z;
        memset(&z, 0, sizeof(z));
        z.gpo_lt = -1;
        z.size = A.n;
        *A.ctl = z;
    }
}

// every triangle u < v < x once (one warp per u, one lane per arc u -> v, v > u)
__global__ void k_tds_count(TdsArgs A) {
    const int lane = threadIdx.x & 31;
    const long long W = (long long)gridDim.x * (blockDim.x >> 5);
    long long cnt = 0;
    for (long long u = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); u < A.n; u += W) {
        const long long b = A.rp[u], e = A.rp[u + 1];
        for (long long j = b + lane; j < e; j += 32) {
            const int v = head(A, j);
            if (v <= (int)u) continue;
            long long a = j + 1, c = row_after(A, v, v);
            const long long ce = A.rp[v + 1];
            while (a < e && c < ce) {
                const int xa = head(A, a), xc = head(A, c);
                if (xa < xc) a++;
                else if (xc < xa) c++;
                else {
                    atomicAdd((unsigned long long *)&A.w[u], 1ull);
                    atomicAdd((unsigned long long *)&A.w[v], 1ull);
                    atomicAdd((unsigned long long *)&A.w[xa], 1ull);
                    cnt++;
                    a++;
                    c++;
                }
            }
        }
    }
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, d);
    if (lane == 0 && cnt) atomicAdd((unsigned long long *)&A.ctl->f, (unsigned long long)cnt);
}

__global__ void k_tds_start(TdsArgs A) {
    TdsCtl *c = A.ctl;
    c->round = 0;
    c->size = A.n;
    c->best_round = 0;
    c->best_size = A.n;
    c->bf = c->f;
    c->status = A.n == 0 ? 1 : 0;
    if (A.tr_cap > 0) {
        A.tr_f[0] = c->f;
        A.tr_size[0] = A.n;
        A.tr_peeled[0] = 0;
    }
}

__global__ void k_tds_min(TdsArgs A) {
    const TdsCtl *c = A.ctl;
    if (c->status || c->error) return;
    long long m = 0x7fffffffffffffffLL;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < A.n; u += (long long)gridDim.x * blockDim.x)
        if (A.pr[u] == DUPIN_LIVE && A.w[u] < m) m = A.w[u];
    m = warp_min64(m);
    if ((threadIdx.x & 31) == 0 && m != 0x7fffffffffffffffLL) atomicMin(&A.ctl->minw, m);
}

__device__ __forceinline__ long long tds_floor(u128 x, u128 y) {
    const u128 q = x / y;
    return q > (u128)0x7fffffffffffffffULL ? 0x7fffffffffffffffLL : (long long)q;
}

// ceil(x / y) - 1 (the largest integer strictly below x / y), -1 for x = 0
__device__ __forceinline__ long long tds_below(u128 x, u128 y) {
    if (x == 0) return -1;
    return tds_floor(x - 1, y);
}

__global__ void k_tds_plan(TdsArgs A) {
    TdsCtl *c = A.ctl;
    if (c->status || c->error) return;
    if (c->round + 1 > A.max_rounds) {
        c->error = DUPIN_ERR_NO_PROGRESS;
        return;
    }
    const u128 f = (u128)(unsigned long long)c->f, size = (u128)(unsigned long long)c->size;
    const long long m = c->minw;
    const long long below_g = tds_below(f, size);
    if (A.lpo && c->round > 0 && m <= below_g) {  // Algorithm 4: some live w < g(S)
        c->T = below_g > c->gpo_lt ? below_g : c->gpo_lt;
        c->kind = 2;
    } else {
        long long T = tds_floor((u128)(unsigned long long)A.kD * f, (u128)(unsigned long long)A.D * size);
        if (A.gpo) {  // Algorithm 3: tau_max refined at every main round
            const u128 num = (u128)(unsigned long long)A.D * f, den = (u128)(unsigned long long)A.kD * size;
            const long long le = tds_floor(num, den), lt = tds_below(num, den);
            if (le > c->gpo_le) c->gpo_le = le;
            if (lt > c->gpo_lt) c->gpo_lt = lt;
            if (c->gpo_le > T) T = c->gpo_le;
        }
        c->kind = 0;
        if (m > T) {  // the threshold selects nobody: the minimum rule
            T = m;
            c->kind = 1;
        }
        c->T = T;
    }
    c->ucnt = 0;
    c->df = 0;
}

__global__ void k_tds_select(TdsArgs A) {
    const TdsCtl *c = A.ctl;
    if (c->status || c->error) return;
    const long long T = c->T;
    const int r = (int)(c->round + 1);
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); b < A.n; b += stride) {
        const long long u = b + lane;
        const bool sel = u < A.n && A.pr[u] == DUPIN_LIVE && A.w[u] <= T;
        const unsigned m = __ballot_sync(0xffffffffu, sel);
        if (!m) continue;
        long long base = 0;
        if (lane == 0) base = (long long)atomicAdd((unsigned long long *)&A.ctl->ucnt, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (sel) {
            A.pr[u] = r;
            A.front[base + __popc(m & ((1u << lane) - 1u))] = (int)u;
        }
    }
}

__global__ void k_tds_expand(TdsArgs A) {
    const TdsCtl *c = A.ctl;
    if (c->status || c->error) return;
    const int r = (int)(c->round + 1);
    const long long U = c->ucnt;
    const int lane = threadIdx.x & 31;
    const long long W = (long long)gridDim.x * (blockDim.x >> 5);
    long long dead = 0;
    for (long long k = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); k < U; k += W) {
        const int u = A.front[k];
        const long long b = A.rp[u], e = A.rp[u + 1];
        for (long long j = b + lane; j < e; j += 32) {
            const int v = head(A, j);
            const int pv = A.pr[v];
            if (pv < r) continue;  // left in an earlier round
            long long a = j + 1, cc = row_after(A, v, v);
            const long long ce = A.rp[v + 1];
            while (a < e && cc < ce) {
                const int xa = head(A, a), xc = head(A, cc);
                if (xa < xc) a++;
                else if (xc < xa) cc++;
                else {
                    const int x = xa, px = A.pr[x];
                    if (px >= r) {  // the triangle {u, v, x} of G[S_{i-1}]
                        const bool vu = pv == r, xu = px == r;
                        // counted once: by its smallest member in U_i
                        if (!((vu && v < u) || (xu && x < u))) {
                            dead++;
                            if (!vu) atomicAdd((unsigned long long *)&A.w[v], (unsigned long long)-1ll);
                            if (!xu) atomicAdd((unsigned long long *)&A.w[x], (unsigned long long)-1ll);
                        }
                    }
                    a++;
                    cc++;
                }
            }
        }
    }
    for (int d = 16; d > 0; d >>= 1) dead += __shfl_down_sync(0xffffffffu, dead, d);
    if (lane == 0 && dead) atomicAdd((unsigned long long *)&A.ctl->df, (unsigned long long)dead);
}

// ---- kCLiDS: q-cliques, 3 <= q <= DUPIN_CLIQUE_MAX_Q

constexpr int QMAX = DUPIN_CLIQUE_MAX_Q;
// positions of depth d (2 <= d <= QMAX - 1) start at pos_base(d): d of them,
// one in the row of each member chosen before depth d
__host__ __device__ constexpr int pos_base(int d) { return d * (d - 1) / 2 - 1; }

// first position in [p, end) whose id is at least x (end if none): doubling
// steps from p, then a binary search in the last step, so a long row is
// crossed in O(log gap) reads
__device__ __forceinline__ long long seek(const TdsArgs &A, long long p, long long end, int x) {
    if (p >= end || head(A, p) >= x) return p;
    long long lo = p, hi, step = 1;  // head(lo) < x
    for (;;) {
        hi = lo + step;
        if (hi >= end) {
            hi = end;
            break;
        }
        if (head(A, hi) >= x) break;
        lo = hi;
        step <<= 1;
    }
    lo++;  // the answer is in [lo, hi]
    while (lo < hi) {
        const long long mid = lo + ((hi - lo) >> 1);
        if (head(A, mid) < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// The q-cliques {u, v, y_2, ..., y_{q-1}} with v < y_2 < ... < y_{q-1}, all in
// u's row, whose members pass 'keep' (v is the caller's: u's arc at position
// j).  c[0] = u, c[1] = v; at depth d the candidates y_d are the ids above
// c[d-1] present in the rows of c[0..d-1].  They are found by a leapfrog
// join: the rows take turns, each seeking its position to the largest id
// seen so far, until d rows in a row show the same id (rows are sorted, so
// every position only moves forward and the largest id only grows; a long
// row is crossed by doubling steps).  'emit' gets the q members in c[0..q-1].
template <class Keep, class Emit>
__device__ void clique_walk(const TdsArgs &A, int q, int u, long long j, long long e, int v, Keep keep, Emit emit) {
    int c[QMAX];
    long long end[QMAX];
    long long pos[pos_base(QMAX)];
    c[0] = u;
    c[1] = v;
    end[0] = e;
    end[1] = A.rp[v + 1];
    pos[pos_base(2)] = j + 1;
    pos[pos_base(2) + 1] = row_after(A, v, v);
    int d = 2;
    while (d >= 2) {
        long long *P = pos + pos_base(d);
        bool found = false;
        int y = 0;
        if (P[0] < end[0]) {
            y = head(A, P[0]);
            int agree = 1, t = 1;  // rows in turn that show y
            for (;;) {
                if (agree == d) {  // y is in every row
                    if (keep(y)) {
                        found = true;
                        break;
                    }
                    if (++P[0] >= end[0]) break;
                    y = head(A, P[0]);
                    agree = 1;
                    t = 1;
                    continue;
                }
                P[t] = seek(A, P[t], end[t], y);
                if (P[t] >= end[t]) break;  // a row is used up: no candidate left at this depth
                const int h = head(A, P[t]);
                if (h == y) {
                    agree++;
                } else {
                    y = h;
                    agree = 1;
                }
                t = t + 1 == d ? 0 : t + 1;
            }
        }
        if (!found) {
            d--;
            continue;
        }
        P[0]++;  // this depth resumes after y
        c[d] = y;
        if (d == q - 1) {
            emit(c);
            continue;
        }
        long long *N = pos + pos_base(d + 1);
        for (int t = 0; t < d; t++) N[t] = P[t];
        N[d] = row_after(A, y, y);
        end[d] = A.rp[y + 1];
        d++;
    }
}

// every q-clique once, from its member u of lowest rank (degree, then id):
// the lane of arc u -> v walks when v outranks u and keeps only members that
// outrank u, so a hub lists just the cliques whose other members have higher
// degree still, and the listing spreads over the low-degree vertices' warps
__global__ void k_clq_count(TdsArgs A) {
    const int lane = threadIdx.x & 31;
    const int q = A.q;
    const long long W = (long long)gridDim.x * (blockDim.x >> 5);
    long long cnt = 0;
    for (long long u = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); u < A.n; u += W) {
        const long long b = A.rp[u], e = A.rp[u + 1];
        const auto above = [&](int x) {
            const long long dx = A.rp[x + 1] - A.rp[x];
            return dx > e - b || (dx == e - b && x > (int)u);
        };
        for (long long j = b + lane; j < e; j += 32) {
            const int v = head(A, j);
            if (!above(v)) continue;
            clique_walk(
                A, q, (int)u, j, e, v, above,
                [&](const int *c) {
                    for (int t = 0; t < q; t++) atomicAdd((unsigned long long *)&A.w[c[t]], 1ull);
                    cnt++;
                });
        }
    }
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, d);
    if (lane == 0 && cnt) atomicAdd((unsigned long long *)&A.ctl->f, (unsigned long long)cnt);
}

// the q-cliques of G[S_{i-1}] that die in round i (one warp per removed
// vertex u): each is listed once, by its removed member of lowest rank
// (degree, then id) -- u's walk keeps a member removed in this round only if
// it outranks u -- and lowers f by one and each member outside U_i by one
__global__ void k_clq_expand(TdsArgs A) {
    const TdsCtl *ctl = A.ctl;
    if (ctl->status || ctl->error) return;
    const int r = (int)(ctl->round + 1);
    const long long U = ctl->ucnt;
    const int q = A.q;
    const int lane = threadIdx.x & 31;
    const long long W = (long long)gridDim.x * (blockDim.x >> 5);
    long long dead = 0;
    for (long long k = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); k < U; k += W) {
        const int u = A.front[k];
        const long long b = A.rp[u], e = A.rp[u + 1];
        const auto keep = [&](int x) {
            const int px = A.pr[x];
            if (px < r) return false;  // left in an earlier round
            if (px > r) return true;   // survives the round
            const long long dx = A.rp[x + 1] - A.rp[x];
            return dx > e - b || (dx == e - b && x > u);
        };
        for (long long j = b + lane; j < e; j += 32) {
            const int v = head(A, j);
            if (!keep(v)) continue;
            clique_walk(A, q, u, j, e, v, keep, [&](const int *c) {
                dead++;
                for (int t = 1; t < q; t++)
                    if (A.pr[c[t]] != r) atomicAdd((unsigned long long *)&A.w[c[t]], (unsigned long long)-1ll);
            });
        }
    }
    for (int d = 16; d > 0; d >>= 1) dead += __shfl_down_sync(0xffffffffu, dead, d);
    if (lane == 0 && dead) atomicAdd((unsigned long long *)&A.ctl->df, (unsigned long long)dead);
}

__global__ void k_tds_close(TdsArgs A) {
    TdsCtl *c = A.ctl;
    if (c->status || c->error) return;
    if (c->ucnt == 0) {  // cannot happen (Lemma 4.2 / minimum rule)
        c->error = DUPIN_ERR_NO_PROGRESS;
        return;
    }
    const long long i = c->round + 1;
    c->f -= c->df;
    c->size -= c->ucnt;
    c->round = i;
    c->n_min_rule += c->kind == 1 ? 1 : 0;
    if (c->size > 0 &&
        (u128)(unsigned long long)c->f * (unsigned long long)c->best_size >
            (u128)(unsigned long long)c->bf * (unsigned long long)c->size) {
        c->bf = c->f;
        c->best_size = c->size;
        c->best_round = i;
    }
    if (i < A.tr_cap) {
        A.tr_f[i] = c->f;
        A.tr_size[i] = c->size;
        A.tr_peeled[i] = c->ucnt;
    }
    c->minw = 0x7fffffffffffffffLL;
    if (c->size == 0) c->status = 1;
}

__global__ void k_tds_mask(const int *pr, long long n, const TdsCtl *c, uint8_t *mask) {
    const long long br = c->best_round;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x)
        mask[u] = (long long)pr[u] > br ? 1 : 0;
}

__global__ void k_tds_minw_init(TdsCtl *c) { c->minw = 0x7fffffffffffffffLL; }

}  // namespace

// dupin_peel for the metrics DUPIN_TDS and DUPIN_KCLIDS (parameters checked by the caller).
int tds_peel(dupin_graph *g, const dupin_params *p, dupin_result *r, cudaStream_t s) {
    const long long n = g->n;
    const long long max_rounds = p->max_rounds > 0 ? p->max_rounds : n + 1;
    const long long tr_cap = std::min<long long>(max_rounds, n) + 1;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    TdsArgs A;
    memset(&A, 0, sizeof(A));
    A.n = n;
    A.rp = g->rp;
    A.col = g->col;
    A.hubs = g->hubs;
    A.kD = (long long)p->k_mult * (p->eps_den + p->eps_num);
    A.D = p->eps_den;
    A.gpo = (p->flags & (DUPIN_GPO | DUPIN_LPO)) ? 1 : 0;
    A.lpo = (p->flags & DUPIN_LPO) ? 1 : 0;
    A.q = p->metric == DUPIN_KCLIDS ? p->clique_q : 3;
    const bool tri = p->metric == DUPIN_TDS;  // the triangle kernels; kCLiDS (any q) walks
    A.max_rounds = max_rounds;
    A.tr_cap = tr_cap;
    cudaError_t e = cudaSuccess;
    void *buf[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    auto alloc = [&](int k, size_t bytes) {
        if (e == cudaSuccess) e = cudaMallocAsync(&buf[k], bytes ? bytes : 8, s);
    };
    alloc(0, 8 * (size_t)n);
    alloc(1, 4 * (size_t)n);
    alloc(2, 4 * (size_t)n);
    alloc(3, sizeof(TdsCtl));
    alloc(4, 8 * (size_t)tr_cap);
    alloc(5, 8 * (size_t)tr_cap);
    alloc(6, 8 * (size_t)tr_cap);
    auto release = [&]() {
        for (void *q : buf)
            if (q) cudaFreeAsync(q, s);
        cudaStreamSynchronize(s);
    };
    if (e != cudaSuccess) {
        release();
        cudaGetLastError();
        return dupin_fail(e == cudaErrorMemoryAllocation ? DUPIN_ERR_OOM : DUPIN_ERR_CUDA,
                          std::string("clique peel state: ") + cudaGetErrorString(e));
    }
    A.w = (long long *)buf[0];
    A.pr = (int *)buf[1];
    A.front = (int *)buf[2];
    A.ctl = (TdsCtl *)buf[3];
    A.tr_f = (long long *)buf[4];
    A.tr_size = (long long *)buf[5];
    A.tr_peeled = (long long *)buf[6];
    const int vgrid = sms * 8;
    k_tds_reset<<<vgrid, 256, 0, s>>>(A);
    if (tri) k_tds_count<<<vgrid, 256, 0, s>>>(A);
    else k_clq_count<<<vgrid, 256, 0, s>>>(A);
    k_tds_start<<<1, 1, 0, s>>>(A);
    k_tds_minw_init<<<1, 1, 0, s>>>(A.ctl);
    TdsCtl hc;
    int rc = DUPIN_OK;
    for (long long done_rounds = 0;; done_rounds += 32) {
        for (int j = 0; j < 32; j++) {
            k_tds_min<<<vgrid, 256, 0, s>>>(A);
            k_tds_plan<<<1, 1, 0, s>>>(A);
            k_tds_select<<<vgrid, 256, 0, s>>>(A);
            if (tri) k_tds_expand<<<vgrid, 256, 0, s>>>(A);
            else k_clq_expand<<<vgrid, 256, 0, s>>>(A);
            k_tds_close<<<1, 1, 0, s>>>(A);
        }
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, A.ctl, sizeof(hc), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            rc = dupin_cuda_fail(e, "clique peel rounds");
            break;
        }
        if (hc.error || hc.status) break;
        if (done_rounds > max_rounds + 64) {  // the device stops itself first; a guard only
            rc = dupin_fail(DUPIN_ERR_NO_PROGRESS, "max_rounds reached before the set became empty");
            break;
        }
    }
    if (rc == DUPIN_OK && hc.error)
        rc = dupin_fail(hc.error, hc.error == DUPIN_ERR_NO_PROGRESS ? "max_rounds reached before the set became empty"
                                                                    : "clique peel failed");
    if (rc == DUPIN_OK) {
        r->n_rounds = hc.round;
        r->best_round = hc.best_round;
        r->best_size = hc.best_size;
        r->best_f_hi = 0;
        r->best_f_lo = (unsigned long long)hc.bf;
        r->best_density = hc.best_size > 0 ? (double)hc.bf / (double)hc.best_size : 0.0;
        r->n_min_rule = hc.n_min_rule;
        r->n_bulk_rounds = 0;
        r->tail_arcs = 0;
        r->tail_ctas = 0;
        for (int j = 0; j < 4; j++) r->phase_ms[j] = 0.f;
        const bool dev = (p->flags & DUPIN_RESULT_DEVICE) != 0;
        const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (r->best_mask && n > 0) {
            uint8_t *mk = nullptr;
            e = dev ? cudaSuccess : cudaMallocAsync((void **)&mk, (size_t)n, s);
            if (e == cudaSuccess) {
                k_tds_mask<<<sms * 4, 256, 0, s>>>(A.pr, n, A.ctl, dev ? r->best_mask : mk);
                if (!dev) e = cudaMemcpyAsync(r->best_mask, mk, (size_t)n, cudaMemcpyDeviceToHost, s);
                if (mk) cudaFreeAsync(mk, s);
            }
        }
        if (e == cudaSuccess && r->peel_round && n > 0)
            e = cudaMemcpyAsync(r->peel_round, A.pr, 4 * (size_t)n, kind, s);
        const long long nt = hc.round + 1;
        const long long cnt = std::min<long long>(nt, r->trace_cap);
        if (e == cudaSuccess && cnt > 0) {
            // f of each S_i as a (hi, lo) pair: the counts are below 2^63
            if (r->trace_f_lo) e = cudaMemcpyAsync(r->trace_f_lo, A.tr_f, 8 * (size_t)cnt, kind, s);
            if (e == cudaSuccess && r->trace_f_hi) {
                if (dev) e = cudaMemsetAsync(r->trace_f_hi, 0, 8 * (size_t)cnt, s);
                else memset(r->trace_f_hi, 0, 8 * (size_t)cnt);
            }
            if (e == cudaSuccess && r->trace_size) e = cudaMemcpyAsync(r->trace_size, A.tr_size, 8 * (size_t)cnt, kind, s);
            if (e == cudaSuccess && r->trace_peeled)
                e = cudaMemcpyAsync(r->trace_peeled, A.tr_peeled, 8 * (size_t)cnt, kind, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = dupin_cuda_fail(e, "clique peel results");
        if (rc == DUPIN_OK && (r->trace_f_hi || r->trace_f_lo || r->trace_size || r->trace_peeled) &&
            r->trace_cap < nt)
            rc = dupin_fail(DUPIN_ERR_BUFFER_TOO_SMALL, "trace_cap < n_rounds + 1 (n_rounds is filled)");
    }
    release();
    return rc;
}
