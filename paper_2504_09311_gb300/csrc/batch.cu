// batch.cu -- dupin_peel_batch: many independent graphs, one CTA per graph.
//
// A persistent grid pulls graphs from an atomic queue; each CTA runs a whole
// peel (Algorithm 2, Sec. 4.1) of its graph: initial weights (a warp per row,
// the whole CTA for rows longer than CTA_BIGROW), then the rounds.  The
// graph's weights stay in global memory (L2-resident for window-sized
// graphs) with the vertex state in the sign (w >= 0 live, w = -i removed in
// round i); 64-vertex segment minima, double-buffered by round parity, sit in
// shared memory, so a round scans only segments that can hold selected
// vertices and every warp closes the round itself (two barriers per round),
// exactly as the single-graph tail does.  Graphs with more than CTA_MAX_N
// vertices take the single-graph path.  Results are identical to dupin_peel:
// the arithmetic is the same exact integer peel.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <type_traits>
#include <vector>

#include <map>
#include <mutex>
#include "dupin_internal.h"
#include "peel_device.cuh"

// Two launch shapes of the batched kernel, picked per device (default, or by
// dupin_batch_tune): 128 threads x 4 CTAs per SM, or 256 threads x 2.
#define CTA_MAX_SEG 2048
#define CTA_MAX_N ((long long)CTA_MAX_SEG * TAIL_SEG)
static_assert(CTA_MAX_N == DUPIN_BATCH_CTA_MAX_N, "header limit out of date");
#define CTA_BIGROW 2048
#define CTA_BIGLIST 64

struct CtaJob {
    long long n, arcs;
    const long long *rp;
    const int *col;
    const long long *cw;  // nullptr: DG
    const long long *a;   // nullptr: 0
    const int *hubs;      // heads of hub-coded arcs
    long long kD, D, max_rounds;
    int use_min, gpo, lpo;
    long long *w;      // [n] workspace
    int *front;        // [n] workspace
    int *pr;           // [n] output
    long long *tr_f_hi;
    unsigned long long *tr_f_lo;
    long long *tr_size, *tr_peeled;
    long long tr_cap;
    long long *out;    // [8]: R, best round, best size, best f hi, best f lo, minimum-rule rounds, error, 0
};

template <int NT>
__device__ __forceinline__ void cta_peel_one(const CtaJob &J, long long *segbuf, TailAcc<NT / 32> *s_acc, long long *s_w,
                                             long long *s_pref, long long *s_fs, long long *s_fl, int *s_big,
                                             int *s_nbig, unsigned long long *s_lo, unsigned long long *s_hi) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const long long n = J.n;
    const bool dg = J.cw == nullptr;
    long long *w = J.w;
    const long long *rp = J.rp;
    const int *col = J.col;
    const long long *cw = J.cw;
    const int *hubs = J.hubs;
    const int nseg = (int)((n + TAIL_SEG - 1) / TAIL_SEG);

    // ---- initial peeling weights w_u = a_u + sum_v c_uv (Sec. 2.2)
    if (tid == 0) *s_nbig = 0;
    for (long long u = tid; u < n; u += NT) {
        const long long d = rp[u + 1] - rp[u];
        w[u] = dg ? (d << 32) : (J.a ? J.a[u] : 0);
    }
    __syncthreads();
    if (!dg) {
        for (long long u = wid; u < n; u += (NT / 32)) {
            const long long b = rp[u], e = rp[u + 1];
            if (e - b > CTA_BIGROW) {
                int k = 0;
                if (lane == 0) {
                    k = atomicAdd(s_nbig, 1);
                    if (k < CTA_BIGLIST) s_big[k] = (int)u;
                }
                k = __shfl_sync(0xffffffffu, k, 0);
                if (k < CTA_BIGLIST) continue;  // the whole CTA sums it below
                // list full: this warp sums the row itself
            }
            long long sum = 0;
            for (long long p = b + lane; p < e; p += 32) sum += cw[p];
            sum = warp_sum64(sum);
            if (lane == 0) w[u] += sum;
        }
        __syncthreads();
        const int nb = *s_nbig < CTA_BIGLIST ? *s_nbig : CTA_BIGLIST;
        for (int k = 0; k < nb; k++) {
            const long long u = s_big[k];
            long long sum = 0;
            for (long long p = rp[u] + tid; p < rp[u + 1]; p += NT) sum += cw[p];
            sum = warp_sum64(sum);
            if (lane == 0) s_w[wid] = sum;
            __syncthreads();
            if (tid == 0) {
                long long t = 0;
                for (int q = 0; q < (NT / 32); q++) t += s_w[q];
                w[u] += t;
            }
            __syncthreads();
        }
    }
    __syncthreads();
    // f(V) = sum_u (w_u + a_u) / 2; segment minima of round 1
    {
        unsigned long long lo = 0, hi = 0;
        for (long long u = tid; u < n; u += NT) {
            add128(lo, hi, (unsigned long long)w[u], 0);
            if (!dg && J.a) add128(lo, hi, (unsigned long long)J.a[u], 0);
        }
        warp_sum128(lo, hi);
        if (lane == 0) {
            s_lo[wid] = lo;
            s_hi[wid] = hi;
        }
    }
    long long *first = segbuf + (1 & 1) * nseg;
    for (int q = wid; q < nseg; q += (NT / 32)) {
        const long long p = (long long)q * TAIL_SEG + 2 * lane;
        const long long w0 = p < n ? w[p] : -1, w1 = p + 1 < n ? w[p + 1] : -1;
        long long m = kMaxLL;
        if (w0 >= 0) m = w0;
        if (w1 >= 0 && w1 < m) m = w1;
        m = warp_min64(m);
        if (lane == 0) first[q] = m;
    }
    if (tid < 2) s_acc[tid].F = 0;
    __syncthreads();
    RoundState st;
    {
        unsigned long long lo = 0, hi = 0;
        for (int q = 0; q < (NT / 32); q++) add128(lo, hi, s_lo[q], s_hi[q]);
        st.f = mk128(lo, hi) >> 1;
    }
    st.round = 0;
    st.size = n;
    st.best_round = 0;
    st.best_size = n;
    st.bf = st.f;
    st.gpo_le = 0;
    st.gpo_lt = -1;
    st.gm_f = 0;
    st.gm_s = 0;
    st.n_min_rule = 0;
    st.scan = 0;
    if (tid == 0 && J.tr_cap > 0) {
        J.tr_f_hi[0] = (long long)(unsigned long long)(st.f >> 64);
        J.tr_f_lo[0] = (unsigned long long)st.f;
        J.tr_size[0] = n;
        J.tr_peeled[0] = 0;
    }
    int err = 0;
    // the round loop in two forms: NARROW (f < 2^62, so every sum of a
    // round fits 64 bits: 64-bit adds, 32-bit warp reductions) or wide
    auto rounds = [&](auto narrow_tag) {
        constexpr bool NARROW = decltype(narrow_tag)::value;
        TailRound R = tail_plan<NARROW>(J.kD, J.D, J.use_min, J.gpo, J.lpo, st, seg_global_min(first, nseg));
        while (!R.done) {
            if (R.i > J.max_rounds) {
                err = DUPIN_ERR_NO_PROGRESS;
                break;
            }
            const long long i = R.i;
            const long long *cur = segbuf + (i & 1) * nseg;
            long long *nxt = segbuf + ((i + 1) & 1) * nseg;
            TailAcc<NT / 32> &acc = s_acc[i & 1];
            // ---- select
            unsigned long long wlo = 0, whi = 0;
            long long mins = kMaxLL;  // new minimum over the segments this lane looked at
            for (int q0 = wid * 32; q0 < nseg; q0 += NT) {
                const int q = q0 + lane;
                const long long sm = q < nseg ? cur[q] : kMaxLL;
                if (q < nseg) nxt[q] = sm;
                const bool cand = seg_candidate(sm, R);
                if (!cand) mins = sm < mins ? sm : mins;  // untouched by the select
                unsigned cm = __ballot_sync(0xffffffffu, cand);
                __syncwarp();
                while (cm) {
                    const int qq = q0 + __ffs(cm) - 1;
                    cm &= cm - 1;
                    const long long p = (long long)qq * TAIL_SEG + 2 * lane;
                    const long long w0 = p < n ? w[p] : -1, w1 = p + 1 < n ? w[p + 1] : -1;
                    bool s0, s1;
                    if (R.minrule) {
                        s0 = w0 >= 0 && w0 <= R.minw;
                        s1 = w1 >= 0 && w1 <= R.minw;
                    } else {
                        s0 = w0 >= 0 && (w0 <= R.gle || mul_le(w0, R.Y, R.Xhi, R.Xlo));
                        s1 = w1 >= 0 && (w1 <= R.gle || mul_le(w1, R.Y, R.Xhi, R.Xlo));
                    }
                    long long m = kMaxLL;
                    if (w0 >= 0 && !s0) m = w0;
                    if (w1 >= 0 && !s1 && w1 < m) m = w1;
                    m = warp_min64(m);
                    if (lane == 0) {
                        nxt[qq] = m;
                        mins = m < mins ? m : mins;
                    }
                    const unsigned b0 = __ballot_sync(0xffffffffu, s0), b1 = __ballot_sync(0xffffffffu, s1);
                    if (b0 | b1) {
                        unsigned base = 0;
                        if (lane == 0) base = atomicAdd(&acc.F, (unsigned)(__popc(b0) + __popc(b1)));
                        base = __shfl_sync(0xffffffffu, base, 0);
                        const unsigned lt = (1u << lane) - 1u;
                        unsigned slot = base + __popc(b0 & lt) + __popc(b1 & lt);
                        if (s0) {
                            w[p] = -i;
                            if (NARROW) wlo += (unsigned long long)w0;
                            else add128(wlo, whi, (unsigned long long)w0, 0);
                            J.front[slot] = (int)p;
                            if (slot < TAIL_FAST) {
                                s_fs[slot] = rp[p];
                                s_fl[slot] = rp[p + 1] - rp[p];
                            }
                            slot++;
                        }
                        if (s1) {
                            w[p + 1] = -i;
                            if (NARROW) wlo += (unsigned long long)w1;
                            else add128(wlo, whi, (unsigned long long)w1, 0);
                            J.front[slot] = (int)(p + 1);
                            if (slot < TAIL_FAST) {
                                s_fs[slot] = rp[p + 1];
                                s_fl[slot] = rp[p + 2] - rp[p + 1];
                            }
                        }
                    }
                }
            }
            // the select's sums and minimum stay in registers until the expand's
            __syncthreads();
            if (tid == 0) s_acc[(i + 1) & 1].F = 0;
            const int F = (int)acc.F;
            // ---- expand: every arc of the frontier (heads read from global memory)
            unsigned long long ilo = 0, ihi = 0;
            long long mind = kMaxLL;
            auto arc = [&](long long pos) {
                const int v = arc_head(col[pos], hubs);
                const long long c = dg ? DUPIN_Q_ONE : cw[pos];
                const long long wv = w[v];
                if (wv >= 0) {
                    const long long old = (long long)atomicAdd((unsigned long long *)&w[v], (unsigned long long)(-c));
                    atomicMin(&nxt[v / TAIL_SEG], old - c);
                    mind = old - c < mind ? old - c : mind;
                } else if (wv == -i) {
                    if (NARROW) ilo += (unsigned long long)c;
                    else add128(ilo, ihi, (unsigned long long)c, 0);
                }
            };
            if (F <= TAIL_FAST) {
                // chunks of 32 consecutive arcs of one vertex, chunk c to warp
                // c % (NT / 32); the walk is the same in every lane of a warp
                int e = 0;
                long long cbase = 0, c = wid;
                long long a0 = F > 0 ? s_fs[0] : 0, ln = F > 0 ? s_fl[0] : 0;
                while (e < F) {
                    if (c >= cbase + ((ln + 31) >> 5)) {
                        cbase += (ln + 31) >> 5;
                        e++;
                        if (e < F) {
                            a0 = s_fs[e];
                            ln = s_fl[e];
                        }
                        continue;
                    }
                    const long long off = (c - cbase) * 32 + lane;
                    if (off < ln) arc(a0 + off);
                    c += NT / 32;
                }
            } else {
                for (int c0 = 0; c0 < F; c0 += NT) {
                    const int qq = c0 + tid;
                    long long deg = 0;
                    if (qq < F) {
                        const int p = J.front[qq];
                        deg = rp[p + 1] - rp[p];
                    }
                    long long tot;
                    long long ex = block_excl_scan<NT / 32>(deg, s_w, tot);
                    s_pref[tid] = ex;
                    const int nq = (F - c0) < NT ? (F - c0) : NT;
                    if (tid == 0) s_pref[nq] = tot;
                    __syncthreads();
                    for (long long x = tid; x < tot; x += NT) {
                        const int e = smem_last_le(s_pref, nq, x);
                        const int p = J.front[c0 + e];
                        arc(rp[p] + (x - s_pref[e]));
                    }
                    __syncthreads();
                }
            }
            if (NARROW) {
                if (__any_sync(0xffffffffu, wlo != 0)) wlo = warp_sum64_redux(wlo);
                if (__any_sync(0xffffffffu, ilo != 0)) ilo = warp_sum64_redux(ilo);
            } else {
                if (__any_sync(0xffffffffu, (wlo | whi) != 0)) warp_sum128(wlo, whi);
                if (__any_sync(0xffffffffu, (ilo | ihi) != 0)) warp_sum128(ilo, ihi);
            }
            mins = warp_min64(mind < mins ? mind : mins);
            if (lane == 0) {
                acc.wlo[wid] = wlo;
                acc.whi[wid] = whi;
                acc.ilo[wid] = ilo;
                acc.ihi[wid] = ihi;
                acc.mins[wid] = mins;
            }
            __syncthreads();
            // ---- every warp: close round i, plan round i + 1
            u128 wsel, internal;
            long long mins_all;
            tail_acc_sum<NT / 32, NARROW>(acc, wsel, internal, mins_all);
            st.f = st.f - (wsel - (internal >> 1));
            st.size -= F;
            st.round = i;
            st.n_min_rule += R.minrule ? 1 : 0;
            if (st.size > 0 && frac_gt<NARROW>(st.f, st.size, st.bf, st.best_size)) {
                st.bf = st.f;
                st.best_size = st.size;
                st.best_round = i;
            }
            if (tid == 0 && i < J.tr_cap) {
                J.tr_f_hi[i] = (long long)(unsigned long long)(st.f >> 64);
                J.tr_f_lo[i] = (unsigned long long)st.f;
                J.tr_size[i] = st.size;
                J.tr_peeled[i] = F;
            }
            if (F == 0) {
                err = DUPIN_ERR_NO_PROGRESS;
                break;
            }
            R = tail_plan<NARROW>(J.kD, J.D, J.use_min, J.gpo, J.lpo, st, mins_all);
        }
    };
    // f only decreases and starts as the best f
    if ((unsigned long long)(st.f >> 64) == 0 && (unsigned long long)st.f < (1ull << 62)) rounds(std::true_type{});
    else rounds(std::false_type{});
    __syncthreads();
    for (long long u = tid; u < n; u += NT) {
        const long long wv = w[u];
        J.pr[u] = wv < 0 ? (int)(-wv) : 0x7fffffff;
    }
    if (tid == 0) {
        J.out[0] = st.round;
        J.out[1] = st.best_round;
        J.out[2] = st.best_size;
        J.out[3] = (long long)(unsigned long long)(st.bf >> 64);
        J.out[4] = (long long)(unsigned long long)st.bf;
        J.out[5] = st.n_min_rule;
        J.out[6] = err;
        J.out[7] = 0;
    }
}

template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_peel_cta(const CtaJob *jobs, int njobs, int *next) {
    extern __shared__ __align__(16) long long s_seg[];  // 2 * CTA_MAX_SEG
    __shared__ TailAcc<NT / 32> s_acc[2];
    __shared__ long long s_w[(NT / 32)];
    __shared__ long long s_pref[NT + 1];
    __shared__ long long s_fs[TAIL_FAST], s_fl[TAIL_FAST];
    __shared__ int s_big[CTA_BIGLIST];
    __shared__ int s_nbig;
    __shared__ unsigned long long s_lo[(NT / 32)], s_hi[(NT / 32)];
    __shared__ int s_job;
    for (;;) {
        if (threadIdx.x == 0) s_job = atomicAdd(next, 1);
        __syncthreads();
        const int j = s_job;
        __syncthreads();
        if (j >= njobs) break;
        const CtaJob J = jobs[j];
        const int nseg = (int)((J.n + TAIL_SEG - 1) / TAIL_SEG);
        (void)nseg;
        cta_peel_one<NT>(J, s_seg, s_acc, s_w, s_pref, s_fs, s_fl, s_big, &s_nbig, s_lo, s_hi);
        __syncthreads();
    }
}

// the launch shapes: threads per CTA, CTAs per SM the kernel is bounded for
struct CtaShape {
    int threads;
    const void *fn;
};
static const CtaShape kCtaShapes[2] = {{128, (const void *)k_peel_cta<128, 4>}, {256, (const void *)k_peel_cta<256, 2>}};
// Per device: the shape of launches with more graphs than one wave of the
// widest shape holds ('large', tuned or default), or one shape for every
// launch ('forced').  A launch that fits one wave of 256-thread CTAs leaves
// SMs idle with either shape, so it takes the wider CTAs, which finish each
// graph sooner (the serving case: few requests per launch).
struct ShapeSel {
    int large = 0;
    bool forced = false;
};
static std::mutex g_shape_mu;
static std::map<int, ShapeSel> g_shape;
static thread_local int t_tune_shape = -1;  // the autotuner's shape under test

static ShapeSel shape_sel(int dev) {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    auto it = g_shape.find(dev);
    return it == g_shape.end() ? ShapeSel() : it->second;
}

static int cta_shape_for(int dev, size_t njobs, int sms) {
    if (t_tune_shape >= 0) return t_tune_shape;
    const ShapeSel sel = shape_sel(dev);
    if (sel.forced) return sel.large;
    return njobs <= (size_t)2 * sms ? 1 : sel.large;
}

static int set_cta_smem() {
    static bool done = false;
    if (done) return DUPIN_OK;
    for (const CtaShape &c : kCtaShapes) {
        cudaError_t e = cudaFuncSetAttribute(c.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(2 * CTA_MAX_SEG * sizeof(long long)));
        if (e != cudaSuccess) return dupin_cuda_fail(e, "cudaFuncSetAttribute(k_peel_cta)");
    }
    done = true;
    return DUPIN_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static long long trace_cap_of(const dupin_graph *g, const dupin_params &p) {
    const long long mr = p.max_rounds > 0 ? p.max_rounds : g->n + 1;
    return std::min<long long>(mr, g->n) + 1;
}

long long cta_graph_limit() { return CTA_MAX_N; }

// device bytes one graph takes in a batch arena
long long cta_job_bytes(const dupin_graph *g, const dupin_params *p) {
    const long long n = g->n;
    return (long long)(align256(8 * (size_t)n) + align256(4 * (size_t)n) + align256(4 * (size_t)n) +
                       align256(32 * (size_t)trace_cap_of(g, *p)) + 64 + sizeof(CtaJob) + 256);
}

struct CtaBatch {
    unsigned char *arena = nullptr;
    size_t nj = 0, outs_base = 0;
    std::vector<size_t> off_pr, off_tr;
    std::vector<long long> trcap;
    std::vector<int64_t> idx;
    dupin_graph *const *graphs = nullptr;
    const dupin_params *params = nullptr;
    dupin_result *results = nullptr;
};

// Enqueue one persistent launch for graphs[idx[k]] on stream s (no host
// synchronisation).  Results stay in the arena until cta_batch_finish.
int cta_batch_enqueue(dupin_graph *const *graphs, const dupin_params *params, dupin_result *results,
                      const std::vector<int64_t> &idx, cudaStream_t s, CtaBatch **out) {
    *out = nullptr;
    if (idx.empty()) return DUPIN_OK;
    int rc = set_cta_smem();
    if (rc) return rc;
    CtaBatch *B = new CtaBatch();
    B->graphs = graphs;
    B->params = params;
    B->results = results;
    B->idx = idx;
    const size_t nj = idx.size();
    B->nj = nj;
    std::vector<size_t> off_w(nj), off_f(nj);
    B->off_pr.resize(nj);
    B->off_tr.resize(nj);
    B->trcap.resize(nj);
    size_t at = align256(sizeof(CtaJob) * nj) + 256;
    B->outs_base = at;
    at = align256(at + 64 * nj);
    for (size_t k = 0; k < nj; k++) {
        const dupin_graph *g = graphs[idx[k]];
        const long long n = g->n;
        B->trcap[k] = trace_cap_of(g, params[idx[k]]);
        off_w[k] = at;
        at = align256(at + 8 * (size_t)n);
        off_f[k] = at;
        at = align256(at + 4 * (size_t)n);
        B->off_pr[k] = at;
        at = align256(at + 4 * (size_t)n);
        B->off_tr[k] = at;
        at = align256(at + 32 * (size_t)B->trcap[k]);
    }
    cudaError_t e = cudaMallocAsync((void **)&B->arena, at, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete B;
        return dupin_fail(e == cudaErrorMemoryAllocation ? DUPIN_ERR_OOM : DUPIN_ERR_CUDA,
                          std::string("batch arena: ") + cudaGetErrorString(e));
    }
    unsigned char *arena = B->arena;
    std::vector<CtaJob> jobs(nj);
    for (size_t k = 0; k < nj; k++) {
        const dupin_graph *g = graphs[idx[k]];
        const dupin_params &p = params[idx[k]];
        const DevGraph dgr = dev_graph(g, p.metric);
        CtaJob &J = jobs[k];
        J.n = g->n;
        J.arcs = g->arcs;
        J.rp = dgr.rp;
        J.col = dgr.col;
        J.cw = dgr.cw;
        J.a = dgr.a;
        J.hubs = dgr.hubs;
        J.kD = (long long)p.k_mult * (p.eps_den + p.eps_num);
        J.D = p.eps_den;
        J.max_rounds = p.max_rounds > 0 ? p.max_rounds : g->n + 1;
        J.use_min = J.kD < 2 * J.D ? 1 : 0;
        J.gpo = (p.flags & (DUPIN_GPO | DUPIN_LPO)) ? 1 : 0;
        J.lpo = (p.flags & DUPIN_LPO) ? 1 : 0;
        J.w = (long long *)(arena + off_w[k]);
        J.front = (int *)(arena + off_f[k]);
        const bool dev = (p.flags & DUPIN_RESULT_DEVICE) != 0;
        dupin_result &r = results[idx[k]];
        J.pr = (dev && r.peel_round) ? r.peel_round : (int *)(arena + B->off_pr[k]);
        long long *tr = (long long *)(arena + B->off_tr[k]);
        const long long tc = B->trcap[k];
        const bool user_tr = dev && r.trace_f_hi && r.trace_f_lo && r.trace_size && r.trace_peeled;
        J.tr_f_hi = user_tr ? (long long *)r.trace_f_hi : tr;
        J.tr_f_lo = user_tr ? (unsigned long long *)r.trace_f_lo : (unsigned long long *)(tr + tc);
        J.tr_size = user_tr ? (long long *)r.trace_size : tr + 2 * tc;
        J.tr_peeled = user_tr ? (long long *)r.trace_peeled : tr + 3 * tc;
        J.tr_cap = user_tr ? std::min<long long>(tc, r.trace_cap) : tc;
        J.out = (long long *)(arena + B->outs_base + 64 * k);
    }
    // largest graphs first: the queue hands them out before the small ones,
    // so the launch does not end waiting for a big graph started last
    {
        std::vector<size_t> order(nj);
        for (size_t k = 0; k < nj; k++) order[k] = k;
        std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
            return jobs[x].arcs + jobs[x].n > jobs[y].arcs + jobs[y].n;
        });
        std::vector<CtaJob> sorted(nj);
        for (size_t k = 0; k < nj; k++) sorted[k] = jobs[order[k]];
        jobs.swap(sorted);
    }
    int *next = (int *)(arena + align256(sizeof(CtaJob) * nj));
    int sms = 0, dev = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const CtaShape &shape = kCtaShapes[cta_shape_for(dev, nj, sms)];
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, shape.fn, shape.threads, 2 * CTA_MAX_SEG * sizeof(long long));
    if (occ < 1) occ = 1;
    const int grid = (int)std::min<long long>((long long)nj, (long long)sms * occ);
    e = cudaMemcpyAsync(arena, jobs.data(), sizeof(CtaJob) * nj, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(next, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        const CtaJob *jobs_dev = (const CtaJob *)arena;
        int njobs = (int)nj;
        void *args[] = {(void *)&jobs_dev, (void *)&njobs, (void *)&next};
        e = cudaLaunchKernel(shape.fn, dim3(grid), dim3(shape.threads), args, 2 * CTA_MAX_SEG * sizeof(long long), s);
    }
    if (e != cudaSuccess) {
        cudaFreeAsync(B->arena, s);
        delete B;
        return dupin_cuda_fail(e, "batched peel launch");
    }
    *out = B;
    return DUPIN_OK;
}

// Copy a finished batch's results into the callers' result structs and free
// its arena.  'status' gets the first failing graph's code (0 if none).
int cta_batch_finish(CtaBatch *B, cudaStream_t s, std::vector<int> *per_job_status) {
    if (!B) return DUPIN_OK;
    const size_t nj = B->nj;
    unsigned char *arena = B->arena;
    std::vector<long long> outs(8 * nj);
    cudaError_t e = cudaMemcpyAsync(outs.data(), arena + B->outs_base, 64 * nj, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int status = DUPIN_OK;
    std::string msg;
    if (per_job_status) per_job_status->assign(nj, DUPIN_OK);
    for (size_t k = 0; k < nj && e == cudaSuccess; k++) {
        const int64_t j = B->idx[k];
        const dupin_graph *g = B->graphs[j];
        const dupin_params &p = B->params[j];
        dupin_result &r = B->results[j];
        const long long *o = &outs[8 * k];
        r.n_rounds = o[0];
        r.n_min_rule = o[5];
        r.n_bulk_rounds = 0;
        for (int q = 0; q < 4; q++) r.phase_ms[q] = 0.f;
        if (o[6]) {
            if (per_job_status) (*per_job_status)[k] = (int)o[6];
            if (!status) {
                status = (int)o[6];
                msg = "graph " + std::to_string((long long)j) + ": max_rounds reached before the set became empty";
            }
            continue;
        }
        r.best_round = o[1];
        r.best_size = o[2];
        r.best_f_hi = o[3];
        r.best_f_lo = (unsigned long long)o[4];
        const u128 bf = mk128((unsigned long long)o[4], (unsigned long long)o[3]);
        r.best_density = o[2] > 0 ? (double)bf / 4294967296.0 / (double)o[2] : 0.0;
        const bool dev = (p.flags & DUPIN_RESULT_DEVICE) != 0;
        const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        const long long n = g->n;
        const int *pr_dev = dev && r.peel_round ? r.peel_round : (const int *)(arena + B->off_pr[k]);
        if (r.peel_round && !dev && n > 0) e = cudaMemcpyAsync(r.peel_round, pr_dev, 4 * (size_t)n, kind, s);
        const long long nt = o[0] + 1;
        const bool want_tr = r.trace_f_hi || r.trace_f_lo || r.trace_size || r.trace_peeled;
        const bool user_tr = dev && r.trace_f_hi && r.trace_f_lo && r.trace_size && r.trace_peeled;
        if (want_tr && !user_tr && e == cudaSuccess) {
            const long long cnt = std::min<long long>(nt, (long long)r.trace_cap);
            const long long *tr = (const long long *)(arena + B->off_tr[k]);
            const long long tc = B->trcap[k];
            if (cnt > 0) {
                if (r.trace_f_hi) e = cudaMemcpyAsync(r.trace_f_hi, tr, 8 * (size_t)cnt, kind, s);
                if (r.trace_f_lo && e == cudaSuccess) e = cudaMemcpyAsync(r.trace_f_lo, tr + tc, 8 * (size_t)cnt, kind, s);
                if (r.trace_size && e == cudaSuccess) e = cudaMemcpyAsync(r.trace_size, tr + 2 * tc, 8 * (size_t)cnt, kind, s);
                if (r.trace_peeled && e == cudaSuccess) e = cudaMemcpyAsync(r.trace_peeled, tr + 3 * tc, 8 * (size_t)cnt, kind, s);
            }
        }
        if (want_tr && r.trace_cap < nt) {
            if (per_job_status) (*per_job_status)[k] = DUPIN_ERR_BUFFER_TOO_SMALL;
            if (!status) {
                status = DUPIN_ERR_BUFFER_TOO_SMALL;
                msg = "graph " + std::to_string((long long)j) + ": trace_cap < n_rounds + 1";
            }
        }
        if (r.best_mask && n > 0 && e == cudaSuccess) {
            if (dev) {
                launch_mask(pr_dev, n, o[1], r.best_mask, s);
            } else {
                e = cudaStreamSynchronize(s);
                std::vector<int> tmp;
                const int *prh = r.peel_round;
                if (!prh) {
                    tmp.resize((size_t)n);
                    if (e == cudaSuccess) e = cudaMemcpy(tmp.data(), pr_dev, 4 * (size_t)n, cudaMemcpyDeviceToHost);
                    prh = tmp.data();
                }
                for (long long u = 0; u < n && e == cudaSuccess; u++) r.best_mask[u] = prh[u] > o[1] ? 1 : 0;
            }
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(arena, s);
    delete B;
    if (e != cudaSuccess) return dupin_cuda_fail(e, "batched peel");
    if (status) return dupin_fail(status, msg);
    return DUPIN_OK;
}

// Streams for concurrent tails, created once per device and reused.
// peels whose tails may overlap later grid-wide stages
#define TAIL_OVERLAP_MAX 8

static cudaStream_t tail_stream(int dev, size_t q) {
    static std::mutex mu;
    static std::map<int, std::vector<cudaStream_t>> pool;
    const size_t kMax = 32;
    std::lock_guard<std::mutex> lk(mu);
    std::vector<cudaStream_t> &v = pool[dev];
    const size_t want = std::min(q + 1, kMax);
    while (v.size() < want) {
        cudaStream_t t = nullptr;
        if (cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking) != cudaSuccess) break;
        v.push_back(t);
    }
    return v.empty() ? nullptr : v[q % v.size()];
}

// Several peels of large graphs (or of one graph under several parameter
// sets).  The initial weights are computed once per graph and metric; the
// grid-wide stages run one after another on 'stream' (each is a
// cooperative launch); each peel's tail sub-graph is built on 'stream' and
// its one-CTA tail runs on a stream of its own, so the latency-bound tails,
// one SM each, run side by side.  A graph that appears several times gets
// one cached workspace per appearance.
static int peel_large_concurrent(dupin_graph *const *graphs, const dupin_params *params, dupin_result *results,
                                 const std::vector<int64_t> &idx, cudaStream_t s) {
    const size_t k = idx.size();
    std::vector<PeelPlan> plans(k);
    std::vector<PeelWorkspace *> ws(k, nullptr);
    std::map<dupin_graph *, int> uses;
    int dev = 0;
    cudaGetDevice(&dev);
    auto fail_at = [&](size_t q, int rc) {
        char buf[512];
        dupin_last_error(buf, sizeof(buf));
        return dupin_fail(rc, "graph " + std::to_string((long long)idx[q]) + ": " + buf);
    };
    for (size_t q = 0; q < k; q++) {
        dupin_graph *g = graphs[idx[q]];
        if (g->device != dev) return dupin_fail(DUPIN_ERR_INVALID_ARG, "batched graphs must live on the current device");
        int rc = peel_resolve(g, &params[idx[q]], &plans[q]);
        if (rc) return fail_at(q, rc);
        ws[q] = workspace_slot(g, uses[g]++, plans[q], &rc);
        if (rc) return fail_at(q, rc);
    }
    // initial weights: once per (graph, metric); the other peels of the pair
    // copy them (before any grid-wide round changes them)
    for (size_t q = 0; q < k; q++) {
        const PeelWorkspace *from = nullptr;
        for (size_t q2 = 0; q2 < q && !from; q2++)
            if (graphs[idx[q2]] == graphs[idx[q]] && params[idx[q2]].metric == params[idx[q]].metric) from = ws[q2];
        int rc = enqueue_peel_stages(graphs[idx[q]], ws[q], &params[idx[q]], plans[q], PEEL_INIT, s, from);
        if (rc) return fail_at(q, rc);
    }
    // With few peels, peel q's grid-wide stage runs beside the tails of peels
    // 0 .. q-1 on one block per SM fewer per SM a running tail may hold (one
    // for the one-CTA tail, the cluster's CTAs for the cluster tail), so that
    // its cooperative grid always fits; with many peels every grid-wide stage
    // runs first, on all SMs, and the tails after them.
    const int cl_sms = cluster_ctas();
    bool overlap = k <= TAIL_OVERLAP_MAX;
    {
        long long held = 0;
        for (size_t q = 0; q + 1 < k; q++) held += plans[q].cl_cap > 0 ? cl_sms : 1;
        if (overlap && ws[0] && held > ws[0]->grid / 2) overlap = false;
    }
    if (!overlap) {
        for (size_t q = 0; q < k; q++) {
            int rc = enqueue_peel_stages(graphs[idx[q]], ws[q], &params[idx[q]], plans[q], PEEL_BULK, s);
            if (rc) return fail_at(q, rc);
        }
    }
    std::vector<cudaEvent_t> ev(2 * k, nullptr);
    int rc = DUPIN_OK;
    int held = 0;  // SMs the tails queued so far may hold
    for (size_t q = 0; q < k && rc == DUPIN_OK; q++) {
        if (overlap) {
            const int grid = ws[q]->grid - held;
            rc = enqueue_peel_stages(graphs[idx[q]], ws[q], &params[idx[q]], plans[q], PEEL_BULK, s, nullptr,
                                     grid > 0 ? grid : 1);
            if (rc) break;
            // the later peels' grid-wide rounds run narrow beside this one's tail if it is a cluster
            for (size_t q2 = q + 1; q2 < k; q2++) enqueue_note_cluster(ws[q], ws[q2], s);
        }
        rc = enqueue_peel_stages(graphs[idx[q]], ws[q], &params[idx[q]], plans[q], PEEL_BUILD, s);
        if (rc) break;
        cudaStream_t t = tail_stream(dev, q);
        if (!t) {
            rc = dupin_fail(DUPIN_ERR_CUDA, "could not create a stream for the tails");
            break;
        }
        cudaError_t e = cudaEventCreateWithFlags(&ev[2 * q], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[2 * q + 1], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2 * q], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(t, ev[2 * q], 0);
        if (e != cudaSuccess) {
            rc = dupin_cuda_fail(e, "tail stream setup");
            break;
        }
        rc = enqueue_peel_stages(graphs[idx[q]], ws[q], &params[idx[q]], plans[q], PEEL_TAIL, t);
        if (rc) break;
        held += plans[q].cl_cap > 0 ? cl_sms : 1;
        e = cudaEventRecord(ev[2 * q + 1], t);
        if (e != cudaSuccess) rc = dupin_cuda_fail(e, "tail stream join");
    }
    // join the tails only after all of them are queued: a join inside the loop
    // would queue each build behind the previous tail
    for (size_t q = 0; q < k && rc == DUPIN_OK; q++) {
        cudaError_t e = cudaStreamWaitEvent(s, ev[2 * q + 1], 0);
        if (e != cudaSuccess) rc = dupin_cuda_fail(e, "tail stream join");
    }
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    if (rc) return rc;
    for (size_t q = 0; q < k; q++) {
        rc = peel_finish(graphs[idx[q]], ws[q], &params[idx[q]], &results[idx[q]], s);
        if (rc) return fail_at(q, rc);
    }
    return DUPIN_OK;
}

extern "C" int dupin_peel_batch(dupin_graph *const *graphs, const dupin_params *params, dupin_result *results,
                                int64_t count, void *stream) {
    if (count < 0) return dupin_fail(DUPIN_ERR_INVALID_ARG, "count < 0");
    if (count > 0 && (!graphs || !params || !results))
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "graphs, params and results must be non-NULL");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int64_t> cta, big;
    for (int64_t j = 0; j < count; j++) {
        if (!graphs[j]) return dupin_fail(DUPIN_ERR_INVALID_ARG, "graph " + std::to_string((long long)j) + " is NULL");
        PeelPlan plan;
        int rc = peel_resolve(graphs[j], &params[j], &plan);
        if (rc == DUPIN_OK && is_clique_metric(params[j].metric))
            rc = dupin_fail(DUPIN_ERR_INVALID_ARG, "the clique metrics (TDS, kCLiDS) are served by dupin_peel only");
        if (rc) {
            char buf[512];
            dupin_last_error(buf, sizeof(buf));
            return dupin_fail(rc, "graph " + std::to_string((long long)j) + ": " + buf);
        }
        if (graphs[j]->n >= 1 && graphs[j]->n <= CTA_MAX_N) cta.push_back(j);
        else big.push_back(j);
    }
    CtaBatch *B = nullptr;
    int rc = cta_batch_enqueue(graphs, params, results, cta, s, &B);
    if (rc) return rc;
    rc = cta_batch_finish(B, s, nullptr);
    if (rc) return rc;
    if (big.size() > 1) return peel_large_concurrent(graphs, params, results, big, s);
    for (int64_t j : big) {
        rc = dupin_peel(graphs[j], &params[j], &results[j], stream);
        if (rc) {
            char buf[512];
            dupin_last_error(buf, sizeof(buf));
            return dupin_fail(rc, "graph " + std::to_string((long long)j) + ": " + buf);
        }
    }
    return DUPIN_OK;
}

extern "C" int dupin_batch_set_threads(int threads) {
    ShapeSel sel;
    if (threads == 128) sel = ShapeSel{0, true};
    else if (threads == 256) sel = ShapeSel{1, true};
    else if (threads != 0) return dupin_fail(DUPIN_ERR_INVALID_ARG, "threads must be 0, 128 or 256");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return dupin_cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_shape_mu);
    g_shape[dev] = sel;
    return DUPIN_OK;
}

extern "C" int dupin_batch_get_threads(int *threads) {
    if (!threads) return dupin_fail(DUPIN_ERR_INVALID_ARG, "threads is NULL");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return dupin_cuda_fail(e, "cudaGetDevice");
    *threads = kCtaShapes[shape_sel(dev).large].threads;
    return DUPIN_OK;
}

// The autotuner: time every launch shape on the caller's own batch and keep
// the fastest for this device's launches of more than one wave.
extern "C" int dupin_batch_tune(dupin_graph *const *graphs, const dupin_params *params, int64_t count,
                                void *stream, int *threads) {
    if (count < 0) return dupin_fail(DUPIN_ERR_INVALID_ARG, "count < 0");
    if (count > 0 && (!graphs || !params)) return dupin_fail(DUPIN_ERR_INVALID_ARG, "graphs and params must be non-NULL");
    std::vector<dupin_graph *> gs;
    std::vector<dupin_params> ps;
    for (int64_t j = 0; j < count; j++) {
        if (!graphs[j]) return dupin_fail(DUPIN_ERR_INVALID_ARG, "graph " + std::to_string((long long)j) + " is NULL");
        if (graphs[j]->n < 1 || graphs[j]->n > CTA_MAX_N) continue;
        dupin_params p = params[j];
        p.flags &= ~DUPIN_RESULT_DEVICE;  // results stay in the batch arena
        gs.push_back(graphs[j]);
        ps.push_back(p);
    }
    if (gs.empty()) return dupin_fail(DUPIN_ERR_INVALID_ARG, "no graph of the batch fits one CTA");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return dupin_cuda_fail(e, "cudaGetDevice");
    std::vector<dupin_result> res(gs.size());
    const int nshape = (int)(sizeof(kCtaShapes) / sizeof(kCtaShapes[0]));
    std::vector<double> best(nshape, 1e300);
    int rc = DUPIN_OK;
    for (int rep = 0; rep < 3 && rc == DUPIN_OK; rep++) {
        for (int i = 0; i < nshape && rc == DUPIN_OK; i++) {
            t_tune_shape = i;
            memset(res.data(), 0, sizeof(dupin_result) * res.size());
            const auto t0 = std::chrono::steady_clock::now();
            rc = dupin_peel_batch(gs.data(), ps.data(), res.data(), (int64_t)gs.size(), stream);
            const double t = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            t_tune_shape = -1;
            if (rep > 0) best[i] = std::min(best[i], t);  // the first pass warms up
        }
    }
    if (rc) return rc;
    int pick = 0;
    for (int i = 1; i < nshape; i++)
        if (best[i] < best[pick]) pick = i;
    {
        std::lock_guard<std::mutex> lk(g_shape_mu);
        g_shape[dev] = ShapeSel{pick, false};
    }
    if (threads) *threads = kCtaShapes[pick].threads;
    return DUPIN_OK;
}
