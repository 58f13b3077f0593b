// cluster.cu -- the tail of a peel (Algorithm 2, Sec. 4.1, with Algorithms 3
// and 4 of Sec. 5) on a thread-block cluster of C CTAs (C = 16 where the
// device allows a cluster that large, else 8).
//
// Once the live set S fits the cluster's shared memory, the rounds left
// are many and small (k(1+eps) < 2 removes a few vertices per round on a
// skewed graph), so a grid-wide round pays three grid barriers for little
// work and the one-CTA tail is limited by the arcs one SM can fetch.  Here
// the live sub-graph's vertex state is spread over the cluster's shared
// memory: local vertex p (0 <= p < L, the tail sub-graph's numbering) is
// owned by CTA p mod C at slot p / C, which holds its peeling weight (>= 0
// while live, -i once removed in round i) and its arc range.  A round:
//
//   S  every CTA selects from its own slots (64-slot segments with an exact
//      minimum each, double-buffered by round parity, so only segments that
//      can hold a selected vertex are scanned), lists the selected slots and
//      the prefix of their arc counts, and publishes its partial results;
//   -- cluster barrier --
//   E  the round's arcs, concatenated over the CTAs' lists, are split evenly
//      over the CTAs; each arc u -> v reads v's state in its owner's shared
//      memory, subtracts c_uv with a returning 64-bit atomic add there when v
//      survives (and marks v's segment dirty with a 32-bit atomic OR), or adds
//      c_uv to the sum over arcs inside U_i when v left in this round;
//   -- cluster barrier --
//   C  every CTA reads all partials and closes the round identically:
//      f_i = f_{i-1} - (sum_{u in U_i} w_u - internal/2), |S_i|, the best prefix,
//      the exact minimum live weight (survivors' minima before the round and
//      every decrement's result), and plans round i+1.
//
// Before its next select every CTA recomputes the exact minimum of each of
// its dirty segments.  (A 64-bit atomic minimum on another CTA's shared
// memory was measured to lose updates when several SMs hit one word; 64-bit
// adds and 32-bit ORs there stay atomic, so only those are used remotely.)
//
// Partials are double-buffered by round parity: round i+2 writes a buffer
// only after the barrier that every CTA reaches after closing round i.
// Every decision that ends the loop is taken from cluster-wide totals, so all
// CTAs leave together; a last barrier keeps every CTA's shared memory alive
// until no other CTA can read it.  All arithmetic is exact integer
// arithmetic, identical to the one-CTA tail's.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "dupin_internal.h"
#include "peel_device.cuh"

#define CL_THREADS 256
#define CL_WARPS (CL_THREADS / 32)
#define CL_SEG 64
#define CL_WIN 512  // frontier entries per expand window
#define CL_ILP 4    // arcs in flight per thread in the expand
#define CL_MAXSEG 1024  // segments per CTA (slots are 16-bit: at most 65,536 per CTA)
static const long long kPad = (long long)0x8000000000000000ULL;  // slots past the owned ones

// ------------------------------------------------------------- cluster PTX

__device__ __forceinline__ unsigned cl_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cl_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// all threads of every CTA of the cluster; release/acquire orders the
// shared-memory writes (local and remote) before it against reads after it
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// the shared::cluster address of 'p' (this CTA's shared memory) in CTA 'rank'
__device__ __forceinline__ uint32_t cl_map(const void *p, unsigned rank) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t o;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(o) : "r"(a), "r"(rank));
    return o;
}

__device__ __forceinline__ long long cl_ld_s64(uint32_t a) {
    long long v;
    asm volatile("ld.shared::cluster.s64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long cl_ld_u64(uint32_t a) {
    unsigned long long v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ unsigned cl_ld_u32(uint32_t a) {
    unsigned v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ unsigned cl_ld_u16(uint32_t a) {
    unsigned short v;
    asm volatile("ld.shared::cluster.u16 %0, [%1];" : "=h"(v) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long cl_atom_add_u64(uint32_t a, unsigned long long x) {
    unsigned long long v;
    asm volatile("atom.shared::cluster.add.u64 %0, [%1], %2;" : "=l"(v) : "r"(a), "l"(x) : "memory");
    return v;
}

// an empty instruction that reads x: the thread waits for x's producer here
__device__ __forceinline__ void consume(unsigned x) { asm volatile("" ::"r"(x)); }

__device__ __forceinline__ unsigned cl_atom_or_b32(uint32_t a, unsigned x) {
    unsigned v;
    asm volatile("atom.shared::cluster.or.b32 %0, [%1], %2;" : "=r"(v) : "r"(a), "r"(x) : "memory");
    return v;
}

// Largest k in [0, U] with le(k) true, for a predicate that is true on a
// prefix of [0, U] and at k = 0.  One warp, 32 probes per step.
template <class LeF>
__device__ __forceinline__ long long warp_search_last_le_fn(long long U, LeF le) {
    const int lane = threadIdx.x & 31;
    long long lo = 0, hi = U;
    while (lo < hi) {
        const long long span = hi - lo;  // candidates lo+1 .. hi
        long long p;
        if (span <= 32) p = lo + 1 + lane;
        else p = lo + 1 + (long long)(((unsigned long long)(span - 1) * (unsigned)lane) / 31u);
        const bool valid = p <= hi;
        const bool ok = valid && le(p);
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (m == 0) {
            hi = __shfl_sync(0xffffffffu, p, 0) - 1;
        } else {
            const int Lh = 31 - __clz(m);
            const long long pl = __shfl_sync(0xffffffffu, p, Lh);
            const long long pn = __shfl_sync(0xffffffffu, p, Lh < 31 ? Lh + 1 : 31);
            const bool nvalid = __shfl_sync(0xffffffffu, (int)valid, Lh < 31 ? Lh + 1 : 31);
            lo = pl;
            if (Lh < 31 && nvalid) hi = pn - 1;
        }
    }
    return lo;
}

// ------------------------------------------------------------ shared state

// One CTA's partial results of a round (written by its thread 0).
struct ClPart {
    unsigned cnt;                    // vertices selected
    unsigned arcs;                   // their arcs
    unsigned long long wlo, whi;     // sum of their peeling weights
    long long mins;                  // minimum over the CTA's survivors before the decrements
    unsigned long long ilo, ihi;     // expand: sum of c over arcs inside U
    long long mind;                  // expand: minimum weight after a decrement
};

struct ClShared {
    ClPart part[2];                 // by round parity
    unsigned F[2];                  // frontier counter, by round parity
    long long initmin;              // the CTA's minimum live weight at the start
    long long red_mn[CL_WARPS];
    unsigned long long red_lo[CL_WARPS], red_hi[CL_WARPS];
    long long scan[CL_WARPS];
    unsigned wbase[CL_WIN + 1];     // expand window: arc prefix of entries e0 ..
    unsigned wstart[CL_WIN + 1];    // ... and their first arcs in the sub-graph
    long long win_e0;
    unsigned dirty[CL_MAXSEG / 32];  // segments whose vertices lost weight in the last expand
    int err;
};

// Dynamic shared memory per CTA for P slots (P a multiple of CL_SEG):
// tw (8 B), arc start and degree (4 + 4 B), frontier slot (2 B), frontier
// arc prefix (4 B) per slot, two segment minima per segment.
__host__ __device__ __forceinline__ long long cl_smem_bytes(long long P) {
    const long long nseg = P / CL_SEG;
    return 8 * P + 4 * P + 4 * P + 16 * nseg + 4 * (P + 1) + 2 * P + 16;
}

// ------------------------------------------------------------------ kernel

__device__ __forceinline__ long long block_min64(long long x, long long *s) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    x = warp_min64(x);
    __syncthreads();
    if (lane == 0) s[wid] = x;
    __syncthreads();
    long long m = lane < CL_WARPS ? s[lane] : kMaxLL;
    m = warp_min64(m);
    return m;
}

__global__ void __launch_bounds__(CL_THREADS, 1) k_peel_cluster(PeelArgs A, int P) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ClShared S;
    PeelCtl *ctl = A.ctl;
    if (ctl->status != ST_CLUSTER || ctl->error) return;  // identical in every CTA
    const unsigned C = cl_size(), r = cl_rank();
    const int lg = C == 16 ? 4 : (C == 8 ? 3 : (C == 4 ? 2 : (C == 2 ? 1 : 0)));
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const long long L = ctl->live_len;
    const int *live = ctl->live_sel ? A.live1 : A.live0;
    const long long nown = L > (long long)r ? (L - (long long)r + C - 1) / C : 0;
    const int nseg = P / CL_SEG;                      // segment minima buffers hold nseg entries
    const int nsl = (int)((nown + CL_SEG - 1) / CL_SEG);  // segments that hold this CTA's vertices
    long long *tw = (long long *)smem;                           // [P]
    unsigned *tst = (unsigned *)(smem + 8 * (size_t)P);          // [P] first arc
    unsigned *tdg = tst + P;                                     // [P] arcs
    long long *segbuf = (long long *)(tdg + P);                  // [2 nseg]
    unsigned *fpre = (unsigned *)(segbuf + 2 * nseg);            // [P + 1]
    unsigned short *fl = (unsigned short *)(fpre + P + 1);       // [P]
    const bool dg = A.tcw == nullptr;
    const int *tcol = A.tcol;
    const long long *tcw = A.tcw;

    // this CTA's slots: weights, arc ranges
    for (long long s = tid; s < P; s += CL_THREADS) {
        if (s < nown) {
            const long long p = s * C + r;
            tw[s] = A.w[live[p]];
            const long long a0 = A.tlrp[p], a1 = A.tlrp[p + 1];
            tst[s] = (unsigned)a0;
            tdg[s] = (unsigned)(a1 - a0);
        } else {
            tw[s] = kPad;
            tst[s] = 0;
            tdg[s] = 0;
        }
    }
    RoundState st;  // identical in every thread of every CTA
    st.round = ctl->round;
    st.size = ctl->size;
    st.f = mk128(ctl->f_lo, ctl->f_hi);
    st.best_round = ctl->best_round;
    st.best_size = ctl->best_size;
    st.bf = mk128(ctl->bf_lo, ctl->bf_hi);
    st.gpo_le = ctl->gpo_le;
    st.gpo_lt = ctl->gpo_lt;
    st.gm_f = 0;
    st.gm_s = 0;
    st.n_min_rule = ctl->n_min_rule;
    st.scan = ctl->scan_volume;
    if (tid == 0) {
        S.F[0] = 0;
        S.F[1] = 0;
        S.err = 0;
    }
    for (int k = tid; k < CL_MAXSEG / 32; k += CL_THREADS) S.dirty[k] = 0;
    __syncthreads();
    // round i reads the minima in buffer (i & 1)
    {
        long long *first = segbuf + ((st.round + 1) & 1) * nseg;
        long long mn = kMaxLL;
        for (int q = wid; q < nsl; q += CL_WARPS) {
            const longlong2 v = *(const longlong2 *)&tw[(long long)q * CL_SEG + 2 * lane];
            long long m = kMaxLL;
            if (v.x >= 0) m = v.x;
            if (v.y >= 0 && v.y < m) m = v.y;
            m = warp_min64(m);
            if (lane == 0) first[q] = m;
            mn = m < mn ? m : mn;
        }
        mn = block_min64(mn, S.red_mn);
        if (tid == 0) S.initmin = mn;
    }
    cl_sync();
    long long m0 = kMaxLL;
    if (lane < (int)C) m0 = cl_ld_s64(cl_map(&S.initmin, lane));
    m0 = warp_min64(m0);
    TailRound R = tail_plan<false>(A.kD, A.D, A.use_min, A.gpo, A.lpo, st, m0);
    int err = 0;
    while (!R.done) {
        if (R.i > A.max_rounds) {
            err = DUPIN_ERR_NO_PROGRESS;
            break;
        }
        const long long i = R.i;
        const int par = (int)(i & 1);
        long long *cur = segbuf + par * nseg;
        long long *nxt = segbuf + (par ^ 1) * nseg;
        // ---- the exact minimum of every segment the last expand touched
        for (int q = wid; q < nsl; q += CL_WARPS) {
            if (!((S.dirty[q >> 5] >> (q & 31)) & 1u)) continue;  // warp-uniform
            const longlong2 v = *(const longlong2 *)&tw[(long long)q * CL_SEG + 2 * lane];
            long long m = kMaxLL;
            if (v.x >= 0) m = v.x;
            if (v.y >= 0 && v.y < m) m = v.y;
            m = warp_min64(m);
            if (lane == 0) cur[q] = m;
        }
        __syncthreads();
        for (int k = tid; k < (nsl + 31) / 32; k += CL_THREADS) S.dirty[k] = 0;
        // ---- S: select this CTA's slots
        unsigned long long wlo = 0, whi = 0;
        long long mins = kMaxLL;  // survivors' minimum over the segments this lane looked at
        for (int q0 = wid * 32; q0 < nsl; q0 += CL_THREADS) {
            const int q = q0 + lane;
            const long long sm = q < nsl ? cur[q] : kMaxLL;
            if (q < nsl) nxt[q] = sm;
            const bool cand = seg_candidate(sm, R);
            if (!cand) mins = sm < mins ? sm : mins;
            unsigned cm = __ballot_sync(0xffffffffu, cand);
            __syncwarp();  // every lane's copy above lands before lane 0 overwrites a scanned segment's minimum
            while (cm) {
                const int qq = q0 + __ffs(cm) - 1;
                cm &= cm - 1;
                const long long p = (long long)qq * CL_SEG + 2 * lane;
                const longlong2 v = *(const longlong2 *)&tw[p];
                bool s0, s1;
                if (R.minrule) {
                    s0 = v.x >= 0 && v.x <= R.minw;
                    s1 = v.y >= 0 && v.y <= R.minw;
                } else {
                    s0 = v.x >= 0 && (v.x <= R.gle || mul_le(v.x, R.Y, R.Xhi, R.Xlo));
                    s1 = v.y >= 0 && (v.y <= R.gle || mul_le(v.y, R.Y, R.Xhi, R.Xlo));
                }
                long long m = kMaxLL;
                if (v.x >= 0 && !s0) m = v.x;
                if (v.y >= 0 && !s1 && v.y < m) m = v.y;
                m = warp_min64(m);
                if (lane == 0) {
                    nxt[qq] = m;
                    mins = m < mins ? m : mins;
                }
                const unsigned b0 = __ballot_sync(0xffffffffu, s0), b1 = __ballot_sync(0xffffffffu, s1);
                if (b0 | b1) {
                    unsigned base = 0;
                    if (lane == 0) base = atomicAdd(&S.F[par], (unsigned)(__popc(b0) + __popc(b1)));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    const unsigned lt = (1u << lane) - 1u;
                    unsigned slot = base + __popc(b0 & lt) + __popc(b1 & lt);
                    if (s0) {
                        tw[p] = -i;
                        add128(wlo, whi, (unsigned long long)v.x, 0);
                        fl[slot++] = (unsigned short)p;
                    }
                    if (s1) {
                        tw[p + 1] = -i;
                        add128(wlo, whi, (unsigned long long)v.y, 0);
                        fl[slot] = (unsigned short)(p + 1);
                    }
                }
            }
        }
        __syncthreads();
        const unsigned F = S.F[par];
        if (tid == 0) S.F[par ^ 1] = 0;  // round i+1's counter (last read in round i-1)
        // the frontier's arc prefix
        {
            unsigned carry = 0;
            for (unsigned e0 = 0; e0 < F; e0 += CL_THREADS) {
                const unsigned e = e0 + tid;
                const long long d = e < F ? (long long)tdg[fl[e]] : 0;
                long long tot;
                const long long ex = block_excl_scan<CL_WARPS>(d, S.scan, tot);
                if (e < F) fpre[e] = carry + (unsigned)ex;
                carry += (unsigned)tot;
            }
            if (tid == 0) fpre[F] = carry;
        }
        warp_sum128(wlo, whi);
        mins = warp_min64(mins);
        if (lane == 0) {
            S.red_lo[wid] = wlo;
            S.red_hi[wid] = whi;
            S.red_mn[wid] = mins;
        }
        __syncthreads();
        if (wid == 0) {
            unsigned long long l = lane < CL_WARPS ? S.red_lo[lane] : 0, h = lane < CL_WARPS ? S.red_hi[lane] : 0;
            long long m = lane < CL_WARPS ? S.red_mn[lane] : kMaxLL;
            warp_sum128(l, h);
            m = warp_min64(m);
            if (lane == 0) {
                ClPart &pp = S.part[par];
                pp.cnt = F;
                pp.arcs = fpre[F];
                pp.wlo = l;
                pp.whi = h;
                pp.mins = m;
            }
        }
        cl_sync();  // A: every CTA's selection, list and partials are visible
        // ---- E: expand the round's arcs, split evenly over the CTAs
        unsigned long long ilo = 0, ihi = 0;
        long long mind = kMaxLL;
        {
            // per-CTA arc counts -> exclusive prefix (every warp holds it in lanes 0..C-1)
            unsigned a = 0;
            if (lane < (int)C) a = cl_ld_u32(cl_map(&S.part[par].arcs, lane));
            unsigned incl = a;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned o = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += o;
            }
            const unsigned Atot = __shfl_sync(0xffffffffu, incl, 31);
            const unsigned excl = incl - a;
            const unsigned E0 = (unsigned)split_at(Atot, r, C), E1 = (unsigned)split_at(Atot, r + 1, C);
            unsigned x = E0;
            while (x < E1) {  // block-uniform
                // owner CTA q of global arc x and its local arc index
                const unsigned m = __ballot_sync(0xffffffffu, lane < (int)C && excl <= x && a > 0 && x < excl + a);
                if (m == 0) {  // cannot happen for x < Atot; leave the expand rather than map rank -1
                    if (tid == 0) S.err = DUPIN_ERR_CUDA;
                    break;
                }
                const int q = __ffs(m) - 1;
                const unsigned qbase = __shfl_sync(0xffffffffu, excl, q), qcnt = __shfl_sync(0xffffffffu, a, q);
                const unsigned lo = x - qbase;
                const unsigned hi = (E1 - qbase < qcnt ? E1 - qbase : qcnt);
                const unsigned Fq = cl_ld_u32(cl_map(&S.part[par].cnt, q));
                const uint32_t rfpre = cl_map(fpre, q), rfl = cl_map(fl, q), rtst = cl_map(tst, q);
                // the window's first entry: the last e with fpre_q[e] <= lo
                // (fpre_q[0] = 0 <= lo < fpre_q[Fq]); warp 0, 32 probes a step
                if (wid == 0) {
                    const long long e = warp_search_last_le_fn(
                        (long long)Fq - 1, [&](long long k) { return cl_ld_u32(rfpre + 4 * (uint32_t)k) <= lo; });
                    if (lane == 0) S.win_e0 = e;
                }
                __syncthreads();
                const long long e0 = S.win_e0;
                for (int t = tid; t <= CL_WIN; t += CL_THREADS) {
                    const long long e = e0 + t;
                    unsigned b = 0xffffffffu, s0 = 0;
                    if (e <= (long long)Fq) b = cl_ld_u32(rfpre + 4 * (uint32_t)e);
                    if (e < (long long)Fq) s0 = cl_ld_u32(rtst + 4 * cl_ld_u16(rfl + 2 * (uint32_t)e));
                    S.wbase[t] = e <= (long long)Fq ? b : 0xffffffffu;
                    S.wstart[t] = s0;
                }
                __syncthreads();
                const unsigned wend = S.wbase[CL_WIN] < hi ? S.wbase[CL_WIN] : hi;
                for (unsigned xb = lo + tid; xb < wend; xb += CL_ILP * CL_THREADS) {
                    long long pos[CL_ILP];
#pragma unroll
                    for (int u = 0; u < CL_ILP; u++) {
                        const unsigned xx = xb + u * CL_THREADS;
                        pos[u] = -1;
                        if (xx < wend) {
                            int lo2 = 0, hi2 = CL_WIN;  // last t with wbase[t] <= xx
                            while (lo2 < hi2) {
                                const int mid = (lo2 + hi2 + 1) >> 1;
                                if (S.wbase[mid] <= xx) lo2 = mid;
                                else hi2 = mid - 1;
                            }
                            pos[u] = (long long)S.wstart[lo2] + (xx - S.wbase[lo2]);
                        }
                    }
                    int cv[CL_ILP];
                    long long cc[CL_ILP];
#pragma unroll
                    for (int u = 0; u < CL_ILP; u++) {
                        if (pos[u] >= 0) {
                            cv[u] = tcol[pos[u]];
                            cc[u] = dg ? DUPIN_Q_ONE : tcw[pos[u]];
                        }
                    }
                    long long wv[CL_ILP];
                    uint32_t wa[CL_ILP];
#pragma unroll
                    for (int u = 0; u < CL_ILP; u++) {
                        if (pos[u] >= 0) {
                            wa[u] = cl_map(&tw[cv[u] >> lg], (unsigned)cv[u] & (C - 1));
                            wv[u] = cl_ld_s64(wa[u]);
                        }
                    }
                    long long nv[CL_ILP];
#pragma unroll
                    for (int u = 0; u < CL_ILP; u++) {
                        nv[u] = kMaxLL;
                        if (pos[u] < 0) continue;
                        if (wv[u] >= 0) {
                            nv[u] = (long long)cl_atom_add_u64(wa[u], (unsigned long long)(-cc[u])) - cc[u];
                            mind = nv[u] < mind ? nv[u] : mind;
                        } else if (wv[u] == -i) {
                            add128(ilo, ihi, (unsigned long long)cc[u], 0);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < CL_ILP; u++) {
                        if (nv[u] != kMaxLL) {
                            const int sg = (cv[u] >> lg) / CL_SEG;
                            // the returned word is consumed, so the OR has been
                            // performed at its target before this thread reaches
                            // the next cluster barrier
                            consume(cl_atom_or_b32(cl_map(&S.dirty[sg >> 5], (unsigned)cv[u] & (C - 1)), 1u << (sg & 31)));
                        }
                    }
                }
                x = qbase + wend;
                __syncthreads();  // the window is reused
            }
        }
        warp_sum128(ilo, ihi);
        mind = warp_min64(mind);
        if (lane == 0) {
            S.red_lo[wid] = ilo;
            S.red_hi[wid] = ihi;
            S.red_mn[wid] = mind;
        }
        __syncthreads();
        if (wid == 0) {
            unsigned long long l = lane < CL_WARPS ? S.red_lo[lane] : 0, h = lane < CL_WARPS ? S.red_hi[lane] : 0;
            long long m = lane < CL_WARPS ? S.red_mn[lane] : kMaxLL;
            warp_sum128(l, h);
            m = warp_min64(m);
            if (lane == 0) {
                S.part[par].ilo = l;
                S.part[par].ihi = h;
                S.part[par].mind = m;
            }
        }
        cl_sync();  // B: every decrement and partial of round i is visible
        // ---- C: close round i and plan round i+1 (every warp, same values)
        unsigned long long Wl = 0, Wh = 0, Il = 0, Ih = 0;
        long long Un = 0, Mn = kMaxLL;
        if (lane < (int)C) {
            const uint32_t pa = cl_map(&S.part[par], lane);
            Un = cl_ld_u32(pa + offsetof(ClPart, cnt));
            Wl = cl_ld_u64(pa + offsetof(ClPart, wlo));
            Wh = cl_ld_u64(pa + offsetof(ClPart, whi));
            Il = cl_ld_u64(pa + offsetof(ClPart, ilo));
            Ih = cl_ld_u64(pa + offsetof(ClPart, ihi));
            const long long m1 = cl_ld_s64(pa + offsetof(ClPart, mins)), m2 = cl_ld_s64(pa + offsetof(ClPart, mind));
            Mn = m1 < m2 ? m1 : m2;
        }
        Un = warp_sum64(Un);
        Un = __shfl_sync(0xffffffffu, Un, 0);
        warp_sum128(Wl, Wh);
        warp_sum128(Il, Ih);
        Wl = __shfl_sync(0xffffffffu, Wl, 0);
        Wh = __shfl_sync(0xffffffffu, Wh, 0);
        Il = __shfl_sync(0xffffffffu, Il, 0);
        Ih = __shfl_sync(0xffffffffu, Ih, 0);
        Mn = warp_min64(Mn);
        const u128 wsel = mk128(Wl, Wh), internal = mk128(Il, Ih);
        st.f = st.f - (wsel - (internal >> 1));
        st.scan += st.size;
        st.size -= Un;
        st.round = i;
        st.n_min_rule += R.minrule ? 1 : 0;
        if (st.size > 0 && frac_gt(st.f, st.size, st.bf, st.best_size)) {
            st.bf = st.f;
            st.best_size = st.size;
            st.best_round = i;
        }
        if (r == 0 && tid == 0 && i < A.tr_cap) {
            A.tr_f_hi[i] = (long long)(unsigned long long)(st.f >> 64);
            A.tr_f_lo[i] = (unsigned long long)st.f;
            A.tr_size[i] = st.size;
            A.tr_peeled[i] = Un;
        }
        if (Un == 0) {  // cannot happen (Lemma 4.2 / minimum rule); every CTA sees it
            err = DUPIN_ERR_NO_PROGRESS;
            break;
        }
        R = tail_plan<false>(A.kD, A.D, A.use_min, A.gpo, A.lpo, st, Mn);
    }
    if (tid == 0 && S.err) set_error(ctl, S.err);
    // peel rounds of this CTA's vertices
    for (long long s = tid; s < nown; s += CL_THREADS) {
        const long long wv = tw[s];
        if (wv < 0) A.pr[live[s * C + r]] = (int)(-wv);
    }
    if (r == 0 && tid == 0) {
        if (err) set_error(ctl, err);
        ctl->round = st.round;
        ctl->size = st.size;
        ctl->f_lo = (unsigned long long)st.f;
        ctl->f_hi = (unsigned long long)(st.f >> 64);
        ctl->best_round = st.best_round;
        ctl->best_size = st.best_size;
        ctl->bf_lo = (unsigned long long)st.bf;
        ctl->bf_hi = (unsigned long long)(st.bf >> 64);
        ctl->gpo_le = st.gpo_le;
        ctl->gpo_lt = st.gpo_lt;
        ctl->n_min_rule = st.n_min_rule;
        ctl->scan_volume = st.scan;
        ctl->tail_ctas = (int)C;
    }
    cl_sync();  // no CTA leaves while another may still read its shared memory
    if (r == 0 && tid == 0 && !err) ctl->status = ST_DONE;
}

// ------------------------------------------------------------------- host

namespace {
struct ClConfig {
    int C = 0;       // CTAs per cluster (0: not set up)
    int P = 0;       // slots per CTA
    int rc = 0;
};
std::mutex g_cl_mu;
ClConfig g_cl[64];
}  // namespace

// The cluster shape for the current device, set up once per device: 16 CTAs
// where a cluster that large can be resident, else 8; P slots per CTA as the
// shared memory allows (a multiple of 64, at most 65,536 so that a slot fits
// 16 bits).
static int cluster_config(ClConfig *out) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return dupin_fail(DUPIN_ERR_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_cl_mu);
    ClConfig &c = g_cl[dev];
    if (c.C == 0 && c.rc == 0) {
        int smem = 0;
        cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, k_peel_cluster);
        if (e != cudaSuccess) {
            c.rc = dupin_cuda_fail(e, "cudaFuncGetAttributes(k_peel_cluster)");
            return c.rc;
        }
        const int dyn = smem - (int)fa.sharedSizeBytes;
        long long P = (dyn - 16) / 22;
        P = (P / CL_SEG) * CL_SEG;
        while (P > 0 && cl_smem_bytes(P) > dyn) P -= CL_SEG;
        if (P > 65536) P = 65536;
        e = cudaFuncSetAttribute(k_peel_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cl_smem_bytes(P));
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_peel_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess || P <= 0) {
            c.rc = dupin_cuda_fail(e, "cudaFuncSetAttribute(k_peel_cluster)");
            return c.rc;
        }
        int best = 0;
        for (int C : {16, 8}) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(C);
            cfg.blockDim = dim3(CL_THREADS);
            cfg.dynamicSmemBytes = (size_t)cl_smem_bytes(P);
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = C;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nc = 0;
            if (cudaOccupancyMaxActiveClusters(&nc, (void *)k_peel_cluster, &cfg) == cudaSuccess && nc > 0) {
                best = C;
                break;
            }
            cudaGetLastError();
        }
        if (best == 0) {
            c.rc = dupin_fail(DUPIN_ERR_CUDA, "no thread-block cluster of 8 or 16 CTAs fits this device");
            return c.rc;
        }
        c.C = best;
        c.P = (int)P;
    }
    if (c.rc) return c.rc;
    *out = c;
    return DUPIN_OK;
}

long long cluster_cap_limit() {
    ClConfig c;
    if (cluster_config(&c) != DUPIN_OK) return 0;
    return (long long)c.C * c.P;
}

int cluster_ctas() {
    ClConfig c;
    if (cluster_config(&c) != DUPIN_OK) return 0;
    return c.C;
}

int launch_cluster_tail(const PeelArgs &A, cudaStream_t s) {
    ClConfig c;
    int rc = cluster_config(&c);
    if (rc) return rc;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c.C);
    cfg.blockDim = dim3(CL_THREADS);
    cfg.dynamicSmemBytes = (size_t)cl_smem_bytes(c.P);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c.C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_peel_cluster, A, c.P);
    if (e != cudaSuccess) return dupin_cuda_fail(e, "cluster launch of k_peel_cluster");
    return DUPIN_OK;
}
