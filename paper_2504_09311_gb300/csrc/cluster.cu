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
// while live, -i once removed in round i), its arc range and, per 64 slots,
// the segment's exact minimum.  Every CTA also keeps its own copy of two
// bitmaps over all local ids: the vertices removed through the previous round
// and through the current one.  A round:
//
//   S  every CTA selects from its own slots (only segments whose minimum can
//      pass the round's threshold are scanned), lists the selected slots with
//      the prefix of their arc counts, prefetches their arcs into L2 (one bulk
//      request per vertex), and pushes its count, arcs, weight sum and
//      survivors' minimum into every CTA's inbox;
//   -- cluster barrier --
//   E  every CTA reads all CTAs' lists once: it extends its bitmap with U_i
//      and, when the lists are short (the common case), builds the window of
//      all listed vertices' arc ranges in the same pass; it walks an equal
//      share of the round's arcs: an arc into an earlier round's removals is
//      skipped, one into U_i adds c to the sum over arcs inside U_i, and one
//      into a survivor subtracts c in its owner's shared memory with a
//      returning 64-bit atomic add and lowers the owner's segment minimum by
//      compare-and-swap; it pushes that sum and the smallest decremented
//      weight into every CTA's inbox;
//   -- cluster barrier --
//   C  every CTA closes the round from its inbox, identically:
//      f_i = f_{i-1} - (sum_{u in U_i} w_u - internal/2), |S_i|, the best
//      prefix, the exact minimum live weight (survivors' minima before the
//      round and every decrement's result) and the plan of round i+1.
//
// A 64-bit atomic minimum on another CTA's shared memory was measured to lose
// updates when several SMs hit one word, while 64-bit adds and
// compare-and-swap there stay atomic: so the segment minima are lowered by a
// compare-and-swap loop.  The selection inbox is double-buffered by round
// parity; lists, prefixes and bitmaps are rewritten only after the barrier
// that follows every CTA's last read of them.  Every decision that ends the
// loop is taken from cluster-wide values, so all CTAs leave together; a last
// barrier keeps every CTA's shared memory alive until no other CTA can read
// it.  All arithmetic is exact integer arithmetic, identical to the one-CTA
// tail's.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "dupin_internal.h"
#include "peel_device.cuh"

#define CL_THREADS 256
#define CL_WARPS (CL_THREADS / 32)
#define CL_WIN 512  // list entries per expand window
#define CL_ILP 4    // arcs in flight per thread in the expand
#define CL_MAXC 16
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

// One CTA's selection of a round, pushed into every CTA's inbox before the
// first barrier (double-buffered by round parity).
struct ClSel {
    unsigned cnt;                 // vertices selected
    unsigned arcs;                // their arcs
    unsigned long long w_lo, w_hi;  // sum of their weights
    long long mins;               // minimum over the CTA's survivors before the decrements
};

// One CTA's expand results, pushed into every CTA's inbox before the second barrier.
struct ClRes {
    unsigned long long i_lo, i_hi;  // sum of c over the arcs it expanded that end inside U_i
    long long mind;                 // minimum weight after one of its decrements
};

struct ClShared {
    ClSel sel[2][CL_MAXC];  // [parity][CTA]
    ClRes res[CL_MAXC];     // [CTA]
    unsigned F[2];          // list counter, by round parity
    long long initmin;
    long long red_mn[CL_WARPS];
    unsigned long long red_lo[CL_WARPS], red_hi[CL_WARPS];
    long long scan[CL_WARPS];
    unsigned qcnt[CL_MAXC], qarc[CL_MAXC];  // the round: per CTA selected vertices and arcs ...
    unsigned qcex[CL_MAXC], qaex[CL_MAXC];  // ... and their exclusive prefixes
    unsigned wbase[CL_WIN + 1];             // expand window: arc prefix of its entries ...
    unsigned wstart[CL_WIN + 1];            // ... and their first arcs in the sub-graph
    long long win_e0;
    int err;
};

// Dynamic shared memory per CTA for P slots (P a multiple of 64) in a cluster
// of C CTAs: tw (8 B), arc start and degree (4 + 4 B), the list entry (2 B),
// its arc prefix (4 B) and first arc (4 B) per slot, one exact minimum per
// 64-slot segment, and two bitmaps over all C P local ids.
__host__ __device__ __forceinline__ long long cl_smem_bytes(long long P, long long C) {
    const long long nw = (C * P + 31) / 32;
    return 8 * P + 4 * P + 4 * P + 8 * (P / 64) + 4 * (P + 1) + 4 * P + 2 * P + 32 + 8 * nw;
}

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

__device__ __forceinline__ long long cl_cas_b64(uint32_t a, long long cmp, long long x) {
    long long v;
    asm volatile("atom.shared::cluster.cas.b64 %0, [%1], %2, %3;" : "=l"(v) : "r"(a), "l"(cmp), "l"(x) : "memory");
    return v;
}

__device__ __forceinline__ void cl_st_u32(uint32_t a, unsigned x) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(x) : "memory");
}

__device__ __forceinline__ void cl_st_u64(uint32_t a, unsigned long long x) {
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(a), "l"(x) : "memory");
}

// L2 prefetch of bytes [off, off + len) of an array of 'total' bytes, in
// 16-byte granules inside the array (one bulk request, no data returned)
__device__ __forceinline__ void prefetch_l2(const void *base, unsigned long long total, unsigned long long off,
                                            unsigned long long len) {
    const unsigned long long a = off & ~15ull;
    unsigned long long b = (off + len + 15) & ~15ull;
    const unsigned long long end = total & ~15ull;
    if (b > end) b = end;
    if (b > a)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"((const char *)base + a), "r"((unsigned)(b - a))
                     : "memory");
}

// NARROW: f < 2^62 and the best f < 2^64 when the cluster starts, so every
// sum a round forms fits 64 bits and the products are 64 x 64 -> 128-bit.
template <bool NARROW>
__device__ __forceinline__ void cluster_body(const PeelArgs &A, const int P, unsigned char *smem, ClShared &S) {
    PeelCtl *ctl = A.ctl;
    const unsigned C = cl_size(), r = cl_rank();
    const int lg = C == 16 ? 4 : (C == 8 ? 3 : (C == 4 ? 2 : (C == 2 ? 1 : 0)));
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const long long L = ctl->live_len;
    const int *live = ctl->live_sel ? A.live1 : A.live0;
    const long long nown = L > (long long)r ? (L - (long long)r + C - 1) / C : 0;
    const int nsl = (int)((nown + 63) / 64);           // segments that hold this CTA's vertices
    const long long NW = ((long long)C * P + 31) / 32;  // bitmap words
    const int nwl = (int)((L + 31) / 32);               // ... that cover the live set
    long long *tw = (long long *)smem;                         // [P]
    unsigned *tst = (unsigned *)(smem + 8 * (size_t)P);        // [P] first arc
    unsigned *tdg = tst + P;                                   // [P] arcs
    long long *segmin = (long long *)(tdg + P);                // [P / 64]
    unsigned *pre = (unsigned *)(segmin + P / 64);             // [P + 1] list arc prefix
    unsigned *first = pre + P + 1;                             // [P] first arc of each list entry
    unsigned short *lst = (unsigned short *)(first + P);       // [P] list of selected slots
    unsigned *bm = (unsigned *)(((uintptr_t)(lst + P) + 15) & ~(uintptr_t)15);  // [2][NW]
    const bool dg = A.tcw == nullptr;
    const int *tcol = A.tcol;
    const long long *tcw = A.tcw;

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
    {  // nothing of the live set is removed before the first round
        unsigned *b0 = bm + (st.round & 1) * NW;
        for (int k = tid; k < nwl; k += CL_THREADS) b0[k] = 0;
    }
    __syncthreads();
    {
        long long mn = kMaxLL;
        for (int q = wid; q < nsl; q += CL_WARPS) {
            const longlong2 v = *(const longlong2 *)&tw[(long long)q * 64 + 2 * lane];
            long long m = kMaxLL;
            if (v.x >= 0) m = v.x;
            if (v.y >= 0 && v.y < m) m = v.y;
            m = warp_min64(m);
            if (lane == 0) segmin[q] = m;
            mn = m < mn ? m : mn;
        }
        mn = block_min64(mn, S.red_mn);
        if (tid == 0) S.initmin = mn;
    }
    cl_sync();
    long long m0 = kMaxLL;
    if (lane < (int)C) m0 = cl_ld_s64(cl_map(&S.initmin, lane));
    m0 = warp_min64(m0);
    TailRound R = tail_plan<NARROW>(A.kD, A.D, A.use_min, A.gpo, A.lpo, st, m0);
    int err = 0;
    while (!R.done) {
        if (R.i > A.max_rounds) {
            err = DUPIN_ERR_NO_PROGRESS;
            break;
        }
        const long long i = R.i;
        const int par = (int)(i & 1);
        unsigned *bmc = bm + par * NW;              // removed through round i (built below)
        const unsigned *bmp = bm + (par ^ 1) * NW;  // removed through round i-1
        // ---- S: select this CTA's slots (segments that may hold selected vertices)
        unsigned long long wlo = 0, whi = 0;
        long long mins = kMaxLL;  // survivors' minimum over the segments this lane looked at
        for (int q0 = wid * 32; q0 < nsl; q0 += CL_THREADS) {
            const int q = q0 + lane;
            const long long sm = q < nsl ? segmin[q] : kMaxLL;
            const bool cand = seg_candidate(sm, R);
            if (!cand) mins = sm < mins ? sm : mins;
            unsigned cm = __ballot_sync(0xffffffffu, cand);
            __syncwarp();
            while (cm) {
                const int qq = q0 + __ffs(cm) - 1;
                cm &= cm - 1;
                const long long p = (long long)qq * 64 + 2 * lane;
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
                    segmin[qq] = m;  // the survivors' minimum; the expand lowers it further
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
                        if (NARROW) wlo += (unsigned long long)v.x;
                        else add128(wlo, whi, (unsigned long long)v.x, 0);
                        lst[slot++] = (unsigned short)p;
                    }
                    if (s1) {
                        tw[p + 1] = -i;
                        if (NARROW) wlo += (unsigned long long)v.y;
                        else add128(wlo, whi, (unsigned long long)v.y, 0);
                        lst[slot] = (unsigned short)(p + 1);
                    }
                }
            }
        }
        if (NARROW) wlo = warp_sum64_redux(wlo);
        else warp_sum128(wlo, whi);
        mins = warp_min64(mins);
        if (lane == 0) {
            S.red_lo[wid] = wlo;
            S.red_hi[wid] = whi;
            S.red_mn[wid] = mins;
        }
        __syncthreads();
        const unsigned F = S.F[par];
        if (tid == 0) S.F[par ^ 1] = 0;  // round i+1's counter (last read in round i-1)
        // the list's arc prefix and first arcs; each listed vertex's arcs are
        // prefetched into L2 now (the expand reads them after the barrier)
        if (F <= 32) {
            if (wid == 0) {
                unsigned d = 0;
                if (lane < (int)F) {
                    const unsigned sl = lst[lane];
                    d = tdg[sl];
                    first[lane] = tst[sl];
                    prefetch_l2(tcol, 4ull * A.tarc_cap, 4ull * tst[sl], 4ull * d);
                    if (!dg) prefetch_l2(tcw, 8ull * A.tarc_cap, 8ull * tst[sl], 8ull * d);
                }
                unsigned incl = d;
#pragma unroll
                for (int k = 1; k < 32; k <<= 1) {
                    const unsigned o = __shfl_up_sync(0xffffffffu, incl, k);
                    if (lane >= k) incl += o;
                }
                if (lane < (int)F) pre[lane] = incl - d;
                if (lane == 31) pre[F] = incl;
            }
        } else {
            unsigned carry = 0;
            for (unsigned e0 = 0; e0 < F; e0 += CL_THREADS) {
                const unsigned e = e0 + tid;
                unsigned d = 0;
                if (e < F) {
                    const unsigned sl = lst[e];
                    d = tdg[sl];
                    first[e] = tst[sl];
                    prefetch_l2(tcol, 4ull * A.tarc_cap, 4ull * tst[sl], 4ull * d);
                    if (!dg) prefetch_l2(tcw, 8ull * A.tarc_cap, 8ull * tst[sl], 8ull * d);
                }
                long long tot;
                const long long ex = block_excl_scan<CL_WARPS>((long long)d, S.scan, tot);
                if (e < F) pre[e] = carry + (unsigned)ex;
                carry += (unsigned)tot;
            }
            if (tid == 0) pre[F] = carry;
        }
        if (wid == 0) {  // the CTA's totals, pushed into every CTA's inbox
            unsigned long long l = lane < CL_WARPS ? S.red_lo[lane] : 0, h = lane < CL_WARPS ? S.red_hi[lane] : 0;
            long long m = lane < CL_WARPS ? S.red_mn[lane] : kMaxLL;
            warp_sum128(l, h);
            m = warp_min64(m);
            l = __shfl_sync(0xffffffffu, l, 0);
            h = __shfl_sync(0xffffffffu, h, 0);
            m = __shfl_sync(0xffffffffu, m, 0);
            __syncwarp();
            const unsigned arcs = pre[F];
            if (lane < (int)C) {
                const uint32_t b = cl_map(&S.sel[par][r], lane);
                cl_st_u32(b + offsetof(ClSel, cnt), F);
                cl_st_u32(b + offsetof(ClSel, arcs), arcs);
                cl_st_u64(b + offsetof(ClSel, w_lo), l);
                cl_st_u64(b + offsetof(ClSel, w_hi), h);
                cl_st_u64(b + offsetof(ClSel, mins), (unsigned long long)m);
            }
        }
        cl_sync();  // A: every CTA's selection, list and prefix are visible
        // ---- E: the removed set U_i and the round's arcs
        if (wid == 0) {  // per CTA: selected vertices and arcs, and their prefixes
            unsigned c = 0, a = 0;
            if (lane < (int)C) {
                c = S.sel[par][lane].cnt;
                a = S.sel[par][lane].arcs;
            }
            unsigned ic = c, ia = a;
#pragma unroll
            for (int k = 1; k < 32; k <<= 1) {
                const unsigned oc = __shfl_up_sync(0xffffffffu, ic, k), oa = __shfl_up_sync(0xffffffffu, ia, k);
                if (lane >= k) {
                    ic += oc;
                    ia += oa;
                }
            }
            if (lane < (int)C) {
                S.qcnt[lane] = c;
                S.qarc[lane] = a;
                S.qcex[lane] = ic - c;
                S.qaex[lane] = ia - a;
            }
        }
        // removed through round i = removed through round i-1, plus U_i
        for (int k = tid; k < nwl; k += CL_THREADS) bmc[k] = bmp[k];
        __syncthreads();
        const unsigned Ltot = S.qcex[C - 1] + S.qcnt[C - 1];
        const unsigned Atot = S.qaex[C - 1] + S.qarc[C - 1];
        // A short round (its lists fit one window): the window over all CTAs'
        // lists is built here, in the same pass that extends the bitmap
        const bool gwin = Ltot <= CL_WIN;
        for (unsigned g = tid; g < Ltot; g += CL_THREADS) {
            int q = 0;  // the last CTA whose entries start at or before g
            for (int step = 8; step > 0; step >>= 1)
                if (q + step < (int)C && S.qcex[q + step] <= g) q += step;
            const unsigned e = g - S.qcex[q];
            const unsigned sl = cl_ld_u16(cl_map(lst, q) + 2 * e);
            if (gwin) {
                S.wbase[g] = S.qaex[q] + cl_ld_u32(cl_map(pre, q) + 4 * e);
                S.wstart[g] = cl_ld_u32(cl_map(first, q) + 4 * e);
            }
            const unsigned p = sl * C + q;
            atomicOr(&bmc[p >> 5], 1u << (p & 31));
        }
        if (gwin)
            for (unsigned t = Ltot + tid; t <= CL_WIN; t += CL_THREADS) S.wbase[t] = t == Ltot ? Atot : 0xffffffffu;
        __syncthreads();
        unsigned long long ilo = 0, ihi = 0;
        long long mind = kMaxLL;
        // one arc: a survivor loses c in its owner's shared memory (returning
        // 64-bit add; the owner's segment minimum lowered by compare-and-swap),
        // an arc into U_i adds c to 'internal', an arc into an earlier round's
        // removals is skipped (the bitmaps are local copies)
        auto arcs = [&](const long long (&pos)[CL_ILP]) {
            int cv[CL_ILP];
            long long cc[CL_ILP];
#pragma unroll
            for (int u = 0; u < CL_ILP; u++) {
                if (pos[u] >= 0) {
                    cv[u] = tcol[pos[u]];
                    cc[u] = dg ? DUPIN_Q_ONE : tcw[pos[u]];
                }
            }
            uint32_t sa[CL_ILP];
            long long nv[CL_ILP], sm[CL_ILP];
#pragma unroll
            for (int u = 0; u < CL_ILP; u++) {
                nv[u] = kMaxLL;
                if (pos[u] < 0) continue;
                const unsigned v = (unsigned)cv[u];
                if (!((bmc[v >> 5] >> (v & 31)) & 1u)) {
                    const unsigned o = v & (C - 1), sl = v >> lg;
                    sa[u] = cl_map(&segmin[sl >> 6], o);
                    sm[u] = cl_ld_s64(sa[u]);
                    nv[u] = (long long)cl_atom_add_u64(cl_map(&tw[sl], o), (unsigned long long)(-cc[u])) - cc[u];
                    mind = nv[u] < mind ? nv[u] : mind;
                } else if (!((bmp[v >> 5] >> (v & 31)) & 1u)) {
                    if (NARROW) ilo += (unsigned long long)cc[u];
                    else add128(ilo, ihi, (unsigned long long)cc[u], 0);
                }
            }
#pragma unroll
            for (int u = 0; u < CL_ILP; u++) {
                if (nv[u] == kMaxLL) continue;
                long long cur = sm[u];
                while (nv[u] < cur) {
                    const long long prev = cl_cas_b64(sa[u], cur, nv[u]);
                    if (prev == cur) break;
                    cur = prev;
                }
            }
        };
        {
            const unsigned E0 = (unsigned)split_at(Atot, r, C), E1 = (unsigned)split_at(Atot, r + 1, C);
            if (gwin) {
                for (unsigned xb = E0 + tid; xb < E1; xb += CL_ILP * CL_THREADS) {
                    long long pos[CL_ILP];
#pragma unroll
                    for (int u = 0; u < CL_ILP; u++) {
                        const unsigned xx = xb + u * CL_THREADS;
                        pos[u] = -1;
                        if (xx < E1) {
                            int lo2 = 0, hi2 = (int)Ltot;  // last t with wbase[t] <= xx
                            while (lo2 < hi2) {
                                const int mid = (lo2 + hi2 + 1) >> 1;
                                if (S.wbase[mid] <= xx) lo2 = mid;
                                else hi2 = mid - 1;
                            }
                            pos[u] = (long long)S.wstart[lo2] + (xx - S.wbase[lo2]);
                        }
                    }
                    arcs(pos);
                }
            } else {
                unsigned x = E0;
                int q = 0;
                while (x < E1) {  // block-uniform: a window of one CTA's list at a time
                    while (q + 1 < (int)C && (S.qaex[q + 1] <= x || S.qarc[q] == 0)) q++;
                    if (!(S.qaex[q] <= x && x < S.qaex[q] + S.qarc[q])) {  // cannot happen for x < Atot
                        if (tid == 0) S.err = DUPIN_ERR_CUDA;
                        break;
                    }
                    const unsigned qbase = S.qaex[q], qcnt = S.qarc[q], Fq = S.qcnt[q];
                    const unsigned lo = x - qbase;
                    const unsigned hi = (E1 - qbase < qcnt ? E1 - qbase : qcnt);
                    const uint32_t rpre = cl_map(pre, q), rfirst = cl_map(first, q);
                    if (wid == 0) {  // the window's first entry: the last e with pre_q[e] <= lo
                        const long long e = warp_search_last_le_fn(
                            (long long)Fq - 1, [&](long long k) { return cl_ld_u32(rpre + 4 * (uint32_t)k) <= lo; });
                        if (lane == 0) S.win_e0 = e;
                    }
                    __syncthreads();
                    const long long e0 = S.win_e0;
                    for (int t = tid; t <= CL_WIN; t += CL_THREADS) {
                        const long long e = e0 + t;
                        unsigned b = 0xffffffffu, s0 = 0;
                        if (e <= (long long)Fq) b = cl_ld_u32(rpre + 4 * (uint32_t)e);
                        if (e < (long long)Fq) s0 = cl_ld_u32(rfirst + 4 * (uint32_t)e);
                        S.wbase[t] = b;
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
                        arcs(pos);
                    }
                    x = qbase + wend;
                    __syncthreads();  // the window is reused
                }
            }
        }
        if (NARROW) ilo = warp_sum64_redux(ilo);
        else warp_sum128(ilo, ihi);
        mind = warp_min64(mind);
        if (lane == 0) {
            S.red_lo[wid] = ilo;
            S.red_hi[wid] = ihi;
            S.red_mn[wid] = mind;
        }
        __syncthreads();
        if (wid == 0) {  // this CTA's results, pushed into every CTA's inbox
            unsigned long long l = lane < CL_WARPS ? S.red_lo[lane] : 0, h = lane < CL_WARPS ? S.red_hi[lane] : 0;
            long long m = lane < CL_WARPS ? S.red_mn[lane] : kMaxLL;
            warp_sum128(l, h);
            m = warp_min64(m);
            l = __shfl_sync(0xffffffffu, l, 0);
            h = __shfl_sync(0xffffffffu, h, 0);
            m = __shfl_sync(0xffffffffu, m, 0);
            if (lane < (int)C) {
                const uint32_t b = cl_map(&S.res[r], lane);
                cl_st_u64(b + offsetof(ClRes, i_lo), l);
                cl_st_u64(b + offsetof(ClRes, i_hi), h);
                cl_st_u64(b + offsetof(ClRes, mind), (unsigned long long)m);
            }
        }
        cl_sync();  // B: every decrement and every CTA's results of round i are visible
        // ---- C: close round i and plan round i+1 (every warp, same values, local reads)
        unsigned long long Wl = 0, Wh = 0, Il = 0, Ih = 0;
        unsigned Uq = 0;
        long long Mn = kMaxLL;
        if (lane < (int)C) {
            const ClSel &x = S.sel[par][lane];
            const ClRes &y = S.res[lane];
            Uq = x.cnt;
            Wl = x.w_lo;
            Wh = x.w_hi;
            Il = y.i_lo;
            Ih = y.i_hi;
            Mn = x.mins < y.mind ? x.mins : y.mind;
        }
        const long long Un = (long long)__reduce_add_sync(0xffffffffu, Uq);
        if (NARROW) {
            Wl = warp_sum64_redux(Wl);
            Il = warp_sum64_redux(Il);
            Wh = 0;
            Ih = 0;
        } else {
            warp_sum128(Wl, Wh);
            warp_sum128(Il, Ih);
            Wl = __shfl_sync(0xffffffffu, Wl, 0);
            Wh = __shfl_sync(0xffffffffu, Wh, 0);
            Il = __shfl_sync(0xffffffffu, Il, 0);
            Ih = __shfl_sync(0xffffffffu, Ih, 0);
        }
        Mn = warp_min64(Mn);
        const u128 wsel = mk128(Wl, Wh), internal = mk128(Il, Ih);
        st.f = st.f - (wsel - (internal >> 1));
        st.scan += st.size;
        st.size -= Un;
        st.round = i;
        st.n_min_rule += R.minrule ? 1 : 0;
        if (st.size > 0 && frac_gt<NARROW>(st.f, st.size, st.bf, st.best_size)) {
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
        R = tail_plan<NARROW>(A.kD, A.D, A.use_min, A.gpo, A.lpo, st, Mn);
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

__global__ void __launch_bounds__(CL_THREADS, 1) k_peel_cluster(PeelArgs A, int P) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ClShared S;
    const PeelCtl *ctl = A.ctl;
    if (ctl->status != ST_CLUSTER || ctl->error) return;  // identical in every CTA
    if (ctl->f_hi == 0 && ctl->f_lo < (1ull << 62) && ctl->bf_hi == 0) cluster_body<true>(A, P, smem, S);
    else cluster_body<false>(A, P, smem, S);
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
// shared memory allows (a multiple of 64, at most 65,536).
static long long slots_for(int C, int dyn) {
    long long P = (long long)dyn / (26 + C / 4);
    P = (P / 64) * 64;
    while (P > 0 && cl_smem_bytes(P, C) > dyn) P -= 64;
    return P > 65536 ? 65536 : P;  // a list entry keeps the slot in 16 bits
}

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
        const long long P16 = slots_for(16, dyn), P8 = slots_for(8, dyn);
        const long long most = std::max(cl_smem_bytes(P16, 16), cl_smem_bytes(P8, 8));
        e = cudaFuncSetAttribute(k_peel_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_peel_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess || P8 <= 0) {
            c.rc = dupin_cuda_fail(e, "cudaFuncSetAttribute(k_peel_cluster)");
            return c.rc;
        }
        int best = 0;
        long long bestP = 0;
        for (int C : {16, 8}) {
            const long long P = C == 16 ? P16 : P8;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(C);
            cfg.blockDim = dim3(CL_THREADS);
            cfg.dynamicSmemBytes = (size_t)cl_smem_bytes(P, C);
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = C;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nc = 0;
            if (P > 0 && cudaOccupancyMaxActiveClusters(&nc, (void *)k_peel_cluster, &cfg) == cudaSuccess && nc > 0) {
                best = C;
                bestP = P;
                break;
            }
            cudaGetLastError();
        }
        if (best == 0) {
            c.rc = dupin_fail(DUPIN_ERR_CUDA, "no thread-block cluster of 8 or 16 CTAs fits this device");
            return c.rc;
        }
        c.C = best;
        c.P = (int)bestP;
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
    cfg.dynamicSmemBytes = (size_t)cl_smem_bytes(c.P, c.C);
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
