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
// the segment's exact minimum.  The tail sub-graph's rows are stored with
// each row's arcs grouped by the owner of their head, with every group's
// bounds, so that each CTA reads exactly the arcs into its own vertices and
// every update of a vertex's state is made by its owner.  A round i:
//
//   S  the removed set U_i.  When round i takes the minimum rule (the common
//      case of a skewed graph at k(1+eps) < 2), U_i is every live vertex at
//      the minimum weight, and every CTA already holds it: each CTA listed its
//      own vertices at its own minimum with its results of round i-1.  The
//      CTAs at the cluster's minimum mark theirs; nothing is exchanged.
//      Otherwise every CTA selects from its own slots (only segments whose
//      minimum can pass the round's threshold are scanned), lists them,
//      prefetches their arcs and group bounds into L2, and pushes its count
//      and weight sum -- and a short list itself -- into every CTA's inbox,
//      followed by a cluster barrier.
//   E  every CTA walks the round's list and, for each removed vertex u, the
//      group of u's arcs whose heads it owns: an arc into an earlier round's
//      removal is skipped, one into U_i adds c to the sum over arcs inside
//      U_i, and one into a survivor subtracts c with a shared-memory atomic
//      and lowers the segment minimum -- all local.
//   P  every CTA finds its minimum live weight and its live vertices at that
//      weight (prefetching their arcs into L2), and pushes them with its
//      internal sum into every CTA's inbox by asynchronous shared-memory
//      stores that complete on the receiver's mbarrier.
//   -- every CTA waits on its own mbarrier: all C pushes have arrived --
//   C  every CTA closes the round from its inbox, identically:
//      f_i = f_{i-1} - (sum_{u in U_i} w_u - internal/2), |S_i|, the best
//      prefix, the cluster's minimum live weight and the plan of round i+1.
//
// So a minimum-rule round has no cluster barrier at all: each CTA waits only
// for the data it needs.  The only traffic between CTAs is the inboxes (and
// the list of a CTA that selected more than a short list holds, read
// remotely).  No CTA can get more than one round ahead of another (it needs
// everyone's results of a round to start the next), so inboxes
// double-buffered by round parity are never overwritten before they are
// read.  Every decision that ends the loop is taken from cluster-wide
// values, so all CTAs leave together; a last barrier keeps every CTA's
// shared memory alive until no other CTA can read it.  All arithmetic is
// exact integer arithmetic, identical to the one-CTA tail's.
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
#define CL_INL 32   // a list this short travels in the inboxes
#define CL_SPEC 32  // a CTA lists its vertices at its minimum weight up to this many ...
#define CL_PUSH 8   // ... and pushes them into the inboxes up to this many
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

__device__ __forceinline__ unsigned cl_ld_u16(uint32_t a) {
    unsigned short v;
    asm volatile("ld.shared::cluster.u16 %0, [%1];" : "=h"(v) : "r"(a) : "memory");
    return v;
}

// ------------------------------------------------------------ shared state

// One CTA's selection of a round that is not taken by the minimum rule from
// the listed minima, pushed into every CTA's inbox before the first barrier
// (double-buffered by round parity).
struct ClSel {
    unsigned cnt;                   // vertices selected
    unsigned pad;
    unsigned long long w_lo, w_hi;  // sum of their weights
};

// One CTA's results of a round, pushed into every CTA's inbox at the round's
// end (double-buffered by round parity): 64 bytes, four 16-byte asynchronous
// stores that complete on the receiver's mbarrier.
struct __align__(16) ClRes {
    unsigned long long i_lo, i_hi;  // sum of c over the arcs it expanded that end inside U_i
    long long mn;                   // minimum weight of its live vertices after the round (kMaxLL: none)
    unsigned long long scnt;        // its live vertices at that weight ...
    unsigned spec[CL_PUSH];         // ... by local id, when scnt <= CL_PUSH
};

struct ClShared {
    ClSel sel[2][CL_MAXC];                // [parity][CTA]
    ClRes res[2][CL_MAXC];                // [parity][CTA]
    unsigned long long mb[2];             // [parity]: complete once every CTA's ClRes has arrived
    unsigned inl[CL_MAXC][CL_INL];        // [CTA]: its selected local ids, when it selected at most CL_INL
    unsigned F;                           // list counter
    unsigned nspec, nseg;                 // this CTA's vertices at its minimum ...
    unsigned short myslot[CL_SPEC];       // ... their slots ...
    int myseg[CL_SPEC];                   // ... their segments ...
    long long myalt[CL_SPEC];             // ... and each segment's minimum over its other live vertices
    long long red_mn[CL_WARPS];
    unsigned long long red_lo[CL_WARPS], red_hi[CL_WARPS];
    long long scan[CL_WARPS];
    unsigned qcnt[CL_MAXC], qcex[CL_MAXC];  // the round: per CTA selected vertices, exclusive prefix
    unsigned wbase[CL_WIN + 1];             // expand window: arc prefix of its entries ...
    unsigned wstart[CL_WIN + 1];            // ... and the first arc of each entry's group
    int err;
};

// Dynamic shared memory per CTA for P slots (P a multiple of 64): tw (8 B),
// arc start and degree (4 + 4 B) and the list entry (2 B) per slot, and one
// exact minimum per 64-slot segment.
__host__ __device__ __forceinline__ long long cl_smem_bytes(long long P, long long) {
    return 8 * P + 4 * P + 4 * P + 8 * (P / 64) + 2 * P + 16;
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

__device__ __forceinline__ void cl_st_u32(uint32_t a, unsigned x) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(x) : "memory");
}

// 16 bytes into another CTA's shared memory, completing (as 16 transaction
// bytes) on the mbarrier at 'mbar' in that CTA
__device__ __forceinline__ void cl_st_async_v4(uint32_t a, uint32_t mbar, unsigned x, unsigned y, unsigned z,
                                               unsigned w) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(a),
                 "r"(x), "r"(y), "r"(z), "r"(w), "r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mb_init(unsigned long long *mb, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(mb)), "r"(count)
                 : "memory");
}

// this thread's arrival, announcing 'tx' transaction bytes for the current phase
__device__ __forceinline__ void mb_arrive_expect_tx(unsigned long long *mb, unsigned tx) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
            (unsigned)__cvta_generic_to_shared(mb)),
        "r"(tx)
        : "memory");
}

// has the phase of parity 'parity' completed? (acquire at cluster scope: the
// asynchronous stores that completed it are visible)
__device__ __forceinline__ bool mb_try_wait(unsigned long long *mb, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, "
        "1, 0, p;\n\t}"
        : "=r"(done)
        : "r"((unsigned)__cvta_generic_to_shared(mb)), "r"(parity)
        : "memory");
    return done != 0;
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
    const int nsl = (int)((nown + 63) / 64);  // segments that hold this CTA's vertices
    long long *tw = (long long *)smem;                          // [P]
    unsigned *tst = (unsigned *)(smem + 8 * (size_t)P);         // [P] first arc
    unsigned *tdg = tst + P;                                    // [P] arcs
    long long *segmin = (long long *)(tdg + P);                 // [P / 64]
    unsigned short *lst = (unsigned short *)(segmin + P / 64);  // [P] list of selected slots
    const bool dg = A.tcw == nullptr;
    const int *tcol = A.tcol;
    const long long *tcw = A.tcw;
    const unsigned long long grp_bytes = 4ull * DUPIN_GRP_STRIDE * (unsigned long long)(A.hcap + 1);

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
        S.F = 0;
        S.err = 0;
    }
    __syncthreads();
    for (int q = wid; q < nsl; q += CL_WARPS) {  // exact segment minima
        const longlong2 v = *(const longlong2 *)&tw[(long long)q * 64 + 2 * lane];
        long long m = kMaxLL;
        if (v.x >= 0) m = v.x;
        if (v.y >= 0 && v.y < m) m = v.y;
        m = warp_min64(m);
        if (lane == 0) segmin[q] = m;
    }

    // The results of a round (and, once, of the state before the first): this
    // CTA's minimum live weight, its live vertices at that weight -- the
    // minimum rule's choice here, should the next round take it and this CTA
    // hold the cluster's minimum -- with each of their segments' minimum over
    // its other live vertices, L2 prefetches of their arcs and group bounds,
    // and the push of all that and the round's internal sum into every CTA's
    // inbox (buffer pb).
    auto publish = [&](int pb, unsigned long long il, unsigned long long ih) {
        if (NARROW) il = warp_sum64_redux(il);
        else warp_sum128(il, ih);
        if (lane == 0) {
            S.red_lo[wid] = il;
            S.red_hi[wid] = ih;
        }
        if (tid == 0) {
            S.nspec = 0;
            S.nseg = 0;
        }
        __syncthreads();  // the round's decrements and segment minima are final
        long long mn = kMaxLL;
        for (int q = tid; q < nsl; q += CL_THREADS) mn = segmin[q] < mn ? segmin[q] : mn;
        mn = block_min64(mn, S.red_mn);
        if (mn != kMaxLL) {
            unsigned k = 0;  // rank of the next segment at the minimum (the same in every warp)
            for (int q0 = 0; q0 < nsl; q0 += 32) {  // every warp finds every such segment ...
                const int q = q0 + lane;
                unsigned cm = __ballot_sync(0xffffffffu, q < nsl && segmin[q] == mn);
                while (cm) {
                    const int qq = q0 + __ffs(cm) - 1;
                    cm &= cm - 1;
                    if ((k++ & (CL_WARPS - 1)) != (unsigned)wid) continue;  // ... and scans its share
                    const long long p = (long long)qq * 64 + 2 * lane;
                    const longlong2 v = *(const longlong2 *)&tw[p];
                    const bool s0 = v.x == mn, s1 = v.y == mn;
                    long long m = kMaxLL;
                    if (v.x >= 0 && !s0) m = v.x;
                    if (v.y >= 0 && !s1 && v.y < m) m = v.y;
                    m = warp_min64(m);
                    const unsigned b0 = __ballot_sync(0xffffffffu, s0), b1 = __ballot_sync(0xffffffffu, s1);
                    unsigned base = 0;
                    if (lane == 0) {
                        base = atomicAdd(&S.nspec, (unsigned)(__popc(b0) + __popc(b1)));
                        const unsigned j = atomicAdd(&S.nseg, 1u);
                        if (j < CL_SPEC) {
                            S.myseg[j] = qq;
                            S.myalt[j] = m;
                        }
                    }
                    base = __shfl_sync(0xffffffffu, base, 0);
                    const unsigned lt = (1u << lane) - 1u;
                    unsigned slot = base + __popc(b0 & lt) + __popc(b1 & lt);
                    if (s0) {
                        if (slot < CL_SPEC) S.myslot[slot] = (unsigned short)p;
                        slot++;
                    }
                    if (s1 && slot < CL_SPEC) S.myslot[slot] = (unsigned short)(p + 1);
                }
            }
        }
        __syncthreads();
        const unsigned ns = S.nspec;
        if (ns <= CL_SPEC && tid >= 32) {  // one prefetch per thread (warp 0 pushes)
            const unsigned x = (unsigned)tid - 32, e = x / 3, k = x - 3 * e;
            if (e < ns && (k != 1 || !dg)) {
                const unsigned sl = S.myslot[e];
                if (k == 0) prefetch_l2(tcol, 4ull * A.tarc_cap, 4ull * tst[sl], 4ull * tdg[sl]);
                else if (k == 1) prefetch_l2(tcw, 8ull * A.tarc_cap, 8ull * tst[sl], 8ull * tdg[sl]);
                else
                    prefetch_l2(A.tgrp, grp_bytes, 4ull * DUPIN_GRP_STRIDE * ((unsigned long long)sl * C + r),
                                4ull * DUPIN_GRP_STRIDE);
            }
        }
        if (wid == 0) {  // lane o pushes this CTA's results into CTA o's inbox
            unsigned long long l = lane < CL_WARPS ? S.red_lo[lane] : 0, h = lane < CL_WARPS ? S.red_hi[lane] : 0;
            warp_sum128(l, h);
            l = __shfl_sync(0xffffffffu, l, 0);
            h = __shfl_sync(0xffffffffu, h, 0);
            if (lane < (int)C) {
                const uint32_t b = cl_map(&S.res[pb][r], lane), m = cl_map(&S.mb[pb], lane);
                unsigned x[CL_PUSH];
#pragma unroll
                for (int k = 0; k < CL_PUSH; k++) x[k] = (unsigned)k < ns ? (unsigned)S.myslot[k] * C + r : 0u;
                cl_st_async_v4(b, m, (unsigned)l, (unsigned)(l >> 32), (unsigned)h, (unsigned)(h >> 32));
                cl_st_async_v4(b + 16, m, (unsigned)mn, (unsigned)((unsigned long long)mn >> 32), ns, 0u);
                cl_st_async_v4(b + 32, m, x[0], x[1], x[2], x[3]);
                cl_st_async_v4(b + 48, m, x[4], x[5], x[6], x[7]);
            }
        }
    };
    // every CTA's results (buffer pb), read by every warp alike: the
    // cluster's minimum live weight, whether a CTA holding it listed more
    // vertices than its inbox list takes, and the round's internal sum
    auto results = [&](int pb, long long &Mn, bool &over, unsigned long long &Il, unsigned long long &Ih) {
        long long mn = kMaxLL;
        unsigned sc = 0;
        unsigned long long il = 0, ih = 0;
        if (lane < (int)C) {
            const ClRes &x = S.res[pb][lane];
            mn = x.mn;
            sc = x.scnt;
            il = x.i_lo;
            ih = x.i_hi;
        }
        Mn = warp_min64(mn);
        over = __any_sync(0xffffffffu, lane < (int)C && mn == Mn && sc > CL_PUSH) != 0;
        if (NARROW) {
            Il = warp_sum64_redux(il);
            Ih = 0;
        } else {
            warp_sum128(il, ih);
            Il = __shfl_sync(0xffffffffu, il, 0);
            Ih = __shfl_sync(0xffffffffu, ih, 0);
        }
    };

    // every CTA's results of a round arrive by asynchronous stores that
    // complete on the receiver's mbarrier of the round's parity: one local
    // arrival (announcing C ClRes of transaction bytes) and the C pushes
    // complete a phase.  A CTA can push round i+2's results (same parity)
    // only after it has received this CTA's results of round i+1, which this
    // CTA sends after its wait for round i: phases never overlap.
    unsigned phase = 0;  // bit b: parity of mbarrier b's current phase
    int werr = 0;
    auto expect = [&](int pb) {  // warp 1: warp 0's loads in flight need not complete first
        if (tid == 32) mb_arrive_expect_tx(&S.mb[pb], (unsigned)(C * sizeof(ClRes)));
    };
    auto wait_results = [&](int pb) {
        int bad = 0;
        if (!mb_try_wait(&S.mb[pb], (phase >> pb) & 1)) {
            const long long t0 = clock64();
            while (!mb_try_wait(&S.mb[pb], (phase >> pb) & 1)) {
                if (clock64() - t0 > (1ll << 32)) {  // a lost push: cannot happen; give up rather than hang
                    bad = 1;
                    break;
                }
            }
        }
        phase ^= 1u << pb;
        if (__syncthreads_or(bad)) werr = DUPIN_ERR_TIMEOUT;
    };
    if (tid == 0) {
        mb_init(&S.mb[0], 1);
        mb_init(&S.mb[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    expect((int)(st.round & 1));
    cl_sync();  // every CTA's mbarriers are set up before any push
    publish((int)(st.round & 1), 0, 0);
    wait_results((int)(st.round & 1));
    // Warp 0, after a round's results: should the next round take the
    // minimum rule, its list is every CTA's vertices at the minimum Mn; lane
    // q (a CTA at Mn) loads the bounds of its entries' groups for this CTA
    // now, so that the loads are in flight while the round closes (nothing
    // here waits for them).
    bool pre = false;
    unsigned pc = 0, ptot = 0, pg0[CL_PUSH], pg1[CL_PUSH];
    auto preload = [&](int pb, long long Mn, bool over) {
        if (wid != 0) return;
        pc = lane < (int)C && S.res[pb][lane].mn == Mn ? (unsigned)S.res[pb][lane].scnt : 0;
        ptot = __reduce_add_sync(0xffffffffu, pc);
        pre = !over && ptot <= 32;
        if (!pre) return;
#pragma unroll
        for (int e = 0; e < CL_PUSH; e++) {
            if ((unsigned)e < pc) {
                const unsigned *gr = A.tgrp + (size_t)S.res[pb][lane].spec[e] * DUPIN_GRP_STRIDE + r;
                pg0[e] = __ldg(gr);
                pg1[e] = __ldg(gr + 1);
            }
        }
    };
    TailRound R;
    bool fast;
    {
        long long m0;
        bool over;
        unsigned long long il, ih;
        results((int)(st.round & 1), m0, over, il, ih);
        preload((int)(st.round & 1), m0, over);
        R = tail_plan<NARROW>(A.kD, A.D, A.use_min, A.gpo, A.lpo, st, m0);
        fast = R.minrule && !over;
        pre = pre && fast;
    }
    int err = werr;
    while (!R.done && !err) {
        if (R.i > A.max_rounds) {
            err = DUPIN_ERR_NO_PROGRESS;
            break;
        }
        const long long i = R.i;
        const int par = (int)(i & 1), ppar = par ^ 1;
        expect(par);
        unsigned long long Wl = 0, Wh = 0;  // sum of the removed vertices' weights
        // entry g of the round's list (CTA by CTA) -> its local id
        auto entry = [&](unsigned g) -> unsigned {
            int q = 0;  // the last CTA whose entries start at or before g
            for (int step = 8; step > 0; step >>= 1)
                if (q + step < (int)C && S.qcex[q + step] <= g) q += step;
            const unsigned e = g - S.qcex[q];
            if (fast) return S.res[ppar][q].spec[e];
            if (S.qcnt[q] <= CL_INL) return S.inl[q][e];
            return cl_ld_u16(cl_map(lst, q) + 2 * e) * C + q;
        };
        // the group bounds of entry g's row for this CTA
        auto group = [&](unsigned g, unsigned &gs, unsigned &len) {
            const unsigned p = entry(g);
            const unsigned *gr = A.tgrp + (size_t)p * DUPIN_GRP_STRIDE + r;
            gs = gr[0];
            len = gr[1] - gs;
        };
        // warp 0: the window of list entries [w0, w0 + nw), nw <= 32: each
        // entry's group start and the prefix of the group lengths
        auto build_window = [&](unsigned w0, unsigned nw) {
            unsigned gs = 0, len = 0;
            if (lane < (int)nw) group(w0 + lane, gs, len);
            unsigned incl = len;
#pragma unroll
            for (int k = 1; k < 32; k <<= 1) {
                const unsigned o = __shfl_up_sync(0xffffffffu, incl, k);
                if (lane >= k) incl += o;
            }
            if (lane < (int)nw) {
                S.wbase[lane] = incl - len;
                S.wstart[lane] = gs;
            }
            if (lane == 31) S.wbase[nw] = incl;
        };
        if (fast) {
            // U_i: the vertices at the minimum weight, listed by the CTAs that
            // hold it with the previous round's results; each marks its own
            if (wid > 0 && S.res[ppar][r].mn == R.minw) {  // warp 0 builds the list's window meanwhile
                const unsigned ns = (unsigned)S.res[ppar][r].scnt;
                const unsigned ng = S.nseg < ns ? S.nseg : ns;
                for (unsigned e = tid - 32; e < ns; e += CL_THREADS - 32) tw[S.myslot[e]] = -i;
                for (unsigned k = tid - 32; k < ng; k += CL_THREADS - 32) segmin[S.myseg[k]] = S.myalt[k];
            }
            if (wid == 0 && pre) {  // the list and its group bounds, loaded while round i-1 closed
                unsigned len[CL_PUSH], tot = 0;
#pragma unroll
                for (int e = 0; e < CL_PUSH; e++) {
                    len[e] = (unsigned)e < pc ? pg1[e] - pg0[e] : 0u;
                    tot += len[e];
                }
                unsigned ic = pc, it = tot;
#pragma unroll
                for (int k = 1; k < 32; k <<= 1) {
                    const unsigned oc = __shfl_up_sync(0xffffffffu, ic, k), ot = __shfl_up_sync(0xffffffffu, it, k);
                    if (lane >= k) {
                        ic += oc;
                        it += ot;
                    }
                }
                const unsigned exc = ic - pc;
                if (lane < (int)C) {
                    S.qcnt[lane] = pc;
                    S.qcex[lane] = exc;
                }
                unsigned run = it - tot;
#pragma unroll
                for (int e = 0; e < CL_PUSH; e++) {
                    if ((unsigned)e < pc) {
                        S.wbase[exc + e] = run;
                        S.wstart[exc + e] = pg0[e];
                        run += len[e];
                    }
                }
                if (lane == 31) S.wbase[ptot] = it;
            } else if (wid == 0) {
                const unsigned c =
                    lane < (int)C && S.res[ppar][lane].mn == R.minw ? (unsigned)S.res[ppar][lane].scnt : 0;
                unsigned ic = c;
#pragma unroll
                for (int k = 1; k < 32; k <<= 1) {
                    const unsigned oc = __shfl_up_sync(0xffffffffu, ic, k);
                    if (lane >= k) ic += oc;
                }
                if (lane < (int)C) {
                    S.qcnt[lane] = c;
                    S.qcex[lane] = ic - c;
                }
                __syncwarp();
                const unsigned Un = __shfl_sync(0xffffffffu, ic, 31);
                if (Un <= 32) build_window(0, Un);  // the list's only window, before the barrier below
            }
            __syncthreads();
            const unsigned Un = S.qcex[C - 1] + S.qcnt[C - 1];
            const u128 W = (u128)(unsigned long long)R.minw * Un;
            Wl = (unsigned long long)W;
            Wh = (unsigned long long)(W >> 64);
        } else {
            // ---- S: select this CTA's slots (segments that may hold selected vertices)
            unsigned long long wlo = 0, whi = 0;
            for (int q0 = wid * 32; q0 < nsl; q0 += CL_THREADS) {
                const int q = q0 + lane;
                const long long sm = q < nsl ? segmin[q] : kMaxLL;
                unsigned cm = __ballot_sync(0xffffffffu, seg_candidate(sm, R));
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
                    if (lane == 0) segmin[qq] = m;  // the survivors' minimum; the expand lowers it further
                    const unsigned b0 = __ballot_sync(0xffffffffu, s0), b1 = __ballot_sync(0xffffffffu, s1);
                    if (b0 | b1) {
                        unsigned base = 0;
                        if (lane == 0) base = atomicAdd(&S.F, (unsigned)(__popc(b0) + __popc(b1)));
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
            if (lane == 0) {
                S.red_lo[wid] = wlo;
                S.red_hi[wid] = whi;
            }
            __syncthreads();
            const unsigned F = S.F;
            // each listed vertex's arcs and group bounds are prefetched into
            // L2 now (the owners read them after the barrier); a short list
            // goes into every CTA's inbox
            for (unsigned e = tid; e < F; e += CL_THREADS) {
                const unsigned sl = lst[e];
                const unsigned long long p = (unsigned long long)sl * C + r;
                prefetch_l2(tcol, 4ull * A.tarc_cap, 4ull * tst[sl], 4ull * tdg[sl]);
                if (!dg) prefetch_l2(tcw, 8ull * A.tarc_cap, 8ull * tst[sl], 8ull * tdg[sl]);
                prefetch_l2(A.tgrp, grp_bytes, 4ull * DUPIN_GRP_STRIDE * p, 4ull * DUPIN_GRP_STRIDE);
            }
            if (F <= CL_INL)
                for (unsigned x = tid; x < F * C; x += CL_THREADS) {
                    const unsigned e = x >> lg, o = x & (C - 1);
                    cl_st_u32(cl_map(&S.inl[r][e], o), (unsigned)lst[e] * C + r);
                }
            if (wid == 0) {  // the CTA's count and weight sum, pushed into every CTA's inbox
                unsigned long long l = lane < CL_WARPS ? S.red_lo[lane] : 0, h = lane < CL_WARPS ? S.red_hi[lane] : 0;
                warp_sum128(l, h);
                l = __shfl_sync(0xffffffffu, l, 0);
                h = __shfl_sync(0xffffffffu, h, 0);
                if (lane < (int)C) {
                    const uint32_t b = cl_map(&S.sel[par][r], lane);
                    cl_st_u32(b + offsetof(ClSel, cnt), F);
                    cl_st_u64(b + offsetof(ClSel, w_lo), l);
                    cl_st_u64(b + offsetof(ClSel, w_hi), h);
                }
            }
            cl_sync();  // A: every CTA's selection and list are visible
            if (tid == 0) S.F = 0;  // every thread has read it
            if (wid == 0) {  // per CTA: selected vertices and their prefix
                const unsigned c = lane < (int)C ? S.sel[par][lane].cnt : 0;
                unsigned ic = c;
#pragma unroll
                for (int k = 1; k < 32; k <<= 1) {
                    const unsigned oc = __shfl_up_sync(0xffffffffu, ic, k);
                    if (lane >= k) ic += oc;
                }
                if (lane < (int)C) {
                    S.qcnt[lane] = c;
                    S.qcex[lane] = ic - c;
                }
            }
            Wl = lane < (int)C ? S.sel[par][lane].w_lo : 0;
            Wh = lane < (int)C ? S.sel[par][lane].w_hi : 0;
            if (NARROW) {
                Wl = warp_sum64_redux(Wl);
                Wh = 0;
            } else {
                warp_sum128(Wl, Wh);
                Wl = __shfl_sync(0xffffffffu, Wl, 0);
                Wh = __shfl_sync(0xffffffffu, Wh, 0);
            }
            __syncthreads();
        }
        // ---- E: this CTA's groups of the removed vertices' arcs
        const unsigned Ltot = S.qcex[C - 1] + S.qcnt[C - 1];
        unsigned long long ilo = 0, ihi = 0;
        // arcs into vertices this CTA owns: a survivor loses c (a returning
        // 64-bit shared-memory atomic; the segment minimum lowered by
        // atomicMin when the result falls below it), an arc into U_i adds c
        // to 'internal', an arc into an earlier round's removals is skipped.
        // The heads' states are read before any update (removal marks do not
        // change during the expand).
        auto arcs = [&](const long long (&pos)[CL_ILP]) {
            int cv[CL_ILP];
            long long cc[CL_ILP], wv[CL_ILP];
#pragma unroll
            for (int u = 0; u < CL_ILP; u++) {
                if (pos[u] >= 0) {
                    cv[u] = tcol[pos[u]];
                    cc[u] = dg ? DUPIN_Q_ONE : tcw[pos[u]];
                }
            }
#pragma unroll
            for (int u = 0; u < CL_ILP; u++) {
                wv[u] = kPad;
                if (pos[u] < 0) continue;
                const unsigned v = (unsigned)cv[u], sl = v >> lg;
                if ((v & (C - 1)) != r || (long long)sl >= nown) {  // not this CTA's vertex: a broken group
                    S.err = DUPIN_ERR_CUDA;
                    continue;
                }
                wv[u] = tw[sl];
            }
#pragma unroll
            for (int u = 0; u < CL_ILP; u++) {
                if (wv[u] >= 0) {
                    const unsigned sl = (unsigned)cv[u] >> lg;
                    const long long nv =
                        (long long)atomicAdd((unsigned long long *)&tw[sl], (unsigned long long)(-cc[u])) - cc[u];
                    if (nv < segmin[sl >> 6]) atomicMin(&segmin[sl >> 6], nv);  // segment minima only fall here
                } else if (wv[u] == -i) {
                    if (NARROW) ilo += (unsigned long long)cc[u];
                    else add128(ilo, ihi, (unsigned long long)cc[u], 0);
                }
            }
        };
        const bool built = fast && Ltot <= 32;  // the fast path built the only window
        for (unsigned w0 = 0; w0 < Ltot; w0 += CL_WIN) {  // block-uniform: a window of list entries
            const unsigned nw = Ltot - w0 < CL_WIN ? Ltot - w0 : CL_WIN;
            if (built) {
            } else if (nw <= 32) {
                if (wid == 0) build_window(w0, nw);
            } else {
                unsigned carry = 0;
                for (unsigned t0 = 0; t0 < nw; t0 += CL_THREADS) {
                    const unsigned t = t0 + tid;
                    unsigned gs = 0, len = 0;
                    if (t < nw) group(w0 + t, gs, len);
                    long long tot;
                    const long long ex = block_excl_scan<CL_WARPS>((long long)len, S.scan, tot);
                    if (t < nw) {
                        S.wbase[t] = carry + (unsigned)ex;
                        S.wstart[t] = gs;
                    }
                    carry += (unsigned)tot;
                }
                if (tid == 0) S.wbase[nw] = carry;
            }
            if (!built) __syncthreads();
            const unsigned wt = S.wbase[nw];
            for (unsigned xb = tid; xb < wt; xb += CL_ILP * CL_THREADS) {
                long long pos[CL_ILP];
#pragma unroll
                for (int u = 0; u < CL_ILP; u++) {
                    const unsigned xx = xb + u * CL_THREADS;
                    pos[u] = -1;
                    if (xx < wt) {
                        int lo2 = 0, hi2 = (int)nw - 1;  // last t with wbase[t] <= xx
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
            __syncthreads();  // the window is reused
        }
        publish(par, ilo, ihi);
        wait_results(par);  // every CTA's results of round i have arrived
        if (werr) {
            err = werr;
            break;
        }
        // ---- C: close round i and plan round i+1 (every warp, same values, local reads)
        long long Mn;
        bool over;
        unsigned long long Il, Ih;
        results(par, Mn, over, Il, Ih);
        preload(par, Mn, over);
        const long long Un = (long long)Ltot;
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
        fast = R.minrule && !over;
        pre = pre && fast;
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
    long long P = (long long)dyn / 18;
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
