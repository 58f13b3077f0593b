// dupin_common.cuh -- shared device/host definitions of libdupin (sm_103a).
//
// Data layout in HBM (one symmetric adjacency per graph, Sec. 2.1):
//   rp[n+1]  int64  row offsets          col[A] int32 neighbour ids
//   cw[A]    int64  Q32.32 arc weights (absent for DG: every arc weighs 1.0)
//   a[n]     int64  Q32.32 vertex weights (absent: 0)
// Peeling state (Algorithm 2, Sec. 4.1):
//   w[n]  int64  current peeling weight w_u(S)      pr[n] int32 round u left S
//   live lists (int32 ids), per-block staging, the round's frontier and the
//   per-round trace.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dupin.h"

typedef unsigned __int128 u128;

#define DUPIN_Q_ONE (1LL << 32)
#define DUPIN_LIVE 0x7fffffff

// In-kernel waits give up after this many polls (about a second with the
// back-off below) and report DUPIN_ERR_TIMEOUT instead of hanging.
#define DUPIN_SPIN_LIMIT (1ll << 21)

// A grid-wide round that removed at most this many vertices, or expanded at
// most DUPIN_TAIL_SMALL_ARCS arcs, is "small": once S fits a tail, the tail
// takes over after such a round whatever the live arc count.
#define DUPIN_TAIL_SMALL_ROUND 64
#define DUPIN_TAIL_SMALL_ARCS (1LL << 18)
// The one-CTA tail takes a live set of at most tail_cap vertices only when
// its sub-graph has at most this many arcs (one SM fetches them); larger
// ones go to the cluster tail.
#define DUPIN_ONE_CTA_ARCS (1LL << 20)
// ... provided its live sub-graph fits the tail's arc buffer (2^27 arcs)
#define DUPIN_TAIL_BUF_ARCS (1LL << 27)
#define DUPIN_GRP_STRIDE 17  // per tail row: its first arc, then each owner group's end (16 owners at most)

// Peeling phases recorded in PeelCtl::status
#define ST_RUNNING 0
#define ST_DONE 1
#define ST_TAIL 2     // the one-CTA tail finishes the peel
#define ST_CLUSTER 3  // the cluster tail finishes the peel

// Device-resident control block of one peel.  'bar_*' is the grid barrier;
// the rest is the state after the last completed round.
struct PeelCtl {
    unsigned int bar_count;
    unsigned int bar_gen;
    int error;
    int status;
    long long round;
    long long size;
    unsigned long long f_lo, f_hi;
    long long live_len;
    int live_sel;
    int pad0;
    long long minw;
    long long best_round, best_size;
    unsigned long long bf_lo, bf_hi;
    long long gpo_le;
    long long gpo_lt;  // Algorithm 4's strict form of tau_max: ceil(...) - 1
    long long n_min_rule;
    long long scan_volume;
    long long bulk_rounds;
    long long elive;      // |E(S)|: undirected edges with both ends live
    long long tail_arcs;  // arcs of the tail sub-graph (0 if the tail did not run)
    unsigned long long init_lo, init_hi;  // sum over u of (w_u + a_u) = 2 f(V)
    long long init_min;
    int init_overflow;
    int tail_ctas;  // CTAs of the tail that finished the peel (0: none ran)
    // loading checks (the initial-weight pass with its checks on): a row not
    // strictly increasing, and the symmetry fingerprint (0 when symmetric)
    int check_unsorted;
    int beside_cluster;  // a batched call's earlier peel is on a cluster tail: the grid-wide rounds run narrow
    unsigned long long check_fp;
};

// Per-block partial results of one bulk round (one 128-byte line each)
struct BlockPart {
    long long sel_cnt;    // vertices selected
    long long stage_cnt;  // selected vertices with at least one arc (frontier entries)
    long long sel_deg;    // their arcs
    unsigned long long ws_lo, ws_hi;  // sum of their peeling weights
    long long surv_cnt;   // live survivors in the block's range
    long long min_surv;   // minimum survivor weight
    unsigned long long in_lo, in_hi;  // expand: sum of c over arcs inside U
    long long min_dec;    // expand: minimum weight after a decrement
    long long rem_cnt;    // expand: 2 per arc from U to S \ U, 1 per arc inside U
    long long mc_cnt;     // minimum-rule candidates (live vertices of weight min_surv)
    long long mc_stage;   // ... with at least one arc
    long long mc_deg;     // ... and their arcs
    long long min_surv2;  // the smallest live weight above min_surv (minimum-rule blocks)
    long long pad[1];
};

// Hubs: up to DUPIN_HUB_MAX highest-degree vertices (degree >= DUPIN_HUB_MIN_DEG).
// An arc whose head is hub number h is stored in col[] as -(h + 1), so the
// expand can aggregate a round's decrements of a hub in shared memory.
#define DUPIN_HUB_MAX 1024
#define DUPIN_HUB_MIN_DEG 1024

struct DevGraph {
    long long n;
    long long arcs;
    const long long *rp;
    const int *col;       // neighbour ids; -(h + 1) for hub number h
    const long long *cw;  // nullptr: DG weights
    const long long *a;   // nullptr: 0
    const int *hubs;      // hub number -> vertex id
    int n_hubs;
    unsigned long long key;  // the symmetry fingerprint's key (loading checks only)
};

// neighbour id of an arc's stored column value
__device__ __forceinline__ int arc_head(int cv, const int *hubs) { return cv >= 0 ? cv : hubs[-cv - 1]; }

struct PeelArgs {
    DevGraph g;
    long long *w;
    int *pr;
    int *live0, *live1;
    int *stage_id;      // minimum-rule candidates: live-list positions
    long long *stage_start, *stage_off;
    long long *fstart, *fbase;
    long long *cstart;
    BlockPart *part;
    PeelCtl *ctl;
    long long *tr_f_hi;
    unsigned long long *tr_f_lo;
    long long *tr_size, *tr_peeled;
    long long tr_cap;
    long long kD;       // k (D + N)
    long long D;        // eps denominator
    int use_min;        // k (1 + eps) < 2: the minimum rule can fire
    int gpo;            // Algorithm 3
    int lpo;            // Algorithm 4 (with gpo)
    long long max_rounds;
    long long tail_cap;     // the one-CTA tail takes |S| <= tail_cap ...
    long long one_arcs;     // ... with 2 |E(S)| <= one_arcs; otherwise the cluster tail
    long long cl_cap;       // the cluster tail takes |S| <= cl_cap (0: no cluster tail)
    long long hcap;         // max(tail_cap, cl_cap): the grid-wide rounds hand over below it ...
    long long tail_arcs;    // ... once 2 |E(S)| <= tail_arcs or after a small round
    // tail sub-graph
    int *loc;           // global id -> local id (valid for live vertices)
    long long *tdeg;    // tail: full degree prefix [L+1]
    long long *tlrp;    // tail: live-degree prefix [L+1]
    int *tcnt;          // tail: per-row live-arc counts [L]
    int *tfill;         // tail: per-row fill counters [L]
    int *tcol;          // tail arcs: local neighbour ids
    long long *tcw;     // tail arcs: weights (nullptr for DG)
    long long tarc_cap;
    // cluster tail: each row's arcs grouped by the owner of their head (local
    // id mod cl_c); row p's group o is [tgrp[p G + o], tgrp[p G + o + 1]) for
    // G = DUPIN_GRP_STRIDE
    unsigned *tgrp;
    int cl_c;           // CTAs of the cluster tail (0: none)
};

// ---------------------------------------------------------------- helpers

// Arc counts stay below 2^40 (checked when a graph is loaded), so the even
// split of an arc or vertex range over at most 2^16 parts has a 64-bit product.
__host__ __device__ __forceinline__ long long split_at(long long T, long long c, long long G) {
    return (long long)(((unsigned long long)T * (unsigned long long)c) / (unsigned long long)G);
}

__host__ __device__ __forceinline__ u128 mk128(unsigned long long lo, unsigned long long hi) {
    return ((u128)hi << 64) | (u128)lo;
}

// floor((u1 2^64 + u0) / v) for u1 < v (the quotient fits in 64 bits):
// Knuth's Algorithm D (TAOCP vol. 2, 4.3.1) with 32-bit digits -- normalise v,
// estimate each of the two quotient digits from the top two dividend digits
// and the top divisor digit, and correct the estimate (at most twice).
__host__ __device__ __forceinline__ unsigned long long div_u128_u64(unsigned long long u1, unsigned long long u0,
                                                                    unsigned long long v) {
    const unsigned long long B = 1ull << 32;
#ifdef __CUDA_ARCH__
    const int s = __clzll((long long)v);
#else
    const int s = __builtin_clzll(v);
#endif
    v <<= s;
    const unsigned long long vn1 = v >> 32, vn0 = v & 0xffffffffull;
    const unsigned long long un32 = s ? (u1 << s) | (u0 >> (64 - s)) : u1;
    const unsigned long long un10 = u0 << s;
    const unsigned long long un1 = un10 >> 32, un0 = un10 & 0xffffffffull;
    unsigned long long q1 = un32 / vn1, rhat = un32 - q1 * vn1;
    while (q1 >= B || q1 * vn0 > ((rhat << 32) | un1)) {
        q1--;
        rhat += vn1;
        if (rhat >= B) break;
    }
    const unsigned long long un21 = (un32 << 32) + un1 - q1 * v;  // exact: the true value is below 2^64
    unsigned long long q0 = un21 / vn1;
    rhat = un21 - q0 * vn1;
    while (q0 >= B || q0 * vn0 > ((rhat << 32) | un0)) {
        q0--;
        rhat += vn1;
        if (rhat >= B) break;
    }
    return (q1 << 32) | q0;
}

// floor(X / Y) for 1 <= Y < 2^64, saturated to INT64_MAX, with integer
// operations only (the quotient is below 2^63 once saturation is ruled out,
// so X's high word is below Y).  Used once per round.
__host__ __device__ __forceinline__ long long floor_div_sat(u128 X, unsigned long long Y) {
    if (X >= ((u128)Y << 63)) return 0x7fffffffffffffffLL;
    return (long long)div_u128_u64((unsigned long long)(X >> 64), (unsigned long long)X, Y);
}

// exact threshold floor(num_mul * f / (den_mul * size)), saturated to INT64_MAX
__device__ __forceinline__ long long floor_ratio(unsigned long long num_mul, u128 f, unsigned long long den_mul,
                                                 long long size) {
    const u128 num = (u128)num_mul * f;
    const u128 den = (u128)den_mul * (u128)(unsigned long long)size;
    if (den >> 64) {  // only when den_mul * size >= 2^64 (not reached with the limits on eps and n)
        u128 q = num / den;
        return q > (u128)0x7fffffffffffffffULL ? 0x7fffffffffffffffLL : (long long)q;
    }
    return floor_div_sat(num, (unsigned long long)den);
}

// ceil(num_mul * f / (den_mul * size)) - 1 (the largest w with w < the
// ratio), saturated to INT64_MAX; -1 when the ratio is 0
__device__ __forceinline__ long long below_ratio(unsigned long long num_mul, u128 f, unsigned long long den_mul,
                                                 long long size) {
    const u128 num = (u128)num_mul * f;
    if (num == 0) return -1;
    const u128 den = (u128)den_mul * (u128)(unsigned long long)size;
    if (den >> 64) {
        u128 q = (num - 1) / den;
        return q > (u128)0x7fffffffffffffffULL ? 0x7fffffffffffffffLL : (long long)q;
    }
    return floor_div_sat(num - 1, (unsigned long long)den);
}

// w * Y <= X exactly, for 0 <= w < 2^63 (the division-free form of w <= floor(X / Y))
__device__ __forceinline__ bool mul_le(long long w, unsigned long long Y, unsigned long long Xhi,
                                       unsigned long long Xlo) {
    const unsigned long long lo = (unsigned long long)w * Y;
    const unsigned long long hi = __umul64hi((unsigned long long)w, Y);
    return hi < Xhi || (hi == Xhi && lo <= Xlo);
}

// a * b mod 2^128 for a 64-bit b (three multiplies instead of a 128x128 product)
__device__ __forceinline__ u128 mul_u128_u64(u128 a, unsigned long long b) {
    const unsigned long long alo = (unsigned long long)a, ahi = (unsigned long long)(a >> 64);
    const unsigned long long lo = alo * b;
    const unsigned long long hi = __umul64hi(alo, b) + ahi * b;
    return ((u128)hi << 64) | (u128)lo;
}

// a/b > c/d for the best-prefix rule (strict: earliest round wins ties);
// a, c < 2^96 and b, d < 2^31, so both products fit in 128 bits.  NARROW:
// a, c < 2^64 (one 64 x 64 -> 128-bit product each).
template <bool NARROW = false>
__device__ __forceinline__ bool frac_gt(u128 a, long long b, u128 c, long long d) {
    if (NARROW)
        return (u128)(unsigned long long)a * (unsigned long long)d > (u128)(unsigned long long)c * (unsigned long long)b;
    return mul_u128_u64(a, (unsigned long long)d) > mul_u128_u64(c, (unsigned long long)b);
}

__device__ __forceinline__ void add128(unsigned long long &lo, unsigned long long &hi, unsigned long long xlo,
                                       unsigned long long xhi) {
    unsigned long long s = lo + xlo;
    hi += xhi + (s < lo ? 1ull : 0ull);
    lo = s;
}

__device__ __forceinline__ void warp_sum128(unsigned long long &lo, unsigned long long &hi) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        unsigned long long olo = __shfl_down_sync(0xffffffffu, lo, d);
        unsigned long long ohi = __shfl_down_sync(0xffffffffu, hi, d);
        add128(lo, hi, olo, ohi);
    }
}

__device__ __forceinline__ long long warp_sum64(long long x) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_down_sync(0xffffffffu, x, d);
    return x;
}

// minimum over the warp, in every lane: the high words' minimum, then the
// minimum low word among the lanes that hold it (two 32-bit warp reductions)
__device__ __forceinline__ long long warp_min64(long long x) {
    const int hi = (int)(x >> 32);
    const int mh = __reduce_min_sync(0xffffffffu, hi);
    const unsigned ml = __reduce_min_sync(0xffffffffu, hi == mh ? (unsigned)x : 0xffffffffu);
    return (long long)(((unsigned long long)(unsigned)mh << 32) | ml);
}

// sum over the warp, in every lane, exact while the total is below 2^64:
// three 32-bit warp reductions of 21-bit chunks (a chunk's sum over 32
// lanes stays below 2^27)
__device__ __forceinline__ unsigned long long warp_sum64_redux(unsigned long long x) {
    const unsigned M = (1u << 21) - 1;
    const unsigned s0 = __reduce_add_sync(0xffffffffu, (unsigned)x & M);
    const unsigned s1 = __reduce_add_sync(0xffffffffu, (unsigned)(x >> 21) & M);
    const unsigned s2 = __reduce_add_sync(0xffffffffu, (unsigned)(x >> 42));
    return (unsigned long long)s0 + ((unsigned long long)s1 << 21) + ((unsigned long long)s2 << 42);
}

// inclusive warp scan of a 64-bit value
__device__ __forceinline__ long long warp_incl_scan64(long long x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        long long o = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += o;
    }
    return x;
}

// A keyed 64-bit fingerprint of an arc (u -> v, weight c) for symmetry
// checks: summed over all arcs with a wrapping add, sym_mix(u, v, c) and
// sym_mix(v, u, c) give the same total when every arc has a reverse arc of
// the same weight (the multiset of arcs equals its reverse); a missing or
// re-weighted reverse arc leaves the totals different except with
// probability about 2^-64 over the key.  (SplitMix64's finaliser.)
__host__ __device__ __forceinline__ unsigned long long fmix64(unsigned long long x) {
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ULL;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebULL;
    x ^= x >> 31;
    return x;
}
__host__ __device__ __forceinline__ unsigned long long sym_mix(unsigned long long key, long long u, long long v,
                                                               long long c) {
    const unsigned long long h = fmix64(key ^ (((unsigned long long)u << 32) | (unsigned long long)(unsigned)v));
    return fmix64(h + (unsigned long long)c * 0x9e3779b97f4a7c15ULL + key);
}

__device__ __forceinline__ void set_error(PeelCtl *ctl, int code) { atomicCAS(&ctl->error, 0, code); }

__device__ __forceinline__ unsigned ld_volatile_u32(const unsigned *p) {
    return *(volatile const unsigned *)p;
}

__device__ __forceinline__ int ld_volatile_i32(const int *p) { return *(volatile const int *)p; }

// Grid-wide barrier for a cooperative launch (every block resident).
// ctl->bar_count counts the arrivals since the control block was reset; a
// barrier is complete once it reaches the running total of the block counts
// of all barriers so far (kept by the caller, advanced here by nblocks;
// thread 0's copy is the one used).  One release-add to arrive and acquire
// loads to wait, with no reset step between barriers; the error flag is read
// alongside.
// Waiting is bounded: after DUPIN_SPIN_LIMIT polls the block records
// DUPIN_ERR_TIMEOUT and every block leaves at its next barrier.  Returns
// false when the peel must stop.
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned atom_add_release_u32(unsigned *p, unsigned x) {
    unsigned v;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "r"(x) : "memory");
    return v;
}

__device__ __forceinline__ bool grid_barrier(PeelCtl *ctl, unsigned nblocks, unsigned &target_acc) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        target_acc += nblocks;
        const unsigned target = target_acc;  // wraps consistently with the counter
        __threadfence();  // the block's writes (ordered by the block barrier) before the arrival
        unsigned v = atom_add_release_u32(&ctl->bar_count, 1u) + 1u;
        int err = ld_volatile_i32(&ctl->error);
        int ok = 1;
        long long it = 0;
        while ((int)(v - target) < 0 && err == 0) {
            if (++it > DUPIN_SPIN_LIMIT) {
                set_error(ctl, DUPIN_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            if (it > 256) __nanosleep(it > 8192 ? 256 : 20);
            v = ld_acquire_u32(&ctl->bar_count);
            err = ld_volatile_i32(&ctl->error);
        }
        __threadfence();
        s_ok = ok && err == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

// Largest k in [0, U] with base[k] <= x, for non-decreasing base with
// base[0] <= x.  One warp, 32 probes per step (log_32 U dependent loads).
__device__ __forceinline__ long long warp_search_last_le(const long long *base, long long U, long long x) {
    const int lane = threadIdx.x & 31;
    long long lo = 0, hi = U;
    while (lo < hi) {
        long long span = hi - lo;  // candidates lo+1 .. hi
        long long p;
        if (span <= 32) p = lo + 1 + lane;
        else p = lo + 1 + (long long)(((unsigned long long)(span - 1) * (unsigned)lane) / 31u);
        bool valid = p <= hi;
        bool le = valid && base[p] <= x;
        unsigned m = __ballot_sync(0xffffffffu, le);
        if (m == 0) {
            long long p0 = __shfl_sync(0xffffffffu, p, 0);
            hi = p0 - 1;
        } else {
            int L = 31 - __clz(m);
            long long pl = __shfl_sync(0xffffffffu, p, L);
            long long pn = __shfl_sync(0xffffffffu, p, L < 31 ? L + 1 : 31);
            bool nvalid = __shfl_sync(0xffffffffu, (int)valid, L < 31 ? L + 1 : 31);
            lo = pl;
            if (L < 31 && nvalid) hi = pn - 1;
        }
    }
    return lo;
}
