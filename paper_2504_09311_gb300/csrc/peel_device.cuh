// peel_device.cuh -- device building blocks shared by the peel kernels
// (single graph: peel.cu; many graphs, one CTA each: batch.cu).
#pragma once
#include "dupin_common.cuh"

#define BULK_THREADS 1024
#define BULK_WARPS (BULK_THREADS / 32)
#define WALK_WIN 1024
#ifndef BULK_ILP
#define BULK_ILP 1  // arcs in flight per thread in the grid-wide expand (1 measured best)
#endif
#define INIT_THREADS 256
#define INIT_WARPS (INIT_THREADS / 32)
#ifndef INIT_UNROLL
#define INIT_UNROLL 4  // 32-arc chunks whose loads a warp issues together in the initial weights
#endif
#ifndef TAIL_THREADS
#define TAIL_THREADS 256
#endif
#define TAIL_WARPS (TAIL_THREADS / 32)
#define SCAN_THREADS 1024


static const long long kMaxLL = 0x7fffffffffffffffLL;

// ------------------------------------------------------------ block helpers

// Block-wide reduction of NV 64-bit sums, one u128 sum and one minimum.
// All threads get the results.  Two __syncthreads.
template <int NWARPS, int NV>
struct BlockRed {
    long long v[NV];
    unsigned long long lo, hi;
    long long mn;
};

template <int NWARPS, int NV>
__device__ __forceinline__ void block_reduce(BlockRed<NWARPS, NV> &r, long long (*s_v)[NV], unsigned long long *s_lo,
                                             unsigned long long *s_hi, long long *s_mn) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; j++) r.v[j] = warp_sum64(r.v[j]);
    warp_sum128(r.lo, r.hi);
    r.mn = warp_min64(r.mn);
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < NV; j++) s_v[wid][j] = r.v[j];
        s_lo[wid] = r.lo;
        s_hi[wid] = r.hi;
        s_mn[wid] = r.mn;
    }
    __syncthreads();
    if (wid == 0) {
        bool in = lane < NWARPS;
#pragma unroll
        for (int j = 0; j < NV; j++) r.v[j] = in ? s_v[lane][j] : 0;
        r.lo = in ? s_lo[lane] : 0;
        r.hi = in ? s_hi[lane] : 0;
        r.mn = in ? s_mn[lane] : kMaxLL;
#pragma unroll
        for (int j = 0; j < NV; j++) r.v[j] = warp_sum64(r.v[j]);
        warp_sum128(r.lo, r.hi);
        r.mn = warp_min64(r.mn);
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < NV; j++) s_v[0][j] = r.v[j];
            s_lo[0] = r.lo;
            s_hi[0] = r.hi;
            s_mn[0] = r.mn;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; j++) r.v[j] = s_v[0][j];
    r.lo = s_lo[0];
    r.hi = s_hi[0];
    r.mn = s_mn[0];
    __syncthreads();
}

// Exclusive block scan of one 64-bit value per thread; 'total' gets the sum.
template <int NWARPS>
__device__ __forceinline__ long long block_excl_scan(long long x, long long *s_w, long long &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long incl = warp_incl_scan64(x);
    if (lane == 31) s_w[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        long long v = lane < NWARPS ? s_w[lane] : 0;
        v = warp_incl_scan64(v);
        if (lane < NWARPS) s_w[lane] = v;
    }
    __syncthreads();
    long long before = wid ? s_w[wid - 1] : 0;
    total = s_w[NWARPS - 1];
    __syncthreads();
    return before + incl - x;
}

// last t in [0, WALK_WIN] with s[t] <= x (s non-decreasing, s[0] <= x):
// a fixed number of predicated steps, so that several searches interleave
__device__ __forceinline__ int smem_last_le_fixed(const long long *s, long long x) {
    static_assert((WALK_WIN & (WALK_WIN - 1)) == 0, "WALK_WIN: a power of two");
    int t = 0;
#pragma unroll
    for (int step = WALK_WIN; step > 0; step >>= 1)
        if (t + step <= WALK_WIN && s[t + step] <= x) t += step;
    return t;
}

// last t in [0, n) with s[t] <= x (s non-decreasing, s[0] <= x)
__device__ __forceinline__ int smem_last_le(const long long *s, int n, long long x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (s[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Walk the arcs [e0, e1) of a segmented arc space.  Entry k (0 <= k < U)
// covers [base(k), base(k+1)) and its arcs sit at col positions start(k) + (x -
// base(k)); base(U) is the total.  k0 must satisfy base(k0) <= e0.  The
// block loads WALK_WIN entries at a time into shared memory and calls
// fn(k, pos) once per arc, consecutive threads on consecutive arcs.
template <class BaseF, class StartF, class ArcF>
__device__ __forceinline__ void walk_arcs(BaseF base, StartF start, long long U, long long e0, long long e1,
                                          long long k0, long long *s_base, long long *s_start, ArcF fn) {
    long long e = e0, k = k0;
    while (e < e1) {
        __syncthreads();
        for (int t = threadIdx.x; t <= WALK_WIN; t += blockDim.x) {
            long long idx = k + t;
            s_base[t] = idx <= U ? base(idx) : kMaxLL;
            s_start[t] = idx < U ? start(idx) : 0;
        }
        __syncthreads();
        long long wend = s_base[WALK_WIN];
        long long hi = e1 < wend ? e1 : wend;
        for (long long x = e + threadIdx.x; x < hi; x += blockDim.x) {
            int t = smem_last_le(s_base, WALK_WIN, x);
            fn(k + t, s_start[t] + (x - s_base[t]));
        }
        int t2 = smem_last_le(s_base, WALK_WIN + 1, hi);
        k += t2;
        e = hi;
    }
}


struct RoundState {
    long long round, size;
    u128 f;
    long long live_len;
    int live_sel;
    long long minw;
    long long best_round, best_size;
    u128 bf;
    long long gpo_le, gpo_lt, n_min_rule, scan;
    u128 gm_f;       // the largest g(S) = gm_f / gm_s a main round has started from
    long long gm_s;  // (0: none yet); tau_max only changes when g(S) exceeds it
};


// Shared accumulator of one tail round (double-buffered by round parity).
// F is a 32-bit shared counter; the sums are written per warp by its lane 0
// and added up by every thread when it closes the round: shared-memory
// atomics on 64-bit words are compare-and-swap loops that collapse when
// several warps hit one word.
template <int NW>
struct TailAcc {
    unsigned F;                          // |U_i|
    unsigned long long wlo[NW], whi[NW];  // sum of the removed vertices' weights
    unsigned long long ilo[NW], ihi[NW];  // sum of c over arcs inside U
    long long mins[NW];                   // minimum live weight after the round
};

// the round's totals from the warps' parts: lane j < NW loads part j and a
// butterfly over the lanes leaves the totals in every lane (NW a power of
// two, <= 32).  NARROW: the totals are below 2^64 (high words unused), and
// 32-bit warp reductions replace the butterfly.
template <int NW, bool NARROW = false>
__device__ __forceinline__ void tail_acc_sum(const TailAcc<NW> &acc, u128 &wsel, u128 &internal, long long &mins) {
    static_assert(NW > 0 && NW <= 32 && (NW & (NW - 1)) == 0, "warps per block: a power of two");
    const int lane = threadIdx.x & 31;
    const bool in = lane < NW;
    if (NARROW) {
        wsel = (u128)warp_sum64_redux(in ? acc.wlo[lane] : 0ull);
        internal = (u128)warp_sum64_redux(in ? acc.ilo[lane] : 0ull);
        mins = warp_min64(in ? acc.mins[lane] : 0x7fffffffffffffffLL);
        return;
    }
    unsigned long long wl = in ? acc.wlo[lane] : 0, wh = in ? acc.whi[lane] : 0;
    unsigned long long il = in ? acc.ilo[lane] : 0, ih = in ? acc.ihi[lane] : 0;
    long long m = in ? acc.mins[lane] : 0x7fffffffffffffffLL;
#pragma unroll
    for (int d = 1; d < NW; d <<= 1) {
        const unsigned long long owl = __shfl_xor_sync(0xffffffffu, wl, d), owh = __shfl_xor_sync(0xffffffffu, wh, d);
        const unsigned long long oil = __shfl_xor_sync(0xffffffffu, il, d), oih = __shfl_xor_sync(0xffffffffu, ih, d);
        const long long om = __shfl_xor_sync(0xffffffffu, m, d);
        add128(wl, wh, owl, owh);
        add128(il, ih, oil, oih);
        m = om < m ? om : m;
    }
    // lanes 0 .. NW-1 hold the totals (a power-of-two NW); broadcast lane 0's
    wl = __shfl_sync(0xffffffffu, wl, 0);
    wh = __shfl_sync(0xffffffffu, wh, 0);
    il = __shfl_sync(0xffffffffu, il, 0);
    ih = __shfl_sync(0xffffffffu, ih, 0);
    m = __shfl_sync(0xffffffffu, m, 0);
    wsel = mk128(wl, wh);
    internal = mk128(il, ih);
    mins = m;
}

// The parameters of one round, computed identically by every warp.
struct TailRound {
    long long i;                  // round number
    unsigned long long Xhi, Xlo;  // X = k (D+N) f
    unsigned long long Y;         // Y = D |S|
    long long gle;                // Algorithm 3's floor(tau_max), -1 without GPO
    long long minw;               // minimum live weight
    int minrule;                  // threshold selects nobody: take the minimum
    int trim;                     // Algorithm 4's trim round
    int done;                     // S is empty
};

#define TAIL_FAST 32
#define TAIL_SEG 64  // vertices per segment (one warp, two per lane)
#define TAIL_ILP 4   // arcs in flight per thread in the tail's expand

// can segment minimum sm hold a vertex that round R selects?
__device__ __forceinline__ bool seg_candidate(long long sm, const TailRound &R) {
    if (sm == kMaxLL) return false;
    return R.minrule ? sm == R.minw : (sm <= R.gle || mul_le(sm, R.Y, R.Xhi, R.Xlo));
}

// Every warp (all lanes, identical result): plan round st.round + 1 from the
// state and the minimum live weight m -- thresholds and the minimum rule.
// With Algorithm 4 (lpo) the round is a trim round while some live w < g(S),
// i.e. m |S| <= f - 1: it removes w < max(tau_max, g), in the same
// division-free form (w <= gpo_lt or w |S| <= f - 1).  A main round refines
// tau_max (Algorithm 3) in both its forms.  NARROW: f and the g(S) it is compared with
// are below 2^64.
template <bool NARROW = false>
__device__ __forceinline__ TailRound tail_plan(long long kD, long long D, int use_min, int gpo, int lpo,
                                               RoundState &st, long long m) {
    TailRound R;
    R.i = st.round + 1;
    R.minw = m;
    R.done = st.size == 0 ? 1 : 0;
    R.minrule = 0;
    R.trim = 0;
    if (lpo && st.round > 0 && st.size > 0 && st.f != 0) {  // trims follow a round
        const u128 X = st.f - 1;
        const unsigned long long Xhi = (unsigned long long)(X >> 64), Xlo = (unsigned long long)X;
        if (mul_le(m, (unsigned long long)st.size, Xhi, Xlo)) {
            R.trim = 1;
            R.Xhi = Xhi;
            R.Xlo = Xlo;
            R.Y = (unsigned long long)st.size;
            R.gle = st.gpo_lt;
            return R;
        }
    }
    const u128 X = NARROW ? (u128)(unsigned long long)st.f * (unsigned long long)kD
                          : mul_u128_u64(st.f, (unsigned long long)kD);
    R.Xhi = (unsigned long long)(X >> 64);
    R.Xlo = (unsigned long long)X;
    R.Y = (unsigned long long)D * (unsigned long long)st.size;
    R.gle = -1;
    if (gpo && st.size > 0) {
        // floor and ceil-1 are monotone in g, so tau_max's integer forms can
        // only grow when g(S) exceeds the largest g seen so far
        if (st.gm_s == 0 || frac_gt<NARROW>(st.f, st.size, st.gm_f, st.gm_s)) {
            st.gm_f = st.f;
            st.gm_s = st.size;
            const long long le = floor_ratio((unsigned long long)D, st.f, (unsigned long long)kD, st.size);
            st.gpo_le = le > st.gpo_le ? le : st.gpo_le;
            if (lpo) {
                const long long lt = below_ratio((unsigned long long)D, st.f, (unsigned long long)kD, st.size);
                st.gpo_lt = lt > st.gpo_lt ? lt : st.gpo_lt;
            }
        }
        R.gle = st.gpo_le;
    }
    R.minrule = (use_min && st.size > 0 && !mul_le(m, R.Y, R.Xhi, R.Xlo) && m > R.gle) ? 1 : 0;
    return R;
}

// minimum of segment minima (one warp; all lanes get the result)
__device__ __forceinline__ long long seg_global_min(const long long *segmin, int nseg) {
    const int lane = threadIdx.x & 31;
    long long m = kMaxLL;
    for (int q = lane; q < nseg; q += 32) m = segmin[q] < m ? segmin[q] : m;
    m = warp_min64(m);
    return __shfl_sync(0xffffffffu, m, 0);
}
