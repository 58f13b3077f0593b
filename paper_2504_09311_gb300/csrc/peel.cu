// peel.cu -- Dupin's parallel batch peeling (Algorithm 2, Sec. 4.1) on sm_103a.
//
// One peel = four stages, all on the caller's stream:
//  (a) initial peeling weights w_u(V) = a_u + sum_v c_uv: an arc-balanced
//      segmented sum over the CSR (each warp streams a contiguous arc range,
//      carries the open row across chunks, so a hub row costs one atomic per
//      warp), then f(V) = sum_u (w_u + a_u) / 2 and min_u w_u;
//  (b)-(c) the bulk rounds in one persistent cooperative kernel, three grid
//      barriers per round:
//        A  select: scan this block's slice of the live list, peel every u
//           with w_u <= T_i (T_i = floor(k (D+N) f / (D |S|)), or the minimum
//           live weight when T_i selects nobody); stage the frontier with one
//           packed (count, arcs) shared atomic per warp;
//        B  place: prefix the per-block counts, write the frontier with its
//           arc offsets, record where each consumer block's equal share of
//           the round's arcs starts (merge path), compact the live list when
//           it has halved;
//        C  expand: walk this block's share of the frontier's arcs, subtract
//           c_uv from every surviving neighbour with an int64 atomic, sum c
//           over arcs inside U_i, and take the minimum post-decrement weight
//           (the next round's minimum-rule candidate);
//        D  (every block, redundantly) f_i = f_{i-1} - (sum_{u in U} w_u -
//           internal/2), |S_i|, the best prefix, the trace;
//  (d) once |S| <= tail_cap: the live vertices' induced subgraph is built
//      (local ids, live arcs only) and one CTA runs the remaining rounds with
//      w and the vertex states in shared memory.
// Every step is exact integer arithmetic, so the per-round sets, the trace
// and the best set equal the single-threaded oracle's bit for bit.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <string>

#include <chrono>
#include <mutex>

#include "dupin_internal.h"
#include "peel_device.cuh"



// ------------------------------------------------------------- (a) init

// w_u = a_u (DW/FD) or deg_u * 1.0 (DG); every vertex live; live list = ids.
__global__ void k_init_vertex(DevGraph g, int dg, long long *w, int *pr, int *live0, PeelCtl *ctl) {
    long long n = g.n;
    unsigned long long lo = 0, hi = 0;
    long long mn = kMaxLL;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
        long long wu;
        if (dg) {
            wu = (g.rp[u + 1] - g.rp[u]) << 32;
            add128(lo, hi, (unsigned long long)wu, 0);
            mn = wu < mn ? wu : mn;
        } else {
            wu = g.a ? g.a[u] : 0;
            if (wu < 0) atomicExch(&ctl->init_overflow, 2);
        }
        w[u] = wu;
        if (pr) pr[u] = DUPIN_LIVE;
        if (live0) live0[u] = (int)u;
    }
    if (dg) {
        warp_sum128(lo, hi);
        mn = warp_min64(mn);
        if ((threadIdx.x & 31) == 0) {
            unsigned long long old = atomicAdd(&ctl->init_lo, lo);
            if (old + lo < old) hi += 1;
            if (hi) atomicAdd(&ctl->init_hi, hi);
            atomicMin(&ctl->init_min, mn);
        }
    }
}

// Arc-balanced segmented sum: w_u += sum of c over row u.  The arc range is
// split evenly over all warps of the grid; each warp walks its range in
// 32-arc chunks, finds each arc's row from 32 cached row ends (5 shuffle
// steps), reduces rows within the chunk with a segmented scan and keeps the
// open last row in registers, so a row spanning many chunks is flushed once
// per warp.  The loads of INIT_UNROLL chunks are issued together; registers
// are held to what 6 resident blocks per SM allow (measured 3% faster on
// R-MAT-24 than the default budget).  CHECK also validates ids, self-loops
// and int64 overflow.
template <bool CHECK>
__global__ void __launch_bounds__(INIT_THREADS, CHECK ? 1 : 6) k_init_arcs(DevGraph g, long long *w, PeelCtl *ctl) {
    const int lane = threadIdx.x & 31;
    const long long NW = (long long)gridDim.x * INIT_WARPS;
    const long long W = blockIdx.x * (long long)INIT_WARPS + (threadIdx.x >> 5);
    const long long A = g.arcs, n = g.n;
    const long long we0 = split_at(A, W, NW);
    const long long we1 = split_at(A, W + 1, NW);
    if (we0 >= we1) return;
    long long r = warp_search_last_le(g.rp, n, we0);  // row of the first arc
    long long carry_own = -1, carry_val = 0;
    bool bad = false;
    // CHECK: rows strictly increasing (each arc against the next, across
    // chunks through the last arc seen, across warps through the arc before
    // the range) and the symmetry fingerprint
    bool unsorted = false;
    unsigned long long fp = 0;
    long long prev_row = -1;
    int prev_col = 0;
    if (CHECK && g.rp[r] < we0) {  // the range starts inside row r: compare with the arc before it
        prev_row = r;
        prev_col = g.col[we0 - 1];
    }
    auto check_chunk = [&](const long long own, const int cvx, const long long val, const long long x,
                           const bool valid) {
        const int ncol = __shfl_down_sync(0xffffffffu, cvx, 1);
        const long long nown = __shfl_down_sync(0xffffffffu, own, 1);
        if (valid && lane < 31 && x + 1 < we1 && nown == own && ncol <= cvx) unsorted = true;
        if (lane == 0 && valid && own == prev_row && cvx <= prev_col) unsorted = true;
        if (valid) fp += sym_mix(g.key, own, cvx, val) - sym_mix(g.key, cvx, own, val);
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        const int lst = 31 - __clz(vm);
        prev_row = __shfl_sync(0xffffffffu, own, lst);
        prev_col = __shfl_sync(0xffffffffu, cvx, lst);
    };
    long long r_end = g.rp[r + 1];  // end of row r
    long long lacc = 0;             // per-lane partial sum of row r over whole-row chunks
    // one 32-arc chunk whose weights (and, with CHECK, heads) are already loaded
    auto chunk = [&](const long long x0, const long long val, const int cvx) {
        const long long x = x0 + lane;
        const bool valid = x < we1;
        if (CHECK && valid) {
            if (cvx < 0 || cvx >= n || val < 0) bad = true;
        }
        // fast path: the whole chunk lies in row r (long rows, hubs)
        const long long cend = x0 + 32 < we1 ? x0 + 32 : we1;
        if (cend <= r_end) {
            if (CHECK) check_chunk(r, cvx, val, x, valid);
            if (CHECK && valid && cvx == r) bad = true;  // self-loop
            if (CHECK && (unsigned long long)lacc + (unsigned long long)val < (unsigned long long)lacc) bad = true;
            lacc += val;
            return;
        }
        // leaving row r inside this chunk: fold the lanes' partials into the carry
        {
            long long sum = warp_sum64(lacc);
            sum = __shfl_sync(0xffffffffu, sum, 0);
            lacc = 0;
            if (sum != 0) {
                if (carry_own == r) carry_val += sum;
                else {
                    if (carry_own >= 0 && lane == 0)
                        atomicAdd((unsigned long long *)&w[carry_own], (unsigned long long)carry_val);
                    carry_own = r;
                    carry_val = sum;
                }
            }
        }
        // Row of each lane's arc: with the 32 row ends rp[rr+1 .. rr+32] held
        // one per lane, a lane whose arc x has rp[rr] <= x < rp[rr+32] lies in
        // row rr + #{j : rp[rr+1+j] <= x} (5 shuffle steps).  Lanes further
        // out wait while the window moves on by 32 rows.
        long long owner = valid ? -1 : kMaxLL;
        long long rr = r;
        for (;;) {
            const long long idx = rr + 1 + lane;
            const long long bj = idx <= n ? g.rp[idx] : kMaxLL;
            // count in [0, 32]: 33 outcomes, so six halving steps
            int lo = 0, hi = 32;
#pragma unroll
            for (int s = 0; s < 6; s++) {
                const int mid = (lo + hi) >> 1;
                const long long bm = __shfl_sync(0xffffffffu, bj, mid & 31);
                if (lo < hi) {
                    if (bm <= x) lo = mid + 1;
                    else hi = mid;
                }
            }
            if (owner < 0 && lo < 32) owner = rr + lo;
            if (!__any_sync(0xffffffffu, owner < 0)) break;
            rr += 32;
        }
        if (CHECK && valid && cvx == owner) bad = true;
        if (CHECK) check_chunk(owner, cvx, val, x, valid);
        // segmented inclusive scan by owner
        long long sv = val;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            long long ov = __shfl_up_sync(0xffffffffu, sv, d);
            long long oo = __shfl_up_sync(0xffffffffu, owner, d);
            if (lane >= d && oo == owner) {
                if (CHECK && (unsigned long long)sv + (unsigned long long)ov < (unsigned long long)sv) bad = true;
                sv += ov;
            }
        }
        long long on = __shfl_down_sync(0xffffffffu, owner, 1);
        const unsigned vmask = __ballot_sync(0xffffffffu, valid);
        const int last = 31 - __clz(vmask);
        const bool is_end = valid && (lane == last || on != owner);
        const long long o0 = __shfl_sync(0xffffffffu, owner, 0);
        const long long oL = __shfl_sync(0xffffffffu, owner, last);
        if (carry_own >= 0 && carry_own != o0) {
            if (lane == 0) {
                if (CHECK) {
                    unsigned long long old = atomicAdd((unsigned long long *)&w[carry_own], (unsigned long long)carry_val);
                    if (old + (unsigned long long)carry_val < old) bad = true;
                } else {
                    atomicAdd((unsigned long long *)&w[carry_own], (unsigned long long)carry_val);
                }
            }
            carry_own = -1;
            carry_val = 0;
        }
        const long long add = (carry_own == o0) ? carry_val : 0;
        if (is_end && owner != oL) {
            long long tot = sv + (owner == o0 ? add : 0);
            if (CHECK) {
                unsigned long long old = atomicAdd((unsigned long long *)&w[owner], (unsigned long long)tot);
                if (old + (unsigned long long)tot < old) bad = true;
            } else {
                atomicAdd((unsigned long long *)&w[owner], (unsigned long long)tot);
            }
        }
        long long lastsum = __shfl_sync(0xffffffffu, sv, last);
        carry_val = lastsum + (oL == o0 ? add : 0);
        carry_own = oL;
        r = oL;  // the next chunk starts in this row or later
        r_end = g.rp[r + 1];
    };
    // INIT_UNROLL chunks per step: their loads are issued before any is processed
    for (long long xb = we0; xb < we1; xb += 32 * INIT_UNROLL) {
        long long vals[INIT_UNROLL];
        int cvs[INIT_UNROLL];
#pragma unroll
        for (int u = 0; u < INIT_UNROLL; u++) {
            const long long x = xb + 32 * u + lane;
            vals[u] = x < we1 ? g.cw[x] : 0;
            cvs[u] = (CHECK && x < we1) ? g.col[x] : 0;
        }
#pragma unroll
        for (int u = 0; u < INIT_UNROLL; u++)
            if (xb + 32 * u < we1) chunk(xb + 32 * u, vals[u], cvs[u]);
    }
    {
        long long sum = warp_sum64(lacc);
        sum = __shfl_sync(0xffffffffu, sum, 0);
        if (sum != 0) {
            if (carry_own == r) carry_val += sum;
            else {
                if (carry_own >= 0 && lane == 0)
                    atomicAdd((unsigned long long *)&w[carry_own], (unsigned long long)carry_val);
                carry_own = r;
                carry_val = sum;
            }
        }
    }
    if (carry_own >= 0 && lane == 0) {
        if (CHECK) {
            unsigned long long old = atomicAdd((unsigned long long *)&w[carry_own], (unsigned long long)carry_val);
            if (old + (unsigned long long)carry_val < old) bad = true;
        } else {
            atomicAdd((unsigned long long *)&w[carry_own], (unsigned long long)carry_val);
        }
    }
    if (CHECK && __any_sync(0xffffffffu, bad) && lane == 0) atomicExch(&ctl->init_overflow, 1);
    if (CHECK) {
        if (__any_sync(0xffffffffu, unsorted) && lane == 0) atomicExch(&ctl->check_unsorted, 1);
        for (int d = 16; d > 0; d >>= 1) fp += __shfl_down_sync(0xffffffffu, fp, d);  // wrapping sum
        if (lane == 0 && fp) atomicAdd(&ctl->check_fp, fp);
    }
}

// sum over u of (w_u + a_u) and min w (DW/FD)
__global__ void k_init_reduce(DevGraph g, const long long *w, PeelCtl *ctl) {
    unsigned long long lo = 0, hi = 0;
    long long mn = kMaxLL;
    bool bad = false;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < g.n; u += (long long)gridDim.x * blockDim.x) {
        long long wu = w[u];
        if (wu < 0) bad = true;  // wrapped past 2^63
        add128(lo, hi, (unsigned long long)wu, 0);
        if (g.a) add128(lo, hi, (unsigned long long)g.a[u], 0);
        mn = wu < mn ? wu : mn;
    }
    warp_sum128(lo, hi);
    mn = warp_min64(mn);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(&ctl->init_overflow, 1);
    if ((threadIdx.x & 31) == 0) {
        unsigned long long old = atomicAdd(&ctl->init_lo, lo);
        if (old + lo < old) hi += 1;
        if (hi) atomicAdd(&ctl->init_hi, hi);
        atomicMin(&ctl->init_min, mn);
    }
}

int launch_init_weights(const DevGraph &dg, int metric, long long *w, int *pr, int *live0, PeelCtl *ctl, bool check,
                        cudaStream_t s) {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int vgrid = sms * 8;
    const bool isdg = metric == DUPIN_DG || dg.cw == nullptr;
    k_init_vertex<<<vgrid, 256, 0, s>>>(dg, isdg ? 1 : 0, w, pr, live0, ctl);
    if (!isdg) {
        if (dg.arcs > 0) {
            int agrid = sms * 8;
            if (check) k_init_arcs<true><<<agrid, INIT_THREADS, 0, s>>>(dg, w, ctl);
            else k_init_arcs<false><<<agrid, INIT_THREADS, 0, s>>>(dg, w, ctl);
        }
        k_init_reduce<<<vgrid, 256, 0, s>>>(dg, w, ctl);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return dupin_cuda_fail(e, "init kernels");
    return DUPIN_OK;
}

// f(V), |V|, round 0, best = S_0, trace entry 0
__global__ void k_init_finish(PeelArgs A, long long n) {
    PeelCtl *c = A.ctl;
    u128 s = mk128(c->init_lo, c->init_hi);
    u128 f = s >> 1;
    c->round = 0;
    c->size = n;
    c->f_lo = (unsigned long long)f;
    c->f_hi = (unsigned long long)(f >> 64);
    c->live_len = n;
    c->live_sel = 0;
    c->minw = n > 0 ? c->init_min : 0;
    c->best_round = 0;
    c->best_size = n;
    c->bf_lo = c->f_lo;
    c->bf_hi = c->f_hi;
    c->gpo_le = 0;
    c->gpo_lt = -1;
    c->n_min_rule = 0;
    c->scan_volume = 0;
    c->bar_count = 0;
    c->bar_gen = 0;
    c->elive = A.g.arcs / 2;
    c->tail_arcs = 0;
    if (c->init_overflow) c->error = DUPIN_ERR_OVERFLOW;
    c->tail_ctas = 0;
    if (n == 0) c->status = ST_DONE;
    else if (n <= A.hcap && A.g.arcs <= A.tail_arcs)
        c->status = n <= A.tail_cap && A.g.arcs <= A.one_arcs ? ST_TAIL : ST_CLUSTER;
    else c->status = ST_RUNNING;
    if (A.tr_cap > 0) {
        A.tr_f_hi[0] = (long long)c->f_hi;
        A.tr_f_lo[0] = c->f_lo;
        A.tr_size[0] = n;
        A.tr_peeled[0] = 0;
    }
}

// ------------------------------------------------------ (b)-(c) bulk rounds

// Stage one warp's frontier entries (lanes with 'stage' set) at block-local
// slots from a 32-bit shared counter: each entry's first arc and degree (the
// arc offsets follow from a scan in phase B).  Shared-memory atomics stay
// 32-bit: 64-bit ones are compare-and-swap loops that collapse under
// contention.
__device__ __forceinline__ void stage_entry(const PeelArgs &A, long long j0, bool stage, long long start,
                                            long long deg, unsigned *s_nst) {
    const int lane = threadIdx.x & 31;
    const unsigned bal = __ballot_sync(0xffffffffu, stage);
    if (!bal) return;
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(s_nst, (unsigned)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (stage) {
        const long long slot = (long long)base + __popc(bal & ((1u << lane) - 1u));
        A.stage_start[j0 + slot] = start;
        A.stage_off[j0 + slot] = deg;
    }
}

// The grid-wide rounds of one peel, run by blocks b = 0 .. G-1 of a cooperative
// launch (all of it, or one group of it).
__device__ __forceinline__ void peel_bulk_body(const PeelArgs &A, const int b, const unsigned G) {
    __shared__ long long s_v[BULK_WARPS][6];
    __shared__ unsigned long long s_lo[BULK_WARPS], s_hi[BULK_WARPS];
    __shared__ long long s_mn[BULK_WARPS];
    __shared__ unsigned s_nst;   // frontier entries staged by the block
    __shared__ unsigned s_surv;  // candidates / survivors placed by the block
    __shared__ long long s_scan[BULK_WARPS];
    __shared__ long long s_base[WALK_WIN + 1];
    __shared__ long long s_start[WALK_WIN + 1];
    __shared__ int s_hub[DUPIN_HUB_MAX];
    // a round's decrements of each hub, as two 32-bit words (hi gets the carries)
    __shared__ unsigned s_hlo[DUPIN_HUB_MAX], s_hhi[DUPIN_HUB_MAX];
    // The state after the last completed round lives in shared memory, not in
    // registers: thread 0 updates it at the end of a round (phase D) and a
    // block barrier publishes it.  s_rd carries phase B's totals to phase D.
    __shared__ RoundState s_st;
    __shared__ long long s_elive;  // |E(S)|
    __shared__ struct {
        unsigned long long wlo, whi;  // sum of the selected vertices' weights
        long long U_sel, newSize;
        long long arcs;     // arcs the round expanded
        long long minsurv;  // minimum weight of this round's survivors before its decrements
        int minrule, compact;
    } s_rd;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    PeelCtl *ctl = A.ctl;
    const DevGraph g = A.g;
    const bool dg = g.cw == nullptr;
    const int nh = g.n_hubs;
    for (int h = tid; h < nh; h += BULK_THREADS) {
        s_hub[h] = g.hubs[h];
        s_hlo[h] = 0;
        s_hhi[h] = 0;
    }
    unsigned bar_target = 0;  // running total of the arrivals the grid barriers wait for
    if (tid == 0) {
        RoundState &st = s_st;
        st.round = ctl->round;
        st.size = ctl->size;
        st.f = mk128(ctl->f_lo, ctl->f_hi);
        st.live_len = ctl->live_len;
        st.live_sel = ctl->live_sel;
        st.minw = ctl->minw;
        st.best_round = ctl->best_round;
        st.best_size = ctl->best_size;
        st.bf = mk128(ctl->bf_lo, ctl->bf_hi);
        st.gpo_le = ctl->gpo_le;
        st.gpo_lt = ctl->gpo_lt;
        st.gm_f = 0;
        st.gm_s = 0;
        st.n_min_rule = ctl->n_min_rule;
        st.scan = ctl->scan_volume;
        s_elive = ctl->elive;
        s_rd.U_sel = kMaxLL;  // no round yet
        s_rd.arcs = kMaxLL;
    }
    __syncthreads();
    if (ctl->status != ST_RUNNING || ctl->error) return;

    for (;;) {
        const long long size = s_st.size;
        // a tail (one CTA or a cluster) takes over once S fits it and either
        // its arcs are few or the rounds have become small (a round of few
        // vertices or arcs costs a tail microseconds and the grid-wide kernel
        // its barriers)
        const bool small_round = s_rd.U_sel <= DUPIN_TAIL_SMALL_ROUND || s_rd.arcs <= DUPIN_TAIL_SMALL_ARCS;
        if (size == 0 || (size <= A.hcap && (2 * s_elive <= A.tail_arcs || (small_round && 2 * s_elive <= A.tarc_cap))))
            break;
        if (s_st.round >= A.max_rounds) {
            if (b == 0 && tid == 0) set_error(ctl, DUPIN_ERR_NO_PROGRESS);
            break;
        }
        const long long i = s_st.round + 1;
        long long T;
        {
            const u128 f = s_st.f;
            const u128 f1 = f - 1;
            if (A.lpo && s_st.round > 0 && f != 0 &&
                mul_le(s_st.minw, (unsigned long long)size, (unsigned long long)(f1 >> 64), (unsigned long long)f1)) {
                // Algorithm 4's trim round: some live w < g(S) (the exact minimum
                // live weight says so); it removes w < max(tau_max, g(S))
                const long long bg = floor_div_sat(f1, (unsigned long long)size);
                T = bg > s_st.gpo_lt ? bg : s_st.gpo_lt;
            } else {
                T = floor_ratio((unsigned long long)A.kD, f, (unsigned long long)A.D, size);
                if (A.gpo) {
                    const long long le = floor_ratio((unsigned long long)A.D, f, (unsigned long long)A.kD, size);
                    const long long gl = le > s_st.gpo_le ? le : s_st.gpo_le;
                    long long gt = s_st.gpo_lt;
                    if (A.lpo) {
                        const long long lt = below_ratio((unsigned long long)A.D, f, (unsigned long long)A.kD, size);
                        gt = lt > gt ? lt : gt;
                    }
                    T = gl > T ? gl : T;
                    __syncthreads();  // every thread has read s_st.gpo_le / gpo_lt
                    if (tid == 0) {
                        s_st.gpo_le = gl;
                        s_st.gpo_lt = gt;
                    }
                }
            }
        }
        const int live_sel = s_st.live_sel;
        int *live = live_sel ? A.live1 : A.live0;
        int *nlive = live_sel ? A.live0 : A.live1;
        const long long L = s_st.live_len;
        const long long j0 = split_at(L, b, G), j1 = split_at(L, b + 1, G);
        // Phase A selects w <= T.  When k(1+eps) < 2 the threshold can select
        // nobody, and the round then takes the minimum rule (U_i = the live
        // vertices of minimum weight).  So that this needs no second pass, a
        // block that selected nothing also stages its own minimum-weight
        // vertices as candidates; after the barrier, if no block selected
        // anything, the blocks whose minimum is the global one commit theirs.
        const long long thr = T;
        bool minrule = false;
        long long U_sel = 0, U_stage = 0, totArcs = 0, slotBase = 0, arcBase = 0, survBase = 0;
        // ---------------- phase A: select
        if (tid == 0) s_nst = 0;
        __syncthreads();
        {
            long long cnt = 0, surv = 0, minsurv = kMaxLL, sdeg = 0;
            unsigned long long wlo = 0, whi = 0;
            for (long long jb = j0 + wid * 32; jb < j1; jb += BULK_THREADS) {
                const long long j = jb + lane;
                int id = j < j1 ? live[j] : -1;
                long long wv = 0;
                if (id >= 0) wv = A.w[id];
                const bool sel = id >= 0 && wv <= thr;
                if (id >= 0 && !sel) {
                    surv++;
                    minsurv = wv < minsurv ? wv : minsurv;
                }
                long long start = 0, deg = 0;
                if (sel) {
                    cnt++;
                    add128(wlo, whi, (unsigned long long)wv, 0);
                    A.pr[id] = (int)i;
                    live[j] = -1;
                    start = g.rp[id];
                    deg = g.rp[id + 1] - start;
                    sdeg += deg;
                }
                stage_entry(A, j0, sel && deg > 0, start, deg, &s_nst);
            }
            BlockRed<BULK_WARPS, 6> r;
            r.v[0] = cnt; r.v[1] = surv; r.v[2] = sdeg; r.v[3] = 0; r.v[4] = 0; r.v[5] = 0;
            r.lo = wlo; r.hi = whi; r.mn = minsurv;
            block_reduce<BULK_WARPS, 6>(r, s_v, s_lo, s_hi, s_mn);
            BlockPart &p = A.part[b];
            if (tid == 0) {
                p.sel_cnt = r.v[0];
                p.surv_cnt = r.v[1];
                p.ws_lo = r.lo;
                p.ws_hi = r.hi;
                p.min_surv = r.mn;
                p.stage_cnt = (long long)s_nst;
                p.sel_deg = r.v[2];
            }
            const long long m = r.mn;
            if (A.use_min && r.v[0] == 0 && m != kMaxLL) {
                // minimum-rule candidates: the live vertices of weight m (their
                // list positions in stage_id, the ones with arcs staged as usual)
                __syncthreads();  // thread 0 has read s_nst
                if (tid == 0) {
                    s_nst = 0;
                    s_surv = 0;
                }
                __syncthreads();
                long long cdeg = 0, min2 = kMaxLL;  // min2: the smallest live weight above m
                for (long long jb = j0 + wid * 32; jb < j1; jb += BULK_THREADS) {
                    const long long j = jb + lane;
                    const int id = j < j1 ? live[j] : -1;
                    const long long wv = id >= 0 ? A.w[id] : kMaxLL;
                    const bool c = id >= 0 && wv == m;
                    if (id >= 0 && wv > m && wv < min2) min2 = wv;
                    const unsigned cb = __ballot_sync(0xffffffffu, c);
                    long long start = 0, deg = 0;
                    if (cb) {
                        unsigned base = 0;
                        if (lane == 0) base = atomicAdd(&s_surv, (unsigned)__popc(cb));
                        base = __shfl_sync(0xffffffffu, base, 0);
                        if (c) {
                            A.stage_id[j0 + (long long)base + __popc(cb & ((1u << lane) - 1u))] = (int)j;
                            start = g.rp[id];
                            deg = g.rp[id + 1] - start;
                            cdeg += deg;
                        }
                    }
                    stage_entry(A, j0, c && deg > 0, start, deg, &s_nst);
                }
                BlockRed<BULK_WARPS, 6> rc;
                for (int q = 0; q < 6; q++) rc.v[q] = 0;
                rc.v[0] = cdeg;
                rc.lo = 0; rc.hi = 0; rc.mn = min2;
                block_reduce<BULK_WARPS, 6>(rc, s_v, s_lo, s_hi, s_mn);
                if (tid == 0) {
                    p.mc_cnt = (long long)s_surv;
                    p.mc_stage = (long long)s_nst;
                    p.mc_deg = rc.v[0];
                    p.min_surv2 = rc.mn;
                }
            } else if (tid == 0) {
                p.mc_cnt = 0;
                p.mc_stage = 0;
                p.mc_deg = 0;
                p.min_surv2 = kMaxLL;
            }
        }
        if (!grid_barrier(ctl, G, bar_target)) return;
        // ---------------- phase B (part 1): totals and this block's offsets
        long long myStage, myDeg, myCand = 0;
        {
            BlockRed<BULK_WARPS, 6> r;
            for (int j = 0; j < 6; j++) r.v[j] = 0;
            r.lo = 0; r.hi = 0; r.mn = kMaxLL;
            // v: 0 sel_cnt, 1 stage_cnt, 2 sel_deg, 3 survivors before b,
            //    4 stage entries before b, 5 arcs before b
            for (int t = tid; t < (int)G; t += BULK_THREADS) {
                const BlockPart &p = A.part[t];
                r.v[0] += p.sel_cnt;
                r.v[1] += p.stage_cnt;
                r.v[2] += p.sel_deg;
                if (t < b) {
                    r.v[3] += p.surv_cnt;
                    r.v[4] += p.stage_cnt;
                    r.v[5] += p.sel_deg;
                }
                add128(r.lo, r.hi, p.ws_lo, p.ws_hi);
                r.mn = p.min_surv < r.mn ? p.min_surv : r.mn;
            }
            block_reduce<BULK_WARPS, 6>(r, s_v, s_lo, s_hi, s_mn);
            U_sel = r.v[0]; U_stage = r.v[1]; totArcs = r.v[2];
            survBase = r.v[3]; slotBase = r.v[4]; arcBase = r.v[5];
            if (tid == 0) {
                s_rd.wlo = r.lo;
                s_rd.whi = r.hi;
                s_rd.minsurv = r.mn;  // the survivors' minimum (before this round's decrements)
            }
            myStage = A.part[b].stage_cnt;
            myDeg = A.part[b].sel_deg;
            const long long minAll = r.mn;
            if (U_sel == 0 && A.use_min && minAll != kMaxLL) {
                // minimum rule: U_i = the candidates of the blocks whose
                // minimum is the global minimum
                minrule = true;
                for (int j = 0; j < 6; j++) r.v[j] = 0;
                r.lo = 0; r.hi = 0; r.mn = kMaxLL;
                for (int t = tid; t < (int)G; t += BULK_THREADS) {
                    const BlockPart &p = A.part[t];
                    const bool q = p.min_surv == minAll;
                    const long long ms = q ? p.min_surv2 : p.min_surv;  // survivors of the minimum rule
                    r.mn = ms < r.mn ? ms : r.mn;
                    if (q) {
                        r.v[0] += p.mc_cnt;
                        r.v[1] += p.mc_stage;
                        r.v[2] += p.mc_deg;
                    }
                    if (t < b) {
                        r.v[3] += p.surv_cnt - (q ? p.mc_cnt : 0);
                        if (q) {
                            r.v[4] += p.mc_stage;
                            r.v[5] += p.mc_deg;
                        }
                    }
                }
                block_reduce<BULK_WARPS, 6>(r, s_v, s_lo, s_hi, s_mn);
                U_sel = r.v[0]; U_stage = r.v[1]; totArcs = r.v[2];
                survBase = r.v[3]; slotBase = r.v[4]; arcBase = r.v[5];
                const BlockPart &pb = A.part[b];
                const bool mine = pb.min_surv == minAll;
                myStage = mine ? pb.mc_stage : 0;
                myDeg = mine ? pb.mc_deg : 0;
                myCand = mine ? pb.mc_cnt : 0;
                if (tid == 0) {
                    const u128 ws = (u128)(unsigned long long)U_sel * (unsigned long long)minAll;
                    s_rd.wlo = (unsigned long long)ws;
                    s_rd.whi = (unsigned long long)(ws >> 64);
                    s_rd.minsurv = r.mn;
                }
            }
        }
        if (U_sel == 0) {  // cannot happen (Lemma 4.2 / minimum rule): stop rather than spin
            if (b == 0 && tid == 0) set_error(ctl, DUPIN_ERR_NO_PROGRESS);
            return;
        }
        if (myCand > 0) {  // commit this block's minimum-rule candidates
            for (long long c = tid; c < myCand; c += BULK_THREADS) {
                const long long j = A.stage_id[j0 + c];
                A.pr[live[j]] = (int)i;
                live[j] = -1;
            }
            __syncthreads();
        }
        const long long newSize = size - U_sel;
        const bool compact = newSize > 0 && (2 * newSize <= L || newSize <= A.hcap);
        if (tid == 0) {
            s_rd.U_sel = U_sel;
            s_rd.arcs = totArcs;
            s_rd.newSize = newSize;
            s_rd.minrule = minrule ? 1 : 0;
            s_rd.compact = compact ? 1 : 0;
        }
        // Consumer block c expands the arcs [split_at(totArcs, c, G), split_at(totArcs, c + 1, G))
        // and starts its walk at the frontier entry holding its first arc.  The
        // consumers whose first arc lies in this block's entries, global arcs
        // [arcBase, arcBase + myDeg), are c_lo .. c_lo + nc - 1; their first
        // arcs go to shared memory (s_base is free until phase C), and every
        // entry finds its consumers there by binary search.
        long long *s_cs = s_base;
        long long c_lo = 0, nc = 0;
        if (myDeg > 0) {
            const unsigned long long T = (unsigned long long)totArcs;
            c_lo = (long long)(((unsigned long long)arcBase * G + T - 1) / T);
            long long c_hi = (long long)(((unsigned long long)(arcBase + myDeg) * G + T - 1) / T);
            if (c_hi > (long long)G) c_hi = G;
            nc = c_hi - c_lo;
        }
        for (long long t = tid; t < nc; t += BULK_THREADS) s_cs[t] = split_at(totArcs, c_lo + t, G);
        __syncthreads();
        // the staged entries' arc offsets: a block scan of their degrees
        long long carry = 0;
        for (long long q0 = 0; q0 < myStage; q0 += BULK_THREADS) {
            const long long q = q0 + tid;
            const long long deg = q < myStage ? A.stage_off[j0 + q] : 0;
            long long chunk;
            const long long off = carry + block_excl_scan<BULK_WARPS>(deg, s_scan, chunk);
            carry += chunk;
            if (q < myStage) {
                const long long gs = slotBase + q;
                const long long goff = arcBase + off;
                const long long gend = goff + deg;
                A.fstart[gs] = A.stage_start[j0 + q];
                A.fbase[gs] = goff;
                int lo = 0, hi = (int)nc;  // first consumer whose first arc is >= goff
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (s_cs[mid] < goff) lo = mid + 1;
                    else hi = mid;
                }
                for (int t = lo; t < (int)nc && s_cs[t] < gend; t++) A.cstart[c_lo + t] = gs;
            }
        }
        if (b == 0 && tid == 0) A.fbase[U_stage] = totArcs;
        if (compact) {
            if (tid == 0) s_surv = 0;
            __syncthreads();
            for (long long jb = j0 + wid * 32; jb < j1; jb += BULK_THREADS) {
                const long long j = jb + lane;
                int id = j < j1 ? live[j] : -1;
                const bool keep = id >= 0;
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                if (bal) {
                    unsigned base = 0;
                    if (lane == 0) base = atomicAdd(&s_surv, (unsigned)__popc(bal));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (keep) nlive[survBase + (long long)base + __popc(bal & ((1u << lane) - 1u))] = id;
                }
            }
        }
        if (!grid_barrier(ctl, G, bar_target)) return;

        // ---------------- phase C: expand
        // The block walks an equal share [E0, E1) of the round's arcs through
        // windows of WALK_WIN frontier entries in shared memory; each thread
        // takes BULK_ILP arcs at a time and issues their loads together.
        unsigned long long ilo = 0, ihi = 0;
        long long nrem = 0;  // 2 per arc from U to S \ U, 1 per arc inside U
        long long mindec = kMaxLL;  // with Algorithm 4: the smallest weight after a decrement
        if (totArcs > 0) {
            const long long E0 = split_at(totArcs, b, G);
            const long long E1 = split_at(totArcs, b + 1, G);
            const long long *fb = A.fbase;
            const long long *fs = A.fstart;
            const int *col = g.col;
            const long long *cw = g.cw;
            int *pr = A.pr;
            long long *w = A.w;
            long long e = E0, kk = E0 < E1 ? A.cstart[b] : 0;
            while (e < E1) {  // block-uniform
                __syncthreads();
                for (int t = tid; t <= WALK_WIN; t += BULK_THREADS) {
                    const long long idx = kk + t;
                    s_base[t] = idx <= U_stage ? fb[idx] : kMaxLL;
                    s_start[t] = idx < U_stage ? fs[idx] : 0;
                }
                __syncthreads();
                const long long wend = s_base[WALK_WIN];
                const long long hi = E1 < wend ? E1 : wend;
                for (long long xb = e + tid; xb < hi; xb += (long long)BULK_ILP * BULK_THREADS) {
                    long long pos[BULK_ILP];
#pragma unroll
                    for (int u = 0; u < BULK_ILP; u++) {
                        const long long x = xb + (long long)u * BULK_THREADS;
                        const int t = smem_last_le_fixed(s_base, x);
                        pos[u] = x < hi ? s_start[t] + (x - s_base[t]) : -1;
                    }
                    int cv[BULK_ILP];
                    long long cc[BULK_ILP];
#pragma unroll
                    for (int u = 0; u < BULK_ILP; u++) {
                        if (pos[u] >= 0) {
                            cv[u] = col[pos[u]];
                            cc[u] = dg ? DUPIN_Q_ONE : cw[pos[u]];
                        }
                    }
                    int pp[BULK_ILP];
#pragma unroll
                    for (int u = 0; u < BULK_ILP; u++)
                        if (pos[u] >= 0) pp[u] = pr[cv[u] >= 0 ? cv[u] : s_hub[-cv[u] - 1]];
#pragma unroll
                    for (int u = 0; u < BULK_ILP; u++) {
                        if (pos[u] < 0) continue;
                        const int p = pp[u];
                        const long long c = cc[u];
                        if (p > (int)i) {
                            const int cvu = cv[u];
                            if (cvu >= 0) {
                                if (A.lpo) {
                                    const long long nv =
                                        (long long)atomicAdd((unsigned long long *)&w[cvu], (unsigned long long)(-c)) - c;
                                    mindec = nv < mindec ? nv : mindec;
                                } else {
                                    // result unused: a fire-and-forget reduction
                                    atomicAdd((unsigned long long *)&w[cvu], (unsigned long long)(-c));
                                }
                            } else {  // hub head: aggregate in shared memory
                                const int h = -cvu - 1;
                                const unsigned cl = (unsigned)c;
                                const unsigned old = atomicAdd(&s_hlo[h], cl);
                                const unsigned ch =
                                    (unsigned)((unsigned long long)c >> 32) + (old + cl < old ? 1u : 0u);
                                if (ch) atomicAdd(&s_hhi[h], ch);
                            }
                            nrem += 2;
                        } else if (p == (int)i) {
                            add128(ilo, ihi, (unsigned long long)c, 0);
                            nrem++;
                        }
                    }
                }
                kk += smem_last_le(s_base, WALK_WIN + 1, hi);
                e = hi;
            }
        }
        if (nh > 0) {  // one reduction per hub touched by this block
            __syncthreads();
            for (int h = tid; h < nh; h += BULK_THREADS) {
                const unsigned long long a = ((unsigned long long)s_hhi[h] << 32) + s_hlo[h];
                if (a) {
                    const long long nv =
                        (long long)(atomicAdd((unsigned long long *)&A.w[s_hub[h]], (unsigned long long)0 - a) - a);
                    mindec = nv < mindec ? nv : mindec;
                    s_hlo[h] = 0;
                    s_hhi[h] = 0;
                }
            }
        }
        {
            BlockRed<BULK_WARPS, 6> r;
            for (int j = 0; j < 6; j++) r.v[j] = 0;
            r.v[0] = nrem;
            r.lo = ilo; r.hi = ihi; r.mn = mindec;
            block_reduce<BULK_WARPS, 6>(r, s_v, s_lo, s_hi, s_mn);
            if (tid == 0) {
                A.part[b].in_lo = r.lo;
                A.part[b].in_hi = r.hi;
                A.part[b].min_dec = r.mn;
                A.part[b].rem_cnt = r.v[0];
            }
        }
        if (!grid_barrier(ctl, G, bar_target)) return;

        // ---------------- phase D: close the round (every block)
        {
            BlockRed<BULK_WARPS, 6> r;
            for (int j = 0; j < 6; j++) r.v[j] = 0;
            r.lo = 0; r.hi = 0; r.mn = kMaxLL;
            for (int t = tid; t < (int)G; t += BULK_THREADS) {
                add128(r.lo, r.hi, A.part[t].in_lo, A.part[t].in_hi);
                r.mn = A.part[t].min_dec < r.mn ? A.part[t].min_dec : r.mn;
                r.v[0] += A.part[t].rem_cnt;
            }
            block_reduce<BULK_WARPS, 6>(r, s_v, s_lo, s_hi, s_mn);
            if (tid == 0) {
                RoundState &st = s_st;
                // an edge leaves E(S) with its first removed end: counted 2 on
                // its one arc from U to S \ U, 1 on each of its two arcs inside U
                s_elive -= r.v[0] / 2;
                // exact minimum live weight (Algorithm 4 needs it): a survivor's
                // last decrement result is its final weight
                if (A.lpo) st.minw = s_rd.minsurv < r.mn ? s_rd.minsurv : r.mn;
                const u128 internal = mk128(r.lo, r.hi);
                const u128 wsel = mk128(s_rd.wlo, s_rd.whi);
                st.f = st.f - (wsel - (internal >> 1));
                st.scan += L;
                st.size = s_rd.newSize;
                st.round = i;
                st.n_min_rule += s_rd.minrule;
                if (s_rd.compact) {
                    st.live_sel ^= 1;
                    st.live_len = s_rd.newSize;
                }
                if (st.size > 0 && frac_gt(st.f, st.size, st.bf, st.best_size)) {
                    st.bf = st.f;
                    st.best_size = st.size;
                    st.best_round = i;
                }
                if (b == 0 && i < A.tr_cap) {
                    A.tr_f_hi[i] = (long long)(unsigned long long)(st.f >> 64);
                    A.tr_f_lo[i] = (unsigned long long)st.f;
                    A.tr_size[i] = st.size;
                    A.tr_peeled[i] = s_rd.U_sel;
                }
            }
            __syncthreads();
        }
    }
    if (b == 0 && tid == 0) {
        const RoundState &st = s_st;
        ctl->round = st.round;
        ctl->size = st.size;
        ctl->f_lo = (unsigned long long)st.f;
        ctl->f_hi = (unsigned long long)(st.f >> 64);
        ctl->live_len = st.live_len;
        ctl->live_sel = st.live_sel;
        ctl->minw = st.minw;
        ctl->best_round = st.best_round;
        ctl->best_size = st.best_size;
        ctl->bf_lo = (unsigned long long)st.bf;
        ctl->bf_hi = (unsigned long long)(st.bf >> 64);
        ctl->gpo_le = st.gpo_le;
        ctl->gpo_lt = st.gpo_lt;
        ctl->n_min_rule = st.n_min_rule;
        ctl->scan_volume = st.scan;
        ctl->bulk_rounds = st.round;
        ctl->elive = s_elive;
        if (ctl->error == 0)
            ctl->status = st.size == 0 ? ST_DONE
                          : (st.size <= A.tail_cap && 2 * s_elive <= A.one_arcs ? ST_TAIL : ST_CLUSTER);
    }
}

// Beside a cluster tail (a batched call's earlier peel) the rounds run on a
// quarter of the launched blocks and the rest leave at once: the cluster's
// rounds are bound by the latency of their loads, which a full-width stage's
// memory traffic raises.  The flag is set before the launch, so every block
// reads the same value.
__global__ void __launch_bounds__(BULK_THREADS, 1) k_peel_bulk(PeelArgs A) {
    unsigned G = gridDim.x;
    if (A.ctl->beside_cluster) G = G / 4 > 0 ? G / 4 : 1;
    if (blockIdx.x >= G) return;
    peel_bulk_body(A, blockIdx.x, G);
}

// a later peel of a batched call learns whether this one's tail is a cluster
// (read right after this peel's grid-wide rounds, before its tail starts)
__global__ void k_note_cluster(const PeelCtl *prev, PeelCtl *next) {
    if (prev->status == ST_CLUSTER) next->beside_cluster = 1;
}

void enqueue_note_cluster(const PeelWorkspace *prev, PeelWorkspace *next, cudaStream_t s) {
    k_note_cluster<<<1, 1, 0, s>>>(prev->ctl, next->ctl);
}

// ------------------------------------------------------- (d) tail sub-graph

// local ids and full degrees of the live vertices
__global__ void k_tail_prep(PeelArgs A) {
    const PeelCtl *c = A.ctl;
    if ((c->status != ST_TAIL && c->status != ST_CLUSTER) || c->error) return;
    const long long L = c->live_len;
    const int *live = c->live_sel ? A.live1 : A.live0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < L; p += (long long)gridDim.x * blockDim.x) {
        int gid = live[p];
        A.loc[gid] = (int)p;
        A.tdeg[p] = A.g.rp[gid + 1] - A.g.rp[gid];
    }
}

// exclusive prefix of x[0..L) in place, x[L] = total (one block)
__global__ void __launch_bounds__(SCAN_THREADS) k_tail_scan(PeelArgs A, long long *x, const int *cnt) {
    __shared__ long long s_w[SCAN_THREADS / 32];
    const PeelCtl *c = A.ctl;
    if ((c->status != ST_TAIL && c->status != ST_CLUSTER) || c->error) return;
    const long long L = c->live_len;
    long long carry = 0;
    for (long long b0 = 0; b0 < L; b0 += SCAN_THREADS) {
        long long p = b0 + threadIdx.x;
        long long v = p < L ? (cnt ? (long long)cnt[p] : x[p]) : 0;
        long long tot;
        long long ex = block_excl_scan<SCAN_THREADS / 32>(v, s_w, tot);
        if (p < L) x[p] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        x[L] = carry;
        if (cnt) {
            A.ctl->tail_arcs = carry;
            if (carry > A.tarc_cap) set_error(A.ctl, DUPIN_ERR_OOM);
        }
    }
}

// pass 0: count live neighbours per live vertex; pass 1: fill local arcs
template <int PASS>
__global__ void __launch_bounds__(BULK_THREADS) k_tail_arcs(PeelArgs A) {
    __shared__ long long s_base[WALK_WIN + 1];
    __shared__ long long s_start[WALK_WIN + 1];
    __shared__ long long s_k0;
    const PeelCtl *c = A.ctl;
    if ((c->status != ST_TAIL && c->status != ST_CLUSTER) || c->error) return;
    const long long L = c->live_len;
    const int *live = c->live_sel ? A.live1 : A.live0;
    const long long tot = A.tdeg[L];
    const unsigned G = gridDim.x;
    const long long e0 = split_at(tot, blockIdx.x, G);
    const long long e1 = split_at(tot, blockIdx.x + 1, G);
    if (e0 >= e1) return;
    const long long *tdeg = A.tdeg;
    const long long *rp = A.g.rp;
    if (threadIdx.x < 32) {
        long long k = warp_search_last_le(tdeg, L, e0);
        if (threadIdx.x == 0) s_k0 = k;
    }
    __syncthreads();
    const long long k0 = s_k0;
    const int *col = A.g.col;
    const int *hubs = A.g.hubs;
    const long long *cw = A.g.cw;
    const int *pr = A.pr;
    const bool grp = c->status == ST_CLUSTER && A.tgrp != nullptr && A.cl_c > 0;
    walk_arcs([=](long long k) { return tdeg[k]; },
              [=](long long k) { return rp[live[k]]; }, L, e0, e1, k0, s_base, s_start,
              [&](long long k, long long pos) {
                  const int v = arc_head(col[pos], hubs);
                  if (pr[v] != DUPIN_LIVE) return;
                  if (PASS == 0) {  // per row (per row and owner for the cluster; k_tail_rowcnt adds them up)
                      if (grp) atomicAdd(&A.tgrp[k * DUPIN_GRP_STRIDE + 1 + (A.loc[v] & (A.cl_c - 1))], 1u);
                      else atomicAdd(&A.tcnt[k], 1);
                  } else {
                      const long long slot =
                          grp ? (long long)atomicAdd(&A.tgrp[k * DUPIN_GRP_STRIDE + 1 + (A.loc[v] & (A.cl_c - 1))], 1u)
                              : A.tlrp[k] + atomicAdd(&A.tfill[k], 1);
                      A.tcol[slot] = A.loc[v];
                      if (A.tcw) A.tcw[slot] = cw ? cw[pos] : DUPIN_Q_ONE;
                  }
              });
}

// For the cluster tail: each row's live-arc count, from its owner groups' counts
__global__ void k_tail_rowcnt(PeelArgs A) {
    const PeelCtl *c = A.ctl;
    if (c->status != ST_CLUSTER || c->error || A.tgrp == nullptr || A.cl_c <= 0) return;
    const long long L = c->live_len;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < L; k += (long long)gridDim.x * blockDim.x) {
        const unsigned *g = A.tgrp + k * DUPIN_GRP_STRIDE + 1;
        unsigned t = 0;
        for (int o = 0; o < A.cl_c; o++) t += g[o];
        A.tcnt[k] = (int)t;
    }
}

// For the cluster tail: each row's owner-group counts become the groups' first
// arcs (the fill pointers of pass 1, which leaves each group's end there).
__global__ void k_tail_grp(PeelArgs A) {
    const PeelCtl *c = A.ctl;
    if (c->status != ST_CLUSTER || c->error || A.tgrp == nullptr || A.cl_c <= 0) return;
    const long long L = c->live_len;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < L; k += (long long)gridDim.x * blockDim.x) {
        unsigned *g = A.tgrp + k * DUPIN_GRP_STRIDE;
        unsigned run = (unsigned)A.tlrp[k];
        g[0] = run;
        for (int o = 0; o < A.cl_c; o++) {
            const unsigned cnt = g[1 + o];
            g[1 + o] = run;
            run += cnt;
        }
    }
}

// One CTA finishes the peel on the live sub-graph held in shared memory.
// tw[p] is the peeling weight of local vertex p while it is live (>= 0) and
// -i once it left in round i.  The live vertices are grouped in segments of
// 64 with an exact minimum per segment, kept in two buffers by round parity:
// round i reads its thresholds from one buffer and writes the new minima to
// the other (recomputed for segments that lose vertices, lowered by
// atomicMin on every decrement).  A round scans only segments that can hold
// selected vertices, expands the frontier's arcs (from L2) with shared-memory
// atomics, and then every warp closes the round and plans the next one
// itself from the same shared data: two block barriers per round.
// NARROW: f < 2^62 and the best f < 2^64 when the tail starts, so every sum
// a round forms (at most 2f) fits 64 bits; the sums then take 64-bit adds
// and 32-bit warp reductions, the products 64 x 64 -> 128-bit multiplies.
template <bool NARROW>
__device__ __forceinline__ void peel_tail_body(const PeelArgs &A, unsigned char *smem, TailAcc<TAIL_WARPS> *s_acc,
                                               long long *s_w, long long *s_pref) {
    PeelCtl *ctl = A.ctl;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const long long L = ctl->live_len;
    const int nseg = (int)((L + TAIL_SEG - 1) / TAIL_SEG);
    const long long LP = (long long)nseg * TAIL_SEG;
    long long *tw = (long long *)smem;                                  // [LP]
    long long *segbuf = (long long *)(smem + 8 * LP);                   // [2 nseg]
    int *toff = (int *)(smem + 8 * LP + 16 * nseg);                     // [L+1]
    unsigned short *tf = (unsigned short *)(smem + 8 * LP + 16 * nseg + 4 * (L + 1));  // [L]
    const int *live = ctl->live_sel ? A.live1 : A.live0;
    const bool dg = A.tcw == nullptr;
    const int *tcol = A.tcol;
    const long long *tcw = A.tcw;

    RoundState st;  // identical in every thread
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
    for (long long p = tid; p <= L; p += TAIL_THREADS) toff[p] = (int)A.tlrp[p];
    for (long long p = tid; p < LP; p += TAIL_THREADS) tw[p] = p < L ? A.w[live[p]] : -1;  // pads: gone
    if (tid < 2) s_acc[tid].F = 0;
    __syncthreads();
    // round i reads the minima in buffer (i & 1): fill the first round's buffer
    long long *first = segbuf + ((st.round + 1) & 1) * nseg;
    for (int q = wid; q < nseg; q += TAIL_WARPS) {
        const longlong2 v = *(const longlong2 *)&tw[(long long)q * TAIL_SEG + 2 * lane];
        long long m = kMaxLL;
        if (v.x >= 0) m = v.x;
        if (v.y >= 0 && v.y < m) m = v.y;
        m = warp_min64(m);
        if (lane == 0) first[q] = m;
    }
    __syncthreads();
    TailRound R = tail_plan<NARROW>(A.kD, A.D, A.use_min, A.gpo, A.lpo, st, seg_global_min(first, nseg));
    int err = 0;
    while (!R.done) {
        if (R.i > A.max_rounds) {
            err = DUPIN_ERR_NO_PROGRESS;
            break;
        }
        const long long i = R.i;
        const long long *cur = segbuf + (i & 1) * nseg;  // minima at the start of round i
        long long *nxt = segbuf + ((i + 1) & 1) * nseg;  // minima after round i
        TailAcc<TAIL_WARPS> &acc = s_acc[i & 1];
        // ---- select: lanes test segments in parallel; a candidate segment
        // is then scanned by its warp (two vertices per lane)
        unsigned long long wlo = 0, whi = 0;
        long long mins = kMaxLL;  // new minimum over the segments this lane looked at
        for (int q0 = wid * 32; q0 < nseg; q0 += TAIL_THREADS) {
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
                const longlong2 v = *(const longlong2 *)&tw[p];
                bool s0, s1;
                if (R.minrule) {
                    s0 = v.x >= 0 && v.x <= R.minw;
                    s1 = v.y >= 0 && v.y <= R.minw;
                } else {
                    s0 = v.x >= 0 && (v.x <= R.gle || mul_le(v.x, R.Y, R.Xhi, R.Xlo));
                    s1 = v.y >= 0 && (v.y <= R.gle || mul_le(v.y, R.Y, R.Xhi, R.Xlo));
                }
                long long m = kMaxLL;  // the segment's minimum over its survivors
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
                    if (lane == 0) base = atomicAdd(&acc.F, (unsigned)(__popc(b0) + __popc(b1)));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    const unsigned lt = (1u << lane) - 1u;
                    unsigned slot = base + __popc(b0 & lt) + __popc(b1 & lt);
                    if (s0) {
                        tw[p] = -i;
                        if (NARROW) wlo += (unsigned long long)v.x;
                        else add128(wlo, whi, (unsigned long long)v.x, 0);
                        tf[slot++] = (unsigned short)p;
                    }
                    if (s1) {
                        tw[p + 1] = -i;
                        if (NARROW) wlo += (unsigned long long)v.y;
                        else add128(wlo, whi, (unsigned long long)v.y, 0);
                        tf[slot] = (unsigned short)(p + 1);
                    }
                }
            }
        }
        // the select's sums and minimum stay in registers: they are reduced
        // with the expand's after it, off the path to the first barrier
        __syncthreads();
        // round i+1's counter was last read in round i-1: reset it now
        if (tid == 0) s_acc[(i + 1) & 1].F = 0;
        const int F = (int)acc.F;
        // ---- expand
        unsigned long long ilo = 0, ihi = 0;
        long long mind = kMaxLL;
        auto apply = [&](int v, long long c) {
            const long long wv = tw[v];
            if (wv >= 0) {
                const long long old = (long long)atomicAdd((unsigned long long *)&tw[v], (unsigned long long)(-c));
                atomicMin(&nxt[v / TAIL_SEG], old - c);
                mind = old - c < mind ? old - c : mind;
            } else if (wv == -i) {
                if (NARROW) ilo += (unsigned long long)c;
                else add128(ilo, ihi, (unsigned long long)c, 0);
            }
        };
        // TAIL_ILP arcs per thread at a time: their loads from L2 are issued
        // together before any of them is applied
        auto arcs = [&](const long long (&pos)[TAIL_ILP]) {
            int cv[TAIL_ILP];
            long long cc[TAIL_ILP];
#pragma unroll
            for (int u = 0; u < TAIL_ILP; u++) {
                if (pos[u] >= 0) {
                    cv[u] = tcol[pos[u]];
                    cc[u] = dg ? DUPIN_Q_ONE : tcw[pos[u]];
                }
            }
#pragma unroll
            for (int u = 0; u < TAIL_ILP; u++)
                if (pos[u] >= 0) apply(cv[u], cc[u]);
        };
        if (F <= TAIL_FAST) {
            // the frontier's arcs in chunks of 32 consecutive arcs of one
            // vertex: chunk c goes to warp c % TAIL_WARPS, TAIL_ILP of a warp's
            // chunks in flight at once; the walk is the same in every lane
            // (broadcast shared loads, no divergence)
            int e = 0, cbase = 0;
            int p0 = F > 0 ? tf[0] : 0;
            int a0 = F > 0 ? toff[p0] : 0, a1 = F > 0 ? toff[p0 + 1] : 0;
            int c = wid;
            while (e < F) {
                long long pos[TAIL_ILP];
                int got = 0;
#pragma unroll
                for (int u = 0; u < TAIL_ILP; u++) {
                    pos[u] = -1;
                    while (e < F && c >= cbase + ((a1 - a0 + 31) >> 5)) {
                        cbase += (a1 - a0 + 31) >> 5;
                        e++;
                        if (e < F) {
                            p0 = tf[e];
                            a0 = toff[p0];
                            a1 = toff[p0 + 1];
                        }
                    }
                    if (e < F) {
                        const int a = a0 + (c - cbase) * 32 + lane;
                        if (a < a1) pos[u] = a;
                        c += TAIL_WARPS;
                        got++;
                    }
                }
                if (got == 1) {  // one chunk: no predicated-off slots to issue
                    if (pos[0] >= 0) apply(tcol[pos[0]], dg ? DUPIN_Q_ONE : tcw[pos[0]]);
                } else {
                    arcs(pos);
                }
            }
        } else {
            for (int c0 = 0; c0 < F; c0 += TAIL_THREADS) {
                const int qq = c0 + tid;
                long long deg = 0;
                if (qq < F) {
                    const int p = tf[qq];
                    deg = toff[p + 1] - toff[p];
                }
                long long tot;
                long long ex = block_excl_scan<TAIL_WARPS>(deg, s_w, tot);
                s_pref[tid] = ex;
                const int nq = (F - c0) < TAIL_THREADS ? (F - c0) : TAIL_THREADS;
                if (tid == 0) s_pref[nq] = tot;
                __syncthreads();
                for (long long x0 = tid; x0 < tot; x0 += TAIL_ILP * TAIL_THREADS) {
                    long long pos[TAIL_ILP];
#pragma unroll
                    for (int u = 0; u < TAIL_ILP; u++) {
                        const long long x = x0 + (long long)u * TAIL_THREADS;
                        pos[u] = -1;
                        if (x < tot) {
                            const int e = smem_last_le(s_pref, nq, x);
                            const int p = tf[c0 + e];
                            pos[u] = toff[p] + (x - s_pref[e]);
                        }
                    }
                    arcs(pos);
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
        // ---- every warp: close round i and plan round i + 1 (same values everywhere)
        u128 wsel, internal;
        long long mins_all;
        tail_acc_sum<TAIL_WARPS, NARROW>(acc, wsel, internal, mins_all);
        st.f = st.f - (wsel - (internal >> 1));
        st.scan += L;
        st.size -= F;
        st.round = i;
        st.n_min_rule += R.minrule ? 1 : 0;
        // the best prefix and the trace are kept by the last warp alone: its
        // select covers the fewest segments (the tail has at most 234 of 64)
        if (wid == TAIL_WARPS - 1 && st.size > 0 && frac_gt<NARROW>(st.f, st.size, st.bf, st.best_size)) {
            st.bf = st.f;
            st.best_size = st.size;
            st.best_round = i;
        }
        if (tid == (TAIL_WARPS - 1) * 32 && i < A.tr_cap) {
            A.tr_f_hi[i] = (long long)(unsigned long long)(st.f >> 64);
            A.tr_f_lo[i] = (unsigned long long)st.f;
            A.tr_size[i] = st.size;
            A.tr_peeled[i] = F;
        }
        if (F == 0) {  // cannot happen (Lemma 4.2 / minimum rule); stop instead of spinning
            err = DUPIN_ERR_NO_PROGRESS;
            break;
        }
        R = tail_plan<NARROW>(A.kD, A.D, A.use_min, A.gpo, A.lpo, st, mins_all);
    }
    if (tid == (TAIL_WARPS - 1) * 32) {
        s_pref[0] = st.best_round;
        s_pref[1] = st.best_size;
        s_pref[2] = (long long)(unsigned long long)st.bf;
        s_pref[3] = (long long)(unsigned long long)(st.bf >> 64);
    }
    __syncthreads();
    for (long long p = tid; p < L; p += TAIL_THREADS) {
        const long long wv = tw[p];
        if (wv < 0) A.pr[live[p]] = (int)(-wv);
    }
    if (tid == 0) {
        st.best_round = s_pref[0];
        st.best_size = s_pref[1];
        st.bf = mk128((unsigned long long)s_pref[2], (unsigned long long)s_pref[3]);
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
        ctl->tail_ctas = 1;
        if (!err) ctl->status = ST_DONE;
    }
}

__global__ void __launch_bounds__(TAIL_THREADS, 1) k_peel_tail(PeelArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ TailAcc<TAIL_WARPS> s_acc[2];
    __shared__ long long s_w[TAIL_WARPS];
    __shared__ long long s_pref[TAIL_THREADS + 1];
    const PeelCtl *ctl = A.ctl;
    if (ctl->status != ST_TAIL || ctl->error) return;
    // f only decreases, and a round's sums (removed weights, arcs inside
    // the removed set) are at most 2f; the best f so far must fit 64 bits too
    if (ctl->f_hi == 0 && ctl->f_lo < (1ull << 62) && ctl->bf_hi == 0)
        peel_tail_body<true>(A, smem, s_acc, s_w, s_pref);
    else peel_tail_body<false>(A, smem, s_acc, s_w, s_pref);
}

// best_mask[u] = (peel_round[u] > best_round) for a best round known on the host
__global__ void k_mask_rounds(const int *pr, long long n, long long br, uint8_t *mask) {
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x)
        mask[u] = (long long)pr[u] > br ? 1 : 0;
}

void launch_mask(const int *pr, long long n, long long best_round, uint8_t *mask, cudaStream_t s) {
    const int grid = (int)std::min<long long>(1024, (n + 255) / 256);
    k_mask_rounds<<<grid > 0 ? grid : 1, 256, 0, s>>>(pr, n, best_round, mask);
}

// best_mask[u] = (peel_round[u] > best_round)
__global__ void k_finalize(const int *pr, long long n, const PeelCtl *ctl, uint8_t *mask) {
    const long long br = ctl->best_round;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x)
        mask[u] = (long long)pr[u] > br ? 1 : 0;
}

// ------------------------------------------------------------------- host

long long tail_cap_limit() {
    int dev = 0, smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // static shared memory of k_peel_tail is about 5 KB; 14 bytes per vertex
    // plus padding to whole 64-vertex segments and 16 bytes per segment
    long long avail = (long long)smem - 8 * 1024 - 8 * TAIL_SEG - 32;
    long long cap = avail / (14 + 1);
    if (cap > 65535) cap = 65535;
    return cap < 0 ? 0 : cap;
}

long long tail_cap_default() {
    long long lim = tail_cap_limit();
    return lim < 16384 ? lim : 16384;
}

int peel_grid_size() {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_peel_bulk, BULK_THREADS, 0);
    if (occ < 1) occ = 1;
    if (occ > 2) occ = 2;
    // the consumer starts of one round are staged in s_base (WALK_WIN + 1 entries)
    return std::min(sms * occ, WALK_WIN);
}

// raise k_peel_tail's dynamic shared-memory limit, once per device (the
// limit is a per-device attribute of the function)
static int set_tail_smem() {
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0, smem = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return dupin_fail(DUPIN_ERR_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return DUPIN_OK;
    cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_peel_tail);
    if (e != cudaSuccess) return dupin_cuda_fail(e, "cudaFuncGetAttributes(k_peel_tail)");
    int dyn = smem - (int)fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(k_peel_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return dupin_cuda_fail(e, "cudaFuncSetAttribute(k_peel_tail)");
    done[dev] = true;
    return DUPIN_OK;
}

static long long tail_smem_bytes(long long cap) {
    const long long nseg = (cap + TAIL_SEG - 1) / TAIL_SEG;
    return 8 * nseg * TAIL_SEG + 16 * nseg + 4 * (cap + 1) + 2 * cap + 16;
}

static int check_params(const dupin_graph *g, const dupin_params *p) {
    if (!p) return dupin_fail(DUPIN_ERR_INVALID_ARG, "params is NULL");
    if (p->metric < DUPIN_DG || p->metric > DUPIN_KCLIDS) return dupin_fail(DUPIN_ERR_INVALID_ARG, "unknown metric");
    if (p->metric == DUPIN_KCLIDS && (p->clique_q < 3 || p->clique_q > DUPIN_CLIQUE_MAX_Q))
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "DUPIN_KCLIDS needs clique_q in 3..DUPIN_CLIQUE_MAX_Q");
    if (p->k_mult < 1 || p->k_mult > 64) return dupin_fail(DUPIN_ERR_INVALID_ARG, "k_mult must be in 1..64");
    if (p->eps_den < 1 || p->eps_den > (1LL << 24) || p->eps_num < 0 || p->eps_num > (1LL << 30))
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "eps must be eps_num/eps_den with 0 <= eps_num <= 2^30, 1 <= eps_den <= 2^24");
    if (p->flags & ~(uint32_t)(DUPIN_GPO | DUPIN_LPO | DUPIN_RESULT_DEVICE | DUPIN_TIMING | DUPIN_TAIL_ONE_CTA |
                               DUPIN_TAIL_CLUSTER))
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "unknown flag");
    if ((p->flags & DUPIN_TAIL_ONE_CTA) && (p->flags & DUPIN_TAIL_CLUSTER))
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "DUPIN_TAIL_ONE_CTA and DUPIN_TAIL_CLUSTER exclude each other");
    if (p->metric != DUPIN_DG && !is_clique_metric(p->metric) && g->cw == nullptr)
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "DW/FD need edge weights; the graph was loaded without them");
    return DUPIN_OK;
}

DevGraph dev_graph(const dupin_graph *g, int metric) {
    DevGraph d;
    d.n = g->n;
    d.arcs = g->arcs;
    d.rp = g->rp;
    d.col = g->col;
    d.cw = metric == DUPIN_DG ? nullptr : g->cw;
    d.a = metric == DUPIN_DG ? nullptr : g->a;
    d.hubs = g->hubs;
    d.n_hubs = g->n_hubs;
    return d;
}

// Arcs the tail buffer holds: the live sub-graph has at most
// min(all arcs, |S| (|S| - 1)) arcs, and the grid-wide rounds go on while it
// has more than DUPIN_TAIL_BUF_ARCS.
static long long tail_arc_buffer(long long arcs, const PeelPlan &plan) {
    const long long tc = plan.hcap();
    return std::min<long long>(std::min<long long>(arcs, tc * (tc > 0 ? tc - 1 : 0)), DUPIN_TAIL_BUF_ARCS);
}

long long workspace_bytes(long long n, long long arcs, bool has_cw, const PeelPlan &plan, int grid) {
    const long long tail_cap = plan.hcap(), tr_cap = plan.tr_cap;
    const long long tarc = tail_arc_buffer(arcs, plan);
    long long b = 0;
    // w, pr, live0, live1, stage_id, stage_start, stage_off, fstart, loc, mask; fbase
    b += n * (8 + 4 + 4 + 4 + 4 + 8 + 8 + 8 + 4 + 1) + 8 * (n + 1);
    b += 8 * (grid + 1) + (long long)sizeof(BlockPart) * grid + (long long)sizeof(PeelCtl);
    b += 32 * tr_cap;
    b += (tail_cap + 1) * (8 + 8 + 4 + 4 + 4 * DUPIN_GRP_STRIDE);
    b += tarc * (4 + (has_cw ? 8 : 0));
    return b;
}

void workspace_free(PeelWorkspace *ws, cudaStream_t s) {
    if (!ws) return;
    void *ptrs[] = {ws->w, ws->pr, ws->live0, ws->live1, ws->stage_id, ws->stage_start, ws->stage_off,
                    ws->fstart, ws->fbase, ws->cstart, ws->part, ws->ctl, ws->tr_f_hi, ws->tr_f_lo,
                    ws->tr_size, ws->tr_peeled, ws->loc, ws->tdeg, ws->tlrp, ws->tcnt, ws->tfill,
                    ws->tgrp, ws->tcol, ws->tcw, ws->mask};
    for (void *q : ptrs) {
        if (!q) continue;
        if (ws->async) cudaFreeAsync(q, s);
        else cudaFree(q);
    }
    for (int j = 0; j < 7; j++)
        if (ws->ev[j]) cudaEventDestroy(ws->ev[j]);
    delete ws;
}

void workspace_free(PeelWorkspace *ws) { workspace_free(ws, 0); }

PeelWorkspace *workspace_create(long long n, long long arcs, bool has_cw, const PeelPlan &plan, bool async,
                                cudaStream_t s, int *rc) {
    const long long tail_cap = plan.hcap(), tr_cap = plan.tr_cap;
    PeelWorkspace *ws = new PeelWorkspace();
    cudaGetDevice(&ws->device);
    ws->n = n;
    ws->arcs = arcs;
    ws->tail_cap = tail_cap;
    ws->tr_cap = tr_cap;
    ws->tarc_cap = tail_arc_buffer(arcs, plan);
    ws->grid = peel_grid_size();
    ws->async = async;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto **ptr, long long count) {
        if (e != cudaSuccess) return;
        size_t sz = sizeof(**ptr) * (size_t)(count > 0 ? count : 1);
        e = async ? cudaMallocAsync((void **)ptr, sz, s) : cudaMalloc((void **)ptr, sz);
        if (e == cudaSuccess) ws->bytes += (long long)sz;
    };
    A(&ws->w, n);
    A(&ws->pr, n);
    A(&ws->live0, n);
    A(&ws->live1, n);
    A(&ws->stage_id, n);
    A(&ws->stage_start, n);
    A(&ws->stage_off, n);
    A(&ws->fstart, n);
    A(&ws->fbase, n + 1);
    A(&ws->cstart, ws->grid + 1);
    A(&ws->part, ws->grid);
    A(&ws->ctl, 1);
    A(&ws->tr_f_hi, tr_cap);
    A(&ws->tr_f_lo, tr_cap);
    A(&ws->tr_size, tr_cap);
    A(&ws->tr_peeled, tr_cap);
    A(&ws->loc, n);
    A(&ws->tdeg, tail_cap + 1);
    A(&ws->tlrp, tail_cap + 1);
    A(&ws->tcnt, tail_cap + 1);
    A(&ws->tfill, tail_cap + 1);
    A(&ws->tgrp, (tail_cap + 1) * DUPIN_GRP_STRIDE);
    A(&ws->tcol, ws->tarc_cap);
    if (has_cw) A(&ws->tcw, ws->tarc_cap);
    A(&ws->mask, n);
    if (e != cudaSuccess) {
        workspace_free(ws, s);
        cudaGetLastError();
        *rc = dupin_fail(e == cudaErrorMemoryAllocation ? DUPIN_ERR_OOM : DUPIN_ERR_CUDA,
                         std::string("peel workspace allocation failed: ") + cudaGetErrorString(e));
        return nullptr;
    }
    *rc = DUPIN_OK;
    return ws;
}

// Workspaces of freed graphs wait here for a later graph they fit (a caller
// that loads a new graph for every peel then pays no cudaMalloc / cudaFree for
// the peel state), at most WS_POOL_MAX of them; dupin_trim_cache frees them.
#define WS_POOL_MAX 8
static std::mutex g_pool_mu;
static std::vector<PeelWorkspace *> g_pool;

static bool workspace_fits(const PeelWorkspace *ws, int dev, long long n, long long tarc, bool has_cw,
                           const PeelPlan &plan) {
    return ws->device == dev && !ws->async && ws->n >= n && ws->tarc_cap >= tarc && ws->tail_cap >= plan.hcap() &&
           ws->tr_cap >= plan.tr_cap && (ws->tcw != nullptr || !has_cw);
}

// the smallest pooled workspace that fits, taken out of the pool (or null)
static PeelWorkspace *workspace_take(int dev, long long n, long long tarc, bool has_cw, const PeelPlan &plan) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    int best = -1;
    for (int j = 0; j < (int)g_pool.size(); j++)
        if (workspace_fits(g_pool[j], dev, n, tarc, has_cw, plan) &&
            (best < 0 || g_pool[j]->bytes < g_pool[best]->bytes))
            best = j;
    if (best < 0) return nullptr;
    PeelWorkspace *ws = g_pool[best];
    g_pool.erase(g_pool.begin() + best);
    return ws;
}

void workspace_release(PeelWorkspace *ws) {
    if (!ws) return;
    if (!ws->async) {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if ((int)g_pool.size() < WS_POOL_MAX) {
            g_pool.push_back(ws);
            return;
        }
    }
    workspace_free(ws);
}

extern "C" int dupin_trim_cache(void) {
    std::vector<PeelWorkspace *> v;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        v.swap(g_pool);
    }
    int dev = 0;
    cudaGetDevice(&dev);
    for (PeelWorkspace *ws : v) {
        cudaSetDevice(ws->device);
        workspace_free(ws);
    }
    cudaSetDevice(dev);
    graph_pool_trim();
    return DUPIN_OK;
}

static int workspace_ensure_ref(dupin_graph *g, PeelWorkspace *&slot, const PeelPlan &plan) {
    PeelWorkspace *ws = slot;
    const long long tarc = tail_arc_buffer(g->arcs, plan);
    const bool has_cw = g->cw != nullptr;
    if (ws && workspace_fits(ws, g->device, g->n, tarc, has_cw, plan)) return DUPIN_OK;
    PeelPlan big = plan;
    if (ws) {  // grow to cover both the old and the new caps
        big.cl_cap = std::max(plan.hcap(), ws->tail_cap);
        big.tr_cap = std::max(plan.tr_cap, ws->tr_cap);
        workspace_release(ws);
        slot = nullptr;
    }
    slot = workspace_take(g->device, g->n, tail_arc_buffer(g->arcs, big), has_cw, big);
    if (slot) return DUPIN_OK;
    int rc;
    slot = workspace_create(g->n, g->arcs, has_cw, big, false, 0, &rc);
    return rc;
}

int workspace_ensure(dupin_graph *g, const PeelPlan &plan) { return workspace_ensure_ref(g, g->ws, plan); }

PeelWorkspace *workspace_slot(dupin_graph *g, int k, const PeelPlan &plan, int *rc) {
    if (k == 0) {
        *rc = workspace_ensure(g, plan);
        return *rc ? nullptr : g->ws;
    }
    if ((int)g->ws_more.size() < k) g->ws_more.resize(k, nullptr);
    *rc = workspace_ensure_ref(g, g->ws_more[k - 1], plan);
    return *rc ? nullptr : g->ws_more[k - 1];
}

static PeelArgs make_args(const dupin_graph *g, const PeelWorkspace *ws, const dupin_params *p,
                          const PeelPlan &plan) {
    PeelArgs A;
    A.g = dev_graph(g, p->metric);
    A.w = ws->w;
    A.pr = ws->pr;
    A.live0 = ws->live0;
    A.live1 = ws->live1;
    A.stage_id = ws->stage_id;
    A.stage_start = ws->stage_start;
    A.stage_off = ws->stage_off;
    A.fstart = ws->fstart;
    A.fbase = ws->fbase;
    A.cstart = ws->cstart;
    A.part = ws->part;
    A.ctl = ws->ctl;
    A.tr_f_hi = ws->tr_f_hi;
    A.tr_f_lo = ws->tr_f_lo;
    A.tr_size = ws->tr_size;
    A.tr_peeled = ws->tr_peeled;
    A.tr_cap = ws->tr_cap;
    A.kD = (long long)p->k_mult * (p->eps_den + p->eps_num);
    A.D = p->eps_den;
    A.use_min = A.kD < 2 * A.D ? 1 : 0;
    A.gpo = (p->flags & (DUPIN_GPO | DUPIN_LPO)) ? 1 : 0;  // Algorithm 4 carries Algorithm 3
    A.lpo = (p->flags & DUPIN_LPO) ? 1 : 0;
    A.max_rounds = plan.max_rounds;
    A.tail_cap = plan.tail_cap;
    A.one_arcs = plan.one_arcs;
    A.cl_cap = plan.cl_cap;
    A.hcap = plan.hcap();
    A.tail_arcs = std::min<long long>(plan.tail_arcs, ws->tarc_cap);
    A.loc = ws->loc;
    A.tdeg = ws->tdeg;
    A.tlrp = ws->tlrp;
    A.tcnt = ws->tcnt;
    A.tfill = ws->tfill;
    A.tcol = ws->tcol;
    A.tcw = p->metric == DUPIN_DG ? nullptr : ws->tcw;
    A.tarc_cap = ws->tarc_cap;
    A.tgrp = ws->tgrp;
    A.cl_c = plan.cl_cap > 0 ? cluster_ctas() : 0;
    return A;
}

// Enqueue a whole peel on 'stream' (no host synchronisation).
__global__ void k_ctl_reset(PeelCtl *c) {
    PeelCtl z;
    memset(&z, 0, sizeof(z));
    z.init_min = kMaxLL;
    *c = z;
}

// A follower of a batched call: the initial weights of the same graph and
// metric copied from another workspace, the live state set up as the
// initial-weight kernels would, and the sums f(V) and min w copied.
__global__ void k_init_follow(long long n, const long long *src_w, long long *w, int *pr, int *live0) {
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
        w[u] = src_w[u];
        pr[u] = DUPIN_LIVE;
        live0[u] = (int)u;
    }
}

__global__ void k_init_follow_ctl(const PeelCtl *src, PeelCtl *dst) {
    dst->init_lo = src->init_lo;
    dst->init_hi = src->init_hi;
    dst->init_min = src->init_min;
    dst->init_overflow = src->init_overflow;
}

int enqueue_peel_stages(const dupin_graph *g, PeelWorkspace *ws, const dupin_params *p, const PeelPlan &plan,
                        int stages, cudaStream_t s, const PeelWorkspace *init_from, int bulk_grid) {
    PeelArgs A = make_args(g, ws, p, plan);
    const long long tail_cap = plan.hcap();  // tail buffers hold this many vertices
    const bool timing = (p->flags & DUPIN_TIMING) != 0;
    if (timing && !ws->ev[0]) {
        for (int j = 0; j < 7; j++) DUPIN_CUDA_TRY(cudaEventCreate(&ws->ev[j]));
    }
    int rc;
    if (stages & PEEL_INIT) {
        if (timing) DUPIN_CUDA_TRY(cudaEventRecord(ws->ev[0], s));
        k_ctl_reset<<<1, 1, 0, s>>>(ws->ctl);
        if (init_from) {
            int sms = 0, dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            k_init_follow<<<sms * 8, 256, 0, s>>>(g->n, init_from->w, ws->w, ws->pr, ws->live0);
            k_init_follow_ctl<<<1, 1, 0, s>>>(init_from->ctl, ws->ctl);
        } else {
            rc = launch_init_weights(A.g, p->metric, ws->w, ws->pr, ws->live0, ws->ctl, false, s);
            if (rc) return rc;
        }
        k_init_finish<<<1, 1, 0, s>>>(A, g->n);
        if (timing) DUPIN_CUDA_TRY(cudaEventRecord(ws->ev[1], s));
    }
    if (stages & PEEL_BULK) {
        if (timing) DUPIN_CUDA_TRY(cudaEventRecord(ws->ev[2], s));
        if (g->n > A.hcap || g->arcs > A.tail_arcs) {
            const int grid = bulk_grid > 0 && bulk_grid < ws->grid ? bulk_grid : ws->grid;
            void *args[] = {&A};
            cudaError_t e =
                cudaLaunchCooperativeKernel((void *)k_peel_bulk, dim3(grid), dim3(BULK_THREADS), args, 0, s);
            if (e != cudaSuccess) return dupin_cuda_fail(e, "cooperative launch of k_peel_bulk");
        }
        if (timing) DUPIN_CUDA_TRY(cudaEventRecord(ws->ev[3], s));
    }
    if (stages & PEEL_BUILD) {
        int sms = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (timing) DUPIN_CUDA_TRY(cudaEventRecord(ws->ev[4], s));
        DUPIN_CUDA_TRY(cudaMemsetAsync(ws->tcnt, 0, sizeof(int) * (size_t)(tail_cap + 1), s));
        DUPIN_CUDA_TRY(cudaMemsetAsync(ws->tfill, 0, sizeof(int) * (size_t)(tail_cap + 1), s));
        if (A.cl_c > 0)
            DUPIN_CUDA_TRY(cudaMemsetAsync(ws->tgrp, 0, sizeof(unsigned) * (size_t)(tail_cap + 1) * DUPIN_GRP_STRIDE, s));
        k_tail_prep<<<sms * 2, 256, 0, s>>>(A);
        k_tail_scan<<<1, SCAN_THREADS, 0, s>>>(A, ws->tdeg, nullptr);
        k_tail_arcs<0><<<sms * 2, BULK_THREADS, 0, s>>>(A);
        if (A.cl_c > 0) k_tail_rowcnt<<<sms, 256, 0, s>>>(A);
        // tcnt -> tlrp
        PeelArgs A2 = A;
        k_tail_scan<<<1, SCAN_THREADS, 0, s>>>(A2, ws->tlrp, ws->tcnt);
        if (A.cl_c > 0) k_tail_grp<<<sms, 256, 0, s>>>(A);
        k_tail_arcs<1><<<sms * 2, BULK_THREADS, 0, s>>>(A);
        if (timing) DUPIN_CUDA_TRY(cudaEventRecord(ws->ev[5], s));
    }
    if (stages & PEEL_TAIL) {
        // the status the grid-wide stage (or the set-up) left picks one of
        // the two tails; the other returns at once
        if (plan.tail_cap > 0) {
            rc = set_tail_smem();
            if (rc) return rc;
            k_peel_tail<<<1, TAIL_THREADS, (size_t)tail_smem_bytes(plan.tail_cap), s>>>(A);
        }
        if (plan.cl_cap > 0) {
            rc = launch_cluster_tail(A, s);
            if (rc) return rc;
        }
        if (timing) DUPIN_CUDA_TRY(cudaEventRecord(ws->ev[6], s));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return dupin_cuda_fail(e, "peel kernels");
    return DUPIN_OK;
}

int enqueue_peel(const dupin_graph *g, PeelWorkspace *ws, const dupin_params *p, const PeelPlan &plan,
                 cudaStream_t s) {
    return enqueue_peel_stages(g, ws, p, plan, PEEL_ALL, s);
}

int peel_resolve(const dupin_graph *g, const dupin_params *p, PeelPlan *plan) {
    int rc = check_params(g, p);
    if (rc) return rc;
    const long long lim = tail_cap_limit();
    const long long user = p->tail_cap > 0 ? p->tail_cap : 0;
    plan->tail_cap = user ? std::min<long long>(user, lim) : tail_cap_default();
    plan->cl_cap = 0;
    plan->one_arcs = DUPIN_ONE_CTA_ARCS;
    if (!(p->flags & DUPIN_TAIL_ONE_CTA)) {
        const long long climit = cluster_cap_limit();
        if (climit <= 0) {
            if (p->flags & DUPIN_TAIL_CLUSTER) return dupin_fail(DUPIN_ERR_CUDA, "no cluster tail on this device");
        } else {
            plan->cl_cap = user ? std::min<long long>(user, climit) : climit;
        }
    }
    if (p->flags & DUPIN_TAIL_ONE_CTA) plan->one_arcs = 0x7fffffffffffffffLL;  // every tail on one CTA
    if (plan->cl_cap == 0) plan->one_arcs = 0x7fffffffffffffffLL;
    if (p->flags & DUPIN_TAIL_CLUSTER) plan->tail_cap = 0;  // every tail on the cluster
    plan->tail_arcs = p->tail_arc_cap > 0 ? p->tail_arc_cap : DUPIN_TAIL_ARCS_DEFAULT;
    plan->max_rounds = p->max_rounds > 0 ? p->max_rounds : g->n + 1;
    plan->tr_cap = std::min<long long>(plan->max_rounds, g->n) + 1;
    return DUPIN_OK;
}

int peel_finish(const dupin_graph *g, PeelWorkspace *ws, const dupin_params *p, dupin_result *r, cudaStream_t s) {
    PeelCtl c;
    DUPIN_CUDA_TRY(cudaMemcpyAsync(&c, ws->ctl, sizeof(PeelCtl), cudaMemcpyDeviceToHost, s));
    DUPIN_CUDA_TRY(cudaStreamSynchronize(s));
    r->n_rounds = c.round;
    r->n_min_rule = c.n_min_rule;
    r->n_bulk_rounds = c.bulk_rounds;
    r->tail_arcs = c.tail_arcs;
    r->tail_ctas = c.tail_ctas;
    for (int j = 0; j < 4; j++) r->phase_ms[j] = 0.f;
    if ((p->flags & DUPIN_TIMING) && ws->ev[0]) {
        // init, grid-wide rounds, tail build, tail (the stages of several peels
        // run together interleave, so each has its own start event)
        cudaEventElapsedTime(&r->phase_ms[0], ws->ev[0], ws->ev[1]);
        cudaEventElapsedTime(&r->phase_ms[1], ws->ev[2], ws->ev[3]);
        cudaEventElapsedTime(&r->phase_ms[2], ws->ev[4], ws->ev[5]);
        cudaEventElapsedTime(&r->phase_ms[3], ws->ev[5], ws->ev[6]);
    }
    if (c.error) {
        const char *why = c.error == DUPIN_ERR_NO_PROGRESS ? "max_rounds reached before the set became empty"
                          : c.error == DUPIN_ERR_TIMEOUT   ? "an in-kernel grid barrier timed out"
                          : c.error == DUPIN_ERR_OVERFLOW  ? "peeling weight overflow"
                          : c.error == DUPIN_ERR_OOM       ? "tail sub-graph exceeds its buffer"
                                                           : "peel failed";
        return dupin_fail(c.error, why);
    }
    if (c.status != ST_DONE) return dupin_fail(DUPIN_ERR_CUDA, "peel did not complete");
    r->best_round = c.best_round;
    r->best_size = c.best_size;
    r->best_f_hi = (long long)c.bf_hi;
    r->best_f_lo = c.bf_lo;
    {
        u128 bf = mk128(c.bf_lo, c.bf_hi);
        r->best_density = c.best_size > 0 ? (double)bf / 4294967296.0 / (double)c.best_size : 0.0;
    }
    const bool dev = (p->flags & DUPIN_RESULT_DEVICE) != 0;
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const long long n = g->n;
    if (r->best_mask && n > 0) {
        int sms = 0, d = 0;
        cudaGetDevice(&d);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
        uint8_t *dst = dev ? r->best_mask : ws->mask;
        k_finalize<<<sms * 4, 256, 0, s>>>(ws->pr, n, ws->ctl, dst);
        if (!dev) DUPIN_CUDA_TRY(cudaMemcpyAsync(r->best_mask, ws->mask, (size_t)n, cudaMemcpyDeviceToHost, s));
    }
    if (r->peel_round && n > 0)
        DUPIN_CUDA_TRY(cudaMemcpyAsync(r->peel_round, ws->pr, sizeof(int) * (size_t)n, kind, s));
    const long long nt = c.round + 1;
    bool trace_short = false;
    if (r->trace_f_hi || r->trace_f_lo || r->trace_size || r->trace_peeled) {
        long long cnt = std::min<long long>(nt, (long long)r->trace_cap);
        if (r->trace_cap < nt) trace_short = true;
        if (cnt > 0) {
            if (r->trace_f_hi) DUPIN_CUDA_TRY(cudaMemcpyAsync(r->trace_f_hi, ws->tr_f_hi, 8 * (size_t)cnt, kind, s));
            if (r->trace_f_lo) DUPIN_CUDA_TRY(cudaMemcpyAsync(r->trace_f_lo, ws->tr_f_lo, 8 * (size_t)cnt, kind, s));
            if (r->trace_size) DUPIN_CUDA_TRY(cudaMemcpyAsync(r->trace_size, ws->tr_size, 8 * (size_t)cnt, kind, s));
            if (r->trace_peeled) DUPIN_CUDA_TRY(cudaMemcpyAsync(r->trace_peeled, ws->tr_peeled, 8 * (size_t)cnt, kind, s));
        }
    }
    DUPIN_CUDA_TRY(cudaStreamSynchronize(s));
    if (trace_short)
        return dupin_fail(DUPIN_ERR_BUFFER_TOO_SMALL, "trace_cap < n_rounds + 1 (n_rounds is filled)");
    return DUPIN_OK;
}

// A whole peel of a graph small enough for the one-CTA kernel, every buffer
// supplied by the caller through A (no allocation): reset the control block,
// initial weights (validated when 'check'), round 0, then all rounds in one CTA.
int launch_small_graph_peel(const PeelArgs &A, int metric, bool check, cudaStream_t s) {
    k_ctl_reset<<<1, 1, 0, s>>>(A.ctl);
    int rc = launch_init_weights(A.g, metric, A.w, A.pr, A.live0, A.ctl, check, s);
    if (rc) return rc;
    k_init_finish<<<1, 1, 0, s>>>(A, A.g.n);
    rc = set_tail_smem();
    if (rc) return rc;
    k_peel_tail<<<1, TAIL_THREADS, (size_t)tail_smem_bytes(A.tail_cap), s>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return dupin_cuda_fail(e, "small-graph peel kernels");
    return DUPIN_OK;
}

// The hand-over autotuner: the peel of this graph under each candidate
// tail_arc_cap (the live-arc count below which the grid-wide rounds hand
// over to a tail even when their last round was large), once to warm up and
// twice more timed; the fastest candidate wins.
static const long long kHandover[DUPIN_TUNE_HANDOVER_N] = {1ll << 16, 1ll << 18, 1ll << 20,
                                                           1ll << 22, 1ll << 24, 1ll << 26};

extern "C" int dupin_tune_handover(dupin_graph *g, const dupin_params *params, void *stream, int64_t *best,
                                   float *times_ms) {
    if (!g || !params) return dupin_fail(DUPIN_ERR_INVALID_ARG, "graph and params must be non-NULL");
    if (is_clique_metric(params->metric))
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "the clique metrics have no tail to hand over to");
    double t_best[DUPIN_TUNE_HANDOVER_N];
    for (int i = 0; i < DUPIN_TUNE_HANDOVER_N; i++) t_best[i] = 1e300;
    for (int rep = 0; rep < 3; rep++) {
        for (int i = 0; i < DUPIN_TUNE_HANDOVER_N; i++) {
            dupin_params p = *params;
            p.tail_arc_cap = kHandover[i];
            p.flags &= ~(DUPIN_RESULT_DEVICE | DUPIN_TIMING);
            dupin_result r;
            memset(&r, 0, sizeof(r));
            const auto t0 = std::chrono::steady_clock::now();
            const int rc = dupin_peel(g, &p, &r, stream);  // returns once the peel is complete
            const double t = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (rc) return rc;
            if (rep > 0) t_best[i] = std::min(t_best[i], t);  // the first pass warms up
        }
    }
    int pick = 0;
    for (int i = 1; i < DUPIN_TUNE_HANDOVER_N; i++)
        if (t_best[i] < t_best[pick]) pick = i;
    if (best) *best = kHandover[pick];
    if (times_ms)
        for (int i = 0; i < DUPIN_TUNE_HANDOVER_N; i++) times_ms[i] = (float)(t_best[i] * 1e3);
    return DUPIN_OK;
}

extern "C" int dupin_peel(dupin_graph *g, const dupin_params *p, dupin_result *r, void *stream) {
    if (!g) return dupin_fail(DUPIN_ERR_INVALID_ARG, "graph is NULL");
    if (!r) return dupin_fail(DUPIN_ERR_INVALID_ARG, "result is NULL");
    PeelPlan plan;
    int rc = peel_resolve(g, p, &plan);
    if (rc) return rc;
    DUPIN_CUDA_TRY(cudaSetDevice(g->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (is_clique_metric(p->metric)) return tds_peel(g, p, r, s);
    rc = workspace_ensure(g, plan);
    if (rc) return rc;
    rc = enqueue_peel(g, g->ws, p, plan, s);
    if (rc) return rc;
    return peel_finish(g, g->ws, p, r, s);
}
