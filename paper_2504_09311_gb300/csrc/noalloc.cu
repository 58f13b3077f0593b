// noalloc.cu -- dupin_peel_noalloc: a peel that allocates no memory.
//
// Who needs it: callers that may not allocate device memory once they are
// running -- services that reserve all GPU memory up front through their own
// pool and forbid later allocation, latency-critical loops in which
// cudaMalloc/cudaFree would synchronise the device and stall concurrent
// work, and plug-ins hosted by a process whose allocator owns the device.
// They pass the graph and every output in memory they already own; the
// working state lives in one file-scope device array of fixed size, so the
// call itself allocates nothing (no cudaMalloc, no cudaFree, no allocating
// library routine).
//
// Limits and sharing: graphs of at most DUPIN_NOALLOC_MAX_N vertices (the
// whole peel then runs in the one-CTA kernel).  Every GPU that loads the
// library holds the array (about 100 KB) until the process exits.  All calls
// on a device share it and it keeps the last call's contents; each call
// clears what must start at zero, but calls that overlap on the GPU (other
// streams, other threads) race on it and must be serialised by the caller.
// The first call on a device looks up the array's device address
// (cudaGetSymbolAddress) and sets the one-CTA kernel's shared-memory limit;
// make that first call before any stream capture.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <string>

#include "dupin_internal.h"

#define NOALLOC_CTL_BYTES 512
#define NOALLOC_FLAG_BYTES 256
#define NOALLOC_BYTES \
    (NOALLOC_CTL_BYTES + NOALLOC_FLAG_BYTES + 8 * DUPIN_NOALLOC_MAX_N + 4 * DUPIN_NOALLOC_MAX_N)

static_assert(sizeof(PeelCtl) <= NOALLOC_CTL_BYTES, "control block must fit its slot");

// The working state of dupin_peel_noalloc: control block | flags | w | live.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {

std::mutex g_mu;
void *g_addr[256];  // device address of g_noalloc_scratch, per device ordinal

// Set-up, once per device with that device current: the array's device
// address.  The host-side name of the array is only a stand-in and must not
// be given to a kernel.
int scratch_address(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= 256) return dupin_fail(DUPIN_ERR_INVALID_ARG, "device ordinal out of range");
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return dupin_cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_addr[dev] = p;
    }
    *out = (unsigned char *)g_addr[dev];
    return DUPIN_OK;
}

}  // namespace

// flags[0] = 1 when an offset, id or weight is out of range; flags[1..2] = rp[n]
__global__ void k_noalloc_check(const long long *rp, const int *col, const long long *cw, const long long *a,
                                long long n, int *flags) {
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
        const long long b = rp[u], e = rp[u + 1];
        if (b > e || (u == 0 && b != 0)) {
            atomicExch(&flags[0], 1);
            continue;
        }
        if (a && a[u] < 0) atomicExch(&flags[0], 1);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *(long long *)(flags + 2) = rp[n];
    (void)col;
    (void)cw;
}

// ids in range, no self-loops, weights >= 0 (run only after the offsets
// passed); flags[4..5] accumulate the symmetry fingerprint (sum over arcs of
// sym_mix(u, v, c) - sym_mix(v, u, c), zero for a symmetric CSR)
__global__ void k_noalloc_check_arcs(const long long *rp, const int *col, const long long *cw, long long n,
                                     unsigned long long key, int *flags) {
    unsigned long long fp = 0;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
        for (long long p = rp[u]; p < rp[u + 1]; p++) {
            const int v = col[p];
            const long long c = cw ? cw[p] : DUPIN_Q_ONE;
            if (v < 0 || v >= n || v == u || c < 0) {
                atomicExch(&flags[0], 1);
                continue;
            }
            fp += sym_mix(key, u, v, c) - sym_mix(key, v, u, c);
        }
    }
    if (fp) atomicAdd((unsigned long long *)(flags + 4), fp);
}

__global__ void k_noalloc_mask(const int *pr, long long n, long long best_round, uint8_t *mask) {
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x)
        mask[u] = (long long)pr[u] > best_round ? 1 : 0;
}

extern "C" int dupin_peel_noalloc(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const int64_t *arc_w,
                                  const int64_t *vertex_w, const dupin_params *params, int32_t *peel_round,
                                  dupin_result *result, void *stream) {
    if (!params || !result || !row_ptr || !peel_round)
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "row_ptr, params, peel_round and result must be non-NULL");
    if (n < 1 || n > DUPIN_NOALLOC_MAX_N)
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "dupin_peel_noalloc takes 1 <= n <= " +
                                                     std::to_string(DUPIN_NOALLOC_MAX_N) + " vertices (got " +
                                                     std::to_string((long long)n) + ")");
    const dupin_params &p = *params;
    if (p.metric < DUPIN_DG || p.metric > DUPIN_FD) return dupin_fail(DUPIN_ERR_INVALID_ARG, "unknown metric");
    if (p.k_mult < 1 || p.k_mult > 64) return dupin_fail(DUPIN_ERR_INVALID_ARG, "k_mult must be in 1..64");
    if (p.eps_den < 1 || p.eps_den > (1LL << 24) || p.eps_num < 0 || p.eps_num > (1LL << 30))
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "eps must be eps_num/eps_den, 0 <= eps_num <= 2^30, 1 <= eps_den <= 2^24");
    if (p.flags & ~(uint32_t)(DUPIN_GPO | DUPIN_LPO))
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "dupin_peel_noalloc accepts only the DUPIN_GPO and DUPIN_LPO flags");
    if (p.metric != DUPIN_DG && !arc_w) return dupin_fail(DUPIN_ERR_INVALID_ARG, "DW/FD need arc weights");
    if (n > tail_cap_limit())
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "this device's shared memory cannot hold the graph's state");
    if ((result->trace_f_hi || result->trace_f_lo || result->trace_size || result->trace_peeled) && result->trace_cap < 1)
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "trace arrays given with trace_cap < 1");
    int dev = 0;
    DUPIN_CUDA_TRY(cudaGetDevice(&dev));
    unsigned char *base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc) return rc;
    PeelCtl *ctl = (PeelCtl *)base;
    int *flags = (int *)(base + NOALLOC_CTL_BYTES);
    long long *w = (long long *)(base + NOALLOC_CTL_BYTES + NOALLOC_FLAG_BYTES);
    int *live = (int *)(base + NOALLOC_CTL_BYTES + NOALLOC_FLAG_BYTES + 8 * DUPIN_NOALLOC_MAX_N);
    cudaStream_t s = (cudaStream_t)stream;
    const long long *rp = (const long long *)row_ptr;
    const int *col = (const int *)col_idx;
    const long long *cw = p.metric == DUPIN_DG ? nullptr : (const long long *)arc_w;
    const long long *a = p.metric == DUPIN_DG ? nullptr : (const long long *)vertex_w;

    // validate the caller's CSR before any kernel indexes through it
    DUPIN_CUDA_TRY(cudaMemsetAsync(flags, 0, NOALLOC_FLAG_BYTES, s));
    k_noalloc_check<<<32, 256, 0, s>>>(rp, col, cw, a, n, flags);
    DUPIN_CUDA_TRY(cudaGetLastError());
    int hflags[6] = {0, 0, 0, 0, 0, 0};
    DUPIN_CUDA_TRY(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, s));
    DUPIN_CUDA_TRY(cudaStreamSynchronize(s));
    long long arcs = 0;
    memcpy(&arcs, hflags + 2, sizeof(arcs));
    if (hflags[0] || arcs < 0) return dupin_fail(DUPIN_ERR_INVALID_ARG, "invalid CSR offsets or vertex weights");
    if (arcs & 1) return dupin_fail(DUPIN_ERR_INVALID_ARG, "a symmetric CSR has an even arc count");
    if (arcs > 0 && !col) return dupin_fail(DUPIN_ERR_INVALID_ARG, "col_idx is NULL");
    k_noalloc_check_arcs<<<32, 256, 0, s>>>(rp, col, cw, n, fingerprint_key(), flags);
    DUPIN_CUDA_TRY(cudaGetLastError());
    DUPIN_CUDA_TRY(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, s));
    DUPIN_CUDA_TRY(cudaStreamSynchronize(s));
    if (hflags[0]) return dupin_fail(DUPIN_ERR_INVALID_ARG, "invalid CSR: neighbour id out of range, self-loop or negative weight");
    unsigned long long fp = 0;
    memcpy(&fp, hflags + 4, sizeof(fp));
    if (fp) return dupin_fail(DUPIN_ERR_INVALID_ARG, "the CSR is not symmetric (an arc without a reverse arc of equal weight)");

    PeelArgs A;
    memset(&A, 0, sizeof(A));
    A.g.n = n;
    A.g.arcs = arcs;
    A.g.rp = rp;
    A.g.col = col;
    A.g.cw = cw;
    A.g.a = a;
    A.w = w;
    A.pr = (int *)peel_round;
    A.live0 = live;
    A.live1 = live;
    A.ctl = ctl;
    A.tr_f_hi = (long long *)result->trace_f_hi;
    A.tr_f_lo = (unsigned long long *)result->trace_f_lo;
    A.tr_size = (long long *)result->trace_size;
    A.tr_peeled = (long long *)result->trace_peeled;
    const bool tr = A.tr_f_hi && A.tr_f_lo && A.tr_size && A.tr_peeled;
    A.tr_cap = tr ? result->trace_cap : 0;
    A.kD = (long long)p.k_mult * (p.eps_den + p.eps_num);
    A.D = p.eps_den;
    A.use_min = A.kD < 2 * A.D ? 1 : 0;
    A.gpo = (p.flags & (DUPIN_GPO | DUPIN_LPO)) ? 1 : 0;
    A.lpo = (p.flags & DUPIN_LPO) ? 1 : 0;
    A.max_rounds = p.max_rounds > 0 ? p.max_rounds : n + 1;
    // the one-CTA kernel's shared memory follows the graph's size
    A.tail_cap = n;
    A.hcap = n;
    A.cl_cap = 0;
    A.one_arcs = 0x7fffffffffffffffLL;
    A.tail_arcs = arcs;
    // the graph itself is the one-CTA kernel's sub-graph (local ids = ids)
    A.tlrp = (long long *)rp;
    A.tcol = (int *)col;
    A.tcw = (long long *)cw;
    rc = launch_small_graph_peel(A, p.metric, cw != nullptr, s);
    if (rc) return rc;

    PeelCtl c;
    DUPIN_CUDA_TRY(cudaMemcpyAsync(&c, ctl, sizeof(PeelCtl), cudaMemcpyDeviceToHost, s));
    DUPIN_CUDA_TRY(cudaStreamSynchronize(s));
    result->n_rounds = c.round;
    result->n_min_rule = c.n_min_rule;
    result->n_bulk_rounds = 0;
    result->tail_arcs = arcs;
    for (int j = 0; j < 4; j++) result->phase_ms[j] = 0.f;
    if (c.error) {
        return dupin_fail(c.error, c.error == DUPIN_ERR_NO_PROGRESS ? "max_rounds reached before the set became empty"
                                   : c.error == DUPIN_ERR_OVERFLOW  ? "a peeling weight does not fit in int64"
                                                                    : "peel failed");
    }
    if (c.status != ST_DONE) return dupin_fail(DUPIN_ERR_CUDA, "peel did not complete");
    result->best_round = c.best_round;
    result->best_size = c.best_size;
    result->best_f_hi = (long long)c.bf_hi;
    result->best_f_lo = c.bf_lo;
    const u128 bf = mk128(c.bf_lo, c.bf_hi);
    result->best_density = c.best_size > 0 ? (double)bf / 4294967296.0 / (double)c.best_size : 0.0;
    if (result->best_mask) {
        k_noalloc_mask<<<32, 256, 0, s>>>(A.pr, n, c.best_round, result->best_mask);
        DUPIN_CUDA_TRY(cudaGetLastError());
        DUPIN_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (tr && result->trace_cap < c.round + 1)
        return dupin_fail(DUPIN_ERR_BUFFER_TOO_SMALL, "trace_cap < n_rounds + 1 (n_rounds is filled)");
    return DUPIN_OK;
}
