// graph.cu -- loading a graph into HBM as one symmetric adjacency.
//
// Input forms (Sec. 2.1): a bipartite users x items graph as CSR (users ->
// items) plus CSC (items -> users), or a general undirected graph as a
// symmetric CSR.  The device copy is always one CSR over n = users + items
// vertices: rows [0, n_left) are users whose neighbour ids are shifted by
// n_left (items become vertices n_left + i), rows [n_left, n) are items.
// Validation runs on the device: offsets monotone and starting at 0, ids in
// range, no self-loops, weights >= 0 (Property 3.1), every initial peeling
// weight a_u + sum_v c_uv below 2^63 (checked with the same segmented-sum
// kernel the peel uses), every row's neighbour ids strictly increasing (so
// no pair repeats), and the adjacency symmetric with equal weights on an
// arc and its reverse -- for a bipartite graph, the CSC holds exactly the
// CSR's edges -- by a keyed fingerprint of the arc multiset against its
// reverse (a missing or re-weighted reverse arc passes with probability
// about 2^-64).
#include <cuda_runtime.h>
#include <stdint.h>

#include <string.h>

#include <string>

#include <map>
#include <mutex>
#include "dupin_internal.h"

// Device buffers of graphs come from a memory pool of the library's own,
// stream-ordered, that keeps freed memory (dupin_trim_cache releases it): a
// caller that loads a new graph for every peel then pays no cudaMalloc /
// cudaFree for the adjacency and the loader's temporaries.
static cudaMemPool_t graph_pool(int dev) {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lk(mu);
    auto it = pools.find(dev);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    unsigned long long keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = pool;
    return pool;
}

static cudaError_t galloc(void **p, size_t bytes, cudaStream_t s) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool = graph_pool(dev);
    if (!bytes) bytes = 8;
    return pool ? cudaMallocFromPoolAsync(p, bytes, pool, s) : cudaMallocAsync(p, bytes, s);
}

static void gfree(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

void graph_pool_trim() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaMemPool_t pool = graph_pool(dev);
    if (pool) cudaMemPoolTrimTo(pool, 0);
}

__global__ void k_add_offset_i64(long long *x, long long n, long long add) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] += add;
}

__global__ void k_add_offset_i32(int *x, long long n, int add, int limit, int *bad) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int v = x[i];
        if (v < 0 || v >= limit) atomicExch(bad, 1);
        x[i] = v + add;
    }
}

// offsets: rp[0] == 0, non-decreasing, rp[n] == arcs
__global__ void k_check_offsets(const long long *rp, long long n, long long arcs, int *bad) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (rp[i] > rp[i + 1]) atomicExch(bad, 1);
    if (blockIdx.x == 0 && threadIdx.x == 0 && (rp[0] != 0 || rp[n] != arcs)) atomicExch(bad, 1);
}

__global__ void k_fill_i64(long long *x, long long n, long long v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] = v;
}

__global__ void k_check_nonneg(const long long *x, long long n, int *bad) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (x[i] < 0) atomicExch(bad, 1);
}

static cudaMemcpyKind kind_of(bool dev) { return dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }

static int read_last(const int64_t *p, long long idx, bool dev, long long *out) {
    if (!p) return dupin_fail(DUPIN_ERR_INVALID_ARG, "offset array is NULL");
    if (dev) {
        cudaError_t e = cudaMemcpy(out, p + idx, sizeof(long long), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return dupin_cuda_fail(e, "reading an offset");
    } else {
        *out = p[idx];
    }
    return DUPIN_OK;
}

// log2 histogram of degrees >= DUPIN_HUB_MIN_DEG
__global__ void k_deg_hist(const long long *rp, long long n, unsigned long long *hist) {
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
        const long long d = rp[u + 1] - rp[u];
        if (d >= DUPIN_HUB_MIN_DEG) atomicAdd(&hist[63 - __clzll(d)], 1ull);
    }
}

// hubs[] holds 'cap' entries: exactly the number of vertices with degree >= thr
__global__ void k_pick_hubs(const long long *rp, long long n, long long thr, int *slot_of, int *hubs, int *nh,
                            int cap) {
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
        const long long d = rp[u + 1] - rp[u];
        if (d >= thr) {
            const int h = atomicAdd(nh, 1);
            if (h < cap) {
                hubs[h] = (int)u;
                slot_of[u] = h;
            }
        }
    }
}

__global__ void k_encode_hub_arcs(int *col, long long arcs, const int *slot_of) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < arcs; p += (long long)gridDim.x * blockDim.x) {
        const int h = slot_of[col[p]];
        if (h >= 0) col[p] = -(h + 1);
    }
}

__global__ void k_fill_i32(int *x, long long n, int v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] = v;
}

// Pick the hubs (at most DUPIN_HUB_MAX vertices, highest degrees first, degree
// >= DUPIN_HUB_MIN_DEG, threshold a power of two) and re-code their arcs.
static int select_hubs(dupin_graph *g, int grid, cudaStream_t s) {
    if (g->arcs == 0 || g->n == 0) return DUPIN_OK;
    unsigned long long *hist = nullptr;
    int *nh = nullptr, *slot_of = nullptr;
    unsigned long long h[64];
    cudaError_t e = galloc((void **)&hist, 64 * sizeof(unsigned long long) + sizeof(int), s);
    if (e != cudaSuccess) return dupin_cuda_fail(e, "hub histogram");
    nh = (int *)(hist + 64);
    e = cudaMemsetAsync(hist, 0, 64 * sizeof(unsigned long long) + sizeof(int), s);
    if (e == cudaSuccess) {
        k_deg_hist<<<grid, 256, 0, s>>>(g->rp, g->n, hist);
        e = cudaMemcpyAsync(h, hist, sizeof(h), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        gfree(hist, s);
        return dupin_cuda_fail(e, "hub histogram");
    }
    // smallest power-of-two threshold >= DUPIN_HUB_MIN_DEG keeping at most
    // DUPIN_HUB_MAX vertices; cum = number of vertices with degree >= 2^bstar
    const int bmin = 63 - __builtin_clzll((unsigned long long)DUPIN_HUB_MIN_DEG);
    int bstar = -1;
    unsigned long long cum = 0;
    for (int b = 63; b >= bmin; b--) {
        if (cum + h[b] > DUPIN_HUB_MAX) break;
        cum += h[b];
        bstar = b;
    }
    if (bstar < 0 || cum == 0) {
        gfree(hist, s);
        return DUPIN_OK;
    }
    const long long thr = 1LL << bstar;
    e = galloc((void **)&g->hubs, sizeof(int) * (size_t)cum, s);
    if (e == cudaSuccess) e = galloc((void **)&slot_of, sizeof(int) * (size_t)g->n, s);
    if (e == cudaSuccess) {
        k_fill_i32<<<grid, 256, 0, s>>>(slot_of, g->n, -1);
        k_pick_hubs<<<grid, 256, 0, s>>>(g->rp, g->n, thr, slot_of, g->hubs, nh, (int)cum);
        k_encode_hub_arcs<<<grid, 256, 0, s>>>(g->col, g->arcs, slot_of);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    gfree(slot_of, s);
    gfree(hist, s);
    if (e != cudaSuccess) return dupin_cuda_fail(e, "hub selection");
    g->n_hubs = (int)cum;
    g->bytes += (long long)sizeof(int) * (long long)cum;
    return DUPIN_OK;
}

static void graph_release(dupin_graph *g) {
    if (!g) return;
    workspace_release(g->ws);
    for (PeelWorkspace *w : g->ws_more) workspace_release(w);
    // no work on the graph may be in flight when it is freed (as cudaFree would
    // have enforced); then its buffers go back to the pool
    cudaDeviceSynchronize();
    gfree(g->hubs, 0);
    gfree(g->rp, 0);
    gfree(g->col, 0);
    gfree(g->cw, 0);
    gfree(g->a, 0);
    delete g;
}

extern "C" int dupin_graph_load(const dupin_graph_desc *d, void *stream, dupin_graph **out) {
    if (!d || !out) return dupin_fail(DUPIN_ERR_INVALID_ARG, "desc or out is NULL");
    *out = nullptr;
    const bool dev = (d->flags & DUPIN_DEVICE_PTRS) != 0;
    if (d->flags & ~DUPIN_DEVICE_PTRS) return dupin_fail(DUPIN_ERR_INVALID_ARG, "unknown graph flag");
    const long long nL = d->n_left, nR = d->n_right;
    if (nL < 0 || nR < 0 || nL + nR > 0x7ffffffeLL)
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "vertex counts must be >= 0 and n < 2^31 - 1");
    const bool bip = nR > 0;
    if (!d->csr_ptr || (!d->csr_idx && nL > 0)) return dupin_fail(DUPIN_ERR_INVALID_ARG, "csr_ptr / csr_idx missing");
    if (bip && (!d->csc_ptr || !d->csc_idx)) return dupin_fail(DUPIN_ERR_INVALID_ARG, "bipartite graph needs csc_*");
    if (bip && ((d->csr_w == nullptr) != (d->csc_w == nullptr)))
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "csr_w and csc_w must both be given or both be NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    long long m_csr = 0, m_csc = 0;
    if ((rc = read_last(d->csr_ptr, nL, dev, &m_csr))) return rc;
    if (bip && (rc = read_last(d->csc_ptr, nR, dev, &m_csc))) return rc;
    if (m_csr < 0 || (bip && m_csc != m_csr))
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "CSR and CSC hold different edge counts");
    const long long n = nL + nR;
    const long long arcs = bip ? 2 * m_csr : m_csr;
    if (!bip && (arcs & 1)) return dupin_fail(DUPIN_ERR_INVALID_ARG, "a symmetric CSR has an even number of arcs");
    if (arcs >= (1LL << 40)) return dupin_fail(DUPIN_ERR_INVALID_ARG, "a graph holds fewer than 2^40 arcs");

    dupin_graph *g = new dupin_graph();
    cudaGetDevice(&g->device);
    g->n_left = nL;
    g->n_right = nR;
    g->n = n;
    g->arcs = arcs;
    g->m = arcs / 2;
    const bool has_w = d->csr_w != nullptr;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
        if (e != cudaSuccess) return;
        e = galloc(p, bytes ? bytes : 8, s);
        if (e == cudaSuccess) g->bytes += (long long)bytes;
    };
    alloc((void **)&g->rp, sizeof(long long) * (size_t)(n + 1));
    alloc((void **)&g->col, sizeof(int) * (size_t)arcs);
    if (has_w) alloc((void **)&g->cw, sizeof(long long) * (size_t)arcs);
    if (d->vertex_w) alloc((void **)&g->a, sizeof(long long) * (size_t)n);
    int *bad = nullptr;
    if (e == cudaSuccess) e = galloc((void **)&bad, sizeof(int), s);
    if (e != cudaSuccess) {
        graph_release(g);
        gfree(bad, s);
        cudaGetLastError();
        return dupin_fail(e == cudaErrorMemoryAllocation ? DUPIN_ERR_OOM : DUPIN_ERR_CUDA,
                          std::string("graph allocation: ") + cudaGetErrorString(e));
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    const int grid = sms * 4;
    const cudaMemcpyKind k = kind_of(dev);
#define TRY(expr)                                    \
    do {                                             \
        cudaError_t _e = (expr);                     \
        if (_e != cudaSuccess) {                     \
            int _r = dupin_cuda_fail(_e, #expr);     \
            graph_release(g);                        \
            gfree(bad, s);                           \
            return _r;                               \
        }                                            \
    } while (0)
    TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
    const long long m = m_csr;
    if (bip) {
        TRY(cudaMemcpyAsync(g->rp, d->csr_ptr, sizeof(long long) * (size_t)(nL + 1), k, s));
        // item rows: csc_ptr[1..nR] + m
        TRY(cudaMemcpyAsync(g->rp + nL + 1, d->csc_ptr + 1, sizeof(long long) * (size_t)nR, k, s));
        k_add_offset_i64<<<grid, 256, 0, s>>>(g->rp + nL + 1, nR, m);
        if (m > 0) {
            TRY(cudaMemcpyAsync(g->col, d->csr_idx, sizeof(int) * (size_t)m, k, s));
            TRY(cudaMemcpyAsync(g->col + m, d->csc_idx, sizeof(int) * (size_t)m, k, s));
            k_add_offset_i32<<<grid, 256, 0, s>>>(g->col, m, (int)nL, (int)nR, bad);   // items -> global ids
            k_add_offset_i32<<<grid, 256, 0, s>>>(g->col + m, m, 0, (int)nL, bad);     // users stay
            if (has_w) {
                TRY(cudaMemcpyAsync(g->cw, d->csr_w, sizeof(long long) * (size_t)m, k, s));
                TRY(cudaMemcpyAsync(g->cw + m, d->csc_w, sizeof(long long) * (size_t)m, k, s));
            }
        }
        // csc_ptr must itself start at 0
        long long c0 = 0;
        if (dev) TRY(cudaMemcpy(&c0, d->csc_ptr, sizeof(long long), cudaMemcpyDeviceToHost));
        else c0 = d->csc_ptr[0];
        if (c0 != 0) {
            graph_release(g);
            gfree(bad, s);
            return dupin_fail(DUPIN_ERR_INVALID_ARG, "csc_ptr[0] must be 0");
        }
    } else {
        TRY(cudaMemcpyAsync(g->rp, d->csr_ptr, sizeof(long long) * (size_t)(n + 1), k, s));
        if (arcs > 0) {
            TRY(cudaMemcpyAsync(g->col, d->csr_idx, sizeof(int) * (size_t)arcs, k, s));
            if (has_w) TRY(cudaMemcpyAsync(g->cw, d->csr_w, sizeof(long long) * (size_t)arcs, k, s));
        }
    }
    if (d->vertex_w) TRY(cudaMemcpyAsync(g->a, d->vertex_w, sizeof(long long) * (size_t)n, k, s));
    k_check_offsets<<<grid, 256, 0, s>>>(g->rp, n, arcs, bad);
    if (has_w) k_check_nonneg<<<grid, 256, 0, s>>>(g->cw, arcs, bad);
    if (g->a) k_check_nonneg<<<grid, 256, 0, s>>>(g->a, n, bad);
    int hbad = 0;
    TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    if (hbad) {
        graph_release(g);
        gfree(bad, s);
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "invalid CSR: offsets, ids or weights out of range");
    }
    // ids in range, no self-loops, and w_u(V) < 2^63 for the weights given
    {
        long long *w = nullptr;
        PeelCtl *ctl = nullptr;
        TRY(galloc((void **)&w, sizeof(long long) * (size_t)(n > 0 ? n : 1), s));
        e = galloc((void **)&ctl, sizeof(PeelCtl), s);
        if (e != cudaSuccess) {
            gfree(w, s);
            TRY(e);
        }
        PeelCtl hc;
        memset(&hc, 0, sizeof(hc));
        hc.init_min = 0x7fffffffffffffffLL;
        cudaMemcpyAsync(ctl, &hc, sizeof(PeelCtl), cudaMemcpyHostToDevice, s);
        DevGraph dg = {};
        dg.n = n;
        dg.arcs = arcs;
        dg.rp = g->rp;
        dg.col = g->col;
        // without weights every arc is 1.0: validate ids with a temporary unit weight array
        long long *unit = nullptr;
        if (!has_w && arcs > 0) {
            e = galloc((void **)&unit, sizeof(long long) * (size_t)arcs, s);
            if (e == cudaSuccess) k_fill_i64<<<grid, 256, 0, s>>>(unit, arcs, 1LL << 32);
        }
        dg.cw = has_w ? g->cw : unit;
        dg.a = g->a;
        dg.key = fingerprint_key();
        rc = DUPIN_OK;
        if (e == cudaSuccess && dg.cw) rc = launch_init_weights(dg, DUPIN_DW, w, nullptr, nullptr, ctl, true, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, ctl, sizeof(PeelCtl), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        gfree(w, s);
        gfree(ctl, s);
        gfree(unit, s);
        if (e != cudaSuccess || rc) {
            int r2 = rc ? rc : dupin_cuda_fail(e, "graph validation");
            graph_release(g);
            gfree(bad, s);
            return r2;
        }
        if (hc.init_overflow) {
            graph_release(g);
            gfree(bad, s);
            if (hc.init_overflow == 2) return dupin_fail(DUPIN_ERR_INVALID_ARG, "negative vertex weight");
            return dupin_fail(has_w ? DUPIN_ERR_OVERFLOW : DUPIN_ERR_INVALID_ARG,
                              "invalid graph: a neighbour id out of range, a self-loop, a negative weight, or a "
                              "peeling weight >= 2^63");
        }
        // sorted rows without repeats, and symmetry: checked in the same pass
        // (k_init_arcs with its checks on), read here once the ids are known valid
        if (arcs > 0 && (hc.check_unsorted || hc.check_fp)) {
            graph_release(g);
            gfree(bad, s);
            if (hc.check_unsorted)
                return dupin_fail(DUPIN_ERR_INVALID_ARG, "invalid graph: a row's neighbour ids are not strictly "
                                                         "increasing (unsorted, or a repeated pair)");
            return dupin_fail(DUPIN_ERR_INVALID_ARG,
                              bip ? "invalid graph: the CSC does not hold the CSR's edges with the same weights"
                                  : "invalid graph: the CSR is not symmetric (an arc without a reverse arc of "
                                    "equal weight)");
        }
    }
#undef TRY
    gfree(bad, s);
    rc = select_hubs(g, grid, s);
    if (rc) {
        graph_release(g);
        return rc;
    }
    *out = g;
    return DUPIN_OK;
}

extern "C" int dupin_graph_free(dupin_graph *g) {
    if (!g) return DUPIN_OK;
    cudaSetDevice(g->device);
    graph_release(g);
    return DUPIN_OK;
}

extern "C" int dupin_graph_info(const dupin_graph *g, int64_t *n, int64_t *m, int64_t *arcs, int64_t *bytes) {
    if (!g) return dupin_fail(DUPIN_ERR_INVALID_ARG, "graph is NULL");
    if (n) *n = g->n;
    if (m) *m = g->m;
    if (arcs) *arcs = g->arcs;
    if (bytes) *bytes = g->bytes + (g->ws ? g->ws->bytes : 0);
    return DUPIN_OK;
}
