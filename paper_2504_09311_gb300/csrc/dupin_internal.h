// dupin_internal.h -- host-side internals of libdupin shared by the .cu files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dupin.h"
#include "dupin_common.cuh"

// error text for the calling thread (dupin_last_error)
void dupin_set_error(const std::string &msg);
int dupin_fail(int code, const std::string &msg);
// CUDA error -> DUPIN_ERR_CUDA with the runtime's text
int dupin_cuda_fail(cudaError_t e, const char *what);
// the per-process key of the symmetry fingerprints (sym_mix)
unsigned long long fingerprint_key();

#define DUPIN_CUDA_TRY(expr)                                   \
    do {                                                       \
        cudaError_t _e = (expr);                               \
        if (_e != cudaSuccess) return dupin_cuda_fail(_e, #expr); \
    } while (0)

// Per-graph peeling workspace (device memory), allocated on first use and
// reused by later peels of the same graph.
struct PeelWorkspace {
    long long n = 0, arcs = 0, tail_cap = 0, tr_cap = 0, tarc_cap = 0;
    int grid = 0;    // blocks of the persistent kernel
    int device = 0;  // where it was allocated
    long long *w = nullptr;
    int *pr = nullptr;
    int *live0 = nullptr, *live1 = nullptr;
    int *stage_id = nullptr;
    long long *stage_start = nullptr, *stage_off = nullptr;
    long long *fstart = nullptr, *fbase = nullptr;
    long long *cstart = nullptr;
    BlockPart *part = nullptr;
    PeelCtl *ctl = nullptr;
    long long *tr_f_hi = nullptr;
    unsigned long long *tr_f_lo = nullptr;
    long long *tr_size = nullptr, *tr_peeled = nullptr;
    int *loc = nullptr;
    long long *tdeg = nullptr, *tlrp = nullptr;
    int *tcnt = nullptr, *tfill = nullptr;
    unsigned *tgrp = nullptr;
    int *tcol = nullptr;
    long long *tcw = nullptr;
    uint8_t *mask = nullptr;
    bool async = false;  // allocated with cudaMallocAsync (freed with cudaFreeAsync)
    // DUPIN_TIMING: init start, init done, grid-wide rounds start and done,
    // build start and done, tail done
    cudaEvent_t ev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    long long bytes = 0;
};

struct dupin_graph {
    int device = 0;
    long long n_left = 0, n_right = 0, n = 0, m = 0, arcs = 0;
    long long *rp = nullptr;
    int *col = nullptr;
    long long *cw = nullptr;
    long long *a = nullptr;
    int *hubs = nullptr;  // hub number -> vertex id (arcs to hubs are stored as -(h + 1))
    int n_hubs = 0;
    long long bytes = 0;
    PeelWorkspace *ws = nullptr;
    std::vector<PeelWorkspace *> ws_more;  // further workspaces for concurrent peels of this graph
};

// The caps of one peel, resolved from its params and the graph: the tail
// takes over once |S| <= tail_cap and 2 |E(S)| <= tail_arcs.
struct PeelPlan {
    long long tail_cap = 0, tail_arcs = 0, max_rounds = 0, tr_cap = 0;
    long long cl_cap = 0;    // cluster tail capacity (0: none)
    long long one_arcs = 0;  // the one-CTA tail's live-arc limit
    long long hcap() const { return tail_cap > cl_cap ? tail_cap : cl_cap; }
};

DevGraph dev_graph(const dupin_graph *g, int metric);
long long workspace_bytes(long long n, long long arcs, bool has_cw, const PeelPlan &plan, int grid);
PeelWorkspace *workspace_create(long long n, long long arcs, bool has_cw, const PeelPlan &plan, bool async,
                                cudaStream_t s, int *rc);
void workspace_free(PeelWorkspace *ws);
void workspace_free(PeelWorkspace *ws, cudaStream_t s);
// a freed graph's workspace: kept for a later graph it fits, or freed
void workspace_release(PeelWorkspace *ws);
// release the freed graph buffers the library's memory pool keeps (current device)
void graph_pool_trim();
int workspace_ensure(dupin_graph *g, const PeelPlan &plan);
// workspace k of graph g (0: the one dupin_peel uses), allocated or grown for plan
PeelWorkspace *workspace_slot(dupin_graph *g, int k, const PeelPlan &plan, int *rc);

// the three steps of dupin_peel: caps from params, kernels on a stream, results
int peel_resolve(const dupin_graph *g, const dupin_params *p, PeelPlan *plan);
int enqueue_peel(const dupin_graph *g, PeelWorkspace *ws, const dupin_params *p, const PeelPlan &plan,
                 cudaStream_t s);
// The stages of one peel: PEEL_INIT = control reset and initial weights,
// PEEL_BULK = the grid-wide rounds (a cooperative launch over the whole GPU),
// PEEL_BUILD = the tail sub-graph, PEEL_TAIL = the one-CTA rounds.
enum { PEEL_INIT = 1, PEEL_BUILD = 2, PEEL_TAIL = 4, PEEL_BULK = 8, PEEL_FRONT = 9, PEEL_ALL = 15 };
// 'init_from' (stage PEEL_INIT only): a workspace whose initial weights for
// the same graph and metric are already computed on this stream and not yet
// changed by its grid-wide rounds; they are copied instead of recomputed.
// 'bulk_grid' (stage PEEL_BULK): blocks of the cooperative launch, 0 = one per
// SM; fewer leave SMs to one-CTA tails that run at the same time.
int enqueue_peel_stages(const dupin_graph *g, PeelWorkspace *ws, const dupin_params *p, const PeelPlan &plan,
                        int stages, cudaStream_t s, const PeelWorkspace *init_from = nullptr, int bulk_grid = 0);
int peel_finish(const dupin_graph *g, PeelWorkspace *ws, const dupin_params *p, dupin_result *r, cudaStream_t s);

// kernels shared by loading and peeling
int launch_init_weights(const DevGraph &dg, int metric, long long *w, int *pr, int *live0, PeelCtl *ctl,
                        bool check, cudaStream_t s);

// batched one-CTA-per-graph peels (batch.cu)
#include <vector>
struct CtaBatch;
long long cta_graph_limit();
long long cta_job_bytes(const dupin_graph *g, const dupin_params *p);
int cta_batch_enqueue(dupin_graph *const *graphs, const dupin_params *params, dupin_result *results,
                      const std::vector<int64_t> &idx, cudaStream_t s, CtaBatch **out);
int cta_batch_finish(CtaBatch *B, cudaStream_t s, std::vector<int> *per_job_status);

// best_mask[u] = (peel_round[u] > best_round) on the device
void launch_mask(const int *pr, long long n, long long best_round, uint8_t *mask, cudaStream_t s);

// a whole peel of a small graph with caller-supplied buffers (no allocation)
int launch_small_graph_peel(const PeelArgs &A, int metric, bool check, cudaStream_t s);

// the cluster tail (cluster.cu): its live-set capacity on the current device,
// its CTAs per cluster, and its launch (the kernel returns at once unless the
// peel's status says the cluster finishes it)
long long cluster_cap_limit();
// records in 'next' whether 'prev' (its grid-wide rounds enqueued on s) went to the cluster tail
void enqueue_note_cluster(const PeelWorkspace *prev, PeelWorkspace *next, cudaStream_t s);
int cluster_ctas();
int launch_cluster_tail(const PeelArgs &A, cudaStream_t s);

// dupin_peel under the clique metrics TDS and kCLiDS (tds.cu)
int tds_peel(dupin_graph *g, const dupin_params *p, dupin_result *r, cudaStream_t s);
inline bool is_clique_metric(int metric) { return metric == DUPIN_TDS || metric == DUPIN_KCLIDS; }

// the largest live set the single-CTA tail accepts, and the default caps
long long tail_cap_limit();
long long tail_cap_default();
#define DUPIN_TAIL_ARCS_DEFAULT (1LL << 16)
int peel_grid_size();
