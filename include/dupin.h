/*
 * dupin.h -- C ABI of the GB300 batch-peeling library (libdupin.so).
 *
 * The library finds dense subgraphs by Dupin's parallel batch peeling
 * (arXiv 2504.09311, Algorithm 2, Sec. 4.1) on one NVIDIA GB300 (sm_103a):
 * every round removes all live vertices whose peeling weight is at most
 * k(1+eps) times the current density and keeps the densest prefix.
 *
 * Definitions (Sec. 2.1, Eq. 1 and Sec. 2.2):
 *   f(S)    = sum_{u in S} a_u + sum_{(u,v) in E[S]} c_uv
 *   g(S)    = f(S) / |S|
 *   w_u(S)  = a_u + sum_{v in N(u) cap S} c_uv   (the drop of f when u leaves S)
 * Metrics (Sec. 2.1): DUPIN_DG uses a = 0, c = 1 (supplied weights ignored);
 * DUPIN_DW and DUPIN_FD use the supplied a and c (FD's c_e = 1/log(x + 5)
 * with x the object vertex's degree is computed by the caller, as the
 * paper's ESusp plug-in does in Listing 1).
 *
 * Numbers: every weight is Q32.32 fixed point in an int64 (value * 2^32),
 * non-negative (Property 3.1).  f is kept exactly in 128 bits.  The round
 * threshold is the exact integer floor(k (D+N) f / (D |S|)) for eps = N/D,
 * so the per-round removal sets, the density trace and the best subgraph are
 * fully determined and reproducible bit for bit.
 *
 * Readings of points the paper leaves open:
 *   - k = k_mult (Algorithm 2 uses k = 2 for DG/DW/FD; k_mult = 1 gives the
 *     (1+eps) g threshold).  If a round's threshold selects no vertex (only
 *     possible when k(1+eps) < 2), every live vertex of minimum peeling
 *     weight is removed instead, which keeps Thm 4.3's 2(1+eps) bound.
 *   - Candidates for the best set are S_0 .. S_{R-1} (non-empty); ties keep
 *     the earliest round (Algorithm 1's strict ">").
 *   - DUPIN_GPO adds Algorithm 3's global threshold tau_max.
 *   - DUPIN_LPO adds Algorithm 4's local trims: after every round, while some
 *     live w_u < g(S), a trim round removes {u : w_u < max(tau_max, g(S))};
 *     each trim is a round of its own (peel_round, trace, best candidate).
 *
 * Conventions for every function:
 *   - returns DUPIN_OK (0) or a negative DUPIN_ERR_* code and never throws;
 *     dupin_last_error() gives the calling thread's last message;
 *   - 'stream' is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream); work is ordered on it;
 *   - host pointers are read (or written) only during the call; the library
 *     never keeps a caller pointer after returning.
 */
#ifndef DUPIN_H
#define DUPIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ error codes */
#define DUPIN_OK 0
#define DUPIN_ERR_INVALID_ARG -1    /* bad CSR, id out of range, negative weight, bad eps/k */
#define DUPIN_ERR_OVERFLOW -2       /* some initial peeling weight does not fit in int64 */
#define DUPIN_ERR_OOM -3            /* device memory exhausted (or serving budget) */
#define DUPIN_ERR_BUFFER_TOO_SMALL -4 /* trace_cap < n_rounds + 1 (n_rounds still filled) */
#define DUPIN_ERR_NO_PROGRESS -5    /* max_rounds reached before S became empty */
#define DUPIN_ERR_CUDA -6           /* CUDA runtime error; message has the CUDA text */
#define DUPIN_ERR_TIMEOUT -7        /* an in-kernel wait hit its iteration limit */
#define DUPIN_ERR_NOT_FOUND -8      /* unknown serving ticket */

/* ----------------------------------------------------------------- metrics */
#define DUPIN_DG 0
#define DUPIN_DW 1
#define DUPIN_FD 2
#define DUPIN_TDS 3 /* triangle density (Sec. 2.1): f(S) = triangles of G[S], w_u = those through u;
                       plain counts, not Q32.32 (the paper's k for TDS is 3); dupin_peel only */
#define DUPIN_KCLIDS 4 /* q-clique density kCLiDS (Sec. 2.1): f(S) = q-cliques of G[S], w_u = those
                          through u, q = dupin_params.clique_q (3 .. DUPIN_CLIQUE_MAX_Q; q = 3 gives
                          the same results as DUPIN_TDS); plain counts (the paper's k for kCLiDS is
                          q); dupin_peel only */
#define DUPIN_CLIQUE_MAX_Q 8

/* --------------------------------------------------------- graph loading */

/* dupin_graph_desc.flags */
#define DUPIN_DEVICE_PTRS 1u /* the arrays below are device pointers (still copied) */

typedef struct dupin_graph dupin_graph;

/*
 * A graph is given in one of two forms (Sec. 2.1: V, E, a_i, c_ij):
 *
 *  (a) bipartite users x items: n_left users, n_right > 0 items.  The CSR
 *      (csr_ptr[n_left+1], csr_idx[m] item ids in [0, n_right), csr_w[m])
 *      lists each user's items; the CSC (csc_ptr[n_right+1], csc_idx[m] user
 *      ids in [0, n_left), csc_w[m]) lists each item's users and must hold
 *      the same edge set with the same weights.  Vertex ids of the result are
 *      users [0, n_left) then items [n_left, n_left + n_right).
 *  (b) general undirected: n_right = 0, csr_* is a symmetric CSR over
 *      n_left vertices (each edge in both rows, equal weights), csc_* NULL.
 *
 * csr_w / csc_w may be NULL (all c = 1.0); vertex_w (length n) may be NULL
 * (all a = 0).  The edge set must be simple: no self-loops, no repeated
 * pairs.  Every row lists its neighbour ids in strictly increasing order.
 * Offsets are int64 and start at 0; ids are int32.
 */
typedef struct {
    int64_t n_left, n_right;
    const int64_t *csr_ptr;
    const int32_t *csr_idx;
    const int64_t *csr_w;
    const int64_t *csc_ptr;
    const int32_t *csc_idx;
    const int64_t *csc_w;
    const int64_t *vertex_w;
    uint32_t flags;
} dupin_graph_desc;

/*
 * Copy a graph to the current CUDA device as one symmetric adjacency
 * (int64 row offsets, int32 neighbour ids, int64 Q32.32 arc weights) and
 * validate it on the device: offsets monotone from 0, ids in range, no
 * self-loops, weights >= 0, every initial peeling weight a_u + sum_v c_uv <
 * 2^63, fewer than 2^40 arcs, every row strictly increasing (no repeated
 * pair), and symmetry -- every arc u -> v has the reverse arc v -> u with
 * the same weight; for form (a), the CSC holds exactly the CSR's edges and
 * weights.  Symmetry is checked by comparing a keyed 64-bit fingerprint of
 * the arcs with that of the reversed arcs (the key is drawn once per
 * process), so an asymmetric input is rejected except with probability
 * about 2^-64.  On success *out owns the device copy until
 * dupin_graph_free.  Errors: INVALID_ARG (any check above), OVERFLOW, OOM,
 * CUDA.  Synchronises 'stream'.
 */
int dupin_graph_load(const dupin_graph_desc *desc, void *stream, dupin_graph **out);

/*
 * Release a graph (after all work on it is done; the call waits for the
 * device).  NULL is accepted.  Its arrays return to the library's memory
 * pool and its peeling workspaces are kept, at most 8 per process, for later
 * graphs they fit; dupin_trim_cache() releases both.
 */
int dupin_graph_free(dupin_graph *g);

/* Free the peeling workspaces kept from freed graphs and release the graph
 * memory the library's pool keeps on the current device (see dupin_graph_free). */
int dupin_trim_cache(void);

/* n = vertices, m = undirected edges, arcs = 2m, device_bytes = bytes held. */
int dupin_graph_info(const dupin_graph *g, int64_t *n, int64_t *m, int64_t *arcs, int64_t *device_bytes);

/* ----------------------------------------------------------------- peeling */

/* dupin_params.flags */
#define DUPIN_GPO 1u           /* Algorithm 3: global threshold tau_max (Sec. 5.1) */
#define DUPIN_LPO 2u           /* Algorithm 4: after every round, trim rounds while some
                                  w_u < g(S) (Sec. 5.2); implies DUPIN_GPO */
#define DUPIN_RESULT_DEVICE 8u /* best_mask / peel_round / trace_* are device pointers */
#define DUPIN_TIMING 16u       /* fill the phase_ms[] durations (CUDA events on 'stream') */
#define DUPIN_TAIL_ONE_CTA 32u /* every tail runs in the one-CTA kernel (no cluster tail) */
#define DUPIN_TAIL_CLUSTER 64u /* every tail runs in the cluster kernel (never one CTA) */

typedef struct {
    int32_t metric;     /* DUPIN_DG, DUPIN_DW, DUPIN_FD, DUPIN_TDS or DUPIN_KCLIDS */
    int32_t k_mult;     /* k of Algorithm 2, 1..64 (2 is the paper's value for DG/DW/FD) */
    int64_t eps_num;    /* eps = eps_num / eps_den, eps_num >= 0 */
    int64_t eps_den;    /* 1 .. 2^24 */
    int64_t max_rounds; /* <= 0: n + 1 */
    uint32_t flags;
    int32_t tail_cap;   /* <= 0: automatic; else the live-set size at or below which
                           a tail (one CTA or a cluster) may finish the peel */
    int64_t tail_arc_cap; /* <= 0: automatic (2^16); else, once |S| fits a tail, the
                             tail takes over when the live sub-graph has at most
                             this many arcs (2 |E(S)|) or after a round that removed
                             at most 64 vertices or expanded at most 2^18 arcs (if the
                             sub-graph has at most 2^27 arcs), whichever comes first */
    int32_t clique_q;   /* DUPIN_KCLIDS: the clique size q, 3 .. DUPIN_CLIQUE_MAX_Q;
                           ignored by the other metrics */
} dupin_params;

/*
 * Result of one peel.  Arrays are caller-owned (host memory, or device
 * memory with DUPIN_RESULT_DEVICE); each may be NULL.
 *   best_mask[n]   1 for the vertices of the densest prefix S_best
 *   peel_round[n]  round (1..n_rounds) in which each vertex was removed
 *   trace_*[i]     for i = 0..n_rounds: f(S_i) as (hi, lo) words, |S_i|,
 *                  |U_i| (vertices removed in round i; 0 for i = 0)
 * Scalars (always host): n_rounds R, best_round b (S_b = {u : peel_round[u]
 * > b}), |S_b|, f(S_b) as (hi, lo), g(S_b) as a double (value, not Q32.32),
 * how many rounds used the minimum-weight rule, how many rounds ran in the
 * grid-wide kernel (the rest ran in a tail), the tail's arc count (0 when
 * the grid-wide rounds emptied S), with DUPIN_TIMING the device time of
 * each phase: [0] initial weights, [1] grid-wide rounds, [2] tail sub-graph
 * build, [3] tail rounds; and the CTAs of the tail that ran (1: the one-CTA
 * tail, 8 or 16: the cluster tail, 0: no tail).
 *
 * The tail: once the live set is small, one of two kernels finishes the
 * peel on the live sub-graph -- one CTA with the state in its shared memory
 * (live sets of at most about 14,900 vertices whose sub-graph has at most
 * 2^20 arcs), or a thread-block cluster of 8 or 16 CTAs with the state
 * spread over their shared memory (live sets of up to about 195,000
 * vertices).  Both give identical results; the flags DUPIN_TAIL_ONE_CTA and
 * DUPIN_TAIL_CLUSTER force one of them.
 */
typedef struct {
    uint8_t *best_mask;
    int32_t *peel_round;
    int64_t *trace_f_hi;
    uint64_t *trace_f_lo;
    int64_t *trace_size;
    int64_t *trace_peeled;
    int64_t trace_cap;
    int64_t n_rounds;
    int64_t best_round;
    int64_t best_size;
    int64_t best_f_hi;
    uint64_t best_f_lo;
    double best_density;
    int64_t n_min_rule;
    int64_t n_bulk_rounds;
    int64_t tail_arcs;  /* arcs of the live sub-graph the tail started on */
    float phase_ms[4];
    int64_t tail_ctas;  /* CTAs of the tail that ran: 1, 8 or 16 (0: none) */
} dupin_result;

/*
 * Algorithm 2 (Sec. 4.1) on a loaded graph: rounds i = 1, 2, ... remove
 * U_i = {u in S_{i-1} : w_u(S_{i-1}) <= T_i} (minimum rule if empty) until S
 * is empty; the result names the densest S_i.  Runs on 'stream' and returns
 * when the result is complete.  Errors: INVALID_ARG (params), NO_PROGRESS
 * (max_rounds), BUFFER_TOO_SMALL (trace_cap < n_rounds + 1 with a non-NULL
 * trace; everything else is still filled), OOM, TIMEOUT, CUDA.
 *
 * With metric DUPIN_TDS (DUPIN_KCLIDS), f and the weights are triangle
 * (q-clique) counts, not Q32.32: the trace's f words and best_f hold counts,
 * best_density is f / |S|, the graph's weights are ignored, and each round
 * runs as a few short launches (the graph's cliques are listed once at the
 * start, and every round lists only the cliques through its removed
 * vertices).  The graph's rows must be sorted (the loader checks it); f
 * stays below 2^63 (a count that large could not be listed).  The tail
 * fields of the result are 0.  INVALID_ARG for DUPIN_KCLIDS with clique_q
 * outside 3 .. DUPIN_CLIQUE_MAX_Q.
 */
int dupin_peel(dupin_graph *g, const dupin_params *params, dupin_result *result, void *stream);

/*
 * The hand-over autotuner.  tail_arc_cap decides when the grid-wide rounds
 * hand over to a tail although their last round was large (once |S| fits a
 * tail and 2 |E(S)| <= tail_arc_cap; small rounds hand over regardless).
 * dupin_tune_handover peels 'g' under each of the DUPIN_TUNE_HANDOVER_N
 * candidates 2^16, 2^18, ..., 2^26 (params otherwise as given; results are
 * identical under every candidate, and none is returned), once to warm up
 * and twice more timed on the host, and writes the fastest candidate to
 * *best and each candidate's best time in ms to times_ms[0 ..
 * DUPIN_TUNE_HANDOVER_N - 1] (either may be NULL).  The caller passes the
 * winner as params.tail_arc_cap to later peels of similar graphs.  Errors as
 * dupin_peel; INVALID_ARG for DUPIN_TDS and DUPIN_KCLIDS.
 */
#define DUPIN_TUNE_HANDOVER_N 6
int dupin_tune_handover(dupin_graph *g, const dupin_params *params, void *stream, int64_t *best, float *times_ms);

/*
 * Peel 'count' independent graphs in few launches (one persistent launch
 * for all graphs small enough for one CTA, the single-graph path for the
 * rest).  params and results are arrays of length count; results are
 * identical to 'count' separate dupin_peel calls.  A graph may appear more
 * than once.  Errors as dupin_peel; the first failing index is named in
 * the message.
 */
int dupin_peel_batch(dupin_graph *const *graphs, const dupin_params *params, dupin_result *results,
                     int64_t count, void *stream);

/*
 * Launch shape of the one-CTA-per-graph kernel used by dupin_peel_batch (and
 * by the server) for graphs of at most DUPIN_BATCH_CTA_MAX_N vertices: CTAs of
 * 128 threads (4 per SM) or of 256 threads (2 per SM).  Results do not depend
 * on the shape; only the time does.  The choice is per device and process.
 * By default a launch of at most 2 x (SM count) graphs (one wave of 256-thread
 * CTAs: the GPU is not full, and wider CTAs finish each graph sooner) takes
 * 256 threads and a larger launch 128.
 *
 * dupin_batch_set_threads: threads = 128 or 256 makes every launch on the
 * current device take that shape; 0 restores the default rule; INVALID_ARG
 * otherwise.
 * dupin_batch_get_threads: writes the shape that launches of more than one
 * wave take on the current device to *threads.
 * dupin_batch_tune: the autotuner.  Peels the batch's graphs of at most
 * DUPIN_BATCH_CTA_MAX_N vertices (larger ones are ignored) once per shape to
 * warm up, then twice more per shape, timing each call on the host (the call
 * synchronises 'stream'); the faster shape becomes the one that launches of
 * more than one wave take on the current device (smaller launches keep 256
 * threads), and its thread count is written to *threads (if non-NULL).  No
 * result is returned; the graphs are not changed.  Errors as
 * dupin_peel_batch, the shape then unchanged; INVALID_ARG if no graph of the
 * batch is small enough.
 */
#define DUPIN_BATCH_CTA_MAX_N 131072
int dupin_batch_set_threads(int threads);
int dupin_batch_get_threads(int *threads);
int dupin_batch_tune(dupin_graph *const *graphs, const dupin_params *params, int64_t count, void *stream,
                     int *threads);

/* ------------------------------------------------- peel without allocation */

/*
 * No counterpart in the paper: an entry point for callers that may not
 * allocate device memory once running (services that reserve all GPU memory
 * up front in their own pool, latency-critical loops where cudaMalloc /
 * cudaFree would synchronise the device and stall other work, plug-ins in a
 * process whose allocator owns the device).  It runs the same peel as
 * dupin_peel on a graph of at most DUPIN_NOALLOC_MAX_N vertices given as a
 * symmetric CSR in DEVICE memory (row_ptr[n+1] int64, col_idx[row_ptr[n]]
 * int32, arc_w Q32.32 or NULL for DG, vertex_w or NULL), writes peel_round[n]
 * (device), the scalars of *result, and -- when non-NULL -- result->best_mask
 * and result->trace_* (device pointers, trace_cap entries).  It calls no
 * cudaMalloc, cudaFree or allocating library routine: its working state is
 * one fixed file-scope device array (about 100 KB, held by every GPU that
 * loads the library until exit).  Every call on a device shares that array
 * and it keeps the last call's contents: calls that overlap on the GPU race
 * and must be serialised by the caller.  The first call on a device performs
 * set-up (looks up the array's device address, sets a kernel's shared-memory
 * limit); make it before any stream capture.  Errors: INVALID_ARG (n outside
 * 1..DUPIN_NOALLOC_MAX_N, bad CSR or params), OVERFLOW, NO_PROGRESS,
 * BUFFER_TOO_SMALL, CUDA.  Synchronises 'stream'.
 */
#define DUPIN_NOALLOC_MAX_N 8192
int dupin_peel_noalloc(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const int64_t *arc_w,
                       const int64_t *vertex_w, const dupin_params *params, int32_t *peel_round,
                       dupin_result *result, void *stream);

/* ----------------------------------------------------------------- serving */

typedef struct dupin_server dupin_server;

typedef struct {
    int64_t memory_budget; /* device bytes the server may hold for per-request state (> 0) */
    int32_t max_slots;     /* requests on the device at once, 1..4096 */
    int32_t device;        /* CUDA device ordinal */
} dupin_serve_config;

typedef struct {
    int64_t submitted, completed, rejected, in_flight, queued;
    double p50_ms, p99_ms;   /* submit -> completion latency over completed requests */
    double graphs_per_s;     /* completed / (last completion - first submit) */
} dupin_serve_stats_t;

/*
 * Continuous-batching server over resident graphs.  submit() queues a peel
 * of 'graph' (which must stay loaded until the ticket completes) and returns
 * at once with a ticket; a worker thread admits queued requests into free
 * slots while the device-memory budget allows, launches them alongside the
 * requests already running, and writes each result into the caller's
 * 'result' (host arrays) when it completes.  poll() reports completion,
 * wait() blocks until it.  Results equal dupin_peel's exactly.
 */
int dupin_serve_create(const dupin_serve_config *cfg, dupin_server **out);
int dupin_serve_submit(dupin_server *s, dupin_graph *graph, const dupin_params *params, dupin_result *result,
                       uint64_t *ticket);
int dupin_serve_poll(dupin_server *s, uint64_t ticket, int *done, int *status);
int dupin_serve_wait(dupin_server *s, uint64_t ticket, int *status);
int dupin_serve_stats(dupin_server *s, dupin_serve_stats_t *out);
int dupin_serve_destroy(dupin_server *s);

/* ------------------------------------------------------------------- misc */

/* Copy the calling thread's last error message (NUL-terminated) into buf. */
int dupin_last_error(char *buf, size_t cap);

/* Library version as "major.minor.patch". */
const char *dupin_version(void);

/*
 * sizeof() of a public struct as this library was compiled, by type name
 * ("dupin_graph_desc", "dupin_params", "dupin_result", "dupin_serve_config",
 * "dupin_serve_stats_t"), so that a binding can check its layouts; -1 for an
 * unknown name or NULL.  Touches no device.
 */
int64_t dupin_struct_size(const char *name);

#ifdef __cplusplus
}
#endif

#endif /* DUPIN_H */
