/*
 * mincut.h -- C ABI of the GB300 exact minimum-cut library (libmincut.so).
 *
 * Problem (Sec. 2, "Basic Concepts"): G = (V, E, c) undirected with
 * non-negative integer edge weights.  A cut (A, V \ A) splits V into two
 * non-empty sides; its capacity is the total weight of the edges between
 * them; lambda(G) is the smallest capacity.  The library computes lambda(G)
 * exactly with the contraction rounds of Sec. 2.1 / Algorithm 2: bounds from
 * vertex degrees (trivial and collapsed-vertex cuts) and label propagation,
 * edge marking by the Padberg-Rinaldi tests and by concurrent CAPFOREST
 * passes (Algorithm 1), union-find over the marked edges and CSR contraction,
 * until the graph is trivial or the bound is proven.  All arithmetic is exact
 * integer: int32 input weights, int64 cut values.
 *
 * Conventions shared by every call
 *   - Graph input: a symmetric CSR.  row_ptr int64[n+1] (row_ptr[0] = 0,
 *     non-decreasing), col int32[M] with values in [0, n), w int32[M] >= 0.
 *     Every undirected edge {u, v} appears in row u and in row v with the same
 *     total weight.  Rows need not be sorted; duplicate entries are summed,
 *     self-loops and zero weights are dropped.
 *   - Streams: every call is ordered on the CUDA stream given at graph
 *     creation and returns after that stream's work for the call finished.
 *   - Ownership: the library copies inputs; callers own every buffer they
 *     pass; the library owns a graph's device memory until
 *     mincut_graph_destroy().
 *   - Errors: every int-returning call returns a mincut_status; on error
 *     mincut_last_error() gives a per-thread message.  Calls on distinct
 *     graphs are thread-safe; calls on one graph must not overlap.
 *   - Device waits inside kernels are bounded; a wait that runs out sets an
 *     error status (MINCUT_ERR_DEVICE_TIMEOUT) instead of hanging.
 */
#ifndef MINCUT_H
#define MINCUT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MINCUT_OK = 0,
    MINCUT_ERR_INVALID = -1,        /* bad argument or malformed graph */
    MINCUT_ERR_OOM = -2,            /* device allocation failed */
    MINCUT_ERR_OVERFLOW = -3,       /* a size or sum exceeds the supported range */
    MINCUT_ERR_DEVICE_TIMEOUT = -4, /* a bounded device wait ran out */
    MINCUT_ERR_CUDA = -5,           /* a CUDA runtime call failed */
    MINCUT_ERR_INTERNAL = -6        /* an internal consistency check failed */
} mincut_status;

/* flags of mincut_graph_from_csr */
#define MINCUT_HOST_PTRS 0u      /* row_ptr/col/w are host pointers */
#define MINCUT_DEVICE_PTRS 1u    /* row_ptr/col/w are device pointers */
#define MINCUT_SKIP_VALIDATE 2u  /* caller guarantees symmetry; skip that check */

/* Device allocator used for all of a graph's device memory.  alloc returns a
 * device pointer of at least `bytes` (256-byte aligned) or NULL; free releases
 * it.  Both are called on the host thread that makes the library call, with
 * the graph's stream.  NULL allocator: stream-ordered allocations from a pool
 * per device owned by the library (see mincut_release_cached). */
typedef struct mincut_allocator {
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void (*free)(void* ptr, size_t bytes, void* stream, void* ctx);
    void* ctx;
} mincut_allocator;

typedef struct mincut_graph mincut_graph; /* opaque, device-resident */

/* Options of a full solve.  mincut_default_options() fills the defaults. */
typedef struct mincut_options {
    int32_t lp_iters;        /* label-propagation sweeps per bound (default 2; 0 = off) */
    int32_t lp_min_n;        /* run LP only on graphs with n >= lp_min_n (default 10000) */
    int32_t lp_every_round;  /* 0: LP bound in the first round only (default, the paper's
                                once-per-solve bound); 1: in every round */
    uint32_t pr_mask;        /* PR1..PR4 as bits 0..3 (default 0xF) */
    int64_t pr_budget;       /* PR3/PR4 only if min(|N(u)|,|N(v)|) <= budget (default 16; <0 = all) */
    int32_t passes;          /* concurrent CAPFOREST passes per wave (0 = auto) */
    int32_t pass_table;      /* per-pass table slots, power of two in [256, 2048] (0 = auto) */
    int32_t waves;           /* CAPFOREST waves per round (0 = auto) */
    uint64_t seed;           /* start-vertex seed of the concurrent passes */
    int32_t deterministic;   /* 1: one sequential CAPFOREST pass from vertex 0 per round */
    int32_t max_rounds;      /* 0 = unlimited */
    int64_t spin_limit;      /* iteration limit of bounded device waits (0 = default) */
    int32_t profile;         /* 1: time every kernel with CUDA events (mincut_profile_read) */
    int32_t init_bound;      /* 0: bounds inside the rounds only (default); 1: first run the
                                coarsening heuristic of Sec. 2.1 "Lowering the upper bound"
                                (label-propagation clusters contracted, PR tests, repeated, then
                                the coarse graph solved exactly) on graphs with n >= lp_min_n */
    int32_t cf_visit;        /* visit array of the concurrent CAPFOREST passes (Sec. 4, parallel
                                session (1)): 0 shared (default), 1 private to each pass,
                                2 alternate over the first two rounds and keep the faster */
    int32_t seq_passes;      /* passes of the sequential CAPFOREST a round runs when the
                                concurrent passes mark nothing, each a whole pass from its own
                                start vertex with private arrays: 1 = the single pass of
                                Algorithm 2; 0 = auto (one per SM, device memory permitting) */
    int32_t batch_small_n;   /* mincut_batch_solve: graphs of at most this many vertices (and at
                                most 2048) are solved one per warp, each running all its rounds
                                alone (one CAPFOREST pass per round; of pr_mask only PR1/PR2);
                                the others share the batch's round kernels.  0 = auto (chosen
                                by timing candidate thresholds on the first solve of the batch,
                                then kept); < 0 = every graph in the round kernels */
    int32_t seq_kernel;      /* kernel of the whole-graph CAPFOREST passes: 0 (default) one
                                warp per pass, the next vertex among those of highest priority
                                taken from the last scanned row when it holds one (else the
                                smaller id), keys in 1, 2 or 4 bytes as the bound requires, as
                                many passes as keep their arrays within a share of L2 (or
                                seq_passes); 1 one thread block per pass, ties to the smaller
                                id.  Bounds of 2^32 - 1 and more always use 1. */
} mincut_options;

/* Statistics of a solve (all optional to read). */
typedef struct mincut_stats {
    int64_t n_input, m_input;    /* canonical input: vertices, undirected edges */
    int32_t rounds;              /* contraction rounds run */
    int32_t seq_passes;          /* rounds that needed the sequential CAPFOREST pass */
    int64_t marks_pr;            /* edges marked by PR1..PR4 over all rounds */
    int64_t marks_cf;            /* edges marked by CAPFOREST over all rounds */
    int64_t entries_processed;   /* sum over rounds of the round graph's directed entries */
    int32_t lambda_source;       /* 1 degree, 2 label propagation, 3 CAPFOREST alpha,
                                    4 coarsening heuristic (init_bound = 1) */
    int32_t kernel_launches;     /* kernels launched by the solve */
    double ms_total;             /* host wall time of the solve */
} mincut_stats;

/* One round, for testing and for callers that drive the loop themselves.
 * Zero-initialise, then set what you need (mincut_default_round_options()). */
typedef struct mincut_round_options {
    int64_t lambda_in;       /* carried-in upper bound (INT64_MAX: none) */
    int32_t lp_iters, lp_min_n;
    uint32_t pr_mask;
    int64_t pr_budget;
    int32_t capforest;       /* 0 none; 1 concurrent passes (+ sequential pass if no
                                marks); 2 one sequential pass from cf_start, ties to the
                                smaller vertex id; 3 as 1 with visit sets private to each
                                pass; 4 one sequential pass from cf_start driven by one warp,
                                ties to the first vertex of the last scanned row that holds
                                the highest priority, else the smaller id */
    int32_t cf_start;
    int32_t passes, pass_table, waves;
    uint64_t seed;
    /* optional external marking (host pointers; replaces all marking):   */
    const int32_t* groups;   /* [n] group id in [0, n) per vertex: contract each group */
    int64_t npairs;          /* or: contract the components of these pairs */
    const int32_t* pair_u;
    const int32_t* pair_v;
    /* optional outputs (host pointers, sized for the round's input graph): */
    uint8_t* pr_flags_out;   /* [M] PR flags (bit0..3 = PR1..PR4) per directed entry */
    int32_t* cf_order_out;   /* [n] visit order of the sequential pass (capforest 2 or 4) */
    int32_t* cf_marks_out;   /* [2*cf_marks_cap] marked pairs (x, y) of that pass, in scan
                                order */
    int64_t cf_marks_cap;
    int32_t* lp_labels_out;  /* [n] labels after the LP sweeps (when LP ran) */
} mincut_round_options;

typedef struct mincut_round_result {
    int64_t n_in, m_in;      /* round input: vertices, directed entries */
    int64_t n_out, m_out;    /* contracted graph */
    int64_t lambda_out;      /* bound after the round */
    int64_t marks_pr, marks_cf;
    int32_t stopped;         /* 1: n <= 2 or bound 0 after the degree bound (no contraction) */
    int32_t seq_pass;        /* 1: the sequential CAPFOREST pass ran */
    int64_t cf_nscanned;     /* vertices visited by the sequential pass */
    int64_t cf_nmarks;       /* marks of the sequential pass */
} mincut_round_result;

void mincut_default_options(mincut_options* o);
void mincut_default_round_options(mincut_round_options* ro);

/* Build a device graph from a CSR (Sec. 2, G = (V, E, c)).  The graph is
 * validated (indices in range, weights >= 0, symmetric unless
 * MINCUT_SKIP_VALIDATE) and brought to canonical form: rows sorted, duplicates
 * summed, self-loops and zero weights dropped.  n >= 2 (a cut needs two
 * non-empty sides, Sec. 2) else MINCUT_ERR_INVALID.  cuda_stream is a
 * cudaStream_t (NULL: the legacy default stream).  On success *out owns the
 * graph.  Host col / w arrays in pinned (page-locked, mapped) memory are read
 * in place by the device; pageable ones are copied first.  The caller's
 * arrays are not referenced after the call returns.  Symmetry of an input
 * already in canonical form is checked by a 128-bit fingerprint of its edge
 * triples (an asymmetric input passes only on a collision); other inputs are
 * checked exactly after canonicalisation.  Sizes: n <= 2^31 - 2 and
 * M = row_ptr[n] <= 2^31 - 1 (MINCUT_ERR_OVERFLOW beyond, before any device
 * work); in practice device memory bounds them first (about 208 bytes per
 * vertex and 126 per entry, mincut_graph_footprint). */
int mincut_graph_from_csr(int64_t n, const int64_t* row_ptr, const int32_t* col,
                          const int32_t* w, uint32_t flags, void* cuda_stream,
                          const mincut_allocator* alloc, mincut_graph** out);

/* Exact minimum cut (Algorithm 2 with the round of Sec. 2.1).  *cut_value =
 * lambda(G).  side_bitmap (nullable; host or device memory, ceil(n/64)
 * words): bit v (word v/64, bit v%64) is 1 iff vertex v is on the side of a
 * minimum cut that does not contain vertex 0; both sides are non-empty.
 * stats is nullable.  Starts from the input graph (solve does not consume
 * the rounds run by mincut_contract_round). */
int mincut_solve(mincut_graph* g, const mincut_options* opts, int64_t* cut_value,
                 uint64_t* side_bitmap, mincut_stats* stats);

/* Run one contraction round on the graph's current state and replace it by
 * the contracted graph (Algorithm 2, one loop iteration; Algorithm 1 for the
 * CAPFOREST marking).  With ro->groups or ro->pair_u/pair_v set, only the
 * contraction runs, with that marking.  res is required. */
int mincut_contract_round(mincut_graph* g, const mincut_round_options* ro,
                          mincut_round_result* res);

/* Size of the graph's current state: vertices and directed CSR entries. */
int mincut_graph_info(const mincut_graph* g, int64_t* n, int64_t* m_directed);

/* Copy the current canonical CSR to host buffers sized by mincut_graph_info:
 * row_ptr[n+1], col[M], w[M] (weights widened to int64). */
int mincut_graph_export_csr(const mincut_graph* g, int64_t* row_ptr, int32_t* col,
                            int64_t* w);

/* Return the current state to the canonical input graph. */
int mincut_graph_reset(mincut_graph* g);

/* Release a graph and its device memory (NULL is ignored). */
void mincut_graph_destroy(mincut_graph* g);

/* Packed batch of independent graphs (many small solves at once).  Graph i
 * owns the vertices [vertex_offsets[i], vertex_offsets[i+1]) of one CSR over
 * all vertices (vertex_offsets: host int64[num_graphs+1], vertex_offsets[0] =
 * 0, every graph at least 2 vertices); no edge may join two graphs
 * (MINCUT_ERR_INVALID).  Other arguments as mincut_graph_from_csr; the total
 * weight must stay below 2^31 (MINCUT_ERR_OVERFLOW).  The result is a graph
 * object usable only with mincut_batch_solve / mincut_graph_destroy. */
int mincut_batch_from_csr(int64_t num_graphs, const int64_t* vertex_offsets,
                          const int64_t* row_ptr, const int32_t* col, const int32_t* w,
                          uint32_t flags, void* cuda_stream, const mincut_allocator* alloc,
                          mincut_graph** out);

/* Exact minimum cut of every graph of a batch (Algorithm 2 per graph; label
 * propagation is not used).  Graphs of at most opts->batch_small_n vertices
 * are solved one per warp in one persistent launch (a work queue, largest
 * first); the others share one set of round kernels, each graph with its own
 * bound, stop test and witness.  cut_values: host int64[num_graphs].  side_bitmap (nullable, host or device, ceil(n/64)
 * words): bit v = 1 iff vertex v is on the side of its graph's minimum cut
 * that does not hold the graph's first vertex.  When every graph takes the
 * one-warp solver and profiling is off, the second solve of the batch with
 * the same split captures that solve's launches as a CUDA graph (on a stream
 * the library creates) and later solves replay it on the batch's stream;
 * both are released by mincut_graph_destroy. */
int mincut_batch_solve(mincut_graph* g, const mincut_options* opts, int64_t* cut_values,
                       uint64_t* side_bitmap, mincut_stats* stats);

/* How the last mincut_batch_solve split the batch: *small_n = the vertex
 * threshold of the one-warp-per-graph solver it used (the timed choice when
 * opts->batch_small_n was 0; -1 before any solve), *small_graphs = the graphs
 * it solved that way.  MINCUT_ERR_INVALID if g is not a batch. */
int mincut_batch_info(const mincut_graph* g, int32_t* small_n, int64_t* small_graphs);

/* Per-kernel-category timing collected by solves run with opts->profile = 1
 * (CUDA events recorded on the graph's stream around each launch).  Fills up
 * to `cap` entries (out may be NULL to count), sets *count to the number of
 * categories with at least one launch; reset != 0 clears the totals.
 * `units` is the work each launch was given (directed entries for the edge
 * kernels, vertices for the vertex kernels). */
typedef struct mincut_profile_entry {
    char name[24];
    int64_t launches;
    int64_t units;
    double ms;
} mincut_profile_entry;
int mincut_profile_read(mincut_graph* g, mincut_profile_entry* out, int32_t cap, int32_t* count,
                        int32_t reset);

/* Contraction without device allocation.  The paper has no counterpart: this
 * entry point serves callers that cannot allocate device memory -- a plug-in
 * inside a host application that owns the whole device pool, or a
 * latency-critical loop that cannot afford cudaMalloc's latency and implicit
 * synchronisation.  It contracts a device CSR (row_ptr[n+1], col[M], w[M],
 * M = m_directed = row_ptr[n]; symmetric, weights >= 0, total weight < 2^31)
 * by caller-given labels (labels[v] in [0, n2) names v's contracted vertex)
 * and writes the canonical contracted CSR: row_ptr_out[n2+1], col_out and
 * w_out with capacity M (all device pointers); *m_out (host) gets its number
 * of entries.  Rows are numbered by label, sorted by neighbour, parallel
 * edges summed, self-loops and zero weights dropped -- the same result as
 * mincut_contract_round with groups = labels when the labels are numbered
 * by increasing smallest member.
 * Checked before any other work: row_ptr[0] = 0, row_ptr non-decreasing and
 * row_ptr[n] = m_directed, labels in [0, n2), columns in [0, n), weights
 * >= 0 (MINCUT_ERR_INVALID otherwise), and the sum of the M weights at most
 * 2^31 - 1, so that every contracted weight fits int32
 * (MINCUT_ERR_OVERFLOW otherwise).
 * Limits: n and M at most 262,144 (MINCUT_ERR_OVERFLOW beyond).  All
 * intermediate data lives in one fixed ~7.2 MB device array inside the
 * library, held by every GPU that loads it until the process exits; the
 * library allocates nothing on this path.  The first call on a device looks
 * up that array's device address (cudaGetSymbolAddress); make that first
 * call before any stream capture.  The address is cached per device for the
 * life of the process: do not use this entry point after cudaDeviceReset on
 * that device.  Calls share the array, so calls that
 * overlap on the GPU race: serialise them.  Stream-ordered on cuda_stream;
 * returns after the work finished. */
int mincut_contract_csr_noalloc(int64_t n, const int64_t* row_ptr, const int32_t* col,
                                const int32_t* w, int64_t m_directed, const int32_t* labels,
                                int64_t n2, int64_t* row_ptr_out, int32_t* col_out,
                                int32_t* w_out, int64_t* m_out, void* cuda_stream);

/* Estimated peak device bytes of one graph with n vertices and m_directed
 * CSR entries (creation, a solve with label propagation, total weight below
 * 2^31); used by the server's admission control. */
int64_t mincut_graph_footprint(int64_t n, int64_t m_directed);

/* Graphs created without a user allocator take device memory from a pool per
 * device owned by the library; blocks freed by mincut_graph_destroy stay in
 * the pool for the next graph.  This returns the unused blocks of `device`'s
 * pool to the driver (memory of live graphs is not touched).  The paper has
 * no counterpart: this is memory management of the library.
 * Returns MINCUT_ERR_INVALID for a device index outside [0, 64). */
int mincut_release_cached(int device);

/* ---- Serving: continuous batching of solve requests ------------------------
 * A server owns `workers` device workers, each with its own CUDA stream, so
 * admitted requests run concurrently.  A request is admitted when a worker
 * is free and the summed footprint estimates (mincut_graph_footprint) of the
 * admitted requests stay under hbm_cap_bytes (a request alone is always
 * admitted).  A worker that takes a request with n <= pack_max_n also takes
 * the small requests queued right behind it (up to pack_max_requests and
 * pack_max_vertices) and solves them as one packed batch; larger requests
 * are solved alone.  Values are exact, so a request's value does not depend
 * on what it was solved with. */
typedef struct mincut_server mincut_server;
typedef struct mincut_server_options {
    int32_t workers;            /* default 4 */
    int32_t pack_max_requests;  /* default 256 (1 disables packing) */
    int64_t hbm_cap_bytes;      /* default 60 GiB */
    int64_t pack_max_n;         /* default 4096 */
    int64_t pack_max_vertices;  /* default 2^20 */
    int32_t want_bitmap;        /* keep each request's side bitmap (default 1) */
    int32_t device;             /* CUDA device of the workers (default 0) */
    mincut_options solve;       /* options of every solve */
} mincut_server_options;
typedef struct mincut_server_stats {
    int64_t submitted, completed;
    int64_t packed_batches, packed_requests, single_solves;
    int64_t peak_inflight_bytes, inflight_bytes, queued;
    int32_t peak_inflight, reserved;
} mincut_server_stats;
void mincut_server_default_options(mincut_server_options* o);
int mincut_server_create(const mincut_server_options* opts, mincut_server** out);
/* Queue a request; the host CSR (as for mincut_graph_from_csr with
 * MINCUT_HOST_PTRS) is copied before the call returns.  *request_id names
 * the request in mincut_server_wait. */
int mincut_server_submit(mincut_server* s, int64_t n, const int64_t* row_ptr, const int32_t* col,
                         const int32_t* w, uint64_t* request_id);
/* As mincut_server_submit, but nothing is copied: the server reads the
 * caller's host arrays when a worker takes the request, so they must stay
 * alive and unchanged until mincut_server_wait returns for it.  Pinned
 * (page-locked, mapped) arrays are then read in place by the device, which
 * spares the host both the submit copy and a staging copy. */
int mincut_server_submit_borrowed(mincut_server* s, int64_t n, const int64_t* row_ptr,
                                  const int32_t* col, const int32_t* w, uint64_t* request_id);
/* Block until the request is solved; returns its status and fills the value,
 * the latency from submission to completion (ms) and, if requested and kept,
 * its side bitmap (host, ceil(n/64) words).  The request is then released. */
int mincut_server_wait(mincut_server* s, uint64_t request_id, int64_t* cut_value,
                       double* latency_ms, uint64_t* side_bitmap);
int mincut_server_stats_read(mincut_server* s, mincut_server_stats* out);
/* Finish every queued request, stop the workers and free the server. */
void mincut_server_destroy(mincut_server* s);

/* Static description of a status code. */
const char* mincut_status_string(int status);

/* Message of the last error raised on the calling thread ("" if none). */
const char* mincut_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MINCUT_H */
