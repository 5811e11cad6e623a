/*
 * cbfs.h -- C ABI of the GB300 Cluster-BFS library (libcbfs.so).
 *
 * Cluster-BFS (C-BFS) runs one breadth-first search from a whole cluster S
 * of k <= 64 sources whose pairwise distances are at most d (the paper
 * "Parallel Cluster-BFS and Applications to Shortest Paths", Section 3).
 * For every vertex v it returns the cluster distance vector
 * <S_v[0..d], Delta_v> of Section 3.1:
 *   Delta_v  = min over s in S of delta(s, v),
 *   S_v[i]   = { s in S : delta(s, v) = Delta_v + i },  i = 0..d,
 * with each subset stored as a 64-bit word, bit j standing for S[j]
 * (least significant bit = S[0]).  By Corollary 1 the d+1 subsets cover S
 * for every reachable v, so only S_v[0..d-1] are stored; S_v[d] is
 * ALL & ~(S_v[0] | ... | S_v[d-1]) when Delta_v is finite (ALL = the k low
 * bits) and empty otherwise.
 *
 * Output format (caller-allocated device memory; the library never
 * allocates outputs):
 *   dist  uint8_t [n]      Delta_v, 0xFF when no source reaches v;
 *   masks uint64_t[d][n]   masks[i*n + v] = S_v[i]   (d = 0: may be NULL).
 * Batched calls use [C][n] and [C][d][n] with cluster c at offset c*n and
 * c*d*n.
 *
 * Conventions for every entry point:
 *   - device pointers unless the name starts with host_;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default);
 *   - return value: CBFS_OK (0) or a negative CBFS_E_* status; on error no
 *     output is partially valid;
 *   - the graph is undirected: off/adj hold both arc directions.
 * Stream ordering: the traversal calls with device outputs (cbfs_run,
 * cbfs_run_batched), the label append and the queries only enqueue work on
 * `stream` and return; their outputs are complete when the stream reaches
 * that point.  Argument errors are returned at once.  Errors the kernels
 * detect (CBFS_E_DIAMETER, CBFS_E_DEPTH, an out-of-range query id) are kept
 * in a status word of the handle or label store -- the first one sticks --
 * and returned by cbfs_sync_status(stream), or by the next call on the same
 * handle that blocks; the outputs of a call that hit such an error are not
 * valid.  Traversal calls with host outputs or a label store, host-driven
 * rounds (cbfs_tune_t.host_loop) or kernel timing (cbfs_profile) block and
 * return those errors themselves.
 * The library is not thread-safe per handle: calls on one handle must not
 * overlap in time on the host, and since a handle's scratch, class lists and
 * staging buffers are reused by every call, calls on one handle should use
 * one stream (or be ordered between streams by the caller).  Outputs of the
 * traversal calls may also be host memory (see cbfs_run_batched).
 */
#ifndef CBFS_H
#define CBFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    CBFS_OK = 0,
    CBFS_E_INVALID = -1,  /* bad argument: null pointer, k not in [1,64], d not in
                             [0,15], source out of range, duplicate source in a cluster */
    CBFS_E_DIAMETER = -2, /* some vertex saw sources spread more than d rounds apart:
                             the cluster's diameter exceeds d (Corollary 1 violated) */
    CBFS_E_DEPTH = -3,    /* some Delta_v would be >= 255 and does not fit one byte
                             (Section 3.1 stores Delta_v in one byte, D < 256) */
    CBFS_E_NOMEM = -4,    /* device or pinned host allocation failed, or a request
                             exceeds the stated memory budget */
    CBFS_E_TIMEOUT = -5,  /* a bounded device-side wait expired */
    CBFS_E_CUDA = -6,     /* a CUDA runtime call failed */
    CBFS_E_GRAPH = -7     /* graph validation failed: offsets not monotone, ids out
                             of range, self loop, unsorted or duplicate neighbours,
                             or a missing reverse arc */
};

typedef struct cbfs_graph_s* cbfs_graph_t;
typedef struct cbfs_labels_s* cbfs_labels_t;

/* Tuning knobs of the traversal.  Zero fields take the library defaults. */
typedef struct cbfs_tune_s {
    /* Direction optimisation (Appendix A, EdgeMap): a round runs dense (pull)
       when |F| + sum_{u in F} deg(u) > pull_alpha * nnz * (clusters in flight);
       < 0 disables pull.  0 = default, per wave: 0.02 when the wave's
       clusters have at most 4 sources each (their pull stops after a few
       frontier neighbours; a plain BFS is k = 1), else 0.08 (the paper's
       commented rule is 1/10). */
    float pull_alpha;
    /* clusters traversed concurrently in one batched wave; rounded down to a
       power of two in 1..8.  0 = default (4). */
    int slots;
    /* the vertex phase scans every vertex instead of the frontier queue when
       |F| * dense_div > n.  0 = default (16); < 0 = never. */
    int dense_div;
    /* != 0: drive the rounds from the host (one launch per kernel, a
       synchronisation every two rounds) instead of one CUDA graph per call
       whose rounds loop on the device (conditional WHILE nodes).  Calls with
       kernel timing enabled (cbfs_profile) always use the host loop. */
    int host_loop;
    /* degree classes of the dense edge phase: one thread per vertex of degree
       <= small_deg (1..32, rounded down to a power of two), one warp per
       vertex of degree <= mid_deg (small_deg..65536), one CTA per 2048-arc
       piece above.  0 = defaults (32, 16384); the autotuner picks them per
       graph. */
    int small_deg;
    int mid_deg;
    /* warp-per-vertex limit for pull rounds whose frontier holds fewer than
       n/32 vertices (lists rarely end early there).  0 or < 0 = use mid_deg
       in every round (the default: other limits were measured no faster). */
    int sparse_mid_deg;
    /* how the clusters of a call with device outputs are grouped into waves:
       0 = by size (sizes descending, ties in call order: the clusters of a
       wave then finish in similar rounds and small ones pull and stop
       early), 1 = in call order.  Host outputs and label stores always use
       call order. */
    int wave_order;
    /* != 0: a pull round also does the vertex phase of the next round for
       the vertices it finishes (their state, output rows and the sources new
       at them, which the next pull gathers), saving a pass over the
       frontier.  Graphs whose clusters' frontiers rarely meet in time (a
       road grid) gain; on power-law graphs the plain pull is faster.  0 (the
       default) = plain; the autotuner tries both. */
    int fused_pull;
    /* waves with fused pulls, and packed waves (see pack): rounds whose new
       sources are recorded, one whole block per vertex and round, and turned
       into the outputs after the wave (each output word written once,
       together with its neighbours), instead of each output word being
       written in the round it becomes known; rounds past the recorded ones
       write directly.  The records take n * slot-words-per-wave * 8 + n / 8
       bytes of device memory per round.  0 = default: as many as fit a
       quarter of the free device memory, at most 96; > 0 = that many (at
       most 255); < 0 = none (and no packing). */
    int stage_rounds;
    /* calls with device outputs: clusters that fill only part of a 64-bit
       slot word share words (largest first, each into the fullest word with
       room, at most 31 to a word), so a wave traverses as many clusters as
       its words hold; each cluster's outputs are read off its bits of the
       round records.  Used when it saves words and round records fit; the
       outputs are the same either way.  Calls with host outputs or a label
       store, and calls with wave_order = 1, keep one cluster per word.
       0 = default (on); < 0 = one cluster per word. */
    int pack;
} cbfs_tune_t;

/* Work counters of one cluster's traversal (Theorem 1). */
typedef struct cbfs_cluster_stats_s {
    uint64_t frontier_appearances; /* V = sum_i |F_i| */
    uint64_t arcs_scanned;         /* A = sum_i sum_{u in F_i} deg(u) (push model) */
    uint64_t reached_arcs;         /* sum of deg(v) over vertices with finite Delta_v */
    uint64_t rounds;               /* number of non-empty frontiers */
} cbfs_cluster_stats_t;

/*
 * Graph residency.  Copies the CSR (off[n+1], adj[nnz]) into device memory
 * owned by the handle.  off is int64 when off_is_i64 != 0, else int32;
 * adj is int32 vertex ids.  inputs_on_device selects whether off/adj are
 * device or host pointers; the caller keeps ownership of them and may free
 * them when the call returns.  validate != 0 checks the graph (see
 * CBFS_E_GRAPH) on the device before returning.  Offsets that do not start
 * at 0, end at nnz and never decrease always give CBFS_E_GRAPH.  All work
 * after the copies (checks, degree order, relabelled copy) runs on the
 * device.  The traversal runs on an internal copy whose vertices are ordered
 * by degree, highest first, down to degree 32; vertices of degree 1..32
 * follow in power-of-two buckets (32, 16, ..., 2, 1) that keep the caller's
 * order within each bucket, then the isolated ones -- so graphs whose input
 * order has locality (a grid in row-major order) keep most of it.  Outputs
 * are always in the caller's ids.  The call synchronises `stream`.  Limits:
 * 0 <= n < 2^31, 0 <= nnz < 2^40, every degree < 2^31.
 * Problem statement: Section 2 (unweighted graph G = (V, E)).
 */
int cbfs_graph_create(int64_t n, const void* off, int off_is_i64, const int32_t* adj, int64_t nnz,
                      int inputs_on_device, int validate, void* stream, cbfs_graph_t* out);

/* Frees the handle and everything it owns, after the device has finished
 * every call on it.  NULL is accepted.  No paper counterpart: it ends the
 * residency of Section 2's graph G that cbfs_graph_create began. */
int cbfs_graph_destroy(cbfs_graph_t g);

/* n and nnz of the resident graph (host outputs). */
int cbfs_graph_info(cbfs_graph_t g, int64_t* host_n, int64_t* host_nnz);

/*
 * One C-BFS (Algorithm 1, Section 3.2) from the k sources host_sources[0..k)
 * with cluster diameter bound d.  Writes dist[n] and masks[d][n], in device
 * or host memory (see cbfs_run_batched).
 * Sources must be distinct and in [0, n); 1 <= k <= 64; 0 <= d <= 15.  d must
 * bound the pairwise source distances, otherwise CBFS_E_DIAMETER is returned
 * (the library detects the violation rather than producing wrong subsets).
 * With device outputs the call is stream-ordered (see the top of this file):
 * CBFS_E_DIAMETER and CBFS_E_DEPTH then come from cbfs_sync_status(stream).
 * With host outputs it returns when they are complete.  Device scratch is
 * owned by the handle and grown on demand (allocation synchronises the
 * device; a call of the same size or smaller allocates nothing).  The first
 * call of each call shape (clusters per wave, cluster sizes, d) records a
 * CUDA graph of the traversal; later calls of that shape replay it.
 */
int cbfs_run(cbfs_graph_t g, const int32_t* host_sources, int k, int d, uint8_t* dist, uint64_t* masks,
             void* stream);

/*
 * C clusters with one common diameter bound d: cluster c has the sources
 * host_sources_concat[host_cluster_off[c] .. host_cluster_off[c+1]).
 * Outputs dist[C][n], masks[C][d][n].  The clusters are traversed
 * concurrently, several per wave with per-cluster frontiers sharing each
 * round's launches (no paper counterpart: the paper runs clusters one after
 * another, Algorithm "Framework of Landmark Labeling").  tune may be NULL.
 * Same validation, errors and completion rule as cbfs_run.
 *
 * dist and masks may be device memory (written by the kernels) or host
 * memory.  With device memory the call is stream-ordered, like cbfs_run.
 * With host memory every wave's outputs go to a device buffer and are
 * copied out on a second stream while the next wave traverses; pinned
 * memory (cudaHostAlloc / cudaHostRegister) lets the copies overlap,
 * pageable memory is correct but each copy blocks the calling thread; the
 * outputs are complete when the call returns.
 */
int cbfs_run_batched(cbfs_graph_t g, const int32_t* host_sources_concat, const int32_t* host_cluster_off,
                     int C, int d, uint8_t* dist, uint64_t* masks, const cbfs_tune_t* tune, void* stream);

/*
 * cbfs_run_batched that also appends the C clusters, in order, to the label
 * store `labels` (created with this graph's n and the same d): the rows of
 * the landmark labeling (Section 4.2) are written from each wave's outputs
 * while they are still on the device, so building labels costs no second
 * pass over dist/masks.  dist and masks may both be NULL (labels only), or
 * device or host memory as in cbfs_run_batched.  CBFS_E_NOMEM when the
 * store has no room for C more clusters, CBFS_E_INVALID when its n or d
 * differ; on any error the store's count is left as it was.  Always driven
 * from the host (no CUDA-graph replay).
 */
int cbfs_run_batched_labels(cbfs_graph_t g, const int32_t* host_sources_concat, const int32_t* host_cluster_off,
                            int C, int d, uint8_t* dist, uint64_t* masks, cbfs_labels_t labels,
                            const cbfs_tune_t* tune, void* stream);

/*
 * cbfs_run without any allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory -- a process
 * whose GPU memory is entirely held by another allocator (such as a
 * framework's caching pool), or a latency-critical loop where cudaMalloc and
 * cudaFree, which can block and synchronise the device, are not allowed.
 *
 * The caller passes the graph directly (device off int64[n+1] and adj
 * int32[nnz], no handle), the sources on the host and the outputs (device
 * dist[n], masks[d][n]) as for cbfs_run; the results are identical.  The
 * graph is checked on the device before the traversal reads through it:
 * off[0] = 0, off[n] = nnz, offsets that never decrease and ids in [0, n),
 * else CBFS_E_GRAPH (the reads of the check stay inside off[0..n] and
 * adj[0..nnz), so those two sizes must be right).  Symmetry is not checked:
 * a directed CSR gives the C-BFS of its arcs.
 * The traversal's scratch is one fixed array compiled into the library
 * (about 7 MB; every GPU that loads the library keeps it until the process
 * exits), so the sizes are limited: n <= 131072 and nnz <= 4194304, larger
 * graphs return CBFS_E_NOMEM.  The first call on a device looks up the
 * array's device address for that device; make that first call before any
 * stream capture.  All calls share the one array and it keeps the last
 * call's contents (each call clears what must start at zero): calls that
 * overlap on the GPU -- on other streams or from other host threads -- race
 * and corrupt each other's results.  The edge phase runs in push mode only.
 * The call synchronises `stream` (after the graph check, then once per two
 * BFS levels); it calls no cudaMalloc, cudaFree or other allocating routine.
 */
int cbfs_run_noalloc(int64_t n, const int64_t* off, const int32_t* adj, int64_t nnz, const int32_t* host_sources,
                     int k, int d, uint8_t* dist, uint64_t* masks, void* stream);

/*
 * Work counters (Theorem 1) of C clusters computed from their outputs
 * (device dist[C][n], masks[C][d][n], host_ks[C] cluster sizes) on the
 * resident graph g, written to host_out[C].  Each frontier appearance of
 * Algorithm 1 is a pair (v, i) with S_v[i] non-empty, so the counters are a
 * function of the outputs alone.  Synchronises `stream`.  Diagnostic, not on
 * the traversal path.
 */
int cbfs_output_stats(cbfs_graph_t g, const uint8_t* dist, const uint64_t* masks, const int32_t* host_ks,
                      int C, int d, cbfs_cluster_stats_t* host_out, void* stream);

/* Device-time accounting of the traversal kernels of one handle. */
typedef struct cbfs_kernel_times_s {
    /* index 0: wave set-up (seed + source check), 1: vertex phase (phase A),
       2: edge phase (phase B, push or pull) */
    uint64_t launches[3];
    double ms[3]; /* summed CUDA-event durations, milliseconds */
    uint64_t total_launches; /* every kernel the traversal launched */
} cbfs_kernel_times_t;

/*
 * enable != 0 makes later cbfs_run / cbfs_run_batched calls on g bracket each
 * traversal kernel with CUDA events on the call's stream and accumulate the
 * durations; enable == 0 stops that.  host_out (may be NULL) receives the
 * totals accumulated since the previous cbfs_profile call, which resets them.
 * Kernel launch counts are kept even when timing is disabled.
 */
int cbfs_profile(cbfs_graph_t g, int enable, cbfs_kernel_times_t* host_out);

/*
 * Landmark labels (Section 4.2, Algorithm "Framework of Landmark Labeling"):
 * a vertex-major store of the cluster distance vectors of up to C_capacity
 * clusters with common d, in device memory owned by the handle.  The row of
 * vertex v holds, for every stored cluster c: Delta_v(c) (one byte) and
 * S_v[0..d-1](c) (64-bit words); row stride = round_up(C_capacity, 8) +
 * 8 * d * C_capacity bytes.  Fails with CBFS_E_NOMEM when n * stride exceeds
 * hbm_budget_bytes (0 = no budget) or the allocation fails.
 */
int cbfs_labels_create(int64_t n, int C_capacity, int d, size_t hbm_budget_bytes, cbfs_labels_t* out);

/*
 * cbfs_labels_create with w-bit subset words, w in {8, 16, 32, 64}: the
 * store then holds clusters of at most w sources (the word sizes of the
 * paper's landmark-labeling study, Section 5.3), 1 + d * w / 8 bytes per
 * cluster and vertex.  Row layout: [dist C_capacity bytes | pad to 8 |
 * d blocks of round_up(C_capacity * w / 8, 8) bytes].  Appends narrow the
 * C-BFS output words (whose bits at and above the cluster size are zero)
 * and reject clusters larger than w with CBFS_E_INVALID.  w = 64 is
 * cbfs_labels_create.
 */
int cbfs_labels_create_w(int64_t n, int C_capacity, int d, int w, size_t hbm_budget_bytes, cbfs_labels_t* out);
int cbfs_labels_destroy(cbfs_labels_t L);

/*
 * Appends C clusters given in the cluster-major C-BFS output format (device
 * dist[C][n], masks[C][d][n]) with their sizes host_ks[C] (1..64) into the
 * vertex-major rows: the step of Section 4.2's Algorithm "Framework of
 * Landmark Labeling" that stores each cluster's distance vectors in every
 * vertex's label L[v].  CBFS_E_INVALID when the store would exceed
 * C_capacity.  Stream-ordered (asynchronous).
 */
int cbfs_labels_append(cbfs_labels_t L, const uint8_t* dist, const uint64_t* masks, const int32_t* host_ks,
                       int C, void* stream);

/* Forgets every stored cluster (count = 0); the memory stays allocated and
 * later appends overwrite the rows.  Host-side only, no device work. */
int cbfs_labels_reset(cbfs_labels_t L);

/* Number of clusters stored so far (host output). */
int cbfs_labels_count(cbfs_labels_t L, int* host_count);

/* Device pointer to the row store and its stride in bytes (host outputs). */
int cbfs_labels_rows(cbfs_labels_t L, const uint8_t** host_rows, int64_t* host_stride);

/*
 * Distance query of the landmark labeling (Section 4.2, "Answering Queries
 * with Clustered Landmarks"): for each pair (u, v) = (pairs[2t], pairs[2t+1])
 * (device int32), out[t] (device uint16) = min over stored clusters of
 * Delta_u + Delta_v + i + j for the smallest i + j with S_u[i] & S_v[j] != 0
 * (i, j in 0..d, S_d implied), i.e. min over all landmarks s of
 * delta(u, s) + delta(s, v) -- an upper bound of delta(u, v), exact when a
 * landmark lies on a shortest u-v path.  u == v gives 0; no common landmark
 * gives 0xFFFF; a pair with an id outside [0, n) gives 0xFFFF and makes the
 * next cbfs_labels_status return CBFS_E_INVALID.  Stream-ordered
 * (asynchronous); q may be 0.
 */
int cbfs_query_distance(cbfs_labels_t L, const int32_t* pairs, int64_t q, uint16_t* out, void* stream);

/*
 * Distance query with the bounded bidirectional search of Appendix B fused
 * in: for each pair, around u and around v a BFS ball on the resident graph
 * g grows level by level, a level being kept only if the ball (its centre
 * included) then holds at most tau vertices -- the first level that would
 * overflow is dropped whole and that side stops.  The local answer is the
 * minimum over vertices x in both balls of hops(u, x) + hops(x, v) (it is
 * delta(u, v) whenever the balls meet); out[t] = min(local answer, label
 * answer of cbfs_query_distance).  L may be NULL (local search only; no
 * meeting gives 0xFFFF); otherwise its n must be g's.  1 <= tau <= 2048.
 * One CTA per pair with up to 144 KB of shared memory.  Out-of-range ids
 * give 0xFFFF and set the status word of L (or of g when L is NULL).
 * Stream-ordered (asynchronous).
 */
int cbfs_query_local(cbfs_labels_t L, cbfs_graph_t g, const int32_t* pairs, int64_t q, int tau, uint16_t* out,
                     void* stream);

/* Synchronises `stream` and returns (then clears) the label store's device
 * status word: CBFS_OK or CBFS_E_INVALID after an out-of-range query id. */
int cbfs_labels_status(cbfs_labels_t L, void* stream);

/* Synchronises `stream` and returns (then clears) the graph handle's device
 * status word: CBFS_OK or the first error its stream-ordered calls left
 * (CBFS_E_DIAMETER, CBFS_E_DEPTH; CBFS_E_INVALID from a local-search query
 * without labels).  Per handle, where cbfs_sync_status is per stream. */
int cbfs_graph_status(cbfs_graph_t g, void* stream);

/*
 * Synchronises `stream`, then reads and clears the status words of every
 * graph handle and label store that enqueued stream-ordered work on it since
 * the last cbfs_sync_status of that stream, and returns CBFS_OK or the first
 * error found (CBFS_E_DIAMETER, CBFS_E_DEPTH, CBFS_E_INVALID for a bad query
 * id or seed), or CBFS_E_CUDA when the synchronisation itself fails.  The
 * errors are those of Section 3.1's output definition: the distance vector
 * of a vertex is only defined when d bounds the cluster's diameter
 * (Corollary 1) and Delta_v fits the one byte Section 3.1 gives it.
 */
int cbfs_sync_status(void* stream);

/*
 * Distance-query server with continuous batching.  No paper counterpart: it
 * serves the query of Section 4.2 ("Answering Queries with Clustered
 * Landmarks", cbfs_query_distance) to requests that arrive at any time.
 * A native dispatcher thread packs waiting requests, in arrival order, into
 * batches of at most max_batch pairs and launches each on one of `slots`
 * streams of its own (page-locked staging, H2D, the query kernel, D2H) as
 * soon as a slot is free and the batch's device bytes fit the budget; one
 * waiter thread per slot completes requests in the order their batches
 * finish.  Memory: the server allocates its batch buffers at creation
 * (10 bytes per pair: int32 pair + uint16 answer, slots x max_batch pairs)
 * inside device_budget_bytes (0 = a quarter of the device memory free at
 * creation; max_batch shrinks to fit), and admits a batch when the bytes in
 * flight plus its own fit.  The label store must stay alive and unchanged
 * while the server runs.
 *
 * cbfs_server_submit queues host_pairs[q][2] (int32, host memory) and gives
 * a ticket; the answers go to host_out[q] (uint16, host memory).  Both
 * buffers must stay valid until cbfs_server_wait has returned CBFS_OK for
 * the ticket.  cbfs_server_wait blocks until the request is answered
 * (timeout_s < 0: no limit) and releases the ticket, or returns
 * CBFS_E_TIMEOUT and keeps it.  Out-of-range ids answer 0xFFFF and set the
 * label store's status, as in cbfs_query_distance.  cbfs_server_stats
 * fills host_counts[5] = (requests completed, batches, pairs answered,
 * max_batch, budget bytes) and up to `cap` request latencies in
 * milliseconds (arrival at cbfs_server_submit to answers in host_out), in
 * completion order.  cbfs_server_destroy launches what is pending, waits for
 * every batch in flight and frees the server; tickets not yet waited for
 * become invalid.
 */
typedef struct cbfs_server_s* cbfs_server_t;
int cbfs_server_create(cbfs_labels_t L, int64_t max_batch, int slots, size_t device_budget_bytes,
                       cbfs_server_t* out);
int cbfs_server_submit(cbfs_server_t S, const int32_t* host_pairs, int64_t q, uint16_t* host_out,
                       uint64_t* ticket);
int cbfs_server_wait(cbfs_server_t S, uint64_t ticket, double timeout_s);
int cbfs_server_stats(cbfs_server_t S, uint64_t* host_counts, double* host_latency_ms, int64_t cap,
                      int64_t* host_n_latency);
int cbfs_server_destroy(cbfs_server_t S);

/*
 * Page-locked host memory for outputs and inputs (cudaHostAlloc, portable
 * across devices).  No paper counterpart: host outputs of cbfs_run_batched
 * overlap the traversal only from page-locked memory, and buffers pinned
 * by some other allocators were measured to slow those overlapped copies
 * down after earlier large jobs on the machine.  *host_out is NULL on
 * failure (CBFS_E_NOMEM).  cbfs_host_free(NULL) is a no-op.
 */
int cbfs_host_alloc(size_t bytes, void** host_out);
int cbfs_host_free(void* host_ptr);

/* Human-readable name of a status code (static string).  No paper
 * counterpart: it names the codes of this interface. */
const char* cbfs_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* CBFS_H */
