/*
 * meerkat.h -- C ABI of the GB300 slab-hash dynamic graph store.
 *
 * The store keeps a directed graph with 32-bit vertex ids and 32-bit edge
 * weights as one hash table per vertex, each bucket a chain of 128-byte
 * slabs (paper, Sec. "Motivation": SlabGraph on SlabHash; Sec. "Memory
 * Management in Meerkat": all head slabs in one allocation, located through an
 * exclusive scan of per-vertex bucket counts).  A slab is 32 four-byte lanes:
 * lanes 2p and 2p+1 (p = 0..14) hold the destination and the weight of one
 * edge (the weighted ConcurrentMap layout), lane 30 is unused and lane 31
 * holds the index of the next slab of the chain.
 *
 * Conventions for every call:
 *  - Pointers named d_* are DEVICE pointers (for example the data_ptr() of a
 *    CUDA tensor) owned by the caller.  The library never frees them and does
 *    not keep them after the call's work has been enqueued.
 *  - `stream` is a cudaStream_t passed as void* (0 = the legacy default
 *    stream).  Work is enqueued on it and the call returns without waiting,
 *    unless its comment says it synchronises.  Results are valid once the
 *    stream has reached that point.
 *  - The library owns the slab pool, the per-list update metadata, the change
 *    log and the state of every incremental algorithm.  One graph must not be
 *    used from two host threads at once.
 *  - Vertex ids must be < V.  0xFFFFFFFF, 0xFFFFFFFE and 0xFFFFFFFD are
 *    reserved (INF/INVALID, EMPTY key, TOMBSTONE key; paper, footnotes on
 *    EMPTY_KEY and TOMBSTONE_KEY), so V <= 0xFFFFFFFD.
 *  - Errors found on the host (null pointer, bad size, unknown handle) are
 *    returned at once and nothing is enqueued.  Errors found on the device
 *    (a vertex id >= V, a weight of 0, an exhausted slab pool, an expired
 *    bounded wait) are recorded in the graph's sticky status word; every later
 *    kernel of that graph then does nothing until mk_last_error() reads and
 *    clears the word.  A batch rejected this way is not applied (an exhausted
 *    pool is the exception: see mk_insert_batch).
 *  - All arithmetic is unsigned integer; results are exact.
 */
#ifndef MEERKAT_H
#define MEERKAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mk_graph mk_graph;
typedef int mk_status;

enum {
    MK_OK = 0,
    MK_ERR_INVALID_ARG = -1,    /* bad argument (host) or bad vertex id / weight (device) */
    MK_ERR_POOL_EXHAUSTED = -2, /* the slab pool had no free slab for an insert */
    MK_ERR_TIMEOUT = -3,        /* a bounded device loop hit its iteration limit */
    MK_ERR_CUDA = -4,           /* a CUDA runtime call failed */
    MK_ERR_NO_MEMORY = -5,      /* a device or host allocation failed */
    MK_ERR_INTERNAL = -6
};

#define MK_NONE 0xFFFFFFFFu       /* INF distance, INVALID parent, null slab */
#define MK_INVALID_LANE 0xFFu     /* update marker: the marked slab is full */

/* Sizing of a new graph.  Zero fields take the defaults noted. */
typedef struct mk_config {
    uint32_t V;                          /* vertices [0, V) */
    uint64_t edge_capacity_hint;         /* expected peak edge count (pool sizing) */
    uint32_t buckets;                    /* buckets of every vertex when d_bucket_per_vertex is NULL (0 = 1) */
    const uint32_t *d_bucket_per_vertex; /* device, V entries >= 1, or NULL */
    uint64_t pool_slabs;                 /* overflow slabs in the pool (0 = from the hint) */
} mk_config;

/* Graph statistics (mk_graph_stats). */
typedef struct mk_stats {
    uint32_t V;
    uint64_t lists;          /* slab lists = head slabs = sum of bucket counts */
    uint64_t pool_slabs;     /* capacity of the overflow pool */
    uint64_t pool_used;      /* pool slabs marked allocated in the bitmap */
    uint64_t chain_slabs;    /* slabs reachable from the heads (heads included) */
    uint64_t live_edges;     /* valid (dst, weight) pairs */
    uint64_t tombstones;     /* deleted pairs still occupying a lane */
    uint32_t chain_max;      /* longest chain, in slabs */
    double chain_mean;       /* mean chain length, in slabs */
    uint64_t device_bytes;   /* device memory held by the graph */
    uint64_t epoch;          /* number of mk_commit_batch calls so far */
} mk_stats;

/* One line of the optional per-kernel timing (mk_profile_read). */
typedef struct mk_kernel_time {
    char name[48];
    uint64_t launches;
    double total_ms;         /* sum of CUDA-event durations on the launch stream */
} mk_kernel_time;

/* ------------------------------------------------------------------ setup */

/* Per-vertex bucket counts from an initial edge list by the load-factor rule
 * buckets(v) = max(1, ceil(outdeg(v) / (load_factor * 15))) (paper, Sec.
 * "Motivation": a bucket count fixed a priori by the load factor and the
 * number of adjacent vertices).  d_src: n source ids; d_buckets: V outputs.
 * load_factor must be in (0, 1]. */
mk_status mk_bucket_rule(uint32_t V, const uint32_t *d_src, uint64_t n, float load_factor,
                         uint32_t *d_buckets, void *stream);

/* Creates an empty graph: one allocation of sum(buckets) head slabs located
 * by an exclusive scan of the bucket counts (paper, Sec. "Memory Management
 * in Meerkat"), plus a slab pool with an occupancy bitmap.  The pool holds
 * `pool_slabs` slabs, or when 0: edge_capacity_hint / 15 + lists / 8 + 1024
 * rounded up to 32.  Synchronises `stream`.  *out receives the handle. */
mk_status mk_graph_create_ex(const mk_config *cfg, void *stream, mk_graph **out);

/* Same with the arguments of the paper's problem statement:
 * graph_create(V, E, buckets) with an optional per-vertex bucket array. */
mk_status mk_graph_create(uint32_t V, uint64_t edge_capacity_hint, uint32_t buckets,
                          const uint32_t *d_bucket_per_vertex, void *stream, mk_graph **out);

/* Frees every device buffer of the graph after synchronising the device. */
mk_status mk_graph_destroy(mk_graph *g);

/* ---------------------------------------------------------------- updates */

/* Inserts n edges (d_src[i], d_dst[i]) with weight d_w[i] (d_w NULL = weight
 * 1; a weight must be >= 1).  Set semantics (paper, Sec. "Experimental
 * Evaluation", insertion: an edge is stored at the end of its slab list only
 * if it is not already present): an edge already in the graph keeps its
 * weight.  Within the batch the first occurrence of a repeated (src, dst)
 * is the one stored (a hash set of the batch's pairs keeps each pair's
 * first position).  Each tile of 256 edges is sorted and grouped by slab
 * list (source and bucket) in shared memory; one warp handles the edges of
 * one slab list, walks the whole chain once with 128-byte slab loads, claims
 * free pairs with 64-bit atomicCAS and links pool slabs taken from the
 * bitmap allocator.
 * d_inserted (n bytes, nullable): 1 where edge i was stored by this call.
 * If the pool runs out, the status becomes MK_ERR_POOL_EXHAUSTED and the
 * batch is applied partially: exactly the edges flagged 1 were stored.
 * Marks the touched slab lists as updated for the UpdateIterator and records
 * each stored edge <src, dst, weight> in the epoch's inserted-edge log (grown
 * on demand like the staging buffers). */
mk_status mk_insert_batch(mk_graph *g, const uint32_t *d_src, const uint32_t *d_dst, const uint32_t *d_w,
                          uint64_t n, uint8_t *d_inserted, void *stream);

/* mk_insert_batch without any allocation.  The paper has no counterpart:
 * this is a service of this library.  mk_insert_batch grows its staging
 * buffers with cudaMalloc the first time it sees a larger batch (after a
 * cudaStreamSynchronize and cudaFree of the old ones); a caller that must
 * not synchronise or allocate at that point -- a serving loop between
 * requests, or a process whose device memory is owned by another allocator
 * or fixed at start-up -- uses this entry point instead.  Results and flags
 * are identical to mk_insert_batch.
 *  - n <= MK_NOALLOC_MAX_BATCH (65,536); a larger n returns
 *    MK_ERR_INVALID_ARG and enqueues nothing.
 *  - The staging scratch is one fixed 1 MiB device array inside the library
 *    (every GPU that loads the library holds it until the process exits).
 *    The first call on each device (with that device current) is its
 *    set-up: it looks up the array's device address (cudaGetSymbolAddress),
 *    which may make the runtime load the library's device code there, so
 *    make that first call before any stream capture.  The set-up is
 *    repeated if the device's context has changed since (cudaDeviceReset).
 *  - With profiling on (mk_profile_enable) its kernels are counted by
 *    mk_launch_count but not timed: the timing hook creates events and
 *    grows a host list, which this call must not do.
 *  - Every call on a device shares the array; each call clears the part
 *    that must start empty (the hash set) on its stream.  Two calls whose work
 *    overlaps on the GPU (different streams, or different graphs at the same
 *    time) race on it: order them on one stream or with events.
 *  - Calls no cudaMalloc, cudaFree or allocating library routine. */
#define MK_NOALLOC_MAX_BATCH 65536u
mk_status mk_insert_batch_noalloc(mk_graph *g, const uint32_t *d_src, const uint32_t *d_dst, const uint32_t *d_w,
                                  uint64_t n, uint8_t *d_inserted, void *stream);

/* Deletes n edges: a present edge's pair becomes TOMBSTONE (never reused;
 * paper, Sec. "Experimental Evaluation", deletion), an absent edge is a
 * no-op; the first occurrence of a repeated pair is the one that deletes.
 * Staged like mk_insert_batch.  d_deleted (n bytes, nullable):
 * 1 where edge i was removed by this call.  Removed edges enter the graph's
 * change log for the decremental algorithms. */
mk_status mk_delete_batch(mk_graph *g, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                          uint8_t *d_deleted, void *stream);

/* Looks up n edges (paper, Sec. "Experimental Evaluation", query: hash to one
 * bucket, walk its chain).  d_bitmap (ceil(n/32) words, required): bit i%32 of
 * word i/32 is 1 iff edge i is present.  d_w (n words, nullable): the stored
 * weight, or 0 when absent.  Queries are independent and unsorted; one
 * group of 4 or 8 lanes (the tuned shape) with 16-byte loads walks one
 * query's chain. */
mk_status mk_query_batch(mk_graph *g, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                         uint32_t *d_bitmap, uint32_t *d_w, void *stream);

/* Closes the current update epoch: runs UpdateSlabPointers (paper, Sec.
 * "Graph Primitives", Fig. "UpdateSlabPointers()") on every updated slab
 * list -- its marker moves to the first free lane of its last slab (or to
 * MK_INVALID_LANE when that slab is full) and its updated flag is cleared --
 * and empties the change log.  Incremental algorithm states that have seen
 * every batch of the epoch stay incremental; the others recompute statically
 * at their next call. */
mk_status mk_commit_batch(mk_graph *g, void *stream);

/* ----------------------------------------------- batching and autotuning */
/*
 * Batched execution (a project addition; the paper launches one kernel per
 * batch and reads the frontier size on the host every round).
 */

/* One query request: n edges, outputs as in mk_query_batch (device
 * pointers; d_w nullable). */
typedef struct mk_query_req {
    const uint32_t *d_src;
    const uint32_t *d_dst;
    uint64_t n;
    uint32_t *d_bitmap;
    uint32_t *d_w;
} mk_query_req;

/* Answers every request of the host array h_reqs in ONE persistent launch
 * (results identical to one mk_query_batch per request).  The descriptors
 * are copied to the device before the call returns. */
mk_status mk_query_multi(mk_graph *g, const mk_query_req *h_reqs, uint32_t nreq, void *stream);

/* One update request of mk_update_multi. */
typedef struct mk_update_req {
    int kind;               /* MK_REQ_INSERT or MK_REQ_DELETE (serving request kinds, below) */
    const uint32_t *d_src;  /* n edges (device) */
    const uint32_t *d_dst;
    const uint32_t *d_w;    /* insert weights (nullable = weight 1); ignored by a delete */
    uint64_t n;
    uint8_t *d_flags;       /* nullable: n flags as in mk_insert_batch / mk_delete_batch */
} mk_update_req;

/* Applies the host array of update requests in order, with results, flags
 * and change log identical to one mk_insert_batch / mk_delete_batch call per
 * request.  Each run of consecutive requests of one kind is merged into one
 * batch: one gather launch copies the run's edges into a contiguous staging
 * array (in request order, so the first occurrence of a repeated pair is
 * still the one applied, which is what applying the requests one after
 * another gives), one staged insert or delete applies it, and one scatter
 * launch writes each request's flags; a run of one request is applied
 * directly.  So a stream of many small requests costs a few launches per run
 * instead of per request (the paper applies one batch per launch).  The
 * descriptors are copied to the device before the call returns; the staging
 * arrays are stream-ordered allocations (cudaMallocAsync) freed on `stream`.
 * MK_ERR_INVALID_ARG (nothing enqueued) for an unknown kind or a null
 * src/dst with n > 0. */
mk_status mk_update_multi(mk_graph *g, const mk_update_req *h_reqs, uint32_t nreq, void *stream);

/* A batcher captures the multi-request query launch (descriptor copy from
 * pinned memory + kernel) in a CUDA graph once and replays it for every
 * group of requests: mk_batcher_add_query queues a request on the host,
 * mk_batcher_launch enqueues all queued requests as one graph launch on the
 * batcher's private stream, ordered after `stream`'s prior work and before
 * its later work.  max_requests bounds one group.  The graph uses the tuning
 * in force at creation. */
typedef struct mk_batcher mk_batcher;
mk_status mk_batcher_create(mk_graph *g, uint32_t max_requests, mk_batcher **out);
mk_status mk_batcher_destroy(mk_batcher *b);
mk_status mk_batcher_add_query(mk_batcher *b, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                               uint32_t *d_bitmap, uint32_t *d_w);
mk_status mk_batcher_launch(mk_batcher *b, void *stream);

/* Kernel shapes: lanes per slab chain in the query kernels (4, 8, 16 or 32:
 * 32/G words per lane, one vector load each), their block size (128, 256,
 * 512) and the size of the persistent BFS/SSSP round kernel's one block per
 * SM, in units of 256 threads (field rounds_blocks_per_sm; 0 = as large as
 * fits).  Timings (ms) are filled by mk_autotune. */
typedef struct mk_tuning {
    int query_group;
    int query_block;
    int rounds_blocks_per_sm;
    float query_best_ms;
    float rounds_best_ms;
    float query_ms[16];   /* per (group, block) in the order tried */
    float rounds_ms[8];   /* per block size 256 x 1..8 */
} mk_tuning;

/* Autotuner: times the query kernel on the sample (d_src, d_dst, n) for
 * every group x block shape and a static BFS from bfs_source for every
 * blocks-per-SM value, on this graph, and keeps the fastest shapes for this
 * graph (*out receives them and the timings).  Synchronises `stream`.
 * Leaves a valid BFS state for bfs_source. */
mk_status mk_autotune(mk_graph *g, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n, uint32_t bfs_source,
                      void *stream, mk_tuning *out);
mk_status mk_get_tuning(mk_graph *g, mk_tuning *out);
mk_status mk_set_tuning(mk_graph *g, const mk_tuning *t);

/* ---------------------------------------------------------------- serving */
/*
 * Serving engine (a project addition; the paper has no serving layer):
 * continuous batching of mixed requests on one graph.  Requests are queued in
 * arrival order by mk_server_submit and admitted by mk_server_progress while
 * fewer than max_inflight are in flight.  A run of consecutive read requests
 * (queries, BFS/SSSP) is one group: its queries go out as one CUDA-graph
 * replay of the multi-request query kernel, its BFS/SSSP calls on a second
 * stream, overlapping on the device.  A run of consecutive inserts (or
 * deletes) is applied as one mk_update_multi call, up to the next commit
 * point, and is a barrier: it waits for every earlier read and every later
 * read waits for it, so each result equals that of running the requests one
 * at a time in arrival order.  An insert is admitted only if the slab pool
 * has at least n free slabs beyond those its run already claimed (the worst
 * case of one new slab per edge); otherwise it completes with
 * MK_ERR_POOL_EXHAUSTED and changes nothing.  Every commit_every updates
 * (0 = never) the server commits the epoch (mk_commit_batch).
 * Buffers named in a request must stay valid until it completes.
 */
enum { MK_REQ_QUERY = 0, MK_REQ_INSERT = 1, MK_REQ_DELETE = 2, MK_REQ_SSSP = 3, MK_REQ_BFS = 4 };

typedef struct mk_request {
    int kind;               /* MK_REQ_* */
    const uint32_t *d_src;  /* query / insert / delete: n edges (device) */
    const uint32_t *d_dst;
    const uint32_t *d_w;    /* insert weights (nullable = 1) */
    uint64_t n;
    uint32_t source;        /* SSSP / BFS source */
    uint32_t *d_out0;       /* query: bitmap; insert/delete: flags (uint8_t*, nullable); SSSP/BFS: dist */
    uint32_t *d_out1;       /* query: weights (nullable); SSSP/BFS: parent (nullable) */
    uint64_t tag;           /* returned on completion */
} mk_request;

typedef struct mk_server mk_server;
mk_status mk_server_create(mk_graph *g, uint32_t max_inflight, uint32_t commit_every, mk_server **out);
mk_status mk_server_destroy(mk_server *s);
/* Queues one request (host only; nothing is launched). */
mk_status mk_server_submit(mk_server *s, const mk_request *r);
/* Retires finished requests, admits and launches queued ones, and reports up
 * to `cap` completed tags (with their MK_* status, nullable) in completion
 * order.  Never blocks on the device except to re-read the free pool slab
 * count when an insert does not fit the running estimate. */
mk_status mk_server_progress(mk_server *s, uint64_t *done_tags, int *done_status, uint32_t cap, uint32_t *n_done);
/* Requests queued and requests in flight or finished but not yet reported. */
mk_status mk_server_pending(mk_server *s, uint64_t *queued, uint64_t *inflight);

/* ------------------------------------------------------------- algorithms */

/* Single-source shortest paths with uint32 weights (paper, Algorithm "SSSP -
 * Incremental / Decremental").  The first call for `source` runs the static
 * algorithm; later calls update the stored tree from the change log of the
 * current epoch: decremental prologue (invalidate the subtrees below deleted
 * tree edges, then relax every edge from a valid into an invalid vertex),
 * incremental prologue (relax the edges inserted since the last commit: read
 * from the epoch's inserted-edge log when the epoch holds no deletes, the
 * paper's frontier of inserted edges, else found with the UpdateIterator),
 * then frontier rounds until no distance improves.
 * Writes V entries to d_dist (distance, MK_NONE if unreachable) and d_parent
 * (the smallest-id vertex u with dist(u) + w(u,v) = dist(v); the source is
 * its own parent; MK_NONE if unreachable).  Either output may be NULL.  Path
 * lengths must stay below 0xFFFFFFFF. */
mk_status mk_incr_sssp(mk_graph *g, uint32_t source, uint32_t *d_dist, uint32_t *d_parent, void *stream);

/* Breadth-first search: mk_incr_sssp on the unweighted view (every weight
 * read as 1); distances are hop counts.  Separate state from mk_incr_sssp. */
mk_status mk_incr_bfs(mk_graph *g, uint32_t source, uint32_t *d_dist, uint32_t *d_parent, void *stream);

/* Near-Far ordering of the SSSP rounds (an addition to the paper, whose
 * rounds relax every improved vertex's lists at once): with delta > 0, an
 * improvement to a distance at or above the current split distance T puts
 * the vertex on a far pile instead of the next frontier; whenever the
 * frontier holds fewer than 2,048 lists the pile is split at
 * max(T, smallest distance pushed) + delta (the width doubling for each
 * split in a row), the vertices below it joining the frontier.  T starts
 * delta above the smallest source distance of the call's first frontier.  Results are
 * those of the plain rounds (the same fixpoint: shortest distances, smallest
 * tight parents); on graphs of large diameter and weight range fewer
 * vertices are improved more than once.  delta_static applies to the calls
 * that compute from scratch (the first for a source, or after an error),
 * delta_incremental to the others: an incremental call's improvements are
 * spread over the whole distance range, so ordering them costs more splits
 * and can be slower than the plain rounds.  Applies to later mk_incr_sssp
 * calls of this graph (not to BFS, the several-state call or the host-driven
 * fallback); 0 (the default) keeps the plain rounds.  Each SSSP state then
 * holds 12 more bytes per vertex, allocated at its next ordered call. */
mk_status mk_set_sssp_delta(mk_graph *g, uint32_t delta_static, uint32_t delta_incremental);

/* Several BFS/SSSP states of one graph advanced by one call (a service of
 * this library; the paper runs one algorithm per call).  Results are those
 * of one mk_incr_sssp / mk_incr_bfs call per request, but the passes over
 * the change log and over the whole slab array run once for all of them:
 * the incremental prologue walks each updated list once and relaxes its new
 * edges into every state, the decremental relax-into-invalid scan reads each
 * slab once and tests it against every state's invalidated vertices, and the
 * rounds of all states share one cooperative launch and one grid barrier per
 * round (no single-block phase for small frontiers).  Up to MK_MULTI_MAX
 * requests, each MK_REQ_SSSP or MK_REQ_BFS (kinds of the serving section,
 * below) with its source and nullable dist / parent outputs (V words each,
 * device); no two requests may name the same (kind, source).  One request is
 * the same as the single call. */
#define MK_MULTI_MAX 4u
typedef struct mk_algo_req {
    int kind;
    uint32_t source;
    uint32_t *d_dist;
    uint32_t *d_parent;
} mk_algo_req;
mk_status mk_incr_multi(mk_graph *g, const mk_algo_req *h_reqs, uint32_t n, void *stream);

/* Weakly connected components (paper, Sec. "Incremental WCC"): union-find with
 * Union-Async hooking of the larger root under the smaller and full path
 * compression.  The first call, and any call whose epoch holds deletions
 * (the paper has no decremental WCC), runs the static pass over every edge;
 * otherwise only the edges inserted since the last commit are united, read
 * from the epoch's inserted-edge log (or found with the UpdateIterator when
 * an insert of the epoch could not log).  d_label (V words): the smallest vertex id of each
 * vertex's component. */
mk_status mk_incr_wcc(mk_graph *g, uint32_t *d_label, void *stream);

/* ------------------------------------------------------------- analytics */

/* PageRank (paper, Sec. "Dynamic PageRank", Algorithm "Page Rank - Static /
 * Incremental / Decremental", Eq. 1): super-steps PR[v] = (1 - d) / V + d *
 * (sum over live edges u -> v of PR[u] / out(u) + T / V), where T is the
 * rank held by vertices without out-edges (the paper's teleport term), until
 * the L1 distance between two successive rank vectors is <= eps or after
 * max_iter super-steps.  d_pr (V floats, device): with warm_start = 0 the
 * ranks start at 1 / V (static); with warm_start != 0 they start from
 * d_pr's contents (the ranks before the last batch: the incremental and
 * decremental cases); on return d_pr holds the ranks.  Ranks are kept as
 * 64-bit fixed-point values (scale 2^48) and the contributions are pushed
 * along out-edges with integer atomics, so the result does not depend on the
 * order of the atomics; each super-step's rounding is below 2^-48 per term.
 * damping in (0, 1), eps > 0, max_iter >= 1.  *h_iters / *h_delta
 * (nullable, host): super-steps run and the last L1 delta.  Synchronises
 * `stream` once per super-step (the host reads the delta); work arrays are
 * stream-ordered allocations freed before the call returns. */
mk_status mk_pagerank(mk_graph *g, float *d_pr, int warm_start, float damping, float eps, uint32_t max_iter,
                      uint32_t *h_iters, float *h_delta, void *stream);

/* Triangle counting on undirected graphs stored with both directions of
 * every edge and no self-loops (paper, Sec. "Dynamic Triangle Counting").
 * mk_tc_count is the paper's Count kernel: *d_total (device, one uint64)
 * += sum over the n edges (d_src[i], d_dst[i]) of |N_g1(src) ∩ N_g2(dst)|
 * (the walk goes over the side with fewer buckets; the sum is the same).
 * g1 and g2 must have the same V.  The edges are handed to the warps one
 * at a time from an 8-byte stream-ordered counter allocated for the call. */
mk_status mk_tc_count(mk_graph *g1, mk_graph *g2, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                      unsigned long long *d_total, void *stream);

/* Static count into *h_triangles (host): every triangle once, on its two
 * lower-ranked vertices' edge, the vertices ranked by (bucket count, id);
 * equal to Count(g, g, every live edge) / 6 on a graph that meets the
 * conditions above (which this count does not check).  Synchronises
 * `stream`. */
mk_status mk_tc_static(mk_graph *g, uint64_t *h_triangles, void *stream);

/* Change in the triangle count after a batch (paper, Algorithms "Triangle
 * Counting - Incremental / Decremental", inclusion-exclusion): g_post is the
 * graph after the batch, g_upd a graph holding exactly the batch's edges,
 * and (d_src, d_dst, n) those same edges, both directions of each, every one
 * actually inserted (deletion = 0) or actually deleted (deletion != 0).
 * With S1 = Count(g_post, g_post), S2 = Count(g_post, g_upd) and S3 =
 * Count(g_upd, g_upd) over the batch, *h_delta (host) = S1/2 - S2/2 + S3/6
 * new triangles, or -(S1/2 + S2/2 + S3/6) for a deletion.  Synchronises
 * `stream`.  MK_ERR_INTERNAL if a count is not divisible as the formula
 * requires (the graphs break the stated conditions). */
mk_status mk_tc_update(mk_graph *g_post, mk_graph *g_upd, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                       int deletion, int64_t *h_delta, void *stream);

/* ------------------------------------------------ ConcurrentSet layout */
/*
 * An unweighted graph in the ConcurrentSet layout (paper, Sec. "Motivation":
 * SlabHash's ConcurrentSet beside the ConcurrentMap; the paper keeps the
 * graphs of BFS and WCC this way): each 128-byte slab holds 31 destination
 * keys (lanes 0..30) and the next-slab index (lane 31), about twice the 15
 * pairs of the weighted store's slab, so the slab array and the passes that
 * stream it are about half as large.  The conventions of the weighted store
 * hold (head slabs located by an exclusive scan of per-vertex bucket counts,
 * a bitmap pool, EMPTY / TOMBSTONE keys never reused, set semantics with the
 * first occurrence of a repeated pair applied, device errors in a sticky
 * status word read by mk_set_last_error).  BFS and WCC run statically.
 */
typedef struct mk_set_graph mk_set_graph;
/* Bucket counts max(1, ceil(outdeg / (load_factor * 31))) (V outputs). */
mk_status mk_set_bucket_rule(uint32_t V, const uint32_t *d_src, uint64_t n, float load_factor, uint32_t *d_buckets,
                             void *stream);
/* Creates an empty set graph (every vertex `buckets` buckets, or
 * d_bucket_per_vertex[v]); the pool holds edge_capacity_hint / 31 + lists / 8
 * + 1024 slabs.  Synchronises `stream`. */
mk_status mk_set_create(uint32_t V, uint64_t edge_capacity_hint, uint32_t buckets, const uint32_t *d_bucket_per_vertex,
                        void *stream, mk_set_graph **out);
mk_status mk_set_destroy(mk_set_graph *g);
/* Insert / delete / query n edges as mk_insert_batch / mk_delete_batch /
 * mk_query_batch do (no weights; flags and bitmap nullable / required
 * alike).  A warp walks eight chains at once, one per 4-lane group (32
 * bytes of the slab a lane). */
mk_status mk_set_insert_batch(mk_set_graph *g, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                              uint8_t *d_inserted, void *stream);
mk_status mk_set_delete_batch(mk_set_graph *g, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                              uint8_t *d_deleted, void *stream);
mk_status mk_set_query_batch(mk_set_graph *g, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                             uint32_t *d_bitmap, void *stream);
/* Static BFS from `source`, level by level over a frontier of lists (one
 * warp a list; frontier sizes kept on the device, levels launched six at a
 * time, the host reading the frontier size once per six levels): d_dist =
 * hop counts (MK_NONE unreachable), d_parent = the smallest-id u with a live
 * edge u -> v and dist(u) + 1 = dist(v) (the source its own parent).
 * Synchronises `stream`; allocates two frontiers of `lists` words each from
 * the stream-ordered pool. */
mk_status mk_set_bfs(mk_set_graph *g, uint32_t source, uint32_t *d_dist, uint32_t *d_parent, void *stream);
/* Static WCC: d_label = the smallest vertex id of each vertex's component. */
mk_status mk_set_wcc(mk_set_graph *g, uint32_t *d_label, void *stream);
/* Lists (head slabs), slabs in use (heads + pool slabs claimed) and device
 * bytes held (host outputs, nullable).  Synchronises `stream`. */
mk_status mk_set_stats(mk_set_graph *g, uint64_t *h_lists, uint64_t *h_slabs_in_use, uint64_t *h_device_bytes,
                       void *stream);
/* Synchronises the device, returns the sticky device status and clears it. */
mk_status mk_set_last_error(mk_set_graph *g);

/* -------------------------------------------------------- learned sizing */
/*
 * Learned slab sizing.  The paper fixes each vertex's bucket count a priori
 * from the load factor and its degree (Sec. "Motivation"); this library adds
 * a small MLP, trained on the degree traces of the running graph, that
 * predicts how many edges each vertex will gain so a rebuilt graph can give
 * it enough buckets.  The load-factor rule stays the fallback and the
 * yardstick.
 * Bucket counts change the layout (chain lengths) but never a result.
 *
 * Network: 8 -> 64 (ReLU) -> 64 (ReLU) -> 1, MK_MLP_NPARAMS fp32 master
 * parameters laid out as W1[8][64], b1[64], W2[64][64], b2[64], W3[64], b3.
 * Every pass uses the masters rounded to bf16 (round to nearest even) and
 * accumulates in fp32; loss = mean squared error; Adam on the masters.
 */
#define MK_MLP_NPARAMS 4801
typedef struct mk_mlp mk_mlp;

/* New network with He-uniform weights drawn from `seed`, zero biases. */
mk_status mk_mlp_create(uint64_t seed, mk_mlp **out);
mk_status mk_mlp_destroy(mk_mlp *m);
int mk_mlp_num_params(void);
/* Copy the fp32 master parameters to / from host memory (set also resets
 * the Adam moments). */
mk_status mk_mlp_get_params(mk_mlp *m, float *h_out);
mk_status mk_mlp_set_params(mk_mlp *m, const float *h_in);
/* d_y[i] = network(d_x[8*i .. 8*i+7]) for i < n (device arrays). */
mk_status mk_mlp_forward(mk_mlp *m, const float *d_x, uint64_t n, float *d_y, void *stream);
/* d_grad (device, MK_MLP_NPARAMS floats) = gradient of mean((y - t)^2)
 * over the n samples with respect to the parameters; *d_sse (device double,
 * nullable) = sum of squared errors. */
mk_status mk_mlp_gradient(mk_mlp *m, const float *d_x, const float *d_t, uint64_t n, float *d_grad, double *d_sse,
                          void *stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the n samples. */
mk_status mk_mlp_adam_step(mk_mlp *m, const float *d_x, const float *d_t, uint64_t n, float lr, double *d_sse,
                           void *stream);
/* Degree trace: for every edge i with d_flags[i] != 0 (or every edge when
 * d_flags is NULL), d_out_deg[src] += sign and d_in_deg[dst] += sign
 * (sign = +1 or -1; either output may be NULL). */
mk_status mk_degree_update(uint32_t V, const uint32_t *d_src, const uint32_t *d_dst, const uint8_t *d_flags,
                           uint64_t n, int sign, uint32_t *d_out_deg, uint32_t *d_in_deg, void *stream);
/* Per-vertex features (d_x: V x 8 floats) from out-degree snapshots
 * d_out_hist[k*V + v] = out-degree of v k batches ago (k = 0..4), the
 * in-degree and the current bucket count: log1p(d), log1p(d - d_k) for
 * k = 1..4, log1p(in), log1p(in) - log1p(d), d / (15 * buckets). */
mk_status mk_sizing_features(uint32_t V, const uint32_t *d_out_hist, const uint32_t *d_in_deg,
                             const uint32_t *d_buckets, float *d_x, void *stream);
/* Training targets: d_t[v] = log1p(max(0, later[v] - then[v]) / horizon),
 * the out-edges gained per batch between two degree snapshots. */
mk_status mk_sizing_targets(uint32_t V, const uint32_t *d_deg_then, const uint32_t *d_deg_later, float horizon,
                            float *d_t, void *stream);
/* Bucket counts from the network: y = net(x) is log1p of the predicted edges
 * gained per batch; buckets = clamp(ceil((deg + horizon * expm1(max(y, 0)))
 * / (load_factor * 15)), 1, max_buckets).  d_y receives y (V floats). */
mk_status mk_sizing_buckets(mk_mlp *m, const float *d_x, const uint32_t *d_out_deg, uint32_t V, float horizon,
                            float load_factor, uint32_t max_buckets, float *d_y, uint32_t *d_buckets, void *stream);

/* ------------------------------------------------------------- inspection */

/* Writes up to `cap` live edges sorted by (src, dst) to d_src/d_dst/d_w and
 * the total live edge count to *d_count (device, one uint64). */
mk_status mk_graph_export(mk_graph *g, uint64_t cap, uint32_t *d_src, uint32_t *d_dst, uint32_t *d_w,
                          uint64_t *d_count, void *stream);

/* Fills *out (host memory).  Synchronises `stream`. */
mk_status mk_graph_stats(mk_graph *g, mk_stats *out, void *stream);

/* Free slabs of the pool (an exact device counter kept with the bitmap:
 * one word is read).  Synchronises `stream`. */
mk_status mk_pool_free(mk_graph *g, uint64_t *out, void *stream);

/* Synchronises the device, returns the sticky device status (MK_OK or an
 * MK_ERR_* code) and clears it.  After an error status every incremental
 * BFS/SSSP/WCC state of the graph recomputes statically at its next call
 * (a failed call may have left it half updated). */
mk_status mk_last_error(mk_graph *g);

/* UpdateIterator marker of slab list `bucket` of vertex v (host outputs):
 * *slab = index of the marked slab, *lane = first lane of the new entries in
 * it (MK_INVALID_LANE if the slab was full), *updated = the list's flag.
 * Synchronises `stream`. */
mk_status mk_list_marker(mk_graph *g, uint32_t v, uint32_t bucket, uint32_t *slab, uint32_t *lane,
                         uint32_t *updated, void *stream);

/* Work counters accumulated by the kernels since the last reset, in this
 * order: query slabs loaded, insert slabs loaded, insert slabs linked,
 * delete slabs loaded; BFS/SSSP rounds: relaxed lists, slabs loaded, live
 * edges relaxed, improved vertices; vertices invalidated by deletions; WCC
 * slabs loaded, WCC edges united, commit slabs loaded; BFS/SSSP prologue
 * kernels (inserted-edge and invalidated-target seeds): lists, slabs loaded,
 * live edges relaxed, improved vertices; incremental WCC pass: slabs loaded,
 * edges united; BFS/SSSP rounds and grid barriers of the round kernel;
 * decremental scan: slabs in use copied, slabs relaxed, live edges examined, edges
 * into invalidated vertices, invalidated vertices given a finite distance;
 * vertices visited by the invalidation pass; BFS/SSSP tree nodes written to
 * the caller's dist/parent arrays; inserted-edge log entries read by the
 * incremental BFS/SSSP prologue and by the incremental WCC pass (then
 * reserved words up to 32).
 * The BFS/SSSP prologue words above count the inserted-edge prologue only.  Copies up to n
 * (<= 32) values to out (host); reset != 0 zeroes them.  Synchronises
 * `stream`. */
mk_status mk_counters(mk_graph *g, uint64_t *out, int n, int reset, void *stream);

/* Per-kernel timing: when on, every library kernel launch is bracketed by
 * CUDA events on its stream.  mk_profile_read synchronises the device, fills
 * up to `cap` entries of `out` (host) with the totals since the last reset,
 * sets *n_out and resets the totals. */
mk_status mk_profile_enable(mk_graph *g, int on);
mk_status mk_profile_read(mk_graph *g, mk_kernel_time *out, int cap, int *n_out);

/* Number of kernel launches the library has made for this graph since
 * creation (scan and export-sort calls included, counted from their launch
 * plans). */
uint64_t mk_launch_count(mk_graph *g);

/* L2 residency control (a service of this library; the paper has none): an
 * access-policy window on `stream` (cudaStreamAttributeAccessPolicyWindow)
 * that marks one part of the graph as persisting in L2 for the kernels
 * later launched on that stream, with the L2 set-aside of this process's
 * context (cudaLimitPersistingL2CacheSize) sized to the window, at most the
 * device's maximum.  region: MK_L2_VINFO (the per-vertex index, 8 B a
 * vertex), MK_L2_HEADS (the head slabs), MK_L2_POOL (the overflow pool
 * slabs); a window larger than the device's window limit is cut to it, and
 * when it is larger than the set-aside only that share of its lines
 * (hitRatio) persists.  MK_L2_NONE removes the window from `stream`, resets
 * the persisting lines to normal and the set-aside to 0.  Both end with the
 * process's context.  *out (nullable, host): window bytes, hit ratio and the
 * device's maximum set-aside. */
enum { MK_L2_NONE = 0, MK_L2_VINFO = 1, MK_L2_HEADS = 2, MK_L2_POOL = 3 };
typedef struct mk_l2_info {
    uint64_t window_bytes;
    uint64_t max_bytes;
    float hit_ratio;
} mk_l2_info;
mk_status mk_l2_window(mk_graph *g, int region, void *stream, mk_l2_info *out);

/* Test hooks for the failure paths (a service of this library; the paper
 * has none).  knob MK_DEBUG_BARRIER_SPINS: value 0 restores the default
 * poll limit of the BFS/SSSP round kernel's grid barrier (2^24 polls of
 * about 32 ns); value v >= 1 sets it to v - 1 polls, so v = 1 makes a wait
 * give up at once unless every block has arrived: the call then reports
 * MK_ERR_TIMEOUT through mk_last_error.  knob MK_DEBUG_HOST_ROUNDS: value 1
 * runs the rounds with the host-driven fallback (one launch per round, the
 * host reading each frontier size) that is otherwise used only when the
 * cooperative launch is refused; 0 restores the kernel.  Results are the
 * same either way.  After mk_last_error has returned an error status, every
 * incremental algorithm state of the graph recomputes statically at its
 * next call. */
enum { MK_DEBUG_BARRIER_SPINS = 1, MK_DEBUG_HOST_ROUNDS = 2 };
mk_status mk_debug_set(mk_graph *g, int knob, uint64_t value);

/* Library version string. */
const char *mk_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MEERKAT_H */
