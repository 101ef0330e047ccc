/*
 * ipg.h — C ABI of the GB300 Pregel superstep library (libipg.so).
 *
 * A Pregel program (Sec. I of the paper) runs in supersteps: every active
 * vertex runs the compute step, sends messages along its out-edges, the
 * messages are combined into each recipient's mailbox (Sec. III), and a vertex
 * that received a message is active in the next superstep.  This library runs
 * the paper's three benchmarks (Sec. VI-C) on one GPU:
 *   PageRank            — pull ("single broadcast", Sec. IV) over the in-edges,
 *                         sum combiner, FP32 ranks;
 *   Hashmin components  — push with a min combiner over the active-vertex list
 *                         ("selection bypass", Sec. VI-C);
 *   SSSP                — push with a min combiner over the active-vertex list.
 *
 * Conventions for every call:
 *   - Graphs are CSR: the out-edges of vertex u are columns[offsets[u] ..
 *     offsets[u+1]-1]; offsets has n+1 entries, offsets[0] = 0,
 *     offsets[n] = m, offsets non-decreasing, every column < n.  Self-loops and
 *     parallel edges are allowed; each stored edge carries one message.
 *   - Plain pointers and sizes only.  "host" pointers are ordinary CPU memory
 *     (page-locked memory, best from ipg_host_alloc, makes copies faster);
 *     "dev" pointers are CUDA device
 *     memory on the device that was current when the graph was created.
 *   - A `stream` argument is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream).  *_dev calls enqueue on that stream and return after
 *     the result is complete on it (the library reads a few bytes back to
 *     decide termination: per superstep, or per 64 supersteps when the
 *     superstep loop runs on the device).
 *   - Every call returns an ipg_status; on failure, ipg_last_error() gives a
 *     message for the calling thread, outputs are unspecified and the stats
 *     count is 0.
 *   - A graph is not thread-safe: calls on one graph must not overlap (they
 *     share the graph's device workspace).  Different graphs are independent.
 *   - Memory: the library allocates the graph's device copy and workspace with
 *     cudaMalloc and frees it in ipg_graph_destroy.  The caller owns every
 *     buffer it passes in; the library never keeps a caller pointer.
 */
#ifndef IPG_H
#define IPG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IPG_OK = 0,
    IPG_EINVAL = 1,    /* bad argument or malformed CSR */
    IPG_ENOMEM = 2,    /* device or pinned-host allocation failed */
    IPG_ECUDA = 3,     /* a CUDA runtime call failed */
    IPG_ETIMEOUT = 4,  /* a bounded device-side wait ran out */
    IPG_EDEVICE = 5,   /* a kernel reported an internal inconsistency */
    IPG_ENOTSUP = 6,   /* operation not supported for this graph */
    IPG_EOVERFLOW = 7, /* an SSSP distance would reach UINT32_MAX */
    IPG_ECANCELED = 8  /* a served query was cancelled before it was dispatched */
} ipg_status;

typedef struct ipg_graph ipg_graph; /* opaque; owns its device copy */

/* One record per superstep, numbered as in the Pregel model (superstep 0 is
 * the one where every vertex is active). */
typedef struct {
    uint32_t superstep;
    uint32_t flags;          /* IPG_STAT_* bits telling which fields were measured */
    uint64_t active;         /* vertices that ran the compute step: n in superstep 0
                                (and in every PageRank superstep), else the previous
                                superstep's receivers; valid with IPG_STAT_RECEIVERS */
    uint64_t senders;        /* vertices that broadcast to their out-neighbours */
    uint64_t messages_sent;  /* messages sent = edges scanned from the senders */
    uint64_t receivers;      /* distinct vertices that received >= 1 of those
                                messages; valid with IPG_STAT_RECEIVERS */
    float kernel_ms;         /* device time of the superstep's main kernel; valid with IPG_STAT_TIMING */
    float superstep_ms;      /* device time of all of the superstep's kernels; valid with IPG_STAT_TIMING */
} ipg_superstep_stats;

#define IPG_STAT_RECEIVERS 1u /* count receivers (costs one extra atomic per message) */
#define IPG_STAT_TIMING 2u    /* time every superstep with CUDA events */
#define IPG_STAT_PULL 4u      /* set by the library: the superstep ran in pull form */

/* Caller-owned statistics buffer.  The library writes min(count, cap) records
 * and sets `count` to the number of supersteps executed, which is also the
 * superstep count of the Pregel run.  buf may be NULL when cap is 0. */
typedef struct {
    ipg_superstep_stats* buf;
    uint32_t cap;
    uint32_t count;  /* out */
    uint32_t flags;  /* in: IPG_STAT_RECEIVERS | IPG_STAT_TIMING */
    uint32_t reserved;
} ipg_stats;

/*
 * ipg_graph_create — copy a host CSR graph to the current device.
 *   offsets  host, n+1 entries;  columns host, m entries (may be NULL if m = 0);
 *   weights  host, m entries or NULL (SSSP then uses length 1 per edge, the
 *            paper's unweighted SSSP, Sec. VI-C);
 *   directed nonzero: arbitrary directed graph.  zero: undirected, stored with
 *            both directions of every edge (the paper's graphs, Sec. VI-B);
 *            creation does not check the symmetry (ipg_graph_check_symmetric
 *            does, on request).
 * The CSR is validated on the device; a malformed one returns IPG_EINVAL.
 * The in-edge (CSC) copy needed by PageRank on a directed graph is built on
 * the first ipg_pagerank call and kept.
 */
ipg_status ipg_graph_create(const uint64_t* offsets, const uint32_t* columns, const uint32_t* weights, uint32_t n,
                            uint64_t m, int directed, ipg_graph** out);

/* ipg_graph_create_dev — same from device arrays, copied on `stream`. */
ipg_status ipg_graph_create_dev(const uint64_t* offsets_dev, const uint32_t* columns_dev,
                                const uint32_t* weights_dev, uint32_t n, uint64_t m, int directed, void* stream,
                                ipg_graph** out);

/*
 * ipg_graph_create_batch — one graph object holding `count` independent
 * graphs (instances) side by side, so one call runs a Pregel program on all of
 * them together (batched queries on many small graphs; not in the paper).
 *   offsets[i], columns[i], weights[i] (or weights = NULL), n[i], m[i]: host CSR
 *   of instance i, as for ipg_graph_create (columns < n[i]); weights for all
 *   instances or for none;  directed: applies to every instance.
 * Instance i's vertex v is vertex base_i + v of the batch graph, with
 * base_i = n[0] + ... + n[i-1]; per-vertex outputs follow that layout.
 */
ipg_status ipg_graph_create_batch(uint32_t count, const uint64_t* const* offsets, const uint32_t* const* columns,
                                  const uint32_t* const* weights, const uint32_t* n, const uint64_t* m, int directed,
                                  ipg_graph** out);

/* Number of instances (1 for a plain graph) and, if bases is not NULL, the
 * count + 1 instance bases (bases[count] = total n). */
ipg_status ipg_graph_instances(const ipg_graph* g, uint32_t* count, uint32_t* bases);

/* Free the graph and all device memory it owns.  NULL is ignored. */
void ipg_graph_destroy(ipg_graph* g);

/* Sizes and kind of a graph (any output pointer may be NULL). */
ipg_status ipg_graph_info(const ipg_graph* g, uint32_t* n, uint64_t* m, int* directed, int* weighted);

/*
 * Where ipg_graph_create / _dev spent its time (a measurement aid; not in the
 * paper).  Milliseconds:
 *   alloc_ms         host wall time of the device allocations and the stream;
 *   upload_issue_ms  host wall time to issue the three copies (pageable host
 *                    memory makes this the whole copy; page-locked returns at once);
 *   upload_ms        device time of the copies (CUDA events on the copy stream);
 *   validate_ms      device time of the CSR checks;
 *   renumber_ms      host wall time of the degree renumbering (sorts, row renaming,
 *                    weight narrowing), including its waits;
 *   total_ms         host wall time of the whole call.
 * In-edge (CSC) building is not part of creation: it happens on first use.
 */
typedef struct {
    float alloc_ms, upload_issue_ms, upload_ms, validate_ms, renumber_ms, total_ms;
} ipg_create_profile;
ipg_status ipg_graph_create_profile(const ipg_graph* g, ipg_create_profile* out);

/*
 * ipg_graph_check_symmetric — does the stored graph equal its reverse?
 *   symmetric  out: 1 if the multiset of stored edges (u, v, w) equals the
 *              multiset of their reverses (v, u, w) (w omitted for an
 *              unweighted graph), else 0.  An undirected graph as the paper uses
 *              them (Sec. VI-B: both directions of every edge stored, with the
 *              same weight) gives 1; parallel edges count with multiplicity and
 *              self-loops are their own reverse.
 *   stream     cudaStream_t as void* (NULL = legacy default); the call returns
 *              after the check is complete on it.
 * ipg_graph_create does not run this check (it costs two sorts of the edges);
 * call it once after creating a graph with directed = 0 to confirm the input.
 * Works on directed and undirected graphs alike.  Temporary device memory: about
 * 32 bytes per edge (unweighted) or 48 (weighted), freed before returning;
 * IPG_ENOMEM if it cannot be had.  IPG_EINVAL for a NULL argument.
 */
ipg_status ipg_graph_check_symmetric(const ipg_graph* g, int* symmetric, void* stream);

/*
 * ipg_host_alloc — page-locked host memory for the host-buffer calls.
 *   bytes  size of the buffer; 0 sets *out = NULL and returns IPG_OK;
 *   out    receives the buffer: zero-filled, aligned to the transparent huge
 *          page size (2 MiB on most kernels) when bytes is at least that size,
 *          else to the base page size.
 * The memory is an anonymous mapping advised to use transparent huge pages
 * and registered with the CUDA runtime (portable to every context).  Host <->
 * device copies from it keep full speed in a long-lived process, where the
 * runtime's own page-locked buffers can end up on scattered small pages and
 * slow a large upload (ipg_graph_create of a 15 GB graph) to half speed.
 * The caller owns the buffer and releases it with ipg_host_free.  Returns
 * IPG_EINVAL for out = NULL, IPG_ENOMEM when the mapping or the page lock
 * fails for lack of memory, IPG_ECUDA for any other CUDA runtime error
 * (including no usable device).  Thread-safe.
 */
ipg_status ipg_host_alloc(size_t bytes, void** out);

/* Release a buffer from ipg_host_alloc.  NULL is ignored; a pointer that
 * ipg_host_alloc did not return (or one already freed) gives IPG_EINVAL and
 * nothing is released.  Thread-safe. */
ipg_status ipg_host_free(void* p);

/*
 * ipg_pagerank — PageRank (Sec. VI-C), pull form over the in-edges ("single
 * broadcast", Sec. IV): rank_0 = 1/n; for t = 1..updates,
 *   rank_t(v) = 0.15/n + 0.85 * sum over edges u->v of rank_{t-1}(u)/outdeg(u);
 * vertices without out-edges send nothing (their mass is dropped).
 *   ranks_out  host, n floats (FP32), written on success.
 * Sums are taken in a fixed order: results are bit-identical from run to run.
 * Stats: updates+1 supersteps (superstep 0 only sends the initial ranks).
 */
ipg_status ipg_pagerank(ipg_graph* g, uint32_t updates, float* ranks_out, ipg_stats* stats);
ipg_status ipg_pagerank_dev(ipg_graph* g, uint32_t updates, float* ranks_dev, ipg_stats* stats, void* stream);

/*
 * ipg_hashmin_cc — Hashmin connected components (Sec. VI-C, CC): every vertex
 * starts with its own id, sends the smallest label it has seen to its
 * neighbours whenever it drops, and the run ends when no message is sent.
 *   labels_out  host, n uint32 (smallest vertex id of the component).
 * Requires an undirected graph (directed = 0), else IPG_EINVAL.
 */
ipg_status ipg_hashmin_cc(ipg_graph* g, uint32_t* labels_out, ipg_stats* stats);
ipg_status ipg_hashmin_cc_dev(ipg_graph* g, uint32_t* labels_dev, ipg_stats* stats, void* stream);

/*
 * ipg_hashmin_cc_batch — Hashmin on every instance of a batch graph at once.
 *   labels_out      host, total n uint32: instance i's labels at [base_i, base_i + n_i),
 *                   as instance-local ids (equal to ipg_hashmin_cc on that instance alone);
 *   supersteps_out  host, one entry per instance or NULL: each instance's superstep count.
 * ipg_hashmin_cc_batch_dev writes the labels to device memory on `stream`.
 */
ipg_status ipg_hashmin_cc_batch(ipg_graph* g, uint32_t* labels_out, uint32_t* supersteps_out);
ipg_status ipg_hashmin_cc_batch_dev(ipg_graph* g, uint32_t* labels_dev, uint32_t* supersteps_out, void* stream);

/*
 * ipg_sssp — single-source shortest paths (Sec. VI-C, SSSP) with a min
 * combiner: the source starts at 0, every other vertex at UINT32_MAX
 * (unreached); a vertex whose distance drops sends distance + w along each
 * out-edge.  Edge lengths are the graph's weights, or 1 without weights.
 *   source    vertex id < n, else IPG_EINVAL;
 *   dist_out  host, n uint32 (UINT32_MAX = unreachable).
 * A path length that would reach UINT32_MAX returns IPG_EOVERFLOW.
 */
ipg_status ipg_sssp(ipg_graph* g, uint32_t source, uint32_t* dist_out, ipg_stats* stats);
ipg_status ipg_sssp_dev(ipg_graph* g, uint32_t source, uint32_t* dist_dev, ipg_stats* stats, void* stream);

/*
 * ipg_sssp_batch — k independent SSSP runs, each exactly as ipg_sssp from
 * sources[i], executed together on one graph (batched queries; not in the
 * paper, whose runs are one source at a time).  Up to 256 queries share each
 * superstep, in lines of 32: the 32 values of a line of a vertex sit in one
 * 128-byte line of memory, so one coalesced read per in-edge and line serves 32
 * queries.  The queries start together, those whose source has out-edges first,
 * in the fewest lines (1 to 8) that hold them; further queries take the
 * lanes that finish.
 *   sources         host, k vertex ids < n (repeats allowed), else IPG_EINVAL;
 *   dist_out        host, k * n uint32: row i holds the distances from sources[i]
 *                   (UINT32_MAX = unreachable);
 *   supersteps_out  host, k entries or NULL: the superstep count of each run.
 * ipg_sssp_batch_dev writes the k * n result to device memory on `stream`.
 * Uses about 264 bytes per vertex and line of device workspace, kept with the
 * graph (fewer lines are used when that would not fit in three quarters of free
 * device memory); ipg_sssp_batch also stages up to 256 rows of n words.
 */
ipg_status ipg_sssp_batch(ipg_graph* g, const uint32_t* sources, uint32_t k, uint32_t* dist_out,
                          uint32_t* supersteps_out);
ipg_status ipg_sssp_batch_dev(ipg_graph* g, const uint32_t* sources, uint32_t k, uint32_t* dist_dev,
                              uint32_t* supersteps_out, void* stream);

/*
 * Totals of the graph's last ipg_sssp_batch[_dev] call (a measurement aid; not
 * in the paper): queries run, supersteps of the lane loop (each serves every
 * lane holding a query), how many of them ran in pull form, supersteps after
 * which finished lanes were harvested, graph launches, and the lanes the call
 * used (32 per line).  All zero before the first call.  IPG_EINVAL for NULL
 * arguments.
 */
typedef struct {
    uint64_t queries, supersteps, pull_supersteps, harvests, launches, lanes;
} ipg_batch_info;
ipg_status ipg_sssp_batch_info(const ipg_graph* g, ipg_batch_info* out);

/*
 * ipg_sssp_noalloc — the same SSSP as ipg_sssp, for callers that may not
 * allocate device memory (the paper has no counterpart to this call).
 * Callers whose device memory belongs to another allocator (a framework's
 * pool, a budget fixed at start-up) or that run on a latency-critical path
 * cannot afford cudaMalloc/cudaFree, which can fail and stall the device; they
 * cannot create an ipg_graph, since that copies the graph and allocates.  This
 * call reads the caller's device CSR in place and allocates nothing: its working
 * state lives in one fixed scratch array inside the library's device image,
 * 16 MiB on every GPU that loads the library, held until the process exits.
 *   offsets_dev, columns_dev, weights_dev (or NULL), n, m: a device CSR on the
 *       current device, as for ipg_graph_create; it is validated on every call;
 *   n <= IPG_NOALLOC_MAX_VERTICES, else IPG_EINVAL;  source < n;
 *   dist_dev: device, n uint32 (UINT32_MAX = unreachable), caller-owned;
 *   supersteps_out: optional, the Pregel superstep count;
 *   stream: cudaStream_t as void* (NULL = legacy default stream).
 * The first call on a device looks up the scratch array's device address (with
 * that device current).  Under CUDA's default lazy module loading that lookup
 * is also what loads this part of the library's device code onto the device and
 * reserves the 16 MiB array, so the first call on each device does take device
 * memory and can fail (IPG_ECUDA) when none is left; later calls take none.
 * Callers on a fixed budget should therefore make one warm-up call at start-up
 * (a one-vertex graph will do) while memory is still available.
 * Every call on a device shares the one scratch array and finds the previous
 * call's contents there (it clears what must start at zero): calls that overlap
 * on the GPU, from several streams or threads, race and give wrong results.
 * The call synchronizes `stream` once per superstep to read the frontier size,
 * so it cannot be issued while that stream is being captured into a CUDA graph.
 */
#define IPG_NOALLOC_MAX_VERTICES (1u << 20)
ipg_status ipg_sssp_noalloc(const uint64_t* offsets_dev, const uint32_t* columns_dev, const uint32_t* weights_dev,
                            uint32_t n, uint64_t m, uint32_t source, uint32_t* dist_dev, uint32_t* supersteps_out,
                            void* stream);

/*
 * General combiners (Sec. III, Fig. 1).  The calls below run vertex programs
 * whose messages are wider than 32 bits and whose combine is not a hardware
 * atomic, through the hybrid combiner of include/ipg_combiner.cuh: each
 * mailbox is a flag plus a message slot; the first message takes a per-vertex
 * lock, stores itself and raises the flag, later ones combine into the slot by
 * compare-and-swap.  A vertex is active in the next superstep exactly when it
 * received a message (its flag was raised), as in the Pregel model, whatever
 * the combined value.  Every superstep record has IPG_STAT_RECEIVERS set: the
 * receivers are counted exactly, for free, by the first-message path.
 * A bounded wait inside the combiner that runs out returns IPG_ETIMEOUT.
 */

/*
 * ipg_sssp_tree — SSSP that also returns a shortest-path tree.  Each message
 * is the 64-bit pair (distance, sender id), combined by the lexicographic
 * minimum, so a vertex keeps the smallest (distance, parent) it ever heard of.
 * It sends only when its distance drops, so the senders, messages and
 * superstep count equal ipg_sssp's.
 *   source      vertex id < n, else IPG_EINVAL;
 *   dist_out    host, n uint32 (UINT32_MAX = unreachable) — equal to ipg_sssp's;
 *   parent_out  host, n uint32: for a reached vertex v other than the source,
 *               the smallest u with an edge u -> v and dist[u] + w(u,v) = dist[v];
 *               the source's parent is the source; UINT32_MAX if unreached.
 * A path length that would reach UINT32_MAX returns IPG_EOVERFLOW.
 */
ipg_status ipg_sssp_tree(ipg_graph* g, uint32_t source, uint32_t* dist_out, uint32_t* parent_out, ipg_stats* stats);
ipg_status ipg_sssp_tree_dev(ipg_graph* g, uint32_t source, uint32_t* dist_dev, uint32_t* parent_dev,
                             ipg_stats* stats, void* stream);

/*
 * ipg_bfs_paths — number of shortest paths from a source, by breadth-first
 * levels.  Each message is the 128-bit pair (level, count); the combine keeps
 * the smallest level and adds the counts of messages at that level.  Every
 * edge has length 1 (weights are ignored) and is one message, so parallel
 * edges count as distinct paths.  Counts are exact modulo 2^64.
 *   source     vertex id < n, else IPG_EINVAL;
 *   level_out  host, n uint32: hop distance from the source (UINT32_MAX = unreachable);
 *   paths_out  host, n uint64: shortest paths from the source modulo 2^64 (0 = unreachable).
 */
ipg_status ipg_bfs_paths(ipg_graph* g, uint32_t source, uint32_t* level_out, uint64_t* paths_out, ipg_stats* stats);
ipg_status ipg_bfs_paths_dev(ipg_graph* g, uint32_t source, uint32_t* level_dev, uint64_t* paths_dev,
                             ipg_stats* stats, void* stream);

/*
 * ipg_combine_dev — the combination step alone: deliver k messages, message i
 * to vertex dst[i], into n mailboxes that start empty.
 *   kind       an ipg_combine_kind (the message size follows from it);
 *   dst_dev    device, k uint32, each < n (else IPG_EINVAL, nothing is
 *              written out of bounds);
 *   msgs_dev   device, k messages of the kind's size, 16-byte aligned for the
 *              128-bit kind (a (key u64, count u64) pair);
 *   flags_dev  device, n uint32, out: 1 where the vertex received a message, 0
 *              elsewhere (cleared by the call);
 *   mail_dev   device, n messages of the kind's size, out: the combined message
 *              where flags_dev is 1, untouched elsewhere;
 *   receivers_out  host, optional: number of vertices that received a message;
 *   options    IPG_COMBINE_WARP (fold same-destination messages within a warp
 *              before the mailbox) and/or IPG_COMBINE_NATIVE (IPG_COMBINE_MIN_U64
 *              only: a hardware 64-bit atomicMin on a slot preset to the maximum
 *              instead of the hybrid combiner; same result — a comparison point);
 *              IPG_COMBINE_STALLED (hybrid combiner only) starts every mailbox
 *              CLAIMED by a first sender that never publishes — the state a
 *              stalled writer would leave — and lets a send poll such a flag
 *              only 64 times: every send's bounded wait runs out, no message is
 *              delivered, flags_dev is left CLAIMED (2) and the call returns
 *              IPG_ETIMEOUT within milliseconds.  It exercises the timeout path
 *              of the combiner without any hang.
 * Returns after the result is complete on `stream`.  k may be 0.
 */
typedef enum {
    IPG_COMBINE_XOR_U32 = 0,       /* 4-byte messages, bitwise exclusive or */
    IPG_COMBINE_MIN_U64 = 1,       /* 8-byte messages, minimum */
    IPG_COMBINE_SUM_U64 = 2,       /* 8-byte messages, sum modulo 2^64 */
    IPG_COMBINE_MINCOUNT_U128 = 3  /* 16-byte (key, count): smallest key, counts at that key added modulo 2^64 */
} ipg_combine_kind;
#define IPG_COMBINE_WARP 1u
#define IPG_COMBINE_NATIVE 2u
#define IPG_COMBINE_STALLED 4u
ipg_status ipg_combine_dev(int kind, uint32_t n, const uint32_t* dst_dev, const void* msgs_dev, uint64_t k,
                           uint32_t* flags_dev, void* mail_dev, uint64_t* receivers_out, uint32_t options,
                           void* stream);

/*
 * Serving (not in the paper): a resident set of graphs answering a stream of
 * queries with continuous batching.  Worker threads take the graph whose head
 * query has waited longest (one worker per graph at a time).  SSSP queries at
 * the head of a graph's queue run one source at a time, or, from
 * min_sssp_batch queued queries on, in a lane session of the batched engine
 * (32 lanes): queries that arrive while the session is on the GPU take lanes
 * that free up, at the next superstep boundary (continuous batching); queued Hashmin
 * queries (or PageRank queries with the same update count) on one graph share
 * one run, as they compute the same result (in flight only: completed results
 * are never reused).  Different graphs run concurrently on their own
 * streams.  Before a dispatch the server checks that the graph's workspace
 * fits (free device memory minus reserve_bytes, or workspace_budget when
 * nonzero), releasing idle graphs' workspaces least recently used first.
 * Each result equals that of the matching single-query call.
 * The graphs stay owned by the caller and must outlive the server; while the
 * server exists, the caller must not call other functions on them.
 */
typedef struct ipg_server ipg_server;

typedef enum { IPG_Q_SSSP = 0, IPG_Q_HASHMIN = 1, IPG_Q_PAGERANK = 2 } ipg_query_kind;

typedef struct {
    uint32_t graph;    /* index into the server's graph array */
    uint32_t kind;     /* ipg_query_kind */
    uint32_t source;   /* SSSP source (< n) */
    uint32_t updates;  /* PageRank updates */
    void* out;         /* host buffer, caller-owned until the completion: n uint32 (SSSP
                          distances, Hashmin labels) or n float (PageRank) */
    uint64_t user;     /* caller's tag, returned in the completion */
} ipg_query;

typedef struct {
    uint64_t user;
    ipg_status status;
    uint32_t supersteps;  /* superstep count of the query's run */
    uint32_t batch;       /* queries dispatched together with this one (itself included); for an
                             SSSP query of a lane session: the session's queries on the device
                             once it was seeded */
    uint32_t joined;      /* 1: an SSSP query seeded into a lane session that was already running,
                             at a superstep boundary (continuous batching); else 0 */
    double t_submit;      /* seconds on the server clock (ipg_server_now) */
    double t_start;
    double t_done;
} ipg_completion;

typedef struct {
    uint32_t workers;           /* worker threads = graphs in flight at once; 0 -> 8 */
    uint32_t max_batch;         /* SSSP queries dispatched together at most; 0 -> 256 */
    uint64_t workspace_budget;  /* bytes of graph workspace held at once; 0 -> free memory */
    uint64_t reserve_bytes;     /* device memory kept free when budget is 0; 0 -> 1 GiB */
    uint32_t min_sssp_batch;    /* fewer queued SSSP queries run one source at a time; 0 -> per
                                   graph, 3 * 2^(0.375 * (log2 m - 18)) clamped to [2, 32] */
    uint32_t flags;             /* IPG_SERVER_* bits */
} ipg_server_options;

/* ipg_server_create runs ipg_autotune on every graph before it starts serving
 * (PageRank, SSSP, batched SSSP, and Hashmin on undirected graphs); a graph
 * already tuned for a program keeps its values.  Tuning times each graph alone;
 * under concurrent load other choices can be faster, so it is off by default. */
#define IPG_SERVER_AUTOTUNE 1u
/* ipg_server_create runs every program the server dispatches once on every graph
 * (one SSSP, one batched SSSP of 32 sources, PageRank with 10 updates, and
 * Hashmin on undirected graphs) into a scratch buffer, so that the graphs' device
 * workspaces and captured superstep loops exist before the first query instead
 * of being made while queries wait.  With a workspace budget, workers may
 * release them later. */
#define IPG_SERVER_PREPARE 2u

/* graphs: count graph handles (all on the same device); opt may be NULL. */
ipg_status ipg_server_create(ipg_graph* const* graphs, uint32_t count, const ipg_server_options* opt,
                             ipg_server** out);
/* Queue a query (copied); returns at once.  IPG_EINVAL for a bad graph index,
 * kind, source, or Hashmin on a directed graph. */
ipg_status ipg_server_submit(ipg_server* s, const ipg_query* q);
/* Up to cap completed queries into out; waits up to wait_ms for the first one
 * (0: no wait, < 0: until one completes or nothing is in flight). */
uint32_t ipg_server_poll(ipg_server* s, ipg_completion* out, uint32_t cap, int wait_ms);
/* Cancel every queued query whose user tag equals `user` and that no worker has
 * dispatched yet.  Each completes at once with status IPG_ECANCELED (supersteps
 * 0, batch 0, t_start = t_done = the time of the cancel); its out buffer is not
 * written and is the caller's again after that completion is polled.  A query
 * already dispatched runs to completion: no running kernel is interrupted.
 * *cancelled (may be NULL) receives the number cancelled.  IPG_EINVAL for a
 * NULL server. */
ipg_status ipg_server_cancel(ipg_server* s, uint64_t user, uint32_t* cancelled);
/* Wait until every submitted query has completed (completions stay pollable). */
ipg_status ipg_server_drain(ipg_server* s);
/* Seconds since the server was created (the clock of the completion times). */
double ipg_server_now(const ipg_server* s);
/* Drain, stop the workers, free the server (not the graphs). */
void ipg_server_destroy(ipg_server* s);

/*
 * Process-wide tuning knobs (not in the paper; they change speed, never results):
 *   "pull_divisor"  Hashmin/SSSP superstep direction.  A superstep whose messages
 *                   (sum of the senders' out-degrees) reach m / pull_divisor runs in
 *                   pull form (every vertex scans its in-edges, as the paper's
 *                   pull-based CC version does, Sec. VI-C) instead of push form.
 *                   0 = always push.  Default 6.
 *   "combine_warp"  ipg_sssp_tree / ipg_bfs_paths: 1 = lanes of a warp that send to
 *                   the same vertex fold their messages first (IPG_COMBINE_WARP),
 *                   0 = every message goes to the mailbox.  Default 0.
 *   "pr_engine"     PageRank pull kernel: 0 = messages staged in shared memory,
 *                   1 = messages loaded into registers, row ends as a bit mask.
 *                   Both add in the same order: ranks are bit-identical.  Default 0.
 *   "pr_threads"    PageRank pull kernel: 256 or 512 threads per merge-path tile.
 *                   The per-thread summation runs change with it, so ranks may
 *                   differ in the last bits (both stay within the float tolerance).
 *                   Default 256.
 *   "pr_carveout"   pull kernels: shared-memory carveout in percent of the SM's
 *                   unified L1/shared array; -1 = the smallest that keeps the
 *                   kernel's full occupancy, leaving the rest to L1, which caches
 *                   the messages of the most-connected senders.  Default -1.
 *   "batch_divisor" ipg_sssp_batch: a superstep whose senders (union over the
 *                   sources of a group) have fewer than m / batch_divisor out-edges
 *                   runs in push form, else in pull form.  0 = always pull.
 *                   Default 6.
 *   "push_loop"     Hashmin/SSSP: 1 = the superstep loop runs on the device inside a
 *                   CUDA graph (a conditional WHILE node; a few host synchronisations
 *                   per run) whenever no per-superstep timing is asked for and the
 *                   stats buffer holds at most 65536 records; 0 = the host drives
 *                   every superstep.  Default 1.
 *   "pull_filter"   Hashmin/SSSP pull supersteps whose messages are below this
 *                   percentage of m read a one-bit-per-vertex sender array before
 *                   each gather and gather only from senders; 0 = never (default:
 *                   measured slower on R-MAT 26/28), 100 = every pull superstep.
 *   "batch_chunk"   batched SSSP: in-edges per warp task of the pull form with one
 *                   line of 32 lanes (the engine's tile size), a multiple of 32 in
 *                   [32, 65536], as its largest size: on smaller graphs the engine
 *                   halves it (not below 64) until each warp of the launch has at
 *                   least 3 tasks; a tile the autotuner stored in the graph is used
 *                   as it is.  Default 256.
 *   "batch_wide_chunk" the same for the pull form with more lines, as its largest
 *                   size: on smaller graphs the engine halves it (not below 128)
 *                   until each warp of the launch has at least 3 tasks.  Default 512.
 *   "batch_tile_tasks" batched SSSP: the tasks per warp of the launch that the two
 *                   tile sizes above are halved to reach, in [0, 64]; 0 uses them
 *                   as they are set.  Halving keeps a tile a multiple of 32.
 *                   Default 3.
 *   "batch_loop"    batched SSSP: 1 = the superstep loop runs on the device inside a
 *                   CUDA graph (one host synchronisation per 1024 supersteps); 0 = the
 *                   host launches every superstep's kernels and reads the loop state
 *                   back after each (for profilers that do not follow kernels inside
 *                   conditional graph nodes).  Results are the same.  Default 1.
 * Unknown names or invalid values return IPG_EINVAL.  Set knobs between calls,
 * not while a call runs.  A graph tuned by ipg_autotune uses its own values of
 * pull_divisor, batch_divisor, batch_chunk, pr_engine and pr_carveout instead of these.
 */
ipg_status ipg_set_tuning(const char* name, int64_t value);
ipg_status ipg_get_tuning(const char* name, int64_t* value);

/*
 * ipg_autotune — pick the launch shape of the calls above for one graph by
 * timing them on it (no counterpart in the paper: its OpenMP versions fix one
 * schedule per benchmark, Sec. V-B and VI-C).
 *   programs     IPG_TUNE_* bits: which programs to tune.  IPG_TUNE_HASHMIN
 *                needs an undirected graph (IPG_EINVAL otherwise).
 *   sssp_source  caller id of the SSSP source to time with; >= n picks the
 *                vertex of largest total degree.
 *   report       optional, out: the chosen values and the timings.
 *   stream       cudaStream_t as void* for the timed runs.
 * Candidates, all of which give bit-identical results (min combiners are
 * order-free; both PageRank engines and every carveout add in one order):
 *   Hashmin, SSSP  pull_divisor in {0, 2, 4, 6, 10, 16, 32};
 *   batched SSSP   (batch_divisor, batch_chunk) in {(6, 256), (0, 256), (2, 256),
 *                  (16, 256), (6, 64), (6, 128), (6, 512), (6, 1024)}: the push/pull
 *                  switch and the tile size of the pull form (in-edges per warp
 *                  task), which the graph then uses as it is;
 *   PageRank       (pr_engine, pr_carveout) in {(0,-1), (0,60), (1,-1), (1,5)}.
 * Each candidate runs twice (the faster run counts): Hashmin and SSSP to
 * quiescence, batched SSSP on 32 sources (sssp_source and 31 caller ids spread
 * evenly over [0, n)), PageRank for 3 updates, into a scratch buffer (32 n
 * words with IPG_TUNE_SSSP_BATCH, else n) that the call allocates and frees.
 * The winners are stored in the graph and used by
 * every later call on it.  Results are cached per graph and in a process-wide
 * table keyed by the graph's shape (n, m, directedness, weights, the largest
 * out-degree and 64 sampled offsets), so tuning an identical graph again costs
 * nothing; IPG_TUNE_FORCE re-times.  Errors: IPG_EINVAL (NULL graph, unknown
 * bits, Hashmin on a directed graph), IPG_ECUDA/IPG_ENOMEM; the graph then keeps
 * its previous tuning.
 */
#define IPG_TUNE_PAGERANK 1u
#define IPG_TUNE_HASHMIN 2u
#define IPG_TUNE_SSSP 4u
#define IPG_TUNE_SSSP_BATCH 8u
#define IPG_TUNE_FORCE 0x100u

typedef struct {
    uint32_t programs;          /* programs the graph is tuned for after the call */
    uint32_t cached;            /* 1: every requested program came from a cache */
    int64_t hashmin_pull_divisor, sssp_pull_divisor, sssp_batch_divisor, pr_engine, pr_carveout;  /* -1 = not tuned */
    float hashmin_ms, sssp_ms, sssp_batch_ms, pagerank_ms;  /* best candidate's run, 0 if not timed */
    float hashmin_default_ms, sssp_default_ms, sssp_batch_default_ms, pagerank_default_ms;  /* process-wide knobs */
    uint32_t candidates_timed;  /* runs made by this call */
    uint32_t sssp_batch_chunk;  /* batched SSSP: in-edges per warp task of its pull form (0 = not tuned) */
} ipg_tune_report;

ipg_status ipg_autotune(ipg_graph* g, uint32_t programs, uint32_t sssp_source, ipg_tune_report* report,
                        void* stream);

/* Message for the last failed call on this thread ("" if none). */
const char* ipg_last_error(void);

/* Static name of a status code. */
const char* ipg_status_string(ipg_status s);

/* Library version, major*10000 + minor*100 + patch. */
int ipg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* IPG_H */
