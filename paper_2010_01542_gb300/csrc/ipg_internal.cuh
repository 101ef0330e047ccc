// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ipg.h"

namespace ipg {

constexpr uint32_t kInf = 0xFFFFFFFFu;

// device status word bits (written by kernels, read by the host after a run)
constexpr uint32_t kStatusOverflow = 1u;    // an SSSP distance reached UINT32_MAX
constexpr uint32_t kStatusBadCsr = 2u;      // validation: offsets not monotone / wrong ends
constexpr uint32_t kStatusBadColumn = 4u;   // validation: a column >= n
constexpr uint32_t kStatusInternal = 8u;    // a kernel found an inconsistent index

// counters the push drivers read back every superstep (one 64-byte block)
struct PushCounters {
    unsigned long long edges;      // messages of the current superstep (sum of frontier degrees)
    unsigned long long receivers;  // distinct receivers (stats mode)
    unsigned int next_size;        // vertices appended to the next frontier
    unsigned int tiles;            // merge-path tiles of the current superstep
    unsigned int status;           // kStatus* bits
    unsigned int pad[9];
};

// Device-resident state of a Hashmin/SSSP superstep loop run inside a CUDA graph
// (ipg_push.cu): the kernels read the frontier from it, so their launch
// parameters never change, and the step kernel advances it.
struct PushLoop {
    unsigned int cur;      // frontier buffer holding the senders
    unsigned int f;        // senders
    unsigned int s;        // Pregel superstep number
    unsigned int pull;     // 1: this superstep runs in pull form
    unsigned int iter;     // supersteps run by the current graph launch
    unsigned int done;     // 1: no superstep left
    unsigned int count;    // superstep count once done
    unsigned int nrec;     // stats records written
    unsigned int status;   // kStatus* bits
    unsigned int filter;   // 1: this pull superstep checks the sender bits before each gather
    unsigned long long divisor;         // pull when messages * divisor >= m (0: never)
    unsigned long long prev_receivers;  // receivers of the previous superstep (stats mode)
    unsigned int filter_pct;            // filter a pull superstep whose messages are below this % of m
    unsigned int pad;
};

// frontier of a loop-driven superstep (loop != NULL) or of a host-driven one
__device__ __forceinline__ const uint32_t* loop_frontier(const uint32_t* F0, const uint32_t* F1,
                                                         const PushLoop* loop) {
    return loop && loop->cur ? F1 : F0;
}
__device__ __forceinline__ uint32_t* loop_next(uint32_t* N0, uint32_t* N1, const PushLoop* loop) {
    return loop && loop->cur ? N0 : N1;
}
__device__ __forceinline__ uint32_t loop_f(uint32_t f, const PushLoop* loop) { return loop ? loop->f : f; }

ipg_status set_error(ipg_status s, const char* fmt, ...);
ipg_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define IPG_CUDA(call)                                                        \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return ::ipg::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define IPG_TRY(expr)                          \
    do {                                       \
        ipg_status s_ = (expr);                \
        if (s_ != IPG_OK) return s_;           \
    } while (0)

// grows a device buffer (contents are not kept)
ipg_status ensure_buffer(void** p, size_t* cap, size_t bytes);

template <typename T>
inline ipg_status ensure(T** p, size_t* cap, size_t count) {
    return ensure_buffer(reinterpret_cast<void**>(p), cap, count * sizeof(T));
}

// RAII guard: makes the graph's device current for the duration of a call
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// knobs an autotuned graph carries instead of the process-wide ones
struct GraphTuning {
    bool pr = false, cc = false, sssp = false, batch = false;
    long long pr_engine = 0, pr_carveout = -1;
    long long cc_divisor = 6, sssp_divisor = 6, batch_divisor = 6, batch_chunk = 256;
};

// per-superstep CUDA events (IPG_STAT_TIMING)
struct StepTimer {
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    ipg_status init();
    void destroy();
};

}  // namespace ipg

struct ipg_graph {
    int device = 0;
    uint32_t n = 0;
    uint64_t m = 0;
    int directed = 1;
    int weighted = 0;

    // CSR (out-edges) in the library's internal vertex numbering: vertices are
    // relabelled by decreasing total degree when the graph is created, so the
    // most-accessed values sit together; perm/inv translate at the boundary.
    uint64_t* off = nullptr;
    uint32_t* col = nullptr;
    uint32_t* w = nullptr;       // u32 weights (only when some weight exceeds 255)
    uint8_t* w8 = nullptr;       // u8 weights (when every weight fits in a byte)
    uint64_t max_outdeg = 0;     // largest out-degree (bounds a frontier's messages)
    uint32_t* perm = nullptr;    // internal id -> caller's id
    uint32_t* inv = nullptr;     // caller's id -> internal id

    // CSC (in-edges) for pull; aliases the CSR on undirected graphs
    uint64_t* csc_off = nullptr;
    uint32_t* csc_src = nullptr;
    uint8_t* csc_w8 = nullptr;    // in-edge weights, same kind as the CSR's
    uint32_t* csc_w = nullptr;
    bool csc_ready = false;
    bool csc_owned = false;
    long long in_nonempty = -1;  // vertices with in-degree > 0 (PageRank receivers), lazily counted

    // PageRank state
    float* inv_outdeg = nullptr;
    float* pr_box[2] = {nullptr, nullptr};  // outbox double buffer
    uint32_t* pr_tile_row = nullptr;        // merge-path tile boundaries over the CSC
    float* pr_head = nullptr;               // per tile: partial of the row that began in an earlier tile
    float* pr_tail = nullptr;               // per tile: partial of the row that continues past it
                                            // (4-byte slots, also used as u32 by pull-min supersteps)
    uint64_t pr_tiles = 0;
    float* pr_out_stage = nullptr;          // host-variant output staging
    size_t pr_out_stage_cap = 0;
    cudaGraphExec_t pr_exec = nullptr;      // captured superstep loop (ipg_pagerank.cu)
    uint64_t pr_exec_key = 0;               // updates and launch shape it was captured for

    // push (Hashmin / SSSP) workspace
    uint32_t* stamp = nullptr;       // superstep in which the vertex was last appended to a frontier
    uint32_t* rstamp = nullptr;      // superstep in which the vertex last received (stats mode)
    uint32_t* frontier[2] = {nullptr, nullptr};
    unsigned long long* fr_prefix = nullptr;  // exclusive prefix of frontier out-degrees (f+1)
    unsigned long long* fr_rowstart = nullptr;
    uint32_t* fr_val = nullptr;               // value snapshot of each frontier vertex
    unsigned long long* block_sums = nullptr;
    size_t block_sums_cap = 0;
    uint32_t* push_tile_row = nullptr;
    size_t push_tile_cap = 0;
    uint32_t* val_stage = nullptr;            // host-variant value buffer
    uint32_t* val = nullptr;                  // values in internal numbering
    float* pr_rank = nullptr;                 // final ranks in internal numbering
    uint32_t* sval = nullptr;                 // pull supersteps: value sent by each vertex, kInf if none
    uint32_t* sbits = nullptr;                // pull supersteps: one bit per vertex, set for the senders
    ipg_create_profile create_profile{};      // where ipg_graph_create spent its time
    ipg::PushCounters* counters = nullptr;    // device
    ipg::PushCounters* h_counters = nullptr;  // pinned host mirror

    ipg::PushLoop* loop = nullptr;            // device loop state (graph-driven runs)
    ipg_superstep_stats* loop_rec = nullptr;  // device stats records of a graph-driven run
    ipg::PushLoop* h_loop = nullptr;          // pinned mirror
    cudaGraphExec_t push_exec[16] = {};       // loop graphs: program x receivers x pull x instances (ipg_push.cu)

    void* batch = nullptr;          // batched-SSSP workspace (ipg_batch.cu)
    void* generic = nullptr;        // general-combiner workspace (ipg_generic.cu)

    // graphs created by ipg_graph_create_batch: instance i owns caller ids
    // [inst_base[i], inst_base[i+1])
    uint32_t instances = 0;
    uint32_t* inst_base_host = nullptr;  // instances + 1
    uint32_t* inst_base = nullptr;       // device copy
    unsigned long long* inst_msgs = nullptr;  // device, per instance
    uint32_t* inst_steps = nullptr;           // device, per instance: supersteps of a loop-driven run

    cudaStream_t stream = nullptr;  // used by the host-buffer entry points
    ipg::StepTimer timer;
    ipg::GraphTuning tuned;         // set by ipg_autotune
};

namespace ipg {
// in ipg_graph.cu
ipg_status ensure_csc(ipg_graph* g, cudaStream_t st);
ipg_status ensure_pull_partition(ipg_graph* g, cudaStream_t st);
ipg_status count_in_nonempty(ipg_graph* g, cudaStream_t st);
ipg_status ensure_push_workspace(ipg_graph* g, bool receivers);
int sm_count_of(int dev);
// SMs of the current device (queried once per device and cached)
int sm_count_current();
// in ipg_graph.cu: shared by create and create_batch
ipg_status create_graph(const uint64_t* offsets, const uint32_t* columns, const uint32_t* weights, uint32_t n,
                        uint64_t m, int directed, cudaStream_t user_stream, bool from_device, ipg_graph** out);
// in ipg_push.cu: the frontier's out-degree prefix, row starts and (if val is not
// NULL) value snapshot, and the merge-path split of (frontier rows + their edges)
// into tiles of kFrontierTile items; edges and tiles land in g->counters
constexpr uint32_t kFrontierTile = 2048;
ipg_status frontier_prepare(ipg_graph* g, const uint32_t* F, uint32_t f, const uint32_t* val, cudaStream_t st);
ipg_status frontier_partition(ipg_graph* g, uint32_t f, cudaStream_t st);
// in ipg_batch.cu
void batch_free(ipg_graph* g);
// Lane sessions of the batched SSSP engine driven by the host (the server): up to
// 32 queries run at once, one per lane; seeds join at superstep boundaries.
struct LaneReport {
    uint32_t live;          // lanes holding a query after the launch
    uint32_t finished;      // lanes whose query finished in the launch's last superstep
    uint32_t row[32];       // output (staging) row of each lane's query
    uint32_t count[32];     // superstep count of each lane's query (final for finished lanes)
};
// stage_dev: 32 rows of n words; a finished query's distances land in its row.
ipg_status lanes_open(ipg_graph* g, uint32_t* stage_dev, cudaStream_t st);
// Seeds nseed queries (caller-id sources, staging rows; at most the free lanes),
// then runs supersteps until a lane finishes or the admit flag is raised.
ipg_status lanes_step(ipg_graph* g, const uint32_t* sources, const uint32_t* rows, uint32_t nseed,
                      cudaStream_t st, LaneReport* rep);
void lanes_close(ipg_graph* g);
// mapped host flag that ends a running launch at the next superstep boundary
volatile unsigned int* lanes_admit_flag(ipg_graph* g);
ipg_status sssp_batch_run(ipg_graph* g, const uint32_t* sources, uint32_t k, uint32_t* dist_dev,
                          uint32_t* supersteps_out, cudaStream_t st);
// in ipg_generic.cu
void generic_free(ipg_graph* g);
// caller ids -> internal ids, in place on the device
ipg_status map_to_internal(ipg_graph* g, uint32_t* ids, uint32_t k, cudaStream_t st);
// in ipg_pull_min.cu
ipg_status pull_min_superstep(ipg_graph* g, bool sssp, bool recv, bool filter, const uint32_t* F, const uint32_t* fval, uint32_t f,
                              uint32_t* val, uint32_t* next, cudaStream_t st, cudaEvent_t ev_kernel);
// the pull form of a loop-driven superstep: every kernel returns at once unless
// loop->pull is set; frontiers and sizes come from the loop block
ipg_status pull_min_enqueue_loop(ipg_graph* g, bool sssp, bool recv, uint32_t* val, cudaStream_t st);
ipg_status pull_min_prepare(ipg_graph* g, cudaStream_t st);
// process-wide tuning knobs (ipg_set_tuning)
struct Tuning {
    long long pull_divisor = 6;  // pull when a superstep's messages reach m / pull_divisor; 0 = never
    long long combine_warp = 0;  // general combiners: fold same-destination messages within a warp first
    long long pr_threads = 256;  // PageRank pull kernel: threads per CTA (256 or 512)
    long long pr_carveout = -1;  // PageRank pull kernel: shared-memory carveout percent (-1 = smallest)
    long long batch_divisor = 6; // batched SSSP: push when the senders' out-edges < m / batch_divisor (0 = pull)
    long long push_loop = 1;     // Hashmin/SSSP: 1 = superstep loop in a CUDA graph where possible, 0 = host loop
    long long pr_engine = 0;     // PageRank pull kernel: 0 staged messages, 1 direct (registers)
    long long pull_filter = 0;   // Hashmin/SSSP pull: check sender bits first below this % of m messages; 0 = never
    long long batch_chunk = 256; // batched SSSP pull: in-edges per warp task (the engine's tile size)
    long long batch_loop = 1;    // batched SSSP: 1 = superstep loop in a CUDA graph, 0 = launched from the host
    long long batch_wide_chunk = 512;  // batched SSSP pull with more than one line: in-edges per warp task
    long long batch_tile_tasks = 3;    // batched SSSP pull: tasks per warp the tile is halved to reach (0: off)
};
Tuning& tuning();
// the graph's tuned value where it has one, else the process-wide knob
long long pull_divisor_for(const ipg_graph* g, bool sssp);
long long pr_engine_for(const ipg_graph* g);
long long pr_carveout_for(const ipg_graph* g);
long long batch_divisor_for(const ipg_graph* g);
long long batch_chunk_for(const ipg_graph* g);
// stats helpers
void stats_begin(ipg_stats* s);
void stats_put(ipg_stats* s, uint32_t idx, const ipg_superstep_stats& rec);
}  // namespace ipg
