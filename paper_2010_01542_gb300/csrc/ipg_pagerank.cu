// PageRank superstep, pull form ("single broadcast", Sec. IV): every vertex
// publishes one outbox value rank/outdeg, and each vertex sums the outboxes of
// its in-neighbours:
//     rank_t(v) = 0.15/N + 0.85 * sum_{u -> v} outbox_{t-1}(u),
//     outbox_t(v) = rank_t(v) / outdeg(v)      (0 for a vertex with no out-edge).
// The outbox, the reciprocal out-degree and the rank live in separate arrays:
// the paper's externalisation of the hot {flag, message} pair (Sec. IV), taken
// to a struct-of-arrays layout.
//
// Work split (Sec. V-A, edges as the workload proxy): the in-edge lists (CSC)
// are cut into tiles of equal length along the merge path of row ends and
// edges, so a vertex with millions of in-edges is spread over many CTAs and a
// run of vertices without in-edges costs one item each.  Each CTA
//   1. stages the tile's row ends and gathers outbox[src] for its edges into
//      shared memory (coalesced streaming loads of the source ids),
//   2. lets each thread walk 8 consecutive merge items, then combines the
//      per-thread carries with a segmented scan in a fixed tree order,
//   3. writes rank/outbox of every vertex whose in-edges began in this tile.
// A vertex whose in-edges began in an earlier tile is finished by a fix-up
// kernel that adds the per-tile partial sums in tile order, in double
// precision.  Every sum therefore has a fixed order: results are
// bit-reproducible.
#include "ipg_mergepath.cuh"

namespace ipg {

__global__ void mp_partition_kernel(const uint64_t* __restrict__ off, uint32_t n, uint64_t m, uint64_t tiles,
                                    uint32_t* __restrict__ tile_row) {
    const uint64_t total = (uint64_t)n + m;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= tiles; t += stride) {
        uint64_t diag = t * kMpTile;
        if (diag > total) diag = total;
        tile_row[t] = mp_rows_before(off + 1, n, m, diag);
    }
}

static unsigned grid_cap(uint64_t work, unsigned cap = 0) {
    if (!cap) cap = (unsigned)sm_count_current() * 16;
    uint64_t b = (work + 255) / 256;
    if (b < 1) b = 1;
    return (unsigned)(b < cap ? b : cap);
}

ipg_status mp_partition(const uint64_t* off, uint32_t n, uint64_t m, uint64_t tiles, uint32_t* tile_row,
                        cudaStream_t st) {
    mp_partition_kernel<<<grid_cap(tiles + 1), 256, 0, st>>>(off, n, m, tiles, tile_row);
    IPG_CUDA(cudaGetLastError());
    return IPG_OK;
}

ipg_status pull_grid(const void* const* kernels, int nkernels, int threads, int device, uint64_t tiles, int carve,
                     unsigned* grid) {
    if (carve < 0) {
        cudaFuncAttributes fa;
        IPG_CUDA(cudaFuncGetAttributes(&fa, kernels[0]));
        for (int i = 0; i < nkernels; ++i)
            IPG_CUDA(cudaFuncSetAttribute(kernels[i], cudaFuncAttributePreferredSharedMemoryCarveout, 100));
        int per_sm = 0, smem_sm = 0;
        IPG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernels[0], threads, 0));
        IPG_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device));
        // 1 KB per resident CTA is reserved by the runtime
        const double need = (double)per_sm * ((double)fa.sharedSizeBytes + 1024.0);
        carve = (int)(100.0 * need / (smem_sm > 0 ? smem_sm : 1)) + 1;
        if (carve > 100) carve = 100;
    }
    for (int i = 0; i < nkernels; ++i)
        IPG_CUDA(cudaFuncSetAttribute(kernels[i], cudaFuncAttributePreferredSharedMemoryCarveout, carve));
    int blocks = 0;
    IPG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernels[0], threads, 0));
    if (blocks < 1) blocks = 1;
    uint64_t gr = (uint64_t)sm_count_of(device) * blocks;
    if (gr > tiles) gr = tiles;
    *grid = (unsigned)(gr ? gr : 1);
    return IPG_OK;
}

namespace {

__global__ void inv_outdeg_kernel(const uint64_t* __restrict__ off, uint32_t n, float* __restrict__ inv) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        uint64_t d = off[v + 1] - off[v];
        inv[v] = d ? 1.0f / (float)d : 0.0f;
    }
}

__global__ void pr_init_kernel(const float* __restrict__ inv, uint32_t n, float r0, float* __restrict__ box) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) box[v] = r0 * inv[v];
}

__global__ void fill_kernel(float* __restrict__ out, uint32_t n, float value) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) out[v] = value;
}

__global__ void unpermute_kernel(const float* __restrict__ in, const uint32_t* __restrict__ inv, uint32_t n,
                                 float* __restrict__ out) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) out[v] = in[inv[v]];
}

// staged engine: the message of in-edge j0 + k (source ids streamed, outboxes gathered)
struct PrGather {
    const uint32_t* __restrict__ src;
    const float* __restrict__ box;
    template <int kThreads, int kItems>
    __device__ __forceinline__ void stage(uint64_t j0, uint32_t E, int tid, float* s_val) const {
        uint32_t u[kItems];
#pragma unroll
        for (int q = 0; q < kItems; ++q) {
            const uint32_t k = tid + q * kThreads;
            u[q] = k < E ? __ldcs(src + j0 + k) : 0u;
        }
#pragma unroll
        for (int q = 0; q < kItems; ++q) {
            const uint32_t k = tid + q * kThreads;
            if (k < E) s_val[mp_pad(k)] = __ldg(box + u[q]);
        }
    }
};

// direct engine: messages of a thread's in-edges j0 + eidx[q], the senders' outboxes.  The
// source ids are streamed (read once, evict-first), the outboxes gathered
// through L1.  Every load is issued unconditionally so that all of them are in
// flight at once; an item that is not an edge loads edge j0 (the tile has at
// least one edge when this is called) and its value is ignored.
struct PrMsg {
    const uint32_t* __restrict__ src;
    const float* __restrict__ box;
    template <int kItems>
    __device__ __forceinline__ void fetch(uint64_t j0, uint32_t emask, const uint32_t* eidx, float* x) const {
        uint32_t u[kItems];
#pragma unroll
        for (int q = 0; q < kItems; ++q) u[q] = __ldcs(src + j0 + ((emask >> q) & 1u ? eidx[q] : 0u));
#pragma unroll
        for (int q = 0; q < kItems; ++q) x[q] = __ldg(box + u[q]);
    }
};

// rank = 0.15/N + 0.85 * sum; outbox = rank / outdeg; the rank itself only in the last superstep
template <bool kFinal>
struct PrEmit {
    const float* __restrict__ inv_outdeg;
    float* __restrict__ box_out;
    float* __restrict__ rank_out;
    float base, damp;
    __device__ __forceinline__ void operator()(uint32_t row, float sum) const {
        const float r = fmaf(damp, sum, base);
        box_out[row] = r * __ldg(inv_outdeg + row);
        if (kFinal) rank_out[row] = r;
    }
};

// kThreads threads per CTA, each walking 2048 / kThreads merge items of a tile;
// kDirect selects the direct engine (messages loaded into registers) over the
// staged one (messages staged in shared memory).  Both sum in the same order.
template <bool kFinal, int kThreads, bool kDirect>
__global__ void __launch_bounds__(kThreads) pr_pull_kernel(
    const uint64_t* __restrict__ csc_off, const uint32_t* __restrict__ csc_src, const float* __restrict__ box_in,
    const float* __restrict__ inv_outdeg, float* __restrict__ box_out, float* __restrict__ rank_out,
    const uint32_t* __restrict__ tile_row, float* __restrict__ tile_head, float* __restrict__ tile_tail,
    uint64_t tiles, uint32_t n, uint64_t m, float base, float damp) {
    constexpr int kItems = (int)kMpTile / kThreads;
    PrEmit<kFinal> emit{inv_outdeg, box_out, rank_out, base, damp};
    if (kDirect) {
        __shared__ MpDirectShared<kThreads, float> sh;
        mp_direct_init(sh);
        const PrMsg msg{csc_src, box_in};
        for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x)
            mp_tile_direct<kThreads, kItems, SumF32>(sh, csc_off, n, m, tile_row, tile, tile_head, tile_tail, msg,
                                                     emit);
    } else {
        __shared__ MpShared<kThreads, kItems, float> sh;
        PrGather gather{csc_src, box_in};
        for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x)
            mp_tile<kThreads, kItems, SumF32>(sh, csc_off, n, m, tile_row, tile, tile_head, tile_tail, gather, emit);
    }
}

// rows whose in-edges span several tiles: the partial sums, added in tile order in double precision
template <bool kFinal>
__global__ void pr_fixup_kernel(const uint64_t* __restrict__ csc_off, const uint32_t* __restrict__ tile_row,
                                const float* __restrict__ tile_head, const float* __restrict__ tile_tail,
                                const float* __restrict__ inv_outdeg, float* __restrict__ box_out,
                                float* __restrict__ rank_out, uint64_t tiles, uint32_t n, float base, float damp) {
    PrEmit<kFinal> emit{inv_outdeg, box_out, rank_out, base, damp};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tiles; t += stride) {
        uint32_t row;
        uint64_t q;
        if (!mp_fixup_span(csc_off, tile_row, t, n, &row, &q)) continue;
        double acc = 0.0;
        for (; q < t; ++q) acc += (double)tile_tail[q];
        acc += (double)tile_head[t];
        emit(row, (float)acc);
    }
}

ipg_status pr_prepare(ipg_graph* g, cudaStream_t st) {
    IPG_TRY(ensure_csc(g, st));
    const uint32_t n = g->n;
    if (!g->inv_outdeg) {
        IPG_CUDA(cudaMalloc(&g->inv_outdeg, sizeof(float) * (n ? n : 1)));
        inv_outdeg_kernel<<<grid_cap(n), 256, 0, st>>>(g->off, n, g->inv_outdeg);
        IPG_CUDA(cudaGetLastError());
    }
    for (int b = 0; b < 2; ++b)
        if (!g->pr_box[b]) IPG_CUDA(cudaMalloc(&g->pr_box[b], sizeof(float) * (n ? n : 1)));
    if (!g->pr_rank) IPG_CUDA(cudaMalloc(&g->pr_rank, sizeof(float) * (n ? n : 1)));
    IPG_TRY(ensure_pull_partition(g, st));
    return IPG_OK;
}

// Launch shape of the pull kernel: engine (knob pr_engine: 0 staged, 1 direct),
// threads per CTA (knob pr_threads: 256 or 512), the shared-memory carveout
// (knob pr_carveout: -1 = the smallest that keeps full occupancy, leaving the
// rest of the unified array to L1; 0..100 = that percentage) and the grid
// (every resident CTA, persistent over tiles).  Only speed depends on it.
struct PrLaunch {
    int threads = 256;
    bool direct = false;
    unsigned grid = 1;
};

template <bool kFinal>
static const void* pr_kernel_for(int threads, bool direct) {
    if (direct)
        return threads == 512 ? reinterpret_cast<const void*>(&pr_pull_kernel<kFinal, 512, true>)
                              : reinterpret_cast<const void*>(&pr_pull_kernel<kFinal, 256, true>);
    return threads == 512 ? reinterpret_cast<const void*>(&pr_pull_kernel<kFinal, 512, false>)
                          : reinterpret_cast<const void*>(&pr_pull_kernel<kFinal, 256, false>);
}

ipg_status pr_launch_shape(ipg_graph* g, PrLaunch* L) {
    const Tuning& tu = tuning();
    L->threads = tu.pr_threads == 512 ? 512 : 256;
    L->direct = pr_engine_for(g) == 1;
    const void* k[2] = {pr_kernel_for<false>(L->threads, L->direct), pr_kernel_for<true>(L->threads, L->direct)};
    return pull_grid(k, 2, L->threads, g->device, g->pr_tiles, (int)pr_carveout_for(g), &L->grid);
}

template <bool kFinal, int kThreads, bool kDirect>
static void pr_launch1(const PrLaunch& L, ipg_graph* g, const float* in, float* outb, cudaStream_t st, float base,
                       float damp) {
    pr_pull_kernel<kFinal, kThreads, kDirect><<<L.grid, kThreads, 0, st>>>(
        g->csc_off, g->csc_src, in, g->inv_outdeg, outb, g->pr_rank, g->pr_tile_row, g->pr_head, g->pr_tail,
        g->pr_tiles, g->n, g->m, base, damp);
}

template <bool kFinal>
static void pr_launch(const PrLaunch& L, ipg_graph* g, const float* in, float* outb, cudaStream_t st, float base,
                      float damp) {
    if (L.direct) {
        if (L.threads == 512)
            pr_launch1<kFinal, 512, true>(L, g, in, outb, st, base, damp);
        else
            pr_launch1<kFinal, 256, true>(L, g, in, outb, st, base, damp);
    } else {
        if (L.threads == 512)
            pr_launch1<kFinal, 512, false>(L, g, in, outb, st, base, damp);
        else
            pr_launch1<kFinal, 256, false>(L, g, in, outb, st, base, damp);
    }
}

}  // namespace

// Enqueues PageRank's `updates` supersteps (initial outbox, then pull + fix-up per
// superstep) on st; the final ranks land in g->pr_rank.
static ipg_status pr_enqueue_loop(ipg_graph* g, const PrLaunch& L, uint32_t updates, float base, float damp,
                                  cudaStream_t st) {
    const uint32_t n = g->n;
    pr_init_kernel<<<grid_cap(n), 256, 0, st>>>(g->inv_outdeg, n, 1.0f / (float)n, g->pr_box[0]);
    int cur = 0;
    for (uint32_t t = 1; t <= updates; ++t) {
        const bool fin = t == updates;
        const float* in = g->pr_box[cur];
        float* outb = g->pr_box[cur ^ 1];
        if (fin)
            pr_launch<true>(L, g, in, outb, st, base, damp);
        else
            pr_launch<false>(L, g, in, outb, st, base, damp);
        const unsigned fg = grid_cap(g->pr_tiles);
        if (fin)
            pr_fixup_kernel<true><<<fg, 256, 0, st>>>(g->csc_off, g->pr_tile_row, g->pr_head, g->pr_tail,
                                                      g->inv_outdeg, outb, g->pr_rank, g->pr_tiles, n, base, damp);
        else
            pr_fixup_kernel<false><<<fg, 256, 0, st>>>(g->csc_off, g->pr_tile_row, g->pr_head, g->pr_tail,
                                                       g->inv_outdeg, outb, g->pr_rank, g->pr_tiles, n, base, damp);
        cur ^= 1;
    }
    IPG_CUDA(cudaGetLastError());
    return IPG_OK;
}

// Captures the superstep loop into g->pr_exec unless one for the same update
// count and launch shape exists.  The graph refers to the graph's own buffers
// only (never to a caller's), and is destroyed with them.
ipg_status pr_loop_graph(ipg_graph* g, uint32_t updates, float base, float damp) {
    PrLaunch L;
    IPG_TRY(pr_launch_shape(g, &L));
    const uint64_t key = ((uint64_t)updates << 32) ^ ((uint64_t)L.grid << 8) ^ ((uint64_t)L.threads << 1) ^
                         (uint64_t)L.direct ^ ((uint64_t)(pr_carveout_for(g) + 1) << 20);
    if (g->pr_exec && g->pr_exec_key == key) return IPG_OK;
    if (g->pr_exec) cudaGraphExecDestroy(g->pr_exec);
    g->pr_exec = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    IPG_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    ipg_status rc = IPG_OK;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = pr_enqueue_loop(g, L, updates, base, damp, cap);
        e = cudaStreamEndCapture(cap, &graph);
        if (rc == IPG_OK && e == cudaSuccess) e = cudaGraphInstantiate(&g->pr_exec, graph, 0);
    }
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    if (rc != IPG_OK) return rc;
    if (e != cudaSuccess) {
        g->pr_exec = nullptr;
        return cuda_fail(e, "PageRank superstep graph", __FILE__, __LINE__);
    }
    g->pr_exec_key = key;
    return IPG_OK;
}

// events for per-superstep timing (per host thread)
static thread_local cudaEvent_t* t_events = nullptr;
static thread_local size_t t_events_cap = 0;

ipg_status ensure_events(ipg_graph*, size_t count, cudaEvent_t** evs) {
    if (count > t_events_cap) {
        cudaEvent_t* nv = new cudaEvent_t[count];
        for (size_t i = 0; i < t_events_cap; ++i) nv[i] = t_events[i];
        for (size_t i = t_events_cap; i < count; ++i) IPG_CUDA(cudaEventCreate(&nv[i]));
        delete[] t_events;
        t_events = nv;
        t_events_cap = count;
    }
    *evs = t_events;
    return IPG_OK;
}

static ipg_status pagerank_run(ipg_graph* g, uint32_t updates, float* ranks_dev, ipg_stats* stats,
                               cudaStream_t st) {
    stats_begin(stats);
    if (!g) return set_error(IPG_EINVAL, "ipg_pagerank: graph is NULL");
    if (g->n && !ranks_dev) return set_error(IPG_EINVAL, "ipg_pagerank: output is NULL");
    DeviceGuard guard(g->device);
    if (!guard.ok) return set_error(IPG_ECUDA, "ipg_pagerank: cannot select the graph's device");
    const uint32_t n = g->n;
    const uint64_t m = g->m;
    const bool timing = stats && (stats->flags & IPG_STAT_TIMING);
    const bool recv = stats && (stats->flags & IPG_STAT_RECEIVERS);
    const float N = (float)n;
    const float base = n ? 0.15f / N : 0.f;
    const float damp = 0.85f;
    cudaEvent_t* ev = nullptr;
    if (n) {
        IPG_TRY(pr_prepare(g, st));
        if (recv) IPG_TRY(count_in_nonempty(g, st));
        if (timing) IPG_TRY(ensure_events(g, 3 * (size_t)updates + 1, &ev));
        if (updates == 0) {
            fill_kernel<<<grid_cap(n), 256, 0, st>>>(ranks_dev, n, 1.0f / N);
            IPG_CUDA(cudaGetLastError());
        } else if (!timing) {
            // the whole superstep loop as one captured graph (built once per shape)
            IPG_TRY(pr_loop_graph(g, updates, base, damp));
            IPG_CUDA(cudaGraphLaunch(g->pr_exec, st));
            unpermute_kernel<<<grid_cap(n), 256, 0, st>>>(g->pr_rank, g->inv, n, ranks_dev);
            IPG_CUDA(cudaGetLastError());
        } else {
            pr_init_kernel<<<grid_cap(n), 256, 0, st>>>(g->inv_outdeg, n, 1.0f / N, g->pr_box[0]);
            IPG_CUDA(cudaGetLastError());
            const uint64_t tiles = g->pr_tiles;
            PrLaunch L;
            IPG_TRY(pr_launch_shape(g, &L));
            int cur = 0;
            for (uint32_t t = 1; t <= updates; ++t) {
                const bool fin = t == updates;
                const float* in = g->pr_box[cur];
                float* outb = g->pr_box[cur ^ 1];
                if (timing) IPG_CUDA(cudaEventRecord(ev[3 * (t - 1)], st));
                if (fin)
                    pr_launch<true>(L, g, in, outb, st, base, damp);
                else
                    pr_launch<false>(L, g, in, outb, st, base, damp);
                IPG_CUDA(cudaGetLastError());
                if (timing) IPG_CUDA(cudaEventRecord(ev[3 * (t - 1) + 1], st));
                if (fin)
                    pr_fixup_kernel<true><<<grid_cap(tiles), 256, 0, st>>>(g->csc_off, g->pr_tile_row, g->pr_head,
                                                                           g->pr_tail, g->inv_outdeg, outb,
                                                                           g->pr_rank, tiles, n, base, damp);
                else
                    pr_fixup_kernel<false><<<grid_cap(tiles), 256, 0, st>>>(g->csc_off, g->pr_tile_row, g->pr_head,
                                                                            g->pr_tail, g->inv_outdeg, outb,
                                                                            g->pr_rank, tiles, n, base, damp);
                IPG_CUDA(cudaGetLastError());
                if (timing) IPG_CUDA(cudaEventRecord(ev[3 * (t - 1) + 2], st));
                cur ^= 1;
            }
            unpermute_kernel<<<grid_cap(n), 256, 0, st>>>(g->pr_rank, g->inv, n, ranks_dev);
            IPG_CUDA(cudaGetLastError());
        }
        IPG_CUDA(cudaStreamSynchronize(st));
    }
    // Pregel numbering: superstep 0 sends the initial ranks, superstep t applies update t
    if (stats) {
        for (uint32_t s = 0; s <= updates; ++s) {
            ipg_superstep_stats r{};
            r.superstep = s;
            r.flags = (recv ? IPG_STAT_RECEIVERS : 0u) | (timing && n && s < updates ? IPG_STAT_TIMING : 0u);
            r.active = n;
            r.senders = s < updates ? n : 0;
            r.messages_sent = s < updates ? m : 0;
            r.receivers = (recv && s < updates) ? (uint64_t)g->in_nonempty : 0;
            if (timing && n && s < updates) {
                float a = 0.f, b = 0.f;
                cudaEventElapsedTime(&a, ev[3 * s], ev[3 * s + 1]);
                cudaEventElapsedTime(&b, ev[3 * s], ev[3 * s + 2]);
                r.kernel_ms = a;
                r.superstep_ms = b;
            }
            stats_put(stats, s, r);
        }
        stats->count = updates + 1;
    }
    return IPG_OK;
}

}  // namespace ipg

using namespace ipg;

extern "C" {

ipg_status ipg_pagerank_dev(ipg_graph* g, uint32_t updates, float* ranks_dev, ipg_stats* stats, void* stream) {
    return pagerank_run(g, updates, ranks_dev, stats, (cudaStream_t)stream);
}

ipg_status ipg_pagerank(ipg_graph* g, uint32_t updates, float* ranks_out, ipg_stats* stats) {
    stats_begin(stats);
    if (!g) return set_error(IPG_EINVAL, "ipg_pagerank: graph is NULL");
    if (g->n && !ranks_out) return set_error(IPG_EINVAL, "ipg_pagerank: output is NULL");
    DeviceGuard guard(g->device);
    IPG_TRY(ensure(&g->pr_out_stage, &g->pr_out_stage_cap, (size_t)g->n));
    IPG_TRY(pagerank_run(g, updates, g->pr_out_stage, stats, g->stream));
    if (g->n) {
        IPG_CUDA(cudaMemcpyAsync(ranks_out, g->pr_out_stage, sizeof(float) * g->n, cudaMemcpyDeviceToHost,
                                 g->stream));
        IPG_CUDA(cudaStreamSynchronize(g->stream));
    }
    return IPG_OK;
}

}  // extern "C"
