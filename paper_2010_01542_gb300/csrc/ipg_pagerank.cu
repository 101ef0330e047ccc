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
#include "ipg_internal.cuh"

namespace ipg {
namespace {

constexpr int kPrThreads = 256;
constexpr int kPrItems = 8;
constexpr uint32_t kPrTile = kPrThreads * kPrItems;

// number of row ends consumed at merge-path diagonal `diag` (Merrill & Garland
// merge-path search; row_end[i] = end offset of row i)
__device__ __forceinline__ uint32_t merge_path_rows(const uint64_t* __restrict__ row_end, uint32_t nrows,
                                                    uint64_t nedges, uint64_t diag) {
    uint64_t lo = diag > nedges ? diag - nedges : 0;
    uint64_t hi = diag < nrows ? diag : nrows;
    while (lo < hi) {
        uint64_t mid = (lo + hi) >> 1;
        if (row_end[mid] <= diag - mid - 1)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (uint32_t)lo;
}

__global__ void pr_partition_kernel(const uint64_t* __restrict__ csc_off, uint32_t n, uint64_t m, uint64_t tiles,
                                    uint32_t* __restrict__ tile_row) {
    uint64_t total = (uint64_t)n + m;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= tiles; t += stride) {
        uint64_t diag = t * kPrTile;
        if (diag > total) diag = total;
        tile_row[t] = merge_path_rows(csc_off + 1, n, m, diag);
    }
}

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

template <bool kFinal>
__global__ void __launch_bounds__(kPrThreads) pr_pull_kernel(
    const uint64_t* __restrict__ csc_off, const uint32_t* __restrict__ csc_src, const float* __restrict__ box_in,
    const float* __restrict__ inv_outdeg, float* __restrict__ box_out, float* __restrict__ rank_out,
    const uint32_t* __restrict__ tile_row, float* __restrict__ tile_head, float* __restrict__ tile_tail, uint32_t n,
    uint64_t m, float base, float damp) {
    __shared__ uint32_t s_end[kPrTile + 1];
    __shared__ float s_val[kPrTile];
    __shared__ float s_wsum[kPrThreads / 32];
    __shared__ int s_wflag[kPrThreads / 32];
    __shared__ unsigned long long s_first_start;

    const uint64_t tile = blockIdx.x;
    const uint64_t total = (uint64_t)n + m;
    const uint64_t d0 = tile * kPrTile;
    const uint64_t d1 = d0 + kPrTile < total ? d0 + kPrTile : total;
    const uint32_t i0 = tile_row[tile];
    const uint32_t i1 = tile_row[tile + 1];
    const uint64_t j0 = d0 - i0;
    const uint32_t R = i1 - i0;
    const uint32_t E = (uint32_t)((d1 - i1) - j0);
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;

    // 1. stage: row ends relative to j0 (clamped past the tile), then gathered outboxes
    for (uint32_t k = tid; k <= R; k += kPrThreads) {
        uint32_t row = i0 + k;
        uint64_t rel = row < n ? csc_off[row + 1] - j0 : (uint64_t)E + 1;
        s_end[k] = rel < (uint64_t)E + 1 ? (uint32_t)rel : E + 1;
    }
    if (tid == 0) s_first_start = i0 < n ? csc_off[i0] : m;
    uint32_t src[kPrItems];
#pragma unroll
    for (int q = 0; q < kPrItems; ++q) {
        uint32_t k = tid + q * kPrThreads;
        src[q] = k < E ? __ldcs(csc_src + j0 + k) : 0u;
    }
#pragma unroll
    for (int q = 0; q < kPrItems; ++q) {
        uint32_t k = tid + q * kPrThreads;
        if (k < E) s_val[k] = __ldg(box_in + src[q]);
    }
    __syncthreads();

    // 2. this thread's slice of the tile's merge path
    const uint32_t items = R + E;
    const uint32_t ds = min((uint32_t)tid * kPrItems, items);
    const uint32_t de = min(ds + kPrItems, items);
    uint32_t lo = ds > E ? ds - E : 0, hi = min(ds, R);
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (s_end[mid] <= ds - mid - 1)
            lo = mid + 1;
        else
            hi = mid;
    }
    const uint32_t ti = lo, tj = ds - lo;

    // pass 1: partial sum of the row this slice ends in, and whether a row ended
    float run = 0.f;
    int ended = 0;
    {
        uint32_t i = ti, j = tj;
        for (uint32_t d = ds; d < de; ++d) {
            if (j < s_end[i]) {
                run += s_val[j];
                ++j;
            } else {
                run = 0.f;
                ++i;
                ended = 1;
            }
        }
    }
    // segmented inclusive scan over threads: (f, v) then (g, w) -> (f|g, g ? w : v + w)
    float v = run;
    int f = ended;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        float vu = __shfl_up_sync(0xFFFFFFFFu, v, o);
        int fu = __shfl_up_sync(0xFFFFFFFFu, f, o);
        if (lane >= o) {
            if (!f) v = vu + v;
            f |= fu;
        }
    }
    if (lane == 31) {
        s_wsum[warp] = v;
        s_wflag[warp] = f;
    }
    __syncthreads();
    float wc = 0.f;
    for (int q = 0; q < warp; ++q) wc = s_wflag[q] ? s_wsum[q] : wc + s_wsum[q];
    const float incl = f ? v : wc + v;
    float excl = __shfl_up_sync(0xFFFFFFFFu, incl, 1);
    if (lane == 0) excl = wc;
    if (tid == kPrThreads - 1) tile_tail[tile] = incl;  // partial of row i1 inside this tile

    // pass 2: walk again from the carry-in and finish every row that ends here
    {
        const bool head_open = s_first_start < j0;  // row i0 began in an earlier tile
        run = excl;
        uint32_t i = ti, j = tj;
        for (uint32_t d = ds; d < de; ++d) {
            if (j < s_end[i]) {
                run += s_val[j];
                ++j;
            } else {
                const uint32_t row = i0 + i;
                if (i == 0 && head_open) {
                    tile_head[tile] = run;
                } else {
                    const float r = fmaf(damp, run, base);
                    box_out[row] = r * __ldg(inv_outdeg + row);
                    if (kFinal) rank_out[row] = r;
                }
                run = 0.f;
                ++i;
            }
        }
    }
}

// rows whose in-edges span several tiles: add the tiles' partial sums in order
template <bool kFinal>
__global__ void pr_fixup_kernel(const uint64_t* __restrict__ csc_off, const uint32_t* __restrict__ tile_row,
                                const float* __restrict__ tile_head, const float* __restrict__ tile_tail,
                                const float* __restrict__ inv_outdeg, float* __restrict__ box_out,
                                float* __restrict__ rank_out, uint64_t tiles, uint32_t n, float base, float damp) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tiles; t += stride) {
        const uint32_t i0 = tile_row[t];
        if (i0 >= n || tile_row[t + 1] == i0) continue;  // no row ends in this tile
        const uint64_t j0 = t * kPrTile - i0;
        if (csc_off[i0] >= j0) continue;  // began here: finished by the pull kernel
        double acc = 0.0;
        uint64_t q = t;
        while (q > 0 && tile_row[q] == i0) --q;  // first tile holding edges of row i0
        for (; q < t; ++q) acc += (double)tile_tail[q];
        acc += (double)tile_head[t];
        const float r = fmaf(damp, (float)acc, base);
        box_out[i0] = r * inv_outdeg[i0];
        if (kFinal) rank_out[i0] = r;
    }
}

unsigned grid_cap(uint64_t work, unsigned cap = 152 * 16) {
    uint64_t b = (work + 255) / 256;
    if (b < 1) b = 1;
    return (unsigned)(b < cap ? b : cap);
}

ipg_status pr_prepare(ipg_graph* g, cudaStream_t st) {
    IPG_TRY(ensure_csc(g, st));
    const uint32_t n = g->n;
    const uint64_t m = g->m;
    if (!g->inv_outdeg) {
        IPG_CUDA(cudaMalloc(&g->inv_outdeg, sizeof(float) * (n ? n : 1)));
        inv_outdeg_kernel<<<grid_cap(n), 256, 0, st>>>(g->off, n, g->inv_outdeg);
        IPG_CUDA(cudaGetLastError());
    }
    for (int b = 0; b < 2; ++b)
        if (!g->pr_box[b]) IPG_CUDA(cudaMalloc(&g->pr_box[b], sizeof(float) * (n ? n : 1)));
    if (!g->pr_tile_row) {
        const uint64_t tiles = ((uint64_t)n + m + kPrTile - 1) / kPrTile;
        IPG_CUDA(cudaMalloc(&g->pr_tile_row, sizeof(uint32_t) * (tiles + 1)));
        IPG_CUDA(cudaMalloc(&g->pr_head, sizeof(float) * (tiles ? tiles : 1)));
        IPG_CUDA(cudaMalloc(&g->pr_tail, sizeof(float) * (tiles ? tiles : 1)));
        pr_partition_kernel<<<grid_cap(tiles + 1), 256, 0, st>>>(g->csc_off, n, m, tiles, g->pr_tile_row);
        IPG_CUDA(cudaGetLastError());
        g->pr_tiles = tiles;
    }
    return IPG_OK;
}

}  // namespace

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
        } else {
            pr_init_kernel<<<grid_cap(n), 256, 0, st>>>(g->inv_outdeg, n, 1.0f / N, g->pr_box[0]);
            IPG_CUDA(cudaGetLastError());
            const uint64_t tiles = g->pr_tiles;
            int cur = 0;
            for (uint32_t t = 1; t <= updates; ++t) {
                const bool fin = t == updates;
                float* in = g->pr_box[cur];
                float* outb = g->pr_box[cur ^ 1];
                if (timing) IPG_CUDA(cudaEventRecord(ev[3 * (t - 1)], st));
                if (tiles) {
                    if (fin)
                        pr_pull_kernel<true><<<(unsigned)tiles, kPrThreads, 0, st>>>(
                            g->csc_off, g->csc_src, in, g->inv_outdeg, outb, ranks_dev, g->pr_tile_row, g->pr_head,
                            g->pr_tail, n, m, base, damp);
                    else
                        pr_pull_kernel<false><<<(unsigned)tiles, kPrThreads, 0, st>>>(
                            g->csc_off, g->csc_src, in, g->inv_outdeg, outb, ranks_dev, g->pr_tile_row, g->pr_head,
                            g->pr_tail, n, m, base, damp);
                    IPG_CUDA(cudaGetLastError());
                }
                if (timing) IPG_CUDA(cudaEventRecord(ev[3 * (t - 1) + 1], st));
                if (fin)
                    pr_fixup_kernel<true><<<grid_cap(tiles), 256, 0, st>>>(g->csc_off, g->pr_tile_row, g->pr_head,
                                                                           g->pr_tail, g->inv_outdeg, outb,
                                                                           ranks_dev, tiles, n, base, damp);
                else
                    pr_fixup_kernel<false><<<grid_cap(tiles), 256, 0, st>>>(g->csc_off, g->pr_tile_row, g->pr_head,
                                                                            g->pr_tail, g->inv_outdeg, outb,
                                                                            ranks_dev, tiles, n, base, damp);
                IPG_CUDA(cudaGetLastError());
                if (timing) IPG_CUDA(cudaEventRecord(ev[3 * (t - 1) + 2], st));
                cur ^= 1;
            }
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
