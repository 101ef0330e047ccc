// Pull form of a min-combiner superstep (Hashmin, SSSP), used when the frontier
// is dense.  Push costs a random read and often an atomic per message; when most
// vertices send, it is cheaper to let every vertex scan its in-edges, as the
// paper's pull-based "single broadcast" version does for CC (Sec. VI-C), and to
// reuse PageRank's merge-path tile engine with a min instead of a sum.
//
// Superstep s in pull form:
//   sval[u] = value u sends in s (its snapshot, kInf if u is not a sender);
//   for every vertex v:  m = min over in-edges (u -> v) of sval[u] (+ w(u,v));
//   if m < val[v]: val[v] = m and v joins the next frontier.
// This is the same synchronous superstep as the push form — same values, same
// next frontier, same counts — because both take the minimum of the same
// messages and activate on the same strict drop.
// When a minority of the edges carry messages, the superstep is filtered: a
// one-bit-per-vertex sender array (n/8 bytes, cached in L1 and L2) is read
// first, and only in-edges whose source sends gather its value; the others
// contribute kInf without touching the value array.  Each vertex is finished by
// exactly one thread (min is exact and order-free), so no atomics on values are
// needed; next-frontier appends go through a per-CTA shared-memory queue.
#include "ipg_mergepath.cuh"

namespace ipg {
namespace {

constexpr int kPmThreads = 256;
constexpr int kPmItems = 8;

// loop-driven supersteps (loop != NULL) return at once unless they run in pull form
__device__ __forceinline__ bool pull_skip(const PushLoop* loop) { return loop && !loop->pull; }

__global__ void sval_fill_kernel(uint32_t* __restrict__ sval, uint32_t* __restrict__ sbits, uint32_t n,
                                 const PushLoop* __restrict__ loop) {
    if (pull_skip(loop)) return;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) sval[i] = kInf;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n / 32; i += stride) sbits[i] = 0;
}

__global__ void sval_scatter_kernel(const uint32_t* F0, const uint32_t* F1, const uint32_t* __restrict__ fval,
                                    uint32_t f, const PushLoop* __restrict__ loop, uint32_t* __restrict__ sval,
                                    uint32_t* __restrict__ sbits) {
    if (pull_skip(loop)) return;
    const uint32_t* __restrict__ F = loop_frontier(F0, F1, loop);
    f = loop_f(f, loop);
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < f; i += stride) {
        const uint32_t u = F[i];
        sval[u] = fval[i];
        atomicOr(&sbits[u >> 5], 1u << (u & 31));
    }
}

// message carried by in-edge j0 + k (kInf when its source does not send)
template <bool kAddWeight, int kWeightKind>
struct PmGather {
    const uint32_t* __restrict__ src;
    const uint8_t* __restrict__ w8;
    const uint32_t* __restrict__ w32;
    const uint32_t* __restrict__ sval;
    const uint32_t* __restrict__ sbits;
    bool filter;  // read the sender bit before gathering (uniform over the grid)
    unsigned int* status;
    template <int kThreads, int kItems>
    __device__ __forceinline__ void stage(uint64_t j0, uint32_t E, int tid, uint32_t* s_val) const {
        uint32_t u[kItems], w[kItems];
#pragma unroll
        for (int q = 0; q < kItems; ++q) {
            const uint32_t k = tid + q * kThreads;
            u[q] = k < E ? __ldcs(src + j0 + k) : 0u;
            w[q] = 1u;
            if (kAddWeight && kWeightKind == 1 && k < E) w[q] = __ldcs(w8 + j0 + k);
            if (kAddWeight && kWeightKind == 2 && k < E) w[q] = __ldcs(w32 + j0 + k);
        }
        bool sends[kItems];
#pragma unroll
        for (int q = 0; q < kItems; ++q) sends[q] = true;
        if (filter) {
            uint32_t bits[kItems];
#pragma unroll
            for (int q = 0; q < kItems; ++q) bits[q] = tid + q * kThreads < E ? __ldg(sbits + (u[q] >> 5)) : 0u;
#pragma unroll
            for (int q = 0; q < kItems; ++q) sends[q] = (bits[q] >> (u[q] & 31)) & 1u;
        }
#pragma unroll
        for (int q = 0; q < kItems; ++q) {
            const uint32_t k = tid + q * kThreads;
            if (k < E) {
                const uint32_t s = sends[q] ? __ldg(sval + u[q]) : kInf;
                uint32_t msg = s;
                if (kAddWeight && s != kInf) {
                    unsigned long long d = (unsigned long long)s + w[q];
                    if (d >= kInf) {
                        atomicOr(status, kStatusOverflow);
                        d = kInf - 1;
                    }
                    msg = (uint32_t)d;
                }
                s_val[mp_pad(k)] = msg;
            }
        }
    }
};

// A strict drop lowers the value and queues the vertex for the next frontier in
// shared memory; the CTA flushes its queue with one atomic per tile.  Only a
// row that began in this tile can be emitted here, and it can drop only if it
// has an in-edge in the tile, so a tile emits at most min(R, E) <= kMpTile / 2
// drops and the queue never fills; a full queue would append straight to the
// global frontier.
constexpr unsigned kPmQueue = kMpTile / 2;

template <bool kRecv>
struct PmEmit {
    uint32_t* __restrict__ val;
    uint32_t* q;          // shared-memory queue of this tile's new frontier vertices
    unsigned int* qn;     // shared-memory queue length
    unsigned int* nrecv;  // shared-memory receiver count
    uint32_t* next0;      // the next frontier: picked at each use, see loop_next
    uint32_t* next1;
    const PushLoop* loop;
    PushCounters* ctr;
    __device__ __forceinline__ void operator()(uint32_t row, uint32_t m) const {
        if (kRecv && m != kInf) atomicAdd(nrecv, 1u);
        if (m < val[row]) {
            val[row] = m;
            const unsigned slot = atomicAdd(qn, 1u);
            if (slot < kPmQueue)
                q[slot] = row;
            else
                loop_next(next0, next1, loop)[atomicAdd(&ctr->next_size, 1u)] = row;
        }
    }
};

template <bool kAddWeight, int kWeightKind, bool kRecv>
__global__ void __launch_bounds__(kPmThreads) pull_min_kernel(
    const uint64_t* __restrict__ csc_off, const uint32_t* __restrict__ csc_src, const uint8_t* __restrict__ csc_w8,
    const uint32_t* __restrict__ csc_w32, const uint32_t* __restrict__ sval, const uint32_t* __restrict__ sbits,
    bool filter, uint32_t* __restrict__ val, const uint32_t* __restrict__ tile_row, uint32_t* __restrict__ tile_head,
    uint32_t* __restrict__ tile_tail, uint64_t tiles, uint32_t n, uint64_t m, uint32_t* next0, uint32_t* next1,
    const PushLoop* __restrict__ loop, PushCounters* __restrict__ ctr) {
    if (pull_skip(loop)) return;
    if (loop) filter = loop->filter != 0;
    __shared__ MpShared<kPmThreads, kPmItems, uint32_t> sh;
    __shared__ uint32_t s_q[kPmQueue];
    __shared__ unsigned int s_qn, s_recv, s_base;
    if (threadIdx.x == 0) {
        s_qn = 0;
        s_recv = 0;
    }
    PmGather<kAddWeight, kWeightKind> gather{csc_src, csc_w8, csc_w32, sval, sbits, filter, &ctr->status};
    PmEmit<kRecv> emit{val, s_q, &s_qn, &s_recv, next0, next1, loop, ctr};
    for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        mp_tile<kPmThreads, kPmItems, MinU32>(sh, csc_off, n, m, tile_row, tile, tile_head, tile_tail, gather, emit);
        __syncthreads();
        const unsigned qn = min(s_qn, kPmQueue);
        if (qn) {
            if (threadIdx.x == 0) s_base = atomicAdd(&ctr->next_size, qn);
            __syncthreads();
            const unsigned base = s_base;
            uint32_t* __restrict__ next = loop_next(next0, next1, loop);  // picked here: no register for the tile walk
            for (unsigned k = threadIdx.x; k < qn; k += kPmThreads) next[base + k] = s_q[k];
            __syncthreads();
            if (threadIdx.x == 0) s_qn = 0;
        }
    }
    if (kRecv) {
        __syncthreads();
        if (threadIdx.x == 0 && s_recv) atomicAdd(&ctr->receivers, (unsigned long long)s_recv);
    }
}

template <bool kRecv>
__global__ void pull_min_fixup_kernel(const uint64_t* __restrict__ csc_off, const uint32_t* __restrict__ tile_row,
                                      const uint32_t* __restrict__ tile_head, const uint32_t* __restrict__ tile_tail,
                                      uint32_t* __restrict__ val, uint64_t tiles, uint32_t n, uint32_t* next0,
                                      uint32_t* next1, const PushLoop* __restrict__ loop,
                                      PushCounters* __restrict__ ctr) {
    if (pull_skip(loop)) return;
    uint32_t* __restrict__ next = loop_next(next0, next1, loop);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tiles; t += stride) {
        uint32_t row;
        uint64_t q;
        if (!mp_fixup_span(csc_off, tile_row, t, n, &row, &q)) continue;
        uint32_t mn = kInf;
        for (; q < t; ++q) mn = min(mn, tile_tail[q]);
        mn = min(mn, tile_head[t]);
        if (kRecv && mn != kInf) atomicAdd(&ctr->receivers, 1ull);
        if (mn < val[row]) {
            val[row] = mn;
            next[atomicAdd(&ctr->next_size, 1u)] = row;
        }
    }
}

template <bool kAddWeight, int kWeightKind, bool kRecv>
ipg_status launch(ipg_graph* g, bool filter, uint32_t* val, uint32_t* next0, uint32_t* next1, const PushLoop* loop,
                  cudaStream_t st) {
    const void* k = reinterpret_cast<const void*>(&pull_min_kernel<kAddWeight, kWeightKind, kRecv>);
    unsigned grid = 1;
    IPG_TRY(pull_grid(&k, 1, kPmThreads, g->device, g->pr_tiles, (int)pr_carveout_for(g), &grid));
    pull_min_kernel<kAddWeight, kWeightKind, kRecv><<<grid, kPmThreads, 0, st>>>(
        g->csc_off, g->csc_src, g->csc_w8, g->csc_w, g->sval, g->sbits, filter, val, g->pr_tile_row,
        (uint32_t*)g->pr_head,
        (uint32_t*)g->pr_tail, g->pr_tiles, g->n, g->m, next0, next1, loop, g->counters);
    IPG_CUDA(cudaGetLastError());
    return IPG_OK;
}

template <bool kAddWeight, int kWeightKind>
ipg_status launch2(bool recv, ipg_graph* g, bool filter, uint32_t* val, uint32_t* next0, uint32_t* next1,
                   const PushLoop* loop, cudaStream_t st) {
    return recv ? launch<kAddWeight, kWeightKind, true>(g, filter, val, next0, next1, loop, st)
                : launch<kAddWeight, kWeightKind, false>(g, filter, val, next0, next1, loop, st);
}

ipg_status launch_any(ipg_graph* g, bool sssp, bool recv, bool filter, uint32_t* val, uint32_t* next0,
                      uint32_t* next1, const PushLoop* loop, cudaStream_t st) {
    if (!sssp) return launch2<false, 0>(recv, g, filter, val, next0, next1, loop, st);
    if (g->csc_w8) return launch2<true, 1>(recv, g, filter, val, next0, next1, loop, st);
    if (g->csc_w) return launch2<true, 2>(recv, g, filter, val, next0, next1, loop, st);
    return launch2<true, 0>(recv, g, filter, val, next0, next1, loop, st);
}

unsigned small_grid(uint64_t work) {
    uint64_t b = (work + 255) / 256;
    if (b < 1) b = 1;
    const uint64_t cap = (uint64_t)sm_count_current() * 16;
    return (unsigned)(b < cap ? b : cap);
}

void launch_fixup(ipg_graph* g, bool recv, uint32_t* val, uint32_t* next0, uint32_t* next1, const PushLoop* loop,
                  cudaStream_t st) {
    if (recv)
        pull_min_fixup_kernel<true><<<small_grid(g->pr_tiles), 256, 0, st>>>(
            g->csc_off, g->pr_tile_row, (const uint32_t*)g->pr_head, (const uint32_t*)g->pr_tail, val, g->pr_tiles,
            g->n, next0, next1, loop, g->counters);
    else
        pull_min_fixup_kernel<false><<<small_grid(g->pr_tiles), 256, 0, st>>>(
            g->csc_off, g->pr_tile_row, (const uint32_t*)g->pr_head, (const uint32_t*)g->pr_tail, val, g->pr_tiles,
            g->n, next0, next1, loop, g->counters);
}


}  // namespace

ipg_status pull_min_prepare(ipg_graph* g, cudaStream_t st) {
    IPG_TRY(ensure_pull_partition(g, st));
    if (!g->sval) IPG_CUDA(cudaMalloc(&g->sval, sizeof(uint32_t) * (g->n ? g->n : 1)));
    if (!g->sbits) IPG_CUDA(cudaMalloc(&g->sbits, sizeof(uint32_t) * ((size_t)g->n / 32 + 1)));
    return IPG_OK;
}

// one pull superstep; the frontier F (f vertices) and its value snapshot fval are
// the senders; new frontier vertices are appended to next via g->counters
ipg_status pull_min_superstep(ipg_graph* g, bool sssp, bool recv, bool filter, const uint32_t* F,
                              const uint32_t* fval, uint32_t f, uint32_t* val, uint32_t* next, cudaStream_t st,
                              cudaEvent_t ev_kernel) {
    IPG_TRY(pull_min_prepare(g, st));
    IPG_CUDA(cudaMemsetAsync(g->sval, 0xFF, sizeof(uint32_t) * g->n, st));
    IPG_CUDA(cudaMemsetAsync(g->sbits, 0, sizeof(uint32_t) * ((size_t)g->n / 32 + 1), st));
    sval_scatter_kernel<<<small_grid(f), 256, 0, st>>>(F, F, fval, f, nullptr, g->sval, g->sbits);
    IPG_CUDA(cudaGetLastError());
    if (ev_kernel) IPG_CUDA(cudaEventRecord(ev_kernel, st));
    IPG_TRY(launch_any(g, sssp, recv, filter, val, next, next, nullptr, st));
    launch_fixup(g, recv, val, next, next, nullptr, st);
    IPG_CUDA(cudaGetLastError());
    return IPG_OK;
}

// the same superstep with sizes and frontiers read from g->loop (graph capture)
ipg_status pull_min_enqueue_loop(ipg_graph* g, bool sssp, bool recv, uint32_t* val, cudaStream_t st) {
    const unsigned fixed = (unsigned)sm_count_of(g->device) * 8;
    sval_fill_kernel<<<fixed, 256, 0, st>>>(g->sval, g->sbits, g->n, g->loop);
    sval_scatter_kernel<<<fixed, 256, 0, st>>>(g->frontier[0], g->frontier[1], g->fr_val, 0, g->loop, g->sval,
                                               g->sbits);
    IPG_CUDA(cudaGetLastError());
    IPG_TRY(launch_any(g, sssp, recv, false, val, g->frontier[0], g->frontier[1], g->loop, st));
    launch_fixup(g, recv, val, g->frontier[0], g->frontier[1], g->loop, st);
    IPG_CUDA(cudaGetLastError());
    return IPG_OK;
}

}  // namespace ipg
