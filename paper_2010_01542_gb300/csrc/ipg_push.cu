// Push supersteps with a min combiner: Hashmin connected components and SSSP
// (Sec. VI-C).  Both keep an explicit list of the vertices that send in the
// current superstep — the paper's "selection bypass" — instead of scanning
// every vertex.
//
// One superstep s, given the frontier F_s (vertices whose value dropped in
// s-1, or the initial senders in superstep 0):
//   prepare    out-degree of every frontier vertex, an exclusive prefix sum of
//              those degrees (two passes plus a single-CTA scan of the block
//              sums), and a snapshot of each sender's value and row start;
//   partition  merge-path split of (frontier rows + their edges) into tiles of
//              2048 items, so a hub's edges are spread over many CTAs and the
//              split costs one short binary search per tile (the paper's
//              edge-centric split had to be recomputed every superstep and lost
//              on small graphs, Sec. VII-A);
//   relax      one thread per edge: candidate = sender value (+ weight for
//              SSSP); if it is below the receiver's current value, atomicMin.
//              For a u32 min the hardware atomic is the whole combiner: it is
//              lock-free and has no empty-mailbox ambiguity (Sec. III), because
//              the value array itself is the mailbox and only a strict drop
//              activates the receiver.  A thread whose atomicMin lowered the
//              value claims the receiver for F_{s+1} with a per-vertex stamp,
//              and the warp appends its claims with one atomicAdd (ballot +
//              popc).
// Senders' values are snapshotted before the relax kernel, so a value that drops
// during superstep s is sent only in s+1: the run is the synchronous Pregel
// execution, superstep for superstep, and the per-superstep counts match the
// model exactly.
#include <algorithm>
#include <vector>

#include "ipg_internal.cuh"

namespace ipg {
namespace {

constexpr int kFrThreads = 256;
constexpr int kFrItems = 8;
constexpr uint32_t kFrBlock = kFrThreads * kFrItems;
constexpr int kScanThreads = 1024;
constexpr int kPushThreads = 256;
constexpr uint32_t kPushTile = kFrontierTile;

enum Kind { kHashmin = 0, kSssp = 1 };

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long x, unsigned long long* s_tmp) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_tmp[warp] = x;
    __syncthreads();
    unsigned long long t = 0;
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += s_tmp[q];
    return t;  // valid in thread 0
}

// exclusive block scan of one u64 per thread; returns this thread's prefix, *total = block total
__device__ __forceinline__ unsigned long long block_exscan_u64(unsigned long long x, unsigned long long* s_tmp,
                                                               unsigned long long* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    unsigned long long incl = x;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_tmp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < nw ? s_tmp[lane] : 0;
        unsigned long long wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) s_tmp[lane] = wi - w;  // exclusive warp offsets
        if (lane == nw - 1) s_tmp[32] = wi;
    }
    __syncthreads();
    *total = s_tmp[32];
    return s_tmp[warp] + incl - x;
}

// labels are the caller's vertex ids, so the result does not depend on the internal numbering
__global__ void hashmin_init_kernel(uint32_t* __restrict__ val, uint32_t* __restrict__ frontier,
                                    const uint32_t* __restrict__ perm, uint32_t n) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        val[v] = perm[v];
        frontier[v] = (uint32_t)v;
    }
}

// `source` is the caller's id; inv maps it to the internal one
__global__ void sssp_init_kernel(uint32_t* __restrict__ val, uint32_t* __restrict__ frontier, uint32_t n,
                                 const uint32_t* __restrict__ inv, uint32_t source) {
    const uint32_t s = inv[source];
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) val[v] = v == s ? 0u : kInf;
    if (blockIdx.x == 0 && threadIdx.x == 0) frontier[0] = s;
}

// The frontier passes take the frontier from the loop block when one is given
// (loop-driven supersteps in a CUDA graph), else from their arguments, and walk
// the frontier's blocks of kFrBlock entries grid-stride.

// pass 1 of the frontier prefix: one degree total per block of 2048 entries
__global__ void __launch_bounds__(kFrThreads) fr_reduce_kernel(const uint32_t* F0, const uint32_t* F1, uint32_t f,
                                                               const PushLoop* __restrict__ loop,
                                                               const uint64_t* __restrict__ off,
                                                               unsigned long long* __restrict__ block_sums) {
    __shared__ unsigned long long s_tmp[33];
    const uint32_t* __restrict__ F = loop_frontier(F0, F1, loop);
    f = loop_f(f, loop);
    const uint32_t nb = (f + kFrBlock - 1) / kFrBlock;
    for (uint32_t blk = blockIdx.x; blk < nb; blk += gridDim.x) {
        const uint64_t b0 = (uint64_t)blk * kFrBlock;
        unsigned long long d = 0;
#pragma unroll
        for (int q = 0; q < kFrItems; ++q) {
            uint64_t i = b0 + (uint64_t)q * kFrThreads + threadIdx.x;
            if (i < f) {
                uint32_t u = F[i];
                d += off[u + 1] - off[u];
            }
        }
        unsigned long long t = block_sum_u64(d, s_tmp);
        if (threadIdx.x == 0) block_sums[blk] = t;
        __syncthreads();  // s_tmp is reused by the next block
    }
}

// single CTA: exclusive scan of the block totals, edge count and tile count; a
// loop-driven superstep also picks its form here (pull when its messages reach
// m / divisor)
__global__ void __launch_bounds__(kScanThreads) fr_scan_kernel(unsigned long long* __restrict__ block_sums,
                                                               uint32_t nb, uint32_t f, PushLoop* __restrict__ loop,
                                                               uint64_t m, unsigned long long* __restrict__ prefix,
                                                               PushCounters* __restrict__ ctr) {
    __shared__ unsigned long long s_tmp[33];
    f = loop_f(f, loop);
    if (loop) nb = (f + kFrBlock - 1) / kFrBlock;
    const uint32_t per = (nb + kScanThreads - 1) / kScanThreads;
    const uint64_t a = (uint64_t)threadIdx.x * per;
    const uint64_t b = a + per < nb ? a + per : nb;
    unsigned long long s = 0;
    for (uint64_t i = a; i < b; ++i) s += block_sums[i];
    unsigned long long total;
    unsigned long long run = block_exscan_u64(s, s_tmp, &total);
    for (uint64_t i = a; i < b; ++i) {
        unsigned long long x = block_sums[i];
        block_sums[i] = run;
        run += x;
    }
    if (threadIdx.x == 0) {
        prefix[f] = total;
        ctr->edges = total;
        ctr->tiles = (unsigned)(((unsigned long long)f + total + kPushTile - 1) / kPushTile);
        ctr->next_size = 0;
        ctr->receivers = 0;
        if (loop) {
            loop->pull = loop->divisor > 0 && total > 0 && (double)total * (double)loop->divisor >= (double)m;
            loop->filter = loop->pull && (double)total * 100.0 < (double)m * (double)loop->filter_pct;
        }
    }
}

__device__ __forceinline__ void fr_write_block(const uint32_t* __restrict__ F, uint32_t f, uint32_t blk,
                                               const uint64_t* __restrict__ off, const uint32_t* __restrict__ val,
                                               const unsigned long long* __restrict__ block_off,
                                               unsigned long long* __restrict__ prefix,
                                               unsigned long long* __restrict__ rowstart, uint32_t* __restrict__ fval,
                                               unsigned long long* s_tmp) {
    const uint64_t i0 = (uint64_t)blk * kFrBlock + (uint64_t)threadIdx.x * kFrItems;
    uint64_t st[kFrItems];
    unsigned long long deg[kFrItems];
    unsigned long long local = 0;
#pragma unroll
    for (int q = 0; q < kFrItems; ++q) {
        uint64_t i = i0 + q;
        deg[q] = 0;
        st[q] = 0;
        if (i < f) {
            uint32_t u = F[i];
            st[q] = off[u];
            deg[q] = off[u + 1] - st[q];
            if (val) fval[i] = val[u];
        }
        local += deg[q];
    }
    unsigned long long total;
    unsigned long long run = block_exscan_u64(local, s_tmp, &total) + block_off[blk];
#pragma unroll
    for (int q = 0; q < kFrItems; ++q) {
        uint64_t i = i0 + q;
        if (i < f) {
            prefix[i] = run;
            rowstart[i] = st[q];
        }
        run += deg[q];
    }
}

// pass 2: per-entry exclusive prefix, row start and value snapshot
__global__ void __launch_bounds__(kFrThreads) fr_write_kernel(
    const uint32_t* F0, const uint32_t* F1, uint32_t f, const PushLoop* __restrict__ loop,
    const uint64_t* __restrict__ off, const uint32_t* __restrict__ val,
    const unsigned long long* __restrict__ block_off, unsigned long long* __restrict__ prefix,
    unsigned long long* __restrict__ rowstart, uint32_t* __restrict__ fval) {
    __shared__ unsigned long long s_tmp[33];
    const uint32_t* __restrict__ F = loop_frontier(F0, F1, loop);
    f = loop_f(f, loop);
    const uint32_t nb = (f + kFrBlock - 1) / kFrBlock;
    for (uint32_t blk = blockIdx.x; blk < nb; blk += gridDim.x) {
        fr_write_block(F, f, blk, off, val, block_off, prefix, rowstart, fval, s_tmp);
        __syncthreads();  // s_tmp is reused by the next block
    }
}


__device__ __forceinline__ uint32_t merge_path_rows(const unsigned long long* __restrict__ row_end, uint32_t nrows,
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

__global__ void push_partition_kernel(const unsigned long long* __restrict__ prefix, uint32_t f,
                                      const PushLoop* __restrict__ loop, const PushCounters* __restrict__ ctr,
                                      uint32_t* __restrict__ tile_row) {
    if (loop && loop->pull) return;
    f = loop_f(f, loop);
    const uint64_t E = ctr->edges;
    const uint64_t tiles = ctr->tiles;
    const uint64_t total = (uint64_t)f + E;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= tiles; t += stride) {
        uint64_t diag = t * kPushTile;
        if (diag > total) diag = total;
        tile_row[t] = merge_path_rows(prefix + 1, f, E, diag);
    }
}

constexpr int kEdgesPerThread = 4;  // independent messages in flight per thread

template <int kWeightKind>
__device__ __forceinline__ uint32_t edge_weight(const uint8_t* __restrict__ w8, const uint32_t* __restrict__ w32,
                                                unsigned long long p) {
    if (kWeightKind == 1) return (uint32_t)__ldcs(w8 + p);
    if (kWeightKind == 2) return __ldcs(w32 + p);
    return 1u;
}

// kWeightKind: 0 = no weights (length 1), 1 = u8 weights, 2 = u32 weights
template <int kKind, int kWeightKind, bool kRecv>
__global__ void __launch_bounds__(kPushThreads) push_relax_kernel(
    const unsigned long long* __restrict__ prefix, const unsigned long long* __restrict__ rowstart,
    const uint32_t* __restrict__ fval, const uint32_t* __restrict__ tile_row, const uint32_t* __restrict__ col,
    const uint8_t* __restrict__ w8, const uint32_t* __restrict__ w32, uint32_t* __restrict__ val,
    uint32_t* __restrict__ stamp, uint32_t* __restrict__ rstamp, uint32_t* next0, uint32_t* next1,
    const PushLoop* __restrict__ loop, PushCounters* __restrict__ ctr, uint32_t f, uint32_t tag) {
    if (loop && loop->pull) return;
    uint32_t* __restrict__ next = loop_next(next0, next1, loop);
    f = loop_f(f, loop);
    if (loop) tag = loop->s + 1;
    __shared__ uint32_t s_start[kPushTile + 1];
    __shared__ unsigned long long s_base[kPushTile + 1];
    __shared__ uint32_t s_val[kPushTile + 1];
    const uint64_t E = ctr->edges;
    const uint32_t tiles = ctr->tiles;
    const uint64_t total = (uint64_t)f + E;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    for (uint32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const uint64_t d0 = (uint64_t)tile * kPushTile;
        const uint64_t d1 = d0 + kPushTile < total ? d0 + kPushTile : total;
        const uint32_t i0 = tile_row[tile];
        const uint32_t i1 = tile_row[tile + 1];
        const uint64_t j0 = d0 - i0;
        const uint32_t R = i1 - i0;
        const uint32_t Et = (uint32_t)((d1 - i1) - j0);
        __syncthreads();  // the previous tile is done with shared memory
        for (uint32_t k = tid; k <= R; k += kPushThreads) {
            const uint32_t r = i0 + k;
            if (r < f) {
                const unsigned long long p = prefix[r];
                s_start[k] = p > j0 ? (uint32_t)(p - j0) : 0u;
                s_base[k] = rowstart[r] + (j0 - p);  // edge position = base + k (mod 2^64)
                s_val[k] = fval[r];
            } else {
                s_start[k] = Et + 1;
                s_base[k] = 0;
                s_val[k] = 0;
            }
        }
        __syncthreads();
        for (uint32_t k0 = 0; k0 < Et; k0 += kPushThreads * kEdgesPerThread) {
            uint32_t v[kEdgesPerThread], cand[kEdgesPerThread], cur[kEdgesPerThread];
            bool ok[kEdgesPerThread];
#pragma unroll
            for (int q = 0; q < kEdgesPerThread; ++q) {
                const uint32_t k = k0 + tid + q * kPushThreads;
                ok[q] = k < Et;
                v[q] = 0;
                cand[q] = 0;
                if (ok[q]) {
                    // row of edge k: the last row whose start is <= k
                    uint32_t lo = 0, hi = R;
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi + 1) >> 1;
                        if (s_start[mid] <= k)
                            lo = mid;
                        else
                            hi = mid - 1;
                    }
                    const unsigned long long p = s_base[lo] + k;
                    v[q] = __ldcs(col + p);
                    if (kKind == kHashmin) {
                        cand[q] = s_val[lo];
                    } else {
                        unsigned long long d = (unsigned long long)s_val[lo] + edge_weight<kWeightKind>(w8, w32, p);
                        if (d >= kInf) {
                            atomicOr(&ctr->status, kStatusOverflow);
                            d = kInf - 1;
                        }
                        cand[q] = (uint32_t)d;
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < kEdgesPerThread; ++q) cur[q] = ok[q] ? val[v[q]] : 0u;  // stale-high, never low
#pragma unroll
            for (int q = 0; q < kEdgesPerThread; ++q) {
                bool app = false, rcv = false;
                if (ok[q]) {
                    if (kRecv) rcv = atomicExch(&rstamp[v[q]], tag) != tag;
                    if (cand[q] < cur[q]) {
                        const uint32_t old = atomicMin(&val[v[q]], cand[q]);
                        if (cand[q] < old) app = atomicExch(&stamp[v[q]], tag) != tag;
                    }
                }
                const unsigned mask = __ballot_sync(0xFFFFFFFFu, app);
                if (mask) {
                    const int leader = __ffs(mask) - 1;
                    uint32_t pos = 0;
                    if (lane == leader) pos = atomicAdd(&ctr->next_size, (unsigned)__popc(mask));
                    pos = __shfl_sync(0xFFFFFFFFu, pos, leader);
                    if (app) next[pos + __popc(mask & ((1u << lane) - 1u))] = v[q];
                }
                if (kRecv) {
                    const unsigned rm = __ballot_sync(0xFFFFFFFFu, rcv);
                    if (lane == 0 && rm) atomicAdd(&ctr->receivers, (unsigned long long)__popc(rm));
                }
            }
        }
    }
}

// instance of caller id c: the last i with bases[i] <= c (empty instances are skipped)
__device__ __forceinline__ uint32_t instance_of(const uint32_t* __restrict__ bases, uint32_t count, uint32_t c) {
    uint32_t lo = 0, hi = count;
    while (lo + 1 < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (bases[mid] <= c)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// per-instance messages of this superstep: sum of the senders' out-degrees, by instance
__global__ void instance_msgs_kernel(const uint32_t* F0, const uint32_t* F1, uint32_t f,
                                     const PushLoop* __restrict__ loop, const uint64_t* __restrict__ off,
                                     const uint32_t* __restrict__ perm, const uint32_t* __restrict__ bases,
                                     uint32_t count, unsigned long long* __restrict__ inst_msgs) {
    extern __shared__ unsigned long long s_acc[];
    const uint32_t* __restrict__ F = loop_frontier(F0, F1, loop);
    f = loop_f(f, loop);
    const bool local = count <= 2048;
    if (local)
        for (uint32_t k = threadIdx.x; k < count; k += blockDim.x) s_acc[k] = 0;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < f; i += stride) {
        const uint32_t u = F[i];
        const unsigned long long d = off[u + 1] - off[u];
        if (!d) continue;
        const uint32_t inst = instance_of(bases, count, perm[u]);
        if (local)
            atomicAdd(&s_acc[inst], d);
        else
            atomicAdd(&inst_msgs[inst], d);
    }
    __syncthreads();
    if (local)
        for (uint32_t k = threadIdx.x; k < count; k += blockDim.x)
            if (s_acc[k]) atomicAdd(&inst_msgs[k], s_acc[k]);
}

// loop-driven runs of a batch graph: one more superstep for every instance whose
// vertices sent messages in this one; the per-instance sums restart at zero
__global__ void instance_step_kernel(unsigned long long* __restrict__ inst_msgs, uint32_t count,
                                     uint32_t* __restrict__ inst_steps) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        if (inst_msgs[i]) ++inst_steps[i];
        inst_msgs[i] = 0;
    }
}

__global__ void fill_u32_kernel(uint32_t* __restrict__ a, uint32_t count, uint32_t value) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) a[i] = value;
}

// labels in caller ids of the union -> instance-local ids
__global__ void local_labels_kernel(uint32_t* __restrict__ labels, uint32_t n, const uint32_t* __restrict__ bases,
                                    uint32_t count) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        labels[v] -= bases[instance_of(bases, count, (uint32_t)v)];
}

unsigned grid_cap(uint64_t work, unsigned cap = 0) {
    if (!cap) cap = (unsigned)sm_count_current() * 16;
    uint64_t b = (work + 255) / 256;
    if (b < 1) b = 1;
    return (unsigned)(b < cap ? b : cap);
}

int sm_count(int dev) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    return v;
}

// next0 / next1: the next frontier of a host-driven superstep (both the same), or
// the two frontier buffers of a loop-driven one, picked by loop->cur
template <int kKind, int kWeightKind, bool kRecv>
void launch_relax(unsigned grid, cudaStream_t st, ipg_graph* g, uint32_t* val, uint32_t* next0, uint32_t* next1,
                  const PushLoop* loop, uint32_t f, uint32_t tag) {
    push_relax_kernel<kKind, kWeightKind, kRecv><<<grid, kPushThreads, 0, st>>>(
        g->fr_prefix, g->fr_rowstart, g->fr_val, g->push_tile_row, g->col, g->w8, g->w, val, g->stamp, g->rstamp,
        next0, next1, loop, g->counters, f, tag);
}

template <int kKind, int kWeightKind>
void launch_relax2(bool recv, unsigned grid, cudaStream_t st, ipg_graph* g, uint32_t* val, uint32_t* next0,
                   uint32_t* next1, const PushLoop* loop, uint32_t f, uint32_t tag) {
    if (recv)
        launch_relax<kKind, kWeightKind, true>(grid, st, g, val, next0, next1, loop, f, tag);
    else
        launch_relax<kKind, kWeightKind, false>(grid, st, g, val, next0, next1, loop, f, tag);
}

void relax_dispatch(int kind, bool recv, unsigned grid, cudaStream_t st, ipg_graph* g, uint32_t* val, uint32_t* next0,
                    uint32_t* next1, const PushLoop* loop, uint32_t f, uint32_t tag) {
    if (kind == kHashmin)
        launch_relax2<kHashmin, 0>(recv, grid, st, g, val, next0, next1, loop, f, tag);
    else if (g->w8)
        launch_relax2<kSssp, 1>(recv, grid, st, g, val, next0, next1, loop, f, tag);
    else if (g->w)
        launch_relax2<kSssp, 2>(recv, grid, st, g, val, next0, next1, loop, f, tag);
    else
        launch_relax2<kSssp, 0>(recv, grid, st, g, val, next0, next1, loop, f, tag);
}

// ---------------------------------------------------------------------------
// Loop-driven runs: the superstep loop inside a CUDA graph (conditional WHILE)

constexpr unsigned kLoopCap = 64;          // supersteps per graph launch
constexpr uint32_t kLoopRecords = 1 << 16; // stats records a loop-driven run keeps

__global__ void loop_init_kernel(PushLoop* __restrict__ loop, uint32_t f, unsigned long long divisor,
                                 unsigned int filter_pct) {
    loop->filter = 0;
    loop->filter_pct = filter_pct;
    loop->cur = 0;
    loop->f = f;
    loop->s = 0;
    loop->pull = 0;
    loop->iter = 0;
    loop->done = f == 0;
    loop->count = 0;
    loop->nrec = 0;
    loop->status = 0;
    loop->divisor = divisor;
    loop->prev_receivers = 0;
}

__device__ __forceinline__ void loop_record(PushLoop* loop, ipg_superstep_stats* rec, const ipg_superstep_stats& r) {
    if (loop->nrec < kLoopRecords) rec[loop->nrec] = r;
    ++loop->nrec;
}

// End of a loop-driven superstep: the stats record, termination (no next
// frontier: the receivers still run one more superstep if messages were sent),
// then the next frontier becomes current and the WHILE condition is set.
__global__ void loop_step_kernel(PushLoop* __restrict__ loop, PushCounters* __restrict__ ctr,
                                 ipg_superstep_stats* __restrict__ rec, uint32_t n, int recv,
                                 cudaGraphConditionalHandle handle) {
    const unsigned long long edges = ctr->edges, receivers = ctr->receivers;
    const uint32_t fn = ctr->next_size, s = loop->s;
    uint32_t status = loop->status | ctr->status;
    if (fn > n) status |= kStatusInternal;
    ipg_superstep_stats r{};
    r.superstep = s;
    r.flags = (recv ? IPG_STAT_RECEIVERS : 0u) | (loop->pull ? IPG_STAT_PULL : 0u);
    r.active = s == 0 ? n : (recv ? loop->prev_receivers : 0);
    r.senders = loop->f;
    r.messages_sent = edges;
    r.receivers = recv ? receivers : 0;
    loop_record(loop, rec, r);
    bool more = false;
    if (status) {
        loop->done = 1;
    } else if (fn == 0) {
        loop->count = s + 1;
        if (edges > 0) {  // the receivers run one more superstep, change nothing, send nothing
            ipg_superstep_stats t{};
            t.superstep = s + 1;
            t.flags = recv ? IPG_STAT_RECEIVERS : 0u;
            t.active = recv ? receivers : 0;
            loop_record(loop, rec, t);
            loop->count = s + 2;
        }
        loop->done = 1;
    } else {
        loop->prev_receivers = receivers;
        loop->f = fn;
        loop->cur ^= 1u;
        loop->s = s + 1;
        more = true;
    }
    loop->status = status;
    const unsigned it = loop->iter + 1;
    const bool again = more && it < kLoopCap;
    loop->iter = again ? it : 0u;
    cudaGraphSetConditional(handle, again ? 1u : 0u);
}

__global__ void unpermute_u32_kernel(const uint32_t* __restrict__ in, const uint32_t* __restrict__ inv, uint32_t n,
                                     uint32_t* __restrict__ out) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) out[v] = in[inv[v]];
}

ipg_status ensure_events_push(size_t count, cudaEvent_t** evs) {
    static thread_local cudaEvent_t* ev = nullptr;
    static thread_local size_t cap = 0;
    if (count > cap) {
        cudaEvent_t* nv = new cudaEvent_t[count];
        for (size_t i = 0; i < cap; ++i) nv[i] = ev[i];
        for (size_t i = cap; i < count; ++i) IPG_CUDA(cudaEventCreate(&nv[i]));
        delete[] ev;
        ev = nv;
        cap = count;
    }
    *evs = ev;
    return IPG_OK;
}

// loop-graph slot: program x receivers counting x pull form allowed x per-instance counts
int loop_slot(int kind, bool recv, bool pull, bool inst) {
    return (inst ? 8 : 0) + (kind == kSssp ? 4 : 0) + (recv ? 2 : 0) + (pull ? 1 : 0);
}

ipg_status ensure_loop_workspace(ipg_graph* g) {
    if (g->loop) return IPG_OK;
    IPG_CUDA(cudaMalloc(&g->loop_rec, sizeof(ipg_superstep_stats) * kLoopRecords));
    IPG_CUDA(cudaHostAlloc(&g->h_loop, sizeof(PushLoop), cudaHostAllocDefault));
    IPG_CUDA(cudaMalloc(&g->loop, sizeof(PushLoop)));
    return IPG_OK;
}

// Builds [WHILE (cond) { superstep }] for one slot.  The body enqueues both forms
// of the superstep; each returns at once unless fr_scan_kernel picked it.
ipg_status push_loop_graph(ipg_graph* g, int kind, bool recv, bool pull, bool inst, cudaGraphExec_t* out) {
    const int sms = sm_count(g->device);
    const unsigned fixed = (unsigned)sms * 8;
    cudaGraph_t graph = nullptr;
    cudaStream_t cap = nullptr;
    ipg_status rc = IPG_OK;
    do {
        cudaError_t e = cudaGraphCreate(&graph, 0);
        cudaGraphConditionalHandle handle;
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = handle;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaStreamBeginCaptureToGraph(cap, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "superstep loop graph", __FILE__, __LINE__);
            break;
        }
        if (inst) {  // per-instance messages of the senders, before the superstep changes anything
            const size_t shm = g->instances <= 2048 ? sizeof(unsigned long long) * g->instances : 0;
            instance_msgs_kernel<<<fixed, 256, shm, cap>>>(g->frontier[0], g->frontier[1], 0, g->loop, g->off,
                                                           g->perm, g->inst_base, g->instances, g->inst_msgs);
            instance_step_kernel<<<grid_cap(g->instances), 256, 0, cap>>>(g->inst_msgs, g->instances,
                                                                         g->inst_steps);
        }
        fr_reduce_kernel<<<fixed, kFrThreads, 0, cap>>>(g->frontier[0], g->frontier[1], 0, g->loop, g->off,
                                                        g->block_sums);
        fr_scan_kernel<<<1, kScanThreads, 0, cap>>>(g->block_sums, 0, 0, g->loop, g->m, g->fr_prefix, g->counters);
        fr_write_kernel<<<fixed, kFrThreads, 0, cap>>>(g->frontier[0], g->frontier[1], 0, g->loop, g->off, g->val,
                                                       g->block_sums, g->fr_prefix, g->fr_rowstart, g->fr_val);
        push_partition_kernel<<<(unsigned)sms * 2, 256, 0, cap>>>(g->fr_prefix, 0, g->loop, g->counters,
                                                                 g->push_tile_row);
        relax_dispatch(kind, recv, (unsigned)sms * 6, cap, g, g->val, g->frontier[0], g->frontier[1], g->loop, 0, 0);
        if (pull) rc = pull_min_enqueue_loop(g, kind == kSssp, recv, g->val, cap);
        loop_step_kernel<<<1, 1, 0, cap>>>(g->loop, g->counters, g->loop_rec, g->n, recv ? 1 : 0, handle);
        cudaGraph_t body = nullptr;
        e = cudaStreamEndCapture(cap, &body);
        if (rc != IPG_OK) break;
        if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
        if (e != cudaSuccess) rc = cuda_fail(e, "superstep loop graph capture", __FILE__, __LINE__);
    } while (false);
    if (cap) cudaStreamDestroy(cap);
    if (graph) cudaGraphDestroy(graph);
    return rc;
}

// Hashmin / SSSP with the superstep loop on the device (no per-superstep timing
// and no per-instance counts): a few host synchronisations per run.
ipg_status push_run_loop(ipg_graph* g, int kind, uint32_t source, uint32_t* out, ipg_stats* stats, cudaStream_t st,
                         const char* name, uint32_t* inst_supersteps) {
    const uint32_t n = g->n;
    const bool recv = stats && (stats->flags & IPG_STAT_RECEIVERS);
    const long long div = pull_divisor_for(g, kind == kSssp);
    const bool pull = div > 0;
    const bool inst = inst_supersteps && g->instances;
    IPG_TRY(ensure_push_workspace(g, recv));
    IPG_TRY(ensure_loop_workspace(g));
    if (inst && !g->inst_steps) IPG_CUDA(cudaMalloc(&g->inst_steps, sizeof(uint32_t) * g->instances));
    if (pull) {
        IPG_TRY(ensure_csc(g, st));
        IPG_TRY(pull_min_prepare(g, st));
    }
    cudaGraphExec_t& exec = g->push_exec[loop_slot(kind, recv, pull, inst)];
    if (!exec) IPG_TRY(push_loop_graph(g, kind, recv, pull, inst, &exec));
    if (inst) {  // every instance runs superstep 0
        IPG_CUDA(cudaMemsetAsync(g->inst_msgs, 0, sizeof(unsigned long long) * g->instances, st));
        fill_u32_kernel<<<grid_cap(g->instances), 256, 0, st>>>(g->inst_steps, g->instances, 1u);
    }
    IPG_CUDA(cudaMemsetAsync(g->stamp, 0, sizeof(uint32_t) * n, st));
    if (recv) IPG_CUDA(cudaMemsetAsync(g->rstamp, 0, sizeof(uint32_t) * n, st));
    IPG_CUDA(cudaMemsetAsync(&g->counters->status, 0, sizeof(unsigned), st));
    uint32_t f;
    if (kind == kHashmin) {
        hashmin_init_kernel<<<grid_cap(n), 256, 0, st>>>(g->val, g->frontier[0], g->perm, n);
        f = n;
    } else {
        sssp_init_kernel<<<grid_cap(n), 256, 0, st>>>(g->val, g->frontier[0], n, g->inv, source);
        f = 1;
    }
    loop_init_kernel<<<1, 1, 0, st>>>(g->loop, f, (unsigned long long)(div > 0 ? div : 0),
                                      (unsigned int)tuning().pull_filter);
    IPG_CUDA(cudaGetLastError());
    // each launch runs up to kLoopCap supersteps; a run has at most n + 1
    const uint64_t max_launches = (uint64_t)n / kLoopCap + 3;
    g->h_loop->done = 0;
    for (uint64_t launches = 0; !g->h_loop->done; ++launches) {
        if (launches > max_launches) return set_error(IPG_EDEVICE, "%s: the superstep loop did not end", name);
        IPG_CUDA(cudaGraphLaunch(exec, st));
        IPG_CUDA(cudaMemcpyAsync(g->h_loop, g->loop, sizeof(PushLoop), cudaMemcpyDeviceToHost, st));
        IPG_CUDA(cudaStreamSynchronize(st));
    }
    const PushLoop h = *g->h_loop;
    if (h.status & kStatusOverflow) return set_error(IPG_EOVERFLOW, "%s: a path length reached UINT32_MAX", name);
    if (h.status) return set_error(IPG_EDEVICE, "%s: frontier overflow", name);
    if (stats) {
        const uint32_t keep = std::min(std::min(h.nrec, kLoopRecords), stats->cap);
        if (keep && stats->buf)
            IPG_CUDA(cudaMemcpyAsync(stats->buf, g->loop_rec, sizeof(ipg_superstep_stats) * keep,
                                     cudaMemcpyDeviceToHost, st));
        stats->count = h.count;
    }
    if (inst)
        IPG_CUDA(cudaMemcpyAsync(inst_supersteps, g->inst_steps, sizeof(uint32_t) * g->instances,
                                 cudaMemcpyDeviceToHost, st));
    unpermute_u32_kernel<<<grid_cap(n), 256, 0, st>>>(g->val, g->inv, n, out);
    IPG_CUDA(cudaGetLastError());
    IPG_CUDA(cudaStreamSynchronize(st));
    return IPG_OK;
}

ipg_status push_run(ipg_graph* g, int kind, uint32_t source, uint32_t* out, ipg_stats* stats, cudaStream_t st,
                    uint32_t* inst_supersteps = nullptr) {
    stats_begin(stats);
    const char* name = kind == kHashmin ? "ipg_hashmin_cc" : "ipg_sssp";
    if (!g) return set_error(IPG_EINVAL, "%s: graph is NULL", name);
    if (kind == kHashmin && g->directed)
        return set_error(IPG_EINVAL, "%s: Hashmin components need an undirected graph (directed = 0)", name);
    if (kind == kSssp && source >= g->n) return set_error(IPG_EINVAL, "%s: source %u >= n = %u", name, source, g->n);
    if (g->n && !out) return set_error(IPG_EINVAL, "%s: output is NULL", name);
    DeviceGuard guard(g->device);
    if (!guard.ok) return set_error(IPG_ECUDA, "%s: cannot select the graph's device", name);
    const uint32_t n = g->n;
    const bool recv = stats && (stats->flags & IPG_STAT_RECEIVERS);
    const bool timing = stats && (stats->flags & IPG_STAT_TIMING);
    if (n == 0) {  // superstep 0 runs on no vertex and sends nothing
        if (stats) {
            ipg_superstep_stats r{};
            r.flags = recv ? IPG_STAT_RECEIVERS : 0u;
            stats_put(stats, 0, r);
            stats->count = 1;
        }
        return IPG_OK;
    }
    if (!timing && (!stats || stats->cap <= kLoopRecords) && tuning().push_loop != 0)
        return push_run_loop(g, kind, source, out, stats, st, name, inst_supersteps);
    IPG_TRY(ensure_push_workspace(g, recv));
    uint32_t* val = g->val;
    cudaEvent_t* ev = nullptr;
    if (timing) IPG_TRY(ensure_events_push(3, &ev));
    const int sms = sm_count(g->device);
    const unsigned relax_grid = (unsigned)sms * 6;

    IPG_CUDA(cudaMemsetAsync(g->stamp, 0, sizeof(uint32_t) * n, st));
    if (recv) IPG_CUDA(cudaMemsetAsync(g->rstamp, 0, sizeof(uint32_t) * n, st));
    IPG_CUDA(cudaMemsetAsync(&g->counters->status, 0, sizeof(unsigned), st));
    uint32_t f;
    if (kind == kHashmin) {
        hashmin_init_kernel<<<grid_cap(n), 256, 0, st>>>(val, g->frontier[0], g->perm, n);
        f = n;
    } else {
        sssp_init_kernel<<<grid_cap(n), 256, 0, st>>>(val, g->frontier[0], n, g->inv, source);
        f = 1;
    }
    IPG_CUDA(cudaGetLastError());

    int cur = 0;
    uint32_t s = 0;
    uint64_t prev_receivers = 0;
    uint32_t count = 0;
    const uint32_t ninst = g->instances;
    const bool per_inst = inst_supersteps && ninst;
    std::vector<unsigned long long> h_inst(per_inst ? ninst : 0);
    if (per_inst)
        for (uint32_t i = 0; i < ninst; ++i) inst_supersteps[i] = 1;
    for (;;) {
        if (timing) IPG_CUDA(cudaEventRecord(ev[0], st));
        IPG_TRY(frontier_prepare(g, g->frontier[cur], f, val, st));
        if (per_inst) {
            IPG_CUDA(cudaMemsetAsync(g->inst_msgs, 0, sizeof(unsigned long long) * ninst, st));
            const size_t shm = ninst <= 2048 ? sizeof(unsigned long long) * ninst : 0;
            instance_msgs_kernel<<<grid_cap(f), 256, shm, st>>>(g->frontier[cur], g->frontier[cur], f, nullptr, g->off,
                                                                g->perm, g->inst_base, ninst, g->inst_msgs);
            IPG_CUDA(cudaGetLastError());
            IPG_CUDA(cudaMemcpyAsync(h_inst.data(), g->inst_msgs, sizeof(unsigned long long) * ninst,
                                     cudaMemcpyDeviceToHost, st));
        }
        // direction: a superstep whose messages reach m / pull_divisor runs in pull form
        bool pull = false, filter = false;
        const long long div = pull_divisor_for(g, kind == kSssp);
        // a frontier of f vertices sends at most f * max_outdeg messages: read the exact
        // count back (one more host sync) only when that bound reaches m / pull_divisor
        if (div > 0 && g->m && (double)f * (double)g->max_outdeg * (double)div >= (double)g->m) {
            IPG_CUDA(cudaMemcpyAsync(&g->h_counters->edges, &g->counters->edges, sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost, st));
            IPG_CUDA(cudaStreamSynchronize(st));
            const unsigned long long es = g->h_counters->edges;
            pull = es > 0 && (double)es * (double)div >= (double)g->m;
            filter = pull && (double)es * 100.0 < (double)g->m * (double)tuning().pull_filter;
        }
        if (pull) {
            IPG_TRY(pull_min_superstep(g, kind == kSssp, recv, filter, g->frontier[cur], g->fr_val, f, val,
                                       g->frontier[cur ^ 1], st, timing ? ev[1] : nullptr));
        } else {
            IPG_TRY(frontier_partition(g, f, st));
            if (timing) IPG_CUDA(cudaEventRecord(ev[1], st));
            relax_dispatch(kind, recv, relax_grid, st, g, val, g->frontier[cur ^ 1], g->frontier[cur ^ 1], nullptr, f,
                           s + 1);
            IPG_CUDA(cudaGetLastError());
        }
        if (timing) IPG_CUDA(cudaEventRecord(ev[2], st));
        IPG_CUDA(cudaMemcpyAsync(g->h_counters, g->counters, sizeof(PushCounters), cudaMemcpyDeviceToHost, st));
        IPG_CUDA(cudaStreamSynchronize(st));
        const PushCounters h = *g->h_counters;
        if (per_inst)
            for (uint32_t i = 0; i < ninst; ++i) inst_supersteps[i] += h_inst[i] > 0 ? 1 : 0;
        if (h.status & kStatusOverflow) {
            if (stats) stats->count = 0;
            return set_error(IPG_EOVERFLOW, "%s: a path length reached UINT32_MAX", name);
        }
        if (stats) {
            ipg_superstep_stats r{};
            r.superstep = s;
            r.flags = (recv ? IPG_STAT_RECEIVERS : 0u) | (timing ? IPG_STAT_TIMING : 0u) | (pull ? IPG_STAT_PULL : 0u);
            r.active = s == 0 ? n : (recv ? prev_receivers : 0);
            r.senders = f;
            r.messages_sent = h.edges;
            r.receivers = recv ? h.receivers : 0;
            if (timing) {
                cudaEventElapsedTime(&r.kernel_ms, ev[1], ev[2]);
                cudaEventElapsedTime(&r.superstep_ms, ev[0], ev[2]);
            }
            stats_put(stats, s, r);
        }
        if (h.next_size == 0) {
            count = s + 1;
            if (h.edges > 0) {  // the receivers still run one more superstep, change nothing, send nothing
                if (stats) {
                    ipg_superstep_stats r{};
                    r.superstep = s + 1;
                    r.flags = recv ? IPG_STAT_RECEIVERS : 0u;
                    r.active = recv ? h.receivers : 0;
                    stats_put(stats, s + 1, r);
                }
                count = s + 2;
            }
            break;
        }
        if (h.next_size > n) return set_error(IPG_EDEVICE, "%s: frontier overflow (%u > n)", name, h.next_size);
        prev_receivers = h.receivers;
        f = h.next_size;
        cur ^= 1;
        ++s;
    }
    unpermute_u32_kernel<<<grid_cap(n), 256, 0, st>>>(val, g->inv, n, out);
    IPG_CUDA(cudaGetLastError());
    IPG_CUDA(cudaStreamSynchronize(st));
    if (stats) stats->count = count;
    return IPG_OK;
}

}  // namespace

ipg_status frontier_prepare(ipg_graph* g, const uint32_t* F, uint32_t f, const uint32_t* val, cudaStream_t st) {
    const uint32_t nb = (f + kFrBlock - 1) / kFrBlock;
    const unsigned grid = nb ? nb : 1;
    fr_reduce_kernel<<<grid, kFrThreads, 0, st>>>(F, F, f, nullptr, g->off, g->block_sums);
    fr_scan_kernel<<<1, kScanThreads, 0, st>>>(g->block_sums, nb, f, nullptr, g->m, g->fr_prefix, g->counters);
    fr_write_kernel<<<grid, kFrThreads, 0, st>>>(F, F, f, nullptr, g->off, val, g->block_sums, g->fr_prefix,
                                                 g->fr_rowstart, g->fr_val);
    IPG_CUDA(cudaGetLastError());
    return IPG_OK;
}

ipg_status frontier_partition(ipg_graph* g, uint32_t f, cudaStream_t st) {
    push_partition_kernel<<<(unsigned)sm_count(g->device) * 2, 256, 0, st>>>(g->fr_prefix, f, nullptr, g->counters,
                                                                            g->push_tile_row);
    IPG_CUDA(cudaGetLastError());
    return IPG_OK;
}

ipg_status ensure_push_workspace(ipg_graph* g, bool receivers) {
    const uint32_t n = g->n;
    if (!g->stamp) {
        IPG_CUDA(cudaMalloc(&g->val, sizeof(uint32_t) * n));
        IPG_CUDA(cudaMalloc(&g->stamp, sizeof(uint32_t) * n));
        IPG_CUDA(cudaMalloc(&g->frontier[0], sizeof(uint32_t) * n));
        IPG_CUDA(cudaMalloc(&g->frontier[1], sizeof(uint32_t) * n));
        IPG_CUDA(cudaMalloc(&g->fr_prefix, sizeof(unsigned long long) * ((size_t)n + 1)));
        IPG_CUDA(cudaMalloc(&g->fr_rowstart, sizeof(unsigned long long) * n));
        IPG_CUDA(cudaMalloc(&g->fr_val, sizeof(uint32_t) * n));
        const size_t nb = ((size_t)n + kFrBlock - 1) / kFrBlock;
        IPG_TRY(ensure(&g->block_sums, &g->block_sums_cap, nb + 1));
        const size_t tiles = ((size_t)n + g->m + kPushTile - 1) / kPushTile + 2;
        IPG_TRY(ensure(&g->push_tile_row, &g->push_tile_cap, tiles + 1));
    }
    if (receivers && !g->rstamp) IPG_CUDA(cudaMalloc(&g->rstamp, sizeof(uint32_t) * n));
    return IPG_OK;
}

}  // namespace ipg

using namespace ipg;

extern "C" {

ipg_status ipg_hashmin_cc_dev(ipg_graph* g, uint32_t* labels_dev, ipg_stats* stats, void* stream) {
    return push_run(g, kHashmin, 0, labels_dev, stats, (cudaStream_t)stream);
}

ipg_status ipg_sssp_dev(ipg_graph* g, uint32_t source, uint32_t* dist_dev, ipg_stats* stats, void* stream) {
    return push_run(g, kSssp, source, dist_dev, stats, (cudaStream_t)stream);
}

static ipg_status host_variant(ipg_graph* g, int kind, uint32_t source, uint32_t* out, ipg_stats* stats) {
    stats_begin(stats);
    if (!g) return set_error(IPG_EINVAL, "graph is NULL");
    if (g->n && !out) return set_error(IPG_EINVAL, "output is NULL");
    DeviceGuard guard(g->device);
    size_t cap = g->val_stage ? (size_t)g->n * sizeof(uint32_t) : 0;
    if (!g->val_stage) IPG_TRY(ensure(&g->val_stage, &cap, (size_t)g->n));
    IPG_TRY(push_run(g, kind, source, g->val_stage, stats, g->stream));
    if (g->n) {
        IPG_CUDA(cudaMemcpyAsync(out, g->val_stage, sizeof(uint32_t) * g->n, cudaMemcpyDeviceToHost, g->stream));
        IPG_CUDA(cudaStreamSynchronize(g->stream));
    }
    return IPG_OK;
}

ipg_status ipg_hashmin_cc(ipg_graph* g, uint32_t* labels_out, ipg_stats* stats) {
    return host_variant(g, kHashmin, 0, labels_out, stats);
}

ipg_status ipg_hashmin_cc_batch_dev(ipg_graph* g, uint32_t* labels_dev, uint32_t* supersteps_out, void* stream) {
    if (!g) return set_error(IPG_EINVAL, "ipg_hashmin_cc_batch: graph is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    DeviceGuard guard(g->device);
    if (!g->instances) {  // a plain graph is one instance
        ipg_stats stats{nullptr, 0, 0, 0, 0};
        IPG_TRY(push_run(g, kHashmin, 0, labels_dev, &stats, st));
        if (supersteps_out) supersteps_out[0] = stats.count;
        return IPG_OK;
    }
    std::vector<uint32_t> counts(g->instances);
    IPG_TRY(push_run(g, kHashmin, 0, labels_dev, nullptr, st, counts.data()));
    if (g->n) {
        local_labels_kernel<<<grid_cap(g->n), 256, 0, st>>>(labels_dev, g->n, g->inst_base, g->instances);
        IPG_CUDA(cudaGetLastError());
        IPG_CUDA(cudaStreamSynchronize(st));
    }
    if (supersteps_out)
        for (uint32_t i = 0; i < g->instances; ++i) supersteps_out[i] = counts[i];
    return IPG_OK;
}

ipg_status ipg_hashmin_cc_batch(ipg_graph* g, uint32_t* labels_out, uint32_t* supersteps_out) {
    if (!g) return set_error(IPG_EINVAL, "ipg_hashmin_cc_batch: graph is NULL");
    if (g->n && !labels_out) return set_error(IPG_EINVAL, "ipg_hashmin_cc_batch: output is NULL");
    DeviceGuard guard(g->device);
    size_t cap = g->val_stage ? (size_t)g->n * sizeof(uint32_t) : 0;
    if (!g->val_stage) IPG_TRY(ensure(&g->val_stage, &cap, (size_t)g->n));
    IPG_TRY(ipg_hashmin_cc_batch_dev(g, g->val_stage, supersteps_out, g->stream));
    if (g->n) {
        IPG_CUDA(cudaMemcpyAsync(labels_out, g->val_stage, sizeof(uint32_t) * g->n, cudaMemcpyDeviceToHost,
                                 g->stream));
        IPG_CUDA(cudaStreamSynchronize(g->stream));
    }
    return IPG_OK;
}

ipg_status ipg_sssp(ipg_graph* g, uint32_t source, uint32_t* dist_out, ipg_stats* stats) {
    return host_variant(g, kSssp, source, dist_out, stats);
}

}  // extern "C"
