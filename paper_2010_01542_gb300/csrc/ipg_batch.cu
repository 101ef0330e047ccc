// Batched SSSP: many sources on one graph, each an independent synchronous
// Pregel SSSP (Sec. VI-C), run together superstep by superstep.
//
// The engine has 32 * L lanes (L = 1 to 8 lines of 32), one query (a source) per
// lane or none.  Values live vertex-major, dist[v][line][lane] with rows of L
// lines, so the 32 lanes of one line of a vertex are one 128-byte line of memory:
// in a pull superstep every in-edge (u -> v) costs one read per line of u's
// sender values that holds a sender, where 32 L separate runs would each pay a
// random 4-byte gather.  A superstep:
//   refill   free lanes take the next queries (from a device list of sources, or
//            from seeds the host wrote at a superstep boundary): the source's
//            value becomes 0 and it joins the current senders;
//   pull     warps walk contiguous chunks of the in-edge lists (CSC), each warp
//            every (warps)-th chunk, with a chunk size halved on smaller graphs
//            until every warp holds about 3 chunks (see batch_chunks).  Lane b of
//            line j keeps a running min of sval[u][j][b] + w over the current
//            destination's edges and flushes it with atomicMin into dist[v][j][b]
//            when the destination changes (a row split across chunks is finished
//            by the atomics).  Lowered lanes are marked in cmask[v][j]; the first
//            mark of a vertex appends it to the next frontier (union over lanes);
//   apply    the previous senders' snapshot rows are reset to kInf, and every
//            vertex of the next frontier publishes dist[v][j][b] for the lanes
//            whose value dropped (kInf for the others), which is the snapshot the
//            next superstep reads; per-lane message counts (sum of the senders'
//            out-degrees) come out of the same pass, and a published value whose
//            messages would reach UINT32_MAX fails the call (IPG_EOVERFLOW);
//   step     a lane whose next senders send nothing has finished its query: its
//            superstep count is final;
//   harvest  finished lanes' distances go to their output rows (in caller ids)
//            and their columns are reset to kInf, which frees the lanes for the
//            next refill.  With a source list, finished lanes wait until their
//            lanes are needed or no lane runs, so that queries started together
//            are harvested in one pass.
// Senders send the value they had at the start of the superstep, as in the
// synchronous model; lanes never share values, so a query's distances and
// superstep count equal those of a standalone ipg_sssp run whichever superstep
// it joined at.
//
// Which vertices send is kept per line: smask[u][j] holds the sending lanes of
// line j, and with L > 1 sany[u] holds one bit per line that has a sender (the
// pull form gathers that word per in-edge and loads only the lines it names).
// With one line, a warp folds each active edge with its 32 lanes, the lanes
// that do not send from the source skipping their load.  With more, the pull
// kernel is instantiated per line count: each thread holds L lanes of a row (a
// 16-byte vector per 4 lines, one word of each line left), and the rows of the
// next edges are staged in a per-warp ring in shared memory by cp.async, so that
// a warp keeps several rows in flight without holding them in registers.  The
// apply and reset passes hold V lanes per thread (V = 2, 4 or 8, the next of L;
// lanes past the row's L lines stay unused).
//
// A sparse superstep runs in push form instead: a task pass cuts the senders'
// out-edge lists into tasks of kPushChunk edges, and a warp per task sends
// sval[u][j][b] + w along each out-edge (u -> v) with atomicMin into
// dist[v][j][b].  Push and pull take the minimum of the same messages and mark
// the same lowered lanes, so they are interchangeable; the refill kernel picks
// push when the senders' out-edges, counted once per sending line, are fewer
// than m / divisor.
//
// ipg_sssp_batch starts its queries together: the synchronous runs from
// different sources go through their dense supersteps (where nearly every edge
// carries a message) at about the same superstep, so one pass over the in-edges
// serves most lanes of every line.  Queries whose source has no out-edges end
// after superstep 0 and are written directly, without a lane; L is the smallest
// line count that holds the others (within free device memory).
//
// The superstep loop runs on the device: a CUDA graph holds a conditional WHILE
// node whose body is one superstep (refill, tasks, pull, push, reset, apply,
// step, harvest).  The kernels read the frontier and the lanes from a device
// control block, so their launch parameters never change, and the step kernel
// decides whether another superstep follows.  ipg_sssp_batch keeps every lane
// busy from its source list inside the loop, so k sources run in one graph launch
// (plus one per kLoopCap supersteps).  The server seeds lanes itself (one line):
// its launches end at the first superstep where a lane finished, or when queries
// wait for a free lane (a flag in mapped host memory), so queries join a running
// batch at the next superstep boundary.
#include <string.h>

#include <vector>

#include "ipg_internal.cuh"

namespace ipg {
namespace {

constexpr int kLanes = 32;                     // lanes per line
constexpr int kMaxLines = 8;                   // lines per vertex at most
constexpr int kMaxSlots = kLanes * kMaxLines;  // lanes at most
constexpr unsigned kLoopCap = 1024;            // supersteps per graph launch
constexpr uint32_t kPushChunk = 256;           // out-edges per push task

struct BatchCounters {
    unsigned long long msgs[kMaxSlots];  // messages the next superstep's senders send, per lane
    unsigned long long edges;            // out-edges of the next senders, once per sending line
    unsigned int next_size;
    unsigned int status;
    unsigned int ntasks;                 // push tasks of the current senders (push supersteps)
    unsigned int pad[11];
};

}  // namespace

// device-resident loop and lane state of one graph's batched engine
struct BatchCtl {
    unsigned int cur;     // frontier buffer holding the current senders
    unsigned int f;       // current senders
    unsigned int iter;    // supersteps run by the current graph launch
    unsigned int done;    // 1: no lane holds a query and none is left to take
    unsigned int status;  // kStatus* bits
    unsigned int push;    // 1: the current superstep runs in push form
    unsigned long long divisor;  // push when the senders' out-edges * divisor < m (0: always pull)
    unsigned long long f_edges;  // out-edges of the current senders, once per sending line
    unsigned int lines;                      // lines of 32 lanes in use
    unsigned int live[kMaxLines];            // lanes holding a query, per line
    unsigned int finished[kMaxLines];        // lanes harvested at the end of the last superstep
    unsigned int pending[kMaxLines];         // lanes whose query ended, not harvested yet (list mode)
    unsigned int final_harvest;              // 1: the last harvest of a session; lanes are not reset
    unsigned int count[kMaxSlots];           // supersteps of each lane's query so far (final once finished)
    unsigned int row[kMaxSlots];             // output row of each lane's query
    // refill from a device list (ipg_sssp_batch): caller ids, nqueries entries
    unsigned int next_query, nqueries;
    const uint32_t* src_list;
    const uint32_t* row_list;  // output row of each listed query (NULL: its index)
    uint32_t* steps_out;       // per output row: the query's superstep count (device), or NULL
    // refill by the host (serving)
    const volatile unsigned int* admit;  // mapped host flag: queries wait for a free lane (or NULL)
    unsigned int stop_on_finish;         // end a graph launch after a superstep in which a lane finished
    unsigned int nseed;                  // seeds below, taken by the next refill
    unsigned int seed_src[kLanes];       // caller ids
    unsigned int seed_row[kLanes];
    // output: rows of n distances in caller order
    uint32_t* out;
    unsigned long long out_stride;
    // totals of the session (ipg_sssp_batch_info)
    unsigned long long supersteps, pull_supersteps, harvests;
};

namespace {

__device__ __forceinline__ uint32_t* fr_cur(uint32_t* fr0, uint32_t* fr1, const BatchCtl* ctl) {
    return ctl->cur ? fr1 : fr0;
}
__device__ __forceinline__ uint32_t* fr_next(uint32_t* fr0, uint32_t* fr1, const BatchCtl* ctl) {
    return ctl->cur ? fr0 : fr1;
}

// index of lane `lane` of line j of vertex v in the [n][L][32] value arrays (rows of L lines)
__device__ __forceinline__ uint64_t slot_at(uint32_t v, uint32_t j, uint32_t lane, uint32_t L) {
    return ((uint64_t)v * L + j) * kLanes + lane;
}

__global__ void chunk_rows_kernel(const uint64_t* __restrict__ off, uint32_t n, uint64_t m, uint64_t chunks,
                                  uint32_t chunk, uint32_t* __restrict__ chunk_row) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < chunks; c += stride) {
        // row holding edge c * chunk: the last row whose start is <= that edge
        const uint64_t e = c * chunk;
        uint32_t lo = 0, hi = n;  // answer in [0, n - 1]
        while (lo + 1 < hi) {
            const uint32_t mid = (uint32_t)(((uint64_t)lo + hi) >> 1);
            if (off[mid] <= e)
                lo = mid;
            else
                hi = mid;
        }
        // skip rows that end at or before e (empty rows sharing the offset)
        while (lo + 1 < n && off[lo + 1] <= e) ++lo;
        chunk_row[c] = lo;
    }
}

// per listed source: 1 if it has out-edges (its query sends), else 0
__global__ void batch_triage_kernel(const uint32_t* __restrict__ list, uint32_t k, const uint32_t* __restrict__ inv,
                                    const uint64_t* __restrict__ off, uint8_t* __restrict__ sends) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) {
        const uint32_t v = inv[list[i]];
        sends[i] = off[v + 1] > off[v] ? 1 : 0;
    }
}

__device__ __forceinline__ bool batch_push_pick(unsigned long long edges, unsigned long long divisor, uint64_t m) {
    return divisor > 0 && (double)edges * (double)divisor < (double)m;
}

// Lanes `mask` of line j of v were lowered: mark them; the first mark of the
// vertex (over all its lines) appends it to the next frontier.
template <int V>
__device__ __forceinline__ void mark_lowered(uint32_t v, uint32_t j, uint32_t L, uint32_t mask,
                                             uint32_t* __restrict__ cmask, uint32_t* __restrict__ cany,
                                             uint32_t* __restrict__ next, BatchCounters* __restrict__ ctr) {
    if (atomicOr(&cmask[(uint64_t)v * L + j], mask) != 0) return;
    if (V > 1 && atomicOr(&cany[v], 1u << j) != 0) return;
    next[atomicAdd(&ctr->next_size, 1u)] = v;
}

// Free lanes take the next queries, in lane order: from the device source list,
// or from the host's seeds.  The source's value becomes 0 and it joins the
// current senders; its count starts at 1 (superstep 0), 2 if it has out-edges
// (its messages make a superstep 1).  Then the superstep's form is picked.
// One block of 32 V threads, thread b = lane b.
template <int V>
__global__ void batch_refill_kernel(BatchCtl* __restrict__ ctl, const uint32_t* __restrict__ inv,
                                    const uint64_t* __restrict__ off, const uint32_t* __restrict__ wmax_out,
                                    uint64_t m, uint32_t L, uint32_t* __restrict__ dist,
                                    uint32_t* __restrict__ sval, uint32_t* __restrict__ smask,
                                    uint32_t* __restrict__ sany, uint32_t* fr0, uint32_t* fr1) {
    __shared__ uint32_t free_sh[V], take_sh[V];
    __shared__ unsigned long long add_sh[V];
    const uint32_t b = threadIdx.x, j = b / kLanes, t = b % kLanes;
    const uint32_t live = ctl->live[j];
    const bool is_free = j < L && !(((live | ctl->pending[j]) >> t) & 1u);  // lines past L are not in the rows
    const unsigned freem = __ballot_sync(0xFFFFFFFFu, is_free);
    if (t == 0) free_sh[j] = __popc(freem);
    __syncthreads();
    uint32_t rank = __popc(freem & ((1u << t) - 1u));
    for (uint32_t i = 0; i < j; ++i) rank += free_sh[i];
    const bool from_list = ctl->nqueries != 0;
    bool take = false;
    uint32_t src = 0, row = 0;
    if (from_list) {
        const uint32_t q = ctl->next_query + rank;
        take = is_free && q < ctl->nqueries;
        if (take) {
            src = ctl->src_list[q];
            row = ctl->row_list ? ctl->row_list[q] : q;
        }
    } else {
        take = is_free && rank < ctl->nseed;
        if (take) {
            src = ctl->seed_src[rank];
            row = ctl->seed_row[rank];
        }
    }
    const unsigned takem = __ballot_sync(0xFFFFFFFFu, take);
    unsigned long long add = 0;
    if (take) {
        const uint32_t v = inv[src];
        const uint64_t at = slot_at(v, j, t, L);
        dist[at] = 0;
        sval[at] = 0;
        const uint64_t deg = off[v + 1] - off[v];
        if (wmax_out[v] == kInf) atomicOr(&ctl->status, kStatusOverflow);  // 0 + w reaches kInf
        if (atomicOr(&smask[(uint64_t)v * L + j], 1u << t) == 0) {
            add = deg;  // a line of v starts sending
            if (V == 1 || atomicOr(&sany[v], 1u << j) == 0) fr_cur(fr0, fr1, ctl)[atomicAdd(&ctl->f, 1u)] = v;
        }
        ctl->count[b] = 1u + (deg > 0 ? 1u : 0u);
        ctl->row[b] = row;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) add += __shfl_down_sync(0xFFFFFFFFu, add, o);
    if (t == 0) {
        ctl->live[j] = live | takem;
        take_sh[j] = __popc(takem);
        add_sh[j] = add;
    }
    __syncthreads();
    if (b == 0) {
        uint32_t took = 0;
        unsigned long long adds = 0;
        for (int i = 0; i < V; ++i) {
            took += take_sh[i];
            adds += add_sh[i];
        }
        if (from_list)
            ctl->next_query += took;
        else
            ctl->nseed = 0;
        ctl->f_edges += adds;
        ctl->push = batch_push_pick(ctl->f_edges, ctl->divisor, m);
    }
}

// Words a thread holds of a vertex's row of 32 V lanes in the wide (V > 1)
// kernels: V <= 4, one vector of V words, lanes V t .. V t + V - 1; V == 8, two
// vectors of 4 words, lanes 4 t .. 4 t + 3 and 128 + 4 t .. 128 + 4 t + 3.  A
// vector never straddles a line of 32 lanes.
template <int V>
struct Wide {
    static constexpr int kVec = V == 8 ? 2 : 1;  // vectors per thread
    static constexpr int kW = V == 8 ? 4 : V;    // words per vector
    // first lane of vector k of thread t
    __device__ __forceinline__ static uint32_t lane0(uint32_t t, int k) { return (uint32_t)k * 128u + kW * t; }
    __device__ __forceinline__ static uint32_t line(uint32_t t, int k) { return lane0(t, k) / kLanes; }
};

// vector k of thread t of row `row` (kW words), or kInf words when `take` is false
template <int V>
__device__ __forceinline__ void wide_load(const uint32_t* __restrict__ row, uint32_t t, int k, bool take,
                                          uint32_t* w) {
    if (V == 2) {
        uint2 x = make_uint2(kInf, kInf);
        if (take) x = __ldg(reinterpret_cast<const uint2*>(row) + t);
        w[0] = x.x, w[1] = x.y;
    } else {
        uint4 x = make_uint4(kInf, kInf, kInf, kInf);
        if (take) x = __ldg(reinterpret_cast<const uint4*>(row) + (size_t)k * 32 + t);
        w[0] = x.x, w[1] = x.y, w[2] = x.z, w[3] = x.w;
    }
}

template <int V>
__device__ __forceinline__ void wide_store(uint32_t* __restrict__ row, uint32_t t, int k, const uint32_t* w) {
    if (V == 2)
        reinterpret_cast<uint2*>(row)[t] = make_uint2(w[0], w[1]);
    else
        reinterpret_cast<uint4*>(row)[(size_t)k * 32 + t] = make_uint4(w[0], w[1], w[2], w[3]);
}

// The one-line pull's lowered minima of one destination, in two steps so that
// the atomic's round trip to L2 overlaps the next destination's edges: issue()
// sends one coalesced row of atomicMin (lane b holds the minimum for lane b) and
// keeps the values it returns; finish() (at the next issue, or at the end of the
// warp's chunk) marks the lanes whose value dropped.  (The wide pull keeps the
// same two steps inside its kernel.)
struct Flush1 {
    uint32_t v = 0, pend = 0;  // destination, and 1 while its atomics are outstanding
    uint32_t r = kInf, old = kInf;

    __device__ __forceinline__ void finish(uint32_t lane, uint32_t* __restrict__ cmask, uint32_t* __restrict__ next,
                                           BatchCounters* __restrict__ ctr) {
        if (pend) {
            const unsigned mask = __ballot_sync(0xFFFFFFFFu, r < old);
            if (mask && lane == 0) mark_lowered<1>(v, 0u, 1u, mask, cmask, nullptr, next, ctr);
        }
        pend = 0;
    }

    __device__ __forceinline__ void issue(uint32_t dst, uint32_t run, uint32_t lane, uint32_t* __restrict__ dist,
                                          uint32_t* __restrict__ cmask, uint32_t* __restrict__ next,
                                          BatchCounters* __restrict__ ctr) {
        finish(lane, cmask, next, ctr);
        r = run;
        old = kInf;
        if (r != kInf) old = atomicMin(&dist[(uint64_t)dst * kLanes + lane], r);
        v = dst;
        pend = 1;
    }
};

// run = min(run, s + w) for a sender value s, and run unchanged for s = kInf (no
// message): min(s, kInf - w) + w is kInf then.  No sum reaches kInf otherwise:
// a value whose messages would is refused when it is published (apply, refill).
__device__ __forceinline__ void batch_fold(uint32_t& run, uint32_t s, uint32_t w) {
    run = min(run, min(s, kInf - w) + w);
}

// end of a row relative to the start of a chunk, clamped to 32 bits: a chunk holds at
// most `chunk` edges, so every value from there up means "ends after this chunk"
__device__ __forceinline__ uint32_t chunk_rel_end(uint64_t row_end, uint64_t e_begin) {
    const uint64_t r = row_end - e_begin;
    return r < 0xFFFFFFFFull ? (uint32_t)r : 0xFFFFFFFFu;
}

// Ends of 32 consecutive rows of the in-edge lists, relative to a chunk's first
// edge, one per lane: the destination row of an edge is found with one ballot,
// and the offsets are loaded once per 32 rows, not once per row.
struct RowWindow {
    uint32_t base;   // row held by lane 0
    uint32_t end_l;  // lane l: end of row base + l (0xFFFFFFFF past the last row)
    __device__ __forceinline__ void load(const uint64_t* __restrict__ csc_off, uint32_t n, uint32_t first,
                                         uint64_t e_begin, uint32_t lane) {
        base = first;
        const uint64_t r = (uint64_t)first + lane;
        end_l = r < n ? chunk_rel_end(csc_off[r + 1], e_begin) : 0xFFFFFFFFu;
    }
    // row and end of the row holding chunk-relative edge e, at or after row `base`
    __device__ __forceinline__ void seek(const uint64_t* __restrict__ csc_off, uint32_t n, uint64_t e_begin,
                                         uint32_t e, uint32_t lane, uint32_t& row, uint32_t& bound) {
        unsigned gt = __ballot_sync(0xFFFFFFFFu, end_l > e);
        while (gt == 0) {  // ends at most at the last row, whose end exceeds every edge of the chunk
            load(csc_off, n, base + 32, e_begin, lane);
            gt = __ballot_sync(0xFFFFFFFFu, end_l > e);
        }
        const int i = __ffs(gt) - 1;
        row = base + (uint32_t)i;
        bound = __shfl_sync(0xFFFFFFFFu, end_l, i);
    }
};

// source and weight of chunk-relative in-edge j (0 and 1 past the chunk's end)
template <int kWeightKind>
__device__ __forceinline__ void edge_ids(const uint32_t* __restrict__ csc_src, const uint8_t* __restrict__ w8,
                                         const uint32_t* __restrict__ w32, uint64_t e_begin, uint32_t j,
                                         uint32_t len, uint32_t& u, uint32_t& w) {
    u = 0;
    w = 1;
    if (j < len) {
        u = __ldcs(csc_src + e_begin + j);
        if (kWeightKind == 1) w = __ldcs(w8 + e_begin + j);
        if (kWeightKind == 2) w = __ldcs(w32 + e_begin + j);
    }
}

// Pull form of a superstep with one line.  A warp per chunk of in-edges: 32
// edges at a time, one ballot keeps the edges whose source sends in some lane,
// and those edges are then taken one after another by the whole warp, kUnroll of
// them in flight; only the lanes that send from the source load their word (the
// line's other sectors are not fetched).  The next group's sender words and the
// one after's ids are loaded while the current group is folded.
template <int kWeightKind>
__global__ void __launch_bounds__(256) batch_pull_kernel(
    const uint64_t* __restrict__ csc_off, const uint32_t* __restrict__ csc_src, const uint8_t* __restrict__ w8,
    const uint32_t* __restrict__ w32, const uint32_t* __restrict__ chunk_row, uint64_t chunks, uint32_t n,
    uint64_t m, const uint32_t* __restrict__ sval, const uint32_t* __restrict__ smask, uint32_t* __restrict__ dist,
    uint32_t* __restrict__ cmask, uint32_t* fr0, uint32_t* fr1, const BatchCtl* __restrict__ ctl,
    BatchCounters* __restrict__ ctr, uint32_t chunk) {
    constexpr int kUnroll = 4;  // edges in flight per warp (8 and 16 measured slower)
    if (ctl->push) return;
    uint32_t* __restrict__ next = fr_next(fr0, fr1, ctl);
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t c = warp; c < chunks; c += nwarps) {
        const uint64_t e_begin = c * chunk;
        const uint32_t len = (uint32_t)(e_begin + chunk < m ? chunk : m - e_begin);
        RowWindow win;
        win.load(csc_off, n, chunk_row[c], e_begin, lane);
        uint32_t row = win.base;
        uint32_t bound = __shfl_sync(0xFFFFFFFFu, win.end_l, 0);  // row end, relative to the chunk (may exceed len)
        uint32_t run[1] = {kInf};
        uint32_t pend = 0;  // some lane folded a message since the last flush (warp-uniform)
        Flush1 fl;
        uint32_t u_l, w_l, u_1, w_1, u_2, w_2;
        edge_ids<kWeightKind>(csc_src, w8, w32, e_begin, lane, len, u_l, w_l);
        uint32_t a_l = lane < len ? __ldg(smask + u_l) : 0u;
        edge_ids<kWeightKind>(csc_src, w8, w32, e_begin, 32 + lane, len, u_1, w_1);
        for (uint32_t j0 = 0; j0 < len; j0 += 32) {
            const uint32_t a_1 = j0 + 32 + lane < len ? __ldg(smask + u_1) : 0u;
            edge_ids<kWeightKind>(csc_src, w8, w32, e_begin, j0 + 64 + lane, len, u_2, w_2);
            // only in-edges whose source sends for some lane
            unsigned active = __ballot_sync(0xFFFFFFFFu, a_l != 0);
            const uint32_t jmax = active ? j0 + 31 - __clz(active) : 0;  // last active edge of the group
            const bool one_row = jmax < bound;  // every active edge belongs to the current row
            while (active) {
                int jj[kUnroll];
                uint32_t wq[kUnroll], s[kUnroll];
#pragma unroll
                for (int q = 0; q < kUnroll; ++q) {
                    jj[q] = active ? __ffs(active) - 1 : -1;
                    if (active) active &= active - 1;
                    const int src_lane = jj[q] < 0 ? 0 : jj[q];
                    const uint32_t u = __shfl_sync(0xFFFFFFFFu, u_l, src_lane);
                    wq[q] = __shfl_sync(0xFFFFFFFFu, w_l, src_lane);
                    const uint32_t a = jj[q] >= 0 ? __shfl_sync(0xFFFFFFFFu, a_l, src_lane) : 0u;
                    s[q] = (a >> lane) & 1u ? __ldg(sval + (uint64_t)u * kLanes + lane) : kInf;
                }
#pragma unroll
                for (int q = 0; q < kUnroll; ++q) {
                    if (jj[q] < 0) continue;
                    if (!one_row) {
                        const uint32_t e = j0 + (uint32_t)jj[q];
                        if (e >= bound) {  // the destination changed (warp-uniform)
                            if (pend) fl.issue(row, run[0], lane, dist, cmask, next, ctr);
                            run[0] = kInf;
                            pend = 0;
                            win.seek(csc_off, n, e_begin, e, lane, row, bound);
                        }
                    }
                    batch_fold(run[0], s[q], wq[q]);
                    pend = 1;
                }
            }
            u_l = u_1, w_l = w_1, a_l = a_1;
            u_1 = u_2, w_1 = w_2;
        }
        if (pend) fl.issue(row, run[0], lane, dist, cmask, next, ctr);
        fl.finish(lane, cmask, next, ctr);
    }
}

// per-thread asynchronous copies into shared memory (cp.async): bytes = 8 or 16
template <int kBytes>
__device__ __forceinline__ void cp_async(uint32_t dst_shared, const void* src) {
    if (kBytes == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst_shared), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(dst_shared), "l"(src), "n"(kBytes)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int kPending>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kPending) : "memory");
}

// Pull form of a superstep with more than one line.  As batch_pull_kernel, but
// the source rows of the active edges are staged in a per-warp ring of
// kRingSlots rows in shared memory: each thread copies its own words of an
// edge's row (in the lines that hold a sender) with cp.async and folds them
// kRingSlots edges later, so that a warp has that many rows in flight without
// holding them in registers.  A thread reads back only what it copied itself;
// the edge's position, weight and sender lines go through a per-warp slot in
// shared memory.
//
// A row of L lines maps to the warp's threads as RowMap<L> says: 16-byte
// vectors for the first 4 (L / 4) lines, then one word per thread for each of
// the L % 4 lines left, so every thread folds exactly L words.
// Dynamic shared memory: ring_smem_bytes(L).
constexpr int kRingWarps = 4;   // warps per block
constexpr int kRingSlots = 16;  // rows in flight per warp

__host__ __device__ constexpr size_t ring_smem_bytes(uint32_t L) {
    return sizeof(uint32_t) * kRingWarps * ((size_t)L * kLanes + (size_t)kRingSlots * L * kLanes) +
           sizeof(uint4) * kRingWarps * kRingSlots;
}

template <int L>
struct RowMap {
    static constexpr int kVec = L / 4;               // vectors: lanes 128 k + 4 t .. + 3 (line 4 k + t / 8)
    static constexpr int kScal = L % 4;              // words: lane 32 (4 kVec + i) + t (line 4 kVec + i)
    static constexpr int kWords = 4 * kVec + kScal;
    static_assert(kWords == L, "every thread holds exactly L lanes of a row");
    __device__ __forceinline__ static uint32_t vec_off(uint32_t t, int k) { return 128u * k + 4u * t; }
    __device__ __forceinline__ static uint32_t vec_line(uint32_t t, int k) { return 4u * k + t / 8u; }
    __device__ __forceinline__ static uint32_t scal_off(uint32_t t, int i) { return 32u * (4 * kVec + i) + t; }
    static constexpr uint32_t scal_line(int i) { return 4u * kVec + i; }
};

// run = min(run, s + w) for a sender value s, run unchanged for s = kInf (as
// batch_fold), with the fused add-min
__device__ __forceinline__ void batch_fold2(uint32_t& run, uint32_t s, uint32_t w, uint32_t lim) {
    run = __viaddmin_u32(min(s, lim), w, run);
}

template <int kWeightKind, int L>
__global__ void __launch_bounds__(kRingWarps * 32) batch_pull_ring_kernel(
    const uint64_t* __restrict__ csc_off, const uint32_t* __restrict__ csc_src, const uint8_t* __restrict__ w8,
    const uint32_t* __restrict__ w32, const uint32_t* __restrict__ chunk_row, uint64_t chunks, uint32_t n,
    uint64_t m, const uint32_t* __restrict__ sval, const uint32_t* __restrict__ sany,
    uint32_t* __restrict__ dist, uint32_t* __restrict__ cmask, uint32_t* __restrict__ cany, uint32_t* fr0,
    uint32_t* fr1, const BatchCtl* __restrict__ ctl, BatchCounters* __restrict__ ctr, uint32_t chunk) {
    using M = RowMap<L>;
    constexpr int kSlots = kRingSlots;
    constexpr uint32_t kRow = L * kLanes;  // words per row
    extern __shared__ __align__(16) uint32_t ring_dyn[];
    if (ctl->push) return;
    uint32_t* __restrict__ next = fr_next(fr0, fr1, ctl);
    const uint32_t lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint4* meta = reinterpret_cast<uint4*>(ring_dyn) + wib * kSlots;  // per slot: edge, weight, lines
    uint32_t* __restrict__ sh = ring_dyn + (kRingWarps * kSlots * 4) + wib * kRow;  // flush buffer
    const uint32_t* ring = ring_dyn + (kRingWarps * kSlots * 4) + kRingWarps * kRow + wib * kSlots * kRow;
    const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(ring);
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t vline[M::kVec > 0 ? M::kVec : 1], voff[M::kVec > 0 ? M::kVec : 1], soff[M::kScal > 0 ? M::kScal : 1];
#pragma unroll
    for (int k = 0; k < M::kVec; ++k) vline[k] = M::vec_line(lane, k), voff[k] = M::vec_off(lane, k);
#pragma unroll
    for (int i = 0; i < M::kScal; ++i) soff[i] = M::scal_off(lane, i);
    for (uint64_t c = warp; c < chunks; c += nwarps) {
        const uint64_t e_begin = c * chunk;
        const uint32_t len = (uint32_t)(e_begin + chunk < m ? chunk : m - e_begin);
        RowWindow win;
        win.load(csc_off, n, chunk_row[c], e_begin, lane);
        uint32_t row = win.base;
        uint32_t bound = __shfl_sync(0xFFFFFFFFu, win.end_l, 0);
        uint32_t run[L];  // the thread's words: vectors, then single words
#pragma unroll
        for (int j = 0; j < L; ++j) run[j] = kInf;
        uint32_t pend = 0;
        uint32_t f_v = 0, f_pend = 0, f_r[L], f_old[L];  // the flush in flight: destination, lines, values
        // the outstanding flush: mark the lanes whose value dropped
        auto finish = [&]() {
#pragma unroll
            for (int j = 0; j < L; ++j) {
                if (!((f_pend >> j) & 1u)) continue;
                const unsigned mask = __ballot_sync(0xFFFFFFFFu, f_r[j] < f_old[j]);
                if (mask && lane == 0) mark_lowered<L>(f_v, (uint32_t)j, L, mask, cmask, cany, next, ctr);
            }
            f_pend = 0;
        };
        // the current destination's minima: to line order, one coalesced row of atomicMin per line
        auto flush = [&]() {
            finish();
#pragma unroll
            for (int k = 0; k < M::kVec; ++k)
                *reinterpret_cast<uint4*>(sh + voff[k]) =
                    make_uint4(run[4 * k], run[4 * k + 1], run[4 * k + 2], run[4 * k + 3]);
#pragma unroll
            for (int i = 0; i < M::kScal; ++i) sh[soff[i]] = run[4 * M::kVec + i];
            __syncwarp();
#pragma unroll
            for (int j = 0; j < L; ++j) {
                f_r[j] = sh[j * kLanes + lane];
                f_old[j] = kInf;
                if (((pend >> j) & 1u) && f_r[j] != kInf)
                    f_old[j] = atomicMin(&dist[slot_at(row, j, lane, L)], f_r[j]);
            }
            __syncwarp();  // the buffer is free for the next flush
            f_v = row;
            f_pend = pend;
        };
        uint32_t issued = 0, folded = 0;
        // fold the oldest staged edge (its copies have completed)
        auto fold_one = [&]() {
            const uint32_t slot = folded % kSlots;
            const uint4 md = meta[slot];  // edge, weight, lines
            const uint32_t e = md.x, w = md.y, a = md.z, lim = kInf - w;
            if (e >= bound) {  // the destination changed (warp-uniform)
                if (pend) flush();
#pragma unroll
                for (int j = 0; j < L; ++j) run[j] = kInf;
                pend = 0;
                win.seek(csc_off, n, e_begin, e, lane, row, bound);
            }
            const uint32_t* x = ring + slot * kRow;
#pragma unroll
            for (int k = 0; k < M::kVec; ++k) {
                if (!((a >> vline[k]) & 1u)) continue;
                const uint4 y = *reinterpret_cast<const uint4*>(x + voff[k]);
                batch_fold2(run[4 * k + 0], y.x, w, lim);
                batch_fold2(run[4 * k + 1], y.y, w, lim);
                batch_fold2(run[4 * k + 2], y.z, w, lim);
                batch_fold2(run[4 * k + 3], y.w, w, lim);
            }
#pragma unroll
            for (int i = 0; i < M::kScal; ++i)
                if ((a >> M::scal_line(i)) & 1u) batch_fold2(run[4 * M::kVec + i], x[soff[i]], w, lim);
            pend |= a;
            ++folded;
        };
        uint32_t u_l, w_l, u_1, w_1, u_2, w_2;
        edge_ids<kWeightKind>(csc_src, w8, w32, e_begin, lane, len, u_l, w_l);
        uint32_t a_l = lane < len ? __ldg(sany + u_l) : 0u;
        edge_ids<kWeightKind>(csc_src, w8, w32, e_begin, 32 + lane, len, u_1, w_1);
        for (uint32_t j0 = 0; j0 < len; j0 += 32) {
            const uint32_t a_1 = j0 + 32 + lane < len ? __ldg(sany + u_1) : 0u;
            edge_ids<kWeightKind>(csc_src, w8, w32, e_begin, j0 + 64 + lane, len, u_2, w_2);
            unsigned active = __ballot_sync(0xFFFFFFFFu, a_l != 0);
            while (active) {
                const int jj = __ffs(active) - 1;
                active &= active - 1;
                const uint32_t u = __shfl_sync(0xFFFFFFFFu, u_l, jj);
                const uint32_t a = __shfl_sync(0xFFFFFFFFu, a_l, jj);
                if (issued - folded == (uint32_t)kSlots) {
                    cp_async_wait<kSlots - 1>();
                    fold_one();
                }
                const uint32_t slot = issued % kSlots;
                const uint32_t* rowp = sval + (uint64_t)u * kRow;
                const uint32_t dst = ring_s + slot * kRow * 4u;
#pragma unroll
                for (int k = 0; k < M::kVec; ++k)
                    if ((a >> vline[k]) & 1u) cp_async<16>(dst + voff[k] * 4u, rowp + voff[k]);
#pragma unroll
                for (int i = 0; i < M::kScal; ++i)
                    if ((a >> M::scal_line(i)) & 1u) cp_async<4>(dst + soff[i] * 4u, rowp + soff[i]);
                cp_async_commit();
                if (lane == (uint32_t)jj) meta[slot] = make_uint4(j0 + (uint32_t)jj, w_l, a_l, 0u);
                __syncwarp();
                ++issued;
            }
            u_l = u_1, w_l = w_1, a_l = a_1;
            u_1 = u_2, w_1 = w_2;
        }
        cp_async_wait<0>();
        while (folded < issued) fold_one();
        if (pend) flush();
        finish();
    }
}

// Push supersteps only: the current senders' out-edge lists as tasks of
// kPushChunk edges, (sender << 32 | chunk).  A warp takes 32 senders at a time
// and claims their tasks with one atomic.
__global__ void batch_tasks_kernel(uint32_t* fr0, uint32_t* fr1, const BatchCtl* __restrict__ ctl,
                                   const uint64_t* __restrict__ off, unsigned long long* __restrict__ tasks,
                                   BatchCounters* __restrict__ ctr) {
    if (!ctl->push) return;
    const uint32_t* __restrict__ F = fr_cur(fr0, fr1, ctl);
    const uint32_t f = ctl->f;
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i0 = warp * 32; i0 < f; i0 += nwarps * 32) {
        const uint64_t i = i0 + lane;
        uint32_t u = 0, nt = 0;
        if (i < f) {
            u = F[i];
            nt = (uint32_t)((off[u + 1] - off[u] + kPushChunk - 1) / kPushChunk);
        }
        uint32_t incl = nt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= (uint32_t)o) incl += x;
        }
        unsigned base = 0;
        if (lane == 31 && incl) base = atomicAdd(&ctr->ntasks, incl);
        base = __shfl_sync(0xFFFFFFFFu, base, 31) + incl - nt;
        for (uint32_t c = 0; c < nt; ++c) tasks[base + c] = ((unsigned long long)u << 32) | c;
    }
}

// candidate s + w for a sender value s < kInf; a sum reaching kInf is reported
__device__ __forceinline__ uint32_t batch_cand(uint32_t s, uint32_t w, BatchCounters* __restrict__ ctr) {
    unsigned long long d = (unsigned long long)s + w;
    if (d >= kInf) {
        atomicOr(&ctr->status, kStatusOverflow);
        d = kInf - 1;
    }
    return (uint32_t)d;
}

// Push form of a superstep: a warp per task (sender u, chunk of its out-edges).
// Per line of u with a sender: when few lanes send (kSparseLanes or fewer),
// lanes take different edges and loop over those lanes, one atomicMin per
// (edge, lane); else lane b sends sval[u][j][b] + w along each edge, one
// coalesced row of atomics per (edge, line).
constexpr int kSparseLanes = 4;

template <int kWeightKind, int V>
__global__ void __launch_bounds__(256) batch_push_kernel(
    const uint64_t* __restrict__ off, const uint32_t* __restrict__ col, const uint8_t* __restrict__ w8,
    const uint32_t* __restrict__ w32, const unsigned long long* __restrict__ tasks, uint32_t L,
    const uint32_t* __restrict__ sval, const uint32_t* __restrict__ smask, const uint32_t* __restrict__ sany,
    uint32_t* __restrict__ dist, uint32_t* __restrict__ cmask, uint32_t* __restrict__ cany, uint32_t* fr0,
    uint32_t* fr1, const BatchCtl* __restrict__ ctl, BatchCounters* __restrict__ ctr) {
    if (!ctl->push) return;
    uint32_t* __restrict__ next = fr_next(fr0, fr1, ctl);
    const uint32_t nt = ctr->ntasks;
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t t = warp; t < nt; t += nwarps) {
        const unsigned long long task = tasks[t];
        const uint32_t u = (uint32_t)(task >> 32);
        const uint64_t e_beg = off[u] + (uint64_t)(uint32_t)task * kPushChunk;
        const uint64_t e_end = min(off[u + 1], e_beg + kPushChunk);
        const uint32_t lines = V == 1 ? (smask[u] ? 1u : 0u) : sany[u];  // lines of u with a sender (warp-uniform)
        uint32_t dense = 0;                                               // lines sent as coalesced rows
#pragma unroll
        for (int j = 0; j < V; ++j) {
            if (!((lines >> j) & 1u)) continue;
            const uint32_t senders = smask[(uint64_t)u * L + j];  // sending lanes of line j (warp-uniform)
            if (__popc(senders) > kSparseLanes) {
                dense |= 1u << j;
                continue;
            }
            // lane per edge (no warp-collective step); the sending lanes one after another
            for (uint64_t e = e_beg + lane; e < e_end; e += 32) {
                const uint32_t v = __ldg(col + e);
                uint32_t w = 1;
                if (kWeightKind == 1) w = __ldg(w8 + e);
                if (kWeightKind == 2) w = __ldg(w32 + e);
                for (uint32_t rest = senders; rest; rest &= rest - 1) {
                    const uint32_t b = __ffs(rest) - 1;
                    const uint32_t s = __ldg(sval + slot_at(u, j, b, L));
                    if (s != kInf) {
                        const uint32_t d = batch_cand(s, w, ctr);
                        if (d < atomicMin(&dist[slot_at(v, j, b, L)], d))
                            mark_lowered<V>(v, (uint32_t)j, L, 1u << b, cmask, cany, next, ctr);
                    }
                }
            }
        }
        if (!dense) continue;
        // kInf: the lane does not send from u in that line
        uint32_t s[V];
#pragma unroll
        for (int j = 0; j < V; ++j) s[j] = (dense >> j) & 1u ? sval[slot_at(u, j, lane, L)] : kInf;
        for (uint64_t j0 = e_beg; j0 < e_end; j0 += 32) {
            const uint32_t cnt = (uint32_t)min((uint64_t)32, e_end - j0);
            uint32_t v_l = 0, w_l = 1;
            if (lane < cnt) {
                v_l = __ldg(col + j0 + lane);
                if (kWeightKind == 1) w_l = __ldg(w8 + j0 + lane);
                if (kWeightKind == 2) w_l = __ldg(w32 + j0 + lane);
            }
            for (uint32_t q = 0; q < cnt; ++q) {
                const uint32_t v = __shfl_sync(0xFFFFFFFFu, v_l, q);
                const uint32_t w = __shfl_sync(0xFFFFFFFFu, w_l, q);
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    if (!((dense >> j) & 1u)) continue;
                    bool changed = false;
                    if (s[j] != kInf) {
                        const uint32_t d = batch_cand(s[j], w, ctr);
                        changed = d < atomicMin(&dist[slot_at(v, j, lane, L)], d);
                    }
                    const unsigned mask = __ballot_sync(0xFFFFFFFFu, changed);
                    if (mask && lane == 0) mark_lowered<V>(v, (uint32_t)j, L, mask, cmask, cany, next, ctr);
                }
            }
        }
    }
}

// previous senders: snapshot rows back to kInf, sender masks cleared
template <int V>
__global__ void batch_reset_kernel(uint32_t* fr0, uint32_t* fr1, const BatchCtl* __restrict__ ctl, uint32_t L,
                                   uint32_t* __restrict__ sval, uint32_t* __restrict__ smask,
                                   uint32_t* __restrict__ sany) {
    using W = Wide<V>;
    const uint32_t* __restrict__ F = fr_cur(fr0, fr1, ctl);
    const uint32_t f = ctl->f;
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t inf[W::kW];
#pragma unroll
    for (int i = 0; i < W::kW; ++i) inf[i] = kInf;
    for (uint64_t i = warp; i < f; i += nwarps) {
        const uint32_t u = F[i];
        if (V == 1) {
            sval[(uint64_t)u * kLanes + lane] = kInf;
            if (lane == 0) smask[u] = 0;
            continue;
        }
        const uint32_t lines = sany[u];
        uint32_t* rowp = sval + (uint64_t)u * (L * kLanes);
#pragma unroll
        for (int k = 0; k < W::kVec; ++k)
            if ((lines >> W::line(lane, k)) & 1u) wide_store<V>(rowp, lane, k, inf);
        if (lane < L && ((lines >> lane) & 1u)) smask[(uint64_t)u * L + lane] = 0;
        __syncwarp();
        if (lane == 0) sany[u] = 0;
    }
}

// Next senders: publish their new values (kInf for the lanes that did not
// change), count their messages per lane, and refuse a value whose messages
// would reach kInf (x + the largest out-edge weight of the vertex >= kInf).
template <int V>
__global__ void batch_apply_kernel(uint32_t* fr0, uint32_t* fr1, const BatchCtl* __restrict__ ctl, uint32_t n,
                                   uint32_t L, const uint64_t* __restrict__ off, const uint32_t* __restrict__ wmax_out,
                                   const uint32_t* __restrict__ dist, uint32_t* __restrict__ sval,
                                   uint32_t* __restrict__ smask, uint32_t* __restrict__ sany,
                                   uint32_t* __restrict__ cmask, uint32_t* __restrict__ cany,
                                   BatchCounters* __restrict__ ctr) {
    using W = Wide<V>;
    const uint32_t* __restrict__ F = fr_next(fr0, fr1, ctl);
    const uint32_t f = min(ctr->next_size, n);  // a larger count is reported by the step kernel
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long msgs[V], edges = 0;
#pragma unroll
    for (int j = 0; j < V; ++j) msgs[j] = 0;
    bool overflow = false;
    if constexpr (V == 1) {
        for (uint64_t i = warp; i < f; i += nwarps) {
            const uint32_t v = F[i];
            const uint64_t deg = off[v + 1] - off[v];
            const uint32_t lim = kInf - wmax_out[v];  // a sent value must stay below this
            const uint32_t mask = cmask[v];
            const bool mine = (mask >> lane) & 1u;
            const uint32_t x = mine ? dist[(uint64_t)v * kLanes + lane] : kInf;
            overflow |= mine && x >= lim;
            sval[(uint64_t)v * kLanes + lane] = x;
            if (mine) msgs[0] += deg;
            edges += deg;
            __syncwarp();
            if (lane == 0) {
                smask[v] = mask;
                cmask[v] = 0;
            }
        }
    } else {
        // only the vectors holding a lowered lane are read and written (the others
        // are kInf already: the previous senders' rows were reset)
        for (uint64_t i = warp; i < f; i += nwarps) {
            const uint32_t v = F[i];
            const uint32_t lines = cany[v];
            const uint64_t deg = off[v + 1] - off[v];
            const uint32_t lim = kInf - wmax_out[v];  // a sent value must stay below this
            const uint64_t rowi = (uint64_t)v * (L * kLanes);
#pragma unroll
            for (int k = 0; k < W::kVec; ++k) {
                const uint32_t j = W::line(lane, k);
                if (!((lines >> j) & 1u)) continue;
                const uint32_t mine =
                    (cmask[(uint64_t)v * L + j] >> (W::lane0(lane, k) % kLanes)) & ((1u << W::kW) - 1u);
                if (!mine) continue;
                uint32_t x[W::kW];
                wide_load<V>(dist + rowi, lane, k, true, x);
#pragma unroll
                for (int q = 0; q < W::kW; ++q) {
                    if ((mine >> q) & 1u) {
                        overflow |= x[q] >= lim;
                        msgs[k * W::kW + q] += deg;
                    } else {
                        x[q] = kInf;
                    }
                }
                wide_store<V>(sval + rowi, lane, k, x);
            }
            edges += deg * (uint64_t)__popc(lines);
            __syncwarp();  // every thread has read the lowered-lane masks
            if (lane < L && ((lines >> lane) & 1u)) {
                const uint64_t wi = (uint64_t)v * L + lane;
                smask[wi] = cmask[wi];
                cmask[wi] = 0;
            }
            if (lane == 0) {
                sany[v] = lines;
                cany[v] = 0;
            }
        }
    }
    if (overflow) atomicOr(&ctr->status, kStatusOverflow);
    if (V == 1) {
        if (msgs[0]) atomicAdd(&ctr->msgs[lane], msgs[0]);
    } else {
#pragma unroll
        for (int k = 0; k < W::kVec; ++k)
#pragma unroll
            for (int q = 0; q < W::kW; ++q)
                if (msgs[k * W::kW + q]) atomicAdd(&ctr->msgs[W::lane0(lane, k) + q], msgs[k * W::kW + q]);
    }
    if (lane == 0 && edges) atomicAdd(&ctr->edges, edges);
}

// largest out-edge weight of each vertex (1 without weights, 0 without out-edges)
__global__ void batch_wmax_kernel(const uint64_t* __restrict__ off, const uint8_t* __restrict__ w8,
                                  const uint32_t* __restrict__ w32, uint32_t n, uint32_t* __restrict__ wmax_out) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        uint32_t mx = 0;
        for (uint64_t e = off[v]; e < off[v + 1]; ++e) {
            const uint32_t w = w8 ? (uint32_t)w8[e] : w32 ? w32[e] : 1u;
            mx = w > mx ? w : mx;
        }
        wmax_out[v] = mx;
    }
}

// Rows of queries whose source has no out-edges: the run ends after superstep 0
// (count 1) with only the source reached.
__global__ void batch_fill_kernel(uint32_t* __restrict__ out, uint64_t stride, uint32_t n,
                                  const uint32_t* __restrict__ src, const uint32_t* __restrict__ rows, uint32_t cnt,
                                  uint32_t* __restrict__ steps) {
    const uint64_t total = (uint64_t)cnt * n;
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += step) {
        const uint32_t r = (uint32_t)(i / n), v = (uint32_t)(i % n);
        out[(uint64_t)rows[r] * stride + v] = v == src[r] ? 0u : kInf;
        if (v == 0 && steps) steps[rows[r]] = 1;
    }
}

// End of a superstep: a live lane whose next senders send nothing has finished
// (its count is final; its distances stay in place until harvested); otherwise
// it runs another superstep.  The next frontier
// becomes current, the counters are cleared, and the WHILE condition says
// whether the graph runs another superstep: while a lane holds a query or the
// source list has more, not past kLoopCap in one launch, and with host seeding
// not past a superstep in which a lane finished (or when queries wait for a
// free lane).  One block of 32 V threads, thread b = lane b.
template <int V>
__global__ void batch_step_kernel(BatchCtl* __restrict__ ctl, BatchCounters* __restrict__ ctr, uint32_t n,
                                  cudaGraphConditionalHandle loop, int in_graph) {
    __shared__ uint32_t live_sh[V], fin_sh[V];
    const uint32_t b = threadIdx.x, j = b / kLanes, t = b % kLanes;
    const uint32_t live = ctl->live[j];
    bool fin = false;
    if ((live >> t) & 1u) {
        if (ctr->msgs[b] > 0)
            ++ctl->count[b];
        else
            fin = true;
    }
    ctr->msgs[b] = 0;
    const unsigned finm = __ballot_sync(0xFFFFFFFFu, fin);
    if (fin && ctl->steps_out) ctl->steps_out[ctl->row[b]] = ctl->count[b];
    if (t == 0) {
        ctl->live[j] = live & ~finm;
        live_sh[j] = live & ~finm;
        fin_sh[j] = finm;
    }
    __syncthreads();
    if (b == 0) {
        const bool from_list = ctl->nqueries != 0;
        uint32_t any_live = 0, any_fin = 0;
        bool some_free = false;
        for (int i = 0; i < V; ++i) {
            any_live |= live_sh[i];
            any_fin |= fin_sh[i];
            some_free |= live_sh[i] != 0xFFFFFFFFu;
        }
        // Finished lanes are harvested when their lanes are needed (queries left in
        // the list), when no lane runs any more, or at once for host seeding; else
        // they wait, so that queries started together are harvested in one pass.
        const bool queued = from_list && ctl->next_query < ctl->nqueries;
        const bool harvest = !from_list || queued || any_live == 0;
        // with a source list and nothing left to run, the lanes are not reused: the
        // harvest leaves their values in place and the next session clears them
        ctl->final_harvest = from_list && !queued && any_live == 0 ? 1u : 0u;
        uint32_t any_harvest = 0;
        for (int i = 0; i < V; ++i) {
            const uint32_t p = ctl->pending[i] | fin_sh[i];
            ctl->finished[i] = harvest ? p : 0u;
            ctl->pending[i] = harvest ? 0u : p;
            any_harvest |= harvest ? p : 0u;
        }
        ++ctl->supersteps;
        if (!ctl->push) ++ctl->pull_supersteps;
        if (any_harvest) ++ctl->harvests;
        const uint32_t fn = ctr->next_size;
        uint32_t status = ctl->status | ctr->status;
        if (fn > n) status |= kStatusInternal;
        ctl->status = status;
        ctl->f = fn <= n ? fn : 0u;
        ctl->cur ^= 1u;
        ctl->f_edges = ctr->edges;
        ctr->next_size = 0;
        ctr->status = 0;
        ctr->edges = 0;
        ctr->ntasks = 0;
        const bool more = (any_live != 0 || queued) && status == 0;
        bool stop = false;
        if (!from_list && ctl->stop_on_finish) {
            stop = any_fin != 0;
            if (ctl->admit && *ctl->admit && some_free) stop = true;
        }
        ctl->done = !more;
        const unsigned it = ctl->iter + 1;
        const bool again = more && !stop && it < kLoopCap;
        ctl->iter = again ? it : 0u;
        if (in_graph) cudaGraphSetConditional(loop, again ? 1u : 0u);
    }
}

// Finished lanes: out[row][v] = dist[inv[v]][line][lane] for every caller id v,
// and the lane's column back to kInf for its next query (not at a session's final
// harvest: the next session clears the array in one pass).  A thread per caller id
// walks the finished lanes of its vertex's row (one row, cached in L1), and the
// warp's writes of one lane cover 32 consecutive words of its output row.
template <int V>
__global__ void batch_harvest_kernel(const BatchCtl* __restrict__ ctl, const uint32_t* __restrict__ inv, uint32_t n,
                                     uint32_t L, uint32_t* __restrict__ dist) {
    __shared__ uint32_t fin_sh[V];
    __shared__ uint32_t row_sh[V * kLanes];
    uint32_t any = 0;
#pragma unroll
    for (int j = 0; j < V; ++j) any |= ctl->finished[j];
    if (!any) return;  // the same for every thread of the block
    for (uint32_t i = threadIdx.x; i < V * kLanes; i += blockDim.x) row_sh[i] = ctl->row[i];
    if (threadIdx.x < V) fin_sh[threadIdx.x] = ctl->finished[threadIdx.x];
    __syncthreads();
    uint32_t* __restrict__ out = ctl->out;
    const uint64_t stride = ctl->out_stride;
    const bool reset = !ctl->final_harvest;
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += step) {
        uint32_t* d = dist + (uint64_t)inv[v] * (L * kLanes);
#pragma unroll
        for (int j = 0; j < V; ++j) {
            for (uint32_t r = fin_sh[j]; r; r &= r - 1) {
                const uint32_t b = __ffs(r) - 1;
                out[(uint64_t)row_sh[j * kLanes + b] * stride + v] = d[j * kLanes + b];
                if (reset) d[j * kLanes + b] = kInf;
            }
        }
    }
}

unsigned grid_for_warps(uint64_t warps, int sms) {
    uint64_t blocks = (warps + 7) / 8;
    const uint64_t cap = (uint64_t)sms * 16;
    if (blocks < 1) blocks = 1;
    return (unsigned)(blocks < cap ? blocks : cap);
}

// lanes per thread of the wide kernels for rows of L lines: the next of 1, 2, 4, 8
int lines_v(uint32_t L) { return L > 4 ? 8 : L > 2 ? 4 : L > 1 ? 2 : 1; }

}  // namespace

// Batch workspace lives with the graph; allocated on first use.
struct BatchWorkspace {
    uint32_t lines = 0;         // lines per vertex the value arrays hold (0: not allocated yet);
                                // a session with L <= lines lines lays its rows out [n][L][32]
    uint32_t* dist = nullptr;   // [n][L][32]
    uint32_t* sval = nullptr;   // [n][L][32]
    uint32_t* smask = nullptr;  // [n][L]
    uint32_t* cmask = nullptr;  // [n][L]
    uint32_t* sany = nullptr;   // [n]: lines with a sender (used with more than one line)
    uint32_t* cany = nullptr;   // [n]: lines with a lowered lane
    uint32_t* fr[2] = {nullptr, nullptr};
    uint32_t* wmax_out = nullptr;  // [n]: largest out-edge weight of each vertex
    // in-edge chunks of the pull form: [0] for one line (knob batch_chunk), [1] for more
    // (knob batch_wide_chunk)
    struct ChunkSet {
        uint32_t* row = nullptr;  // first row of each chunk
        uint64_t count = 0, cap = 0;
        uint32_t size = 0;  // in-edges per chunk (0: not set up yet)
    } cs[2];
    BatchCounters* ctr = nullptr;
    BatchCtl* ctl = nullptr;
    BatchCtl* h_ctl = nullptr;            // pinned mirror
    unsigned int* h_admit = nullptr;      // mapped host flag (serving)
    unsigned int* d_admit = nullptr;      // its device address
    uint32_t* list = nullptr;             // ipg_sssp_batch: sources (caller ids), then their output rows
    uint32_t* steps = nullptr;            // per query: its superstep count
    uint8_t* sends = nullptr;             // per query: 1 if its source has out-edges
    size_t list_cap = 0;
    unsigned long long* tasks = nullptr;  // push tasks of the current senders
    bool clean = false;                   // dist/sval all kInf, masks and counters zero
    bool dist_dirty = false;              // as clean, except dist (left by a final harvest)
    uint32_t dirty_lines = 0;             // lines of the rows that session used
    ipg_batch_info info{};                // totals of the last ipg_sssp_batch call
    cudaGraphExec_t loop[3][kMaxLines] = {};  // superstep loop, per weight kind and line count
};

static void batch_drop_loops(BatchWorkspace* b) {
    for (auto& per_kind : b->loop)
        for (auto& x : per_kind)
            if (x) {
                cudaGraphExecDestroy(x);
                x = nullptr;
            }
}

static void batch_free_values(BatchWorkspace* b) {
    cudaFree(b->dist);
    cudaFree(b->sval);
    cudaFree(b->smask);
    cudaFree(b->cmask);
    cudaFree(b->sany);
    cudaFree(b->cany);
    b->dist = b->sval = b->smask = b->cmask = b->sany = b->cany = nullptr;
    b->lines = 0;
}

void batch_free(ipg_graph* g) {
    BatchWorkspace* b = (BatchWorkspace*)g->batch;
    if (!b) return;
    batch_free_values(b);
    cudaFree(b->fr[0]);
    cudaFree(b->fr[1]);
    cudaFree(b->wmax_out);
    cudaFree(b->cs[0].row);
    cudaFree(b->cs[1].row);
    cudaFree(b->ctr);
    cudaFree(b->ctl);
    cudaFree(b->tasks);
    cudaFree(b->list);
    cudaFree(b->steps);
    cudaFree(b->sends);
    if (b->h_ctl) cudaFreeHost(b->h_ctl);
    if (b->h_admit) cudaFreeHost(b->h_admit);
    batch_drop_loops(b);
    delete b;
    g->batch = nullptr;
}

// device bytes of the value arrays for `lines` lines per vertex
static size_t batch_value_bytes(uint64_t n, uint32_t lines) {
    return (size_t)n * lines * (2 * kLanes + 2) * sizeof(uint32_t) + (size_t)n * 2 * sizeof(uint32_t);
}

// the parts of the workspace that do not depend on the line count
static ipg_status batch_prepare(ipg_graph* g, cudaStream_t st) {
    IPG_TRY(ensure_csc(g, st));
    if (g->batch) return IPG_OK;
    BatchWorkspace* b = new BatchWorkspace();
    g->batch = b;
    const uint32_t n = g->n;
    IPG_CUDA(cudaMalloc(&b->fr[0], sizeof(uint32_t) * (size_t)n));
    IPG_CUDA(cudaMalloc(&b->fr[1], sizeof(uint32_t) * (size_t)n));
    IPG_CUDA(cudaMalloc(&b->wmax_out, sizeof(uint32_t) * (size_t)(n ? n : 1)));
    if (n) {
        const unsigned grid = (n + 255) / 256 < (uint32_t)sm_count_of(g->device) * 8 ? (n + 255) / 256
                                                                                   : (uint32_t)sm_count_of(g->device) * 8;
        batch_wmax_kernel<<<grid, 256, 0, st>>>(g->off, g->w8, g->w, n, b->wmax_out);
        IPG_CUDA(cudaGetLastError());
    }
    IPG_CUDA(cudaMalloc(&b->ctr, sizeof(BatchCounters)));
    IPG_CUDA(cudaMalloc(&b->ctl, sizeof(BatchCtl)));
    // a sender with d out-edges makes ceil(d / kPushChunk) <= d / kPushChunk + 1 tasks
    const size_t max_tasks = (size_t)n + g->m / kPushChunk + 1;
    IPG_CUDA(cudaMalloc(&b->tasks, sizeof(unsigned long long) * max_tasks));
    IPG_CUDA(cudaHostAlloc(&b->h_ctl, sizeof(BatchCtl), cudaHostAllocDefault));
    IPG_CUDA(cudaHostAlloc(&b->h_admit, sizeof(unsigned int), cudaHostAllocMapped));
    *b->h_admit = 0;
    IPG_CUDA(cudaHostGetDevicePointer((void**)&b->d_admit, b->h_admit, 0));
    return IPG_OK;
}

// value arrays for at least `lines` lines per vertex (reallocated, not kept, when
// more are needed: they hold no query between sessions)
static ipg_status batch_values(ipg_graph* g, BatchWorkspace* b, uint32_t lines) {
    if (b->lines >= lines) return IPG_OK;
    batch_drop_loops(b);  // they refer to the old arrays
    batch_free_values(b);
    b->clean = false;
    const size_t n = g->n ? g->n : 1;
    IPG_CUDA(cudaMalloc(&b->dist, sizeof(uint32_t) * kLanes * lines * n));
    IPG_CUDA(cudaMalloc(&b->sval, sizeof(uint32_t) * kLanes * lines * n));
    IPG_CUDA(cudaMalloc(&b->smask, sizeof(uint32_t) * lines * n));
    IPG_CUDA(cudaMalloc(&b->cmask, sizeof(uint32_t) * lines * n));
    IPG_CUDA(cudaMalloc(&b->sany, sizeof(uint32_t) * n));
    IPG_CUDA(cudaMalloc(&b->cany, sizeof(uint32_t) * n));
    b->lines = lines;
    return IPG_OK;
}

// Lines for a session whose `sending` queries should all start at once: the
// fewest lines (at most kMaxLines) that hold them, fewer if the value arrays
// would not fit in three quarters of free device memory.
static uint32_t batch_lines_for(const ipg_graph* g, const BatchWorkspace* b, uint64_t sending) {
    uint32_t want = (uint32_t)((sending + kLanes - 1) / kLanes);
    want = want < 1 ? 1 : want > (uint32_t)kMaxLines ? (uint32_t)kMaxLines : want;
    if (b->lines >= want) return want;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return b->lines ? b->lines : 1;
    const size_t held = b->lines ? batch_value_bytes(g->n, b->lines) : 0;  // freed before the new arrays
    while (want > 1 && batch_value_bytes(g->n, want) > (fr + held) / 4 * 3) --want;
    return want > b->lines ? want : (b->lines ? b->lines : 1);
}

// The in-edge chunks of a pull form (the batched engine's tile sizes, tuning knobs:
// the one-line and the wide pull measure best at different sizes): their first rows
// are recomputed, and the loop graphs that use them, which bake in the chunk count,
// rebuilt, when the size changes.
static ipg_status batch_chunks(ipg_graph* g, BatchWorkspace* b, uint32_t lines, cudaStream_t st) {
    const int wide = lines > 1 ? 1 : 0;
    auto& c = b->cs[wide];
    uint32_t want = (uint32_t)(wide ? tuning().batch_wide_chunk : batch_chunk_for(g));
    // The pull's warps take every (warps)-th chunk.  With fewer than 3 chunks a warp, the
    // warps holding one chunk more set the superstep's time, and with fewer chunks than
    // warps the launch is short of warps; so the knob's tile is halved, while it stays a
    // multiple of 32 and not below a floor (128 in-edges for the wide pull, 64 for one
    // line), until each warp has batch_tile_tasks chunks (3; 0 keeps the knob's tile).
    // A tile the autotuner picked for this graph is kept as it is.
    if (wide || !g->tuned.batch) {
        const uint64_t cap = grid_for_warps(uint64_t(1) << 40, sm_count_of(g->device));
        const uint64_t warps = wide ? 2 * cap * kRingWarps : cap * 8;
        const uint64_t tasks = (uint64_t)tuning().batch_tile_tasks;
        const uint32_t least = wide ? 128u : 64u;
        while (want % 64 == 0 && want / 2 >= least && (g->m + want - 1) / want < tasks * warps) want >>= 1;
    }
    if (c.size == want) return IPG_OK;
    for (auto& per_kind : b->loop)
        for (int l = 0; l < kMaxLines; ++l)
            if (per_kind[l] && ((l > 0) == (wide == 1))) {
                cudaGraphExecDestroy(per_kind[l]);
                per_kind[l] = nullptr;
            }
    const uint64_t chunks = (g->m + want - 1) / want;
    if (chunks > c.cap) {
        cudaFree(c.row);
        c.row = nullptr;
        c.cap = 0;
        IPG_CUDA(cudaMalloc(&c.row, sizeof(uint32_t) * (chunks ? chunks : 1)));
        c.cap = chunks;
    }
    if (chunks) {
        chunk_rows_kernel<<<grid_for_warps(chunks / 32 + 1, sm_count_of(g->device)), 256, 0, st>>>(
            g->csc_off, g->n, g->m, chunks, want, c.row);
        IPG_CUDA(cudaGetLastError());
    }
    c.count = chunks;
    c.size = want;
    return IPG_OK;
}

// the wide pull for rows of L lines (2 <= L <= 8)
template <int K, int L>
static void ring_launch_l(ipg_graph* g, BatchWorkspace* b, unsigned grid, cudaStream_t st) {
    const auto& c = b->cs[1];
    batch_pull_ring_kernel<K, L><<<grid, kRingWarps * 32, ring_smem_bytes(L), st>>>(
        g->csc_off, g->csc_src, g->csc_w8, g->csc_w, c.row, c.count, g->n, g->m, b->sval, b->sany, b->dist, b->cmask,
        b->cany, b->fr[0], b->fr[1], b->ctl, b->ctr, c.size);
}

template <int K>
static void batch_ring_launch(ipg_graph* g, BatchWorkspace* b, uint32_t L, unsigned grid, cudaStream_t st) {
    switch (L) {
        case 2: ring_launch_l<K, 2>(g, b, grid, st); break;
        case 3: ring_launch_l<K, 3>(g, b, grid, st); break;
        case 4: ring_launch_l<K, 4>(g, b, grid, st); break;
        case 5: ring_launch_l<K, 5>(g, b, grid, st); break;
        case 6: ring_launch_l<K, 6>(g, b, grid, st); break;
        case 7: ring_launch_l<K, 7>(g, b, grid, st); break;
        default: ring_launch_l<K, 8>(g, b, grid, st); break;
    }
}

// the superstep body for V lines, enqueued on `st` (captured into the loop graph,
// or launched directly when in_graph is 0)
template <int V>
static void batch_superstep_lines(ipg_graph* g, BatchWorkspace* b, int wkind, uint32_t L,
                                  cudaGraphConditionalHandle loop, int in_graph, cudaStream_t st) {
    const int sms = sm_count_of(g->device);
    const auto& cs = b->cs[L > 1 ? 1 : 0];
    const unsigned grid = grid_for_warps(cs.count, sms);
    const unsigned fixed = (unsigned)sms * 8;  // frontier passes: persistent, the size is read on the device
#define IPG_BATCH_PULL(K)                                                                                           \
    if constexpr (V == 1)                                                                                           \
        batch_pull_kernel<K><<<grid, 256, 0, st>>>(g->csc_off, g->csc_src, g->csc_w8, g->csc_w, cs.row, cs.count,  \
                                                   g->n, g->m, b->sval, b->smask, b->dist, b->cmask, b->fr[0],      \
                                                   b->fr[1], b->ctl, b->ctr, cs.size);                              \
    else                                                                                                            \
        batch_ring_launch<K>(g, b, L, 2 * grid, st)
#define IPG_BATCH_PUSH(K)                                                                                           \
    batch_push_kernel<K, V><<<fixed, 256, 0, st>>>(g->off, g->col, g->w8, g->w, b->tasks, L, b->sval, b->smask,   \
                                                   b->sany, b->dist, b->cmask, b->cany, b->fr[0], b->fr[1], b->ctl, \
                                                   b->ctr)
    batch_refill_kernel<V><<<1, V * kLanes, 0, st>>>(b->ctl, g->inv, g->off, b->wmax_out, g->m, L, b->dist,
                                                     b->sval, b->smask, b->sany, b->fr[0], b->fr[1]);
    batch_tasks_kernel<<<fixed, 256, 0, st>>>(b->fr[0], b->fr[1], b->ctl, g->off, b->tasks, b->ctr);
    if (wkind == 1) {
        IPG_BATCH_PULL(1);
        IPG_BATCH_PUSH(1);
    } else if (wkind == 2) {
        IPG_BATCH_PULL(2);
        IPG_BATCH_PUSH(2);
    } else {
        IPG_BATCH_PULL(0);
        IPG_BATCH_PUSH(0);
    }
#undef IPG_BATCH_PULL
#undef IPG_BATCH_PUSH
    batch_reset_kernel<V><<<fixed, 256, 0, st>>>(b->fr[0], b->fr[1], b->ctl, L, b->sval, b->smask, b->sany);
    batch_apply_kernel<V><<<fixed, 256, 0, st>>>(b->fr[0], b->fr[1], b->ctl, g->n, L, g->off, b->wmax_out,
                                                 b->dist, b->sval, b->smask, b->sany, b->cmask, b->cany, b->ctr);
    batch_step_kernel<V><<<1, V * kLanes, 0, st>>>(b->ctl, b->ctr, g->n, loop, in_graph);
    batch_harvest_kernel<V><<<fixed, 256, 0, st>>>(b->ctl, g->inv, g->n, L, b->dist);
}

static void batch_superstep(ipg_graph* g, BatchWorkspace* b, int wkind, uint32_t lines,
                            cudaGraphConditionalHandle loop, int in_graph, cudaStream_t st) {
    switch (lines_v(lines)) {
        case 8: batch_superstep_lines<8>(g, b, wkind, lines, loop, in_graph, st); break;
        case 4: batch_superstep_lines<4>(g, b, wkind, lines, loop, in_graph, st); break;
        case 2: batch_superstep_lines<2>(g, b, wkind, lines, loop, in_graph, st); break;
        default: batch_superstep_lines<1>(g, b, wkind, lines, loop, in_graph, st); break;
    }
}

// the wide pull's dynamic shared memory for rows of L lines (above the default 48 KB
// limit from 6 lines on); set before the kernel is launched or captured
template <int L>
static cudaError_t ring_smem_allow_l() {
    const int bytes = (int)ring_smem_bytes(L);
    cudaError_t e = cudaFuncSetAttribute(batch_pull_ring_kernel<0, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_pull_ring_kernel<1, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_pull_ring_kernel<2, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

static ipg_status batch_ring_allow(uint32_t lines) {
    cudaError_t e = cudaSuccess;
    switch (lines) {
        case 1: break;
        case 2: e = ring_smem_allow_l<2>(); break;
        case 3: e = ring_smem_allow_l<3>(); break;
        case 4: e = ring_smem_allow_l<4>(); break;
        case 5: e = ring_smem_allow_l<5>(); break;
        case 6: e = ring_smem_allow_l<6>(); break;
        case 7: e = ring_smem_allow_l<7>(); break;
        default: e = ring_smem_allow_l<8>(); break;
    }
    return e == cudaSuccess ? IPG_OK : cuda_fail(e, "batched pull shared memory", __FILE__, __LINE__);
}

// Builds the graph [WHILE (cond) { superstep }] for this workspace, weight kind and line count.
static ipg_status batch_loop_graph(ipg_graph* g, BatchWorkspace* b, int wkind, uint32_t lines) {
    cudaGraphExec_t& exec = b->loop[wkind][lines - 1];
    if (exec) return IPG_OK;
    IPG_TRY(batch_ring_allow(lines));
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
            rc = cuda_fail(e, "batch loop graph", __FILE__, __LINE__);
            break;
        }
        batch_superstep(g, b, wkind, lines, handle, 1, cap);
        cudaGraph_t body = nullptr;
        e = cudaStreamEndCapture(cap, &body);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) rc = cuda_fail(e, "batch loop graph capture", __FILE__, __LINE__);
    } while (false);
    if (cap) cudaStreamDestroy(cap);
    if (graph) cudaGraphDestroy(graph);
    return rc;
}

static int weight_kind(const ipg_graph* g) { return g->csc_w8 ? 1 : g->csc_w ? 2 : 0; }

// Every lane free, values kInf, masks and counters zero (skipped when the last
// session left them so), and the control block set for a new session.
static ipg_status batch_session_begin(ipg_graph* g, BatchWorkspace* b, const BatchCtl& init, cudaStream_t st) {
    const size_t n = g->n;
    IPG_TRY(batch_values(g, b, init.lines));
    IPG_TRY(batch_chunks(g, b, init.lines, st));
    if (b->clean && b->dist_dirty) {
        // only the rows the last session used: its lines
        IPG_CUDA(cudaMemsetAsync(b->dist, 0xFF, sizeof(uint32_t) * kLanes * b->dirty_lines * n, st));
    } else if (!b->clean) {
        const size_t lines = b->lines;
        IPG_CUDA(cudaMemsetAsync(b->dist, 0xFF, sizeof(uint32_t) * kLanes * lines * n, st));
        IPG_CUDA(cudaMemsetAsync(b->sval, 0xFF, sizeof(uint32_t) * kLanes * lines * n, st));
        IPG_CUDA(cudaMemsetAsync(b->smask, 0, sizeof(uint32_t) * lines * n, st));
        IPG_CUDA(cudaMemsetAsync(b->cmask, 0, sizeof(uint32_t) * lines * n, st));
        IPG_CUDA(cudaMemsetAsync(b->sany, 0, sizeof(uint32_t) * n, st));
        IPG_CUDA(cudaMemsetAsync(b->cany, 0, sizeof(uint32_t) * n, st));
        IPG_CUDA(cudaMemsetAsync(b->ctr, 0, sizeof(BatchCounters), st));
    }
    b->clean = false;
    b->dist_dirty = false;
    *b->h_ctl = init;
    IPG_CUDA(cudaMemcpyAsync(b->ctl, b->h_ctl, sizeof(BatchCtl), cudaMemcpyHostToDevice, st));
    return IPG_OK;
}

static BatchCtl batch_ctl_init(const ipg_graph* g, uint32_t lines) {
    BatchCtl c;
    memset(&c, 0, sizeof(c));
    c.divisor = (unsigned long long)batch_divisor_for(g);
    c.lines = lines;
    return c;
}

// one graph launch (or, with the batch_loop knob at 0, the same supersteps launched
// one by one from the host), then the control block back on the host
static ipg_status batch_launch(ipg_graph* g, BatchWorkspace* b, cudaStream_t st, const char* name) {
    if (tuning().batch_loop) {
        IPG_TRY(batch_loop_graph(g, b, weight_kind(g), b->h_ctl->lines));
        IPG_CUDA(cudaGraphLaunch(b->loop[weight_kind(g)][b->h_ctl->lines - 1], st));
        IPG_CUDA(cudaMemcpyAsync(b->h_ctl, b->ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, st));
        IPG_CUDA(cudaStreamSynchronize(st));
    } else {
        // the step kernel leaves iter at 0 where the graph's WHILE condition would end
        IPG_TRY(batch_ring_allow(b->h_ctl->lines));
        for (;;) {
            batch_superstep(g, b, weight_kind(g), b->h_ctl->lines, cudaGraphConditionalHandle{}, 0, st);
            IPG_CUDA(cudaGetLastError());
            IPG_CUDA(cudaMemcpyAsync(b->h_ctl, b->ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, st));
            IPG_CUDA(cudaStreamSynchronize(st));
            if (b->h_ctl->iter == 0) break;
        }
    }
    if (b->h_ctl->status & kStatusOverflow) return set_error(IPG_EOVERFLOW, "%s: a path length reached UINT32_MAX", name);
    if (b->h_ctl->status & kStatusInternal) return set_error(IPG_EDEVICE, "%s: frontier overflow", name);
    return IPG_OK;
}

ipg_status sssp_batch_run(ipg_graph* g, const uint32_t* sources, uint32_t k, uint32_t* dist_dev,
                          uint32_t* supersteps_out, cudaStream_t st) {
    if (!g) return set_error(IPG_EINVAL, "ipg_sssp_batch: graph is NULL");
    if (k == 0) return IPG_OK;
    if (!sources || !dist_dev) return set_error(IPG_EINVAL, "ipg_sssp_batch: NULL argument");
    for (uint32_t i = 0; i < k; ++i)
        if (sources[i] >= g->n)
            return set_error(IPG_EINVAL, "ipg_sssp_batch: source %u (index %u) >= n = %u", sources[i], i, g->n);
    DeviceGuard guard(g->device);
    if (!guard.ok) return set_error(IPG_ECUDA, "ipg_sssp_batch: cannot select the graph's device");
    IPG_TRY(batch_prepare(g, st));
    BatchWorkspace* b = (BatchWorkspace*)g->batch;
    if (b->list_cap < k) {
        cudaFree(b->list);
        cudaFree(b->steps);
        cudaFree(b->sends);
        b->list = b->steps = nullptr;
        b->sends = nullptr;
        b->list_cap = 0;
        IPG_CUDA(cudaMalloc(&b->list, sizeof(uint32_t) * 2 * (size_t)k));
        IPG_CUDA(cudaMalloc(&b->steps, sizeof(uint32_t) * k));
        IPG_CUDA(cudaMalloc(&b->sends, k));
        b->list_cap = k;
    }
    // Queries whose source has no out-edges end after superstep 0: their rows are
    // written directly.  The others take lanes, and start together in the fewest
    // lines that hold them.
    IPG_CUDA(cudaMemcpyAsync(b->list, sources, sizeof(uint32_t) * k, cudaMemcpyHostToDevice, st));
    batch_triage_kernel<<<(k + 255) / 256 < 1024 ? (k + 255) / 256 : 1024, 256, 0, st>>>(b->list, k, g->inv, g->off,
                                                                                      b->sends);
    IPG_CUDA(cudaGetLastError());
    std::vector<uint8_t> sends(k);
    IPG_CUDA(cudaMemcpyAsync(sends.data(), b->sends, k, cudaMemcpyDeviceToHost, st));
    IPG_CUDA(cudaStreamSynchronize(st));
    // sources then output rows: the sending queries first, the others after them
    std::vector<uint32_t> order(2 * (size_t)k);
    uint32_t sending = 0;
    for (uint32_t i = 0; i < k; ++i) sending += sends[i];
    for (uint32_t i = 0, a = 0, z = sending; i < k; ++i) {
        const uint32_t at = sends[i] ? a++ : z++;
        order[at] = sources[i];
        order[(size_t)k + at] = i;
    }
    IPG_CUDA(cudaMemcpyAsync(b->list, order.data(), sizeof(uint32_t) * 2 * (size_t)k, cudaMemcpyHostToDevice, st));
    const uint32_t silent = k - sending;
    if (silent && g->n) {
        const uint64_t total = (uint64_t)silent * g->n;
        const uint64_t cap = (uint64_t)sm_count_of(g->device) * 8;
        const unsigned grid = (unsigned)((total + 255) / 256 < cap ? (total + 255) / 256 : cap);
        batch_fill_kernel<<<grid, 256, 0, st>>>(dist_dev, g->n, g->n, b->list + sending, b->list + k + sending, silent,
                                                b->steps);
        IPG_CUDA(cudaGetLastError());
    }
    b->info = ipg_batch_info{};
    b->info.queries = k;
    if (sending == 0) {
        if (supersteps_out) {
            IPG_CUDA(cudaMemcpyAsync(supersteps_out, b->steps, sizeof(uint32_t) * k, cudaMemcpyDeviceToHost, st));
        }
        IPG_CUDA(cudaStreamSynchronize(st));
        return IPG_OK;
    }
    const uint32_t lines = batch_lines_for(g, b, sending);
    BatchCtl init = batch_ctl_init(g, lines);
    init.nqueries = sending;
    init.src_list = b->list;
    init.row_list = b->list + k;
    init.steps_out = b->steps;
    init.out = dist_dev;
    init.out_stride = g->n;
    IPG_TRY(batch_session_begin(g, b, init, st));
    // every lane is refilled on the device: one launch per kLoopCap supersteps
    const uint64_t bound = ((uint64_t)k + kMaxSlots) * ((uint64_t)g->n + 2) / kLoopCap + 2;
    uint64_t launches = 0;
    for (;; ++launches) {
        if (launches > bound)
            return set_error(IPG_EDEVICE, "ipg_sssp_batch: the superstep loop did not end");
        IPG_TRY(batch_launch(g, b, st, "ipg_sssp_batch"));
        if (b->h_ctl->done) break;
    }
    b->clean = true;  // every lane was harvested; the last harvest left dist in place
    b->dist_dirty = true;
    b->dirty_lines = lines;
    b->info.supersteps = b->h_ctl->supersteps;
    b->info.pull_supersteps = b->h_ctl->pull_supersteps;
    b->info.harvests = b->h_ctl->harvests;
    b->info.launches = launches + 1;
    b->info.lanes = (uint64_t)lines * kLanes;
    if (supersteps_out) {
        IPG_CUDA(cudaMemcpyAsync(supersteps_out, b->steps, sizeof(uint32_t) * k, cudaMemcpyDeviceToHost, st));
        IPG_CUDA(cudaStreamSynchronize(st));
    }
    return IPG_OK;
}

// ---- lane sessions driven by the host (the server): one line of 32 lanes ------

ipg_status lanes_open(ipg_graph* g, uint32_t* stage_dev, cudaStream_t st) {
    DeviceGuard guard(g->device);
    IPG_TRY(batch_prepare(g, st));
    BatchWorkspace* b = (BatchWorkspace*)g->batch;
    *b->h_admit = 0;
    BatchCtl init = batch_ctl_init(g, 1);
    init.stop_on_finish = 1;
    init.admit = b->d_admit;
    init.out = stage_dev;
    init.out_stride = g->n;
    return batch_session_begin(g, b, init, st);
}

volatile unsigned int* lanes_admit_flag(ipg_graph* g) {
    BatchWorkspace* b = (BatchWorkspace*)g->batch;
    return b ? b->h_admit : nullptr;
}

ipg_status lanes_step(ipg_graph* g, const uint32_t* sources, const uint32_t* rows, uint32_t nseed,
                      cudaStream_t st, LaneReport* rep) {
    DeviceGuard guard(g->device);
    BatchWorkspace* b = (BatchWorkspace*)g->batch;
    if (!b) return set_error(IPG_EINVAL, "lanes_step: no open session");
    BatchCtl* h = b->h_ctl;  // mirrors the device block after the previous launch
    if (nseed > (uint32_t)__builtin_popcount(~h->live[0])) return set_error(IPG_EINVAL, "lanes_step: too many seeds");
    if (nseed) {
        h->nseed = nseed;
        for (uint32_t i = 0; i < nseed; ++i) {
            if (sources[i] >= g->n) return set_error(IPG_EINVAL, "lanes_step: source %u >= n", sources[i]);
            h->seed_src[i] = sources[i];
            h->seed_row[i] = rows[i];
        }
        const size_t beg = offsetof(BatchCtl, nseed), end = offsetof(BatchCtl, out);
        IPG_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(b->ctl) + beg, reinterpret_cast<char*>(h) + beg, end - beg,
                                 cudaMemcpyHostToDevice, st));
    }
    if (!nseed && h->live[0] == 0) {
        rep->live = 0;
        rep->finished = 0;
        return IPG_OK;
    }
    *b->h_admit = 0;
    IPG_TRY(batch_launch(g, b, st, "lanes_step"));
    rep->live = h->live[0];
    rep->finished = h->finished[0];
    for (int l = 0; l < kLanes; ++l) {
        rep->row[l] = h->row[l];
        rep->count[l] = h->count[l];
    }
    return IPG_OK;
}

void lanes_close(ipg_graph* g) {
    BatchWorkspace* b = (BatchWorkspace*)g->batch;
    if (b && b->h_ctl->live[0] == 0 && b->h_ctl->status == 0) b->clean = true;
}

}  // namespace ipg

using namespace ipg;

extern "C" {

ipg_status ipg_sssp_batch_info(const ipg_graph* g, ipg_batch_info* out) {
    if (!g || !out) return set_error(IPG_EINVAL, "ipg_sssp_batch_info: NULL argument");
    const BatchWorkspace* b = (const BatchWorkspace*)g->batch;
    *out = b ? b->info : ipg_batch_info{};
    return IPG_OK;
}

ipg_status ipg_sssp_batch_dev(ipg_graph* g, const uint32_t* sources, uint32_t k, uint32_t* dist_dev,
                              uint32_t* supersteps_out, void* stream) {
    return sssp_batch_run(g, sources, k, dist_dev, supersteps_out, (cudaStream_t)stream);
}

// host output: groups of up to kMaxSlots sources through a device staging buffer
// of group * n words (smaller groups when that would not fit in a quarter of
// free device memory)
ipg_status ipg_sssp_batch(ipg_graph* g, const uint32_t* sources, uint32_t k, uint32_t* dist_out,
                          uint32_t* supersteps_out) {
    if (!g) return set_error(IPG_EINVAL, "ipg_sssp_batch: graph is NULL");
    if (k && (!sources || !dist_out)) return set_error(IPG_EINVAL, "ipg_sssp_batch: NULL argument");
    DeviceGuard guard(g->device);
    const uint64_t n = g->n;
    uint32_t group = k < (uint32_t)kMaxSlots ? k : (uint32_t)kMaxSlots;
    if (k) {
        size_t fr = 0, tot = 0;
        IPG_CUDA(cudaMemGetInfo(&fr, &tot));
        while (group > (uint32_t)kLanes && sizeof(uint32_t) * group * (n ? n : 1) > fr / 4) group /= 2;
    }
    uint32_t* stage = nullptr;
    if (k) IPG_CUDA(cudaMalloc(&stage, sizeof(uint32_t) * group * (n ? n : 1)));
    ipg_status rc = IPG_OK;
    for (uint32_t i0 = 0; i0 < k && rc == IPG_OK; i0 += group) {
        const uint32_t kk = k - i0 < group ? k - i0 : group;
        rc = sssp_batch_run(g, sources + i0, kk, stage, supersteps_out ? supersteps_out + i0 : nullptr, g->stream);
        if (rc == IPG_OK && n) {
            cudaError_t e = cudaMemcpyAsync(dist_out + (uint64_t)i0 * n, stage, sizeof(uint32_t) * kk * n,
                                            cudaMemcpyDeviceToHost, g->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
            if (e != cudaSuccess) rc = cuda_fail(e, "copy of batched distances", __FILE__, __LINE__);
        }
    }
    if (stage) cudaFree(stage);
    return rc;
}

}  // extern "C"
