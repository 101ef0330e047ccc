// Batched SSSP: many sources on one graph, each an independent synchronous
// Pregel SSSP (Sec. VI-C), run together superstep by superstep.
//
// The engine has 32 lanes, one per warp lane; each lane holds one query (a
// source) or is free.  Values live vertex-major, dist[v][lane], so the 32
// lanes' values of a vertex are one 128-byte line: in a pull superstep every
// in-edge (u -> v) costs one read of u's sender values for the lanes that send
// from u (only their sectors of the line), where 32 separate runs would each pay
// a random 4-byte gather.  A superstep:
//   refill   free lanes take the next queries (from a device list of sources, or
//            from seeds the host wrote at a superstep boundary): the source's
//            value becomes 0 and it joins the current senders;
//   pull     warps walk contiguous chunks of the in-edge lists (CSC).  Lane b keeps
//            a running min of sval[u][b] + w over the current destination's edges
//            and flushes it with atomicMin into dist[v][b] when the destination
//            changes (a row split across chunks is finished by the atomics).  A
//            lane whose atomicMin lowered the value marks v in cmask[v]; the first
//            marker appends v to the next frontier (union over the lanes);
//   apply    the previous senders' snapshot rows are reset to kInf, and every
//            vertex of the next frontier publishes dist[v][b] for the lanes
//            whose value dropped (kInf for the others), which is the snapshot the
//            next superstep reads; per-lane message counts (sum of the senders'
//            out-degrees) come out of the same pass;
//   step     a lane whose next senders send nothing has finished its query: its
//            superstep count is final and the lane is marked for harvest;
//   harvest  finished lanes' distances go to their output rows (in caller ids)
//            and their columns are reset to kInf, which frees the lanes for the
//            next refill.
// Senders send the value they had at the start of the superstep, as in the
// synchronous model; lanes never share values, so a query's distances and
// superstep count equal those of a standalone ipg_sssp run whichever superstep
// it joined at.
//
// A sparse superstep runs in push form instead: a task pass cuts the senders'
// out-edge lists into tasks of kPushChunk edges, and a warp per task sends
// sval[u][b] + w along each out-edge (u -> v) with atomicMin into dist[v][b].
// Push and pull take the minimum of the same messages and mark the same
// lowered lanes, so they are interchangeable; the refill kernel picks push when
// the senders' out-edges are fewer than m / divisor.
//
// The superstep loop runs on the device: a CUDA graph holds a conditional WHILE
// node whose body is one superstep (refill, tasks, pull, push, reset, apply,
// step, harvest).  The kernels read the frontier and the lanes from a device
// control block, so their launch parameters never change, and the step kernel
// decides whether another superstep follows.  ipg_sssp_batch keeps all 32 lanes
// busy from its source list inside the loop, so k sources run in one graph launch
// (plus one per kLoopCap supersteps).  The server seeds lanes itself: its launches
// end at the first superstep where a lane finished, or when queries wait for a
// free lane (a flag in mapped host memory), so queries join a running batch at
// the next superstep boundary.
#include "ipg_internal.cuh"

namespace ipg {
namespace {

constexpr int kLanes = 32;
constexpr int kUnroll = 4;  // sender lines in flight per warp (8 and 16 measured slower)

constexpr unsigned kLoopCap = 1024;    // supersteps per graph launch
constexpr uint32_t kPushChunk = 256;   // out-edges per push task

struct BatchCounters {
    unsigned long long msgs[kLanes];  // messages the next superstep's senders send, per lane
    unsigned long long edges;         // out-edges of the next senders (union over lanes)
    unsigned int next_size;
    unsigned int status;
    unsigned int ntasks;              // push tasks of the current senders (push supersteps)
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
    unsigned long long f_edges;  // out-edges of the current senders (union over lanes)
    unsigned int live;           // lanes holding a query
    unsigned int finished;       // lanes whose query ended in the last superstep
    unsigned int count[kLanes];  // supersteps of each lane's query so far (final once finished)
    unsigned int row[kLanes];    // output row of each lane's query
    // refill from a device list (ipg_sssp_batch): caller ids, nqueries entries
    unsigned int next_query, nqueries;
    const uint32_t* src_list;
    uint32_t* steps_out;  // per query: its superstep count (device), or NULL
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

__device__ __forceinline__ bool batch_push_pick(unsigned long long edges, unsigned long long divisor, uint64_t m) {
    return divisor > 0 && (double)edges * (double)divisor < (double)m;
}

// Free lanes take the next queries, in lane order: from the device source list,
// or from the host's seeds.  The source's value becomes 0 and it joins the
// current senders; its count starts at 1 (superstep 0), 2 if it has out-edges
// (its messages make a superstep 1).  Then the superstep's form is picked.
__global__ void batch_refill_kernel(BatchCtl* __restrict__ ctl, const uint32_t* __restrict__ inv,
                                    const uint64_t* __restrict__ off, uint64_t m, uint32_t* __restrict__ dist,
                                    uint32_t* __restrict__ sval, uint32_t* __restrict__ smask, uint32_t* fr0,
                                    uint32_t* fr1) {
    const uint32_t b = threadIdx.x;
    const uint32_t live = ctl->live;
    const bool is_free = !((live >> b) & 1u);
    const unsigned freem = __ballot_sync(0xFFFFFFFFu, is_free);
    const uint32_t rank = __popc(freem & ((1u << b) - 1u));
    const bool from_list = ctl->nqueries != 0;
    bool take = false;
    uint32_t src = 0, row = 0;
    if (from_list) {
        const uint32_t q = ctl->next_query + rank;
        take = is_free && q < ctl->nqueries;
        if (take) {
            src = ctl->src_list[q];
            row = q;
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
        dist[(uint64_t)v * kLanes + b] = 0;
        sval[(uint64_t)v * kLanes + b] = 0;
        const uint64_t deg = off[v + 1] - off[v];
        if (atomicOr(&smask[v], 1u << b) == 0) {
            fr_cur(fr0, fr1, ctl)[atomicAdd(&ctl->f, 1u)] = v;
            add = deg;
        }
        ctl->count[b] = 1u + (deg > 0 ? 1u : 0u);
        ctl->row[b] = row;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) add += __shfl_down_sync(0xFFFFFFFFu, add, o);
    if (b == 0) {
        ctl->live = live | takem;
        if (from_list)
            ctl->next_query += __popc(takem);
        else
            ctl->nseed = 0;
        ctl->f_edges += add;
        ctl->push = batch_push_pick(ctl->f_edges, ctl->divisor, m);
    }
}

__device__ __forceinline__ void batch_flush(uint32_t v, uint32_t run, uint32_t lane, uint32_t* __restrict__ dist,
                                            uint32_t* __restrict__ cmask, uint32_t* __restrict__ next,
                                            BatchCounters* __restrict__ ctr) {
    bool changed = false;
    if (run != kInf) {
        const uint32_t old = atomicMin(&dist[(uint64_t)v * kLanes + lane], run);
        changed = run < old;
    }
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, changed);
    if (mask && lane == 0) {
        const unsigned old = atomicOr(&cmask[v], mask);
        if (old == 0) next[atomicAdd(&ctr->next_size, 1u)] = v;
    }
}

// end of a row relative to the start of a chunk, clamped to 32 bits: a chunk holds at
// most `chunk` edges, so every value from there up means "ends after this chunk"
__device__ __forceinline__ uint32_t chunk_rel_end(uint64_t row_end, uint64_t e_begin) {
    const uint64_t r = row_end - e_begin;
    return r < 0xFFFFFFFFull ? (uint32_t)r : 0xFFFFFFFFu;
}

template <int kWeightKind>
__global__ void __launch_bounds__(256) batch_pull_kernel(
    const uint64_t* __restrict__ csc_off, const uint32_t* __restrict__ csc_src, const uint8_t* __restrict__ w8,
    const uint32_t* __restrict__ w32, const uint32_t* __restrict__ chunk_row, uint64_t chunks, uint32_t n, uint64_t m,
    const uint32_t* __restrict__ sval, const uint32_t* __restrict__ smask, uint32_t* __restrict__ dist,
    uint32_t* __restrict__ cmask, uint32_t* fr0, uint32_t* fr1, const BatchCtl* __restrict__ ctl,
    BatchCounters* __restrict__ ctr, uint32_t chunk) {
    if (ctl->push) return;
    uint32_t* __restrict__ next = fr_next(fr0, fr1, ctl);
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t c = warp; c < chunks; c += nwarps) {
        const uint64_t e_begin = c * chunk;
        const uint32_t len = (uint32_t)(e_begin + chunk < m ? chunk : m - e_begin);
        uint32_t row = chunk_row[c];
        uint32_t bound = chunk_rel_end(csc_off[row + 1], e_begin);  // row end, relative to the chunk (may exceed len)
        uint32_t run = kInf;
        bool pending = false;  // some lane folded a message into run (warp-uniform)
        for (uint32_t j0 = 0; j0 < len; j0 += 32) {
            const uint32_t jl = j0 + lane;
            uint32_t u_l = 0, w_l = 1, sm_l = 0;
            if (jl < len) {
                u_l = __ldcs(csc_src + e_begin + jl);
                sm_l = __ldg(smask + u_l);
                if (kWeightKind == 1) w_l = __ldcs(w8 + e_begin + jl);
                if (kWeightKind == 2) w_l = __ldcs(w32 + e_begin + jl);
            }
            // only in-edges whose source sends for some lane of the group
            unsigned active = __ballot_sync(0xFFFFFFFFu, sm_l != 0);
            if (!active) continue;
            const uint32_t jmax = j0 + 31 - __clz(active);  // last active edge of the group
            if (jmax < bound) {
                // fast path: every active edge of the group belongs to the current row
                while (active) {
                    uint32_t s[kUnroll], lim[kUnroll];
#pragma unroll
                    for (int q = 0; q < kUnroll; ++q) {
                        const int jj = active ? __ffs(active) - 1 : 0;
                        const bool ok = active != 0;
                        if (active) active &= active - 1;
                        const uint32_t u = __shfl_sync(0xFFFFFFFFu, u_l, jj);
                        const uint32_t w = __shfl_sync(0xFFFFFFFFu, w_l, jj);
                        const uint32_t sm = __shfl_sync(0xFFFFFFFFu, sm_l, jj);
                        lim[q] = kInf - w;  // s + w stays below kInf iff s < lim
                        // only lanes whose source sends from u load: the line's other sectors stay untouched
                        s[q] = ok && ((sm >> lane) & 1u) ? __ldg(sval + ((uint64_t)u * kLanes + lane)) : kInf;
                    }
#pragma unroll
                    for (int q = 0; q < kUnroll; ++q) {
                        if (s[q] < lim[q]) {
                            run = min(run, s[q] + (kInf - lim[q]));
                        } else if (s[q] != kInf) {
                            atomicOr(&ctr->status, kStatusOverflow);
                            run = min(run, kInf - 1);
                        }
                    }
                }
                pending = true;
                continue;
            }
            while (active) {
                int jj[kUnroll];
                uint32_t s[kUnroll], lim[kUnroll];
#pragma unroll
                for (int q = 0; q < kUnroll; ++q) {
                    jj[q] = active ? __ffs(active) - 1 : -1;
                    if (active) active &= active - 1;
                    const int src_lane = jj[q] < 0 ? 0 : jj[q];
                    const uint32_t u = __shfl_sync(0xFFFFFFFFu, u_l, src_lane);
                    const uint32_t w = __shfl_sync(0xFFFFFFFFu, w_l, src_lane);
                    const uint32_t sm = __shfl_sync(0xFFFFFFFFu, sm_l, src_lane);
                    lim[q] = kInf - w;
                    s[q] = jj[q] >= 0 && ((sm >> lane) & 1u) ? __ldg(sval + ((uint64_t)u * kLanes + lane)) : kInf;
                }
#pragma unroll
                for (int q = 0; q < kUnroll; ++q) {
                    if (jj[q] >= 0) {
                        const uint32_t e = j0 + (uint32_t)jj[q];
                        if (e >= bound) {  // the destination changed (warp-uniform)
                            if (pending) batch_flush(row, run, lane, dist, cmask, next, ctr);
                            run = kInf;
                            pending = false;
                            do {
                                ++row;
                                bound = chunk_rel_end(csc_off[row + 1], e_begin);
                            } while (e >= bound);
                        }
                        if (s[q] < lim[q]) {
                            run = min(run, s[q] + (kInf - lim[q]));
                        } else if (s[q] != kInf) {
                            atomicOr(&ctr->status, kStatusOverflow);
                            run = min(run, kInf - 1);
                        }
                        pending = true;
                    }
                }
            }
        }
        if (pending) batch_flush(row, run, lane, dist, cmask, next, ctr);
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
// When few sources send from u (kSparseLanes or fewer), lanes take different
// edges and loop over those sources, one atomicMin per (edge, source); else
// lane b sends sval[u][b] + w along each edge, one coalesced row per edge.
constexpr int kSparseLanes = 4;

template <int kWeightKind>
__global__ void __launch_bounds__(256) batch_push_kernel(
    const uint64_t* __restrict__ off, const uint32_t* __restrict__ col, const uint8_t* __restrict__ w8,
    const uint32_t* __restrict__ w32, const unsigned long long* __restrict__ tasks,
    const uint32_t* __restrict__ sval, const uint32_t* __restrict__ smask, uint32_t* __restrict__ dist,
    uint32_t* __restrict__ cmask, uint32_t* fr0, uint32_t* fr1, const BatchCtl* __restrict__ ctl,
    BatchCounters* __restrict__ ctr) {
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
        const uint32_t senders = smask[u];  // sources that send from u (warp-uniform)
        if (__popc(senders) <= kSparseLanes) {
            // lane per edge (no warp-collective step); the sending sources one after another
            for (uint64_t j = e_beg + lane; j < e_end; j += 32) {
                const uint32_t v = __ldg(col + j);
                uint32_t w = 1;
                if (kWeightKind == 1) w = __ldg(w8 + j);
                if (kWeightKind == 2) w = __ldg(w32 + j);
                for (uint32_t rest = senders; rest; rest &= rest - 1) {
                    const uint32_t b = __ffs(rest) - 1;
                    const uint32_t s = __ldg(sval + (uint64_t)u * kLanes + b);
                    if (s != kInf) {
                        const uint32_t d = batch_cand(s, w, ctr);
                        if (d < atomicMin(&dist[(uint64_t)v * kLanes + b], d)) {
                            if (atomicOr(&cmask[v], 1u << b) == 0) next[atomicAdd(&ctr->next_size, 1u)] = v;
                        }
                    }
                }
            }
            continue;
        }
        // kInf: lane b does not send from u (its sector is not loaded)
        const uint32_t s = (senders >> lane) & 1u ? sval[(uint64_t)u * kLanes + lane] : kInf;
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
                bool changed = false;
                if (s != kInf) {
                    const uint32_t d = batch_cand(s, w, ctr);
                    changed = d < atomicMin(&dist[(uint64_t)v * kLanes + lane], d);
                }
                const unsigned mask = __ballot_sync(0xFFFFFFFFu, changed);
                if (mask && lane == 0) {
                    const unsigned prev = atomicOr(&cmask[v], mask);
                    if (prev == 0) next[atomicAdd(&ctr->next_size, 1u)] = v;
                }
            }
        }
    }
}

// previous senders: snapshot rows back to kInf
__global__ void batch_reset_kernel(uint32_t* fr0, uint32_t* fr1, const BatchCtl* __restrict__ ctl,
                                   uint32_t* __restrict__ sval, uint32_t* __restrict__ smask) {
    const uint32_t* __restrict__ F = fr_cur(fr0, fr1, ctl);
    const uint32_t f = ctl->f;
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < f; i += nwarps) {
        const uint32_t u = F[i];
        sval[(uint64_t)u * kLanes + lane] = kInf;
        if (lane == 0) smask[u] = 0;
    }
}

// next senders: publish their new values, count their messages per source
__global__ void batch_apply_kernel(uint32_t* fr0, uint32_t* fr1, const BatchCtl* __restrict__ ctl, uint32_t n,
                                   const uint64_t* __restrict__ off, const uint32_t* __restrict__ dist,
                                   uint32_t* __restrict__ sval, uint32_t* __restrict__ smask,
                                   uint32_t* __restrict__ cmask, BatchCounters* __restrict__ ctr) {
    const uint32_t* __restrict__ F = fr_next(fr0, fr1, ctl);
    const uint32_t f = min(ctr->next_size, n);  // a larger count is reported by the step kernel
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long msgs = 0, edges = 0;
    for (uint64_t i = warp; i < f; i += nwarps) {
        const uint32_t v = F[i];
        const uint32_t mask = cmask[v];
        const bool mine = (mask >> lane) & 1u;
        const uint64_t deg = off[v + 1] - off[v];
        sval[(uint64_t)v * kLanes + lane] = mine ? dist[(uint64_t)v * kLanes + lane] : kInf;
        if (mine) msgs += deg;
        edges += deg;
        __syncwarp();
        if (lane == 0) {
            smask[v] = mask;
            cmask[v] = 0;
        }
    }
    if (msgs) atomicAdd(&ctr->msgs[lane], msgs);
    if (lane == 0 && edges) atomicAdd(&ctr->edges, edges);
}

// End of a superstep: a live lane whose next senders send nothing has finished
// (its count is final); otherwise it runs another superstep.  The next frontier
// becomes current, the counters are cleared, and the WHILE condition says
// whether the graph runs another superstep: while a lane holds a query or the
// source list has more, not past kLoopCap in one launch, and with host seeding
// not past a superstep in which a lane finished (or when queries wait for a
// free lane).
__global__ void batch_step_kernel(BatchCtl* __restrict__ ctl, BatchCounters* __restrict__ ctr, uint32_t n,
                                  cudaGraphConditionalHandle loop) {
    const uint32_t b = threadIdx.x;
    const uint32_t live = ctl->live;
    bool fin = false;
    if ((live >> b) & 1u) {
        if (ctr->msgs[b] > 0)
            ++ctl->count[b];
        else
            fin = true;
    }
    ctr->msgs[b] = 0;
    const unsigned finm = __ballot_sync(0xFFFFFFFFu, fin);
    if (fin && ctl->steps_out) ctl->steps_out[ctl->row[b]] = ctl->count[b];
    if (b == 0) {
        ++ctl->supersteps;
        if (!ctl->push) ++ctl->pull_supersteps;
        if (finm) ++ctl->harvests;
        const uint32_t fn = ctr->next_size;
        uint32_t status = ctl->status | ctr->status;
        if (fn > n) status |= kStatusInternal;
        ctl->status = status;
        ctl->f = fn <= n ? fn : 0u;
        ctl->cur ^= 1u;
        ctl->f_edges = ctr->edges;
        const uint32_t now_live = live & ~finm;
        ctl->live = now_live;
        ctl->finished = finm;
        ctr->next_size = 0;
        ctr->status = 0;
        ctr->edges = 0;
        ctr->ntasks = 0;
        const bool from_list = ctl->nqueries != 0;
        const bool more = (now_live != 0 || (from_list && ctl->next_query < ctl->nqueries)) && status == 0;
        bool stop = false;
        if (!from_list && ctl->stop_on_finish) {
            stop = finm != 0;
            if (ctl->admit && *ctl->admit && now_live != 0xFFFFFFFFu) stop = true;
        }
        ctl->done = !more;
        const unsigned it = ctl->iter + 1;
        const bool again = more && !stop && it < kLoopCap;
        ctl->iter = again ? it : 0u;
        cudaGraphSetConditional(loop, again ? 1u : 0u);
    }
}

// Finished lanes: out[row][v] = dist[inv[v]][lane] for every caller id v, and the
// lane's column back to kInf for its next query.
__global__ void batch_harvest_kernel(const BatchCtl* __restrict__ ctl, const uint32_t* __restrict__ inv, uint32_t n,
                                     uint32_t* __restrict__ dist) {
    const uint32_t fin = ctl->finished;
    if (!fin) return;
    uint32_t* __restrict__ out = ctl->out;
    const uint64_t stride = ctl->out_stride;
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += step) {
        uint32_t* d = dist + (uint64_t)inv[v] * kLanes;
        for (uint32_t r = fin; r; r &= r - 1) {
            const uint32_t b = __ffs(r) - 1;
            out[(uint64_t)ctl->row[b] * stride + v] = d[b];
            d[b] = kInf;
        }
    }
}

unsigned grid_for_warps(uint64_t warps, int sms) {
    uint64_t blocks = (warps + 7) / 8;
    const uint64_t cap = (uint64_t)sms * 16;
    if (blocks < 1) blocks = 1;
    return (unsigned)(blocks < cap ? blocks : cap);
}

}  // namespace

// Batch workspace lives with the graph; allocated on first use.
struct BatchWorkspace {
    uint32_t* dist = nullptr;   // [n][32]
    uint32_t* sval = nullptr;   // [n][32]
    uint32_t* smask = nullptr;  // [n]
    uint32_t* cmask = nullptr;  // [n]
    uint32_t* fr[2] = {nullptr, nullptr};
    uint32_t* chunk_row = nullptr;
    uint64_t chunks = 0, chunk_cap = 0;
    uint32_t chunk = 0;  // in-edges per warp task of the pull form (0: not set up yet)
    BatchCounters* ctr = nullptr;
    BatchCtl* ctl = nullptr;
    BatchCtl* h_ctl = nullptr;            // pinned mirror
    unsigned int* h_admit = nullptr;      // mapped host flag (serving)
    unsigned int* d_admit = nullptr;      // its device address
    uint32_t* list = nullptr;             // source list (caller ids) of ipg_sssp_batch
    uint32_t* steps = nullptr;            // per-query superstep counts of ipg_sssp_batch
    size_t list_cap = 0;
    unsigned long long* tasks = nullptr;  // push tasks of the current senders
    bool clean = false;                   // dist/sval all kInf, masks and counters zero
    ipg_batch_info info{};                // totals of the last ipg_sssp_batch call
    cudaGraphExec_t loop[3] = {nullptr, nullptr, nullptr};  // superstep loop, per weight kind
};

void batch_free(ipg_graph* g) {
    BatchWorkspace* b = (BatchWorkspace*)g->batch;
    if (!b) return;
    cudaFree(b->dist);
    cudaFree(b->sval);
    cudaFree(b->smask);
    cudaFree(b->cmask);
    cudaFree(b->fr[0]);
    cudaFree(b->fr[1]);
    cudaFree(b->chunk_row);
    cudaFree(b->ctr);
    cudaFree(b->ctl);
    cudaFree(b->tasks);
    cudaFree(b->list);
    cudaFree(b->steps);
    if (b->h_ctl) cudaFreeHost(b->h_ctl);
    if (b->h_admit) cudaFreeHost(b->h_admit);
    for (int i = 0; i < 3; ++i)
        if (b->loop[i]) cudaGraphExecDestroy(b->loop[i]);
    delete b;
    g->batch = nullptr;
}

static ipg_status batch_prepare(ipg_graph* g, cudaStream_t st) {
    IPG_TRY(ensure_csc(g, st));
    if (g->batch) return IPG_OK;
    BatchWorkspace* b = new BatchWorkspace();
    g->batch = b;
    const uint32_t n = g->n;
    IPG_CUDA(cudaMalloc(&b->dist, sizeof(uint32_t) * kLanes * (size_t)n));
    IPG_CUDA(cudaMalloc(&b->sval, sizeof(uint32_t) * kLanes * (size_t)n));
    IPG_CUDA(cudaMalloc(&b->smask, sizeof(uint32_t) * (size_t)n));
    IPG_CUDA(cudaMalloc(&b->cmask, sizeof(uint32_t) * (size_t)n));
    IPG_CUDA(cudaMalloc(&b->fr[0], sizeof(uint32_t) * (size_t)n));
    IPG_CUDA(cudaMalloc(&b->fr[1], sizeof(uint32_t) * (size_t)n));
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

// The in-edge chunks of the pull form (the batched engine's tile size, a tuning knob):
// their first rows are recomputed, and the loop graphs, which bake in the chunk
// count, rebuilt, when the size changes.
static ipg_status batch_chunks(ipg_graph* g, BatchWorkspace* b, cudaStream_t st) {
    const uint32_t want = (uint32_t)batch_chunk_for(g);
    if (b->chunk == want) return IPG_OK;
    for (auto& x : b->loop)
        if (x) {
            cudaGraphExecDestroy(x);
            x = nullptr;
        }
    const uint64_t chunks = (g->m + want - 1) / want;
    if (chunks > b->chunk_cap) {
        cudaFree(b->chunk_row);
        b->chunk_row = nullptr;
        b->chunk_cap = 0;
        IPG_CUDA(cudaMalloc(&b->chunk_row, sizeof(uint32_t) * (chunks ? chunks : 1)));
        b->chunk_cap = chunks;
    }
    if (chunks) {
        chunk_rows_kernel<<<grid_for_warps(chunks / 32 + 1, sm_count_of(g->device)), 256, 0, st>>>(
            g->csc_off, g->n, g->m, chunks, want, b->chunk_row);
        IPG_CUDA(cudaGetLastError());
    }
    b->chunks = chunks;
    b->chunk = want;
    return IPG_OK;
}

// the superstep body, enqueued on `st` (captured into the loop graph)
static void batch_superstep(ipg_graph* g, BatchWorkspace* b, int wkind, cudaGraphConditionalHandle loop,
                            cudaStream_t st) {
    const int sms = sm_count_of(g->device);
    const unsigned grid = grid_for_warps(b->chunks, sms);
    const unsigned fixed = (unsigned)sms * 8;  // frontier passes: persistent, the size is read on the device
#define IPG_BATCH_PULL(K)                                                                                         \
    batch_pull_kernel<K><<<grid, 256, 0, st>>>(g->csc_off, g->csc_src, g->csc_w8, g->csc_w, b->chunk_row,       \
                                               b->chunks, g->n, g->m, b->sval, b->smask, b->dist, b->cmask,      \
                                               b->fr[0], b->fr[1], b->ctl, b->ctr, b->chunk)
#define IPG_BATCH_PUSH(K)                                                                                         \
    batch_push_kernel<K><<<fixed, 256, 0, st>>>(g->off, g->col, g->w8, g->w, b->tasks, b->sval, b->smask, b->dist,  \
                                                b->cmask, b->fr[0], b->fr[1], b->ctl, b->ctr)
    batch_refill_kernel<<<1, kLanes, 0, st>>>(b->ctl, g->inv, g->off, g->m, b->dist, b->sval, b->smask, b->fr[0],
                                              b->fr[1]);
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
    batch_reset_kernel<<<fixed, 256, 0, st>>>(b->fr[0], b->fr[1], b->ctl, b->sval, b->smask);
    batch_apply_kernel<<<fixed, 256, 0, st>>>(b->fr[0], b->fr[1], b->ctl, g->n, g->off, b->dist, b->sval, b->smask,
                                              b->cmask, b->ctr);
    batch_step_kernel<<<1, kLanes, 0, st>>>(b->ctl, b->ctr, g->n, loop);
    batch_harvest_kernel<<<fixed, 256, 0, st>>>(b->ctl, g->inv, g->n, b->dist);
}

// Builds the graph [WHILE (cond) { superstep }] for this workspace and weight kind.
static ipg_status batch_loop_graph(ipg_graph* g, BatchWorkspace* b, int wkind) {
    if (b->loop[wkind]) return IPG_OK;
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
        batch_superstep(g, b, wkind, handle, cap);
        cudaGraph_t body = nullptr;
        e = cudaStreamEndCapture(cap, &body);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->loop[wkind], graph, 0);
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
    IPG_TRY(batch_chunks(g, b, st));
    IPG_TRY(batch_loop_graph(g, b, weight_kind(g)));
    if (!b->clean) {
        IPG_CUDA(cudaMemsetAsync(b->dist, 0xFF, sizeof(uint32_t) * kLanes * n, st));
        IPG_CUDA(cudaMemsetAsync(b->sval, 0xFF, sizeof(uint32_t) * kLanes * n, st));
        IPG_CUDA(cudaMemsetAsync(b->smask, 0, sizeof(uint32_t) * n, st));
        IPG_CUDA(cudaMemsetAsync(b->cmask, 0, sizeof(uint32_t) * n, st));
        IPG_CUDA(cudaMemsetAsync(b->ctr, 0, sizeof(BatchCounters), st));
    }
    b->clean = false;
    *b->h_ctl = init;
    IPG_CUDA(cudaMemcpyAsync(b->ctl, b->h_ctl, sizeof(BatchCtl), cudaMemcpyHostToDevice, st));
    return IPG_OK;
}

static BatchCtl batch_ctl_init(const ipg_graph* g) {
    BatchCtl c;
    memset(&c, 0, sizeof(c));
    c.divisor = (unsigned long long)batch_divisor_for(g);
    return c;
}

// one graph launch, then the control block back on the host
static ipg_status batch_launch(ipg_graph* g, BatchWorkspace* b, cudaStream_t st, const char* name) {
    IPG_CUDA(cudaGraphLaunch(b->loop[weight_kind(g)], st));
    IPG_CUDA(cudaMemcpyAsync(b->h_ctl, b->ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, st));
    IPG_CUDA(cudaStreamSynchronize(st));
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
        b->list = b->steps = nullptr;
        b->list_cap = 0;
        IPG_CUDA(cudaMalloc(&b->list, sizeof(uint32_t) * k));
        IPG_CUDA(cudaMalloc(&b->steps, sizeof(uint32_t) * k));
        b->list_cap = k;
    }
    IPG_CUDA(cudaMemcpyAsync(b->list, sources, sizeof(uint32_t) * k, cudaMemcpyHostToDevice, st));
    BatchCtl init = batch_ctl_init(g);
    init.nqueries = k;
    init.src_list = b->list;
    init.steps_out = b->steps;
    init.out = dist_dev;
    init.out_stride = g->n;
    IPG_TRY(batch_session_begin(g, b, init, st));
    // every lane is refilled on the device: one launch per kLoopCap supersteps
    const uint64_t bound = ((uint64_t)k + kLanes) * ((uint64_t)g->n + 2) / kLoopCap + 2;
    uint64_t launches = 0;
    for (;; ++launches) {
        if (launches > bound)
            return set_error(IPG_EDEVICE, "ipg_sssp_batch: the superstep loop did not end");
        IPG_TRY(batch_launch(g, b, st, "ipg_sssp_batch"));
        if (b->h_ctl->done) break;
    }
    b->clean = true;  // every lane was harvested
    b->info.queries = k;
    b->info.supersteps = b->h_ctl->supersteps;
    b->info.pull_supersteps = b->h_ctl->pull_supersteps;
    b->info.harvests = b->h_ctl->harvests;
    b->info.launches = launches + 1;
    if (supersteps_out) {
        IPG_CUDA(cudaMemcpyAsync(supersteps_out, b->steps, sizeof(uint32_t) * k, cudaMemcpyDeviceToHost, st));
        IPG_CUDA(cudaStreamSynchronize(st));
    }
    return IPG_OK;
}

// ---- lane sessions driven by the host (the server) ------------------------------

ipg_status lanes_open(ipg_graph* g, uint32_t* stage_dev, cudaStream_t st) {
    DeviceGuard guard(g->device);
    IPG_TRY(batch_prepare(g, st));
    BatchWorkspace* b = (BatchWorkspace*)g->batch;
    *b->h_admit = 0;
    BatchCtl init = batch_ctl_init(g);
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
    if (nseed > (uint32_t)__builtin_popcount(~h->live)) return set_error(IPG_EINVAL, "lanes_step: too many seeds");
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
    if (!nseed && h->live == 0) {
        rep->live = 0;
        rep->finished = 0;
        return IPG_OK;
    }
    *b->h_admit = 0;
    IPG_TRY(batch_launch(g, b, st, "lanes_step"));
    rep->live = h->live;
    rep->finished = h->finished;
    for (int l = 0; l < kLanes; ++l) {
        rep->row[l] = h->row[l];
        rep->count[l] = h->count[l];
    }
    return IPG_OK;
}

void lanes_close(ipg_graph* g) {
    BatchWorkspace* b = (BatchWorkspace*)g->batch;
    if (b && b->h_ctl->live == 0 && b->h_ctl->status == 0) b->clean = true;
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

// host output: groups of 32 sources through a 32 x n device staging buffer
ipg_status ipg_sssp_batch(ipg_graph* g, const uint32_t* sources, uint32_t k, uint32_t* dist_out,
                          uint32_t* supersteps_out) {
    if (!g) return set_error(IPG_EINVAL, "ipg_sssp_batch: graph is NULL");
    if (k && (!sources || !dist_out)) return set_error(IPG_EINVAL, "ipg_sssp_batch: NULL argument");
    DeviceGuard guard(g->device);
    const uint64_t n = g->n;
    uint32_t* stage = nullptr;
    const uint32_t group = k < 32 ? k : 32;
    if (k) IPG_CUDA(cudaMalloc(&stage, sizeof(uint32_t) * group * (n ? n : 1)));
    ipg_status rc = IPG_OK;
    for (uint32_t i0 = 0; i0 < k && rc == IPG_OK; i0 += 32) {
        const uint32_t kk = k - i0 < 32 ? k - i0 : 32;
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
