// General combiners (Sec. III, Fig. 1): vertex programs whose messages are wider
// than 32 bits and whose combine is not a hardware atomic, run through the
// hybrid combiner of ipg_combiner.cuh.
//
// One push superstep s, given the senders F_s:
//   split    the frontier's out-degree prefix and merge-path tiles of
//            (frontier rows + their edges), shared with the min-combiner push
//            path (frontier_prepare / frontier_partition);
//   scatter  one thread per edge u -> v: msg = message(sender state of u, w);
//            deliver it to v's mailbox with ipg_mail_send.  The thread whose
//            message was v's first (it took the lock and raised the flag)
//            appends v to the receiver list — so the receivers, the vertices
//            that are active in superstep s+1, are exactly those with a message,
//            found without scanning all n mailboxes, and counted exactly;
//   apply    one thread per receiver: read the combined message, reset the flag
//            to empty, run the program's compute step (apply), and append the
//            vertex to F_{s+1} if it sends.
// The state of a sender is only read during scatter and only written during
// apply, so no snapshot is needed: the execution is synchronous Pregel,
// superstep for superstep.
//
// Programs:
//   TreeProgram   SSSP with a parent: the 64-bit message (distance << 32 | caller
//                 id of the sender), combined by the minimum, which is the
//                 lexicographic minimum of (distance, sender); a vertex sends when
//                 its distance drops.
//   PathsProgram  shortest-path counting by BFS levels: the 128-bit message
//                 (level, count), combined by the smallest level with the counts
//                 of equal levels added (modulo 2^64); a vertex sends once, when
//                 it first gets a level.
// ipg_combine_dev runs the combination step alone on a caller's message list.
#include <utility>

#include "ipg_combiner.cuh"
#include "ipg_internal.cuh"

namespace ipg {
namespace {

constexpr int kGenThreads = 256;
constexpr uint32_t kTile = kFrontierTile;
constexpr int kEdgesPerThread = 4;
constexpr unsigned long long kUnreached64 = ~0ull;

struct GenCounters {
    unsigned int recv;    // receivers appended in this superstep
    unsigned int next;    // senders of the next superstep
    unsigned int status;  // kStatusOverflow | IPG_MAIL_STATUS_TIMEOUT | kStatusInternal
    unsigned int pad;
};

struct GenWork {
    size_t cap = 0;                      // vertices the buffers hold
    void* state = nullptr;               // 16 B per vertex (either program)
    void* mail = nullptr;                // 16 B per vertex
    uint32_t* flag = nullptr;            // mailbox flags
    uint32_t* recv = nullptr;            // receiver list
    GenCounters* gc = nullptr;           // device
    GenCounters* h_gc = nullptr;         // pinned host mirror
};

// ---------------------------------------------------------------------------
// vertex programs

struct TreeProgram {
    using Msg = unsigned long long;    // (distance << 32) | caller id of the sender
    using State = unsigned long long;  // (distance << 32) | caller id of the parent
    struct Sender {
        uint32_t dist, id;
    };
    struct Combine {
        __device__ Msg operator()(const Msg& a, const Msg& b) const { return a < b ? a : b; }
    };
    static constexpr bool kWeighted = true;
    __device__ static State initial(bool is_source, uint32_t source_id) {
        return is_source ? (unsigned long long)source_id : kUnreached64;
    }
    __device__ static Sender sender(const State* st, const uint32_t* perm, uint32_t u) {
        return Sender{(uint32_t)(st[u] >> 32), perm[u]};
    }
    __device__ static Msg message(const Sender& s, uint32_t w, unsigned int* status) {
        unsigned long long d = (unsigned long long)s.dist + w;
        if (d >= kInf) {
            atomicOr(status, kStatusOverflow);
            d = kInf - 1;
        }
        return (d << 32) | s.id;
    }
    // compute step of a receiver: returns whether it sends; *changed if its state moved
    __device__ static bool apply(State* st, const Msg& m, bool* changed) {
        const State old = *st;
        *changed = m < old;
        if (!*changed) return false;
        *st = m;
        return (m >> 32) < (old >> 32);
    }
};

struct alignas(16) LevelCount {
    unsigned long long level, count;
};

struct PathsProgram {
    using Msg = LevelCount;
    using State = LevelCount;
    using Sender = LevelCount;
    struct Combine {
        __device__ Msg operator()(const Msg& a, const Msg& b) const {
            if (a.level < b.level) return a;
            if (b.level < a.level) return b;
            return Msg{a.level, a.count + b.count};
        }
    };
    static constexpr bool kWeighted = false;
    __device__ static State initial(bool is_source, uint32_t) {
        return is_source ? State{0ull, 1ull} : State{kUnreached64, 0ull};
    }
    __device__ static Sender sender(const State* st, const uint32_t*, uint32_t u) { return st[u]; }
    __device__ static Msg message(const Sender& s, uint32_t, unsigned int*) { return Msg{s.level + 1, s.count}; }
    __device__ static bool apply(State* st, const Msg& m, bool* changed) {
        *changed = st->level == kUnreached64;
        if (*changed) *st = m;
        return *changed;
    }
};

// ---------------------------------------------------------------------------
// kernels

template <class P>
__global__ void gen_init_kernel(typename P::State* __restrict__ state, uint32_t* __restrict__ flag, uint32_t n,
                                const uint32_t* __restrict__ inv, uint32_t source, uint32_t* __restrict__ frontier) {
    const uint32_t s = inv[source];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        state[v] = P::initial(v == s, source);
        flag[v] = IPG_MAIL_EMPTY;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) frontier[0] = s;
}

template <int kWeightKind>
__device__ __forceinline__ uint32_t gen_weight(const uint8_t* __restrict__ w8, const uint32_t* __restrict__ w32,
                                               unsigned long long p) {
    if (kWeightKind == 1) return (uint32_t)__ldcs(w8 + p);
    if (kWeightKind == 2) return __ldcs(w32 + p);
    return 1u;
}

// warp-aggregated append of `v` (where `take`) to list[*size]; every lane of the warp calls it
__device__ __forceinline__ void warp_append(bool take, uint32_t v, uint32_t* __restrict__ list, unsigned int* size) {
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, take);
    if (!mask) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned pos = 0;
    if (lane == leader) pos = atomicAdd(size, (unsigned)__popc(mask));
    pos = __shfl_sync(0xFFFFFFFFu, pos, leader);
    if (take) list[pos + __popc(mask & ((1u << lane) - 1u))] = v;
}

template <class P>
constexpr size_t scatter_smem() {
    return (sizeof(typename P::Sender) + sizeof(unsigned long long) + sizeof(uint32_t)) * (kTile + 1);
}

// kWeightKind: 0 = length 1, 1 = u8 weights, 2 = u32 weights.  kWarp: pre-combine within warps.
template <class P, int kWeightKind, bool kWarp>
__global__ void __launch_bounds__(kGenThreads) gen_scatter_kernel(
    const unsigned long long* __restrict__ prefix, const unsigned long long* __restrict__ rowstart,
    const uint32_t* __restrict__ F, const uint32_t* __restrict__ tile_row, const uint32_t* __restrict__ col,
    const uint8_t* __restrict__ w8, const uint32_t* __restrict__ w32, const typename P::State* __restrict__ state,
    const uint32_t* __restrict__ perm, uint32_t* __restrict__ flag, typename P::Msg* __restrict__ mail,
    uint32_t* __restrict__ recv, const PushCounters* __restrict__ pc, GenCounters* __restrict__ gc, uint32_t f) {
    using Sender = typename P::Sender;
    using Msg = typename P::Msg;
    using Combine = typename P::Combine;
    extern __shared__ __align__(16) unsigned char gen_smem[];
    Sender* s_snd = reinterpret_cast<Sender*>(gen_smem);
    unsigned long long* s_base = reinterpret_cast<unsigned long long*>(s_snd + kTile + 1);
    uint32_t* s_start = reinterpret_cast<uint32_t*>(s_base + kTile + 1);
    const uint64_t E = pc->edges;
    const uint32_t tiles = pc->tiles;
    const uint64_t total = (uint64_t)f + E;
    const int tid = threadIdx.x;
    for (uint32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const uint64_t d0 = (uint64_t)tile * kTile;
        const uint64_t d1 = d0 + kTile < total ? d0 + kTile : total;
        const uint32_t i0 = tile_row[tile];
        const uint32_t i1 = tile_row[tile + 1];
        const uint64_t j0 = d0 - i0;
        const uint32_t R = i1 - i0;
        const uint32_t Et = (uint32_t)((d1 - i1) - j0);
        __syncthreads();  // the previous tile is done with shared memory
        for (uint32_t k = tid; k <= R; k += kGenThreads) {
            const uint32_t r = i0 + k;
            if (r < f) {
                const unsigned long long p = prefix[r];
                s_start[k] = p > j0 ? (uint32_t)(p - j0) : 0u;
                s_base[k] = rowstart[r] + (j0 - p);  // edge position = base + k (mod 2^64)
                s_snd[k] = P::sender(state, perm, F[r]);
            } else {
                s_start[k] = Et + 1;
                s_base[k] = 0;
            }
        }
        __syncthreads();
        for (uint32_t k0 = 0; k0 < Et; k0 += kGenThreads * kEdgesPerThread) {
            uint32_t v[kEdgesPerThread];
            Msg msg[kEdgesPerThread];
            bool ok[kEdgesPerThread];
#pragma unroll
            for (int q = 0; q < kEdgesPerThread; ++q) {
                const uint32_t k = k0 + tid + q * kGenThreads;
                ok[q] = k < Et;
                v[q] = 0;
                if (ok[q]) {
                    uint32_t lo = 0, hi = R;  // row of edge k: the last row whose start is <= k
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi + 1) >> 1;
                        if (s_start[mid] <= k)
                            lo = mid;
                        else
                            hi = mid - 1;
                    }
                    const unsigned long long p = s_base[lo] + k;
                    v[q] = __ldcs(col + p);
                    msg[q] = P::message(s_snd[lo], P::kWeighted ? gen_weight<kWeightKind>(w8, w32, p) : 1u,
                                        &gc->status);
                }
            }
#pragma unroll
            for (int q = 0; q < kEdgesPerThread; ++q) {
                bool send = ok[q];
                if (kWarp) {
                    const unsigned act = __ballot_sync(0xFFFFFFFFu, ok[q]);
                    if (ok[q]) send = ipg_warp_combine<Combine>(act, v[q], &msg[q]);
                }
                bool first = false;
                if (send) first = ipg_mail_send<Combine>(&flag[v[q]], &mail[v[q]], msg[q], &gc->status) == 1;
                warp_append(first, v[q], recv, &gc->recv);
            }
        }
    }
}

template <class P>
__global__ void __launch_bounds__(kGenThreads) gen_apply_kernel(const uint32_t* __restrict__ recv,
                                                                 uint32_t* __restrict__ flag,
                                                                 const typename P::Msg* __restrict__ mail,
                                                                 typename P::State* __restrict__ state,
                                                                 uint32_t* __restrict__ next,
                                                                 GenCounters* __restrict__ gc, uint32_t n) {
    const uint32_t r = gc->recv;
    if (r > n) {  // cannot happen: each vertex is appended by its first message only
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&gc->status, kStatusInternal);
        return;
    }
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < r; base += stride) {
        const uint64_t i = base + threadIdx.x;
        bool send = false;
        uint32_t v = 0;
        if (i < r) {
            v = recv[i];
            const typename P::Msg m = mail[v];
            flag[v] = IPG_MAIL_EMPTY;
            typename P::State s = state[v];
            bool changed;
            send = P::apply(&s, m, &changed);
            if (changed) state[v] = s;
        }
        warp_append(send, v, next, &gc->next);
    }
}

__global__ void tree_output_kernel(const unsigned long long* __restrict__ state, const uint32_t* __restrict__ inv,
                                   uint32_t n, uint32_t* __restrict__ dist, uint32_t* __restrict__ parent) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
        const unsigned long long s = state[inv[c]];
        dist[c] = (uint32_t)(s >> 32);
        parent[c] = (uint32_t)s;
    }
}

__global__ void paths_output_kernel(const LevelCount* __restrict__ state, const uint32_t* __restrict__ inv, uint32_t n,
                                    uint32_t* __restrict__ level, unsigned long long* __restrict__ paths) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
        const LevelCount s = state[inv[c]];
        level[c] = s.level == kUnreached64 ? kInf : (uint32_t)s.level;
        paths[c] = s.count;
    }
}

unsigned grid_for(uint64_t work, unsigned cap) {
    uint64_t b = (work + 255) / 256;
    if (b < 1) b = 1;
    return (unsigned)(b < cap ? b : cap);
}

// ---------------------------------------------------------------------------
// host side

ipg_status ensure_work(ipg_graph* g, GenWork** out) {
    GenWork* w = static_cast<GenWork*>(g->generic);
    if (!w) {
        w = new GenWork();
        g->generic = w;
    }
    const size_t n = g->n ? g->n : 1;
    if (w->cap < n) {
        cudaFree(w->state);
        cudaFree(w->mail);
        cudaFree(w->flag);
        cudaFree(w->recv);
        w->state = w->mail = nullptr;
        w->flag = w->recv = nullptr;
        w->cap = 0;
        IPG_CUDA(cudaMalloc(&w->state, 16 * n));
        IPG_CUDA(cudaMalloc(&w->mail, 16 * n));
        IPG_CUDA(cudaMalloc(&w->flag, sizeof(uint32_t) * n));
        IPG_CUDA(cudaMalloc(&w->recv, sizeof(uint32_t) * n));
        w->cap = n;
    }
    if (!w->gc) IPG_CUDA(cudaMalloc(&w->gc, sizeof(GenCounters)));
    if (!w->h_gc) IPG_CUDA(cudaHostAlloc(&w->h_gc, sizeof(GenCounters), cudaHostAllocDefault));
    *out = w;
    return IPG_OK;
}

template <class P, int kWeightKind>
ipg_status launch_scatter(ipg_graph* g, GenWork* w, uint32_t f, bool warp, cudaStream_t st) {
    constexpr size_t smem = scatter_smem<P>();
    auto kern = warp ? gen_scatter_kernel<P, kWeightKind, true> : gen_scatter_kernel<P, kWeightKind, false>;
    IPG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGenThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const unsigned grid = (unsigned)(sm_count_of(g->device) * per_sm);
    kern<<<grid, kGenThreads, smem, st>>>(g->fr_prefix, g->fr_rowstart, g->frontier[0], g->push_tile_row, g->col,
                                          g->w8, g->w, static_cast<const typename P::State*>(w->state), g->perm,
                                          w->flag, static_cast<typename P::Msg*>(w->mail), w->recv, g->counters,
                                          w->gc, f);
    IPG_CUDA(cudaGetLastError());
    return IPG_OK;
}

template <class P>
ipg_status scatter_dispatch(ipg_graph* g, GenWork* w, uint32_t f, bool warp, cudaStream_t st) {
    if (!P::kWeighted || (!g->w8 && !g->w)) return launch_scatter<P, 0>(g, w, f, warp, st);
    if (g->w8) return launch_scatter<P, 1>(g, w, f, warp, st);
    return launch_scatter<P, 2>(g, w, f, warp, st);
}

// Runs program P from `source` (a caller id).  The frontier ping-pongs between
// g->frontier[0] and [1]; the scatter kernel always reads frontier[0], so the
// two pointers are swapped on the host between supersteps.
template <class P>
ipg_status gen_run(ipg_graph* g, uint32_t source, ipg_stats* stats, cudaStream_t st, const char* name,
                   GenWork** work_out) {
    stats_begin(stats);
    if (!g) return set_error(IPG_EINVAL, "%s: graph is NULL", name);
    if (source >= g->n) return set_error(IPG_EINVAL, "%s: source %u >= n = %u", name, source, g->n);
    DeviceGuard guard(g->device);
    if (!guard.ok) return set_error(IPG_ECUDA, "%s: cannot select the graph's device", name);
    const uint32_t n = g->n;
    const bool timing = stats && (stats->flags & IPG_STAT_TIMING);
    IPG_TRY(ensure_push_workspace(g, false));
    GenWork* w;
    IPG_TRY(ensure_work(g, &w));
    if (timing) IPG_TRY(g->timer.init());
    cudaEvent_t* ev = g->timer.ev;
    const unsigned sms = (unsigned)sm_count_of(g->device);
    IPG_CUDA(cudaMemsetAsync(w->gc, 0, sizeof(GenCounters), st));
    gen_init_kernel<P><<<grid_for(n, sms * 8), 256, 0, st>>>(static_cast<typename P::State*>(w->state), w->flag, n,
                                                             g->inv, source, g->frontier[0]);
    IPG_CUDA(cudaGetLastError());
    const bool warp = tuning().combine_warp != 0;
    uint32_t f = 1;
    uint32_t s = 0;
    uint32_t count = 0;
    uint64_t prev_recv = 0;
    ipg_status rc = IPG_OK;
    for (;;) {
        if (timing) IPG_CUDA(cudaEventRecord(ev[0], st));
        IPG_TRY(frontier_prepare(g, g->frontier[0], f, nullptr, st));
        IPG_TRY(frontier_partition(g, f, st));
        IPG_CUDA(cudaMemsetAsync(w->gc, 0, 2 * sizeof(unsigned int), st));  // recv, next
        if (timing) IPG_CUDA(cudaEventRecord(ev[1], st));
        IPG_TRY(scatter_dispatch<P>(g, w, f, warp, st));
        gen_apply_kernel<P><<<sms * 8, kGenThreads, 0, st>>>(w->recv, w->flag,
                                                             static_cast<const typename P::Msg*>(w->mail),
                                                             static_cast<typename P::State*>(w->state),
                                                             g->frontier[1], w->gc, n);
        IPG_CUDA(cudaGetLastError());
        if (timing) IPG_CUDA(cudaEventRecord(ev[2], st));
        IPG_CUDA(cudaMemcpyAsync(g->h_counters, g->counters, sizeof(PushCounters), cudaMemcpyDeviceToHost, st));
        IPG_CUDA(cudaMemcpyAsync(w->h_gc, w->gc, sizeof(GenCounters), cudaMemcpyDeviceToHost, st));
        IPG_CUDA(cudaStreamSynchronize(st));
        const unsigned long long edges = g->h_counters->edges;
        const GenCounters h = *w->h_gc;
        if (h.status & kStatusOverflow) rc = set_error(IPG_EOVERFLOW, "%s: a path length reached UINT32_MAX", name);
        if (h.status & IPG_MAIL_STATUS_TIMEOUT)
            rc = set_error(IPG_ETIMEOUT, "%s: a bounded wait in the message combiner ran out", name);
        if (h.status & kStatusInternal) rc = set_error(IPG_EDEVICE, "%s: inconsistent receiver count", name);
        if (rc == IPG_OK && (h.recv > n || h.next > n))
            rc = set_error(IPG_EDEVICE, "%s: list overflow (%u, %u > n)", name, h.recv, h.next);
        if (rc != IPG_OK) {
            if (stats) stats->count = 0;
            return rc;
        }
        if (stats) {
            ipg_superstep_stats r{};
            r.superstep = s;
            r.flags = IPG_STAT_RECEIVERS | (timing ? IPG_STAT_TIMING : 0u);
            r.active = s == 0 ? n : prev_recv;
            r.senders = f;
            r.messages_sent = edges;
            r.receivers = h.recv;
            if (timing) {
                cudaEventElapsedTime(&r.kernel_ms, ev[1], ev[2]);
                cudaEventElapsedTime(&r.superstep_ms, ev[0], ev[2]);
            }
            stats_put(stats, s, r);
        }
        if (h.next == 0) {
            count = s + 1;
            if (edges > 0) {  // the receivers run one more superstep and send nothing
                if (stats) {
                    ipg_superstep_stats r{};
                    r.superstep = s + 1;
                    r.flags = IPG_STAT_RECEIVERS;
                    r.active = h.recv;
                    stats_put(stats, s + 1, r);
                }
                count = s + 2;
            }
            break;
        }
        prev_recv = h.recv;
        f = h.next;
        std::swap(g->frontier[0], g->frontier[1]);
        ++s;
    }
    if (stats) stats->count = count;
    *work_out = w;
    return IPG_OK;
}

// ---------------------------------------------------------------------------
// the combination step alone

template <class Msg>
struct XorCombine {
    __device__ Msg operator()(const Msg& a, const Msg& b) const { return a ^ b; }
};
template <class Msg>
struct MinCombine {
    __device__ Msg operator()(const Msg& a, const Msg& b) const { return a < b ? a : b; }
};
template <class Msg>
struct SumCombine {
    __device__ Msg operator()(const Msg& a, const Msg& b) const { return a + b; }
};

template <class Combine, class Msg, bool kWarp>
__global__ void __launch_bounds__(kGenThreads) combine_kernel(const uint32_t* __restrict__ dst,
                                                               const Msg* __restrict__ msgs, uint64_t k, uint32_t n,
                                                               uint32_t* __restrict__ flag, Msg* __restrict__ mail,
                                                               GenCounters* __restrict__ gc, unsigned int spin_limit) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned int first_count = 0;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < k; base += stride) {
        const uint64_t i = base + threadIdx.x;
        bool ok = i < k;
        uint32_t v = 0;
        Msg m{};
        if (ok) {
            v = __ldcs(dst + i);
            m = msgs[i];
            if (v >= n) {
                atomicOr(&gc->status, kStatusInternal);
                ok = false;
            }
        }
        bool send = ok;
        if (kWarp) {
            const unsigned act = __ballot_sync(0xFFFFFFFFu, ok);
            if (ok) send = ipg_warp_combine<Combine>(act, v, &m);
        }
        if (send && ipg_mail_send<Combine>(&flag[v], &mail[v], m, &gc->status, spin_limit) == 1) ++first_count;
    }
    for (int o = 16; o > 0; o >>= 1) first_count += __shfl_down_sync(0xFFFFFFFFu, first_count, o);
    if ((threadIdx.x & 31) == 0 && first_count) atomicAdd(&gc->recv, first_count);
}

// hardware 64-bit atomicMin on slots preset to the maximum (a comparison point)
template <bool kWarp>
__global__ void __launch_bounds__(kGenThreads) combine_native_min_kernel(const uint32_t* __restrict__ dst,
                                                                          const unsigned long long* __restrict__ msgs,
                                                                          uint64_t k, uint32_t n,
                                                                          uint32_t* __restrict__ flag,
                                                                          unsigned long long* __restrict__ mail,
                                                                          GenCounters* __restrict__ gc) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < k; base += stride) {
        const uint64_t i = base + threadIdx.x;
        bool ok = i < k;
        uint32_t v = 0;
        unsigned long long m = 0;
        if (ok) {
            v = __ldcs(dst + i);
            m = msgs[i];
            if (v >= n) {
                atomicOr(&gc->status, kStatusInternal);
                ok = false;
            }
        }
        bool send = ok;
        if (kWarp) {
            const unsigned act = __ballot_sync(0xFFFFFFFFu, ok);
            if (ok) send = ipg_warp_combine<MinCombine<unsigned long long>>(act, v, &m);
        }
        if (send) {
            flag[v] = IPG_MAIL_FULL;  // idempotent
            atomicMin(&mail[v], m);
        }
    }
}

__global__ void preset_max_kernel(unsigned long long* __restrict__ mail, uint32_t n) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) mail[v] = ~0ull;
}

__global__ void fill_flags_kernel(uint32_t* __restrict__ flag, uint32_t n, uint32_t value) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) flag[v] = value;
}

__global__ void count_flags_kernel(const uint32_t* __restrict__ flag, uint32_t n, GenCounters* __restrict__ gc) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned int c = 0;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) c += flag[v] != 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&gc->recv, c);
}

template <class Combine, class Msg>
void launch_combine(bool warp, unsigned grid, cudaStream_t st, const uint32_t* dst, const void* msgs, uint64_t k,
                    uint32_t n, uint32_t* flag, void* mail, GenCounters* gc, unsigned spin_limit) {
    if (warp)
        combine_kernel<Combine, Msg, true><<<grid, kGenThreads, 0, st>>>(dst, static_cast<const Msg*>(msgs), k, n, flag,
                                                                         static_cast<Msg*>(mail), gc, spin_limit);
    else
        combine_kernel<Combine, Msg, false><<<grid, kGenThreads, 0, st>>>(dst, static_cast<const Msg*>(msgs), k, n,
                                                                          flag, static_cast<Msg*>(mail), gc, spin_limit);
}

// polls of a CLAIMED flag allowed under IPG_COMBINE_STALLED before a send gives up
constexpr unsigned kStalledSpinLimit = 64;

struct MinCount128 {
    __device__ LevelCount operator()(const LevelCount& a, const LevelCount& b) const {
        return PathsProgram::Combine{}(a, b);
    }
};

}  // namespace

void generic_free(ipg_graph* g) {
    GenWork* w = static_cast<GenWork*>(g->generic);
    if (!w) return;
    cudaFree(w->state);
    cudaFree(w->mail);
    cudaFree(w->flag);
    cudaFree(w->recv);
    cudaFree(w->gc);
    if (w->h_gc) cudaFreeHost(w->h_gc);
    delete w;
    g->generic = nullptr;
}

}  // namespace ipg

using namespace ipg;

extern "C" {

ipg_status ipg_sssp_tree_dev(ipg_graph* g, uint32_t source, uint32_t* dist_dev, uint32_t* parent_dev,
                             ipg_stats* stats, void* stream) {
    const char* name = "ipg_sssp_tree";
    if (g && g->n && (!dist_dev || !parent_dev)) {
        stats_begin(stats);
        return set_error(IPG_EINVAL, "%s: output is NULL", name);
    }
    cudaStream_t st = (cudaStream_t)stream;
    GenWork* w = nullptr;
    IPG_TRY(gen_run<TreeProgram>(g, source, stats, st, name, &w));
    DeviceGuard guard(g->device);
    tree_output_kernel<<<grid_for(g->n, (unsigned)sm_count_of(g->device) * 8), 256, 0, st>>>(
        static_cast<const unsigned long long*>(w->state), g->inv, g->n, dist_dev, parent_dev);
    IPG_CUDA(cudaGetLastError());
    IPG_CUDA(cudaStreamSynchronize(st));
    return IPG_OK;
}

ipg_status ipg_bfs_paths_dev(ipg_graph* g, uint32_t source, uint32_t* level_dev, uint64_t* paths_dev,
                             ipg_stats* stats, void* stream) {
    const char* name = "ipg_bfs_paths";
    if (g && g->n && (!level_dev || !paths_dev)) {
        stats_begin(stats);
        return set_error(IPG_EINVAL, "%s: output is NULL", name);
    }
    cudaStream_t st = (cudaStream_t)stream;
    GenWork* w = nullptr;
    IPG_TRY(gen_run<PathsProgram>(g, source, stats, st, name, &w));
    DeviceGuard guard(g->device);
    paths_output_kernel<<<grid_for(g->n, (unsigned)sm_count_of(g->device) * 8), 256, 0, st>>>(
        static_cast<const LevelCount*>(w->state), g->inv, g->n, level_dev,
        reinterpret_cast<unsigned long long*>(paths_dev));
    IPG_CUDA(cudaGetLastError());
    IPG_CUDA(cudaStreamSynchronize(st));
    return IPG_OK;
}

// host variants: results staged in one device buffer (4 + 8 bytes per vertex)
static ipg_status gen_host(ipg_graph* g, bool tree, uint32_t source, void* out_a, void* out_b, ipg_stats* stats) {
    const char* name = tree ? "ipg_sssp_tree" : "ipg_bfs_paths";
    if (!g) {
        stats_begin(stats);
        return set_error(IPG_EINVAL, "%s: graph is NULL", name);
    }
    if (g->n && (!out_a || !out_b)) {
        stats_begin(stats);
        return set_error(IPG_EINVAL, "%s: output is NULL", name);
    }
    DeviceGuard guard(g->device);
    const size_t n = g->n;
    const size_t a_bytes = (4 * (n ? n : 1) + 15) & ~size_t(15);  // b starts 16-byte aligned
    void* buf = nullptr;
    IPG_CUDA(cudaMallocAsync(&buf, a_bytes + 8 * (n ? n : 1), g->stream));
    uint32_t* a = static_cast<uint32_t*>(buf);
    void* b = static_cast<char*>(buf) + a_bytes;
    ipg_status rc;
    if (tree)
        rc = ipg_sssp_tree_dev(g, source, a, static_cast<uint32_t*>(b), stats, g->stream);
    else
        rc = ipg_bfs_paths_dev(g, source, a, static_cast<uint64_t*>(b), stats, g->stream);
    if (rc == IPG_OK && n) {
        if (cudaMemcpyAsync(out_a, a, 4 * n, cudaMemcpyDeviceToHost, g->stream) != cudaSuccess ||
            cudaMemcpyAsync(out_b, b, (tree ? 4 : 8) * n, cudaMemcpyDeviceToHost, g->stream) != cudaSuccess)
            rc = set_error(IPG_ECUDA, "%s: copy to host failed", name);
    }
    cudaFreeAsync(buf, g->stream);
    if (cudaStreamSynchronize(g->stream) != cudaSuccess && rc == IPG_OK)
        rc = set_error(IPG_ECUDA, "%s: stream synchronize failed", name);
    return rc;
}

ipg_status ipg_sssp_tree(ipg_graph* g, uint32_t source, uint32_t* dist_out, uint32_t* parent_out, ipg_stats* stats) {
    return gen_host(g, true, source, dist_out, parent_out, stats);
}

ipg_status ipg_bfs_paths(ipg_graph* g, uint32_t source, uint32_t* level_out, uint64_t* paths_out, ipg_stats* stats) {
    return gen_host(g, false, source, level_out, paths_out, stats);
}

ipg_status ipg_combine_dev(int kind, uint32_t n, const uint32_t* dst_dev, const void* msgs_dev, uint64_t k,
                           uint32_t* flags_dev, void* mail_dev, uint64_t* receivers_out, uint32_t options,
                           void* stream) {
    const char* name = "ipg_combine_dev";
    if (kind < IPG_COMBINE_XOR_U32 || kind > IPG_COMBINE_MINCOUNT_U128)
        return set_error(IPG_EINVAL, "%s: unknown kind %d", name, kind);
    if (options & ~(IPG_COMBINE_WARP | IPG_COMBINE_NATIVE | IPG_COMBINE_STALLED))
        return set_error(IPG_EINVAL, "%s: unknown option bits 0x%x", name, options);
    const bool native = options & IPG_COMBINE_NATIVE;
    const bool warp = options & IPG_COMBINE_WARP;
    const bool stalled = options & IPG_COMBINE_STALLED;
    if (native && kind != IPG_COMBINE_MIN_U64)
        return set_error(IPG_EINVAL, "%s: IPG_COMBINE_NATIVE applies to IPG_COMBINE_MIN_U64 only", name);
    if (native && stalled)
        return set_error(IPG_EINVAL, "%s: IPG_COMBINE_STALLED applies to the hybrid combiner only", name);
    const unsigned spin_limit = stalled ? kStalledSpinLimit : IPG_MAIL_SPIN_LIMIT;
    if (k && (!dst_dev || !msgs_dev)) return set_error(IPG_EINVAL, "%s: messages are NULL", name);
    if (n && (!flags_dev || !mail_dev)) return set_error(IPG_EINVAL, "%s: mailboxes are NULL", name);
    if (k && !n) return set_error(IPG_EINVAL, "%s: messages for an empty vertex set", name);
    if (kind == IPG_COMBINE_MINCOUNT_U128 &&
        ((reinterpret_cast<uintptr_t>(msgs_dev) | reinterpret_cast<uintptr_t>(mail_dev)) & 15))
        return set_error(IPG_EINVAL, "%s: 128-bit messages and mailboxes must be 16-byte aligned", name);
    const size_t size = kind == IPG_COMBINE_XOR_U32 ? 4 : kind == IPG_COMBINE_MINCOUNT_U128 ? 16 : 8;
    if (((reinterpret_cast<uintptr_t>(msgs_dev) | reinterpret_cast<uintptr_t>(mail_dev)) & (size - 1)))
        return set_error(IPG_EINVAL, "%s: messages and mailboxes must be aligned to their size", name);
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    IPG_CUDA(cudaGetDevice(&dev));
    const unsigned sms = (unsigned)sm_count_of(dev);
    GenCounters* gc = nullptr;
    IPG_CUDA(cudaMallocAsync(&gc, sizeof(GenCounters), st));
    ipg_status rc = IPG_OK;
    GenCounters h{};
    do {
        if (cudaMemsetAsync(gc, 0, sizeof(GenCounters), st) != cudaSuccess ||
            (n && !stalled && cudaMemsetAsync(flags_dev, 0, sizeof(uint32_t) * n, st) != cudaSuccess)) {
            rc = set_error(IPG_ECUDA, "%s: memset failed", name);
            break;
        }
        if (n && stalled) {  // every mailbox held by a first sender that never publishes
            fill_flags_kernel<<<grid_for(n, sms * 8), 256, 0, st>>>(flags_dev, n, IPG_MAIL_CLAIMED);
            if (cudaGetLastError() != cudaSuccess) {
                rc = set_error(IPG_ECUDA, "%s: kernel launch failed", name);
                break;
            }
        }
        const unsigned grid = grid_for(k, sms * 8);
        if (k) {
            if (native) {
                preset_max_kernel<<<grid_for(n, sms * 8), 256, 0, st>>>(static_cast<unsigned long long*>(mail_dev), n);
                if (warp)
                    combine_native_min_kernel<true><<<grid, kGenThreads, 0, st>>>(
                        dst_dev, static_cast<const unsigned long long*>(msgs_dev), k, n, flags_dev,
                        static_cast<unsigned long long*>(mail_dev), gc);
                else
                    combine_native_min_kernel<false><<<grid, kGenThreads, 0, st>>>(
                        dst_dev, static_cast<const unsigned long long*>(msgs_dev), k, n, flags_dev,
                        static_cast<unsigned long long*>(mail_dev), gc);
                count_flags_kernel<<<grid_for(n, sms * 8), 256, 0, st>>>(flags_dev, n, gc);
            } else if (kind == IPG_COMBINE_XOR_U32) {
                launch_combine<XorCombine<unsigned int>, unsigned int>(warp, grid, st, dst_dev, msgs_dev, k, n,
                                                                       flags_dev, mail_dev, gc, spin_limit);
            } else if (kind == IPG_COMBINE_MIN_U64) {
                launch_combine<MinCombine<unsigned long long>, unsigned long long>(warp, grid, st, dst_dev, msgs_dev,
                                                                                   k, n, flags_dev, mail_dev, gc,
                                                                                   spin_limit);
            } else if (kind == IPG_COMBINE_SUM_U64) {
                launch_combine<SumCombine<unsigned long long>, unsigned long long>(warp, grid, st, dst_dev, msgs_dev,
                                                                                   k, n, flags_dev, mail_dev, gc,
                                                                                   spin_limit);
            } else {
                launch_combine<MinCount128, LevelCount>(warp, grid, st, dst_dev, msgs_dev, k, n, flags_dev, mail_dev,
                                                        gc, spin_limit);
            }
            if (cudaGetLastError() != cudaSuccess) {
                rc = set_error(IPG_ECUDA, "%s: kernel launch failed", name);
                break;
            }
        }
        if (cudaMemcpyAsync(&h, gc, sizeof(GenCounters), cudaMemcpyDeviceToHost, st) != cudaSuccess) {
            rc = set_error(IPG_ECUDA, "%s: counter copy failed", name);
            break;
        }
    } while (0);
    cudaFreeAsync(gc, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == IPG_OK)
        rc = set_error(IPG_ECUDA, "%s: stream synchronize failed", name);
    if (rc != IPG_OK) return rc;
    if (h.status & kStatusInternal) return set_error(IPG_EINVAL, "%s: a destination is >= n = %u", name, n);
    if (h.status & IPG_MAIL_STATUS_TIMEOUT)
        return set_error(IPG_ETIMEOUT, "%s: a bounded wait in the message combiner ran out", name);
    if (receivers_out) *receivers_out = h.recv;
    return IPG_OK;
}

}  // extern "C"
