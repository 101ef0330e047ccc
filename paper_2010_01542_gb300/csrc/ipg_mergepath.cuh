// Merge-path tile engine for pull supersteps (in-edge reductions).
//
// The in-edge lists (CSC) are cut into tiles of kMpTile items along the merge
// path of row ends and edges (Merrill & Garland's merge-based split): every tile
// holds the same number of (rows + edges), so a vertex with a million in-edges is
// spread over many CTAs and a run of vertices without in-edges costs one item
// each — the paper's edge-centric workload proxy (Sec. V-A) made exact.
//
// One tile is processed by a CTA as:
//   1. stage   the tile's row ends (relative, clamped) and each edge's message
//              (a caller-supplied gather) into shared memory;
//   2. walk    each thread takes kItems consecutive merge items, sums (or mins)
//              the messages of every row that starts and ends in its slice and
//              keeps the partial of its first and last row;
//   3. scan    a segmented scan of the per-thread carries, in a fixed tree order,
//              gives each thread the carry-in for its first finished row;
//   4. emit    every row whose in-edges began in this tile is handed to the
//              caller's emit functor; a row that began in an earlier tile leaves
//              its partial in tile_head and is finished by the fix-up kernel,
//              which folds the tiles' partials in tile order.
// With a fixed combine order in every step, float sums are bit-reproducible.
#pragma once

#include "ipg_internal.cuh"

namespace ipg {

constexpr uint32_t kMpTile = 2048;

// number of row ends consumed at merge-path diagonal `diag`; row_end[i] = end offset of row i
__device__ __forceinline__ uint32_t mp_rows_before(const uint64_t* __restrict__ row_end, uint32_t nrows,
                                                   uint64_t nedges, uint64_t diag) {
    uint64_t lo = diag > nedges ? diag - nedges : 0;
    uint64_t hi = diag < nrows ? diag : nrows;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (row_end[mid] <= diag - mid - 1)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (uint32_t)lo;
}

__device__ __forceinline__ uint32_t mp_pad(uint32_t j) { return j + (j >> 5); }  // breaks 32-word strides

struct SumF32 {
    typedef float T;
    static __device__ __forceinline__ float identity() { return 0.f; }
    static __device__ __forceinline__ float combine(float a, float b) { return a + b; }
};

struct MinU32 {
    typedef uint32_t T;
    static __device__ __forceinline__ uint32_t identity() { return kInf; }
    static __device__ __forceinline__ uint32_t combine(uint32_t a, uint32_t b) { return a < b ? a : b; }
};

// Staging of one tile.  A tile has R row ends and E edges with R + E <= kTile,
// so the relative row ends (R + 1 words) and the padded messages (E + E/32
// words) share one buffer: end = buf, val = buf + R + 1.  Keeping the staging
// small leaves more of the SM's unified L1/shared array to the L1 cache, which
// holds the most gathered messages.
template <int kThreads, int kItems, typename T>
struct MpShared {
    static_assert(sizeof(T) == sizeof(uint32_t), "messages share the row-end buffer");
    static constexpr uint32_t kTile = kThreads * kItems;
    uint32_t buf[kTile + kTile / 32 + 2];
    T wsum[kThreads / 32];
    int wflag[kThreads / 32];
    unsigned long long first_start;
};

// Geometry of merge-path tile `tile`: rows [i0, i1) end in it, edges [j0, j0 + E) lie in it.
struct MpGeom {
    uint32_t i0, i1, R, E;
    uint64_t j0;
};

__device__ __forceinline__ MpGeom mp_geom(const uint32_t* __restrict__ tile_row, uint64_t tile, uint32_t n,
                                          uint64_t m) {
    const uint64_t total = (uint64_t)n + m;
    const uint64_t d0 = tile * kMpTile;
    const uint64_t d1 = d0 + kMpTile < total ? d0 + kMpTile : total;
    MpGeom g;
    g.i0 = tile_row[tile];
    g.i1 = tile_row[tile + 1];
    g.j0 = d0 - g.i0;
    g.R = g.i1 - g.i0;
    g.E = (uint32_t)((d1 - g.i1) - g.j0);
    return g;
}

// row end of row i0 + k relative to j0, clamped past the tile (E + 1 for the row
// after the last one)
__device__ __forceinline__ uint32_t mp_rel_end(const uint64_t* __restrict__ off, const MpGeom& g, uint32_t k,
                                               uint32_t n) {
    const uint32_t row = g.i0 + k;
    const uint64_t rel = row < n ? off[row + 1] - g.j0 : (uint64_t)g.E + 1;
    return rel < (uint64_t)g.E + 1 ? (uint32_t)rel : g.E + 1;
}

// Steps 3-4 for one thread of the tile: run is the partial of the thread's last
// (unfinished) row, first_row / first_val the first row that ended in the
// thread's slice (-1 if none) and its partial without carry-in; row0_earlier
// says that row 0 of the tile began in an earlier tile.  Contains one
// __syncthreads().
template <int kThreads, class Op, class Emit>
__device__ __forceinline__ void mp_scan_finish(typename Op::T run, int first_row, typename Op::T first_val,
                                               const MpGeom& g, bool row0_earlier, typename Op::T* wsum, int* wflag,
                                               uint64_t tile, typename Op::T* __restrict__ tile_head,
                                               typename Op::T* __restrict__ tile_tail, Emit& emit, int tid) {
    typedef typename Op::T T;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    // segmented inclusive scan of (row ended, partial): (f, v) then (g, w) -> (f|g, g ? w : v + w)
    T v = run;
    int f = first_row >= 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T vu = __shfl_up_sync(0xFFFFFFFFu, v, o);
        const int fu = __shfl_up_sync(0xFFFFFFFFu, f, o);
        if (lane >= o) {
            if (!f) v = Op::combine(vu, v);
            f |= fu;
        }
    }
    if (lane == 31) {
        wsum[warp] = v;
        wflag[warp] = f;
    }
    __syncthreads();
    T wc = Op::identity();
    for (int q = 0; q < warp; ++q) wc = wflag[q] ? wsum[q] : Op::combine(wc, wsum[q]);
    const T incl = f ? v : Op::combine(wc, v);
    T excl = __shfl_up_sync(0xFFFFFFFFu, incl, 1);
    if (lane == 0) excl = wc;
    if (tid == kThreads - 1) tile_tail[tile] = incl;  // partial of row i1 inside this tile
    // the slice's first finished row, with the carry-in
    if (first_row >= 0) {
        const T tot = Op::combine(excl, first_val);
        if (row0_earlier)
            tile_head[tile] = tot;  // row i0 began in an earlier tile
        else
            emit(g.i0 + (uint32_t)first_row, tot);
    }
}

// Steps 2-4 on a staged tile: end[0..R] (relative row ends), val[mp_pad(k)] for
// k < E, and first_start = offset of row i0, all visible to every thread.
// Contains one __syncthreads().
template <int kThreads, int kItems, class Op, class Emit>
__device__ __forceinline__ void mp_reduce(const uint32_t* end, const typename Op::T* val, const MpGeom& g,
                                          unsigned long long first_start, typename Op::T* wsum, int* wflag,
                                          uint64_t tile, typename Op::T* __restrict__ tile_head,
                                          typename Op::T* __restrict__ tile_tail, Emit& emit) {
    typedef typename Op::T T;
    static_assert(kThreads * kItems == (int)kMpTile, "tiles share one partition");
    const int tid = threadIdx.x;
    // walk this thread's slice once
    const uint32_t items = g.R + g.E;
    const uint32_t ds = min((uint32_t)tid * kItems, items);
    const uint32_t de = min(ds + kItems, items);
    uint32_t lo = ds > g.E ? ds - g.E : 0, hi = min(ds, g.R);
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (end[mid] <= ds - mid - 1)
            lo = mid + 1;
        else
            hi = mid;
    }
    uint32_t i = lo, j = ds - lo;
    uint32_t cur_end = end[i];
    T run = Op::identity(), first_val = Op::identity();
    int first_row = -1;
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        if (ds + q < de) {
            if (j < cur_end) {
                run = Op::combine(run, val[mp_pad(j)]);
                ++j;
            } else {
                if (first_row < 0) {
                    first_row = (int)i;
                    first_val = run;
                } else {
                    emit(g.i0 + i, run);
                }
                run = Op::identity();
                ++i;
                cur_end = end[i];
            }
        }
    }
    mp_scan_finish<kThreads, Op>(run, first_row, first_val, g, first_row == 0 && first_start < g.j0, wsum, wflag,
                                 tile, tile_head, tile_tail, emit, tid);
}

// Processes tile `tile` with plain staging.  gather.template stage<kThreads, kItems>
// (j0, E, tid, s_val) writes the message of edge j0 + k to s_val[mp_pad(k)] for
// k < E; emit(row, total) finishes a row.  Begins with a __syncthreads().
template <int kThreads, int kItems, class Op, class Gather, class Emit>
__device__ __forceinline__ void mp_tile(MpShared<kThreads, kItems, typename Op::T>& sh,
                                        const uint64_t* __restrict__ off, uint32_t n, uint64_t m,
                                        const uint32_t* __restrict__ tile_row, uint64_t tile,
                                        typename Op::T* __restrict__ tile_head,
                                        typename Op::T* __restrict__ tile_tail, Gather& gather, Emit& emit) {
    typedef typename Op::T T;
    const MpGeom g = mp_geom(tile_row, tile, n, m);
    const int tid = threadIdx.x;
    uint32_t* end = sh.buf;
    T* val = reinterpret_cast<T*>(sh.buf + g.R + 1);
    __syncthreads();  // shared memory of the previous tile is free
    for (uint32_t k = tid; k <= g.R; k += kThreads) end[k] = mp_rel_end(off, g, k, n);
    if (tid == 0) sh.first_start = g.i0 < n ? off[g.i0] : m;
    gather.template stage<kThreads, kItems>(g.j0, g.E, tid, val);
    __syncthreads();
    mp_reduce<kThreads, kItems, Op>(end, val, g, sh.first_start, sh.wsum, sh.wflag, tile, tile_head, tile_tail, emit);
}

// ---------------------------------------------------------------------------
// Direct variant: no message staging.  The tile's row ends are marked in a
// kMpTile-bit mask (row k of the tile ends at merge item rel_end(k) + k); each
// thread finds the rows before its slice by a popcount prefix of the mask and
// has msg.template fetch<kItems>() load the messages of its own kItems items
// straight into registers.  Walk, scan and combine order are those of the
// staged engine, so results are bit-identical to it.  Shared memory is under
// 1 KB per CTA, which leaves nearly all of the SM's unified L1/shared array to
// the L1 cache: the gathers of the most-connected senders hit there.
template <int kThreads, typename T>
struct MpDirectShared {
    uint32_t bits[kMpTile / 32];  // bit p: merge item p is a row end
    uint32_t pre[kMpTile / 32];   // exclusive prefix of the words' popcounts
    T wsum[kThreads / 32];
    int wflag[kThreads / 32];
};

template <int kThreads, typename T>
__device__ __forceinline__ void mp_direct_init(MpDirectShared<kThreads, T>& sh) {
    for (uint32_t w = threadIdx.x; w < kMpTile / 32; w += kThreads) sh.bits[w] = 0;
}

// msg.template fetch<kItems>(j0, emask, eidx, x): for every q with bit q of
// emask set, x[q] = message of edge j0 + eidx[q].  emask is 0 when the tile
// has no edges.  The mask must be zero on entry (mp_direct_init, and every call
// leaves it zeroed).  Contains four __syncthreads().
template <int kThreads, int kItems, class Op, class Msg, class Emit>
__device__ __forceinline__ void mp_tile_direct(MpDirectShared<kThreads, typename Op::T>& sh,
                                               const uint64_t* __restrict__ off, uint32_t n, uint64_t m,
                                               const uint32_t* __restrict__ tile_row, uint64_t tile,
                                               typename Op::T* __restrict__ tile_head,
                                               typename Op::T* __restrict__ tile_tail, const Msg& msg, Emit& emit) {
    typedef typename Op::T T;
    static_assert(kThreads * kItems == (int)kMpTile, "tiles share one partition");
    static_assert(32 % kItems == 0, "a thread's items lie in one mask word");
    const MpGeom g = mp_geom(tile_row, tile, n, m);
    const int tid = threadIdx.x;
    const uint32_t items = g.R + g.E;
    __syncthreads();  // the previous tile has read the mask and its warp partials
    for (uint32_t k = tid; k < g.R; k += kThreads) {
        const uint32_t p = (uint32_t)(__ldg(off + g.i0 + k + 1) - g.j0) + k;
        if (p < items) atomicOr(&sh.bits[p >> 5], 1u << (p & 31));
    }
    __syncthreads();
    if (tid < 32) {
        const uint32_t c0 = __popc(sh.bits[tid]), c1 = __popc(sh.bits[tid + 32]);
        uint32_t a = c0, b = c1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t ua = __shfl_up_sync(0xFFFFFFFFu, a, o);
            const uint32_t ub = __shfl_up_sync(0xFFFFFFFFu, b, o);
            if (tid >= o) {
                a += ua;
                b += ub;
            }
        }
        const uint32_t tot0 = __shfl_sync(0xFFFFFFFFu, a, 31);
        sh.pre[tid] = a - c0;
        sh.pre[tid + 32] = tot0 + b - c1;
    }
    __syncthreads();
    // this thread's slice [ds, ds + nval) of the tile's merge items
    const uint32_t ds = min((uint32_t)tid * kItems, items);
    const uint32_t nval = min(ds + kItems, items) - ds;
    uint32_t ends = 0, i = 0, j = 0;
    if (nval) {
        const uint32_t word = sh.bits[ds >> 5];
        const uint32_t sft = ds & 31;
        ends = (word >> sft) & ((1u << nval) - 1u);
        i = sh.pre[ds >> 5] + __popc(word & ((1u << sft) - 1u));
        j = ds - i;
    }
    uint32_t emask = 0, eidx[kItems];
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        eidx[q] = j + q - __popc(ends & ((1u << q) - 1u));
        if ((uint32_t)q < nval && !((ends >> q) & 1u)) emask |= 1u << q;
    }
    T x[kItems];
    if (g.E) msg.template fetch<kItems>(g.j0, emask, eidx, x);
    T run = Op::identity(), first_val = Op::identity();
    int first_row = -1;
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        if ((uint32_t)q < nval) {
            if ((ends >> q) & 1u) {
                if (first_row < 0) {
                    first_row = (int)i;
                    first_val = run;
                } else {
                    emit(g.i0 + i, run);
                }
                run = Op::identity();
                ++i;
            } else {
                run = Op::combine(run, x[q]);
            }
        }
    }
    const bool row0_earlier = first_row == 0 && __ldg(off + g.i0) < g.j0;
    mp_scan_finish<kThreads, Op>(run, first_row, first_val, g, row0_earlier, sh.wsum, sh.wflag, tile, tile_head,
                                 tile_tail, emit, tid);
    // every read of the mask happened before the scan's barrier
    for (uint32_t w = tid; w < kMpTile / 32; w += kThreads) sh.bits[w] = 0;
}

// Tile t's first row, if it began in an earlier tile and ends in t: returns the
// row and the first tile q0 holding its edges; the caller folds tile_tail[q0..t)
// and then tile_head[t], in that order.
__device__ __forceinline__ bool mp_fixup_span(const uint64_t* __restrict__ off, const uint32_t* __restrict__ tile_row,
                                              uint64_t t, uint32_t n, uint32_t* row, uint64_t* q0) {
    const uint32_t i0 = tile_row[t];
    if (i0 >= n || tile_row[t + 1] == i0) return false;  // no row ends in this tile
    const uint64_t j0 = t * kMpTile - i0;
    if (off[i0] >= j0) return false;  // began here: finished by the tile itself
    uint64_t q = t;
    while (q > 0 && tile_row[q] == i0) --q;  // first tile holding edges of row i0
    *row = i0;
    *q0 = q;
    return true;
}

// tile boundaries (tiles + 1 entries) of the merge path over a CSR/CSC
ipg_status mp_partition(const uint64_t* off, uint32_t n, uint64_t m, uint64_t tiles, uint32_t* tile_row,
                        cudaStream_t st);

inline uint64_t mp_tile_count(uint32_t n, uint64_t m) { return ((uint64_t)n + m + kMpTile - 1) / kMpTile; }

// Persistent grid for a pull kernel: the SM's unified L1/shared array is split
// with the smallest shared-memory carveout that still holds the most resident
// CTAs (carve < 0), or with carve percent, on every kernel of `kernels`; the
// grid is every resident CTA, at most `tiles`.  The L1 left over caches the
// gathered messages of the most-connected senders.
ipg_status pull_grid(const void* const* kernels, int nkernels, int threads, int device, uint64_t tiles, int carve,
                     unsigned* grid);

}  // namespace ipg
