// Graph object: device copy of the CSR, validation, the in-edge (CSC) copy for
// pull-based supersteps, error reporting and small shared helpers.
#include <stdarg.h>
#include <atomic>
#include <chrono>
#include <stdio.h>
#include <string.h>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "ipg_internal.cuh"
#include "ipg_mergepath.cuh"

namespace ipg {

static thread_local char g_err[512] = "";

ipg_status set_error(ipg_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

ipg_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    const char* base = strrchr(file, '/');
    set_error(e == cudaErrorMemoryAllocation ? IPG_ENOMEM : IPG_ECUDA, "%s failed: %s (%s:%d)", what,
              cudaGetErrorString(e), base ? base + 1 : file, line);
    return e == cudaErrorMemoryAllocation ? IPG_ENOMEM : IPG_ECUDA;
}

ipg_status ensure_buffer(void** p, size_t* cap, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (*p && *cap >= bytes) return IPG_OK;
    if (*p) {
        cudaFree(*p);
        *p = nullptr;
        *cap = 0;
    }
    IPG_CUDA(cudaMalloc(p, bytes));
    *cap = bytes;
    return IPG_OK;
}

ipg_status StepTimer::init() {
    for (auto& e : ev)
        if (!e) IPG_CUDA(cudaEventCreate(&e));
    return IPG_OK;
}

void StepTimer::destroy() {
    for (auto& e : ev)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
}

void stats_begin(ipg_stats* s) {
    if (s) s->count = 0;
}

void stats_put(ipg_stats* s, uint32_t idx, const ipg_superstep_stats& rec) {
    if (s && s->buf && idx < s->cap) s->buf[idx] = rec;
}

// ---------------------------------------------------------------------------
// validation

__global__ void validate_offsets_kernel(const uint64_t* __restrict__ off, uint32_t n, uint64_t m,
                                        unsigned int* status) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
        uint64_t a = off[v];
        bool bad = (v == 0 && a != 0) || (v == n && a != m) || (v < n && off[v + 1] < a);
        if (bad) atomicOr(status, kStatusBadCsr);
    }
}

__global__ void validate_columns_kernel(const uint32_t* __restrict__ col, uint64_t m, uint32_t n,
                                        unsigned int* status) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) bad |= col[e] >= n;
    if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStatusBadColumn);
}

static unsigned grid_for(uint64_t work, int sms, unsigned per_sm = 8) {
    uint64_t want = (work + 255) / 256;
    uint64_t cap = (uint64_t)(sms > 0 ? sms : 152) * per_sm;
    if (want < 1) want = 1;
    return (unsigned)(want < cap ? want : cap);
}

static int device_sms(int dev) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    return v;
}

// ---------------------------------------------------------------------------
// CSC (in-edges) built with a stable radix sort of (destination, source) pairs;
// since the CSR lists sources in increasing order, each vertex's in-edges come
// out sorted by source, so pull sums have a fixed order.

__global__ void expand_sources_kernel(const uint64_t* __restrict__ off, uint32_t n, uint32_t* __restrict__ src) {
    // one warp per row
    uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t lane = threadIdx.x & 31;
    uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t u = warp; u < n; u += nwarps) {
        uint64_t b = off[u], e = off[u + 1];
        for (uint64_t p = b + lane; p < e; p += 32) src[p] = (uint32_t)u;
    }
}

// key of out-edge e of row u: (destination << 32) | u; rows are in source order,
// so a stable sort on the destination bits leaves every in-edge list sorted by source
__global__ void csc_keys_kernel(const uint64_t* __restrict__ off, const uint32_t* __restrict__ col, uint32_t n,
                                unsigned long long* __restrict__ keys) {
    uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t lane = threadIdx.x & 31;
    uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t u = warp; u < n; u += nwarps) {
        uint64_t b = off[u], e = off[u + 1];
        for (uint64_t p = b + lane; p < e; p += 32) keys[p] = ((unsigned long long)col[p] << 32) | u;
    }
}

// CSC offsets from the destinations of the sorted in-edges: entry i starts every
// row after the previous entry's destination up to its own, and the last entry
// also closes the rows after it (offset m).  dst(i) = key(i) >> shift.  A gap of
// up to kGapDirect rows is written by its thread; a longer one goes to a list
// that csc_gap_fill_kernel writes in parallel (at most n / kGapDirect + 1 gaps).
constexpr uint64_t kGapDirect = 256;

struct CscGap {
    unsigned long long first, last, value;  // rows [first, last] start at entry `value`
};

__device__ __forceinline__ void csc_gap(uint64_t first, uint64_t last, uint64_t value, uint64_t* __restrict__ csc_off,
                                        CscGap* __restrict__ gaps, unsigned int* __restrict__ ngaps) {
    if (first > last) return;
    if (last - first < kGapDirect) {
        for (uint64_t r = first; r <= last; ++r) csc_off[r] = value;
    } else {
        gaps[atomicAdd(ngaps, 1u)] = CscGap{first, last, value};
    }
}

template <typename K>
__global__ void csc_offsets_kernel(const K* __restrict__ keys, int shift, uint64_t m, uint32_t n,
                                   uint64_t* __restrict__ csc_off, uint32_t* __restrict__ src_out,
                                   CscGap* __restrict__ gaps, unsigned int* __restrict__ ngaps) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const K k = keys[i];
        const uint64_t v = (uint64_t)(k >> shift);
        const uint64_t vp = i ? (uint64_t)(keys[i - 1] >> shift) + 1 : 0;
        if (vp <= v) csc_gap(vp, v, i, csc_off, gaps, ngaps);
        if (i == m - 1) csc_gap(v + 1, n, m, csc_off, gaps, ngaps);
        if (src_out) src_out[i] = (uint32_t)k;  // 64-bit keys: the source in the low word
    }
}

__global__ void csc_gap_fill_kernel(const CscGap* __restrict__ gaps, const unsigned int* __restrict__ ngaps,
                                    uint64_t* __restrict__ csc_off) {
    const unsigned int count = *ngaps;
    for (unsigned int q = blockIdx.x; q < count; q += gridDim.x) {
        const CscGap gp = gaps[q];
        for (uint64_t r = gp.first + threadIdx.x; r <= gp.last; r += blockDim.x) csc_off[r] = gp.value;
    }
}

__global__ void count_in_degree_kernel(const uint32_t* __restrict__ col, uint64_t m,
                                       unsigned long long* __restrict__ indeg) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride)
        atomicAdd(&indeg[col[e]], 1ull);
}

__global__ void count_nonempty_kernel(const uint64_t* __restrict__ off, uint32_t n, unsigned long long* out) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long c = 0;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) c += off[v + 1] > off[v];
    for (int s = 16; s > 0; s >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, s);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// In-edge copy (CSC) of a directed graph, built on the device: a stable radix
// sort of the out-edges by destination.  Unweighted: (destination, source) pairs
// of 32-bit words.  Weighted: 64-bit keys (destination << 32 | source), sorted on
// the destination bits only, carrying the weight as the value, so sources and
// weights come out in place without a gather.  The offsets follow from the sorted
// destinations in the same pass that unpacks the sources.
ipg_status ensure_csc(ipg_graph* g, cudaStream_t st) {
    if (g->csc_ready) return IPG_OK;
    if (!g->directed) {
        g->csc_off = g->off;
        g->csc_src = g->col;
        g->csc_w8 = g->w8;
        g->csc_w = g->w;
        g->csc_owned = false;
        g->csc_ready = true;
        return IPG_OK;
    }
    const bool weighted = g->w8 || g->w;
    const uint32_t n = g->n;
    const uint64_t m = g->m;
    const int sms = device_sms(g->device);
    uint32_t* src_in = nullptr;
    uint32_t* keys_out = nullptr;
    unsigned long long* wkeys_in = nullptr;
    unsigned long long* wkeys_out = nullptr;
    void* temp = nullptr;
    size_t temp_bytes = 0;
    CscGap* gaps = nullptr;
    unsigned int* ngaps = nullptr;
    ipg_status rc = IPG_OK;
    cudaError_t e;
#define CSC_CUDA(call)                                             \
    do {                                                           \
        e = (call);                                                \
        if (e != cudaSuccess) {                                    \
            rc = cuda_fail(e, #call, __FILE__, __LINE__);          \
            goto done;                                             \
        }                                                          \
    } while (0)
    {
        CSC_CUDA(cudaMalloc(&g->csc_off, sizeof(uint64_t) * ((size_t)n + 1)));
        CSC_CUDA(cudaMalloc(&g->csc_src, sizeof(uint32_t) * (m ? m : 1)));
        if (g->w8) CSC_CUDA(cudaMalloc(&g->csc_w8, m ? m : 1));
        if (g->w) CSC_CUDA(cudaMalloc(&g->csc_w, sizeof(uint32_t) * (m ? m : 1)));
        g->csc_owned = true;
        if (!m) {
            CSC_CUDA(cudaMemsetAsync(g->csc_off, 0, sizeof(uint64_t) * ((size_t)n + 1), st));
        } else {
            int bits = 1;
            while (bits < 32 && (1ull << bits) < (uint64_t)n) ++bits;
            const unsigned grid = grid_for(m, sms, 16);
            const size_t max_gaps = (size_t)n / kGapDirect + 2;
            CSC_CUDA(cudaMalloc(&gaps, sizeof(CscGap) * max_gaps));
            CSC_CUDA(cudaMalloc(&ngaps, sizeof(unsigned int)));
            CSC_CUDA(cudaMemsetAsync(ngaps, 0, sizeof(unsigned int), st));
            if (!weighted) {
                CSC_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, temp_bytes, (const uint32_t*)nullptr,
                                                         (uint32_t*)nullptr, (const uint32_t*)nullptr,
                                                         (uint32_t*)nullptr, (long long)m, 0, bits, st));
                CSC_CUDA(cudaMalloc(&temp, temp_bytes ? temp_bytes : 16));
                CSC_CUDA(cudaMalloc(&src_in, sizeof(uint32_t) * m));
                CSC_CUDA(cudaMalloc(&keys_out, sizeof(uint32_t) * m));
                expand_sources_kernel<<<grid_for((uint64_t)n * 32, sms, 16), 256, 0, st>>>(g->off, n, src_in);
                CSC_CUDA(cudaGetLastError());
                CSC_CUDA(cub::DeviceRadixSort::SortPairs(temp, temp_bytes, (const uint32_t*)g->col, keys_out,
                                                         (const uint32_t*)src_in, g->csc_src, (long long)m, 0, bits,
                                                         st));
                csc_offsets_kernel<uint32_t><<<grid, 256, 0, st>>>(keys_out, 0, m, n, g->csc_off, nullptr, gaps,
                                                                   ngaps);
            } else {
                CSC_CUDA(cudaMalloc(&wkeys_in, sizeof(unsigned long long) * m));
                CSC_CUDA(cudaMalloc(&wkeys_out, sizeof(unsigned long long) * m));
                csc_keys_kernel<<<grid_for((uint64_t)n * 32, sms, 16), 256, 0, st>>>(g->off, g->col, n, wkeys_in);
                CSC_CUDA(cudaGetLastError());
                if (g->w8) {
                    CSC_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, temp_bytes, (const unsigned long long*)nullptr,
                                                             (unsigned long long*)nullptr, (const uint8_t*)nullptr,
                                                             (uint8_t*)nullptr, (long long)m, 32, 32 + bits, st));
                    CSC_CUDA(cudaMalloc(&temp, temp_bytes ? temp_bytes : 16));
                    CSC_CUDA(cub::DeviceRadixSort::SortPairs(temp, temp_bytes, (const unsigned long long*)wkeys_in,
                                                             wkeys_out, (const uint8_t*)g->w8, g->csc_w8, (long long)m,
                                                             32, 32 + bits, st));
                } else {
                    CSC_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, temp_bytes, (const unsigned long long*)nullptr,
                                                             (unsigned long long*)nullptr, (const uint32_t*)nullptr,
                                                             (uint32_t*)nullptr, (long long)m, 32, 32 + bits, st));
                    CSC_CUDA(cudaMalloc(&temp, temp_bytes ? temp_bytes : 16));
                    CSC_CUDA(cub::DeviceRadixSort::SortPairs(temp, temp_bytes, (const unsigned long long*)wkeys_in,
                                                             wkeys_out, (const uint32_t*)g->w, g->csc_w, (long long)m,
                                                             32, 32 + bits, st));
                }
                csc_offsets_kernel<unsigned long long><<<grid, 256, 0, st>>>(wkeys_out, 32, m, n, g->csc_off,
                                                                              g->csc_src, gaps, ngaps);
            }
            csc_gap_fill_kernel<<<(unsigned)sms * 4, 256, 0, st>>>(gaps, ngaps, g->csc_off);
            CSC_CUDA(cudaGetLastError());
        }
        CSC_CUDA(cudaStreamSynchronize(st));
        g->csc_ready = true;
    }
done:
#undef CSC_CUDA
    if (src_in) cudaFree(src_in);
    if (keys_out) cudaFree(keys_out);
    if (wkeys_in) cudaFree(wkeys_in);
    if (wkeys_out) cudaFree(wkeys_out);
    if (temp) cudaFree(temp);
    if (gaps) cudaFree(gaps);
    if (ngaps) cudaFree(ngaps);
    if (rc != IPG_OK) {
        if (g->csc_off) cudaFree(g->csc_off);
        if (g->csc_src) cudaFree(g->csc_src);
        if (g->csc_w8) cudaFree(g->csc_w8);
        if (g->csc_w) cudaFree(g->csc_w);
        g->csc_off = nullptr;
        g->csc_src = nullptr;
        g->csc_w8 = nullptr;
        g->csc_w = nullptr;
        g->csc_owned = false;
    }
    return rc;
}

ipg_status count_in_nonempty(ipg_graph* g, cudaStream_t st) {
    if (g->in_nonempty >= 0) return IPG_OK;
    IPG_TRY(ensure_csc(g, st));
    IPG_CUDA(cudaMemsetAsync(&g->counters->receivers, 0, sizeof(unsigned long long), st));
    if (g->n) {
        count_nonempty_kernel<<<grid_for(g->n, device_sms(g->device)), 256, 0, st>>>(g->csc_off, g->n,
                                                                                    &g->counters->receivers);
        IPG_CUDA(cudaGetLastError());
    }
    IPG_CUDA(cudaMemcpyAsync(&g->h_counters->receivers, &g->counters->receivers, sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, st));
    IPG_CUDA(cudaStreamSynchronize(st));
    g->in_nonempty = (long long)g->h_counters->receivers;
    return IPG_OK;
}

ipg_status ensure_pull_partition(ipg_graph* g, cudaStream_t st) {
    if (g->pr_tile_row) return IPG_OK;
    IPG_TRY(ensure_csc(g, st));
    const uint64_t tiles = mp_tile_count(g->n, g->m);
    IPG_CUDA(cudaMalloc(&g->pr_tile_row, sizeof(uint32_t) * (tiles + 1)));
    IPG_CUDA(cudaMalloc(&g->pr_head, sizeof(float) * (tiles ? tiles : 1)));
    IPG_CUDA(cudaMalloc(&g->pr_tail, sizeof(float) * (tiles ? tiles : 1)));
    IPG_TRY(mp_partition(g->csc_off, g->n, g->m, tiles, g->pr_tile_row, st));
    g->pr_tiles = tiles;
    return IPG_OK;
}

// ---------------------------------------------------------------------------
// Degree-ordered relabelling (done once, when the graph is created).  Random
// accesses in every superstep land on the values of hub vertices; numbering the
// vertices by decreasing total degree packs those values into few cache lines and
// keeps them in L2.  The permutation is invisible to callers: sources are mapped
// in, outputs are mapped back, and Hashmin labels stay the caller's ids.

__global__ void degree_key_kernel(const uint64_t* __restrict__ off, const unsigned long long* __restrict__ indeg,
                                  uint32_t n, uint32_t* __restrict__ key, uint32_t* __restrict__ ids) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        unsigned long long d = (off[v + 1] - off[v]) + (indeg ? indeg[v] : 0ull);
        key[v] = ~(uint32_t)(d < 0xFFFFFFFFull ? d : 0xFFFFFFFFull);  // ascending sort = descending degree
        ids[v] = (uint32_t)v;
    }
}

__global__ void invert_kernel(const uint32_t* __restrict__ perm, uint32_t n, uint32_t* __restrict__ inv,
                              const uint64_t* __restrict__ off, unsigned long long* __restrict__ new_deg) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        const uint32_t o = perm[x];
        inv[o] = (uint32_t)x;
        new_deg[x] = off[o + 1] - off[o];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) new_deg[n] = 0;
}

__global__ void max_degree_kernel(const uint64_t* __restrict__ off, uint32_t n, unsigned long long* out) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long mx = 0;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        mx = max(mx, (unsigned long long)(off[v + 1] - off[v]));
    for (int s = 16; s > 0; s >>= 1) mx = max(mx, __shfl_down_sync(0xFFFFFFFFu, mx, s));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

__global__ void max_weight_kernel(const uint32_t* __restrict__ w, uint64_t m, unsigned int* out) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned mx = 0;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) mx = max(mx, w[e]);
    for (int s = 16; s > 0; s >>= 1) mx = max(mx, __shfl_down_sync(0xFFFFFFFFu, mx, s));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

// one warp per new row: copy the old row, renaming its columns
__global__ void rename_rows_kernel(const uint64_t* __restrict__ off, const uint32_t* __restrict__ col,
                                   const uint32_t* __restrict__ w, const uint32_t* __restrict__ perm,
                                   const uint32_t* __restrict__ inv, const uint64_t* __restrict__ new_off, uint32_t n,
                                   uint32_t* __restrict__ new_col, uint32_t* __restrict__ new_w,
                                   uint8_t* __restrict__ new_w8) {
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t x = warp; x < n; x += nwarps) {
        const uint32_t o = perm[x];
        const uint64_t b = off[o], len = off[o + 1] - b, nb = new_off[x];
        for (uint64_t k = lane; k < len; k += 32) {
            new_col[nb + k] = inv[col[b + k]];
            if (new_w) new_w[nb + k] = w[b + k];
            if (new_w8) new_w8[nb + k] = (uint8_t)w[b + k];
        }
    }
}

static ipg_status relabel(ipg_graph* g, cudaStream_t st) {
    const uint32_t n = g->n;
    const uint64_t m = g->m;
    if (n == 0) return IPG_OK;
    const int sms = device_sms(g->device);
    unsigned long long* indeg = nullptr;
    unsigned long long* new_deg = nullptr;
    uint32_t *key = nullptr, *key_out = nullptr, *ids = nullptr;
    uint64_t* new_off = nullptr;
    uint32_t* new_col = nullptr;
    uint32_t* new_w = nullptr;
    uint8_t* new_w8 = nullptr;
    void* temp = nullptr;
    size_t tb = 0, tb2 = 0;
    ipg_status rc = IPG_OK;
    cudaError_t e;
    unsigned wmax = 0;
#define RL(call)                                          \
    do {                                                  \
        e = (call);                                       \
        if (e != cudaSuccess) {                           \
            rc = cuda_fail(e, #call, __FILE__, __LINE__); \
            goto done;                                    \
        }                                                 \
    } while (0)
    RL(cudaMalloc(&g->perm, sizeof(uint32_t) * n));
    RL(cudaMalloc(&g->inv, sizeof(uint32_t) * n));
    RL(cudaMalloc(&key, sizeof(uint32_t) * n));
    RL(cudaMalloc(&key_out, sizeof(uint32_t) * n));
    RL(cudaMalloc(&ids, sizeof(uint32_t) * n));
    RL(cudaMalloc(&new_deg, sizeof(unsigned long long) * ((size_t)n + 1)));
    RL(cudaMalloc(&new_off, sizeof(uint64_t) * ((size_t)n + 1)));
    if (g->directed && m) {
        RL(cudaMalloc(&indeg, sizeof(unsigned long long) * ((size_t)n + 1)));
        RL(cudaMemsetAsync(indeg, 0, sizeof(unsigned long long) * ((size_t)n + 1), st));
        count_in_degree_kernel<<<grid_for(m, sms, 16), 256, 0, st>>>(g->col, m, indeg);
        RL(cudaGetLastError());
    }
    degree_key_kernel<<<grid_for(n, sms), 256, 0, st>>>(g->off, indeg, n, key, ids);
    RL(cudaGetLastError());
    RL(cub::DeviceRadixSort::SortPairs(nullptr, tb, (const uint32_t*)key, key_out, (const uint32_t*)ids, g->perm,
                                       (long long)n, 0, 32, st));
    RL(cub::DeviceScan::ExclusiveSum(nullptr, tb2, new_deg, (unsigned long long*)new_off, (long long)n + 1, st));
    if (tb2 > tb) tb = tb2;
    RL(cudaMalloc(&temp, tb ? tb : 16));
    tb2 = tb;
    RL(cub::DeviceRadixSort::SortPairs(temp, tb2, (const uint32_t*)key, key_out, (const uint32_t*)ids, g->perm,
                                       (long long)n, 0, 32, st));
    invert_kernel<<<grid_for(n, sms), 256, 0, st>>>(g->perm, n, g->inv, g->off, new_deg);
    RL(cudaGetLastError());
    tb2 = tb;
    RL(cub::DeviceScan::ExclusiveSum(temp, tb2, new_deg, (unsigned long long*)new_off, (long long)n + 1, st));
    if (g->w && m) {
        RL(cudaMemsetAsync(&g->counters->status, 0, sizeof(unsigned), st));
        max_weight_kernel<<<grid_for(m, sms, 16), 256, 0, st>>>(g->w, m, &g->counters->status);
        RL(cudaGetLastError());
        RL(cudaMemcpyAsync(&g->h_counters->status, &g->counters->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        RL(cudaStreamSynchronize(st));
        wmax = g->h_counters->status;
        RL(cudaMemsetAsync(&g->counters->status, 0, sizeof(unsigned), st));
    }
    RL(cudaMalloc(&new_col, sizeof(uint32_t) * (m ? m : 1)));
    if (g->w) {
        if (wmax <= 255)
            RL(cudaMalloc(&new_w8, m ? m : 1));
        else
            RL(cudaMalloc(&new_w, sizeof(uint32_t) * (m ? m : 1)));
    }
    if (m) {
        rename_rows_kernel<<<grid_for((uint64_t)n * 32, sms, 16), 256, 0, st>>>(g->off, g->col, g->w, g->perm, g->inv,
                                                                                new_off, n, new_col, new_w, new_w8);
        RL(cudaGetLastError());
    }
    RL(cudaMemsetAsync(&g->counters->receivers, 0, sizeof(unsigned long long), st));
    max_degree_kernel<<<grid_for(n, sms), 256, 0, st>>>(g->off, n, &g->counters->receivers);
    RL(cudaGetLastError());
    RL(cudaMemcpyAsync(&g->h_counters->receivers, &g->counters->receivers, sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, st));
    RL(cudaStreamSynchronize(st));
    g->max_outdeg = g->h_counters->receivers;
    cudaFree(g->off);
    cudaFree(g->col);
    if (g->w) cudaFree(g->w);
    g->off = new_off;
    g->col = new_col;
    g->w = new_w;
    g->w8 = new_w8;
    new_off = nullptr;
    new_col = nullptr;
    new_w = nullptr;
    new_w8 = nullptr;
done:
#undef RL
    if (indeg) cudaFree(indeg);
    if (new_deg) cudaFree(new_deg);
    if (key) cudaFree(key);
    if (key_out) cudaFree(key_out);
    if (ids) cudaFree(ids);
    if (temp) cudaFree(temp);
    if (new_off) cudaFree(new_off);
    if (new_col) cudaFree(new_col);
    if (new_w) cudaFree(new_w);
    if (new_w8) cudaFree(new_w8);
    return rc;
}

int sm_count_of(int dev) { return device_sms(dev); }

int sm_count_current() {
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return device_sms(0);
    if (dev >= kMaxDev) return device_sms(dev);
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v <= 0) {
        v = device_sms(dev);
        cache[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

__global__ void map_ids_kernel(const uint32_t* __restrict__ inv, uint32_t* __restrict__ ids, uint32_t k) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) ids[i] = inv[ids[i]];
}

ipg_status map_to_internal(ipg_graph* g, uint32_t* ids, uint32_t k, cudaStream_t st) {
    if (!k) return IPG_OK;
    map_ids_kernel<<<(k + 255) / 256, 256, 0, st>>>(g->inv, ids, k);
    IPG_CUDA(cudaGetLastError());
    return IPG_OK;
}

Tuning& tuning() {
    static Tuning t;
    return t;
}

long long pull_divisor_for(const ipg_graph* g, bool sssp) {
    if (sssp ? g->tuned.sssp : g->tuned.cc) return sssp ? g->tuned.sssp_divisor : g->tuned.cc_divisor;
    return tuning().pull_divisor;
}
long long pr_engine_for(const ipg_graph* g) { return g->tuned.pr ? g->tuned.pr_engine : tuning().pr_engine; }
long long pr_carveout_for(const ipg_graph* g) { return g->tuned.pr ? g->tuned.pr_carveout : tuning().pr_carveout; }
long long batch_divisor_for(const ipg_graph* g) {
    return g->tuned.batch ? g->tuned.batch_divisor : tuning().batch_divisor;
}

long long batch_chunk_for(const ipg_graph* g) { return g->tuned.batch ? g->tuned.batch_chunk : tuning().batch_chunk; }

// ---------------------------------------------------------------------------
// creation

// frees the per-algorithm workspace, keeping the graph (CSR, CSC, numbering)
void release_workspace(ipg_graph* g) {
    DeviceGuard guard(g->device);
    if (g->stream) cudaStreamSynchronize(g->stream);
    auto f = [](auto*& p) {
        if (p) cudaFree(p);
        p = nullptr;
    };
    if (g->pr_exec) cudaGraphExecDestroy(g->pr_exec);  // it refers to the buffers below
    g->pr_exec = nullptr;
    for (auto& x : g->push_exec) {  // so do the superstep loop graphs
        if (x) cudaGraphExecDestroy(x);
        x = nullptr;
    }
    f(g->inv_outdeg);
    f(g->pr_box[0]);
    f(g->pr_box[1]);
    f(g->pr_rank);
    f(g->pr_out_stage);
    g->pr_out_stage_cap = 0;
    f(g->stamp);
    f(g->rstamp);
    f(g->frontier[0]);
    f(g->frontier[1]);
    f(g->fr_prefix);
    f(g->fr_rowstart);
    f(g->fr_val);
    f(g->block_sums);
    g->block_sums_cap = 0;
    f(g->push_tile_row);
    g->push_tile_cap = 0;
    f(g->val_stage);
    f(g->val);
    f(g->sval);
    f(g->sbits);
    batch_free(g);
    generic_free(g);
}

static void free_graph(ipg_graph* g) {
    if (!g) return;
    DeviceGuard guard(g->device);
    auto f = [](void* p) {
        if (p) cudaFree(p);
    };
    if (g->csc_owned) {
        f(g->csc_off);
        f(g->csc_src);
        f(g->csc_w8);
        f(g->csc_w);
    }
    f(g->off);
    f(g->col);
    f(g->w);
    f(g->w8);
    f(g->perm);
    f(g->inv);
    f(g->val);
    f(g->sval);
    f(g->sbits);
    f(g->pr_rank);
    f(g->inv_outdeg);
    f(g->pr_box[0]);
    f(g->pr_box[1]);
    f(g->pr_tile_row);
    f(g->pr_head);
    f(g->pr_tail);
    f(g->pr_out_stage);
    f(g->stamp);
    f(g->rstamp);
    f(g->frontier[0]);
    f(g->frontier[1]);
    f(g->fr_prefix);
    f(g->fr_rowstart);
    f(g->fr_val);
    f(g->block_sums);
    f(g->push_tile_row);
    f(g->val_stage);
    f(g->counters);
    f(g->inst_base);
    f(g->inst_msgs);
    f(g->inst_steps);
    delete[] g->inst_base_host;
    if (g->pr_exec) cudaGraphExecDestroy(g->pr_exec);
    for (auto& x : g->push_exec)
        if (x) cudaGraphExecDestroy(x);
    f(g->loop);
    f(g->loop_rec);
    if (g->h_loop) cudaFreeHost(g->h_loop);
    batch_free(g);
    generic_free(g);
    if (g->h_counters) cudaFreeHost(g->h_counters);
    g->timer.destroy();
    if (g->stream) cudaStreamDestroy(g->stream);
    delete g;
}

static ipg_status create_impl(const uint64_t* offsets, const uint32_t* columns, const uint32_t* weights, uint32_t n,
                              uint64_t m, int directed, cudaStream_t user_stream, bool from_device, ipg_graph** out) {
    if (!out) return set_error(IPG_EINVAL, "ipg_graph_create: out is NULL");
    *out = nullptr;
    if (!offsets) return set_error(IPG_EINVAL, "ipg_graph_create: offsets is NULL");
    if (m && !columns) return set_error(IPG_EINVAL, "ipg_graph_create: columns is NULL with m > 0");
    if (m > 0xFFFFFFFF00000000ull) return set_error(IPG_EINVAL, "ipg_graph_create: m too large");
    ipg_graph* g = new (std::nothrow) ipg_graph();
    if (!g) return set_error(IPG_ENOMEM, "ipg_graph_create: host allocation failed");
    ipg_status rc = IPG_OK;
    using clk = std::chrono::steady_clock;
    const auto t_begin = clk::now();
    auto ms_since = [](clk::time_point a) { return std::chrono::duration<float, std::milli>(clk::now() - a).count(); };
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    do {
        if (cudaGetDevice(&g->device) != cudaSuccess) {
            rc = set_error(IPG_ECUDA, "ipg_graph_create: no CUDA device");
            break;
        }
        g->n = n;
        g->m = m;
        g->directed = directed ? 1 : 0;
        g->weighted = weights ? 1 : 0;
        cudaError_t e;
#define CR(call)                                               \
    if ((e = (call)) != cudaSuccess) {                         \
        rc = cuda_fail(e, #call, __FILE__, __LINE__);          \
        break;                                                 \
    }
        CR(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
        CR(cudaMalloc(&g->counters, sizeof(PushCounters)));
        CR(cudaHostAlloc(&g->h_counters, sizeof(PushCounters), cudaHostAllocDefault));
        CR(cudaMalloc(&g->off, sizeof(uint64_t) * ((size_t)n + 1)));
        CR(cudaMalloc(&g->col, sizeof(uint32_t) * (m ? m : 1)));
        if (weights) CR(cudaMalloc(&g->w, sizeof(uint32_t) * (m ? m : 1)));
        for (auto& x : ev) CR(cudaEventCreate(&x));
        g->create_profile.alloc_ms = ms_since(t_begin);
        cudaStream_t st = from_device ? user_stream : g->stream;
        cudaMemcpyKind kind = from_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        CR(cudaMemsetAsync(g->counters, 0, sizeof(PushCounters), st));
        const auto t_copy = clk::now();
        CR(cudaEventRecord(ev[0], st));
        CR(cudaMemcpyAsync(g->off, offsets, sizeof(uint64_t) * ((size_t)n + 1), kind, st));
        if (m) CR(cudaMemcpyAsync(g->col, columns, sizeof(uint32_t) * m, kind, st));
        if (weights && m) CR(cudaMemcpyAsync(g->w, weights, sizeof(uint32_t) * m, kind, st));
        CR(cudaEventRecord(ev[1], st));
        g->create_profile.upload_issue_ms = ms_since(t_copy);
        int sms = device_sms(g->device);
        validate_offsets_kernel<<<grid_for((uint64_t)n + 1, sms), 256, 0, st>>>(g->off, n, m, &g->counters->status);
        CR(cudaGetLastError());
        if (m) {
            validate_columns_kernel<<<grid_for(m, sms, 16), 256, 0, st>>>(g->col, m, n, &g->counters->status);
            CR(cudaGetLastError());
        }
        CR(cudaEventRecord(ev[2], st));
        CR(cudaMemcpyAsync(g->h_counters, g->counters, sizeof(PushCounters), cudaMemcpyDeviceToHost, st));
        CR(cudaStreamSynchronize(st));
        CR(cudaEventElapsedTime(&g->create_profile.upload_ms, ev[0], ev[1]));
        CR(cudaEventElapsedTime(&g->create_profile.validate_ms, ev[1], ev[2]));
#undef CR
        unsigned status = g->h_counters->status;
        if (status & kStatusBadCsr) {
            rc = set_error(IPG_EINVAL,
                           "ipg_graph_create: malformed offsets (need offsets[0]=0, non-decreasing, offsets[n]=m)");
            break;
        }
        if (status & kStatusBadColumn) {
            rc = set_error(IPG_EINVAL, "ipg_graph_create: a column index is >= n");
            break;
        }
        const auto t_relabel = clk::now();
        rc = relabel(g, st);
        if (rc != IPG_OK) break;
        g->create_profile.renumber_ms = ms_since(t_relabel);
        g->create_profile.total_ms = ms_since(t_begin);
        if (!g->directed) {
            g->csc_off = g->off;
            g->csc_src = g->col;
            g->csc_w8 = g->w8;
            g->csc_w = g->w;
            g->csc_ready = true;
        }
    } while (0);
    for (auto& x : ev)
        if (x) cudaEventDestroy(x);
    if (rc != IPG_OK) {
        free_graph(g);
        return rc;
    }
    *out = g;
    return IPG_OK;
}

ipg_status create_graph(const uint64_t* offsets, const uint32_t* columns, const uint32_t* weights, uint32_t n,
                        uint64_t m, int directed, cudaStream_t user_stream, bool from_device, ipg_graph** out) {
    return create_impl(offsets, columns, weights, n, m, directed, user_stream, from_device, out);
}

// ---------------------------------------------------------------------------
// Symmetry check: does the stored edge multiset, weights included, equal its
// reverse?  Both lists are sorted into (key, weight) order and compared entry by
// entry.  Keys are (u << 32 | v) for the forward list and (v << 32 | u) for the
// reverse one, built from the internal (renumbered) CSR: renumbering maps both
// endpoints through one bijection, so it changes no answer.

__global__ void sym_keys_kernel(const uint64_t* __restrict__ off, const uint32_t* __restrict__ col, uint32_t n,
                                unsigned long long* __restrict__ fwd, unsigned long long* __restrict__ rev) {
    // one warp per row
    uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t lane = threadIdx.x & 31;
    uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t u = warp; u < n; u += nwarps) {
        uint64_t b = off[u], e = off[u + 1];
        for (uint64_t p = b + lane; p < e; p += 32) {
            const unsigned long long v = col[p];
            fwd[p] = ((unsigned long long)u << 32) | v;
            rev[p] = (v << 32) | u;
        }
    }
}

__global__ void sym_widen_kernel(const uint8_t* __restrict__ w8, uint64_t m, uint32_t* __restrict__ w) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) w[i] = w8[i];
}

__global__ void sym_compare_kernel(const unsigned long long* __restrict__ a, const unsigned long long* __restrict__ b,
                                   const uint32_t* __restrict__ wa, const uint32_t* __restrict__ wb, uint64_t m,
                                   unsigned int* __restrict__ differ) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
        bad |= a[i] != b[i] || (wa && wa[i] != wb[i]);
    if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) atomicOr(differ, 1u);
}

ipg_status check_symmetric(const ipg_graph* g, int* symmetric, cudaStream_t st) {
    using ull = unsigned long long;
    const uint64_t m = g->m;
    const uint32_t n = g->n;
    *symmetric = 1;
    if (m == 0) return IPG_OK;
    const bool weighted = g->w8 || g->w;
    const int sms = device_sms(g->device);
    int bits = 1;
    while (bits < 32 && (1ull << bits) < (uint64_t)n) ++bits;
    const int key_bits = 32 + bits;       // keys are (hi << 32 | lo) with hi, lo < 2^bits
    const int w_bits = g->w8 ? 8 : 32;
    const unsigned grid = grid_for(m, sms, 16);
    ull *fwd = nullptr, *rev = nullptr, *tmp = nullptr;
    uint32_t *w = nullptr, *w2 = nullptr, *wf = nullptr;
    unsigned int* differ = nullptr;
    unsigned int h_differ = 0;
    void* temp = nullptr;
    size_t temp_bytes = 0, tb = 0;
    ipg_status rc = IPG_OK;
    cudaError_t e = cudaSuccess;
#define SYM_CUDA(call)                                             \
    do {                                                           \
        e = (call);                                                \
        if (e != cudaSuccess) {                                    \
            rc = cuda_fail(e, #call, __FILE__, __LINE__);          \
            goto done;                                             \
        }                                                          \
    } while (0)
    {
        SYM_CUDA(cudaMalloc(&fwd, sizeof(ull) * m));
        SYM_CUDA(cudaMalloc(&rev, sizeof(ull) * m));
        SYM_CUDA(cudaMalloc(&tmp, sizeof(ull) * m));
        SYM_CUDA(cudaMalloc(&differ, sizeof(unsigned int)));
        SYM_CUDA(cudaMemsetAsync(differ, 0, sizeof(unsigned int), st));
        sym_keys_kernel<<<grid_for((uint64_t)n * 32, sms, 16), 256, 0, st>>>(g->off, g->col, n, fwd, rev);
        SYM_CUDA(cudaGetLastError());
        if (!weighted) {
            SYM_CUDA(cub::DeviceRadixSort::SortKeys(nullptr, temp_bytes, (const ull*)nullptr, (ull*)nullptr,
                                                    (long long)m, 0, key_bits, st));
            SYM_CUDA(cudaMalloc(&temp, temp_bytes ? temp_bytes : 16));
            SYM_CUDA(cub::DeviceRadixSort::SortKeys(temp, temp_bytes, (const ull*)fwd, tmp, (long long)m, 0, key_bits,
                                                    st));  // tmp: forward, sorted
            SYM_CUDA(cub::DeviceRadixSort::SortKeys(temp, temp_bytes, (const ull*)rev, fwd, (long long)m, 0, key_bits,
                                                    st));  // fwd: reverse, sorted
            sym_compare_kernel<<<grid, 256, 0, st>>>(tmp, fwd, nullptr, nullptr, m, differ);
            SYM_CUDA(cudaGetLastError());
        } else {
            SYM_CUDA(cudaMalloc(&w, sizeof(uint32_t) * m));
            SYM_CUDA(cudaMalloc(&w2, sizeof(uint32_t) * m));
            SYM_CUDA(cudaMalloc(&wf, sizeof(uint32_t) * m));
            if (g->w8) {
                sym_widen_kernel<<<grid, 256, 0, st>>>(g->w8, m, w);
                SYM_CUDA(cudaGetLastError());
            } else {
                SYM_CUDA(cudaMemcpyAsync(w, g->w, sizeof(uint32_t) * m, cudaMemcpyDeviceToDevice, st));
            }
            SYM_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, (const uint32_t*)nullptr, (uint32_t*)nullptr,
                                                     (const ull*)nullptr, (ull*)nullptr, (long long)m, 0, w_bits, st));
            temp_bytes = tb;
            SYM_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, (const ull*)nullptr, (ull*)nullptr,
                                                     (const uint32_t*)nullptr, (uint32_t*)nullptr, (long long)m, 0,
                                                     key_bits, st));
            if (tb > temp_bytes) temp_bytes = tb;
            SYM_CUDA(cudaMalloc(&temp, temp_bytes ? temp_bytes : 16));
            // each list: by weight, then stably by key, which leaves it in (key, weight) order
            SYM_CUDA(cub::DeviceRadixSort::SortPairs(temp, temp_bytes, (const uint32_t*)w, w2, (const ull*)fwd, tmp,
                                                     (long long)m, 0, w_bits, st));
            SYM_CUDA(cub::DeviceRadixSort::SortPairs(temp, temp_bytes, (const ull*)tmp, fwd, (const uint32_t*)w2, wf,
                                                     (long long)m, 0, key_bits, st));  // (fwd, wf): forward
            SYM_CUDA(cub::DeviceRadixSort::SortPairs(temp, temp_bytes, (const uint32_t*)w, w2, (const ull*)rev, tmp,
                                                     (long long)m, 0, w_bits, st));
            SYM_CUDA(cub::DeviceRadixSort::SortPairs(temp, temp_bytes, (const ull*)tmp, rev, (const uint32_t*)w2, w,
                                                     (long long)m, 0, key_bits, st));  // (rev, w): reverse
            sym_compare_kernel<<<grid, 256, 0, st>>>(fwd, rev, wf, w, m, differ);
            SYM_CUDA(cudaGetLastError());
        }
        SYM_CUDA(cudaMemcpyAsync(&h_differ, differ, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
        SYM_CUDA(cudaStreamSynchronize(st));
        *symmetric = h_differ ? 0 : 1;
    }
done:
#undef SYM_CUDA
    if (fwd) cudaFree(fwd);
    if (rev) cudaFree(rev);
    if (tmp) cudaFree(tmp);
    if (w) cudaFree(w);
    if (w2) cudaFree(w2);
    if (wf) cudaFree(wf);
    if (differ) cudaFree(differ);
    if (temp) cudaFree(temp);
    if (rc != IPG_OK && e == cudaErrorMemoryAllocation)
        return set_error(IPG_ENOMEM, "ipg_graph_check_symmetric: temporary device memory (about %d bytes per edge) "
                                     "could not be allocated", weighted ? 48 : 32);
    return rc;
}

}  // namespace ipg

using namespace ipg;

extern "C" {

ipg_status ipg_graph_create_batch(uint32_t count, const uint64_t* const* offsets, const uint32_t* const* columns,
                                  const uint32_t* const* weights, const uint32_t* n, const uint64_t* m, int directed,
                                  ipg_graph** out) {
    if (!out) return set_error(IPG_EINVAL, "ipg_graph_create_batch: out is NULL");
    *out = nullptr;
    if (count == 0 || !offsets || !n || !m) return set_error(IPG_EINVAL, "ipg_graph_create_batch: empty batch or NULL");
    uint64_t N = 0, M = 0;
    bool any_w = false, all_w = true;
    for (uint32_t i = 0; i < count; ++i) {
        if (!offsets[i]) return set_error(IPG_EINVAL, "ipg_graph_create_batch: offsets[%u] is NULL", i);
        if (m[i] && (!columns || !columns[i]))
            return set_error(IPG_EINVAL, "ipg_graph_create_batch: columns[%u] is NULL", i);
        if (offsets[i][0] != 0 || offsets[i][n[i]] != m[i])
            return set_error(IPG_EINVAL, "ipg_graph_create_batch: instance %u: offsets[0] must be 0 and offsets[n] = m", i);
        const bool w = weights && weights[i];
        any_w |= w;
        all_w &= w;
        N += n[i];
        M += m[i];
    }
    if (any_w && !all_w) return set_error(IPG_EINVAL, "ipg_graph_create_batch: weights for some instances only");
    if (N > 0xFFFFFFFFull) return set_error(IPG_EINVAL, "ipg_graph_create_batch: more than 2^32 - 1 vertices in total");
    uint64_t* off = nullptr;
    uint32_t* col = nullptr;
    uint32_t* w = nullptr;
    uint32_t* bases = new (std::nothrow) uint32_t[count + 1];
    if (cudaMallocHost(&off, sizeof(uint64_t) * (N + 1)) != cudaSuccess ||
        cudaMallocHost(&col, sizeof(uint32_t) * (M ? M : 1)) != cudaSuccess ||
        (any_w && cudaMallocHost(&w, sizeof(uint32_t) * (M ? M : 1)) != cudaSuccess) || !bases) {
        if (off) cudaFreeHost(off);
        if (col) cudaFreeHost(col);
        if (w) cudaFreeHost(w);
        delete[] bases;
        return set_error(IPG_ENOMEM, "ipg_graph_create_batch: pinned staging allocation failed");
    }
    // the disjoint union: instance i's vertex v is vertex base_i + v, its edges follow
    uint64_t vb = 0, eb = 0;
    for (uint32_t i = 0; i < count; ++i) {
        bases[i] = (uint32_t)vb;
        for (uint32_t v = 0; v < n[i]; ++v) off[vb + v] = eb + offsets[i][v];
        for (uint64_t e = 0; e < m[i]; ++e) {
            const uint32_t c = columns[i][e];
            if (c >= n[i]) {  // would silently land in another instance
                cudaFreeHost(off);
                cudaFreeHost(col);
                if (w) cudaFreeHost(w);
                delete[] bases;
                return set_error(IPG_EINVAL, "ipg_graph_create_batch: instance %u has a column >= its n", i);
            }
            col[eb + e] = (uint32_t)vb + c;
        }
        if (any_w && m[i]) memcpy(w + eb, weights[i], sizeof(uint32_t) * m[i]);
        vb += n[i];
        eb += m[i];
    }
    off[N] = M;
    bases[count] = (uint32_t)N;
    ipg_graph* g = nullptr;
    ipg_status rc = create_graph(off, col, any_w ? w : nullptr, (uint32_t)N, M, directed, nullptr, false, &g);
    cudaFreeHost(off);
    cudaFreeHost(col);
    if (w) cudaFreeHost(w);
    if (rc != IPG_OK) {
        delete[] bases;
        return rc;
    }
    g->instances = count;
    g->inst_base_host = bases;
    if (cudaMalloc(&g->inst_base, sizeof(uint32_t) * (count + 1)) != cudaSuccess ||
        cudaMalloc(&g->inst_msgs, sizeof(unsigned long long) * count) != cudaSuccess ||
        cudaMemcpy(g->inst_base, bases, sizeof(uint32_t) * (count + 1), cudaMemcpyHostToDevice) != cudaSuccess) {
        free_graph(g);
        return set_error(IPG_ENOMEM, "ipg_graph_create_batch: instance table allocation failed");
    }
    *out = g;
    return IPG_OK;
}

ipg_status ipg_graph_instances(const ipg_graph* g, uint32_t* count, uint32_t* bases) {
    if (!g) return set_error(IPG_EINVAL, "ipg_graph_instances: graph is NULL");
    const uint32_t c = g->instances ? g->instances : 1;
    if (count) *count = c;
    if (bases) {
        if (g->instances)
            memcpy(bases, g->inst_base_host, sizeof(uint32_t) * (c + 1));
        else {
            bases[0] = 0;
            bases[1] = g->n;
        }
    }
    return IPG_OK;
}

ipg_status ipg_graph_create(const uint64_t* offsets, const uint32_t* columns, const uint32_t* weights, uint32_t n,
                            uint64_t m, int directed, ipg_graph** out) {
    return create_impl(offsets, columns, weights, n, m, directed, nullptr, false, out);
}

ipg_status ipg_graph_create_dev(const uint64_t* offsets_dev, const uint32_t* columns_dev, const uint32_t* weights_dev,
                                uint32_t n, uint64_t m, int directed, void* stream, ipg_graph** out) {
    return create_impl(offsets_dev, columns_dev, weights_dev, n, m, directed, (cudaStream_t)stream, true, out);
}

void ipg_graph_destroy(ipg_graph* g) { free_graph(g); }

ipg_status ipg_graph_create_profile(const ipg_graph* g, ipg_create_profile* out) {
    if (!g || !out) return set_error(IPG_EINVAL, "ipg_graph_create_profile: NULL argument");
    *out = g->create_profile;
    return IPG_OK;
}

ipg_status ipg_graph_info(const ipg_graph* g, uint32_t* n, uint64_t* m, int* directed, int* weighted) {
    if (!g) return set_error(IPG_EINVAL, "ipg_graph_info: graph is NULL");
    if (n) *n = g->n;
    if (m) *m = g->m;
    if (directed) *directed = g->directed;
    if (weighted) *weighted = g->weighted;
    return IPG_OK;
}

ipg_status ipg_graph_check_symmetric(const ipg_graph* g, int* symmetric, void* stream) {
    if (!g) return set_error(IPG_EINVAL, "ipg_graph_check_symmetric: graph is NULL");
    if (!symmetric) return set_error(IPG_EINVAL, "ipg_graph_check_symmetric: symmetric is NULL");
    DeviceGuard guard(g->device);
    if (!guard.ok) return set_error(IPG_ECUDA, "ipg_graph_check_symmetric: cannot select the graph's device");
    return check_symmetric(g, symmetric, static_cast<cudaStream_t>(stream));
}

const char* ipg_last_error(void) { return g_err; }

const char* ipg_status_string(ipg_status s) {
    switch (s) {
        case IPG_OK: return "IPG_OK";
        case IPG_EINVAL: return "IPG_EINVAL";
        case IPG_ENOMEM: return "IPG_ENOMEM";
        case IPG_ECUDA: return "IPG_ECUDA";
        case IPG_ETIMEOUT: return "IPG_ETIMEOUT";
        case IPG_EDEVICE: return "IPG_EDEVICE";
        case IPG_ENOTSUP: return "IPG_ENOTSUP";
        case IPG_EOVERFLOW: return "IPG_EOVERFLOW";
        case IPG_ECANCELED: return "IPG_ECANCELED";
    }
    return "IPG_UNKNOWN";
}

int ipg_version(void) { return 100; }

ipg_status ipg_set_tuning(const char* name, int64_t value) {
    if (!name) return set_error(IPG_EINVAL, "ipg_set_tuning: name is NULL");
    if (!strcmp(name, "pull_divisor")) {
        if (value < 0) return set_error(IPG_EINVAL, "ipg_set_tuning: pull_divisor must be >= 0");
        tuning().pull_divisor = value;
        return IPG_OK;
    }
    if (!strcmp(name, "combine_warp")) {
        if (value != 0 && value != 1) return set_error(IPG_EINVAL, "ipg_set_tuning: combine_warp must be 0 or 1");
        tuning().combine_warp = value;
        return IPG_OK;
    }
    if (!strcmp(name, "push_loop")) {
        if (value != 0 && value != 1) return set_error(IPG_EINVAL, "ipg_set_tuning: push_loop must be 0 or 1");
        tuning().push_loop = value;
        return IPG_OK;
    }
    if (!strcmp(name, "batch_divisor")) {
        if (value < 0) return set_error(IPG_EINVAL, "ipg_set_tuning: batch_divisor must be >= 0");
        tuning().batch_divisor = value;
        return IPG_OK;
    }
    if (!strcmp(name, "pr_engine")) {
        if (value != 0 && value != 1) return set_error(IPG_EINVAL, "ipg_set_tuning: pr_engine must be 0 or 1");
        tuning().pr_engine = value;
        return IPG_OK;
    }
    if (!strcmp(name, "pr_threads")) {
        if (value != 256 && value != 512) return set_error(IPG_EINVAL, "ipg_set_tuning: pr_threads must be 256 or 512");
        tuning().pr_threads = value;
        return IPG_OK;
    }
    if (!strcmp(name, "pr_carveout")) {
        if (value < -1 || value > 100) return set_error(IPG_EINVAL, "ipg_set_tuning: pr_carveout must be in [-1, 100]");
        tuning().pr_carveout = value;
        return IPG_OK;
    }
    if (!strcmp(name, "pull_filter")) {
        if (value < 0 || value > 100) return set_error(IPG_EINVAL, "ipg_set_tuning: pull_filter must be in [0, 100]");
        tuning().pull_filter = value;
        return IPG_OK;
    }
    if (!strcmp(name, "batch_chunk")) {
        if (value < 32 || value > 65536 || value % 32)
            return set_error(IPG_EINVAL, "ipg_set_tuning: batch_chunk must be a multiple of 32 in [32, 65536]");
        tuning().batch_chunk = value;
        return IPG_OK;
    }
    if (!strcmp(name, "batch_loop")) {
        if (value != 0 && value != 1) return set_error(IPG_EINVAL, "ipg_set_tuning: batch_loop must be 0 or 1");
        tuning().batch_loop = value;
        return IPG_OK;
    }
    if (!strcmp(name, "batch_wide_chunk")) {
        if (value < 32 || value > 65536 || value % 32)
            return set_error(IPG_EINVAL, "ipg_set_tuning: batch_wide_chunk must be a multiple of 32 in [32, 65536]");
        tuning().batch_wide_chunk = value;
        return IPG_OK;
    }
    if (!strcmp(name, "batch_tile_tasks")) {
        if (value < 0 || value > 64) return set_error(IPG_EINVAL, "ipg_set_tuning: batch_tile_tasks must be in [0, 64]");
        tuning().batch_tile_tasks = value;
        return IPG_OK;
    }
    return set_error(IPG_EINVAL, "ipg_set_tuning: unknown knob '%s'", name);
}

ipg_status ipg_get_tuning(const char* name, int64_t* value) {
    if (!name || !value) return set_error(IPG_EINVAL, "ipg_get_tuning: NULL argument");
    if (!strcmp(name, "pull_divisor")) {
        *value = tuning().pull_divisor;
        return IPG_OK;
    }
    if (!strcmp(name, "combine_warp")) {
        *value = tuning().combine_warp;
        return IPG_OK;
    }
    if (!strcmp(name, "push_loop")) {
        *value = tuning().push_loop;
        return IPG_OK;
    }
    if (!strcmp(name, "batch_divisor")) {
        *value = tuning().batch_divisor;
        return IPG_OK;
    }
    if (!strcmp(name, "pr_engine")) {
        *value = tuning().pr_engine;
        return IPG_OK;
    }
    if (!strcmp(name, "pr_threads")) {
        *value = tuning().pr_threads;
        return IPG_OK;
    }
    if (!strcmp(name, "pr_carveout")) {
        *value = tuning().pr_carveout;
        return IPG_OK;
    }
    if (!strcmp(name, "pull_filter")) {
        *value = tuning().pull_filter;
        return IPG_OK;
    }
    if (!strcmp(name, "batch_chunk")) {
        *value = tuning().batch_chunk;
        return IPG_OK;
    }
    if (!strcmp(name, "batch_loop")) {
        *value = tuning().batch_loop;
        return IPG_OK;
    }
    if (!strcmp(name, "batch_wide_chunk")) {
        *value = tuning().batch_wide_chunk;
        return IPG_OK;
    }
    if (!strcmp(name, "batch_tile_tasks")) {
        *value = tuning().batch_tile_tasks;
        return IPG_OK;
    }
    return set_error(IPG_EINVAL, "ipg_get_tuning: unknown knob '%s'", name);
}

}  // extern "C"
