// Graph object: device copy of the CSR, validation, the in-edge (CSC) copy for
// pull-based supersteps, error reporting and small shared helpers.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "ipg_internal.cuh"

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

ipg_status ensure_csc(ipg_graph* g, cudaStream_t st) {
    if (g->csc_ready) return IPG_OK;
    if (!g->directed) {
        g->csc_off = g->off;
        g->csc_src = g->col;
        g->csc_owned = false;
        g->csc_ready = true;
        return IPG_OK;
    }
    const uint32_t n = g->n;
    const uint64_t m = g->m;
    const int sms = device_sms(g->device);
    unsigned long long* indeg = nullptr;
    uint32_t* src_in = nullptr;
    uint32_t* keys_out = nullptr;
    void* temp = nullptr;
    size_t temp_bytes = 0, scan_bytes = 0;
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
        g->csc_owned = true;
        CSC_CUDA(cudaMalloc(&indeg, sizeof(unsigned long long) * ((size_t)n + 1)));
        CSC_CUDA(cudaMemsetAsync(indeg, 0, sizeof(unsigned long long) * ((size_t)n + 1), st));
        if (m) {
            count_in_degree_kernel<<<grid_for(m, sms, 16), 256, 0, st>>>(g->col, m, indeg);
            CSC_CUDA(cudaGetLastError());
        }
        CSC_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, indeg, (unsigned long long*)g->csc_off,
                                               (long long)n + 1, st));
        if (m) {
            int bits = 1;
            while (bits < 32 && (1ull << bits) < (uint64_t)n) ++bits;
            CSC_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, temp_bytes, (const uint32_t*)nullptr, (uint32_t*)nullptr,
                                                     (const uint32_t*)nullptr, (uint32_t*)nullptr, (long long)m, 0,
                                                     bits, st));
        }
        if (scan_bytes > temp_bytes) temp_bytes = scan_bytes;
        CSC_CUDA(cudaMalloc(&temp, temp_bytes ? temp_bytes : 16));
        CSC_CUDA(cub::DeviceScan::ExclusiveSum(temp, scan_bytes, indeg, (unsigned long long*)g->csc_off,
                                               (long long)n + 1, st));
        if (m) {
            CSC_CUDA(cudaMalloc(&src_in, sizeof(uint32_t) * m));
            CSC_CUDA(cudaMalloc(&keys_out, sizeof(uint32_t) * m));
            expand_sources_kernel<<<grid_for((uint64_t)n * 32, sms, 16), 256, 0, st>>>(g->off, n, src_in);
            CSC_CUDA(cudaGetLastError());
            int bits = 1;
            while (bits < 32 && (1ull << bits) < (uint64_t)n) ++bits;
            size_t tb = temp_bytes;
            CSC_CUDA(cub::DeviceRadixSort::SortPairs(temp, tb, (const uint32_t*)g->col, keys_out,
                                                     (const uint32_t*)src_in, g->csc_src, (long long)m, 0, bits,
                                                     st));
        }
        CSC_CUDA(cudaStreamSynchronize(st));
        g->csc_ready = true;
    }
done:
#undef CSC_CUDA
    if (indeg) cudaFree(indeg);
    if (src_in) cudaFree(src_in);
    if (keys_out) cudaFree(keys_out);
    if (temp) cudaFree(temp);
    if (rc != IPG_OK) {
        if (g->csc_off) cudaFree(g->csc_off);
        if (g->csc_src) cudaFree(g->csc_src);
        g->csc_off = nullptr;
        g->csc_src = nullptr;
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

// ---------------------------------------------------------------------------
// creation

static void free_graph(ipg_graph* g) {
    if (!g) return;
    DeviceGuard guard(g->device);
    auto f = [](void* p) {
        if (p) cudaFree(p);
    };
    if (g->csc_owned) {
        f(g->csc_off);
        f(g->csc_src);
    }
    f(g->off);
    f(g->col);
    f(g->w);
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
        cudaStream_t st = from_device ? user_stream : g->stream;
        cudaMemcpyKind kind = from_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        CR(cudaMemsetAsync(g->counters, 0, sizeof(PushCounters), st));
        CR(cudaMemcpyAsync(g->off, offsets, sizeof(uint64_t) * ((size_t)n + 1), kind, st));
        if (m) CR(cudaMemcpyAsync(g->col, columns, sizeof(uint32_t) * m, kind, st));
        if (weights && m) CR(cudaMemcpyAsync(g->w, weights, sizeof(uint32_t) * m, kind, st));
        int sms = device_sms(g->device);
        validate_offsets_kernel<<<grid_for((uint64_t)n + 1, sms), 256, 0, st>>>(g->off, n, m, &g->counters->status);
        CR(cudaGetLastError());
        if (m) {
            validate_columns_kernel<<<grid_for(m, sms, 16), 256, 0, st>>>(g->col, m, n, &g->counters->status);
            CR(cudaGetLastError());
        }
        CR(cudaMemcpyAsync(g->h_counters, g->counters, sizeof(PushCounters), cudaMemcpyDeviceToHost, st));
        CR(cudaStreamSynchronize(st));
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
        if (!g->directed) {
            g->csc_off = g->off;
            g->csc_src = g->col;
            g->csc_ready = true;
        }
    } while (0);
    if (rc != IPG_OK) {
        free_graph(g);
        return rc;
    }
    *out = g;
    return IPG_OK;
}

}  // namespace ipg

using namespace ipg;

extern "C" {

ipg_status ipg_graph_create(const uint64_t* offsets, const uint32_t* columns, const uint32_t* weights, uint32_t n,
                            uint64_t m, int directed, ipg_graph** out) {
    return create_impl(offsets, columns, weights, n, m, directed, nullptr, false, out);
}

ipg_status ipg_graph_create_dev(const uint64_t* offsets_dev, const uint32_t* columns_dev, const uint32_t* weights_dev,
                                uint32_t n, uint64_t m, int directed, void* stream, ipg_graph** out) {
    return create_impl(offsets_dev, columns_dev, weights_dev, n, m, directed, (cudaStream_t)stream, true, out);
}

void ipg_graph_destroy(ipg_graph* g) { free_graph(g); }

ipg_status ipg_graph_info(const ipg_graph* g, uint32_t* n, uint64_t* m, int* directed, int* weighted) {
    if (!g) return set_error(IPG_EINVAL, "ipg_graph_info: graph is NULL");
    if (n) *n = g->n;
    if (m) *m = g->m;
    if (directed) *directed = g->directed;
    if (weighted) *weighted = g->weighted;
    return IPG_OK;
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
    }
    return "IPG_UNKNOWN";
}

int ipg_version(void) { return 100; }

}  // extern "C"
