// ipg_sssp_noalloc: SSSP for callers that must not allocate device memory.
//
// Who needs this: code that links this library into a process whose device memory
// is owned by someone else (a host framework's pooling allocator, a fixed budget
// carved out at start-up) and code on a latency-critical path, where a cudaMalloc
// or cudaFree would stall the whole device and may fail at the worst moment.  Such
// callers hold their graph in their own device buffers and cannot create an
// ipg_graph, because graph creation copies the graph and allocates a workspace.
//
// This entry point reads the caller's device CSR in place and keeps all of its
// working state (visited stamps, two frontier lists, the frontier values and a few
// counters) in one fixed array that lives in the library's own device image:
// about 16 MiB per GPU, held until the process exits.  With CUDA's lazy module
// loading (the default) the array is reserved when this file's device code is
// loaded onto a GPU, which the first call on that GPU triggers through its
// cudaGetSymbolAddress; every later call takes no device memory.  It therefore
// handles at most IPG_NOALLOC_MAX_VERTICES vertices and rejects larger graphs.
// It calls no cudaMalloc, cudaFree or other allocating routine.
//
// The kernels are a simpler variant of the push superstep in ipg_push.cu: one warp
// per frontier vertex instead of the merge-path split, with the same synchronous
// semantics (sender values snapshotted between supersteps, atomicMin combine,
// stamp-deduplicated frontier appends), so distances and superstep counts equal
// those of ipg_sssp.
#include <mutex>

#include "ipg_internal.cuh"

namespace ipg {
namespace {

constexpr uint32_t kNaMax = IPG_NOALLOC_MAX_VERTICES;

struct NaCounters {
    unsigned int next_size;
    unsigned int status;
    unsigned long long edges;
    unsigned int pad[12];
};

// layout: stamp[kNaMax] | frontier0[kNaMax] | frontier1[kNaMax] | fval[kNaMax] | counters
constexpr size_t kNaScratchBytes = (size_t)4 * kNaMax * sizeof(uint32_t) + sizeof(NaCounters);

static __device__ __align__(256) unsigned char g_na_scratch[kNaScratchBytes];

// Device addresses of g_na_scratch, one per device, looked up on the first call made
// with that device current.  In host code the symbol itself is only a host-side
// stand-in, so kernels are always given the looked-up address.
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mu;
unsigned char* g_na_ptr[kNaMaxDevices] = {};

ipg_status na_scratch(unsigned char** out) {
    int dev = -1;
    IPG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) return set_error(IPG_ENOTSUP, "ipg_sssp_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)", __FILE__, __LINE__);
        g_na_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_na_ptr[dev];
    return IPG_OK;
}

__global__ void na_validate(const uint64_t* __restrict__ off, const uint32_t* __restrict__ col, uint32_t n,
                            uint64_t m, NaCounters* __restrict__ c) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (uint64_t v = t0; v <= n; v += stride) {
        uint64_t a = off[v];
        if ((v == 0 && a != 0) || (v == n && a != m) || (v < n && off[v + 1] < a)) atomicOr(&c->status, kStatusBadCsr);
    }
    for (uint64_t e = t0; e < m; e += stride)
        if (col[e] >= n) atomicOr(&c->status, kStatusBadColumn);
}

__global__ void na_init(uint32_t* __restrict__ dist, uint32_t n, uint32_t source, uint32_t* __restrict__ frontier,
                        uint32_t* __restrict__ fval) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        dist[v] = v == source ? 0u : kInf;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        frontier[0] = source;
        fval[0] = 0;
    }
}

// one warp per frontier vertex; lanes walk its out-edges
template <bool kWeighted>
__global__ void na_relax(const uint64_t* __restrict__ off, const uint32_t* __restrict__ col,
                         const uint32_t* __restrict__ wt, uint32_t* __restrict__ dist, const uint32_t* __restrict__ F,
                         const uint32_t* __restrict__ fval, uint32_t f, uint32_t* __restrict__ stamp,
                         uint32_t* __restrict__ next, NaCounters* __restrict__ c, uint32_t tag) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp; i < f; i += nwarps) {
        const uint32_t u = F[i];
        const uint32_t du = fval[i];
        const uint64_t b = off[u], e = off[u + 1];
        if (lane == 0 && e > b) atomicAdd(&c->edges, (unsigned long long)(e - b));
        for (uint64_t p0 = b; p0 < e; p0 += 32) {
            const uint64_t p = p0 + lane;
            bool app = false;
            uint32_t v = 0;
            if (p < e) {
                v = col[p];
                unsigned long long d = (unsigned long long)du + (kWeighted ? wt[p] : 1u);
                if (d >= kInf) {
                    atomicOr(&c->status, kStatusOverflow);
                    d = kInf - 1;
                }
                const uint32_t cand = (uint32_t)d;
                if (cand < dist[v]) {
                    const uint32_t old = atomicMin(&dist[v], cand);
                    if (cand < old) app = atomicExch(&stamp[v], tag) != tag;
                }
            }
            const unsigned mask = __ballot_sync(0xFFFFFFFFu, app);
            if (mask) {
                const int leader = __ffs(mask) - 1;
                uint32_t pos = 0;
                if (lane == (uint32_t)leader) pos = atomicAdd(&c->next_size, (unsigned)__popc(mask));
                pos = __shfl_sync(0xFFFFFFFFu, pos, leader);
                if (app) next[pos + __popc(mask & ((1u << lane) - 1u))] = v;
            }
        }
    }
}

__global__ void na_snapshot(const uint32_t* __restrict__ dist, const uint32_t* __restrict__ F, uint32_t f,
                            uint32_t* __restrict__ fval) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < f; i += stride) fval[i] = dist[F[i]];
}

unsigned na_grid(uint64_t threads) {
    uint64_t b = (threads + 255) / 256;
    if (b < 1) b = 1;
    const uint64_t cap = (uint64_t)sm_count_current() * 8;
    return (unsigned)(b < cap ? b : cap);
}

}  // namespace
}  // namespace ipg

using namespace ipg;

extern "C" ipg_status ipg_sssp_noalloc(const uint64_t* offsets_dev, const uint32_t* columns_dev,
                                       const uint32_t* weights_dev, uint32_t n, uint64_t m, uint32_t source,
                                       uint32_t* dist_dev, uint32_t* supersteps_out, void* stream) {
    if (supersteps_out) *supersteps_out = 0;
    if (n > kNaMax)
        return set_error(IPG_EINVAL, "ipg_sssp_noalloc: n = %u exceeds the limit of %u vertices of its fixed scratch",
                         n, kNaMax);
    if (!offsets_dev || !dist_dev || (m && !columns_dev))
        return set_error(IPG_EINVAL, "ipg_sssp_noalloc: NULL device pointer");
    if (source >= n) return set_error(IPG_EINVAL, "ipg_sssp_noalloc: source %u >= n = %u", source, n);
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    IPG_TRY(na_scratch(&base));
    uint32_t* stamp = reinterpret_cast<uint32_t*>(base);
    uint32_t* fr[2] = {stamp + kNaMax, stamp + 2 * (size_t)kNaMax};
    uint32_t* fval = stamp + 3 * (size_t)kNaMax;
    NaCounters* ctr = reinterpret_cast<NaCounters*>(stamp + 4 * (size_t)kNaMax);

    // the scratch keeps the previous call's contents: clear what must start at zero
    IPG_CUDA(cudaMemsetAsync(ctr, 0, sizeof(NaCounters), st));
    IPG_CUDA(cudaMemsetAsync(stamp, 0, sizeof(uint32_t) * n, st));
    na_validate<<<na_grid(m > n ? m : (uint64_t)n + 1), 256, 0, st>>>(offsets_dev, columns_dev, n, m, ctr);
    IPG_CUDA(cudaGetLastError());
    NaCounters h;
    IPG_CUDA(cudaMemcpyAsync(&h, ctr, sizeof(h), cudaMemcpyDeviceToHost, st));
    IPG_CUDA(cudaStreamSynchronize(st));
    if (h.status & (kStatusBadCsr | kStatusBadColumn))
        return set_error(IPG_EINVAL, "ipg_sssp_noalloc: malformed CSR (offsets or a column index out of range)");

    na_init<<<na_grid(n), 256, 0, st>>>(dist_dev, n, source, fr[0], fval);
    IPG_CUDA(cudaGetLastError());
    uint32_t f = 1, s = 0, count = 0;
    int cur = 0;
    for (;;) {
        IPG_CUDA(cudaMemsetAsync(ctr, 0, 16, st));  // next_size, status, edges
        const unsigned grid = na_grid((uint64_t)f * 32);
        if (weights_dev)
            na_relax<true><<<grid, 256, 0, st>>>(offsets_dev, columns_dev, weights_dev, dist_dev, fr[cur], fval, f,
                                                 stamp, fr[cur ^ 1], ctr, s + 1);
        else
            na_relax<false><<<grid, 256, 0, st>>>(offsets_dev, columns_dev, nullptr, dist_dev, fr[cur], fval, f,
                                                  stamp, fr[cur ^ 1], ctr, s + 1);
        IPG_CUDA(cudaGetLastError());
        IPG_CUDA(cudaMemcpyAsync(&h, ctr, sizeof(h), cudaMemcpyDeviceToHost, st));
        IPG_CUDA(cudaStreamSynchronize(st));
        if (h.status & kStatusOverflow) return set_error(IPG_EOVERFLOW, "ipg_sssp_noalloc: a path length reached UINT32_MAX");
        if (h.next_size == 0) {
            count = s + 1 + (h.edges > 0 ? 1 : 0);
            break;
        }
        if (h.next_size > n) return set_error(IPG_EDEVICE, "ipg_sssp_noalloc: frontier overflow");
        f = h.next_size;
        na_snapshot<<<na_grid(f), 256, 0, st>>>(dist_dev, fr[cur ^ 1], f, fval);
        IPG_CUDA(cudaGetLastError());
        cur ^= 1;
        ++s;
    }
    if (supersteps_out) *supersteps_out = count;
    return IPG_OK;
}
