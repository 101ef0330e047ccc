/*
 * GPU build of the same seeded R-MAT graphs as gen/rmat.c (input tool, no
 * Pregel arithmetic).  Same counter-based splitmix64 stream, same quadrant
 * thresholds, same dedup and weight rule, so for equal parameters the CSR is
 * bit-identical to the CPU build; it exists because the billion-edge graphs
 * take minutes on host cores and about a second here.
 *
 * Steps: one packed key (u << scale | v) per sampled edge (self-loops get a
 * key that sorts last), radix sort, unique, then CSR offsets from a row
 * histogram.  Undirected graphs emit both directions before the sort.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <cub/device/device_select.cuh>

namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t splitmix64_host(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct Cfg {
    uint32_t scale;
    uint32_t ta, tab, tabc;
    uint64_t base;
    int undirected;
};

__global__ void sample_kernel(Cfg c, uint64_t raw, uint64_t* __restrict__ keys) {
    const uint64_t invalid = 1ull << (2 * c.scale);
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < raw; e += stride) {
        uint32_t u = 0, v = 0, lvl = 0;
        for (uint32_t p = 0; lvl < c.scale; ++p) {
            uint64_t r = splitmix64(c.base + 16ull * e + p);
            for (int half = 0; half < 2 && lvl < c.scale; ++half, ++lvl) {
                uint32_t x = half == 0 ? (uint32_t)(r >> 32) : (uint32_t)r;
                uint32_t bit = 1u << (c.scale - 1 - lvl);
                if (x < c.ta) {
                } else if (x < c.tab) {
                    v |= bit;
                } else if (x < c.tabc) {
                    u |= bit;
                } else {
                    u |= bit;
                    v |= bit;
                }
            }
        }
        bool self = u == v;
        if (c.undirected) {
            keys[2 * e] = self ? invalid : ((uint64_t)u << c.scale) | v;
            keys[2 * e + 1] = self ? invalid : ((uint64_t)v << c.scale) | u;
        } else {
            keys[e] = self ? invalid : ((uint64_t)u << c.scale) | v;
        }
    }
}

__global__ void row_hist_kernel(const uint64_t* __restrict__ keys, uint64_t m, uint32_t scale,
                                unsigned long long* __restrict__ hist) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
        atomicAdd(&hist[keys[i] >> scale], 1ull);
}

__global__ void emit_kernel(const uint64_t* __restrict__ keys, uint64_t m, uint32_t scale, uint32_t* __restrict__ cols,
                            uint32_t* __restrict__ w, uint64_t wbase, uint32_t wmax, int symmetric) {
    const uint64_t mask = (1ull << scale) - 1;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        uint64_t k = keys[i];
        uint32_t u = (uint32_t)(k >> scale), v = (uint32_t)(k & mask);
        cols[i] = v;
        if (w) {
            uint32_t lo = u, hi = v;
            if (symmetric && lo > hi) {
                lo = v;
                hi = u;
            }
            uint64_t key = ((uint64_t)lo << 32) | hi;
            w[i] = 1u + (uint32_t)(splitmix64(wbase ^ key) % wmax);
        }
    }
}

struct Plan {
    uint32_t scale, n;
    uint64_t m;
    uint64_t* keys;  // m unique sorted keys
    int undirected;
};

unsigned grid_for(uint64_t work) {
    uint64_t b = (work + 255) / 256;
    if (b < 1) b = 1;
    return (unsigned)(b < 152 * 32 ? b : 152 * 32);
}

}  // namespace

extern "C" {

/* 0 ok, 1 bad argument, 2 out of memory, 3 CUDA error */
int gen_rmat_cuda_plan(uint32_t scale, uint32_t edge_factor, double a, double b, double c, uint64_t seed,
                       int undirected, void* stream, void** plan_out, uint32_t* n_out, uint64_t* m_out) {
    if (!plan_out || scale < 1 || scale > 31 || edge_factor < 1) return 1;
    if (!(a >= 0 && b >= 0 && c >= 0 && a + b + c <= 1.0)) return 1;
    cudaStream_t st = (cudaStream_t)stream;
    Cfg cfg;
    cfg.scale = scale;
    cfg.ta = (uint32_t)(a * 4294967296.0);
    cfg.tab = (uint32_t)((a + b) * 4294967296.0);
    double abc = (a + b + c) * 4294967296.0;
    cfg.tabc = abc >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)abc;
    cfg.base = splitmix64_host(seed);
    cfg.undirected = undirected;
    const uint64_t raw = (uint64_t)edge_factor << scale;
    const uint64_t nkeys = raw * (undirected ? 2 : 1);
    uint64_t *k0 = nullptr, *k1 = nullptr;
    void* temp = nullptr;
    size_t tb = 0, tb2 = 0;
    unsigned long long* nsel = nullptr;
    Plan* p = nullptr;
    int rc = 0;
    const int end_bit = 2 * (int)scale + 1;
    if (cudaMalloc(&k0, nkeys * 8) != cudaSuccess || cudaMalloc(&k1, nkeys * 8) != cudaSuccess ||
        cudaMalloc(&nsel, 8) != cudaSuccess) {
        rc = 2;
        goto fail;
    }
    sample_kernel<<<grid_for(raw), 256, 0, st>>>(cfg, raw, k0);
    if (cudaGetLastError() != cudaSuccess) {
        rc = 3;
        goto fail;
    }
    if (cub::DeviceRadixSort::SortKeys(nullptr, tb, k0, k1, (long long)nkeys, 0, end_bit, st) != cudaSuccess ||
        cub::DeviceSelect::Unique(nullptr, tb2, k1, k0, nsel, (long long)nkeys, st) != cudaSuccess) {
        rc = 3;
        goto fail;
    }
    if (tb2 > tb) tb = tb2;
    if (cudaMalloc(&temp, tb) != cudaSuccess) {
        rc = 2;
        goto fail;
    }
    tb2 = tb;
    if (cub::DeviceRadixSort::SortKeys(temp, tb2, k0, k1, (long long)nkeys, 0, end_bit, st) != cudaSuccess) {
        rc = 3;
        goto fail;
    }
    tb2 = tb;
    if (cub::DeviceSelect::Unique(temp, tb2, k1, k0, nsel, (long long)nkeys, st) != cudaSuccess) {
        rc = 3;
        goto fail;
    }
    {
        unsigned long long uniq = 0;
        if (cudaMemcpyAsync(&uniq, nsel, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = 3;
            goto fail;
        }
        uint64_t m = uniq;
        if (m > 0) {  // the self-loop key sorts last; drop it if present
            uint64_t last = 0;
            if (cudaMemcpy(&last, k0 + (m - 1), 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
                rc = 3;
                goto fail;
            }
            if (last == (1ull << (2 * scale))) --m;
        }
        p = new Plan();
        p->scale = scale;
        p->n = 1u << scale;
        p->m = m;
        p->keys = k0;
        p->undirected = undirected;
        k0 = nullptr;
        *plan_out = p;
        if (n_out) *n_out = p->n;
        if (m_out) *m_out = m;
    }
fail:
    if (k0) cudaFree(k0);
    if (k1) cudaFree(k1);
    if (temp) cudaFree(temp);
    if (nsel) cudaFree(nsel);
    return rc;
}

/* write offsets[n+1], cols[m] and (if w_dev != NULL) weights[m] into device buffers */
int gen_rmat_cuda_emit(void* plan, uint64_t* off_dev, uint32_t* col_dev, uint32_t* w_dev, uint64_t weight_seed,
                       uint32_t wmax, void* stream) {
    Plan* p = (Plan*)plan;
    if (!p || !off_dev || (p->m && !col_dev) || wmax < 1) return 1;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long* hist = nullptr;
    void* temp = nullptr;
    size_t tb = 0;
    int rc = 0;
    const uint64_t n1 = (uint64_t)p->n + 1;
    if (cudaMalloc(&hist, n1 * 8) != cudaSuccess) return 2;
    cudaMemsetAsync(hist, 0, n1 * 8, st);
    if (p->m) row_hist_kernel<<<grid_for(p->m), 256, 0, st>>>(p->keys, p->m, p->scale, hist);
    if (cub::DeviceScan::ExclusiveSum(nullptr, tb, hist, (unsigned long long*)off_dev, (long long)n1, st) !=
            cudaSuccess ||
        cudaMalloc(&temp, tb ? tb : 16) != cudaSuccess) {
        rc = 2;
        goto done;
    }
    if (cub::DeviceScan::ExclusiveSum(temp, tb, hist, (unsigned long long*)off_dev, (long long)n1, st) !=
        cudaSuccess) {
        rc = 3;
        goto done;
    }
    if (p->m)
        emit_kernel<<<grid_for(p->m), 256, 0, st>>>(p->keys, p->m, p->scale, col_dev, w_dev,
                                                   splitmix64_host(weight_seed), wmax, p->undirected);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) rc = 3;
done:
    if (hist) cudaFree(hist);
    if (temp) cudaFree(temp);
    return rc;
}

void gen_rmat_cuda_free(void* plan) {
    Plan* p = (Plan*)plan;
    if (!p) return;
    if (p->keys) cudaFree(p->keys);
    delete p;
}

}  // extern "C"
