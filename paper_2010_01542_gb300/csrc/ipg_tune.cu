// Autotuner: picks, for one graph, the launch shape of its Pregel programs by
// timing candidate knob values on that graph.  The paper fixes one schedule per
// benchmark for its OpenMP versions (Sec. V-B, VI-C); on the GPU the best
// push/pull switch point and pull-kernel shape depend on the graph, so they are
// measured.  Every candidate gives bit-identical results (see include/ipg.h),
// so tuning changes speed only.
#include <map>
#include <mutex>
#include <vector>

#include "ipg_internal.cuh"

namespace ipg {
namespace {

constexpr int kSamples = 64;
const long long kDivisors[] = {0, 2, 4, 6, 10, 16, 32};
const long long kPrShapes[][2] = {{0, -1}, {0, 60}, {1, -1}, {1, 5}};  // (pr_engine, pr_carveout)
// batched SSSP: (push/pull divisor, in-edges per warp task of the pull form: the tile size)
const long long kBatchShapes[][2] = {{6, 256}, {0, 256}, {2, 256}, {16, 256}, {6, 64}, {6, 128}, {6, 512}, {6, 1024}};

__global__ void sample_offsets_kernel(const uint64_t* __restrict__ off, uint32_t n, uint64_t* __restrict__ out) {
    const uint32_t i = threadIdx.x;
    if (i < kSamples) out[i] = off[(uint64_t)n * i / (kSamples - 1)];
}

enum Prog { kProgHashmin = 0, kProgSssp = 1, kProgPagerank = 2, kProgBatch = 3, kProgs = 4 };
const uint32_t kProgBit[kProgs] = {IPG_TUNE_HASHMIN, IPG_TUNE_SSSP, IPG_TUNE_PAGERANK, IPG_TUNE_SSSP_BATCH};
constexpr uint32_t kBatchSources = 32;

struct CacheEntry {
    GraphTuning t;
    float ms[kProgs] = {0.f, 0.f, 0.f, 0.f};  // the chosen candidates' runs
};

bool tuned(const GraphTuning& t, int prog) {
    return prog == kProgHashmin ? t.cc : prog == kProgSssp ? t.sssp : prog == kProgPagerank ? t.pr : t.batch;
}
void untune(GraphTuning& t, int prog) {
    if (prog == kProgHashmin) t.cc = false;
    if (prog == kProgSssp) t.sssp = false;
    if (prog == kProgPagerank) t.pr = false;
    if (prog == kProgBatch) t.batch = false;
}
// candidate c of program prog; a and b are its values (b only for PageRank)
void set_candidate(GraphTuning& t, int prog, long long a, long long b) {
    if (prog == kProgHashmin) t.cc = true, t.cc_divisor = a;
    if (prog == kProgSssp) t.sssp = true, t.sssp_divisor = a;
    if (prog == kProgPagerank) t.pr = true, t.pr_engine = a, t.pr_carveout = b;
    if (prog == kProgBatch) t.batch = true, t.batch_divisor = a, t.batch_chunk = b;
}
void copy_choice(GraphTuning& dst, const GraphTuning& src, int prog) {
    if (prog == kProgHashmin) set_candidate(dst, prog, src.cc_divisor, 0);
    if (prog == kProgSssp) set_candidate(dst, prog, src.sssp_divisor, 0);
    if (prog == kProgPagerank) set_candidate(dst, prog, src.pr_engine, src.pr_carveout);
    if (prog == kProgBatch) set_candidate(dst, prog, src.batch_divisor, src.batch_chunk);
}

std::mutex g_cache_mu;
std::map<std::vector<uint64_t>, CacheEntry>& cache() {
    static std::map<std::vector<uint64_t>, CacheEntry> c;
    return c;
}

ipg_status fingerprint(ipg_graph* g, uint64_t* scratch, cudaStream_t st, std::vector<uint64_t>* key) {
    uint64_t h[kSamples];
    sample_offsets_kernel<<<1, kSamples, 0, st>>>(g->off, g->n, scratch);
    IPG_CUDA(cudaGetLastError());
    IPG_CUDA(cudaMemcpyAsync(h, scratch, sizeof(h), cudaMemcpyDeviceToHost, st));
    IPG_CUDA(cudaStreamSynchronize(st));
    key->assign({(uint64_t)g->n, g->m, (uint64_t)g->directed, (uint64_t)g->weighted, g->max_outdeg,
                 (uint64_t)sm_count_of(g->device)});
    key->insert(key->end(), h, h + kSamples);
    return IPG_OK;
}

// device time of one call on the stream
template <class F>
ipg_status time_call(cudaStream_t st, float* ms, F&& call) {
    cudaEvent_t a, b;
    IPG_CUDA(cudaEventCreate(&a));
    IPG_CUDA(cudaEventCreate(&b));
    ipg_status rc = IPG_OK;
    cudaError_t e = cudaEventRecord(a, st);
    if (e == cudaSuccess) {
        rc = call();
        if (rc == IPG_OK) e = cudaEventRecord(b, st);
        if (rc == IPG_OK && e == cudaSuccess) e = cudaEventSynchronize(b);
        if (rc == IPG_OK && e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc != IPG_OK) return rc;
    IPG_CUDA(e);
    return IPG_OK;
}

// the faster of two timed runs
template <class F>
ipg_status best_of_two(cudaStream_t st, float* ms, uint32_t* runs, F&& call) {
    float t0 = 0.f, t1 = 0.f;
    IPG_TRY(time_call(st, &t0, call));
    IPG_TRY(time_call(st, &t1, call));
    *runs += 2;
    *ms = t0 < t1 ? t0 : t1;
    return IPG_OK;
}

ipg_status autotune(ipg_graph* g, uint32_t programs, uint32_t source, ipg_tune_report* rep, cudaStream_t st) {
    const uint32_t kAll = IPG_TUNE_PAGERANK | IPG_TUNE_HASHMIN | IPG_TUNE_SSSP | IPG_TUNE_SSSP_BATCH;
    if (!g) return set_error(IPG_EINVAL, "ipg_autotune: graph is NULL");
    if (programs & ~(kAll | IPG_TUNE_FORCE)) return set_error(IPG_EINVAL, "ipg_autotune: unknown program bits 0x%x", programs);
    if ((programs & IPG_TUNE_HASHMIN) && g->directed)
        return set_error(IPG_EINVAL, "ipg_autotune: Hashmin components need an undirected graph");
    DeviceGuard guard(g->device);
    if (!guard.ok) return set_error(IPG_ECUDA, "ipg_autotune: cannot select the graph's device");
    const bool force = programs & IPG_TUNE_FORCE;
    programs &= kAll;
    ipg_tune_report r{};
    r.hashmin_pull_divisor = r.sssp_pull_divisor = r.sssp_batch_divisor = r.pr_engine = r.pr_carveout = -1;
    const uint32_t n = g->n;
    if (n == 0 || programs == 0) {
        if (rep) *rep = r;
        return IPG_OK;
    }
    const size_t words = (size_t)n * ((programs & IPG_TUNE_SSSP_BATCH) ? kBatchSources : 1);
    void* scratch = nullptr;
    IPG_CUDA(cudaMalloc(&scratch, sizeof(uint32_t) * (words > 2 * kSamples ? words : 2 * kSamples)));
    ipg_status rc = IPG_OK;
    GraphTuning t = g->tuned;
    float best_ms[kProgs] = {0.f, 0.f, 0.f, 0.f}, def_ms[kProgs] = {0.f, 0.f, 0.f, 0.f};
    do {
        std::vector<uint64_t> key;
        rc = fingerprint(g, static_cast<uint64_t*>(scratch), st, &key);
        if (rc != IPG_OK) break;
        CacheEntry hit;
        bool have = false;
        if (!force) {
            std::lock_guard<std::mutex> lock(g_cache_mu);
            auto it = cache().find(key);
            if (it != cache().end()) {
                hit = it->second;
                have = true;
            }
        }
        // SSSP source: the caller's, else the vertex of largest total degree (internal id 0)
        uint32_t src = source;
        if ((programs & (IPG_TUNE_SSSP | IPG_TUNE_SSSP_BATCH)) && src >= n) {
            cudaError_t e = cudaMemcpy(&src, g->perm, sizeof(uint32_t), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "copy of the tuning source", __FILE__, __LINE__);
                break;
            }
        }
        uint32_t batch_src[kBatchSources];
        batch_src[0] = src;
        for (uint32_t i = 1; i < kBatchSources; ++i) batch_src[i] = (uint32_t)((uint64_t)n * i / kBatchSources);
        uint32_t* out_u = static_cast<uint32_t*>(scratch);
        float* out_f = static_cast<float*>(scratch);
        uint32_t from_cache = 0, requested = 0;
        for (int prog = 0; prog < kProgs && rc == IPG_OK; ++prog) {
            if (!(programs & kProgBit[prog])) continue;
            ++requested;
            if (have && tuned(hit.t, prog)) {
                ++from_cache;
                copy_choice(t, hit.t, prog);
                best_ms[prog] = hit.ms[prog];
                continue;
            }
            auto run = [&]() -> ipg_status {
                if (prog == kProgHashmin) return ipg_hashmin_cc_dev(g, out_u, nullptr, st);
                if (prog == kProgSssp) return ipg_sssp_dev(g, src, out_u, nullptr, st);
                if (prog == kProgBatch) return sssp_batch_run(g, batch_src, kBatchSources, out_u, nullptr, st);
                return ipg_pagerank_dev(g, 3, out_f, nullptr, st);
            };
            // the process-wide knobs first (also a warm-up: workspaces, in-edge copy)
            const GraphTuning saved = g->tuned;
            untune(g->tuned, prog);
            rc = run();
            if (rc == IPG_OK) rc = best_of_two(st, &def_ms[prog], &r.candidates_timed, run);
            float best = -1.f;
            long long best_a = 0, best_b = 0;
            const int count = prog == kProgPagerank ? 4
                              : prog == kProgBatch ? (int)(sizeof(kBatchShapes) / sizeof(kBatchShapes[0]))
                                                   : (int)(sizeof(kDivisors) / sizeof(kDivisors[0]));
            for (int c = 0; c < count && rc == IPG_OK; ++c) {
                const long long a = prog == kProgPagerank ? kPrShapes[c][0]
                                    : prog == kProgBatch  ? kBatchShapes[c][0]
                                                          : kDivisors[c];
                const long long b = prog == kProgPagerank ? kPrShapes[c][1] : prog == kProgBatch ? kBatchShapes[c][1] : 0;
                set_candidate(g->tuned, prog, a, b);
                float ms = 0.f;
                rc = best_of_two(st, &ms, &r.candidates_timed, run);
                if (rc == IPG_OK && (best < 0.f || ms < best)) {
                    best = ms;
                    best_a = a;
                    best_b = b;
                }
            }
            g->tuned = saved;
            if (rc != IPG_OK) break;
            set_candidate(t, prog, best_a, best_b);
            best_ms[prog] = best;
            std::lock_guard<std::mutex> lock(g_cache_mu);
            CacheEntry& ce = cache()[key];
            set_candidate(ce.t, prog, best_a, best_b);
            ce.ms[prog] = best;
        }
        if (rc != IPG_OK) break;
        g->tuned = t;
        r.cached = from_cache > 0 && from_cache == requested;
    } while (false);
    cudaFree(scratch);
    if (rc != IPG_OK) return rc;
    const GraphTuning& gt = g->tuned;
    r.programs = (gt.pr ? IPG_TUNE_PAGERANK : 0u) | (gt.cc ? IPG_TUNE_HASHMIN : 0u) | (gt.sssp ? IPG_TUNE_SSSP : 0u) |
                 (gt.batch ? IPG_TUNE_SSSP_BATCH : 0u);
    if (gt.cc) r.hashmin_pull_divisor = gt.cc_divisor;
    if (gt.sssp) r.sssp_pull_divisor = gt.sssp_divisor;
    if (gt.batch) r.sssp_batch_divisor = gt.batch_divisor, r.sssp_batch_chunk = (uint32_t)gt.batch_chunk;
    if (gt.pr) r.pr_engine = gt.pr_engine, r.pr_carveout = gt.pr_carveout;
    r.hashmin_ms = best_ms[kProgHashmin], r.hashmin_default_ms = def_ms[kProgHashmin];
    r.sssp_ms = best_ms[kProgSssp], r.sssp_default_ms = def_ms[kProgSssp];
    r.sssp_batch_ms = best_ms[kProgBatch], r.sssp_batch_default_ms = def_ms[kProgBatch];
    r.pagerank_ms = best_ms[kProgPagerank], r.pagerank_default_ms = def_ms[kProgPagerank];
    if (rep) *rep = r;
    return IPG_OK;
}

}  // namespace
}  // namespace ipg

extern "C" ipg_status ipg_autotune(ipg_graph* g, uint32_t programs, uint32_t sssp_source, ipg_tune_report* report,
                                   void* stream) {
    return ipg::autotune(g, programs, sssp_source, report, (cudaStream_t)stream);
}
