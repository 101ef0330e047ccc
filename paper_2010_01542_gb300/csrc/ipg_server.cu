// Serving loop: a resident set of graphs answering a stream of mixed queries
// (SSSP, Hashmin CC, PageRank), with continuous batching.
//
// Every graph has a FIFO of pending queries.  Worker threads take the oldest
// waiting graph that no other worker is running (calls on one graph share its
// workspace and must not overlap) and dispatch:
//   - SSSP queries at the head of the graph's queue: with at least
//     min_sssp_batch of them queued (by default 2 to 32, growing with the graph's
//     edge count) a lane session of the batched engine starts: each query takes
//     one of 32 lanes, and whenever a lane's query finishes (its run quiesced)
//     the lane is harvested and the next SSSP query at the head of the queue
//     takes it at the following superstep boundary, so queries that arrive
//     while others are on the GPU join the
//     running batch (continuous batching).  A submit for a graph in a session
//     raises a flag in mapped host memory that ends the running graph launch at
//     the next superstep boundary when a lane is free.  The session admits no
//     query from behind a queued Hashmin or PageRank query (first come, first
//     served per graph), and ends when its lanes are empty.  With fewer SSSP
//     queries queued they run one source at a time, which is faster there;
//   - otherwise the head query's kind (Hashmin, or PageRank with the same update
//     count): every such query queued on the graph shares one run, since they
//     compute the same result (in flight only: finished results are not reused).
// Graphs run on their own streams, so the work of different graphs overlaps on
// the device.  Before a dispatch, the worker checks that the graph's workspace
// fits next to the others (free device memory minus a reserve, or a fixed
// budget); if not, it releases the workspace of idle graphs, least recently
// used first, and otherwise waits for running work to finish.  Results go to
// the caller's host buffers; completions carry timestamps for latency.  A query
// can be cancelled until a worker dispatches it.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include <string.h>

#include "ipg_internal.cuh"

struct ipg_server {
    struct Pending {
        ipg_query q;
        double t_submit;
    };
    struct Slot {
        ipg_graph* g = nullptr;
        std::deque<Pending> pending;
        bool busy = false;
        bool session = false;  // a worker runs an SSSP lane session on this graph
        uint64_t last_used = 0;
        size_t held = 0;  // workspace bytes this graph holds (estimate)
    };
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ipg_completion> done;
    std::vector<std::thread> workers;
    bool stop = false;
    uint64_t inflight = 0;
    uint64_t tick = 0;
    size_t budget = 0;  // 0: use free device memory minus reserve
    size_t reserve = 0;
    uint32_t max_batch = 256;
    uint32_t min_batch = 0;   // fewer queued SSSP queries run one source at a time (0: per graph)
    size_t stage_words = 0;   // per-worker staging allocated at start (IPG_SERVER_PREPARE)
    std::chrono::steady_clock::time_point t0;
    int device = 0;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace ipg {

void release_workspace(ipg_graph* g);  // ipg_graph.cu

namespace {

// Default for ipg_server_options.min_sssp_batch, per graph: fewer queued SSSP
// queries than this run one source at a time.  A lane session's dense supersteps
// scan every in-edge once for all its lanes, so it pays from fewer queries on a
// smaller graph, whose one-source runs are launch-bound.  Measured crossovers of
// ipg_sssp_batch against one-at-a-time runs on directed R-MAT graphs (EF 16): about
// 3 queries at m = 2.6e5, 6 at m = 4.2e6 and 26 at m = 6.5e7; this follows
// 3 * 2^(0.375 * (log2 m - 18)) between 2 and 32.
uint32_t session_threshold(const ipg_server* s, const ipg_graph* g) {
    if (s->min_batch) return s->min_batch;
    const double lg = g->m > 1 ? std::log2((double)g->m) : 0.0;
    const double k = 3.0 * std::exp2(0.375 * (lg - 18.0));
    return k < 2.0 ? 2u : k > 32.0 ? 32u : (uint32_t)std::lround(k);
}

// one run of every program on every graph, so their workspaces exist before serving
ipg_status prepare_graphs(ipg_graph* const* graphs, uint32_t count) {
    size_t nmax = 0;
    for (uint32_t i = 0; i < count; ++i) nmax = graphs[i]->n > nmax ? graphs[i]->n : nmax;
    if (!nmax) return IPG_OK;
    constexpr uint32_t kSources = 32;
    uint32_t* scratch = nullptr;
    IPG_CUDA(cudaMalloc(&scratch, sizeof(uint32_t) * kSources * nmax));
    ipg_status r = IPG_OK;
    for (uint32_t i = 0; i < count && r == IPG_OK; ++i) {
        ipg_graph* g = graphs[i];
        if (!g->n) continue;
        uint32_t src[kSources];
        for (uint32_t k = 0; k < kSources; ++k) src[k] = (uint32_t)((uint64_t)g->n * k / kSources);
        r = ipg_sssp_dev(g, 0, scratch, nullptr, g->stream);
        if (r == IPG_OK) r = sssp_batch_run(g, src, kSources, scratch, nullptr, g->stream);
        // PageRank with the paper's 10 updates: also captures that loop's graph
        if (r == IPG_OK) r = ipg_pagerank_dev(g, 10, reinterpret_cast<float*>(scratch), nullptr, g->stream);
        if (r == IPG_OK && !g->directed) r = ipg_hashmin_cc_dev(g, scratch, nullptr, g->stream);
        // the host-output staging of ipg_sssp / ipg_hashmin_cc / ipg_pagerank
        size_t cap = g->val_stage ? (size_t)g->n * sizeof(uint32_t) : 0;
        if (r == IPG_OK && !g->val_stage) r = ensure(&g->val_stage, &cap, (size_t)g->n);
        if (r == IPG_OK) r = ensure(&g->pr_out_stage, &g->pr_out_stage_cap, (size_t)g->n);
    }
    cudaFree(scratch);
    return r;
}


// device bytes a dispatch may still need to allocate on this graph
size_t workspace_need(const ipg_graph* g, uint32_t kind, uint32_t k, uint32_t min_batch) {
    const size_t n = g->n, m = g->m;
    const size_t tiles = (n + m) / 2048 + 2;
    size_t need = 0;
    if (!g->csc_ready && g->directed) need += m * 9 + n * 8;  // in-edges (sources + weights) and offsets
    if (kind == IPG_Q_PAGERANK) {
        if (!g->pr_box[0]) need += n * 16 + tiles * 12;
    } else {
        if (!g->stamp) need += n * 36 + tiles * 4;
        if (!g->sval) need += n * 4 + tiles * 12;
        // batched SSSP (one line): dist and sender rows [n][32], masks, frontiers, push tasks, chunk rows
        if (kind == IPG_Q_SSSP && k >= min_batch && !g->batch) need += n * 288 + (m / 256 + 1) * 12;
    }
    if (!g->val_stage) need += n * 4;
    return need;
}

size_t device_free(int device) {
    size_t fr = 0, tot = 0;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device) cudaSetDevice(device);
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) fr = 0;
    if (prev != device && prev >= 0) cudaSetDevice(prev);
    return fr;
}

// sources a worker stages at once for batched SSSP (the batched engine's group size)
constexpr size_t kStageSources = 32;

struct WorkerBuffers {
    uint32_t* dev = nullptr;  // kStageSources * n staging for batched SSSP
    size_t cap = 0;
    ipg_status reserve(size_t words) {
        if (cap >= words) return IPG_OK;
        if (dev) cudaFree(dev);
        dev = nullptr;
        cap = 0;
        if (cudaMalloc(&dev, sizeof(uint32_t) * (words ? words : 1)) != cudaSuccess)
            return set_error(IPG_ENOMEM, "server: staging allocation failed");
        cap = words;
        return IPG_OK;
    }
    ~WorkerBuffers() {
        if (dev) cudaFree(dev);
    }
};

// An SSSP lane session on slot `pick` (the caller holds the lock and has marked
// the slot busy; `first` are the head queries to seed, at most 32).  Returns with
// the lock held.
void run_session(ipg_server* s, std::unique_lock<std::mutex>& lock, int pick, std::vector<ipg_server::Pending> first,
                 WorkerBuffers& buf) {
    auto& slot = s->slots[pick];
    ipg_graph* g = slot.g;
    const size_t n = g->n;
    const uint32_t cap = std::min<uint32_t>(32, std::max<uint32_t>(1, s->max_batch));
    slot.session = true;
    lock.unlock();
    struct LiveQuery {
        ipg_server::Pending p;
        double t_start = 0;
        uint32_t batch = 0;
        uint32_t joined = 0;
    };
    std::vector<LiveQuery> by_row(32);
    std::vector<uint32_t> free_rows;
    for (int r = 31; r >= 0; --r) free_rows.push_back((uint32_t)r);
    uint32_t live_count = 0;
    ipg_status rc = buf.reserve(32 * n);
    if (rc == IPG_OK) rc = lanes_open(g, buf.dev, g->stream);
    std::vector<ipg_server::Pending> seeds = std::move(first);
    bool opened = true;
    std::vector<ipg_completion> out;
    for (;;) {
        uint32_t src[32], rows[32];
        const double t_seed = s->now();
        for (size_t i = 0; i < seeds.size(); ++i) {
            const uint32_t r = free_rows.back();
            free_rows.pop_back();
            by_row[r].p = seeds[i];
            by_row[r].t_start = t_seed;
            by_row[r].batch = live_count + (uint32_t)seeds.size();
            by_row[r].joined = opened ? 0u : 1u;
            src[i] = seeds[i].q.source;
            rows[i] = r;
        }
        live_count += (uint32_t)seeds.size();
        LaneReport rep{};
        if (rc == IPG_OK) rc = lanes_step(g, src, rows, (uint32_t)seeds.size(), g->stream, &rep);
        seeds.clear();
        opened = false;
        out.clear();
        if (rc != IPG_OK) {
            // every query of the session fails with the same status
            for (uint32_t r = 0; r < 32; ++r) {
                if (std::find(free_rows.begin(), free_rows.end(), r) != free_rows.end()) continue;
                ipg_completion c{};
                c.user = by_row[r].p.q.user;
                c.status = rc;
                c.batch = by_row[r].batch;
                c.joined = by_row[r].joined;
                c.t_submit = by_row[r].p.t_submit;
                c.t_start = by_row[r].t_start;
                c.t_done = s->now();
                out.push_back(c);
                free_rows.push_back(r);
            }
            live_count = 0;
        } else {
            for (uint32_t fin = rep.finished; fin; fin &= fin - 1) {
                const int l = __builtin_ctz(fin);
                const uint32_t r = rep.row[l];
                cudaError_t e = cudaMemcpyAsync(by_row[r].p.q.out, buf.dev + (size_t)r * n, sizeof(uint32_t) * n,
                                                cudaMemcpyDeviceToHost, g->stream);
                ipg_completion c{};
                c.user = by_row[r].p.q.user;
                c.status = e == cudaSuccess ? IPG_OK : cuda_fail(e, "server result copy", __FILE__, __LINE__);
                c.supersteps = rep.count[l];
                c.batch = by_row[r].batch;
                c.joined = by_row[r].joined;
                c.t_submit = by_row[r].p.t_submit;
                c.t_start = by_row[r].t_start;
                out.push_back(c);
                free_rows.push_back(r);
                --live_count;
            }
            if (!out.empty()) {
                cudaError_t e = cudaStreamSynchronize(g->stream);
                if (e != cudaSuccess) {
                    const ipg_status bad = cuda_fail(e, "server result copy", __FILE__, __LINE__);
                    for (auto& c : out) c.status = bad;
                }
            }
        }
        const double t_done = s->now();
        lock.lock();
        for (auto& c : out) {
            c.t_done = t_done;
            s->done.push_back(c);
        }
        s->inflight -= out.size();
        if (!out.empty()) s->cv_done.notify_all();
        // admission at this superstep boundary: SSSP queries at the head of the queue
        volatile unsigned int* flag = lanes_admit_flag(g);
        if (flag) *flag = 0;
        if (rc == IPG_OK)
            while (!slot.pending.empty() && slot.pending.front().q.kind == IPG_Q_SSSP && live_count + seeds.size() < cap) {
                seeds.push_back(slot.pending.front());
                slot.pending.pop_front();
            }
        if (live_count == 0 && seeds.empty()) break;
        lock.unlock();
    }
    slot.session = false;
    lanes_close(g);
}

void finish(ipg_server* s, const std::vector<ipg_server::Pending>& batch, const std::vector<ipg_status>& rc,
            const std::vector<uint32_t>& steps, double t_start, double t_done) {
    for (size_t i = 0; i < batch.size(); ++i) {
        ipg_completion c{};
        c.user = batch[i].q.user;
        c.status = rc[i];
        c.supersteps = steps[i];
        c.batch = (uint32_t)batch.size();
        c.t_submit = batch[i].t_submit;
        c.t_start = t_start;
        c.t_done = t_done;
        s->done.push_back(c);
    }
}

void worker_main(ipg_server* s) {
    cudaSetDevice(s->device);
    WorkerBuffers buf;
    if (s->stage_words) buf.reserve(s->stage_words);  // IPG_SERVER_PREPARE: before any query
    std::unique_lock<std::mutex> lock(s->mu);
    while (!s->stop) {
        // the idle graph whose head query has waited longest
        int pick = -1;
        double oldest = 0;
        for (size_t i = 0; i < s->slots.size(); ++i) {
            const auto& sl = s->slots[i];
            if (sl.busy || sl.pending.empty()) continue;
            if (pick < 0 || sl.pending.front().t_submit < oldest) {
                pick = (int)i;
                oldest = sl.pending.front().t_submit;
            }
        }
        if (pick < 0) {
            s->cv_work.wait(lock);
            continue;
        }
        auto& slot = s->slots[pick];
        std::vector<ipg_server::Pending> batch;
        const uint32_t kind = slot.pending.front().q.kind;
        size_t head_sssp = 0;  // SSSP queries at the head of the queue
        for (auto it = slot.pending.begin(); it != slot.pending.end() && it->q.kind == IPG_Q_SSSP; ++it) ++head_sssp;
        const uint32_t min_batch = session_threshold(s, slot.g);
        const bool session = kind == IPG_Q_SSSP && head_sssp >= min_batch && s->max_batch > 1;
        if (session) {
            const size_t cap = std::min<size_t>(32, s->max_batch);
            while (batch.size() < cap && !slot.pending.empty() && slot.pending.front().q.kind == IPG_Q_SSSP) {
                batch.push_back(slot.pending.front());
                slot.pending.pop_front();
            }
        } else if (kind == IPG_Q_SSSP) {
            for (auto it = slot.pending.begin(); it != slot.pending.end() && batch.size() < s->max_batch;) {
                if (it->q.kind == IPG_Q_SSSP) {
                    batch.push_back(*it);
                    it = slot.pending.erase(it);
                } else {
                    ++it;
                }
            }
        } else {
            // Hashmin / PageRank queries queued on this graph compute the same result: they
            // share one run (in flight only; finished results are never reused)
            const uint32_t upd = slot.pending.front().q.updates;
            for (auto it = slot.pending.begin(); it != slot.pending.end() && batch.size() < s->max_batch;) {
                if (it->q.kind == kind && (kind != IPG_Q_PAGERANK || it->q.updates == upd)) {
                    batch.push_back(*it);
                    it = slot.pending.erase(it);
                } else {
                    ++it;
                }
            }
        }
        // admission by device memory
        const size_t need = workspace_need(slot.g, kind, session ? min_batch : (uint32_t)batch.size(), min_batch);
        for (;;) {
            size_t avail;
            if (s->budget) {
                size_t used = 0;
                for (auto& o : s->slots) used += o.held;
                avail = s->budget > used ? s->budget - used : 0;
            } else {
                const size_t fr = device_free(s->device);
                avail = fr > s->reserve ? fr - s->reserve : 0;
            }
            if (need <= avail) break;
            // release the least recently used idle workspace
            int lru = -1;
            for (size_t i = 0; i < s->slots.size(); ++i) {
                auto& o = s->slots[i];
                if ((int)i == pick || o.busy || o.held == 0) continue;
                if (lru < 0 || o.last_used < s->slots[lru].last_used) lru = (int)i;
            }
            if (lru >= 0) {
                release_workspace(s->slots[lru].g);
                s->slots[lru].held = 0;
                continue;
            }
            bool others_running = false;
            for (auto& o : s->slots) others_running |= o.busy;
            if (!others_running) break;  // nothing to wait for: try, and report ENOMEM if it fails
            s->cv_done.wait(lock);
        }
        slot.busy = true;
        slot.last_used = ++s->tick;
        slot.held += need;
        ipg_graph* g = slot.g;
        if (session) {
            run_session(s, lock, pick, std::move(batch), buf);
            slot.busy = false;
            s->cv_done.notify_all();
            s->cv_work.notify_all();
            continue;
        }
        lock.unlock();

        const double t_start = s->now();
        std::vector<ipg_status> rc(batch.size(), IPG_OK);
        std::vector<uint32_t> steps(batch.size(), 0);
        if (kind == IPG_Q_SSSP) {
            // a few sources: one-source runs (push for sparse supersteps) beat a lane
            // session, whose pull supersteps stream every in-edge
            for (size_t i = 0; i < batch.size(); ++i) {
                ipg_stats st{nullptr, 0, 0, 0, 0};
                rc[i] = ipg_sssp(g, batch[i].q.source, (uint32_t*)batch[i].q.out, &st);
                steps[i] = st.count;
            }
        } else if (kind == IPG_Q_HASHMIN || kind == IPG_Q_PAGERANK) {
            ipg_stats st{nullptr, 0, 0, 0, 0};
            const ipg_status r = kind == IPG_Q_HASHMIN
                                     ? ipg_hashmin_cc(g, (uint32_t*)batch[0].q.out, &st)
                                     : ipg_pagerank(g, batch[0].q.updates, (float*)batch[0].q.out, &st);
            for (size_t i = 1; i < batch.size() && r == IPG_OK; ++i)
                memcpy(batch[i].q.out, batch[0].q.out, sizeof(uint32_t) * (size_t)g->n);
            std::fill(rc.begin(), rc.end(), r);
            std::fill(steps.begin(), steps.end(), st.count);
        } else {
            rc[0] = set_error(IPG_EINVAL, "server: unknown query kind %u", kind);
        }
        const double t_done = s->now();

        lock.lock();
        slot.busy = false;
        finish(s, batch, rc, steps, t_start, t_done);
        s->inflight -= batch.size();
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

}  // namespace
}  // namespace ipg

using namespace ipg;

extern "C" {

ipg_status ipg_server_create(ipg_graph* const* graphs, uint32_t count, const ipg_server_options* opt,
                             ipg_server** out) {
    if (!out) return set_error(IPG_EINVAL, "ipg_server_create: out is NULL");
    *out = nullptr;
    if (!graphs || count == 0) return set_error(IPG_EINVAL, "ipg_server_create: no graphs");
    for (uint32_t i = 0; i < count; ++i)
        if (!graphs[i]) return set_error(IPG_EINVAL, "ipg_server_create: graph %u is NULL", i);
    ipg_server* s = new (std::nothrow) ipg_server();
    if (!s) return set_error(IPG_ENOMEM, "ipg_server_create: host allocation failed");
    s->t0 = std::chrono::steady_clock::now();
    s->device = graphs[0]->device;
    s->slots.resize(count);
    for (uint32_t i = 0; i < count; ++i) s->slots[i].g = graphs[i];
    uint32_t workers = opt && opt->workers ? opt->workers : 8;
    if (workers > 64) workers = 64;
    s->max_batch = opt && opt->max_batch ? opt->max_batch : 256;
    s->budget = opt ? (size_t)opt->workspace_budget : 0;
    s->reserve = opt && opt->reserve_bytes ? (size_t)opt->reserve_bytes : ((size_t)1 << 30);
    s->min_batch = opt && opt->min_sssp_batch ? opt->min_sssp_batch : 0u;
    if (opt && (opt->flags & IPG_SERVER_PREPARE)) {
        const ipg_status r = prepare_graphs(graphs, count);
        if (r != IPG_OK) {
            delete s;
            return r;
        }
        for (uint32_t i = 0; i < count; ++i)
            s->stage_words = std::max(s->stage_words, kStageSources * (size_t)graphs[i]->n);
    }
    if (opt && (opt->flags & IPG_SERVER_AUTOTUNE)) {
        for (uint32_t i = 0; i < count; ++i) {
            ipg_graph* g = graphs[i];
            const uint32_t progs = IPG_TUNE_PAGERANK | IPG_TUNE_SSSP | IPG_TUNE_SSSP_BATCH |
                                   (g->directed ? 0u : IPG_TUNE_HASHMIN);
            const ipg_status r = ipg_autotune(g, progs, UINT32_MAX, nullptr, g->stream);
            if (r != IPG_OK) {
                delete s;
                return r;
            }
        }
    }
    for (uint32_t w = 0; w < workers; ++w) s->workers.emplace_back(worker_main, s);
    *out = s;
    return IPG_OK;
}

ipg_status ipg_server_submit(ipg_server* s, const ipg_query* q) {
    if (!s || !q) return set_error(IPG_EINVAL, "ipg_server_submit: NULL argument");
    if (q->graph >= s->slots.size()) return set_error(IPG_EINVAL, "ipg_server_submit: graph %u out of range", q->graph);
    const ipg_graph* g = s->slots[q->graph].g;
    if (q->kind > IPG_Q_PAGERANK) return set_error(IPG_EINVAL, "ipg_server_submit: unknown kind %u", q->kind);
    if (q->kind == IPG_Q_SSSP && q->source >= g->n)
        return set_error(IPG_EINVAL, "ipg_server_submit: source %u >= n = %u", q->source, g->n);
    if (q->kind == IPG_Q_HASHMIN && g->directed)
        return set_error(IPG_EINVAL, "ipg_server_submit: Hashmin needs an undirected graph");
    if (g->n && !q->out) return set_error(IPG_EINVAL, "ipg_server_submit: output is NULL");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        auto& slot = s->slots[q->graph];
        slot.pending.push_back({*q, s->now()});
        s->inflight++;
        if (slot.session && q->kind == IPG_Q_SSSP) {
            // end the session's running launch at the next superstep boundary
            volatile unsigned int* flag = lanes_admit_flag(slot.g);
            if (flag) *flag = 1;
        }
    }
    s->cv_work.notify_one();
    return IPG_OK;
}

uint32_t ipg_server_poll(ipg_server* s, ipg_completion* out, uint32_t cap, int wait_ms) {
    if (!s || !out || cap == 0) return 0;
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->done.empty() && wait_ms != 0) {
        if (wait_ms < 0)
            s->cv_done.wait(lock, [&] { return !s->done.empty() || s->inflight == 0; });
        else
            s->cv_done.wait_for(lock, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
    }
    uint32_t k = 0;
    while (k < cap && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    return k;
}

ipg_status ipg_server_cancel(ipg_server* s, uint64_t user, uint32_t* cancelled) {
    if (!s) return set_error(IPG_EINVAL, "ipg_server_cancel: server is NULL");
    uint32_t k = 0;
    {
        // workers take queries off the queues under this lock, so each query is
        // either still queued here (and cancelled) or already dispatched
        std::lock_guard<std::mutex> lock(s->mu);
        const double t = s->now();
        for (auto& sl : s->slots) {
            for (auto it = sl.pending.begin(); it != sl.pending.end();) {
                if (it->q.user != user) {
                    ++it;
                    continue;
                }
                ipg_completion c{};
                c.user = user;
                c.status = IPG_ECANCELED;
                c.t_submit = it->t_submit;
                c.t_start = t;
                c.t_done = t;
                s->done.push_back(c);
                it = sl.pending.erase(it);
                ++k;
            }
        }
        s->inflight -= k;
    }
    if (k) s->cv_done.notify_all();
    if (cancelled) *cancelled = k;
    return IPG_OK;
}

ipg_status ipg_server_drain(ipg_server* s) {
    if (!s) return set_error(IPG_EINVAL, "ipg_server_drain: server is NULL");
    std::unique_lock<std::mutex> lock(s->mu);
    s->cv_done.wait(lock, [&] { return s->inflight == 0; });
    return IPG_OK;
}

double ipg_server_now(const ipg_server* s) { return s ? s->now() : 0.0; }

void ipg_server_destroy(ipg_server* s) {
    if (!s) return;
    {
        std::unique_lock<std::mutex> lock(s->mu);
        s->cv_done.wait(lock, [&] { return s->inflight == 0; });
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    delete s;
}

}  // extern "C"
