/*
 * CPU baseline in the paper's final design: the vertex-centric superstep run on
 * all host cores with OpenMP, for comparison with the GPU library.  It is a
 * measured baseline, not a reference for correctness (that is the oracle), and
 * shares no code with either.
 *
 * Design choices taken from the paper's final versions (Sec. IV-VI):
 *   - vertex attributes externalised into one array per attribute (Sec. IV);
 *   - PageRank and Hashmin pull from their in-neighbours ("single broadcast":
 *     a sender publishes one value that its out-neighbours read, Sec. IV);
 *   - SSSP pushes from the active vertices only ("selection bypass", Sec. VI-C)
 *     into mailboxes combined with a compare-and-swap minimum, the lock-free case
 *     of the hybrid combiner (Sec. III);
 *   - every vertex or frontier loop uses OpenMP's dynamic schedule with chunks
 *     of 256 (Sec. V-B).
 * Supersteps are synchronous: values read in a superstep are those of its start.
 * The superstep count includes the last superstep, in which receivers compute
 * and nothing is sent, as in the Pregel model (Sec. I).
 *
 * Timing (omp_get_wtime) covers the supersteps only; building the in-edge lists
 * for the pull programs is loading work and is timed separately.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define POMP_INF 0xFFFFFFFFu
#define POMP_OK 0
#define POMP_EINVAL 1
#define POMP_ENOMEM 2
#define POMP_EOVERFLOW 7

/* in-edge lists (CSC) of a CSR graph; returns 0 or POMP_ENOMEM */
static int build_csc(uint32_t n, const uint64_t* off, const uint32_t* col, uint64_t** coff_out, uint32_t** csrc_out) {
    const uint64_t m = off[n];
    uint64_t* coff = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    uint32_t* csrc = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint64_t* fill = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    if (!coff || !csrc || !fill) {
        free(coff);
        free(csrc);
        free(fill);
        return POMP_ENOMEM;
    }
#pragma omp parallel for schedule(static)
    for (uint64_t e = 0; e < m; ++e) {
#pragma omp atomic
        coff[col[e] + 1]++;
    }
    for (uint32_t v = 0; v < n; ++v) coff[v + 1] += coff[v];
    memcpy(fill, coff, sizeof(uint64_t) * ((size_t)n + 1));
#pragma omp parallel for schedule(dynamic, 256)
    for (uint32_t u = 0; u < n; ++u) {
        for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
            uint64_t slot;
#pragma omp atomic capture
            slot = fill[col[e]]++;
            csrc[slot] = u;
        }
    }
    free(fill);
    *coff_out = coff;
    *csrc_out = csrc;
    return POMP_OK;
}

/*
 * PageRank, pull form: rank_0 = 1/N; each update reads the in-neighbours'
 * published rank/outdeg (0 for a vertex without out-edges, whose mass is lost)
 * and sets rank = 0.15/N + 0.85 * sum.  FP32 values, sums in float.
 * msgs_out = updates * m (every edge carries one message per update).
 */
int pomp_pagerank(uint32_t n, const uint64_t* off, const uint32_t* col, uint32_t updates, float* rank,
                  uint64_t* msgs_out, double* seconds_out, double* load_seconds_out) {
    if (!off || (n && !rank)) return POMP_EINVAL;
    const uint64_t m = off[n];
    double t0 = omp_get_wtime();
    uint64_t* coff = NULL;
    uint32_t* csrc = NULL;
    if (build_csc(n, off, col, &coff, &csrc)) return POMP_ENOMEM;
    float* outbox = (float*)malloc(sizeof(float) * (n ? n : 1));
    float* inv = (float*)malloc(sizeof(float) * (n ? n : 1));
    if (!outbox || !inv) {
        free(coff);
        free(csrc);
        free(outbox);
        free(inv);
        return POMP_ENOMEM;
    }
#pragma omp parallel for schedule(static)
    for (uint32_t v = 0; v < n; ++v) {
        const uint64_t d = off[v + 1] - off[v];
        inv[v] = d ? 1.0f / (float)d : 0.0f;
    }
    double t1 = omp_get_wtime();
    const float N = (float)n, base = 0.15f / N;
#pragma omp parallel for schedule(static)
    for (uint32_t v = 0; v < n; ++v) rank[v] = 1.0f / N;
    for (uint32_t t = 0; t < updates; ++t) {
#pragma omp parallel for schedule(static)
        for (uint32_t v = 0; v < n; ++v) outbox[v] = rank[v] * inv[v];
#pragma omp parallel for schedule(dynamic, 256)
        for (uint32_t v = 0; v < n; ++v) {
            float s = 0.0f;
            for (uint64_t e = coff[v]; e < coff[v + 1]; ++e) s += outbox[csrc[e]];
            rank[v] = base + 0.85f * s;
        }
    }
    double t2 = omp_get_wtime();
    free(coff);
    free(csrc);
    free(outbox);
    free(inv);
    if (msgs_out) *msgs_out = (uint64_t)updates * m;
    if (seconds_out) *seconds_out = t2 - t1;
    if (load_seconds_out) *load_seconds_out = t1 - t0;
    return POMP_OK;
}

/* append a thread's buffered vertex ids to a shared list with one atomic */
enum { kPompBuf = 1024 };
static uint32_t flush(const uint32_t* buf, uint32_t nb, uint32_t* list, uint64_t* count) {
    if (nb) {
        const uint64_t k = __atomic_fetch_add(count, (uint64_t)nb, __ATOMIC_RELAXED);
        memcpy(list + k, buf, sizeof(uint32_t) * nb);
    }
    return 0;
}

/* lower *p to v if v is smaller; returns 1 if this call lowered it */
static int cas_min(uint32_t* p, uint32_t v) {
    uint32_t cur = __atomic_load_n(p, __ATOMIC_RELAXED);
    while (v < cur) {
        if (__atomic_compare_exchange_n(p, &cur, v, 0, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) return 1;
    }
    return 0;
}

/*
 * SSSP, push form over the active list: superstep 0 activates the source with
 * distance 0; every active vertex sends dist + w along its out-edges into the
 * recipients' mailboxes (CAS minimum); at the barrier a recipient whose mailbox
 * is below its distance takes it and is active in the next superstep.  w = 1
 * when weights is NULL.  A distance that would reach UINT32_MAX is an error.
 */
int pomp_sssp(uint32_t n, const uint64_t* off, const uint32_t* col, const uint32_t* w, uint32_t source,
              uint32_t* dist, uint32_t* supersteps_out, uint64_t* msgs_out, double* seconds_out) {
    if (!off || source >= n || !dist) return POMP_EINVAL;
    uint32_t* mail = (uint32_t*)malloc(sizeof(uint32_t) * n);
    uint8_t* touched = (uint8_t*)calloc(n, 1);
    uint32_t* recv = (uint32_t*)malloc(sizeof(uint32_t) * n);
    uint32_t* front = (uint32_t*)malloc(sizeof(uint32_t) * n);
    if (!mail || !touched || !recv || !front) {
        free(mail);
        free(touched);
        free(recv);
        free(front);
        return POMP_ENOMEM;
    }
    int rc = POMP_OK;
    double t0 = omp_get_wtime();
#pragma omp parallel for schedule(static)
    for (uint32_t v = 0; v < n; ++v) {
        dist[v] = POMP_INF;
        mail[v] = POMP_INF;
    }
    dist[source] = 0;
    front[0] = source;
    uint64_t nf = 1, nrecv = 0, msgs = 0;
    uint32_t s = 0;
    int overflow = 0;
    for (;;) {
        uint64_t sent = 0;
        nrecv = 0;
#pragma omp parallel reduction(+ : sent) reduction(| : overflow)
        {
            uint32_t buf[kPompBuf];
            uint32_t nb = 0;
#pragma omp for schedule(dynamic, 256) nowait
            for (uint64_t i = 0; i < nf; ++i) {
                const uint32_t u = front[i];
                const uint64_t du = dist[u];
                for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
                    const uint32_t v = col[e];
                    uint64_t c = du + (w ? w[e] : 1u);
                    if (c >= POMP_INF) {
                        overflow = 1;
                        c = POMP_INF - 1;
                    }
                    cas_min(&mail[v], (uint32_t)c);
                    if (!__atomic_load_n(&touched[v], __ATOMIC_RELAXED) &&
                        !__atomic_exchange_n(&touched[v], 1, __ATOMIC_RELAXED)) {
                        buf[nb++] = v;
                        if (nb == kPompBuf) nb = flush(buf, nb, recv, &nrecv);
                    }
                }
                sent += off[u + 1] - off[u];
            }
            flush(buf, nb, recv, &nrecv);
        }
        msgs += sent;
        ++s;
        if (sent == 0) break;
        /* barrier: receivers whose mailbox is below their distance are the next senders */
        uint64_t nnext = 0;
#pragma omp parallel
        {
            uint32_t buf[kPompBuf];
            uint32_t nb = 0;
#pragma omp for schedule(dynamic, 256) nowait
            for (uint64_t i = 0; i < nrecv; ++i) {
                const uint32_t v = recv[i];
                touched[v] = 0;
                if (mail[v] < dist[v]) {
                    dist[v] = mail[v];
                    buf[nb++] = v;
                    if (nb == kPompBuf) nb = flush(buf, nb, front, &nnext);
                }
                mail[v] = POMP_INF;
            }
            flush(buf, nb, front, &nnext);
        }
        nf = nnext;
    }
    double t1 = omp_get_wtime();
    if (overflow) rc = POMP_EOVERFLOW;
    free(mail);
    free(touched);
    free(recv);
    free(front);
    if (supersteps_out) *supersteps_out = s;
    if (msgs_out) *msgs_out = msgs;
    if (seconds_out) *seconds_out = t1 - t0;
    return rc;
}

/*
 * Hashmin connected components, pull form, on an undirected graph (both
 * directions stored, so the in-neighbours are the row's own columns):
 * superstep 0 sets label = id and every vertex sends; in a later superstep a
 * vertex takes the minimum label of its in-neighbours that changed in the
 * previous superstep and, if that is smaller, adopts it and sends.
 */
int pomp_hashmin(uint32_t n, const uint64_t* off, const uint32_t* col, uint32_t* label, uint32_t* supersteps_out,
                 uint64_t* msgs_out, double* seconds_out) {
    if (!off || (n && !label)) return POMP_EINVAL;
    uint32_t* prev = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint8_t* act = (uint8_t*)malloc(n ? n : 1);
    uint8_t* act_next = (uint8_t*)malloc(n ? n : 1);
    if (!prev || !act || !act_next) {
        free(prev);
        free(act);
        free(act_next);
        return POMP_ENOMEM;
    }
    double t0 = omp_get_wtime();
#pragma omp parallel for schedule(static)
    for (uint32_t v = 0; v < n; ++v) {
        label[v] = v;
        act[v] = 1;
    }
    uint32_t s = 0;
    uint64_t msgs = 0;
    for (;;) {
        uint64_t sent = 0;
#pragma omp parallel for schedule(static) reduction(+ : sent)
        for (uint32_t v = 0; v < n; ++v)
            if (act[v]) sent += off[v + 1] - off[v];
        msgs += sent;
        ++s;
        if (sent == 0) break;
        memcpy(prev, label, sizeof(uint32_t) * n);
#pragma omp parallel for schedule(dynamic, 256)
        for (uint32_t v = 0; v < n; ++v) {
            uint32_t mn = POMP_INF;
            for (uint64_t e = off[v]; e < off[v + 1]; ++e) {
                const uint32_t u = col[e];
                if (act[u] && prev[u] < mn) mn = prev[u];
            }
            act_next[v] = mn < prev[v];
            if (mn < prev[v]) label[v] = mn;
        }
        uint8_t* t = act;
        act = act_next;
        act_next = t;
    }
    double t1 = omp_get_wtime();
    free(prev);
    free(act);
    free(act_next);
    if (supersteps_out) *supersteps_out = s;
    if (msgs_out) *msgs_out = msgs;
    if (seconds_out) *seconds_out = t1 - t0;
    return POMP_OK;
}

int pomp_threads(void) { return omp_get_max_threads(); }
