/*
 * Seeded synthetic graph inputs: R-MAT edge sampling and CSR assembly.
 *
 * This is an input tool shared by the tests, the benchmark and the oracle
 * side.  It holds none of the Pregel method's arithmetic: it only produces the
 * graphs (CSR offsets / columns / weights) that both the CUDA path and the CPU
 * oracle take as input.  The paper measures on four SNAP social graphs (Sec.
 * VI-B, Table I) that are not available here; R-MAT graphs with the same
 * power-law skew and the same orders of magnitude stand in for them.
 *
 * Random numbers come from one counter-based generator, splitmix64 (Vigna,
 * 2014): output(x) = mix(x + 0x9E3779B97F4A7C15) with the published
 * xor-shift-multiply finaliser.  Every draw is a pure function of
 * (seed, edge index, level pair), so the graph does not depend on the number
 * of threads that build it.
 *
 * R-MAT recipe (Chakrabarti et al., 2004):
 *   - EF * 2^scale raw edges; edge e draws ceil(scale/2) 64-bit words
 *     r_p = splitmix64(splitmix64(seed) + 16*e + p); each word gives two
 *     32-bit uniforms, one per recursion level, most significant level first.
 *   - level uniform x in [0, 2^32): x < A -> quadrant (0,0); x < A+B -> (0,1);
 *     x < A+B+C -> (1,0); else (1,1), with A, B, C the probabilities scaled
 *     to 2^32 and truncated.  Row bit goes to the source, column bit to the
 *     destination.  No noise, no vertex permutation: hubs sit at low ids.
 *   - self-loops are dropped; undirected graphs add the reverse of every
 *     edge; each row is sorted and duplicates are removed.
 * Weights: w(u,v) = 1 + splitmix64(splitmix64(wseed) ^ key) % wmax with
 *   key = u<<32 | v, or min<<32 | max for symmetric graphs so that both
 *   directions of an undirected edge carry the same weight.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define GEN_OK 0
#define GEN_EINVAL 1
#define GEN_ENOMEM 2

static inline uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t gen_splitmix64(uint64_t x) { return splitmix64(x); }

typedef struct {
    uint32_t scale, edge_factor;
    uint32_t ta, tab, tabc; /* quadrant thresholds on a 32-bit uniform */
    uint64_t base;          /* splitmix64(seed) */
    int undirected;
} rmat_cfg;

static inline void rmat_edge(const rmat_cfg* c, uint64_t e, uint32_t* pu, uint32_t* pv) {
    uint32_t u = 0, v = 0;
    uint32_t lvl = 0;
    for (uint32_t p = 0; lvl < c->scale; ++p) {
        uint64_t r = splitmix64(c->base + 16ull * e + p);
        for (int half = 0; half < 2 && lvl < c->scale; ++half, ++lvl) {
            uint32_t x = half == 0 ? (uint32_t)(r >> 32) : (uint32_t)r;
            uint32_t bit = 1u << (c->scale - 1 - lvl);
            if (x < c->ta) {
            } else if (x < c->tab) {
                v |= bit;
            } else if (x < c->tabc) {
                u |= bit;
            } else {
                u |= bit;
                v |= bit;
            }
        }
    }
    *pu = u;
    *pv = v;
}

static int pick_threads(int nthreads) {
    if (nthreads > 0) return nthreads > 256 ? 256 : nthreads;
    long k = sysconf(_SC_NPROCESSORS_ONLN);
    if (k < 1) k = 1;
    if (k > 64) k = 64;
    return (int)k;
}

/* ------------------------------------------------------------------------ */
/* plan: raw edges bucketed by source row, each row sorted and deduplicated   */

typedef struct gen_plan {
    uint32_t n;
    uint64_t m;          /* edges after dedup */
    uint64_t* raw_off;   /* n+1, bucket offsets of raw (pre-dedup) edges */
    uint32_t* raw_cols;  /* raw_off[n] entries, rows sorted, uniques first */
    uint32_t* uniq;      /* n, unique count per row */
    int nthreads;
} gen_plan;

typedef struct {
    const rmat_cfg* cfg;
    uint64_t e0, e1;
    uint32_t* cnt;       /* per-row atomic counters */
    const uint64_t* off; /* NULL in the count pass */
    uint32_t* cols;
} edge_job;

static void* edge_pass(void* arg) {
    edge_job* j = (edge_job*)arg;
    for (uint64_t e = j->e0; e < j->e1; ++e) {
        uint32_t u, v;
        rmat_edge(j->cfg, e, &u, &v);
        if (u == v) continue;
        if (j->off == NULL) {
            __atomic_fetch_add(&j->cnt[u], 1u, __ATOMIC_RELAXED);
            if (j->cfg->undirected) __atomic_fetch_add(&j->cnt[v], 1u, __ATOMIC_RELAXED);
        } else {
            uint32_t k = __atomic_fetch_add(&j->cnt[u], 1u, __ATOMIC_RELAXED);
            j->cols[j->off[u] + k] = v;
            if (j->cfg->undirected) {
                k = __atomic_fetch_add(&j->cnt[v], 1u, __ATOMIC_RELAXED);
                j->cols[j->off[v] + k] = u;
            }
        }
    }
    return NULL;
}

static int run_edge_pass(const rmat_cfg* cfg, int nt, uint32_t* cnt, const uint64_t* off, uint32_t* cols) {
    uint64_t total = (uint64_t)cfg->edge_factor << cfg->scale;
    pthread_t th[256];
    edge_job jobs[256];
    for (int t = 0; t < nt; ++t) {
        jobs[t].cfg = cfg;
        jobs[t].e0 = total * (uint64_t)t / (uint64_t)nt;
        jobs[t].e1 = total * (uint64_t)(t + 1) / (uint64_t)nt;
        jobs[t].cnt = cnt;
        jobs[t].off = off;
        jobs[t].cols = cols;
    }
    for (int t = 1; t < nt; ++t)
        if (pthread_create(&th[t], NULL, edge_pass, &jobs[t]) != 0) return GEN_ENOMEM;
    edge_pass(&jobs[0]);
    for (int t = 1; t < nt; ++t) pthread_join(th[t], NULL);
    return GEN_OK;
}

static int cmp_u32(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

/* sort one row ascending and move the distinct values to its front */
static uint32_t sort_unique(uint32_t* a, uint64_t len) {
    if (len == 0) return 0;
    if (len <= 32) {
        for (uint64_t i = 1; i < len; ++i) {
            uint32_t x = a[i];
            uint64_t k = i;
            while (k > 0 && a[k - 1] > x) {
                a[k] = a[k - 1];
                --k;
            }
            a[k] = x;
        }
    } else {
        qsort(a, (size_t)len, sizeof(uint32_t), cmp_u32);
    }
    uint64_t w = 1;
    for (uint64_t i = 1; i < len; ++i)
        if (a[i] != a[w - 1]) a[w++] = a[i];
    return (uint32_t)w;
}

typedef struct {
    gen_plan* p;
    uint32_t r0, r1;
} row_job;

static void* sort_rows(void* arg) {
    row_job* j = (row_job*)arg;
    for (uint32_t r = j->r0; r < j->r1; ++r)
        j->p->uniq[r] = sort_unique(j->p->raw_cols + j->p->raw_off[r], j->p->raw_off[r + 1] - j->p->raw_off[r]);
    return NULL;
}

/* split rows [0,n) into nt ranges of about equal edge count */
static void split_rows(const uint64_t* off, uint32_t n, int nt, uint32_t* bounds) {
    uint64_t total = off[n];
    bounds[0] = 0;
    for (int t = 1; t < nt; ++t) {
        uint64_t target = total * (uint64_t)t / (uint64_t)nt;
        uint32_t lo = bounds[t - 1], hi = n;
        while (lo < hi) { /* first row whose start offset is >= target */
            uint32_t mid = lo + (hi - lo) / 2;
            if (off[mid] < target) lo = mid + 1;
            else hi = mid;
        }
        bounds[t] = lo;
    }
    bounds[nt] = n;
}

int gen_rmat_plan(uint32_t scale, uint32_t edge_factor, double a, double b, double c, uint64_t seed,
                  int undirected, int nthreads, gen_plan** out, uint32_t* n_out, uint64_t* m_out) {
    if (!out || scale < 1 || scale > 31 || edge_factor < 1) return GEN_EINVAL;
    if (!(a >= 0 && b >= 0 && c >= 0 && a + b + c <= 1.0)) return GEN_EINVAL;
    uint64_t raw = (uint64_t)edge_factor << scale;
    if (raw * (undirected ? 2u : 1u) >= (1ull << 40)) return GEN_EINVAL;
    rmat_cfg cfg;
    cfg.scale = scale;
    cfg.edge_factor = edge_factor;
    cfg.ta = (uint32_t)(a * 4294967296.0);
    cfg.tab = (uint32_t)((a + b) * 4294967296.0);
    double abc = (a + b + c) * 4294967296.0;
    cfg.tabc = abc >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)abc;
    cfg.base = splitmix64(seed);
    cfg.undirected = undirected;

    int nt = pick_threads(nthreads);
    uint32_t n = 1u << scale;
    gen_plan* p = (gen_plan*)calloc(1, sizeof(gen_plan));
    if (!p) return GEN_ENOMEM;
    p->n = n;
    p->nthreads = nt;
    p->raw_off = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    p->uniq = (uint32_t*)calloc((size_t)n, sizeof(uint32_t));
    if (!p->raw_off || !p->uniq) goto oom;

    /* pass 1: count raw edges per row */
    if (run_edge_pass(&cfg, nt, p->uniq, NULL, NULL) != GEN_OK) goto oom;
    p->raw_off[0] = 0;
    for (uint32_t r = 0; r < n; ++r) p->raw_off[r + 1] = p->raw_off[r] + p->uniq[r];
    p->raw_cols = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(p->raw_off[n] ? p->raw_off[n] : 1));
    if (!p->raw_cols) goto oom;
    /* pass 2: regenerate and bucket */
    memset(p->uniq, 0, sizeof(uint32_t) * (size_t)n);
    if (run_edge_pass(&cfg, nt, p->uniq, p->raw_off, p->raw_cols) != GEN_OK) goto oom;
    /* pass 3: sort + dedup rows */
    {
        uint32_t bounds[257];
        split_rows(p->raw_off, n, nt, bounds);
        pthread_t th[256];
        row_job jobs[256];
        for (int t = 0; t < nt; ++t) {
            jobs[t].p = p;
            jobs[t].r0 = bounds[t];
            jobs[t].r1 = bounds[t + 1];
        }
        for (int t = 1; t < nt; ++t)
            if (pthread_create(&th[t], NULL, sort_rows, &jobs[t]) != 0) goto oom;
        sort_rows(&jobs[0]);
        for (int t = 1; t < nt; ++t) pthread_join(th[t], NULL);
    }
    {
        uint64_t m = 0;
        for (uint32_t r = 0; r < n; ++r) m += p->uniq[r];
        p->m = m;
    }
    *out = p;
    if (n_out) *n_out = n;
    if (m_out) *m_out = p->m;
    return GEN_OK;
oom:
    free(p->raw_off);
    free(p->raw_cols);
    free(p->uniq);
    free(p);
    return GEN_ENOMEM;
}

typedef struct {
    const gen_plan* p;
    const uint64_t* off;
    uint32_t* cols;
    uint32_t r0, r1;
} emit_job;

static void* emit_rows(void* arg) {
    emit_job* j = (emit_job*)arg;
    for (uint32_t r = j->r0; r < j->r1; ++r)
        memcpy(j->cols + j->off[r], j->p->raw_cols + j->p->raw_off[r], sizeof(uint32_t) * j->p->uniq[r]);
    return NULL;
}

/* write the deduplicated CSR into caller buffers: offsets[n+1], cols[m] */
int gen_plan_emit(const gen_plan* p, uint64_t* offsets, uint32_t* cols) {
    if (!p || !offsets || (!cols && p->m)) return GEN_EINVAL;
    uint32_t n = p->n;
    offsets[0] = 0;
    for (uint32_t r = 0; r < n; ++r) offsets[r + 1] = offsets[r] + p->uniq[r];
    int nt = p->nthreads;
    uint32_t bounds[257];
    split_rows(offsets, n, nt, bounds);
    pthread_t th[256];
    emit_job jobs[256];
    for (int t = 0; t < nt; ++t) {
        jobs[t].p = p;
        jobs[t].off = offsets;
        jobs[t].cols = cols;
        jobs[t].r0 = bounds[t];
        jobs[t].r1 = bounds[t + 1];
    }
    for (int t = 1; t < nt; ++t)
        if (pthread_create(&th[t], NULL, emit_rows, &jobs[t]) != 0) return GEN_ENOMEM;
    emit_rows(&jobs[0]);
    for (int t = 1; t < nt; ++t) pthread_join(th[t], NULL);
    return GEN_OK;
}

void gen_plan_free(gen_plan* p) {
    if (!p) return;
    free(p->raw_off);
    free(p->raw_cols);
    free(p->uniq);
    free(p);
}

/* ------------------------------------------------------------------------ */
/* weights from endpoints                                                      */

typedef struct {
    const uint64_t* off;
    const uint32_t* cols;
    uint32_t* w;
    uint64_t base;
    uint32_t wmax;
    int symmetric;
    uint32_t r0, r1;
} w_job;

static void* weight_rows(void* arg) {
    w_job* j = (w_job*)arg;
    for (uint32_t u = j->r0; u < j->r1; ++u) {
        for (uint64_t e = j->off[u]; e < j->off[u + 1]; ++e) {
            uint32_t v = j->cols[e];
            uint32_t lo = u, hi = v;
            if (j->symmetric && lo > hi) {
                lo = v;
                hi = u;
            }
            uint64_t key = ((uint64_t)lo << 32) | hi;
            j->w[e] = 1u + (uint32_t)(splitmix64(j->base ^ key) % j->wmax);
        }
    }
    return NULL;
}

int gen_weights(uint32_t n, const uint64_t* offsets, const uint32_t* cols, uint64_t weight_seed, uint32_t wmax,
                int symmetric, int nthreads, uint32_t* weights) {
    if (!offsets || wmax < 1) return GEN_EINVAL;
    if (offsets[n] && (!cols || !weights)) return GEN_EINVAL;
    int nt = pick_threads(nthreads);
    uint32_t bounds[257];
    split_rows(offsets, n, nt, bounds);
    pthread_t th[256];
    w_job jobs[256];
    for (int t = 0; t < nt; ++t) {
        jobs[t].off = offsets;
        jobs[t].cols = cols;
        jobs[t].w = weights;
        jobs[t].base = splitmix64(weight_seed);
        jobs[t].wmax = wmax;
        jobs[t].symmetric = symmetric;
        jobs[t].r0 = bounds[t];
        jobs[t].r1 = bounds[t + 1];
    }
    for (int t = 1; t < nt; ++t)
        if (pthread_create(&th[t], NULL, weight_rows, &jobs[t]) != 0) return GEN_ENOMEM;
    weight_rows(&jobs[0]);
    for (int t = 1; t < nt; ++t) pthread_join(th[t], NULL);
    return GEN_OK;
}
