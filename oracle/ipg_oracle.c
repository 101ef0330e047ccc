/*
 * ORACLE — test infrastructure only.
 *
 * A plain, slow, single-threaded CPU Pregel implementation used to check the
 * CUDA path.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * and reference legs may load it; the library never does.  It shares no code,
 * header or constant with the CUDA path.
 *
 * Execution model (Sec. I, the Pregel description): all vertices start
 * active; in a superstep the user function runs on every active vertex; it may
 * send messages along its out-edges and votes to halt; messages are delivered
 * at the end of the superstep, and a vertex that receives at least one message
 * is active in the next superstep.  Execution stops when no message is in
 * flight (every vertex has halted).
 *
 * Mailbox (Sec. III): each vertex holds, for the next superstep, a flag that
 * says whether any message arrived and the message itself; the first message
 * is stored and the flag raised, every later one is combined into the stored
 * message with the user's combine function (min for Hashmin and SSSP, sum for
 * PageRank).  The flag is what lets a receiver tell "no message" apart from a
 * combined value that happens to equal the combine's neutral element.
 *
 * Messages are delivered in the order they are sent: vertices in increasing id,
 * each along its out-edges in CSR order.  Sums are taken in that order in
 * double precision.
 *
 * Benchmarks (Sec. VI-C): PageRank, connected components, single-source
 * shortest paths.  The paper gives no PageRank formula; the one used here is
 * rank = 0.15/N + 0.85 * (sum of incoming messages), message = rank/outdeg,
 * initial rank 1/N, dangling vertices (out-degree 0) send nothing.  Connected
 * components is Hashmin (labels = vertex ids, min combiner).  SSSP sends
 * dist + w along each edge with a min combiner; without weights every edge
 * has length 1, the paper's unweighted SSSP.
 *
 * Parity pins: closed forms (PageRank on cycles and stars), library routines
 * (connected components, Dijkstra, BFS from scipy), the PageRank fixed point
 * (a dense linear solve), the superstep-count and per-superstep count closed
 * forms, and the rank-mass identity; see tests/test_oracle_pins.py.  The
 * general-combiner functions (orc_combine, orc_sssp_tree, orc_bfs_paths) are
 * pinned by numpy ufunc reductions, the parent rule written out from Dijkstra
 * distances, the shortest-path-count recurrence, grid and hypercube closed
 * forms, networkx path enumeration and the modulo-2^64 wrap of a diamond
 * chain; see tests/test_oracle_pins_combiner.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_EOVERFLOW 3

#define ORC_INF 0xFFFFFFFFu

/* one record per superstep */
typedef struct {
    uint32_t superstep;
    uint32_t reserved;
    uint64_t active;        /* vertices that ran the user function */
    uint64_t senders;       /* vertices that broadcast to their out-neighbours */
    uint64_t messages_sent; /* messages sent (sum of the senders' out-degrees) */
    uint64_t receivers;     /* distinct vertices that received >= 1 of them */
} orc_stats;

static void record(orc_stats* st, uint32_t cap, uint32_t s, uint64_t active, uint64_t senders, uint64_t msgs,
                   uint64_t receivers) {
    if (st && s < cap) {
        st[s].superstep = s;
        st[s].reserved = 0;
        st[s].active = active;
        st[s].senders = senders;
        st[s].messages_sent = msgs;
        st[s].receivers = receivers;
    }
}

static int check_csr(uint32_t n, const uint64_t* off, const uint32_t* col) {
    if (!off) return ORC_EINVAL;
    if (off[0] != 0) return ORC_EINVAL;
    for (uint32_t v = 0; v < n; ++v)
        if (off[v + 1] < off[v]) return ORC_EINVAL;
    if (off[n] && !col) return ORC_EINVAL;
    for (uint64_t e = 0; e < off[n]; ++e)
        if (col[e] >= n) return ORC_EINVAL;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* mailboxes with a min combiner (u32 messages)                              */

typedef struct {
    uint32_t* msg;      /* messages delivered for this superstep */
    uint8_t* has;       /* flag: a message was delivered */
    uint32_t* msg_next; /* messages being combined for the next superstep */
    uint8_t* has_next;
    uint64_t sent;      /* messages sent in the current superstep */
} min_mailboxes;

static void send_min(min_mailboxes* mb, uint32_t dst, uint32_t msg) {
    mb->sent++;
    if (mb->has_next[dst]) {
        if (msg < mb->msg_next[dst]) mb->msg_next[dst] = msg;
    } else {
        mb->msg_next[dst] = msg;
        mb->has_next[dst] = 1;
    }
}

/* end of superstep: deliver the combined messages, return how many vertices got one */
static uint64_t deliver_min(min_mailboxes* mb, uint32_t n) {
    uint32_t* tm = mb->msg;
    mb->msg = mb->msg_next;
    mb->msg_next = tm;
    uint8_t* th = mb->has;
    mb->has = mb->has_next;
    mb->has_next = th;
    memset(mb->has_next, 0, n);
    uint64_t r = 0;
    for (uint32_t v = 0; v < n; ++v) r += mb->has[v];
    return r;
}

static int alloc_min(min_mailboxes* mb, uint32_t n) {
    size_t k = n ? n : 1;
    mb->msg = (uint32_t*)calloc(k, sizeof(uint32_t));
    mb->msg_next = (uint32_t*)calloc(k, sizeof(uint32_t));
    mb->has = (uint8_t*)calloc(k, 1);
    mb->has_next = (uint8_t*)calloc(k, 1);
    mb->sent = 0;
    return (mb->msg && mb->msg_next && mb->has && mb->has_next) ? ORC_OK : ORC_ENOMEM;
}

static void free_min(min_mailboxes* mb) {
    free(mb->msg);
    free(mb->msg_next);
    free(mb->has);
    free(mb->has_next);
}

/*
 * Hashmin connected components.
 * compute(v), superstep 0: value = id(v), send it to every out-neighbour.
 * compute(v), superstep s > 0: m = combined (minimum) message; if m < value,
 *   value = m and send it to every out-neighbour.  Always vote to halt.
 * On an undirected graph (both directions stored) the result is the smallest
 * vertex id of each connected component (Sec. VI-C, CC).
 * max_supersteps = 0 means no limit.
 */
int orc_hashmin(uint32_t n, const uint64_t* off, const uint32_t* col, uint32_t* label, orc_stats* st, uint32_t cap,
                uint32_t max_supersteps, uint32_t* supersteps_out) {
    int rc = check_csr(n, off, col);
    if (rc) return rc;
    if (n && !label) return ORC_EINVAL;
    min_mailboxes mb;
    if (alloc_min(&mb, n)) {
        free_min(&mb);
        return ORC_ENOMEM;
    }
    uint32_t s = 0;
    uint64_t active = n;
    for (;;) {
        uint64_t senders = 0;
        mb.sent = 0;
        for (uint32_t v = 0; v < n; ++v) {
            int runs = (s == 0) || mb.has[v];
            if (!runs) continue;
            int changed;
            if (s == 0) {
                label[v] = v;
                changed = 1;
            } else {
                changed = mb.msg[v] < label[v];
                if (changed) label[v] = mb.msg[v];
            }
            if (changed) {
                senders++;
                for (uint64_t e = off[v]; e < off[v + 1]; ++e) send_min(&mb, col[e], label[v]);
            }
        }
        uint64_t sent = mb.sent;
        uint64_t receivers = deliver_min(&mb, n);
        record(st, cap, s, active, senders, sent, receivers);
        s++;
        if (sent == 0) break;
        if (max_supersteps && s >= max_supersteps) break;
        active = receivers;
    }
    if (supersteps_out) *supersteps_out = s;
    free_min(&mb);
    return ORC_OK;
}

/*
 * Single-source shortest paths (Sec. VI-C, SSSP).
 * Every value starts at infinity (0xFFFFFFFF, "unreached").
 * compute(v), superstep 0: candidate = 0 if v is the source, else infinity.
 * compute(v), superstep s > 0: candidate = combined (minimum) message.
 * If candidate < value: value = candidate and send value + w(v,u) to every
 * out-neighbour u (w = 1 when the graph has no weights).  Vote to halt.
 * value + w is formed in 64 bits; a sum that does not fit below infinity is
 * reported as ORC_EOVERFLOW instead of wrapping.
 */
int orc_sssp(uint32_t n, const uint64_t* off, const uint32_t* col, const uint32_t* w, uint32_t source, uint32_t* dist,
             orc_stats* st, uint32_t cap, uint32_t max_supersteps, uint32_t* supersteps_out) {
    int rc = check_csr(n, off, col);
    if (rc) return rc;
    if (source >= n || !dist) return ORC_EINVAL;
    min_mailboxes mb;
    if (alloc_min(&mb, n)) {
        free_min(&mb);
        return ORC_ENOMEM;
    }
    for (uint32_t v = 0; v < n; ++v) dist[v] = ORC_INF;
    uint32_t s = 0;
    uint64_t active = n;
    rc = ORC_OK;
    for (;;) {
        uint64_t senders = 0;
        mb.sent = 0;
        for (uint32_t v = 0; v < n; ++v) {
            int runs = (s == 0) || mb.has[v];
            if (!runs) continue;
            uint32_t cand = (s == 0) ? (v == source ? 0u : ORC_INF) : mb.msg[v];
            if (cand < dist[v]) {
                dist[v] = cand;
                senders++;
                for (uint64_t e = off[v]; e < off[v + 1]; ++e) {
                    uint64_t len = w ? (uint64_t)w[e] : 1u;
                    uint64_t d = (uint64_t)dist[v] + len;
                    if (d >= ORC_INF) rc = ORC_EOVERFLOW;
                    send_min(&mb, col[e], (uint32_t)(d >= ORC_INF ? ORC_INF - 1 : d));
                }
            }
        }
        uint64_t sent = mb.sent;
        uint64_t receivers = deliver_min(&mb, n);
        record(st, cap, s, active, senders, sent, receivers);
        s++;
        if (sent == 0) break;
        if (max_supersteps && s >= max_supersteps) break;
        active = receivers;
    }
    if (supersteps_out) *supersteps_out = s;
    free_min(&mb);
    return rc;
}

/*
 * PageRank (Sec. VI-C, PR) with `updates` rank updates.
 * compute(v), superstep 0: rank = 1/N; send rank/outdeg(v) to every
 *   out-neighbour (a vertex with no out-edge sends nothing: its mass is lost).
 * compute(v), superstep t in 1..updates: rank = 0.15/N + 0.85 * S, where S is
 *   the combined (summed) message, or 0 if no message arrived; if t < updates
 *   send rank/outdeg(v) again, otherwise halt.
 * Every vertex runs in every superstep (none halts before the last one).
 * Returns rank after `updates` updates; updates + 1 supersteps run.
 */
int orc_pagerank(uint32_t n, const uint64_t* off, const uint32_t* col, uint32_t updates, double* rank, orc_stats* st,
                 uint32_t cap, uint32_t* supersteps_out) {
    int rc = check_csr(n, off, col);
    if (rc) return rc;
    if (n && !rank) return ORC_EINVAL;
    size_t k = n ? n : 1;
    double* msg = (double*)calloc(k, sizeof(double));
    double* msg_next = (double*)calloc(k, sizeof(double));
    uint8_t* has = (uint8_t*)calloc(k, 1);
    uint8_t* has_next = (uint8_t*)calloc(k, 1);
    if (!msg || !msg_next || !has || !has_next) {
        free(msg);
        free(msg_next);
        free(has);
        free(has_next);
        return ORC_ENOMEM;
    }
    const double N = (double)n;
    uint32_t s;
    for (s = 0; s <= updates; ++s) {
        uint64_t senders = 0, sent = 0;
        for (uint32_t v = 0; v < n; ++v) {
            if (s == 0)
                rank[v] = 1.0 / N;
            else
                rank[v] = 0.15 / N + 0.85 * (has[v] ? msg[v] : 0.0);
            if (s < updates) {
                uint64_t outdeg = off[v + 1] - off[v];
                senders++;
                for (uint64_t e = off[v]; e < off[v + 1]; ++e) {
                    uint32_t u = col[e];
                    double m = rank[v] / (double)outdeg;
                    sent++;
                    if (has_next[u]) {
                        msg_next[u] += m;
                    } else {
                        msg_next[u] = m;
                        has_next[u] = 1;
                    }
                }
            }
        }
        /* deliver */
        double* tm = msg;
        msg = msg_next;
        msg_next = tm;
        uint8_t* th = has;
        has = has_next;
        has_next = th;
        memset(has_next, 0, k);
        uint64_t receivers = 0;
        for (uint32_t v = 0; v < n; ++v) receivers += has[v];
        record(st, cap, s, n, senders, sent, receivers);
    }
    if (supersteps_out) *supersteps_out = s;
    free(msg);
    free(msg_next);
    free(has);
    free(has_next);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* mailboxes with an arbitrary combine function and messages of up to 16    */
/* bytes (Sec. III, the hybrid combiner of Fig. 1).  Sequentially there is   */
/* no race, so the lock and the compare-and-swap reduce to their meaning:    */
/* the first message is stored and the flag raised, every later message is   */
/* combined into the stored one.                                             */

typedef struct {
    uint64_t a, b; /* the message's fields; which are used depends on the kind */
} orc_msg;

typedef orc_msg (*orc_combine_fn)(orc_msg x, orc_msg y);

/* kinds of orc_combine */
#define ORC_COMBINE_XOR_U32 0      /* 4-byte messages, bitwise exclusive or */
#define ORC_COMBINE_MIN_U64 1      /* 8-byte messages, minimum */
#define ORC_COMBINE_SUM_U64 2      /* 8-byte messages, sum modulo 2^64 */
#define ORC_COMBINE_MINCOUNT_U128 3 /* 16-byte (key, count): smallest key, counts of equal keys added */

static orc_msg comb_xor32(orc_msg x, orc_msg y) {
    orc_msg r = {(uint32_t)(x.a ^ y.a), 0};
    return r;
}
static orc_msg comb_min64(orc_msg x, orc_msg y) { return x.a <= y.a ? x : y; }
static orc_msg comb_sum64(orc_msg x, orc_msg y) {
    orc_msg r = {x.a + y.a, 0};
    return r;
}
static orc_msg comb_mincount(orc_msg x, orc_msg y) {
    if (x.a < y.a) return x;
    if (y.a < x.a) return y;
    orc_msg r = {x.a, x.b + y.b};
    return r;
}

typedef struct {
    orc_msg* msg_next;
    uint8_t* has_next;
    orc_combine_fn combine;
    uint64_t sent;
} gen_mailboxes;

static void send_gen(gen_mailboxes* mb, uint32_t dst, orc_msg m) {
    mb->sent++;
    if (mb->has_next[dst]) {
        mb->msg_next[dst] = mb->combine(mb->msg_next[dst], m);
    } else {
        mb->msg_next[dst] = m;
        mb->has_next[dst] = 1;
    }
}

static size_t kind_size(int kind) {
    switch (kind) {
        case ORC_COMBINE_XOR_U32: return 4;
        case ORC_COMBINE_MIN_U64: return 8;
        case ORC_COMBINE_SUM_U64: return 8;
        case ORC_COMBINE_MINCOUNT_U128: return 16;
        default: return 0;
    }
}

/*
 * Deliver k messages, message i to vertex dst[i], into n empty mailboxes, in
 * the order given.  msgs holds k records of the kind's size (4, 8 or 16 bytes,
 * little-endian; a 16-byte record is (key u64, count u64)).  On return has[v]
 * is 1 if vertex v received at least one message, and mail[v] (a record of
 * the kind's size) holds the combined message; mail[v] is left untouched where
 * has[v] is 0.  *receivers_out = number of vertices with has[v] = 1.
 */
int orc_combine(int kind, uint32_t n, uint64_t k, const uint32_t* dst, const void* msgs, uint8_t* has, void* mail,
                uint64_t* receivers_out) {
    size_t sz = kind_size(kind);
    if (!sz) return ORC_EINVAL;
    if (k && (!dst || !msgs)) return ORC_EINVAL;
    if (n && (!has || !mail)) return ORC_EINVAL;
    for (uint64_t i = 0; i < k; ++i)
        if (dst[i] >= n) return ORC_EINVAL;
    gen_mailboxes mb;
    mb.msg_next = (orc_msg*)calloc(n ? n : 1, sizeof(orc_msg));
    mb.has_next = has;
    mb.sent = 0;
    if (!mb.msg_next) return ORC_ENOMEM;
    switch (kind) {
        case ORC_COMBINE_XOR_U32: mb.combine = comb_xor32; break;
        case ORC_COMBINE_MIN_U64: mb.combine = comb_min64; break;
        case ORC_COMBINE_SUM_U64: mb.combine = comb_sum64; break;
        default: mb.combine = comb_mincount; break;
    }
    memset(has, 0, n);
    const unsigned char* in = (const unsigned char*)msgs;
    for (uint64_t i = 0; i < k; ++i) {
        orc_msg m = {0, 0};
        if (sz == 4) {
            uint32_t x;
            memcpy(&x, in + i * 4, 4);
            m.a = x;
        } else if (sz == 8) {
            memcpy(&m.a, in + i * 8, 8);
        } else {
            memcpy(&m.a, in + i * 16, 8);
            memcpy(&m.b, in + i * 16 + 8, 8);
        }
        send_gen(&mb, dst[i], m);
    }
    uint64_t r = 0;
    unsigned char* out = (unsigned char*)mail;
    for (uint32_t v = 0; v < n; ++v) {
        if (!has[v]) continue;
        r++;
        if (sz == 4) {
            uint32_t x = (uint32_t)mb.msg_next[v].a;
            memcpy(out + (size_t)v * 4, &x, 4);
        } else if (sz == 8) {
            memcpy(out + (size_t)v * 8, &mb.msg_next[v].a, 8);
        } else {
            memcpy(out + (size_t)v * 16, &mb.msg_next[v].a, 8);
            memcpy(out + (size_t)v * 16 + 8, &mb.msg_next[v].b, 8);
        }
    }
    if (receivers_out) *receivers_out = r;
    free(mb.msg_next);
    return ORC_OK;
}

/* lexicographic order on (distance, parent) pairs held in a message's a and b */
static orc_msg comb_lexmin(orc_msg x, orc_msg y) {
    if (x.a != y.a) return x.a < y.a ? x : y;
    return x.b <= y.b ? x : y;
}

/*
 * Shortest-path tree: SSSP (Sec. VI-C) whose message carries the sender's id
 * as well as the distance, combined by the lexicographic minimum of
 * (distance, sender).
 * State of v: (dist, parent), initially (infinity, infinity).
 * compute(v), superstep 0: the source takes (0, source) and sends.
 * compute(v), superstep s > 0: (d, p) = combined message; if (d, p) is
 *   lexicographically below (dist, parent) the state becomes (d, p); if the
 *   distance itself dropped, send (dist + w(v,u), v) to every out-neighbour u.
 *   Vote to halt.
 * The senders are exactly those of orc_sssp, so the superstep count and every
 * per-superstep count equal SSSP's.  The final parent of a reached vertex v
 * other than the source is the smallest u with an edge u -> v and
 * dist[u] + w(u,v) = dist[v]; the source's parent is itself; an unreached
 * vertex keeps (infinity, infinity).
 */
int orc_sssp_tree(uint32_t n, const uint64_t* off, const uint32_t* col, const uint32_t* w, uint32_t source,
                  uint32_t* dist, uint32_t* parent, orc_stats* st, uint32_t cap, uint32_t max_supersteps,
                  uint32_t* supersteps_out) {
    int rc = check_csr(n, off, col);
    if (rc) return rc;
    if (source >= n || !dist || !parent) return ORC_EINVAL;
    size_t k = n ? n : 1;
    gen_mailboxes mb;
    orc_msg* msg = (orc_msg*)calloc(k, sizeof(orc_msg));
    uint8_t* has = (uint8_t*)calloc(k, 1);
    mb.msg_next = (orc_msg*)calloc(k, sizeof(orc_msg));
    mb.has_next = (uint8_t*)calloc(k, 1);
    mb.combine = comb_lexmin;
    if (!msg || !has || !mb.msg_next || !mb.has_next) {
        free(msg);
        free(has);
        free(mb.msg_next);
        free(mb.has_next);
        return ORC_ENOMEM;
    }
    for (uint32_t v = 0; v < n; ++v) {
        dist[v] = ORC_INF;
        parent[v] = ORC_INF;
    }
    uint32_t s = 0;
    uint64_t active = n;
    rc = ORC_OK;
    for (;;) {
        uint64_t senders = 0;
        mb.sent = 0;
        for (uint32_t v = 0; v < n; ++v) {
            int runs = (s == 0) || has[v];
            if (!runs) continue;
            orc_msg cand;
            if (s == 0) {
                cand.a = v == source ? 0u : ORC_INF;
                cand.b = v == source ? source : ORC_INF;
            } else {
                cand = msg[v];
            }
            int lower = cand.a < dist[v] || (cand.a == dist[v] && cand.b < parent[v]);
            if (!lower) continue;
            int dist_dropped = cand.a < dist[v];
            dist[v] = (uint32_t)cand.a;
            parent[v] = (uint32_t)cand.b;
            if (!dist_dropped) continue;
            senders++;
            for (uint64_t e = off[v]; e < off[v + 1]; ++e) {
                uint64_t len = w ? (uint64_t)w[e] : 1u;
                uint64_t d = (uint64_t)dist[v] + len;
                if (d >= ORC_INF) {
                    rc = ORC_EOVERFLOW;
                    d = ORC_INF - 1;
                }
                orc_msg m = {d, v};
                send_gen(&mb, col[e], m);
            }
        }
        uint64_t sent = mb.sent;
        /* deliver */
        orc_msg* tm = msg;
        msg = mb.msg_next;
        mb.msg_next = tm;
        uint8_t* th = has;
        has = mb.has_next;
        mb.has_next = th;
        memset(mb.has_next, 0, k);
        uint64_t receivers = 0;
        for (uint32_t v = 0; v < n; ++v) receivers += has[v];
        record(st, cap, s, active, senders, sent, receivers);
        s++;
        if (sent == 0) break;
        if (max_supersteps && s >= max_supersteps) break;
        active = receivers;
    }
    if (supersteps_out) *supersteps_out = s;
    free(msg);
    free(has);
    free(mb.msg_next);
    free(mb.has_next);
    return rc;
}

/*
 * Shortest-path counting by breadth-first levels: each message carries
 * (level, number of paths) and the combine keeps the smallest level and adds
 * the counts of messages at that level (ORC_COMBINE_MINCOUNT_U128).  Edges
 * have length 1 whatever the graph's weights; every edge is one message, so
 * parallel edges count as distinct paths.  Counts are taken modulo 2^64.
 * State of v: (level, paths), initially (infinity, 0).
 * compute(v), superstep 0: the source takes (0, 1) and sends.
 * compute(v), superstep s > 0: if v has no level yet, it takes the combined
 *   message as its state and sends (level + 1, paths) to every out-neighbour.
 *   Vote to halt.
 * Result: level = hop distance from the source (infinity if unreached), paths
 * = number of shortest paths from the source modulo 2^64 (0 if unreached).
 */
int orc_bfs_paths(uint32_t n, const uint64_t* off, const uint32_t* col, uint32_t source, uint32_t* level,
                  uint64_t* paths, orc_stats* st, uint32_t cap, uint32_t max_supersteps, uint32_t* supersteps_out) {
    int rc = check_csr(n, off, col);
    if (rc) return rc;
    if (source >= n || !level || !paths) return ORC_EINVAL;
    size_t k = n ? n : 1;
    gen_mailboxes mb;
    orc_msg* msg = (orc_msg*)calloc(k, sizeof(orc_msg));
    uint8_t* has = (uint8_t*)calloc(k, 1);
    mb.msg_next = (orc_msg*)calloc(k, sizeof(orc_msg));
    mb.has_next = (uint8_t*)calloc(k, 1);
    mb.combine = comb_mincount;
    if (!msg || !has || !mb.msg_next || !mb.has_next) {
        free(msg);
        free(has);
        free(mb.msg_next);
        free(mb.has_next);
        return ORC_ENOMEM;
    }
    for (uint32_t v = 0; v < n; ++v) {
        level[v] = ORC_INF;
        paths[v] = 0;
    }
    uint32_t s = 0;
    uint64_t active = n;
    for (;;) {
        uint64_t senders = 0;
        mb.sent = 0;
        for (uint32_t v = 0; v < n; ++v) {
            int runs = (s == 0) || has[v];
            if (!runs) continue;
            if (s == 0) {
                if (v != source) continue;
                level[v] = 0;
                paths[v] = 1;
            } else {
                if (level[v] != ORC_INF) continue;
                level[v] = (uint32_t)msg[v].a;
                paths[v] = msg[v].b;
            }
            senders++;
            for (uint64_t e = off[v]; e < off[v + 1]; ++e) {
                orc_msg m = {(uint64_t)level[v] + 1, paths[v]};
                send_gen(&mb, col[e], m);
            }
        }
        uint64_t sent = mb.sent;
        orc_msg* tm = msg;
        msg = mb.msg_next;
        mb.msg_next = tm;
        uint8_t* th = has;
        has = mb.has_next;
        mb.has_next = th;
        memset(mb.has_next, 0, k);
        uint64_t receivers = 0;
        for (uint32_t v = 0; v < n; ++v) receivers += has[v];
        record(st, cap, s, active, senders, sent, receivers);
        s++;
        if (sent == 0) break;
        if (max_supersteps && s >= max_supersteps) break;
        active = receivers;
    }
    if (supersteps_out) *supersteps_out = s;
    free(msg);
    free(has);
    free(mb.msg_next);
    free(mb.has_next);
    return ORC_OK;
}
