/*
 * Oracle for Cluster-BFS (C-BFS) and the landmark-label query.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, sequential CPU
 * restatement of what the paper ("Parallel Cluster-BFS and Applications to
 * Shortest Paths", arXiv 2410.17226) computes.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or helper with the CUDA library, and the
 * CUDA library never calls it.
 *
 * Conventions (shared with the CUDA path only through the documented output
 * format, never through code):
 *   - graph: CSR, off[n+1] int64, adj[nnz] int32, undirected graphs stored
 *     with both arc directions;
 *   - cluster S = (S[0], ..., S[k-1]), k in [1,64]; bit j (LSB = 0) of a
 *     64-bit word stands for S[j]; ALL = the k low bits;
 *   - output dist[v] = Delta_v = min_j delta(S[j], v) as one byte, 0xFF when
 *     no source reaches v; masks[i*n + v] = S_v[i] for i in [0, d) (the last
 *     subset S_v[d] is implied: ALL minus the stored ones when reachable).
 *
 * Functions:
 *   oracle_bfs            textbook single-source BFS (Appendix A, parallel BFS
 *                         framework, run sequentially).
 *   oracle_cbfs_definition  O1: the definition of the cluster distance vector
 *                         (Section 3.1, the equation defining S_v[i]) computed
 *                         from k independent BFSs.
 *   oracle_cbfs_alg1      O2: Algorithm 1 (Section 3.2) executed sequentially,
 *                         with work counters (Theorem 1).
 *   oracle_certify        exact certificate for a C-BFS output (Bellman
 *                         fixpoint of BFS distances), O(k * m).
 *   oracle_query          landmark-labeling query (Section 4.2, Algorithm
 *                         "Framework of Landmark Labeling"): min over all
 *                         landmarks of delta(u,s) + delta(s,v), decoded from
 *                         the cluster outputs.
 *   oracle_local_search   the bounded bidirectional search added to queries
 *                         (Appendix B): BFS balls of at most tau vertices
 *                         around u and v (whole levels), min over common
 *                         vertices of the two hop counts.
 *
 * Return codes: 0 ok; -1 invalid argument; -2 some vertex sees source
 * distances spread wider than d (the cluster diameter bound of Corollary 1
 * is violated); -3 some Delta_v would be >= 255 (does not fit one byte,
 * Section 3.1 assumes D < 256); -4 out of memory.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_INVALID (-1)
#define OR_DIAMETER (-2)
#define OR_DEPTH (-3)
#define OR_NOMEM (-4)

static uint64_t all_bits(int k) { return k >= 64 ? ~0ull : ((1ull << k) - 1ull); }

static int check_cluster(int64_t n, const int32_t* S, int k, int d) {
    if (k < 1 || k > 64 || d < 0 || d > 15) return OR_INVALID;
    for (int j = 0; j < k; ++j) {
        if (S[j] < 0 || (int64_t)S[j] >= n) return OR_INVALID;
        for (int i = 0; i < j; ++i)
            if (S[i] == S[j]) return OR_INVALID;
    }
    return OR_OK;
}

/* Textbook queue BFS from src.  dist[v] = hop count, -1 when unreachable. */
int oracle_bfs(int64_t n, const int64_t* off, const int32_t* adj, int32_t src, int32_t* dist) {
    if (n <= 0 || src < 0 || (int64_t)src >= n) return OR_INVALID;
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!queue) return OR_NOMEM;
    for (int64_t v = 0; v < n; ++v) dist[v] = -1;
    int64_t head = 0, tail = 0;
    dist[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
            int32_t v = adj[e];
            if (dist[v] < 0) {
                dist[v] = dist[u] + 1;
                queue[tail++] = v;
            }
        }
    }
    free(queue);
    return OR_OK;
}

/*
 * O1 -- the definition (Section 3.1).  Delta_v = min over sources of
 * delta(s, v); S_v[i] = { s : delta(s, v) = Delta_v + i }.  The k distances
 * come from k independent textbook BFSs.
 */
int oracle_cbfs_definition(int64_t n, const int64_t* off, const int32_t* adj, const int32_t* S,
                           int k, int d, uint8_t* dist, uint64_t* masks) {
    int rc = check_cluster(n, S, k, d);
    if (rc) return rc;
    int32_t* delta = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * (size_t)k);
    if (!delta) return OR_NOMEM;
    for (int j = 0; j < k; ++j) {
        rc = oracle_bfs(n, off, adj, S[j], delta + (size_t)j * (size_t)n);
        if (rc) { free(delta); return rc; }
    }
    rc = OR_OK;
    for (int64_t v = 0; v < n; ++v) {
        int32_t lo = -1, hi = -1;
        for (int j = 0; j < k; ++j) {
            int32_t x = delta[(size_t)j * (size_t)n + v];
            if (x < 0) continue;
            if (lo < 0 || x < lo) lo = x;
            if (hi < 0 || x > hi) hi = x;
        }
        for (int i = 0; i < d; ++i) masks[(size_t)i * (size_t)n + v] = 0;
        if (lo < 0) { dist[v] = 0xFF; continue; }
        if (hi - lo > d) rc = OR_DIAMETER;
        if (lo >= 255) { rc = OR_DEPTH; dist[v] = 0xFF; continue; }
        dist[v] = (uint8_t)lo;
        for (int j = 0; j < k; ++j) {
            int32_t x = delta[(size_t)j * (size_t)n + v];
            if (x < 0) { rc = OR_DIAMETER; continue; } /* some source misses v: not one cluster */
            int32_t i = x - lo;
            if (i < d) masks[(size_t)i * (size_t)n + v] |= (1ull << j);
        }
    }
    free(delta);
    return rc;
}

/*
 * O2 -- Algorithm 1 (Section 3.2), executed one step at a time on one core.
 *
 * Readings of the printed algorithm (each documented with the design notes):
 *   (1) initialisation: Snext[S[j]] = {S[j]}, Sseen empty, so that round 0
 *       records S_s[0] = {s};
 *   (2) the output is S_v[0..d] (the last one implied);
 *   (3) the compare-and-swap on r[v] is a once-per-round claim: the first
 *       pusher that grows Snext[v] in round i appends v to F_{i+1};
 *   (4) Fetch_And_Or reports whether it set any new bit;
 *   (5) the edge condition is i - Delta_v < d, with Delta_v = infinity passing.
 * counters (may be NULL): [0] = sum_i |F_i| (frontier appearances),
 * [1] = sum_i sum_{u in F_i} deg(u) (arcs scanned), [2] = number of rounds,
 * [3] = sum over reached v of deg(v) (arcs of the reached part).
 */
int oracle_cbfs_alg1(int64_t n, const int64_t* off, const int32_t* adj, const int32_t* S, int k,
                     int d, uint8_t* dist, uint64_t* masks, int64_t* counters) {
    int rc = check_cluster(n, S, k, d);
    if (rc) return rc;
    const int32_t INF = 0x7fffffff;
    uint64_t* Sseen = (uint64_t*)calloc((size_t)n, sizeof(uint64_t));
    uint64_t* Snext = (uint64_t*)calloc((size_t)n, sizeof(uint64_t));
    int32_t* Delta = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* r = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* F = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* Fnext = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!Sseen || !Snext || !Delta || !r || !F || !Fnext) {
        free(Sseen); free(Snext); free(Delta); free(r); free(F); free(Fnext);
        return OR_NOMEM;
    }
    /* Initialization */
    for (int64_t v = 0; v < n; ++v) { Delta[v] = INF; r[v] = INF; }
    for (int i = 0; i < d; ++i) memset(masks + (size_t)i * (size_t)n, 0, sizeof(uint64_t) * (size_t)n);
    for (int j = 0; j < k; ++j) Snext[S[j]] = 1ull << j;
    int64_t fsize = 0;
    for (int j = 0; j < k; ++j) F[fsize++] = S[j];
    int64_t cnt_v = 0, cnt_a = 0, rounds = 0, reached_arcs = 0;
    int32_t i = 0;
    /* Traversing */
    while (fsize > 0) {
        rounds++;
        /* vertex phase */
        for (int64_t t = 0; t < fsize; ++t) {
            int32_t u = F[t];
            uint64_t Snew = Snext[u] & ~Sseen[u];
            if (Delta[u] == INF) {
                Delta[u] = i;
                reached_arcs += off[u + 1] - off[u];
            }
            int32_t idx = i - Delta[u];
            if (idx < d) masks[(size_t)idx * (size_t)n + u] = Snew;
            else if (idx > d) rc = OR_DIAMETER;
            Sseen[u] |= Snew;
            cnt_v++;
            cnt_a += off[u + 1] - off[u];
        }
        /* edge phase */
        int64_t nsize = 0;
        for (int64_t t = 0; t < fsize; ++t) {
            int32_t u = F[t];
            for (int64_t e = off[u]; e < off[u + 1]; ++e) {
                int32_t v = adj[e];
                if (!(Delta[v] == INF || i - Delta[v] < d)) continue;
                uint64_t before = Snext[v];
                Snext[v] = before | Sseen[u];
                if (Snext[v] != before) {          /* Fetch_And_Or set a bit */
                    if (r[v] != i) {               /* claim v for round i */
                        r[v] = i;
                        Fnext[nsize++] = v;
                    }
                }
            }
        }
        int32_t* tmp = F; F = Fnext; Fnext = tmp;
        fsize = nsize;
        i++;
        if (fsize > 0 && i >= 255) {
            /* a vertex first reached now would need Delta >= 255 */
            for (int64_t t = 0; t < fsize; ++t)
                if (Delta[F[t]] == INF) { rc = OR_DEPTH; break; }
            if (rc == OR_DEPTH) break;
        }
    }
    for (int64_t v = 0; v < n; ++v) dist[v] = (Delta[v] == INF || Delta[v] >= 255) ? 0xFF : (uint8_t)Delta[v];
    if (counters) {
        counters[0] = cnt_v;
        counters[1] = cnt_a;
        counters[2] = rounds;
        counters[3] = reached_arcs;
    }
    free(Sseen); free(Snext); free(Delta); free(r); free(F); free(Fnext);
    return rc;
}

/* delta(S[j], v) decoded from one cluster output; -1 when unreachable. */
static int32_t decode_one(int64_t n, int d, uint64_t all, const uint8_t* dist, const uint64_t* masks,
                          int64_t v, int j) {
    if (dist[v] == 0xFF) return -1;
    uint64_t bit = 1ull << j;
    if (!(all & bit)) return -1;
    for (int i = 0; i < d; ++i)
        if (masks[(size_t)i * (size_t)n + v] & bit) return (int32_t)dist[v] + i;
    return (int32_t)dist[v] + d;
}

/*
 * Exact certificate: the decoded distances x_j(v) must satisfy x_j(S[j]) = 0
 * and, for v != S[j], x_j(v) = 1 + min over neighbours u of x_j(u) (infinity
 * when no neighbour is finite).  BFS distances are the unique solution.  Also
 * checks the output format: masks pairwise disjoint, inside ALL, S_v[0] not
 * empty for reached v, all masks zero for unreached v.
 * Returns -1 when the output is certified, otherwise the first bad vertex
 * (or n when an argument is invalid).
 */
int64_t oracle_certify(int64_t n, const int64_t* off, const int32_t* adj, const int32_t* S, int k,
                       int d, const uint8_t* dist, const uint64_t* masks) {
    if (check_cluster(n, S, k, d)) return n;
    uint64_t all = all_bits(k);
    for (int64_t v = 0; v < n; ++v) {
        uint64_t seen = 0;
        for (int i = 0; i < d; ++i) {
            uint64_t m = masks[(size_t)i * (size_t)n + v];
            if (m & ~all) return v;
            if (m & seen) return v;
            seen |= m;
        }
        if (dist[v] == 0xFF) {
            if (seen) return v;
            continue;
        }
        uint64_t s0 = d > 0 ? masks[v] : all;
        if (s0 == 0) return v;
    }
    for (int j = 0; j < k; ++j) {
        for (int64_t v = 0; v < n; ++v) {
            int32_t x = decode_one(n, d, all, dist, masks, v, j);
            if (v == S[j]) {
                if (x != 0) return v;
                continue;
            }
            int32_t best = -1;
            for (int64_t e = off[v]; e < off[v + 1]; ++e) {
                int32_t y = decode_one(n, d, all, dist, masks, adj[e], j);
                if (y >= 0 && (best < 0 || y < best)) best = y;
            }
            if (best < 0) {
                if (x != -1) return v;
            } else if (x != best + 1) {
                return v;
            }
        }
    }
    return -1;
}

/*
 * Landmark-labeling query (Section 4.2): for each pair (u, v), the minimum
 * over every landmark s of every cluster c of delta(u,s) + delta(s,v), with
 * both distances decoded from cluster c's output.  u == v gives 0; no finite
 * term gives 0xFFFF; sums above 0xFFFE saturate to 0xFFFE.
 * dist is [C][n], masks is [C][d][n], ks[c] = size of cluster c.
 */
int oracle_query(int64_t n, int C, int d, const uint8_t* dist, const uint64_t* masks, const int32_t* ks,
                 int64_t q, const int32_t* pairs, uint16_t* out) {
    if (n < 0 || C < 0 || d < 0 || d > 15 || q < 0) return OR_INVALID;
    for (int64_t t = 0; t < q; ++t) {
        int64_t u = pairs[2 * t], v = pairs[2 * t + 1];
        if (u < 0 || u >= n || v < 0 || v >= n) return OR_INVALID;
        if (u == v) { out[t] = 0; continue; }
        int64_t best = -1;
        for (int c = 0; c < C; ++c) {
            if (ks[c] < 1 || ks[c] > 64) return OR_INVALID;
            uint64_t all = all_bits(ks[c]);
            const uint8_t* dc = dist + (size_t)c * (size_t)n;
            const uint64_t* mc = masks + (size_t)c * (size_t)d * (size_t)n;
            for (int j = 0; j < ks[c]; ++j) {
                int32_t a = decode_one(n, d, all, dc, mc, u, j);
                int32_t b = decode_one(n, d, all, dc, mc, v, j);
                if (a < 0 || b < 0) continue;
                if (best < 0 || a + b < best) best = a + b;
            }
        }
        out[t] = best < 0 ? 0xFFFF : (uint16_t)(best > 0xFFFE ? 0xFFFE : best);
    }
    return OR_OK;
}

/*
 * Vertex-major label rows built from cluster-major C-BFS outputs, the layout
 * the query consumes (Algorithm "Framework of Landmark Labeling" keeps
 * L[v][.] per vertex).  Row of v, for C clusters and d stored subsets:
 *   bytes [0, C)                 : dist of v to cluster c, 0xFF unreachable,
 *   zero padding up to P = round_up(C, 8),
 *   then d blocks of C uint64    : block i holds S_v[i] of cluster c.
 * Row stride = P + 8*d*C bytes.  rows must hold n * stride bytes.
 */
int oracle_label_rows(int64_t n, int C, int d, const uint8_t* dist, const uint64_t* masks, uint8_t* rows) {
    if (n < 0 || C < 0 || d < 0 || d > 15) return OR_INVALID;
    int64_t P = ((int64_t)C + 7) / 8 * 8;
    int64_t stride = P + 8 * (int64_t)d * C;
    for (int64_t v = 0; v < n; ++v) {
        uint8_t* row = rows + v * stride;
        memset(row, 0, (size_t)stride);
        for (int c = 0; c < C; ++c) {
            row[c] = dist[(size_t)c * (size_t)n + v];
            for (int i = 0; i < d; ++i) {
                uint64_t m = masks[((size_t)c * (size_t)d + (size_t)i) * (size_t)n + v];
                memcpy(row + P + 8 * ((int64_t)i * C + c), &m, 8);
            }
        }
    }
    return OR_OK;
}

/*
 * Bounded bidirectional search of a query (Appendix B).  Around each end a
 * BFS grows level by level and keeps a level only if the ball (the end
 * itself included) then holds at most tau vertices; the first level that
 * would overflow is dropped and the search stops.  For every pair, out[t] =
 * min over vertices x in both balls of hops(u, x) + hops(v, x), 0 for u == v
 * and 0xFFFF when the balls do not meet.  Whole levels make the balls
 * independent of the order in which a level's vertices are found; the
 * answer is delta(u, v) whenever it is finite (any common vertex lies on a
 * walk of that length, and a shortest path crosses both balls' boundaries
 * when they meet), so only its presence depends on tau.
 */
static int64_t ball(int64_t n, const int64_t* off, const int32_t* adj, int32_t c, int64_t tau, int32_t* hop,
                    int32_t* list) {
    /* hop[] must be -1 everywhere on entry; the ball's vertices are left in
       list[0, size) with their hops set, everything else stays -1 */
    int64_t size = 1, lo = 0;
    list[0] = c;
    hop[c] = 0;
    for (int32_t h = 1;; ++h) {
        int64_t hi = size, grown = size;
        int overflow = 0;
        for (int64_t i = lo; i < hi && !overflow; ++i) {
            int32_t x = list[i];
            for (int64_t e = off[x]; e < off[x + 1]; ++e) {
                int32_t y = adj[e];
                if (hop[y] >= 0) continue;
                if (grown == tau) { overflow = 1; break; }
                hop[y] = h;
                list[grown++] = y;
            }
        }
        if (overflow) { /* drop the partial level */
            for (int64_t i = hi; i < grown; ++i) hop[list[i]] = -1;
            return hi;
        }
        if (grown == hi) return hi; /* no new level */
        lo = hi;
        size = grown;
    }
    (void)n;
}

int oracle_local_search(int64_t n, const int64_t* off, const int32_t* adj, int64_t q, const int32_t* pairs,
                        int64_t tau, uint16_t* out) {
    if (n < 0 || q < 0 || tau < 1) return OR_INVALID;
    int32_t* hu = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t* hv = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t* lu = (int32_t*)malloc(sizeof(int32_t) * (size_t)(tau < n ? tau : (n > 0 ? n : 1)));
    int32_t* lv = (int32_t*)malloc(sizeof(int32_t) * (size_t)(tau < n ? tau : (n > 0 ? n : 1)));
    if (!hu || !hv || !lu || !lv) {
        free(hu); free(hv); free(lu); free(lv);
        return OR_NOMEM;
    }
    for (int64_t v = 0; v < n; ++v) hu[v] = hv[v] = -1;
    int rc = OR_OK;
    for (int64_t t = 0; t < q; ++t) {
        int32_t u = pairs[2 * t], v = pairs[2 * t + 1];
        if (u < 0 || (int64_t)u >= n || v < 0 || (int64_t)v >= n) { rc = OR_INVALID; break; }
        if (u == v) { out[t] = 0; continue; }
        int64_t su = ball(n, off, adj, u, tau, hu, lu);
        int64_t sv = ball(n, off, adj, v, tau, hv, lv);
        int64_t best = -1;
        for (int64_t i = 0; i < su; ++i) {
            int32_t x = lu[i];
            if (hv[x] >= 0 && (best < 0 || hu[x] + hv[x] < best)) best = hu[x] + hv[x];
        }
        out[t] = best < 0 ? 0xFFFF : (uint16_t)best;
        for (int64_t i = 0; i < su; ++i) hu[lu[i]] = -1;
        for (int64_t i = 0; i < sv; ++i) hv[lv[i]] = -1;
    }
    free(hu); free(hv); free(lu); free(lv);
    return rc;
}
