/*
 * Seeded synthetic graph generation (R-MAT and road-like grids) and CSR
 * construction.  Input generation only: nothing in here computes any part of
 * Cluster-BFS.  Both the CUDA path and the oracle consume the CSR it builds.
 *
 * Randomness: splitmix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based
 * generator: draw(seed, i) = mix(seed + (i + 1) * 0x9E3779B97F4A7C15) with
 * mix the splitmix64 output function.  The stream depends on nothing but the
 * seed and the counter, so the graphs are identical on every machine.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t sm64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t gen_splitmix64(uint64_t seed, uint64_t i) { return sm64(seed, i); }

/*
 * R-MAT edge draws.  m = edge_factor << scale draws; draw e uses the 16-bit
 * fields of words sm64(seed, e * W + w), W = ceil(scale / 4), field f of word
 * w deciding bit level l = 4w + f (most significant level first).  A field r
 * picks quadrant a when r < ta, b when r < tab, c when r < tabc, else d;
 * quadrant (src bit, dst bit) = a (0,0), b (0,1), c (1,0), d (1,1).
 * When perm_seed != 0 every id x is replaced by p[x], p a Fisher-Yates
 * shuffle of 0..n-1 driven by sm64(perm_seed, .).
 */
int gen_rmat_edges(int scale, int64_t edge_factor, uint32_t ta, uint32_t tab, uint32_t tabc, uint64_t seed,
                   uint64_t perm_seed, int64_t* src, int64_t* dst) {
    if (scale < 1 || scale > 30 || edge_factor < 1) return -1;
    int64_t n = (int64_t)1 << scale;
    int64_t m = edge_factor * n;
    int W = (scale + 3) / 4;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        int64_t s = 0, t = 0;
        for (int w = 0; w < W; ++w) {
            uint64_t word = sm64(seed, (uint64_t)e * (uint64_t)W + (uint64_t)w);
            for (int f = 0; f < 4; ++f) {
                int l = 4 * w + f;
                if (l >= scale) break;
                uint32_t r = (uint32_t)((word >> (16 * f)) & 0xFFFFu);
                /* branch-free form of the quadrant table above */
                int sb = r >= tab;
                int db = (r >= ta) ^ (r >= tab) ^ (r >= tabc);
                s |= (int64_t)sb << (scale - 1 - l);
                t |= (int64_t)db << (scale - 1 - l);
            }
        }
        src[e] = s;
        dst[e] = t;
    }
    if (perm_seed) {
        int64_t* p = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
        if (!p) return -4;
        for (int64_t i = 0; i < n; ++i) p[i] = i;
        for (int64_t i = n - 1; i > 0; --i) {
            int64_t j = (int64_t)(sm64(perm_seed, (uint64_t)i) % (uint64_t)(i + 1));
            int64_t x = p[i]; p[i] = p[j]; p[j] = x;
        }
#pragma omp parallel for schedule(static)
        for (int64_t e = 0; e < m; ++e) { src[e] = p[src[e]]; dst[e] = p[dst[e]]; }
        free(p);
    }
    return 0;
}

/*
 * Road-like grid: side x side vertices, id = row * side + col; every
 * horizontal then every vertical grid edge (row-major) is kept unless
 * (sm64(seed, e) >> 32) < del_thr; then n_short shortcut edges whose
 * endpoints are sm64(seed ^ 0xA5A5..., 2i) % n and (..., 2i+1) % n.
 * Returns the number of edges written (buffers hold 2*side*(side-1)+n_short).
 */
int64_t gen_road_grid_edges(int64_t side, uint32_t del_thr, int64_t n_short, uint64_t seed, int64_t* src,
                            int64_t* dst) {
    if (side < 1) return -1;
    int64_t n = side * side, cnt = 0, e = 0;
    for (int dir = 0; dir < 2; ++dir) {
        for (int64_t r = 0; r < side; ++r) {
            for (int64_t c = 0; c < side; ++c) {
                int64_t a = r * side + c, b;
                if (dir == 0) { if (c + 1 >= side) continue; b = a + 1; }
                else { if (r + 1 >= side) continue; b = a + side; }
                uint64_t x = sm64(seed, (uint64_t)e++);
                if ((uint32_t)(x >> 32) < del_thr) continue;
                src[cnt] = a; dst[cnt] = b; cnt++;
            }
        }
    }
    uint64_t s2 = seed ^ 0xA5A5A5A5A5A5A5A5ull;
    for (int64_t i = 0; i < n_short; ++i) {
        src[cnt] = (int64_t)(sm64(s2, 2 * (uint64_t)i) % (uint64_t)n);
        dst[cnt] = (int64_t)(sm64(s2, 2 * (uint64_t)i + 1) % (uint64_t)n);
        cnt++;
    }
    return cnt;
}

/* LSD radix sort of keys over the low `bits` bits, 11-bit digits. */
static int radix_sort_u64(uint64_t* keys, int64_t m, int bits) {
    if (m <= 1) return 0;
    uint64_t* tmp = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)m);
    if (!tmp) return -4;
    const int D = 11, R = 1 << D;
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * R);
    if (!cnt) { free(tmp); return -4; }
    uint64_t *a = keys, *b = tmp;
    for (int sh = 0; sh < bits; sh += D) {
        memset(cnt, 0, sizeof(int64_t) * R);
        for (int64_t i = 0; i < m; ++i) cnt[(a[i] >> sh) & (R - 1)]++;
        int64_t s = 0;
        for (int i = 0; i < R; ++i) { int64_t c = cnt[i]; cnt[i] = s; s += c; }
        for (int64_t i = 0; i < m; ++i) b[cnt[(a[i] >> sh) & (R - 1)]++] = a[i];
        uint64_t* t = a; a = b; b = t;
    }
    if (a != keys) memcpy(keys, a, sizeof(uint64_t) * (size_t)m);
    free(tmp);
    free(cnt);
    return 0;
}

/*
 * Canonical undirected edge keys (lo << 32 | hi, lo < hi), self loops
 * dropped, sorted, duplicates removed.  keys must hold m entries.  Returns
 * the number of unique edges, or a negative error.
 */
int64_t gen_unique_edges(int64_t n, int64_t m, const int64_t* src, const int64_t* dst, uint64_t* keys) {
    if (n < 0 || n > 0x7fffffffLL || m < 0) return -1;
    int64_t k = 0;
    for (int64_t i = 0; i < m; ++i) {
        int64_t a = src[i], b = dst[i];
        if (a < 0 || b < 0 || a >= n || b >= n) return -1;
        if (a == b) continue;
        uint64_t lo = (uint64_t)(a < b ? a : b), hi = (uint64_t)(a < b ? b : a);
        keys[k++] = (lo << 32) | hi;
    }
    int bits = 0;
    while (bits < 31 && ((int64_t)1 << bits) < n) bits++;
    /* dense key lo << bits | hi sorts by (lo, hi) */
    for (int64_t i = 0; i < k; ++i) keys[i] = ((keys[i] >> 32) << bits) | (keys[i] & 0xffffffffull);
    int rc = radix_sort_u64(keys, k, 2 * bits);
    for (int64_t i = 0; i < k; ++i) {
        uint64_t lo = keys[i] >> bits, hi = keys[i] & (((uint64_t)1 << bits) - 1);
        keys[i] = (lo << 32) | hi;
    }
    if (rc) return rc;
    int64_t u = 0;
    for (int64_t i = 0; i < k; ++i)
        if (u == 0 || keys[i] != keys[u - 1]) keys[u++] = keys[i];
    return u;
}

/*
 * CSR of the undirected graph with the U sorted unique canonical keys:
 * off[n+1], adj[2U]; every list sorted ascending (for vertex x, neighbours
 * smaller than x come from keys whose hi is x, larger ones from keys whose lo
 * is x; both groups are written in ascending order).
 */
int gen_csr_fill(int64_t n, int64_t U, const uint64_t* keys, int64_t* off, int32_t* adj) {
    memset(off, 0, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t i = 0; i < U; ++i) {
        off[(keys[i] >> 32) + 1]++;
        off[(keys[i] & 0xffffffffull) + 1]++;
    }
    for (int64_t v = 0; v < n; ++v) off[v + 1] += off[v];
    int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!pos) return -4;
    memcpy(pos, off, sizeof(int64_t) * (size_t)n);
    /* smaller neighbours first: scanning keys in (lo, hi) order, the arc
       hi -> lo arrives in ascending lo for each fixed hi */
    for (int64_t i = 0; i < U; ++i) {
        int64_t lo = (int64_t)(keys[i] >> 32), hi = (int64_t)(keys[i] & 0xffffffffull);
        adj[pos[hi]++] = (int32_t)lo;
    }
    for (int64_t i = 0; i < U; ++i) {
        int64_t lo = (int64_t)(keys[i] >> 32), hi = (int64_t)(keys[i] & 0xffffffffull);
        adj[pos[lo]++] = (int32_t)hi;
    }
    free(pos);
    return 0;
}
