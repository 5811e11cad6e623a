// libcbfs.so, part 1: graph residency, the Cluster-BFS traversal and its
// C ABI entry points (include/cbfs.h).
//
// The traversal follows Algorithm 1 (Section 3.2) level by level for P
// clusters at once ("slots"; P = 1, 2, 4 or 8).  The per-vertex state is
// vertex-major -- vis[v][0..P) and acc[v][0..P) -- so one scan of an
// adjacency list and one gathered block of P subset words serve every
// cluster in flight.  Round i has two kernels:
//
//   phase A (vertex phase): for every queued vertex u and slot s
//     new = acc[u][s] & ~vis[u][s]; vis[u][s] |= new; acc[u][s] = 0;
//     Delta_u = i on the first visit of slot s;  S_u[i - Delta_u] = new
//     (stored when i - Delta_u < d; > d means the cluster diameter exceeds
//     d).  Vertices with new sources are compacted per tile with their arc
//     prefix; lists longer than kBigDeg go to a "big" list cut into
//     kBigDeg-arc pieces.
//
//   phase B (edge phase), one of
//     push (EdgeMap-Sparse, Appendix A): every frontier arc (u, v) ORs the
//       new sources of u into acc[v] where they are not in vis[v] or
//       acc[v] (both checked before the atomic); a pusher that turns some
//       acc[v][s] from 0 to non-zero claims v for F_{i+1} -- the
//       once-per-round claim that r[v] implements in Algorithm 1.  Arcs are
//       spread evenly over the CTAs: big-list pieces first, then tiles whose
//       entries are found by a binary search of the tile's arc prefix in
//       shared memory.
//     pull (EdgeMap-Dense): every vertex v with some unfinished slot ORs the
//       vis blocks of its frontier neighbours (a bitmap test, skipped when
//       the frontier holds more than n/8 vertices: a non-frontier
//       neighbour's sources are already in vis[v]), stops early once every
//       unfinished slot is covered, and keeps the part not in vis[v] as
//       acc[v].  Vertices are handled by a thread, a warp or 2048-arc CTA
//       pieces according to their degree (thresholds per call, see
//       cbfs_tune_t; ranks are sorted by degree, so each class is a rank
//       range), each lane keeping four gathers in flight.
//     The direction is chosen per round from |F| + sum deg(F) against
//     pull_alpha * nnz (the rule of Algorithm "EdgeMap").
//
// Readings of the paper (the oracle takes the same ones):
//   - the sources are seeded into Snext (acc), not Sseen, so round 0 records
//     S_s[0] = {s};
//   - new sources are pushed instead of all of Sseen[u]: a source newly set
//     at v by Sseen[u] must be at distance exactly i from u, so both pushes
//     set the same bits;
//   - the edge condition i - Delta_v < d of Algorithm 1 is replaced by the
//     test new & ~vis[v] & ~acc[v] != 0, which is empty whenever the
//     condition fails (by Corollary 1 vis[v] = ALL after round Delta_v + d)
//     and also skips arcs that would not change Snext[v].
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "cbfs_internal.cuh"

using namespace cbfs;

namespace {

// ----------------------------------------------------------------- helpers

template <class T>
__device__ __forceinline__ void append(T* q, unsigned long long* qlen, T entry) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(qlen, (unsigned long long)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    q[base + __popc(mask & ((1u << lane) - 1u))] = entry;
}

struct ScanSmem {
    uint32_t a[kWarps];
    uint32_t b[kWarps];
};

// Exclusive block-wide scan of two counters (256 threads).
__device__ __forceinline__ void block_scan2(uint32_t a, uint32_t b, uint32_t& ea, uint32_t& eb, uint32_t& ta,
                                            uint32_t& tb, ScanSmem& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t x = __shfl_up_sync(0xffffffffu, ia, o);
        uint32_t y = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) { ia += x; ib += y; }
    }
    if (lane == 31) { sm.a[warp] = ia; sm.b[warp] = ib; }
    __syncthreads();
    uint32_t pa = 0, pb = 0, sa = 0, sb = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        uint32_t x = sm.a[w], y = sm.b[w];
        if (w < warp) { pa += x; pb += y; }
        sa += x; sb += y;
    }
    ea = pa + ia - a;
    eb = pb + ib - b;
    ta = sa;
    tb = sb;
    __syncthreads();
}

__device__ __forceinline__ uint64_t warp_or(uint64_t x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x |= __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ __forceinline__ unsigned long long block_sum(unsigned long long x, unsigned long long* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = x;
    __syncthreads();
    unsigned long long s = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kWarps; ++w) s += red[w];
    __syncthreads();
    return s;  // valid in thread 0
}

// P consecutive words (P * 8 bytes, aligned to P * 8): one 64-bit access
// for P = 1, 128-bit for P = 2, 256-bit accesses for P = 4 and 8.
__device__ __forceinline__ void ld256(const uint64_t* p, uint64_t& a, uint64_t& b, uint64_t& c, uint64_t& d) {
    asm volatile("ld.global.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
}

__device__ __forceinline__ void st256(uint64_t* p, uint64_t a, uint64_t b, uint64_t c, uint64_t d) {
    asm volatile("st.global.v4.u64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(a), "l"(b), "l"(c), "l"(d) : "memory");
}

template <int P>
__device__ __forceinline__ void load_words(const uint64_t* p, uint64_t (&x)[P]) {
    if constexpr (P == 1) {
        x[0] = p[0];
    } else if constexpr (P == 2) {
        const ulonglong2 t = *reinterpret_cast<const ulonglong2*>(p);
        x[0] = t.x;
        x[1] = t.y;
    } else {
#pragma unroll
        for (int i = 0; i < P; i += 4) ld256(p + i, x[i], x[i + 1], x[i + 2], x[i + 3]);
    }
}

template <int P>
__device__ __forceinline__ void store_words(uint64_t* p, const uint64_t (&x)[P]) {
    if constexpr (P == 1) {
        p[0] = x[0];
    } else if constexpr (P == 2) {
        *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2(x[0], x[1]);
    } else {
#pragma unroll
        for (int i = 0; i < P; i += 4) st256(p + i, x[i], x[i + 1], x[i + 2], x[i + 3]);
    }
}

template <int P>
__device__ __forceinline__ void zero_words(uint64_t* p) {
    uint64_t z[P];
#pragma unroll
    for (int i = 0; i < P; ++i) z[i] = 0;
    store_words<P>(p, z);
}

// Gathers kept in flight per lane (two for P = 8 measured slower: the
// register saving did not pay for the lost memory-level parallelism).
template <int P>
struct Gath {
    static constexpr int G = 4;
};

// ORs into acc the src blocks (the sources new at each frontier neighbour)
// of the frontier neighbours among up to G arcs adj[e], adj[e + step], ...
// below o1 (fb == nullptr: every neighbour); all gathers are issued before
// any is used.
template <int P>
__device__ __forceinline__ void gather(const uint64_t* src, const uint32_t* fb, const int32_t* adj, int64_t e,
                                       int64_t step, int64_t o1, uint64_t (&acc)[P]) {
    constexpr int G = Gath<P>::G;
    int32_t u[G];
#pragma unroll
    for (int k = 0; k < G; ++k) u[k] = (e + k * step < o1) ? adj[e + k * step] : -1;
    // only frontier neighbours can carry sources v has not seen
#pragma unroll
    for (int k = 0; k < G; ++k)
        if (fb && u[k] >= 0 && !((fb[u[k] >> 5] >> (u[k] & 31)) & 1u)) u[k] = -1;
    uint64_t x[G][P];
#pragma unroll
    for (int k = 0; k < G; ++k) {
        if (u[k] >= 0) load_words<P>(src + (size_t)u[k] * P, x[k]);
        else {
#pragma unroll
            for (int s = 0; s < P; ++s) x[k][s] = 0;
        }
    }
#pragma unroll
    for (int k = 0; k < G; ++k)
#pragma unroll
        for (int s = 0; s < P; ++s) acc[s] |= x[k][s];
}

// Appends v to the next frontier and adds deg to its degree sum (the
// direction decision of the next round); one atomic pair per warp.
__device__ __forceinline__ void append_next(uint32_t* q, RoundCtl* cn, uint32_t* fbn, uint32_t v, uint32_t deg) {
    atomicOr(fbn + (v >> 5), 1u << (v & 31));
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    // 32 degrees < 2^31 each: sum the high and low halves separately in 32 bits
    const unsigned int hi = __reduce_add_sync(mask, deg >> 16);
    const unsigned int lo = __reduce_add_sync(mask, deg & 0xFFFFu);
    unsigned long long base = 0;
    if (lane == leader) {
        base = atomicAdd(&cn->qlen, (unsigned long long)__popc(mask));
        atomicAdd(&cn->sdeg, ((unsigned long long)hi << 16) + (unsigned long long)lo);
    }
    base = __shfl_sync(mask, base, leader);
    q[base + __popc(mask & ((1u << lane) - 1u))] = v;
}

// Push the new sources fw[0..P) of a frontier vertex along one arc to t.
template <int P>
__device__ __forceinline__ void push_arc(const Wave& w, const uint64_t* fw, uint32_t t, uint32_t stamp, uint32_t* qn,
                                         RoundCtl* cn, uint32_t* fbn) {
    uint64_t vs[P], b[P];
    load_words<P>(w.vis + (size_t)t * P, vs);  // vis is read-only in phase B
    uint64_t any = 0;
#pragma unroll
    for (int s = 0; s < P; ++s) {
        b[s] = fw[s] & ~vs[s];
        any |= b[s];
    }
    if (!any) return;
    uint64_t* ap = w.acc + (size_t)t * P;
    uint64_t ac[P];
    load_words<P>(ap, ac);  // acc only grows in phase B: a stale copy is a subset
    bool claim = false;
#pragma unroll
    for (int s = 0; s < P; ++s) {
        const uint64_t bb = b[s] & ~ac[s];
        if (bb) {
            const unsigned long long old = atomicOr(reinterpret_cast<unsigned long long*>(ap + s), (unsigned long long)bb);
            claim |= (old == 0ull);
        }
    }
    if (!claim) return;
    if (P == 1 || atomicExch(w.rq + t, stamp) != stamp)
        append_next(qn, cn, fbn, t, (uint32_t)(w.off[t + 1] - w.off[t]));
}

// Direction of a round (Algorithm "EdgeMap"): dense when the frontier and
// its arcs are a large part of the graph.
__device__ __forceinline__ bool decide_pull(const Wave& w, const RoundCtl* c) {
    if (!(w.alpha > 0.f)) return false;
    const double work = (double)c->qlen + (double)c->sdeg;
    return work > (double)w.alpha * (double)w.nnz;
}

// Bits still missing at v over the unfinished slots um.
template <int P>
__device__ __forceinline__ uint64_t missing_bits(const uint64_t (&acc)[P], const uint64_t (&vs)[P], const uint64_t* all,
                                                 unsigned int um) {
    uint64_t rem = 0;
#pragma unroll
    for (int s = 0; s < P; ++s)
        if ((um >> s) & 1u) rem |= all[s] & ~(acc[s] | vs[s]);
    return rem;
}

template <int P>
__device__ __forceinline__ unsigned int unfinished(const uint64_t (&vs)[P], const uint64_t* all, unsigned int active) {
    unsigned int um = 0;
#pragma unroll
    for (int s = 0; s < P; ++s)
        if (((active >> s) & 1u) && vs[s] != all[s]) um |= 1u << s;
    return um;
}

// Records the sources fw new at u in round `round` (Algorithm 1's
// S_u[round - Delta_u] = Snew, Delta_u = round on the first visit of a slot)
// either in the wave's internal rows (dist_r path, emitted to the caller's
// arrays after the wave) or, when the wave has no rows (dist_r == nullptr),
// straight into each slot's cluster-major output at the caller's id
// perm[u] (identity when perm is null); those outputs were cleared to
// Delta = 0xFF and empty subsets before the wave.  Returns the slots with
// new sources.
// The P Delta bytes of u's internal row in one load (the row starts at a
// multiple of P bytes).
template <int P>
__device__ __forceinline__ uint64_t load_delta_row(const uint8_t* p) {
    if constexpr (P == 1) return *p;
    else if constexpr (P == 2) return *reinterpret_cast<const uint16_t*>(p);
    else if constexpr (P == 4) return *reinterpret_cast<const uint32_t*>(p);
    else return *reinterpret_cast<const unsigned long long*>(p);
}

template <int P>
__device__ __forceinline__ unsigned int record_rows(const Wave& w, uint32_t u, const uint64_t (&fw)[P], int round,
                                                    const SlotDesc* ss, const uint64_t* dpre = nullptr) {
    unsigned int act = 0;
    if (w.dist_r) {
        // the wave's internal rows of u: P Delta bytes, then each slot's d
        // subset words contiguous (slot s at mr[s*d .. s*d + d))
        uint8_t* dr = w.dist_r + (size_t)u * P;
        uint64_t* mr = w.masks_r + (size_t)u * w.d * P;
        uint16_t* wr = w.wmask_r + (size_t)u * P;
#pragma unroll
        for (int s = 0; s < P; ++s) {
            if (!fw[s]) continue;
            // Delta of the slot: from the row's bytes loaded by the caller, if it did
            const uint8_t dd = dpre ? (uint8_t)(*dpre >> (8 * s)) : dr[s];
            int j;
            uint32_t wm;
            if (dd == 0xFF) {
                if (round >= 255) set_status(w.status, CBFS_E_DEPTH);
                else dr[s] = (uint8_t)round;
                j = 0;
                // first visit of slot s: the rows are not cleared per wave.  A
                // slot's block of at most kZeroWords words (one sector) is
                // zeroed here; longer blocks get a written-word mask instead
                // (k_emit outputs 0 for a word whose bit is clear), which
                // avoids writing d words at the first visit
                wm = 0;
                if (w.d <= kZeroWords)
                    for (int jj = 1; jj < w.d; ++jj) mr[(size_t)s * w.d + jj] = 0ull;
            } else {
                j = round - (int)dd;
                wm = w.d > kZeroWords ? wr[s] : 0u;
            }
            if (j < w.d) {
                mr[(size_t)s * w.d + j] = fw[s];
                if (w.d > kZeroWords) wr[s] = (uint16_t)(wm | (1u << j));
            } else if (j > w.d) {
                set_status(w.status, CBFS_E_DIAMETER);
            }
            act |= 1u << s;
        }
    } else if (w.nmembers) {
        // direct, packed wave: each member cluster's output, from its bits of the word
        const size_t id = w.perm ? (size_t)w.perm[u] : (size_t)u;
#pragma unroll
        for (int s = 0; s < P; ++s) {
            uint64_t x = fw[s];
            if (x) act |= 1u << s;
            while (x) {
                const int b = __ffsll((long long)x) - 1;
                const unsigned int mi = w.bit_member[s * 64 + b];
                if (mi >= (unsigned int)w.nmembers) {  // never for member tables built by the host
                    set_status(w.status, CBFS_E_INVALID);
                    break;
                }
                const MemberDesc& M = w.members[mi];
                x &= ~(M.mask | (1ull << b));  // bit b always goes: the loop ends whatever the tables hold
                const uint64_t bits = (fw[s] & M.mask) >> M.off;
                const uint8_t dd = M.dist[id];
                int j;
                if (dd == 0xFF) {
                    if (round >= 255) set_status(w.status, CBFS_E_DEPTH);
                    else M.dist[id] = (uint8_t)round;
                    j = 0;
                } else {
                    j = round - (int)dd;
                }
                if (j < w.d) M.masks[(size_t)j * (size_t)w.n + id] = bits;
                else if (j > w.d) set_status(w.status, CBFS_E_DIAMETER);
            }
        }
    } else {
        // direct: each slot's cluster-major output at the caller's id
        const size_t id = w.perm ? (size_t)w.perm[u] : (size_t)u;
#pragma unroll
        for (int s = 0; s < P; ++s) {
            if (!fw[s]) continue;
            const SlotDesc& S = ss[s];
            const uint8_t dd = S.dist[id];
            int j;
            if (dd == 0xFF) {
                if (round >= 255) set_status(w.status, CBFS_E_DEPTH);
                else S.dist[id] = (uint8_t)round;
                j = 0;
            } else {
                j = round - (int)dd;
            }
            if (j < w.d) S.masks[(size_t)j * (size_t)w.n + id] = fw[s];
            else if (j > w.d) set_status(w.status, CBFS_E_DIAMETER);
            act |= 1u << s;
        }
    }
    return act;
}

// Waves with round records (hcap > 0) keep the sources new at u in round
// `round` as one whole block hist[round][u] -- a full 32-byte sector at
// P = 4 -- where a direct output write would touch d different output
// words (8 bytes each, partial sectors that the memory must read, merge and
// write back when the neighbouring words of the sector arrive in other
// rounds).  k_flush turns the records into the outputs after the wave;
// rounds past the records write directly.  Returns the slots with new sources.
template <int P>
__device__ __forceinline__ unsigned int record_new(const Wave& w, uint32_t u, const uint64_t (&fw)[P], int round,
                                                   const SlotDesc* ss, const uint64_t* dpre = nullptr) {
    if (round < w.hcap) {
        store_words<P>(w.hist + ((size_t)round * (size_t)w.n + u) * P, fw);
        unsigned int act = 0;
#pragma unroll
        for (int s = 0; s < P; ++s)
            if (fw[s]) act |= 1u << s;
        return act;
    }
    return record_rows<P>(w, u, fw, round, ss, dpre);
}

// Pull result of v.  Fused (FUSE, the call's fused_pull): the vertex phase of
// round rn = round + 1 is done on the spot -- the sources acc & ~vs are new
// at v, they join vis[v], go to v's rows and to nwn[v], the next pull's
// gather source.  Plain: the new sources are stored in acc[v] for the next
// vertex phase.  A pull round writes no queue: the next vertex phase finds
// the frontier in the bitmap.  Counts v and its arcs for the next direction
// decision, notes its slots with new sources (fused), and returns whether v
// joins F_{rn}.
template <int P, bool FUSE>
__device__ __forceinline__ bool pull_finish(const Wave& w, int32_t v, const uint64_t (&acc)[P], const uint64_t (&vs)[P],
                                            uint32_t deg, int rn, uint64_t* nwn, unsigned long long& cnt,
                                            unsigned long long& sdeg, unsigned int& act) {
    uint64_t nw[P], any = 0;
#pragma unroll
    for (int s = 0; s < P; ++s) {
        nw[s] = acc[s] & ~vs[s];
        any |= nw[s];
        if (FUSE && nw[s]) act |= 1u << s;
    }
    if (!any) return false;
    if (FUSE) {
        uint64_t nv[P];
#pragma unroll
        for (int s = 0; s < P; ++s) nv[s] = vs[s] | nw[s];
        store_words<P>(w.vis + (size_t)v * P, nv);
        if (rn >= w.hcap) store_words<P>(nwn + (size_t)v * P, nw);  // else its record is the gather source
        record_new<P>(w, (uint32_t)v, nw, rn, w.slots);
    } else {
        store_words<P>(w.acc + (size_t)v * P, nw);
    }
    cnt += 1;
    sdeg += deg;
    return true;
}

}  // namespace

// --------------------------------------------------------------- kernels
// The traversal kernels have external linkage (declared in
// cbfs_internal.cuh) so that every entry point of the library launches the
// same code.

namespace cbfs {

// Seeds a wave: acc[v][s] = bit j for S_s[j] = v, F_0 = the distinct sources.
__global__ void k_seed(Wave w, const uint64_t* seeds, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const uint64_t e = seeds[i];
        const int s = (int)((e >> 40) & 0xFF), j = (int)((e >> 32) & 0xFF);
        const uint32_t v = (uint32_t)e;
        if ((int64_t)v >= w.n || s >= w.P || j >= 64) {  // never for seeds staged by the host
            set_status(w.status, CBFS_E_INVALID);
            continue;
        }
        // packed clusters of one word may share a source vertex
        atomicOr(reinterpret_cast<unsigned long long*>(w.acc + (size_t)v * w.P + s), 1ull << j);
        if (atomicExch(w.rq + v, 1u) != 1u) {
            append(w.q0, &w.ctl[0].qlen, v);
            atomicAdd(&w.ctl[0].sdeg, (unsigned long long)(w.off[v + 1] - w.off[v]));
            atomicOr(w.fb0 + (v >> 5), 1u << (v & 31));
        }
    }
}

// After a wave: every source must have seen every source of its cluster.
// Otherwise the cluster is not connected within distance d and the implied
// last subset S_v[d] would be wrong, so the call fails with CBFS_E_DIAMETER.
// bound_round > 0: the wave ran exactly bound_round rounds without looking;
// if its frontier was still not empty it is flagged for a rerun instead.
__global__ void k_check_sources(Wave w, const uint64_t* seeds, int count, int bound_round, int* unfinished) {
    if (bound_round > 0 && w.ctl[bound_round].qlen != 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *unfinished = 1;
        return;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const uint64_t e = seeds[i];
        const int s = (int)((e >> 40) & 0xFF);
        const uint32_t v = (uint32_t)e;
        if ((int64_t)v >= w.n || s >= w.P) continue;  // flagged by k_seed
        // each cluster's sources must have seen all of that cluster's sources
        const uint64_t want = w.nmembers ? w.members[(e >> 48) & 0xFF].mask : w.slots[s].all;
        if ((w.vis[(size_t)v * w.P + s] & want) != want) set_status(w.status, CBFS_E_DIAMETER);
    }
}

// A wave without internal rows writes its slots' outputs directly: before
// it, every slot's dist is set to 0xFF and its d subset words to 0.
__global__ void k_clear_outputs(Wave w) {
    const int64_t n = w.n, words = (int64_t)w.d * n;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, step = (int64_t)gridDim.x * blockDim.x;
    for (int s = 0; s < w.nslots; ++s) {
        const SlotDesc S = w.slots[s];
        for (int64_t i = t0; i < n; i += step) S.dist[i] = 0xFF;
        for (int64_t i = t0; i < words; i += step) S.masks[i] = 0ull;
    }
}

// Graph mode: after phase B of the current round, continue the round loop
// while the next frontier is not empty (and the round bound allows it).
__global__ void k_round_cond(Wave w, cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0) return;
    const int r = *w.round_dev;
    unsigned int go = 0;
    // one round; bits 40 and up count the rounds' k_flush launches (waves with round records)
    atomicAdd(w.iters, w.hcap > 0 ? 1ull + (1ull << 40) : 1ull);
    if (w.ctl[r + 1].qlen > 0) {
        if (r + 2 < kMaxRounds) {
            *w.round_dev = r + 1;
            go = 1;
        } else {
            set_status(w.status, CBFS_E_DEPTH);
        }
    }
    cudaGraphSetConditional(h, go);
}

// Phase A: the vertex phase of round `round`, the direction decision and,
// for a push round, the push work lists.  A small frontier is read from the
// queue; a large one (qlen * dense_div > n) by scanning every vertex in
// internal order for its frontier bit, which streams instead of gathering.
// When F_round was produced by a fused pull, that pull already did F_round's
// vertex phase and left its new sources in nw[round & 1]: then this kernel
// only builds the push lists (push round) or returns (pull round).
// Otherwise (F_round pushed or plainly pulled, or the sources) it takes the
// new sources from acc, updates vis and the rows, and before a fused pull
// stores them in nw[round & 1] for the pull to gather.
template <int P>
__global__ void __launch_bounds__(kThreads) k_phase_a(Wave w, int round) {
    constexpr int EPT = Geo<P>::kEpt;
    constexpr int TILE = Geo<P>::kTile;
    __shared__ SlotDesc ss[P];
    __shared__ ScanSmem scan;
    __shared__ unsigned long long red[kWarps];
    __shared__ unsigned int s_active;
    if (w.round_dev) round = *w.round_dev;
    RoundCtl* c = w.ctl + round;
    const unsigned long long qlen = c->qlen;
    if (qlen == 0) return;
    const bool pull = decide_pull(w, c);
    const bool fused = c->fused != 0;  // F_round came from a pull that did its set update
    // this round's pull gathers nw when pulls are fused
    const bool pull_fused = pull && w.fused_pull;
    const bool dense = c->dense || (w.dense_div > 0 && qlen * (unsigned long long)w.dense_div > (unsigned long long)w.n);
    if (blockIdx.x == 0 && threadIdx.x == 0) c->mode = pull ? 1 : 0;
    if (threadIdx.x < w.nslots) ss[threadIdx.x] = w.slots[threadIdx.x];
    if (threadIdx.x == 0) s_active = 0;
    __syncthreads();
    const uint32_t* q = (round & 1) ? w.q1 : w.q0;
    const uint32_t* fbr = (round & 1) ? w.fb1 : w.fb0;  // F_round, set by its producers
    uint64_t* nwc = (round & 1) ? w.nw1 : w.nw0;        // F_round's new sources (pull gathers)
    {
        // F_{round+1}'s bitmap was last read in round - 1: clear it for this round's edge phase.
        // With round records, F_round's bitmap (final now) is kept for k_flush
        uint32_t* fbn = (round & 1) ? w.fb0 : w.fb1;
        const int64_t words = (w.n + 31) / 32;
        uint32_t* keep = round < w.hcap ? w.fbh + (size_t)round * (size_t)words : nullptr;
        for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < words; i += (int64_t)gridDim.x * kThreads) {
            fbn[i] = 0u;
            if (keep) keep[i] = fbr[i];
        }
    }
    if (fused && pull) return;  // nothing left of F_round's vertex phase
    const unsigned long long span = dense ? (unsigned long long)w.n : qlen;
    const unsigned long long ntiles = (span + TILE - 1) / TILE;
    unsigned long long my_nf = 0;
    unsigned int my_active = 0;
    for (unsigned long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        uint32_t keep[EPT], dg[EPT];
        int64_t ost[EPT];
        uint64_t fw[EPT][P];
        uint32_t cnt = 0, arcs = 0;
#pragma unroll
        for (int r = 0; r < EPT; ++r) {
            keep[r] = 0;
            dg[r] = 0;
            ost[r] = 0;
#pragma unroll
            for (int s = 0; s < P; ++s) fw[r][s] = 0;
            const unsigned long long idx = t * TILE + (unsigned long long)threadIdx.x * EPT + r;
            if (idx >= span) continue;
            if (dense && !((fbr[idx >> 5] >> (idx & 31)) & 1u)) continue;  // not in F_round
            const uint32_t u = dense ? (uint32_t)idx : q[idx];
            if (fused) {
                // vis updated by the pull that produced F_round: record the rows
                load_words<P>(round < w.hcap ? w.hist + ((size_t)round * (size_t)w.n + u) * P : nwc + (size_t)u * P,
                              fw[r]);
                // (the fused pull recorded the rows too)
                if (pull) continue;  // the dense edge phase needs no work lists
            } else {
                // u's acc, vis and (with internal rows) Delta bytes, loaded together: a
                // member of F_round always has sources in acc
                uint64_t a[P], vs[P];
                load_words<P>(w.acc + (size_t)u * P, a);
                load_words<P>(w.vis + (size_t)u * P, vs);
                const uint64_t dpre = w.dist_r ? load_delta_row<P>(w.dist_r + (size_t)u * P) : 0ull;
                uint64_t anyacc = 0;
#pragma unroll
                for (int s = 0; s < P; ++s) anyacc |= a[s];
                if (!anyacc) continue;  // not in F_round (dense scan), or nothing new
                uint64_t any = 0;
#pragma unroll
                for (int s = 0; s < P; ++s) {
                    fw[r][s] = a[s] & ~vs[s];
                    any |= fw[r][s];
                    vs[s] |= fw[r][s];
                }
                store_words<P>(w.vis + (size_t)u * P, vs);
                zero_words<P>(w.acc + (size_t)u * P);
                if (!any) continue;
                my_active |= record_new<P>(w, u, fw[r], round, ss, w.dist_r ? &dpre : nullptr);
                my_nf += 1;
                if (pull) {
                    // the pull's gather source (a recorded round gathers from its record)
                    if (pull_fused && round >= w.hcap) store_words<P>(nwc + (size_t)u * P, fw[r]);
                    continue;  // the dense edge phase needs no work lists
                }
            }
            const int64_t o0 = w.off[u], o1 = w.off[u + 1];
            const int64_t deg = o1 - o0;
            if (deg == 0) continue;
            if (deg > kBigDeg) {
                // big list: one entry plus ceil(deg / kBigDeg) piece records
                const unsigned int bi = atomicAdd(&c->nbig, 1u);
                w.big[bi].ost = o0;
                w.big[bi].deg = deg;
                store_words<P>(w.big_fw + (size_t)bi * P, fw[r]);
                const unsigned int np = (unsigned int)((deg + kBigDeg - 1) / kBigDeg);
                const unsigned int p0 = atomicAdd(&c->npieces, np);
                for (unsigned int p = 0; p < np; ++p) {
                    w.piece_ent[p0 + p] = bi;
                    w.piece_no[p0 + p] = p;
                }
                continue;
            }
            keep[r] = 1;
            dg[r] = (uint32_t)deg;
            ost[r] = o0;
            cnt += 1;
            arcs += (uint32_t)deg;
        }
        if (!pull) {
            uint32_t ecnt, earcs, tcnt, tarcs;
            block_scan2(cnt, arcs, ecnt, earcs, tcnt, tarcs, scan);
            const unsigned long long base = t * TILE;
#pragma unroll
            for (int r = 0; r < EPT; ++r) {
                if (!keep[r]) continue;
                const unsigned long long pos = base + ecnt;
                w.t_pre[pos] = earcs;
                w.t_ost[pos] = ost[r];
                store_words<P>(w.t_fw + pos * P, fw[r]);
                ecnt += 1;
                earcs += dg[r];
            }
            if (threadIdx.x == 0) {
                w.tile_cnt[t] = tcnt;
                w.tile_arcs[t] = tarcs;
            }
        }
    }
    if (fused) return;  // the pull counted F_round and its active slots
    const unsigned long long bnf = block_sum(my_nf, red);
    const unsigned int wa = __reduce_or_sync(0xffffffffu, my_active);
    if ((threadIdx.x & 31) == 0 && wa) atomicOr(&s_active, wa);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (bnf) atomicAdd(&c->nf, bnf);
        if (s_active) atomicOr(&c->slot_active, s_active);
    }
}

// The pull (dense edge phase) of round `round`.  FUSE: the round also does
// the set update of round + 1 for the vertices it finishes (see k_phase_b);
// otherwise it leaves their new sources in acc.  Two instantiations keep the
// plain pull's code and registers as they are without the fused work.
template <int P, bool FUSE>
__device__ __forceinline__ void pull_round(const Wave& w, RoundCtl* c, RoundCtl* cn, int round,
                                           unsigned long long qlen, const uint32_t* fb, uint32_t* fbn, uint32_t stamp,
                                           const uint64_t* sall, unsigned int* s_work_p, uint64_t (*sor)[P],
                                           int32_t (*sadj)[32 * kPullSmall]) {
    // ---- pull: dense pass over every vertex that can still gain sources.
    // Plain: every vertex ORs the vis blocks of its frontier neighbours and
    // leaves the new part in acc for the next vertex phase.  Fused: it ORs the
    // sources new at its neighbours this round instead (nw[round & 1]; a
    // frontier neighbour's older sources are already in vis[v], and a
    // non-frontier neighbour's entry -- read without the bitmap test when the
    // frontier is dense; cleared per wave -- holds sources of an earlier
    // round, so neither adds anything), then does v's vertex phase of
    // round + 1 on the spot (pull_finish): vis is updated in place, which is
    // safe because a fused round reads no other vertex's vis.  Fused pulls
    // save the next vertex phase's pass over the frontier; graphs whose
    // clusters' frontiers rarely meet (a road grid) gain, power-law graphs do
    // not: the call's fused_pull chooses (autotuned).
    // Degree classes are consecutive rank ranges: big [0, nb), mid [nb, nb + nm),
    // small [nb + nm, nb + nm + ns).
    const bool sparse_round = w.n_big_s >= 0 && qlen * 32 < (unsigned long long)w.n;
    const int64_t nb = sparse_round ? w.n_big_s : w.n_big;
    const int64_t nm = sparse_round ? w.n_mid_s : w.n_mid;
    const int64_t ns = sparse_round ? w.n_small_s : w.n_small;
    const uint64_t* pieces = sparse_round ? w.pull_pieces_s : w.pull_pieces;
    const int64_t npieces = sparse_round ? w.n_pull_pieces_s : w.n_pull_pieces;
    const unsigned int active = c->slot_active;
    // gather source: vis (plain); fused: the round's record, or nw past the records
    const uint64_t* gsrc = !FUSE               ? w.vis
                           : round < w.hcap ? w.hist + (size_t)round * (size_t)w.n * P
                                            : ((round & 1) ? w.nw1 : w.nw0);
    uint64_t* nwn = (round & 1) ? w.nw0 : w.nw1;  // F_{round+1}'s new sources, written by pull_finish
    const int rn = round + 1;
    unsigned long long my_cnt = 0, my_sdeg = 0;
    unsigned int my_act = 0;
    const uint64_t* all = sall;  // ALL of each slot, read from shared memory where needed
    unsigned int& s_work = *s_work_p;
    // high-degree vertices: their lists are cut into kBigDeg-arc pieces that
    // all CTAs take from a counter; each piece ORs its part into acc[v].
    // Fused, the last piece of v to finish (a per-vertex counter, reset by
    // it) does v's set update; plain, the first piece to make acc[v] non-zero
    // counts v and acc[v] goes to the next vertex phase
    for (;;) {
        if (threadIdx.x == 0) s_work = atomicAdd(&c->piece_ctr, 1u);
        __syncthreads();
        const unsigned int p = s_work;
        __syncthreads();
        if (p >= npieces) break;
        const uint64_t pc = pieces[p];
        const int32_t v = (int32_t)(pc >> 32);
        const int64_t o0 = w.off[v], o1 = w.off[v + 1];
        const int64_t a0 = o0 + (int64_t)(uint32_t)pc * kBigDeg;
        const int64_t a1 = min(o1, a0 + kBigDeg);
        // acc[v] may be growing under other pieces: one thread reads it so that
        // every thread of the block decides on the same snapshot
        if (threadIdx.x == 0) {
            uint64_t vs[P], ac[P];
            load_words<P>(w.vis + (size_t)v * P, vs);
#pragma unroll
            for (int s = 0; s < P; ++s) ac[s] = __ldcg(reinterpret_cast<const unsigned long long*>(w.acc + (size_t)v * P + s));
#pragma unroll
            for (int s = 0; s < P; ++s) sor[1][s] = vs[s] | ac[s];
        }
        __syncthreads();
        uint64_t seen[P];
#pragma unroll
        for (int s = 0; s < P; ++s) seen[s] = sor[1][s];
        __syncthreads();
        const unsigned int um = unfinished<P>(seen, all, active);
        uint64_t acc[P];
#pragma unroll
        for (int s = 0; s < P; ++s) acc[s] = 0;
        if (!FUSE && !um) continue;  // uniform: seen comes from shared memory
        if (um) {
            for (int64_t b0 = a0; b0 < a1; b0 += Gath<P>::G * kThreads) {
                gather<P>(gsrc, fb, w.adj, b0 + threadIdx.x, kThreads, a1, acc);
#pragma unroll
                for (int s = 0; s < P; ++s) {
                    const uint64_t wa = warp_or(acc[s]);
                    if ((threadIdx.x & 31) == 0) sor[threadIdx.x >> 5][s] = wa;
                }
                __syncthreads();
                if (threadIdx.x < P) {
                    uint64_t x = 0;
                    for (int k = 0; k < kWarps; ++k) x |= sor[k][threadIdx.x];
                    sor[0][threadIdx.x] = x;
                }
                __syncthreads();
#pragma unroll
                for (int s = 0; s < P; ++s) acc[s] = sor[0][s];
                __syncthreads();
                if (missing_bits<P>(acc, seen, all, um) == 0) break;
            }
        }
        if (threadIdx.x == 0) {
            bool claim = false;
#pragma unroll
            for (int s = 0; s < P; ++s) {
                const uint64_t nb_ = acc[s] & ~seen[s];
                if (nb_) {
                    const unsigned long long old =
                        atomicOr(reinterpret_cast<unsigned long long*>(w.acc + (size_t)v * P + s), (unsigned long long)nb_);
                    claim |= (old == 0ull);
                }
            }
            if (FUSE) {
                __threadfence();  // this piece's ORs before its count
                const unsigned int npc = (unsigned int)((o1 - o0 + kBigDeg - 1) / kBigDeg);
                if (atomicAdd(w.piece_cnt + v, 1u) == npc - 1) {
                    // every piece of v has ORed its part into acc[v]: v's set update of round + 1
                    __threadfence();
                    w.piece_cnt[v] = 0u;
                    uint64_t vs[P], ac[P];
                    load_words<P>(w.vis + (size_t)v * P, vs);
#pragma unroll
                    for (int s = 0; s < P; ++s)
                        ac[s] = __ldcg(reinterpret_cast<const unsigned long long*>(w.acc + (size_t)v * P + s));
                    zero_words<P>(w.acc + (size_t)v * P);
                    if (pull_finish<P, true>(w, v, ac, vs, (uint32_t)(o1 - o0), rn, nwn, my_cnt, my_sdeg, my_act))
                        atomicOr(fbn + (v >> 5), 1u << (v & 31));
                }
            } else if (claim && atomicExch(w.rq + v, stamp) != stamp) {
                // the first piece to make acc[v] non-zero counts v once for F_{round+1};
                // acc[v] stays for the next vertex phase
                my_cnt += 1;
                my_sdeg += (unsigned long long)(o1 - o0);
                atomicOr(fbn + (v >> 5), 1u << (v & 31));
            }
        }
    }
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t gw = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t nw_total = ((int64_t)gridDim.x * kThreads) >> 5;
    // warp per mid-degree vertex
    for (int64_t i = gw; i < nm; i += nw_total) {
        const int32_t v = (int32_t)(nb + i);
        uint64_t vs[P];
        load_words<P>(w.vis + (size_t)v * P, vs);
        const unsigned int um = unfinished<P>(vs, all, active);
        if (!um) continue;
        const int64_t o0 = w.off[v], o1 = w.off[v + 1];
        uint64_t acc[P];
#pragma unroll
        for (int s = 0; s < P; ++s) acc[s] = 0;
        for (int64_t b0 = o0; b0 < o1; b0 += 32 * Gath<P>::G) {
            gather<P>(gsrc, fb, w.adj, b0 + lane, 32, o1, acc);
#pragma unroll
            for (int s = 0; s < P; ++s) acc[s] = warp_or(acc[s]);
            if (missing_bits<P>(acc, vs, all, um) == 0) break;
        }
        if (lane == 0 && pull_finish<P, FUSE>(w, v, acc, vs, (uint32_t)(o1 - o0), rn, nwn, my_cnt, my_sdeg, my_act))
            atomicOr(fbn + (v >> 5), 1u << (v & 31));
    }
    // low-degree vertices: a warp takes 32 consecutive ones, whose lists are
    // consecutive in the internal order, stages them in shared memory with
    // coalesced loads, then each lane scans its own list
    int32_t* wadj = sadj[wib];
    const int64_t small0 = nb + nm;
    for (int64_t g0 = gw * 32; g0 < ns; g0 += nw_total * 32) {
        const int64_t i = g0 + lane;
        const bool has = i < ns;
        const int32_t v = has ? (int32_t)(small0 + i) : 0;
        const int64_t o0 = has ? w.off[v] : 0, o1 = has ? w.off[v + 1] : 0;
        const int last = (int)((ns - 1 - g0) < 31 ? (ns - 1 - g0) : 31);
        const int64_t lo = __shfl_sync(0xffffffffu, o0, 0);
        const int64_t hi = __shfl_sync(0xffffffffu, o1, last);
        for (int64_t x = lo + lane; x < hi; x += 32) wadj[x - lo] = w.adj[x];
        __syncwarp();
        bool joined = false;
        if (has) {
            uint64_t vs[P];
            load_words<P>(w.vis + (size_t)v * P, vs);
            const unsigned int um = unfinished<P>(vs, all, active);
            if (um) {
                uint64_t acc[P];
#pragma unroll
                for (int s = 0; s < P; ++s) acc[s] = 0;
                for (int64_t e = o0; e < o1; e += Gath<P>::G) {
                    gather<P>(gsrc, fb, wadj - lo, e, 1, o1, acc);
                    if (missing_bits<P>(acc, vs, all, um) == 0) break;
                }
                joined = pull_finish<P, FUSE>(w, v, acc, vs, (uint32_t)(o1 - o0), rn, nwn, my_cnt, my_sdeg, my_act);
            }
        }
        // the 32 vertices are consecutive: their bits span at most two bitmap words
        const unsigned int jm = __ballot_sync(0xffffffffu, joined);
        if (lane == 0 && jm) {
            const int32_t v0 = (int32_t)(small0 + g0);
            const int sh = v0 & 31;
            atomicOr(fbn + (v0 >> 5), jm << sh);
            if (sh && (jm >> (32 - sh))) atomicOr(fbn + (v0 >> 5) + 1, jm >> (32 - sh));
        }
        __syncwarp();
    }
    // publish the next frontier's size, arcs and active slots: one atomic each per CTA
    __shared__ unsigned long long red[kWarps];
    __shared__ unsigned int s_act;
    if (threadIdx.x == 0) s_act = 0;
    const unsigned long long bc = block_sum(my_cnt, red);
    const unsigned long long bs = block_sum(my_sdeg, red);
    const unsigned int wact = __reduce_or_sync(0xffffffffu, my_act);
    if (lane == 0 && wact) atomicOr(&s_act, wact);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (bc) {
            atomicAdd(&cn->qlen, bc);
            atomicAdd(&cn->nf, bc);
        }
        if (bs) atomicAdd(&cn->sdeg, bs);
        if (s_act) atomicOr(&cn->slot_active, s_act);
        if (blockIdx.x == 0) {
            cn->dense = 1;
            cn->fused = FUSE ? 1 : 0;
        }
    }
}

// Phase B: the edge phase of round `round` in the direction phase A chose.
template <int P, bool FUSE>
__global__ void __launch_bounds__(kThreads, (P >= 8 ? 3 : 4)) k_phase_b(Wave w, int round) {
    constexpr int TILE = Geo<P>::kTile;
    // push and pull never run in the same launch: their staging buffers overlap
    constexpr int kPushPre = (4 * (kThreads + 1) + 15) / 16 * 16;
    constexpr int kPushBytes = kPushPre + 8 * kThreads + 8 * kThreads * P;
    constexpr int kPullBytes = 4 * kWarps * 32 * (int)kPullSmall;
    __shared__ __align__(16) unsigned char sraw[kPushBytes > kPullBytes ? kPushBytes : kPullBytes];
    uint32_t* spre = reinterpret_cast<uint32_t*>(sraw);                      // push: [kThreads + 1]
    int64_t* sost = reinterpret_cast<int64_t*>(sraw + kPushPre);             // push: [kThreads]
    uint64_t* sfw = reinterpret_cast<uint64_t*>(sraw + kPushPre + 8 * kThreads);  // push: [kThreads * P]
    int32_t(*sadj)[32 * kPullSmall] = reinterpret_cast<int32_t(*)[32 * kPullSmall]>(sraw);  // pull
    __shared__ uint64_t sall[P];
    __shared__ unsigned int s_work;
    __shared__ uint64_t sor[kWarps][P];
    if (w.round_dev) round = *w.round_dev;
    RoundCtl* c = w.ctl + round;
    const unsigned long long qlen = c->qlen;
    if (qlen == 0) return;
    if (threadIdx.x < P) sall[threadIdx.x] = (int)threadIdx.x < w.nslots ? w.slots[threadIdx.x].all : 0ull;
    __syncthreads();
    uint32_t* qn = (round & 1) ? w.q0 : w.q1;
    RoundCtl* cn = w.ctl + round + 1;
    const uint32_t stamp = (uint32_t)round + 2;  // F_{round+1}
    const bool pull = c->mode != 0;
    // F_round's bitmap (read) and F_{round+1}'s (written by whoever adds a vertex;
    // phase A of this round cleared it)
    // a dense frontier (over n/8) passes the membership test almost always: skip it then,
    // except in fused waves with round records, whose gather sources are not cleared per
    // wave (a non-frontier entry may hold another wave's sources)
    const bool test_all = FUSE && w.hcap > 0;
    const uint32_t* fb =
        (qlen * 8 > (unsigned long long)w.n && !test_all) ? nullptr : ((round & 1) ? w.fb1 : w.fb0);
    uint32_t* fbn = (round & 1) ? w.fb0 : w.fb1;

    if (!pull) {
        // big-list pieces: kBigDeg consecutive arcs of one hub per CTA step
        const unsigned int npieces = c->npieces;
        for (;;) {
            if (threadIdx.x == 0) s_work = atomicAdd(&c->piece_ctr, 1u);
            __syncthreads();
            const unsigned int p = s_work;
            if (p < npieces && threadIdx.x < P) sfw[threadIdx.x] = w.big_fw[(size_t)w.piece_ent[p] * P + threadIdx.x];
            __syncthreads();
            if (p >= npieces) break;
            const BigEntry be = w.big[w.piece_ent[p]];
            const int64_t a0 = (int64_t)w.piece_no[p] * kBigDeg;
            const int64_t a1 = min(be.deg, a0 + kBigDeg);
            for (int64_t a = a0 + threadIdx.x; a < a1; a += kThreads)
                push_arc<P>(w, sfw, (uint32_t)w.adj[be.ost + a], stamp, qn, cn, fbn);
            __syncthreads();
        }
        // tiles: entries of degree <= kBigDeg, arcs spread over the threads
        const bool dense = c->dense || (w.dense_div > 0 && qlen * (unsigned long long)w.dense_div > (unsigned long long)w.n);
        const unsigned long long span = dense ? (unsigned long long)w.n : qlen;
        const unsigned long long ntiles = (span + TILE - 1) / TILE;
        for (;;) {
            if (threadIdx.x == 0) s_work = atomicAdd(&c->tile_ctr, 1u);
            __syncthreads();
            const unsigned long long t = s_work;
            __syncthreads();
            if (t >= ntiles) break;
            const uint32_t cnt = w.tile_cnt[t];
            const uint32_t tarcs = w.tile_arcs[t];
            const unsigned long long base = t * TILE;
            for (uint32_t g0 = 0; g0 < cnt; g0 += kThreads) {
                const uint32_t ge = min((uint32_t)kThreads, cnt - g0);
                if (threadIdx.x < ge) {
                    const unsigned long long pos = base + g0 + threadIdx.x;
                    spre[threadIdx.x] = w.t_pre[pos];
                    sost[threadIdx.x] = w.t_ost[pos];
                }
                for (uint32_t i = threadIdx.x; i < ge * P; i += kThreads) sfw[i] = w.t_fw[(base + g0) * P + i];
                if (threadIdx.x == 0) spre[ge] = (g0 + ge < cnt) ? w.t_pre[base + g0 + ge] : tarcs;
                __syncthreads();
                const uint32_t a_lo = spre[0], a_hi = spre[ge];
                for (uint32_t a = a_lo + threadIdx.x; a < a_hi; a += kThreads) {
                    // last entry e with spre[e] <= a
                    int lo = 0, hi = (int)ge - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (spre[mid] <= a) lo = mid;
                        else hi = mid - 1;
                    }
                    push_arc<P>(w, sfw + lo * P, (uint32_t)w.adj[sost[lo] + (a - spre[lo])], stamp, qn, cn, fbn);
                }
                __syncthreads();
            }
        }
        return;
    }

    pull_round<P, FUSE>(w, c, cn, round, qlen, fb, fbn, stamp, sall, &s_work, sor, sadj);
}

// Writes the wave's internal rows to the caller's outputs: caller vertex v
// reads the row of its internal rank (coalesced writes per cluster).
template <int P>
__global__ void __launch_bounds__(kThreads) k_emit(Wave w, const int32_t* iperm) {
    __shared__ SlotDesc ss[P];
    if (threadIdx.x < w.nslots) ss[threadIdx.x] = w.slots[threadIdx.x];
    __syncthreads();
    const int d = w.d;
    for (int64_t v = (int64_t)blockIdx.x * kThreads + threadIdx.x; v < w.n; v += (int64_t)gridDim.x * kThreads) {
        const int64_t r = iperm ? iperm[v] : v;
        const uint8_t* dr = w.dist_r + (size_t)r * P;
        const uint64_t* mr = w.masks_r + (size_t)r * d * P;
        const uint16_t* wr = w.wmask_r + (size_t)r * P;
        // a slot that never reached v has stale subset words in the row: write zeros
        unsigned int reached = 0;
#pragma unroll
        for (int s = 0; s < P; ++s) {
            if (s >= w.nslots) continue;
            const uint8_t dv = dr[s];
            ss[s].dist[v] = dv;
            if (dv != 0xFF) reached |= 1u << s;
        }
        // slot by slot: a slot's d words are contiguous in the row; a word the
        // vertex phase did not write this wave (empty subset) is 0
#pragma unroll
        for (int s = 0; s < P; ++s) {
            if (s >= w.nslots) continue;
            const uint32_t wm = !((reached >> s) & 1u) || !d ? 0u : d > kZeroWords ? wr[s] : 0xFFFFu;
            for (int j = 0; j < d; ++j)
                ss[s].masks[(size_t)j * (size_t)w.n + v] = ((wm >> j) & 1u) ? mr[(size_t)s * d + j] : 0ull;
        }
    }
}

// Outputs from the round records (Algorithm 1's Delta_v and S_v[i], read off
// the rounds in which v carried new sources): for caller vertex v (internal
// rank u), Delta of a slot is the first recorded round with sources of that
// slot new at u, and S_v[i] is the record of round Delta + i, or empty when
// u was not in that round's frontier.  Every output word is written, the
// empty ones too, by the thread of v; the threads of a warp take consecutive
// v, so the words of a sector are written within a few instructions of one
// another.  at_cap: after phase A of round hcap - 1, rounds 0 .. hcap - 1
// (later rounds then write their outputs directly, over what this wrote);
// otherwise after the wave, its rounds -- unless the wave reached hcap - 1
// (done then) or, with bound_round > 0, its frontier after bound_round rounds
// was not empty (the wave runs again).
template <int P>
__global__ void __launch_bounds__(kThreads, (P >= 8 ? 2 : 4)) k_flush(Wave w, const int32_t* iperm, int round, int at_cap,
                                                     int bound_round) {
    constexpr int U = P >= 8 ? 2 : 4;  // rounds whose records are loaded together
    __shared__ SlotDesc ss[P];
    __shared__ int s_rounds;
    if (w.round_dev) round = *w.round_dev;
    if (threadIdx.x == 0) {
        int R = -1;
        if (at_cap) {
            if (round == w.hcap - 1 && w.ctl[round].qlen > 0) R = w.hcap;
        } else if (!(bound_round > 0 && w.ctl[bound_round].qlen != 0)) {
            int r = 0;
            while (r < w.hcap && w.ctl[r].qlen > 0) ++r;
            if (r < w.hcap) R = r;
        }
        s_rounds = R;
    }
    if (threadIdx.x < w.nslots) ss[threadIdx.x] = w.slots[threadIdx.x];
    __syncthreads();
    const int R = s_rounds;
    if (R < 0) return;
    const int64_t n = w.n;
    const int d = w.d;
    const size_t words = (size_t)((n + 31) / 32);
    for (int64_t v = (int64_t)blockIdx.x * kThreads + threadIdx.x; v < n; v += (int64_t)gridDim.x * kThreads) {
        const uint32_t u = iperm ? (uint32_t)iperm[v] : (uint32_t)v;
        const uint32_t* fbu = w.fbh + (u >> 5);
        const int sh = (int)(u & 31);
        int dl[P];
        uint32_t wm[P];
#pragma unroll
        for (int s = 0; s < P; ++s) {
            dl[s] = -1;
            wm[s] = 0;
        }
        for (int b0 = 0; b0 < R; b0 += 64) {
            // the rounds of this block in which u was in the frontier, from
            // independent bitmap loads; then their records, U at a time
            const int nb = R - b0 < 64 ? R - b0 : 64;
            uint64_t m = 0;
#pragma unroll 8
            for (int k = 0; k < nb; ++k) m |= (uint64_t)((fbu[(size_t)(b0 + k) * words] >> sh) & 1u) << k;
            while (m) {
                int rr[U];
                uint64_t x[U][P];
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    rr[k] = m ? b0 + __ffsll((long long)m) - 1 : -1;
                    m &= m - 1;
                }
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    if (rr[k] >= 0) load_words<P>(w.hist + ((size_t)rr[k] * (size_t)n + u) * P, x[k]);
                    else {
#pragma unroll
                        for (int s = 0; s < P; ++s) x[k][s] = 0;
                    }
                }
#pragma unroll
                for (int k = 0; k < U; ++k) {
#pragma unroll
                    for (int s = 0; s < P; ++s) {
                        if (s >= w.nslots || !x[k][s]) continue;
                        if (dl[s] < 0) dl[s] = rr[k];
                        const int j = rr[k] - dl[s];
                        if (j < d) {
                            ss[s].masks[(size_t)j * (size_t)n + v] = x[k][s];
                            wm[s] |= 1u << j;
                        } else if (j > d) {
                            set_status(w.status, CBFS_E_DIAMETER);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int s = 0; s < P; ++s) {
            if (s >= w.nslots) continue;
            ss[s].dist[v] = dl[s] < 0 ? (uint8_t)0xFF : (uint8_t)dl[s];
            for (int j = 0; j < d; ++j)
                if (!((wm[s] >> j) & 1u)) ss[s].masks[(size_t)j * (size_t)n + v] = 0ull;
        }
    }
}

// k_flush for packed waves: a slot word holds several clusters (members),
// each a contiguous range of its bits.  Caller vertex v's outputs of every
// member come from the same round records, masked to the member's bits and
// shifted down to its own bit order: Delta is the first recorded round with
// bits of the member new at u, S_v[i] the member's bits of the record of
// round Delta + i.  Word by word, in two passes: the first walks v's
// records and keeps each member's Delta in shared memory (the member of a bit
// comes from the wave's bit table); the second writes member by member and
// subset by subset, every lane of a warp at once, so that a warp's stores
// fill whole sectors of an output row.
template <int P>
__global__ void __launch_bounds__(kThreads) k_flush_packed(Wave w, const int32_t* iperm, int round, int at_cap,
                                                            int bound_round) {
    constexpr int U = 4;
    __shared__ MemberDesc sm[P * kWordMembers];
    __shared__ uint8_t sbit[P * 64];
    __shared__ uint8_t sdl[kWordMembers][kThreads];
    __shared__ int s_first[P + 1];
    __shared__ int s_rounds;
    if (w.round_dev) round = *w.round_dev;
    if (threadIdx.x == 0) {
        int R = -1;
        if (at_cap) {
            if (round == w.hcap - 1 && w.ctl[round].qlen > 0) R = w.hcap;
        } else if (!(bound_round > 0 && w.ctl[bound_round].qlen != 0)) {
            int r = 0;
            while (r < w.hcap && w.ctl[r].qlen > 0) ++r;
            if (r < w.hcap) R = r;
        }
        s_rounds = R;
    }
    const int nm = w.nmembers < P * kWordMembers ? w.nmembers : P * kWordMembers;
    for (int i = threadIdx.x; i < nm; i += kThreads) sm[i] = w.members[i];
    for (int i = threadIdx.x; i < P * 64; i += kThreads) sbit[i] = w.bit_member[i];
    if (threadIdx.x <= P) {
        // members are stored word by word: word s holds [s_first[s], s_first[s + 1])
        int f = nm;
        for (int i = 0; i < nm; ++i)
            if (w.members[i].word >= (int)threadIdx.x) {
                f = i;
                break;
            }
        s_first[threadIdx.x] = f;
    }
    __syncthreads();
    const int R = s_rounds;
    if (R < 0) return;
    const int64_t n = w.n;
    const int d = w.d;
    const size_t words = (size_t)((n + 31) / 32);
    const int t = threadIdx.x;
    for (int64_t v = (int64_t)blockIdx.x * kThreads + threadIdx.x; v < n; v += (int64_t)gridDim.x * kThreads) {
        const uint32_t u = iperm ? (uint32_t)iperm[v] : (uint32_t)v;
        const uint32_t* fbu = w.fbh + (u >> 5);
        const int sh = (int)(u & 31);
        // the rounds in which u was in the frontier (R <= 255: four 64-bit blocks)
        uint64_t mk[4] = {0, 0, 0, 0};
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int nb = R - 64 * b < 64 ? R - 64 * b : 64;  // the block's recorded rounds
#pragma unroll 8
            for (int k = 0; k < nb; ++k) mk[b] |= (uint64_t)((fbu[(size_t)(64 * b + k) * words] >> sh) & 1u) << k;
        }
        for (int s = 0; s < w.nslots; ++s) {
            const int m0 = s_first[s], mc = s_first[s + 1] - m0;
            for (int i = 0; i < mc; ++i) sdl[i][t] = 0xFF;
            // pass 1: each member's Delta (its first recorded round), and any member
            // bits arriving more than d rounds after it (CBFS_E_DIAMETER)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                uint64_t m = mk[b];
                while (m) {
                    int rr[U];
                    uint64_t x[U];
#pragma unroll
                    for (int k = 0; k < U; ++k) {
                        rr[k] = m ? 64 * b + __ffsll((long long)m) - 1 : -1;
                        m &= m - 1;
                    }
#pragma unroll
                    for (int k = 0; k < U; ++k)
                        x[k] = rr[k] >= 0 ? w.hist[((size_t)rr[k] * (size_t)n + u) * P + s] : 0ull;
#pragma unroll
                    for (int k = 0; k < U; ++k) {
                        uint64_t left = x[k];
                        while (left) {
                            const int bt = __ffsll((long long)left) - 1;
                            const int i = (int)sbit[s * 64 + bt] - m0;
                            if (i < 0 || i >= mc) {  // a bit outside every member: never for host-built tables
                                set_status(w.status, CBFS_E_INVALID);
                                break;
                            }
                            left &= ~(sm[m0 + i].mask | (1ull << bt));  // bit bt always goes: the loop ends
                            const int dl = sdl[i][t];
                            if (dl == 0xFF) sdl[i][t] = (uint8_t)rr[k];
                            else if (rr[k] - dl > d) set_status(w.status, CBFS_E_DIAMETER);
                        }
                    }
                }
            }
            // pass 2: member by member and subset by subset, every lane at once
            // (consecutive callers' words of one output row), each word written once
            for (int i = 0; i < mc; ++i) {
                const MemberDesc& M = sm[m0 + i];
                const int dl = sdl[i][t];
                M.dist[v] = (uint8_t)dl;
                for (int j = 0; j < d; ++j) {
                    const int r = dl + j;  // dl == 0xFF: never reached, r > 254 >= R
                    // the block of round r by selects (an indexed register array would go to memory)
                    const uint64_t blk = r < 64 ? mk[0] : r < 128 ? mk[1] : r < 192 ? mk[2] : mk[3];
                    uint64_t x = 0;
                    if (r < R && ((blk >> (r & 63)) & 1ull)) x = w.hist[((size_t)r * (size_t)n + u) * P + s];
                    M.masks[(size_t)j * (size_t)n + v] = (x & M.mask) >> M.off;
                }
            }
        }
    }
}

template __global__ void k_phase_a<1>(Wave, int);
template __global__ void k_phase_a<2>(Wave, int);
template __global__ void k_phase_a<4>(Wave, int);
template __global__ void k_phase_a<8>(Wave, int);
template __global__ void k_phase_b<1, false>(Wave, int);
template __global__ void k_phase_b<2, false>(Wave, int);
template __global__ void k_phase_b<4, false>(Wave, int);
template __global__ void k_phase_b<8, false>(Wave, int);
template __global__ void k_phase_b<1, true>(Wave, int);
template __global__ void k_phase_b<2, true>(Wave, int);
template __global__ void k_phase_b<4, true>(Wave, int);
template __global__ void k_phase_b<8, true>(Wave, int);
template __global__ void k_emit<1>(Wave, const int32_t*);
template __global__ void k_emit<2>(Wave, const int32_t*);
template __global__ void k_emit<4>(Wave, const int32_t*);
template __global__ void k_emit<8>(Wave, const int32_t*);
template __global__ void k_flush<1>(Wave, const int32_t*, int, int, int);
template __global__ void k_flush<2>(Wave, const int32_t*, int, int, int);
template __global__ void k_flush<4>(Wave, const int32_t*, int, int, int);
template __global__ void k_flush<8>(Wave, const int32_t*, int, int, int);
template __global__ void k_flush_packed<1>(Wave, const int32_t*, int, int, int);
template __global__ void k_flush_packed<2>(Wave, const int32_t*, int, int, int);
template __global__ void k_flush_packed<4>(Wave, const int32_t*, int, int, int);
template __global__ void k_flush_packed<8>(Wave, const int32_t*, int, int, int);

cudaError_t launch_round(const Wave& w, int round, int grid, cudaStream_t st, int which, const int32_t* iperm) {
    switch (w.P) {
#define CBFS_CASE(PP)                                                       \
    case PP:                                                                \
        if (which == 0) k_phase_a<PP><<<w.grid_a > 0 ? w.grid_a : grid, kThreads, 0, st>>>(w, round); \
        else if (which == 1 && w.fused_pull) k_phase_b<PP, true><<<grid, kThreads, 0, st>>>(w, round); \
        else if (which == 1) k_phase_b<PP, false><<<grid, kThreads, 0, st>>>(w, round); \
        else k_emit<PP><<<grid, kThreads, 0, st>>>(w, iperm);               \
        break;
        CBFS_CASE(1)
        CBFS_CASE(2)
        CBFS_CASE(4)
        CBFS_CASE(8)
#undef CBFS_CASE
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_flush(const Wave& w, int round, int grid, cudaStream_t st, int at_cap, int bound_round,
                         const int32_t* iperm) {
    if (w.nmembers) {
        // twice the edge phase's CTAs: the packed flush holds fewer registers, more of
        // its CTAs fit an SM, and they hide the record loads' latency (measured 1.7 %
        // on a 256-cluster launch)
        grid *= 2;
        switch (w.P) {
            case 1: k_flush_packed<1><<<grid, kThreads, 0, st>>>(w, iperm, round, at_cap, bound_round); break;
            case 2: k_flush_packed<2><<<grid, kThreads, 0, st>>>(w, iperm, round, at_cap, bound_round); break;
            case 4: k_flush_packed<4><<<grid, kThreads, 0, st>>>(w, iperm, round, at_cap, bound_round); break;
            case 8: k_flush_packed<8><<<grid, kThreads, 0, st>>>(w, iperm, round, at_cap, bound_round); break;
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    switch (w.P) {
        case 1: k_flush<1><<<grid, kThreads, 0, st>>>(w, iperm, round, at_cap, bound_round); break;
        case 2: k_flush<2><<<grid, kThreads, 0, st>>>(w, iperm, round, at_cap, bound_round); break;
        case 4: k_flush<4><<<grid, kThreads, 0, st>>>(w, iperm, round, at_cap, bound_round); break;
        case 8: k_flush<8><<<grid, kThreads, 0, st>>>(w, iperm, round, at_cap, bound_round); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}


}  // namespace cbfs

namespace {

// Graph check: ids in range, no self loop, lists strictly increasing (so no
// repeated arc), and symmetry.  Symmetry is checked by counting: with a
// strict order on vertices (the internal rank: higher degree first), every
// arc v -> u whose head u comes after v must have its reverse, found by a
// binary search in u's list -- the shorter one -- and those "forward" arcs
// must be exactly half of all arcs.  (The forward arcs' reverses are
// distinct backward arcs, so any backward arc without a forward partner
// would make the backward ones outnumber the forward ones.)  One thread,
// warp or CTA per vertex by degree class; flag = 1 on any failure.
__device__ __forceinline__ bool arc_ok(int64_t n, const int64_t* off, const int32_t* adj, const int32_t* rank,
                                       int64_t v, int64_t e, int64_t o0, unsigned long long& fwd) {
    const int32_t u = adj[e];
    if (u < 0 || (int64_t)u >= n || (int64_t)u == v) return false;
    if (e > o0 && adj[e - 1] >= u) return false;
    if (rank[u] < rank[v]) return true;  // backward arc: counted from its partner
    fwd += 1;
    int64_t lo = off[u], hi = off[u + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)adj[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo < off[u + 1] && (int64_t)adj[lo] == v;
}

__global__ void k_validate(int64_t n, const int64_t* off, const int32_t* adj, const int32_t* rank,
                           const int32_t* pl_small, int64_t n_small, const int32_t* pl_mid, int64_t n_mid,
                           const int32_t* pl_big, int64_t n_big, int* flag, unsigned long long* forward) {
    bool ok = true;
    unsigned long long fwd = 0;
    for (int64_t i = blockIdx.x; i < n_big; i += gridDim.x) {
        const int64_t v = pl_big[i];
        const int64_t o0 = off[v], o1 = off[v + 1];
        for (int64_t e = o0 + threadIdx.x; e < o1; e += blockDim.x) ok &= arc_ok(n, off, adj, rank, v, e, o0, fwd);
    }
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = gw; i < n_mid; i += nwarps) {
        const int64_t v = pl_mid[i];
        const int64_t o0 = off[v], o1 = off[v + 1];
        for (int64_t e = o0 + lane; e < o1; e += 32) ok &= arc_ok(n, off, adj, rank, v, e, o0, fwd);
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_small; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = pl_small[i];
        const int64_t o0 = off[v], o1 = off[v + 1];
        for (int64_t e = o0; e < o1; ++e) ok &= arc_ok(n, off, adj, rank, v, e, o0, fwd);
    }
    if (!ok) atomicExch(flag, 1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fwd += __shfl_xor_sync(0xffffffffu, fwd, o);
    if (lane == 0 && fwd) atomicAdd(forward, fwd);
}

// Work counters from outputs: per (cluster, vertex) the number of non-empty
// subsets among S_v[0..d] (S_v[d] implied).
__global__ void k_output_stats(int64_t n, int d, const int64_t* off, const uint8_t* dist, const uint64_t* masks,
                               const uint64_t* alls, int C, unsigned long long* out /*[C][4]*/) {
    __shared__ unsigned long long red[kWarps];
    const int c = blockIdx.y;
    if (c >= C) return;
    const uint8_t* dc = dist + (size_t)c * (size_t)n;
    const uint64_t* mc = masks + (size_t)c * (size_t)d * (size_t)n;
    unsigned long long V = 0, A = 0, R = 0, rounds = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t dd = dc[v];
        if (dd == 0xFF) continue;
        const unsigned long long deg = (unsigned long long)(off[v + 1] - off[v]);
        uint64_t seen = 0;
        int cnt = 0, last = 0;
        for (int i = 0; i < d; ++i) {
            const uint64_t m = mc[(size_t)i * (size_t)n + v];
            if (m) { cnt++; last = i; }
            seen |= m;
        }
        if (alls[c] & ~seen) { cnt++; last = d; }
        V += cnt;
        A += (unsigned long long)cnt * deg;
        R += deg;
        const unsigned long long rr = (unsigned long long)dd + (unsigned long long)last + 1;
        rounds = rr > rounds ? rr : rounds;
    }
    const unsigned long long bV = block_sum(V, red);
    const unsigned long long bA = block_sum(A, red);
    const unsigned long long bR = block_sum(R, red);
    unsigned long long m = rounds;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(0xffffffffu, m, o);
        m = x > m ? x : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&out[c * 4 + 3], m);
    if (threadIdx.x == 0) {
        atomicAdd(&out[c * 4 + 0], bV);
        atomicAdd(&out[c * 4 + 1], bA);
        atomicAdd(&out[c * 4 + 2], bR);
    }
}

}  // namespace

// ------------------------------------------------------------- host side

struct cbfs_graph_s {
    int64_t n = 0, nnz = 0;
    int64_t* off = nullptr;    // caller's CSR offsets (kept for output statistics)
    int32_t* adj = nullptr;    // caller's adjacency (freed once relabelled)
    int64_t* off_r = nullptr;  // relabelled CSR the traversal runs on
    int32_t* adj_r = nullptr;
    int32_t* perm = nullptr;   // rank -> caller's id
    int32_t* iperm_d = nullptr;  // caller's id -> rank (device, for the output emit)
    uint8_t* dist_r = nullptr;   // internal output rows of a wave
    uint16_t* wmask_r = nullptr; // per vertex and slot: which subset words the wave wrote
    uint64_t* masks_r = nullptr;
    int64_t masks_r_cap = 0;
    uint64_t* hist = nullptr;    // round records of waves with fused pulls ([rounds][n][P])
    int64_t hist_cap = 0;
    uint32_t* fbh = nullptr;     // their frontier bitmaps ([rounds][bitmap words])
    int64_t fbh_cap = 0;
    uint64_t* pull_pieces = nullptr;  // (rank << 32 | piece) of every vertex of degree > kPullMid
    int64_t n_small = 0, n_mid = 0, n_big = 0;  // degree classes of the default thresholds
    int64_t big_vertices = 0, big_pieces = 0;
    // pull classes for a call's thresholds (cbfs_tune_t small_deg, mid_deg, sparse_mid_deg)
    // are rank ranges sized from this histogram; hub piece lists are kept per mid threshold
    std::vector<unsigned long long> deg_count;  // vertices of degree 0..kMaxMidDeg, then above
    struct HubPieces {
        int mid;
        uint64_t* d;  // owned, except the create-time list (== pull_pieces)
        int64_t count;
    };
    std::vector<HubPieces> pieces;
    int grid_p[4] = {0, 0, 0, 0};  // edge-phase grid for P = 1, 2, 4, 8 (SMs x resident CTAs)
    int grid_a[4] = {0, 0, 0, 0};  // vertex-phase grid (latency-bound: as many CTAs as fit)
    int device = 0;
    // scratch, sized for cap_slots clusters in flight
    int cap_slots = 0;
    uint64_t* vis = nullptr;
    uint64_t* acc = nullptr;
    uint64_t* nw = nullptr;        // nw0 | nw1, [2][n][P]
    uint32_t* piece_cnt = nullptr;
    uint32_t* rq = nullptr;
    uint32_t* q0 = nullptr;
    uint32_t* q1 = nullptr;
    uint32_t* fb = nullptr;  // two frontier bitmaps
    uint32_t* t_pre = nullptr;
    int64_t* t_ost = nullptr;
    uint64_t* t_fw = nullptr;
    uint32_t* tile_cnt = nullptr;
    uint32_t* tile_arcs = nullptr;
    BigEntry* big = nullptr;
    uint64_t* big_fw = nullptr;
    uint32_t* piece_ent = nullptr;
    uint32_t* piece_no = nullptr;
    RoundCtl* ctl = nullptr;
    int* status = nullptr;
    // per-call buffers, grown on demand
    SlotDesc* slots = nullptr;
    int64_t slots_cap = 0;
    uint64_t* seeds = nullptr;
    int64_t seeds_cap = 0;
    MemberDesc* members = nullptr;  // packed waves: member tables and bit tables of a call
    int64_t members_cap = 0;
    uint8_t* bitm = nullptr;
    int64_t bitm_cap = 0;
    // pinned host staging: the slot tables and seeds of a call are uploaded
    // from ring entry (call number % kUploadRing); a call waits for the upload
    // of the call kUploadRing calls earlier before it rewrites that entry, so
    // stream-ordered calls can be queued without the host overwriting a copy
    // still in flight
    unsigned long long* h_q = nullptr;  // [kMaxRounds + 2]
    static constexpr int kUploadRing = 4;
    struct Upload {
        SlotDesc* slots = nullptr;
        int64_t slots_cap = 0;
        uint64_t* seeds = nullptr;
        int64_t seeds_cap = 0;
        MemberDesc* members = nullptr;
        int64_t members_cap = 0;
        uint8_t* bitm = nullptr;
        int64_t bitm_cap = 0;
        cudaEvent_t done = nullptr;
    };
    Upload up[kUploadRing];
    uint64_t calls = 0;
    // kernel accounting (cbfs_profile)
    bool timing = false;
    std::vector<cudaEvent_t> events;  // pool, reused every call
    std::vector<int> event_kind;      // kind of the launch bracketed by events [2i, 2i+1]
    int events_used = 0;
    uint64_t launches[3] = {0, 0, 0};
    double ms[3] = {0, 0, 0};
    uint64_t total_launches = 0;
    // graph mode: device round counter, capture streams, instantiated graphs
    int* round_dev = nullptr;
    unsigned long long* iters = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t cap_stream2 = nullptr;
    struct GraphEntry {
        uint64_t key;
        cudaGraphExec_t exec;
        cudaEvent_t done;  // recorded after the latest launch: an evicted graph is destroyed once it has run
    };
    std::vector<GraphEntry> graphs;  // most recently used last
    int* wave_flags = nullptr;       // host-driven: waves that needed more rounds than enqueued
    int64_t wave_flags_cap = 0;
    // staged outputs (host destinations, or labels without outputs): a ring
    // of wave buffers, copied out on copy_stream while later waves traverse
    uint8_t* stage = nullptr;
    int64_t stage_cap = 0;
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> ev_emit, ev_copy;  // one pair per ring slot
};

namespace {

thread_local cudaError_t g_last_cuda_error = cudaSuccess;

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) {                   \
            g_last_cuda_error = e_;                \
            return e_ == cudaErrorMemoryAllocation \
                       ? CBFS_E_NOMEM              \
                       : CBFS_E_CUDA;              \
        }                                          \
    } while (0)

template <class T>
int dev_alloc(T** p, int64_t count) {
    *p = nullptr;
    if (count < 1) count = 1;
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (size_t)count);
    if (e != cudaSuccess) {
        g_last_cuda_error = e;
        cudaGetLastError();
        *p = nullptr;
        return CBFS_E_NOMEM;
    }
    return CBFS_OK;
}

template <class T>
void dev_free(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

void free_scratch(cbfs_graph_s* g) {
    dev_free(g->vis);
    dev_free(g->acc);
    dev_free(g->nw);
    dev_free(g->piece_cnt);
    dev_free(g->rq);
    dev_free(g->q0);
    dev_free(g->q1);
    dev_free(g->fb);
    dev_free(g->dist_r);
    dev_free(g->wmask_r);
    dev_free(g->t_pre);
    dev_free(g->t_ost);
    dev_free(g->t_fw);
    dev_free(g->tile_cnt);
    dev_free(g->tile_arcs);
    dev_free(g->big);
    dev_free(g->big_fw);
    dev_free(g->piece_ent);
    dev_free(g->piece_no);
    g->cap_slots = 0;
}

int ensure_scratch(cbfs_graph_s* g, int P) {
    if (g->cap_slots >= P) return CBFS_OK;
    free_scratch(g);
    const ScratchSizes z = scratch_sizes(g->n, P);
    int rc = CBFS_OK;
    if (!rc) rc = dev_alloc(&g->vis, z.state);
    if (!rc) rc = dev_alloc(&g->acc, z.state);
    if (!rc) rc = dev_alloc(&g->nw, 2 * z.state);
    if (!rc) rc = dev_alloc(&g->piece_cnt, z.queue);
    if (!rc && cudaMemset(g->piece_cnt, 0, sizeof(uint32_t) * (size_t)std::max<int64_t>(z.queue, 1)) != cudaSuccess)
        rc = CBFS_E_CUDA;
    if (!rc) rc = dev_alloc(&g->rq, z.queue);
    if (!rc) rc = dev_alloc(&g->q0, z.queue);
    if (!rc) rc = dev_alloc(&g->q1, z.queue);
    if (!rc) rc = dev_alloc(&g->fb, 2 * z.bitmap);
    if (!rc) rc = dev_alloc(&g->dist_r, z.state);
    if (!rc) rc = dev_alloc(&g->wmask_r, z.state);
    if (!rc) rc = dev_alloc(&g->t_pre, z.list);
    if (!rc) rc = dev_alloc(&g->t_ost, z.list);
    if (!rc) rc = dev_alloc(&g->t_fw, z.list * P);
    if (!rc) rc = dev_alloc(&g->tile_cnt, z.tiles);
    if (!rc) rc = dev_alloc(&g->tile_arcs, z.tiles);
    if (!rc) rc = dev_alloc(&g->big, g->big_vertices);
    if (!rc) rc = dev_alloc(&g->big_fw, g->big_vertices * P);
    if (!rc) rc = dev_alloc(&g->piece_ent, g->big_pieces);
    if (!rc) rc = dev_alloc(&g->piece_no, g->big_pieces);
    if (rc) {
        free_scratch(g);
        return rc;
    }
    g->cap_slots = P;
    return CBFS_OK;
}

template <class T>
int ensure_dev(T** p, int64_t* cap, int64_t want) {
    if (*cap >= want) return CBFS_OK;
    dev_free(*p);
    *cap = 0;
    int rc = dev_alloc(p, want);
    if (rc) return rc;
    *cap = want;
    return CBFS_OK;
}

template <class T>
int ensure_pinned(T** p, int64_t* cap, int64_t want) {
    if (*cap >= want) return CBFS_OK;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMallocHost((void**)p, sizeof(T) * (size_t)std::max<int64_t>(want, 1));
    if (e != cudaSuccess) {
        g_last_cuda_error = e;
        cudaGetLastError();
        *p = nullptr;
        return CBFS_E_NOMEM;
    }
    *cap = want;
    return CBFS_OK;
}

// Opens the event bracket of one launch of the given kind when timing.
int prof_begin(cbfs_graph_s* g, int kind, cudaStream_t st) {
    g->launches[kind] += 1;
    g->total_launches += 1;
    if (!g->timing) return -1;
    const int i = g->events_used;
    if ((int)g->events.size() < 2 * (i + 1)) {
        for (int j = 0; j < 2; ++j) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            g->events.push_back(e);
        }
        g->event_kind.push_back(kind);
    }
    g->event_kind[i] = kind;
    g->events_used = i + 1;
    cudaEventRecord(g->events[2 * i], st);
    return i;
}

void prof_end(cbfs_graph_s* g, int slot, cudaStream_t st) {
    if (slot >= 0) cudaEventRecord(g->events[2 * slot + 1], st);
}

// Folds the finished brackets into the totals (the stream has been synchronised).
void prof_collect(cbfs_graph_s* g) {
    for (int i = 0; i < g->events_used; ++i) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, g->events[2 * i], g->events[2 * i + 1]) == cudaSuccess) g->ms[g->event_kind[i]] += t;
    }
    g->events_used = 0;
}

int check_clusters(const cbfs_graph_s* g, const int32_t* src, const int32_t* coff, int C, int d) {
    if (d < 0 || d > 15) return CBFS_E_INVALID;
    if (coff[0] != 0) return CBFS_E_INVALID;
    int32_t buf[64];
    for (int c = 0; c < C; ++c) {
        const int64_t k = (int64_t)coff[c + 1] - coff[c];
        if (k < 1 || k > 64) return CBFS_E_INVALID;
        for (int64_t j = 0; j < k; ++j) {
            const int32_t v = src[coff[c] + j];
            if (v < 0 || (int64_t)v >= g->n) return CBFS_E_INVALID;
            buf[j] = v;
        }
        std::sort(buf, buf + k);
        for (int64_t j = 1; j < k; ++j)
            if (buf[j] == buf[j - 1]) return CBFS_E_INVALID;
    }
    return CBFS_OK;
}

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

// Records every wave of a call as one CUDA graph: per wave the state
// memsets, the seed kernel, a conditional WHILE node whose body is phase A,
// phase B and k_round_cond, then the emit and the source check.
int build_graph(cbfs_graph_s* g, const std::vector<Wave>& waves, const std::vector<int64_t>& seed_off, int grid,
                int64_t bm_words, cudaGraphExec_t* out) {
    *out = nullptr;
    if (!g->cap_stream) {
        CK(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&g->cap_stream2, cudaStreamNonBlocking));
    }
    cudaStream_t cs = g->cap_stream, cs2 = g->cap_stream2;
    const int64_t n = g->n;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (size_t wv = 0; wv < waves.size() && e == cudaSuccess; ++wv) {
        const Wave& w = waves[wv];
        const int P = w.P;
        const int cnt = (int)(seed_off[wv + 1] - seed_off[wv]);
        e = cudaMemsetAsync(w.vis, 0, sizeof(uint64_t) * (size_t)P * (size_t)n, cs);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.acc, 0, sizeof(uint64_t) * (size_t)P * (size_t)n, cs);
        if (e == cudaSuccess && w.fused_pull && !w.hcap)  // a fused pull round may read any vertex's entry
            e = cudaMemsetAsync(w.nw0, 0, sizeof(uint64_t) * 2 * (size_t)P * (size_t)n, cs);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.rq, 0, sizeof(uint32_t) * (size_t)n, cs);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.fb0, 0, sizeof(uint32_t) * 2 * (size_t)bm_words, cs);
        if (e == cudaSuccess && w.dist_r) e = cudaMemsetAsync(w.dist_r, 0xFF, (size_t)P * (size_t)n, cs);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.ctl, 0, sizeof(RoundCtl) * kMaxRounds, cs);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.round_dev, 0, sizeof(int), cs);
        if (e != cudaSuccess) break;
        if (!w.dist_r && !w.hcap) k_clear_outputs<<<grid, kThreads, 0, cs>>>(w);
        k_seed<<<1, kThreads, 0, cs>>>(w, g->seeds + seed_off[wv], cnt);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        // the round loop: a conditional WHILE node spliced into the capture
        cudaStreamCaptureStatus cst;
        cudaGraph_t cg = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        if ((e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &ndeps)) != cudaSuccess) break;
        cudaGraphConditionalHandle h;
        if ((e = cudaGraphConditionalHandleCreate(&h, cg, 1, cudaGraphCondAssignDefault)) != cudaSuccess) break;
        cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode;
        if ((e = cudaGraphAddNode(&cnode, cg, deps, nullptr, ndeps, &cp)) != cudaSuccess) break;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if ((e = cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
            cudaSuccess)
            break;
        if ((e = cudaStreamBeginCaptureToGraph(cs2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
            cudaSuccess)
            break;
        cudaError_t eb = launch_round(w, 0, grid, cs2, 0);
        if (eb == cudaSuccess && w.hcap > 0) eb = launch_flush(w, 0, grid, cs2, 1, 0, g->iperm_d);  // at hcap - 1
        if (eb == cudaSuccess) eb = launch_round(w, 0, grid, cs2, 1);
        if (eb == cudaSuccess) {
            k_round_cond<<<1, 32, 0, cs2>>>(w, h);
            eb = cudaGetLastError();
        }
        cudaGraph_t body_out = nullptr;
        e = cudaStreamEndCapture(cs2, &body_out);
        if (e == cudaSuccess) e = eb;
        if (e != cudaSuccess) break;
        if (w.dist_r && (e = launch_round(w, 0, grid, cs, 2, g->iperm_d)) != cudaSuccess) break;
        if (!w.dist_r && w.hcap > 0 && (e = launch_flush(w, 0, grid, cs, 0, 0, g->iperm_d)) != cudaSuccess) break;
        k_check_sources<<<1, kThreads, 0, cs>>>(w, g->seeds + seed_off[wv], cnt, 0, nullptr);
        e = cudaGetLastError();
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = ee;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        g_last_cuda_error = e;
        cudaGetLastError();
        *out = nullptr;
        return CBFS_E_CUDA;
    }
    return CBFS_OK;
}

// Rounds of round records for a wave with fused pulls (cbfs_tune_t
// stage_rounds): < 0 none; > 0 that many (at most 255, so that a recorded
// round is a valid Delta); 0 = as many as fit a quarter of the free device
// memory (records already held count as free), at most kStageAuto.  Grows
// the records to that size.
int stage_rounds(cbfs_graph_s* g, const cbfs_tune_t* tune, int P, int* out) {
    *out = 0;
    const int64_t n = g->n;
    int want = tune ? tune->stage_rounds : 0;
    if (want < 0 || n == 0) return CBFS_OK;
    const int64_t words = (n + 31) / 32;
    const size_t per_round = sizeof(uint64_t) * (size_t)n * (size_t)P + sizeof(uint32_t) * (size_t)words;
    if (want == 0) {
        size_t fr = 0, tot = 0;
        CK(cudaMemGetInfo(&fr, &tot));
        const size_t held = sizeof(uint64_t) * (size_t)g->hist_cap + sizeof(uint32_t) * (size_t)g->fbh_cap;
        want = (int)std::min<size_t>((size_t)kStageAuto, (fr / 4 + held) / per_round);
        if (want == 0) return CBFS_OK;
    }
    want = std::min(want, 255);
    int rc = ensure_dev(&g->hist, &g->hist_cap, (int64_t)want * n * P);
    if (!rc) rc = ensure_dev(&g->fbh, &g->fbh_cap, (int64_t)want * words);
    if (rc) return rc;
    *out = want;
    return CBFS_OK;
}

// Clusters per wave: the requested slot count rounded down to a power of
// two (1, 2, 4, 8), no wider than the number of clusters.
int slots_for(const cbfs_tune_t* tune, int C) {
    int P = (tune && tune->slots > 0) ? tune->slots : 4;
    P = std::min(P, kMaxSlots);
    int p2 = 1;
    while (p2 * 2 <= P) p2 *= 2;
    while (p2 > 1 && p2 / 2 >= C) p2 /= 2;
    return p2;
}

}  // namespace

namespace cbfs {

int graph_view(const cbfs_graph_s* g, GraphView* out) {
    if (!g || !out) return CBFS_E_INVALID;
    out->n = g->n;
    out->off = g->off_r;
    out->adj = g->adj_r;
    out->iperm = g->iperm_d;
    out->device = g->device;
    return CBFS_OK;
}

int* graph_status(cbfs_graph_s* g) { return g->status; }

// (status words registered per stream by stream-ordered calls)
struct PendingStatus {
    cudaStream_t stream;
    int* word;
    const void* owner;
};
static std::mutex g_pending_mu;
static std::vector<PendingStatus> g_pending;

void status_register(cudaStream_t st, int* word, const void* owner) {
    std::lock_guard<std::mutex> lock(g_pending_mu);
    for (const auto& p : g_pending)
        if (p.stream == st && p.word == word) return;
    g_pending.push_back({st, word, owner});
}

void status_forget(const void* owner) {
    std::lock_guard<std::mutex> lock(g_pending_mu);
    g_pending.erase(std::remove_if(g_pending.begin(), g_pending.end(),
                                   [owner](const PendingStatus& p) { return p.owner == owner; }),
                    g_pending.end());
}

}  // namespace cbfs

namespace {

// Destroys one cached graph once its latest launch has run.
void destroy_graph(cbfs_graph_s::GraphEntry& ge) {
    if (ge.done) {
        cudaEventSynchronize(ge.done);
        cudaEventDestroy(ge.done);
    }
    cudaGraphExecDestroy(ge.exec);
}

// Forgets every captured graph of the handle.
void drop_graphs(cbfs_graph_s* g) {
    for (auto& ge : g->graphs) destroy_graph(ge);
    g->graphs.clear();
}

// Pull classes for thresholds (small, mid): class sizes from the degree
// histogram (ranks are sorted by degree, so each class is a rank range) and
// the hub pieces (kBigDeg arcs each, in piece-major order), built once per
// mid threshold and cached.
struct ClassSet {
    int64_t c_small, c_mid, c_big;
    const uint64_t* pieces;
    int64_t npieces;
};

int class_set(cbfs_graph_s* g, int small, int mid, cudaStream_t st, ClassSet* out) {
    const auto& h = g->deg_count;
    unsigned long long total = 0, le_small = 0, le_mid = 0;
    for (int dg = 1; dg < (int)h.size(); ++dg) {
        total += h[dg];
        if (dg <= small) le_small += h[dg];
        if (dg <= mid) le_mid += h[dg];
    }
    out->c_small = (int64_t)le_small;
    out->c_mid = (int64_t)(le_mid - le_small);
    out->c_big = (int64_t)(total - le_mid);
    for (const auto& hp : g->pieces) {
        if (hp.mid != mid) continue;
        out->pieces = hp.d;
        out->npieces = hp.count;
        return CBFS_OK;
    }
    const int64_t c_big = out->c_big;
    std::vector<int64_t> hub_off((size_t)c_big + 1, 0);
    if (c_big > 0) {
        CK(cudaMemcpyAsync(hub_off.data(), g->off_r, sizeof(int64_t) * hub_off.size(), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    std::vector<uint64_t> pcs;
    for (int64_t k = 0;; ++k) {
        bool any = false;
        for (int64_t r = 0; r < c_big; ++r) {
            if (k * kBigDeg >= hub_off[(size_t)r + 1] - hub_off[(size_t)r]) break;  // degrees do not increase
            pcs.push_back(((uint64_t)r << 32) | (uint64_t)k);
            any = true;
        }
        if (!any) break;
    }
    cbfs_graph_s::HubPieces hp{mid, nullptr, (int64_t)pcs.size()};
    int rc = dev_alloc(&hp.d, hp.count);
    if (rc) return rc;
    if (!pcs.empty()) {
        CK(cudaMemcpyAsync(hp.d, pcs.data(), sizeof(uint64_t) * pcs.size(), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));  // pcs dies with this scope
    }
    if (g->pieces.size() >= 8) {  // keep the create-time list, drop the oldest other one
        for (size_t i = 0; i < g->pieces.size(); ++i) {
            if (g->pieces[i].d == g->pull_pieces) continue;
            drop_graphs(g);  // captured graphs may hold its address
            dev_free(g->pieces[i].d);
            g->pieces.erase(g->pieces.begin() + (long)i);
            break;
        }
    }
    g->pieces.push_back(hp);
    out->pieces = hp.d;
    out->npieces = hp.count;
    return CBFS_OK;
}

// True when p is host memory (pinned or pageable): kernels do not write it.
bool is_host_pointer(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged;
}

int run_clusters_inner(cbfs_graph_s* g, const int32_t* src, const int32_t* coff, int C, int d, uint8_t* dist,
                       uint64_t* masks, cbfs_labels_s* L, int lbase, const cbfs_tune_t* tune, cudaStream_t st);

// Outputs go to dist/masks (device or host memory, either may be null when
// L is given) and, when L is not null, are appended to the label store.
int run_clusters(cbfs_graph_s* g, const int32_t* src, const int32_t* coff, int C, int d, uint8_t* dist,
                 uint64_t* masks, cbfs_labels_s* L, const cbfs_tune_t* tune, cudaStream_t st) {
    int rc = check_clusters(g, src, coff, C, d);
    if (rc) return rc;
    if (C == 0) return CBFS_OK;
    CK(cudaSetDevice(g->device));
    int lbase = 0;
    if (L) {
        rc = labels_reserve(L, g->n, d, coff, C, &lbase, st);
        if (rc) return rc;
    }
    rc = run_clusters_inner(g, src, coff, C, d, dist, masks, L, lbase, tune, st);
    if (rc && L) labels_rollback(L, lbase);
    return rc;
}

int run_clusters_inner(cbfs_graph_s* g, const int32_t* src, const int32_t* coff, int C, int d, uint8_t* dist,
                       uint64_t* masks, cbfs_labels_s* L, int lbase, const cbfs_tune_t* tune, cudaStream_t st) {
    int rc = CBFS_OK;
    const int P = slots_for(tune, C);
    // Default switch factor, per wave: a wave of small clusters (at most 4
    // sources each) pulls early -- its pull stops after a few frontier
    // neighbours -- while larger clusters must collect every source bit
    // (measured: 0.02 vs 0.08 is 1.5x faster for k = 2..4, equal from k = 8).
    const bool alpha_given = tune && tune->pull_alpha != 0.f;
    const float alpha = alpha_given ? tune->pull_alpha : 0.08f;
    // order[pos]: one cluster per word, the cluster in wave pos / P, slot pos % P;
    // packed, the order in which clusters go into words (set below)
    std::vector<int> order((size_t)C);
    for (int c = 0; c < C; ++c) order[c] = c;
    // packed waves: the bits used in each slot word (set below); a word's
    // pull stops once all of its bits are in, as one cluster of that size
    std::vector<int> word_bits;
    auto wave_alpha = [&](int wv) -> float {
        if (alpha_given) return alpha;
        int max_k = 0;
        if (!word_bits.empty()) {
            for (int pos = wv * P; pos < std::min((int)word_bits.size(), (wv + 1) * P); ++pos)
                max_k = std::max(max_k, word_bits[pos]);
        } else {
            for (int pos = wv * P; pos < std::min(C, (wv + 1) * P); ++pos) {
                const int c = order[pos];
                max_k = std::max(max_k, coff[c + 1] - coff[c]);
            }
        }
        return max_k <= 4 ? 0.02f : 0.08f;
    };
    int dense_div = 16;
    if (tune && tune->dense_div != 0) dense_div = tune->dense_div < 0 ? 0 : tune->dense_div;
    int small_deg = (tune && tune->small_deg) ? tune->small_deg : (int)kPullSmall;
    // degrees up to kPullSmall are ordered by power-of-two bucket (cbfs_relabel.cu):
    // the thread class ends at a bucket boundary to stay a rank range
    if (small_deg >= 1 && small_deg <= (int)kPullSmall)
        while (small_deg & (small_deg - 1)) small_deg &= small_deg - 1;
    const int mid_deg = (tune && tune->mid_deg) ? tune->mid_deg : kDefaultMidDeg;
    // other classes for sparse pull rounds: off unless asked for (measured no faster warm)
    const int sparse_mid = (tune && tune->sparse_mid_deg) ? tune->sparse_mid_deg : -1;
    if (small_deg < 1 || small_deg > (int)kPullSmall || mid_deg < small_deg || mid_deg > kMaxMidDeg)
        return CBFS_E_INVALID;
    if (sparse_mid > 0 && (sparse_mid < small_deg || sparse_mid > kMaxMidDeg)) return CBFS_E_INVALID;
    ClassSet cls, cls_s;
    rc = class_set(g, small_deg, mid_deg, st, &cls);
    if (!rc && sparse_mid > 0 && sparse_mid != mid_deg) rc = class_set(g, small_deg, sparse_mid, st, &cls_s);
    else cls_s.c_big = -1;
    if (rc) return rc;
    rc = ensure_scratch(g, P);
    if (!rc) rc = ensure_dev(&g->masks_r, &g->masks_r_cap, std::max<int64_t>(1, g->n * d * P));
    if (rc) return rc;
    const int pi = P == 1 ? 0 : P == 2 ? 1 : P == 4 ? 2 : 3;
    const int grid = g->grid_p[pi];
    int nwaves = (C + P - 1) / P;  // slot words / P once packing has been decided
    const int64_t total_src = coff[C];
    const int64_t n = g->n;
    // Where each wave's outputs go.  Device outputs: straight into dist/masks.
    // Host outputs (or labels without outputs): a ring of G wave buffers,
    // [dist G x P x n | masks G x P x d x n] so consecutive slots form one
    // cluster-major array; each wave is copied out on copy_stream while later
    // waves traverse.  Labels are written per group of waves (about
    // kLabelGroup clusters) from wherever the outputs are: the row store is
    // vertex-major, and a wider group writes longer runs of each row.
    constexpr int kLabelGroup = 32;
    constexpr int64_t kStageBudget = (int64_t)3 << 30;
    const bool host_out = (dist && is_host_pointer(dist)) || (masks && is_host_pointer(masks));
    const bool staged = host_out || (L && !dist);
    const int64_t wave_dist = (int64_t)P * n;       // bytes
    const int64_t wave_masks = (int64_t)P * d * n;  // words
    // Host copies go out per group of CG waves (about 16 clusters: each D2H
    // call has a fixed cost that grows with the state of the host's pinned
    // memory), double-buffered in the ring so the next group traverses
    // while the previous one is copied.
    int G = 2, CG = 1;
    if (staged) {
        const int want_cg = host_out ? std::max(1, 16 / P) : 1;
        if (L) G = std::max(2, kLabelGroup / P);
        G = std::max(G, 2 * want_cg);
        const int64_t fit = kStageBudget / std::max<int64_t>(1, wave_dist + 8 * wave_masks);
        G = (int)std::max<int64_t>(2, std::min<int64_t>(G, fit));
        CG = std::max(1, std::min(want_cg, G / 2));
        while (G % CG) CG--;
    }
    const int LG = L ? (staged ? G : std::max(1, kLabelGroup / P)) : 0;  // waves per label write
    // Wave composition.  With device outputs and no label store every slot
    // writes through its own output pointers, so clusters may be traversed in
    // any grouping: clusters of similar size share a wave (sizes descending,
    // ties in call order).  A wave of small clusters then pulls early and its
    // pulls stop early, instead of running as long as one large cluster in
    // its midst.  Staged outputs and label rows are written per wave in call
    // order, so those calls keep it.
    if (!staged && !L && !(tune && tune->wave_order == 1))
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return coff[a + 1] - coff[a] > coff[b + 1] - coff[b]; });
    // Packed waves.  With device outputs and round records, clusters whose
    // sources fill only part of a 64-bit slot word share words: every bit of a
    // word is an independent BFS, so the traversal is that of the words, and
    // each cluster's outputs are its range of bits in the round records
    // (k_flush_packed).  Clusters go to words by best fit, largest first (the
    // fullest word with room, a new word otherwise), at most kWordMembers to a
    // word; the words fill the waves in that order.  Used when it saves words.
    const bool fused = tune && tune->fused_pull > 0;
    const bool want_pack = !staged && !L && C > 1 && !(tune && (tune->wave_order == 1 || tune->pack < 0));
    std::vector<int> word_first;             // packed: word i holds wmem[word_first[i] .. word_first[i + 1])
    std::vector<std::pair<int, int>> wmem;   // (cluster, bit offset)
    if (want_pack) {
        std::vector<std::vector<std::pair<int, int>>> words;
        std::vector<int> used;
        std::vector<std::vector<int>> by_free(65);  // words by free bits (stale entries skipped)
        for (int pos = 0; pos < C; ++pos) {
            const int c = order[pos];
            const int k = coff[c + 1] - coff[c];
            int ws = -1;
            for (int f = k; f <= 64 && ws < 0; ++f) {
                auto& lst = by_free[f];
                while (!lst.empty() && ws < 0) {
                    const int wi = lst.back();
                    lst.pop_back();
                    if (64 - used[wi] == f && (int)words[wi].size() < kWordMembers) ws = wi;
                }
            }
            if (ws < 0) {
                ws = (int)words.size();
                words.emplace_back();
                used.push_back(0);
            }
            words[ws].push_back({c, used[ws]});
            used[ws] += k;
            if (used[ws] < 64 && (int)words[ws].size() < kWordMembers) by_free[64 - used[ws]].push_back(ws);
        }
        if ((int)words.size() < C) {
            word_first.push_back(0);
            for (size_t wi = 0; wi < words.size(); ++wi) {
                for (const auto& m : words[wi]) wmem.push_back(m);
                word_first.push_back((int)wmem.size());
                word_bits.push_back(used[wi]);
            }
            nwaves = ((int)words.size() + P - 1) / P;
        }
    }
    // round records: fused waves and packed waves write their outputs from them
    int hcap = 0;
    if (fused || !word_first.empty()) {
        rc = stage_rounds(g, tune, P, &hcap);
        if (rc) return rc;
        if (hcap == 0 && !word_first.empty()) {  // no room for records: one cluster per word
            word_first.clear();
            wmem.clear();
            word_bits.clear();
            nwaves = (C + P - 1) / P;
        }
    }
    const bool packed = !word_first.empty();
    const int NW = packed ? (int)word_bits.size() : C;  // slot words of the call
    const int64_t stage_dist_bytes = (G * wave_dist + 255) / 256 * 256;
    if (staged) {
        rc = ensure_dev(&g->stage, &g->stage_cap, stage_dist_bytes + 8 * G * wave_masks);
        if (rc) return rc;
        if (!g->copy_stream) CK(cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking));
        while ((int)g->ev_emit.size() < G) {
            cudaEvent_t a = nullptr, b = nullptr;
            CK(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
            g->ev_emit.push_back(a);
            CK(cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
            g->ev_copy.push_back(b);
        }
    }
    uint64_t* stage_masks = staged ? reinterpret_cast<uint64_t*>(g->stage + stage_dist_bytes) : nullptr;
    auto wave_dist_at = [&](int wv) -> uint8_t* {
        return staged ? g->stage + (size_t)(wv % G) * (size_t)wave_dist : dist + (size_t)wv * (size_t)wave_dist;
    };
    auto wave_masks_at = [&](int wv) -> uint64_t* {
        if (!d) return nullptr;
        return staged ? stage_masks + (size_t)(wv % G) * (size_t)wave_masks : masks + (size_t)wv * (size_t)wave_masks;
    };
    // Captured graphs hold these device pointers: when one of them moves, every
    // cached graph goes (a replay would read the freed buffer).
    const void* held[4] = {g->slots, g->seeds, g->members, g->bitm};
    cbfs_graph_s::Upload& up = g->up[g->calls % cbfs_graph_s::kUploadRing];
    if (up.done) CK(cudaEventSynchronize(up.done));  // this entry's previous upload has been read
    rc = ensure_dev(&g->slots, &g->slots_cap, (int64_t)nwaves * P);
    if (!rc) rc = ensure_pinned(&up.slots, &up.slots_cap, (int64_t)nwaves * P);
    if (!rc) rc = ensure_dev(&g->seeds, &g->seeds_cap, total_src);
    if (!rc) rc = ensure_pinned(&up.seeds, &up.seeds_cap, total_src);
    if (!rc && packed) rc = ensure_dev(&g->members, &g->members_cap, C);
    if (!rc && packed) rc = ensure_pinned(&up.members, &up.members_cap, C);
    if (!rc && packed) rc = ensure_dev(&g->bitm, &g->bitm_cap, (int64_t)nwaves * P * 64);
    if (!rc && packed) rc = ensure_pinned(&up.bitm, &up.bitm_cap, (int64_t)nwaves * P * 64);
    if (held[0] != (const void*)g->slots || held[1] != (const void*)g->seeds || held[2] != (const void*)g->members ||
        held[3] != (const void*)g->bitm)
        drop_graphs(g);
    if (rc) return rc;
    if (!up.done) CK(cudaEventCreateWithFlags(&up.done, cudaEventDisableTiming));
    g->calls += 1;
    // slot tables and seeds of every wave, staged once
    std::vector<int64_t> wave_seed_off(nwaves + 1, 0);
    int64_t ns = 0;
    // packed: each word's members (its first member's wave-local index in
    // SlotDesc.cluster, their count in .pad), the bit table, and the seeds with
    // their member index
    for (int wv = 0; packed && wv < nwaves; ++wv) {
        wave_seed_off[wv] = ns;
        const int m0 = word_first[(size_t)wv * P];
        uint8_t* bt = up.bitm + (size_t)wv * P * 64;
        memset(bt, 0xFF, (size_t)P * 64);
        for (int s = 0; s < P; ++s) {
            const int pos = wv * P + s;
            SlotDesc sd;
            memset(&sd, 0, sizeof(sd));
            if (pos < NW) {
                sd.cluster = word_first[pos] - m0;
                sd.pad = word_first[pos + 1] - word_first[pos];
                for (int mi = word_first[pos]; mi < word_first[pos + 1]; ++mi) {
                    const int c = wmem[mi].first, off = wmem[mi].second;
                    const int k = coff[c + 1] - coff[c];
                    MemberDesc md;
                    memset(&md, 0, sizeof(md));
                    md.dist = dist + (size_t)c * (size_t)n;
                    md.masks = d ? masks + (size_t)c * (size_t)d * (size_t)n : nullptr;
                    md.mask = ((k >= 64) ? ~0ull : ((1ull << k) - 1ull)) << off;
                    md.off = off;
                    md.word = s;
                    up.members[mi] = md;
                    sd.all |= md.mask;
                    for (int b = off; b < off + k; ++b) bt[s * 64 + b] = (uint8_t)(mi - m0);
                    for (int j = 0; j < k; ++j)
                        up.seeds[ns++] = ((uint64_t)(mi - m0) << 48) | ((uint64_t)s << 40) | ((uint64_t)(off + j) << 32) |
                                         (uint32_t)src[coff[c] + j];
                }
            }
            up.slots[(size_t)wv * P + s] = sd;
        }
    }
    for (int wv = 0; !packed && wv < nwaves; ++wv) {
        wave_seed_off[wv] = ns;
        for (int s = 0; s < P; ++s) {
            const int pos = wv * P + s;
            SlotDesc sd;
            memset(&sd, 0, sizeof(sd));
            if (pos < C) {
                const int c = order[pos];  // == pos when staged or with labels
                const int k = coff[c + 1] - coff[c];
                if (staged) {
                    sd.dist = wave_dist_at(wv) + (size_t)s * (size_t)n;
                    sd.masks = d ? wave_masks_at(wv) + (size_t)s * (size_t)d * (size_t)n : nullptr;
                } else {
                    sd.dist = dist + (size_t)c * (size_t)n;
                    sd.masks = d ? masks + (size_t)c * (size_t)d * (size_t)n : nullptr;
                }
                sd.all = (k >= 64) ? ~0ull : ((1ull << k) - 1ull);
                sd.cluster = c;
                for (int j = 0; j < k; ++j)
                    up.seeds[ns++] = ((uint64_t)s << 40) | ((uint64_t)j << 32) | (uint32_t)src[coff[c] + j];  // mapped to ranks on the device
            }
            up.slots[(size_t)wv * P + s] = sd;
        }
    }
    wave_seed_off[nwaves] = ns;
    CK(cudaMemcpyAsync(g->slots, up.slots, sizeof(SlotDesc) * (size_t)nwaves * P, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(g->seeds, up.seeds, sizeof(uint64_t) * (size_t)std::max<int64_t>(ns, 1),
                       cudaMemcpyHostToDevice, st));
    if (packed) {
        CK(cudaMemcpyAsync(g->members, up.members, sizeof(MemberDesc) * (size_t)C, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(g->bitm, up.bitm, (size_t)nwaves * P * 64, cudaMemcpyHostToDevice, st));
    }
    CK(cudaEventRecord(up.done, st));
    CK(map_seeds(g->seeds, ns, g->iperm_d, st));
    // The status word is sticky: it is not cleared here, so an error of an
    // earlier stream-ordered call stays until cbfs_sync_status or the next
    // blocking call reads (and clears) it.

    Wave w;
    memset(&w, 0, sizeof(w));
    w.n = n;
    w.nnz = g->nnz;
    w.off = g->off_r;
    w.adj = g->adj_r;
    w.perm = g->perm;
    w.d = d;
    w.P = P;
    w.vis = g->vis;
    w.acc = g->acc;
    w.nw0 = g->nw;
    w.nw1 = g->nw + (size_t)P * (size_t)n;
    w.piece_cnt = g->piece_cnt;
    w.rq = g->rq;
    w.q0 = g->q0;
    w.q1 = g->q1;
    const int64_t bm_words = scratch_sizes(n, P).bitmap;
    w.fb0 = g->fb;
    w.fb1 = g->fb + bm_words;
    w.ctl = g->ctl;
    w.t_pre = g->t_pre;
    w.t_ost = g->t_ost;
    w.t_fw = g->t_fw;
    w.tile_cnt = g->tile_cnt;
    w.tile_arcs = g->tile_arcs;
    w.big = g->big;
    w.big_fw = g->big_fw;
    w.piece_ent = g->piece_ent;
    w.piece_no = g->piece_no;
    w.n_small = cls.c_small;
    w.n_mid = cls.c_mid;
    w.n_big = cls.c_big;
    w.pull_pieces = cls.pieces;
    w.n_pull_pieces = cls.npieces;
    w.n_big_s = cls_s.c_big;  // < 0: every pull round uses the classes above
    if (cls_s.c_big >= 0) {
        w.n_small_s = cls_s.c_small;
        w.n_mid_s = cls_s.c_mid;
        w.pull_pieces_s = cls_s.pieces;
        w.n_pull_pieces_s = cls_s.npieces;
    }
    w.status = g->status;
    w.alpha = alpha;
    w.dist_r = g->dist_r;
    w.wmask_r = g->wmask_r;
    w.masks_r = g->masks_r;
    w.dense_div = dense_div;
    w.grid_a = g->grid_a[pi];
    w.fused_pull = fused ? 1 : 0;
    if (fused || packed) {
        // no internal rows: the vertex phase (in the pull or in phase A) records each
        // round's new sources (round records, then k_flush / k_flush_packed) or, past
        // the records or without them, writes the outputs directly (cleared per wave
        // by k_clear_outputs when there are no records); no emit
        w.dist_r = nullptr;
        w.masks_r = nullptr;
        w.wmask_r = nullptr;
        w.hcap = hcap;
        w.hist = g->hist;
        w.fbh = g->fbh;
    }
    // packed: the wave's members and bit table (per wave, set below)
    auto set_members = [&](Wave& x, int wv) {
        if (!packed) return;
        const int m0 = word_first[(size_t)wv * P];
        const int m1 = word_first[(size_t)std::min(NW, (wv + 1) * P)];
        x.members = g->members + m0;
        x.nmembers = m1 - m0;
        x.bit_member = g->bitm + (size_t)wv * P * 64;
    };

    // Graph mode (device outputs): the call runs as one cached CUDA graph per
    // call shape whose rounds loop on the device, and is stream-ordered: the
    // graph is launched on `st` and the call returns.  Device-detected errors
    // stay in the status word for cbfs_sync_status(st) or the next blocking call.
    if (!g->timing && !(tune && tune->host_loop) && !staged && !L) {
        if (!g->round_dev) {
            rc = dev_alloc(&g->round_dev, 1);
            if (!rc) rc = dev_alloc(&g->iters, 1);
            if (rc) return rc;
            CK(cudaMemsetAsync(g->iters, 0, sizeof(unsigned long long), st));  // rounds run, read by cbfs_profile
        }
        Wave wg = w;
        wg.round_dev = g->round_dev;
        wg.iters = g->iters;
        std::vector<Wave> waves((size_t)nwaves, wg);
        uint64_t key = 1469598103934665603ull;
        for (int wv = 0; wv < nwaves; ++wv) {
            waves[wv].nslots = std::min(P, NW - wv * P);
            waves[wv].alpha = wave_alpha(wv);
            waves[wv].slots = g->slots + (size_t)wv * P;
            set_members(waves[wv], wv);
            key = fnv1a(key, &waves[wv], sizeof(Wave));
        }
        key = fnv1a(key, wave_seed_off.data(), sizeof(int64_t) * wave_seed_off.size());
        key = fnv1a(key, &grid, sizeof(grid));
        key = fnv1a(key, &g->seeds, sizeof(g->seeds));  // baked into k_seed / k_check_sources
        cbfs_graph_s::GraphEntry* ge = nullptr;
        for (size_t i = 0; i < g->graphs.size(); ++i) {
            if (g->graphs[i].key == key) {
                const auto hit = g->graphs[i];
                g->graphs.erase(g->graphs.begin() + (long)i);
                g->graphs.push_back(hit);
                ge = &g->graphs.back();
                break;
            }
        }
        if (!ge) {
            cudaGraphExec_t exec = nullptr;
            rc = build_graph(g, waves, wave_seed_off, grid, bm_words, &exec);
            if (rc) return rc;
            cudaEvent_t done = nullptr;
            if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                cudaGraphExecDestroy(exec);
                return CBFS_E_CUDA;
            }
            if (g->graphs.size() >= 8) {
                destroy_graph(g->graphs.front());
                g->graphs.erase(g->graphs.begin());
            }
            g->graphs.push_back({key, exec, done});
            ge = &g->graphs.back();
        }
        CK(cudaGraphLaunch(ge->exec, st));
        CK(cudaEventRecord(ge->done, st));
        status_register(st, g->status, g);
        // per wave: seed, emit, check; the rounds' three launches are counted
        // on the device and added by cbfs_profile
        g->launches[0] += 3ull * (uint64_t)nwaves;
        g->total_launches += 3ull * (uint64_t)nwaves;
        return CBFS_OK;
    }

    // Host-driven rounds.  A "careful" wave synchronises every two rounds to
    // see its frontier; it tells how many rounds waves of this call take.  The
    // following waves enqueue that many rounds plus a margin without waiting
    // (rounds past the end return at once) and flag themselves when their
    // frontier was still not empty; flagged waves are run carefully again.
    rc = ensure_dev(&g->wave_flags, &g->wave_flags_cap, nwaves);
    if (rc) return rc;
    CK(cudaMemsetAsync(g->wave_flags, 0, sizeof(int) * (size_t)nwaves, st));
    auto run_wave = [&](int wv, int bound, bool rerun, int* rounds_out) -> int {
        const int c0 = wv * P;
        w.nslots = std::min(P, NW - c0);
        w.alpha = wave_alpha(wv);
        w.slots = g->slots + (size_t)wv * P;
        set_members(w, wv);
        CK(cudaMemsetAsync(g->vis, 0, sizeof(uint64_t) * (size_t)P * (size_t)n, st));
        CK(cudaMemsetAsync(g->acc, 0, sizeof(uint64_t) * (size_t)P * (size_t)n, st));
        if (w.fused_pull && !w.hcap)  // a fused pull round may read any vertex's entry
            CK(cudaMemsetAsync(g->nw, 0, sizeof(uint64_t) * 2 * (size_t)P * (size_t)n, st));
        CK(cudaMemsetAsync(g->rq, 0, sizeof(uint32_t) * (size_t)n, st));
        CK(cudaMemsetAsync(g->fb, 0, sizeof(uint32_t) * 2 * (size_t)bm_words, st));
        if (w.dist_r) CK(cudaMemsetAsync(g->dist_r, 0xFF, (size_t)P * (size_t)n, st));
        CK(cudaMemsetAsync(g->ctl, 0, sizeof(RoundCtl) * kMaxRounds, st));
        const int cnt = (int)(wave_seed_off[wv + 1] - wave_seed_off[wv]);
        // direct outputs are written from the wave's start: its ring slot must have
        // been copied out first (wave wv - G)
        if (!w.dist_r && host_out) CK(cudaStreamWaitEvent(st, g->ev_copy[wv % G], 0));
        int ev = prof_begin(g, 0, st);
        if (!w.dist_r && !w.hcap) k_clear_outputs<<<grid, kThreads, 0, st>>>(w);
        k_seed<<<1, kThreads, 0, st>>>(w, g->seeds + wave_seed_off[wv], cnt);
        prof_end(g, ev, st);
        CK(cudaGetLastError());
        int rounds = 0;
        if (bound > 0) {
            for (int r = 0; r < bound; ++r) {
                ev = prof_begin(g, 1, st);
                CK(launch_round(w, r, grid, st, 0));
                prof_end(g, ev, st);
                if (r == w.hcap - 1) {
                    ev = prof_begin(g, 0, st);
                    CK(launch_flush(w, r, grid, st, 1, 0, g->iperm_d));
                    prof_end(g, ev, st);
                }
                ev = prof_begin(g, 2, st);
                CK(launch_round(w, r, grid, st, 1));
                prof_end(g, ev, st);
            }
            rounds = bound;
        } else {
            bool done = false;
            for (int r = 0; r < kMaxRounds - 1 && !done; ++r) {
                ev = prof_begin(g, 1, st);
                CK(launch_round(w, r, grid, st, 0));
                prof_end(g, ev, st);
                if (r == w.hcap - 1) {
                    ev = prof_begin(g, 0, st);
                    CK(launch_flush(w, r, grid, st, 1, 0, g->iperm_d));
                    prof_end(g, ev, st);
                }
                ev = prof_begin(g, 2, st);
                CK(launch_round(w, r, grid, st, 1));
                prof_end(g, ev, st);
                CK(cudaMemcpyAsync(&g->h_q[r + 1], &g->ctl[r + 1].qlen, sizeof(unsigned long long),
                                   cudaMemcpyDeviceToHost, st));
                if (r % 2 == 1 || r == kMaxRounds - 2) {
                    CK(cudaStreamSynchronize(st));
                    if (g->h_q[r] == 0 || g->h_q[r + 1] == 0) done = true;
                }
                rounds = r + 1;
            }
            if (!done) {
                // the call fails here: it returns (and clears) the status word like any
                // blocking call, so the next call does not report the same error again
                int status = 0;
                CK(cudaMemcpyAsync(&status, g->status, sizeof(int), cudaMemcpyDeviceToHost, st));
                CK(cudaMemsetAsync(g->status, 0, sizeof(int), st));
                CK(cudaStreamSynchronize(st));
                prof_collect(g);
                return status ? status : CBFS_E_DEPTH;
            }
        }
        const int b = wv % G;
        if (host_out && w.dist_r) CK(cudaStreamWaitEvent(st, g->ev_copy[b], 0));  // ring slot b copied out (wave wv - G)
        if (w.dist_r) {
            ev = prof_begin(g, 0, st);
            CK(launch_round(w, 0, grid, st, 2, g->iperm_d));
            prof_end(g, ev, st);
        } else if (w.hcap > 0) {
            ev = prof_begin(g, 0, st);
            CK(launch_flush(w, 0, grid, st, 0, bound, g->iperm_d));
            prof_end(g, ev, st);
        }
        if (host_out && (rerun || (wv + 1) % CG == 0 || wv == nwaves - 1)) {
            // the group's waves sit in consecutive ring slots (G is a multiple of CG)
            const int g0 = rerun ? wv : wv / CG * CG;
            const int64_t nc = (int64_t)std::min(C, (wv + 1) * P) - (int64_t)g0 * P;
            CK(cudaEventRecord(g->ev_emit[b], st));
            CK(cudaStreamWaitEvent(g->copy_stream, g->ev_emit[b], 0));
            if (dist)
                CK(cudaMemcpyAsync(dist + (size_t)g0 * P * (size_t)n, wave_dist_at(g0), (size_t)nc * (size_t)n,
                                   cudaMemcpyDefault, g->copy_stream));
            if (masks && d)
                CK(cudaMemcpyAsync(masks + (size_t)g0 * P * (size_t)d * (size_t)n, wave_masks_at(g0),
                                   sizeof(uint64_t) * (size_t)nc * (size_t)d * (size_t)n, cudaMemcpyDefault,
                                   g->copy_stream));
            for (int x = g0; x <= wv; ++x) CK(cudaEventRecord(g->ev_copy[x % G], g->copy_stream));
        }
        if (L) {
            if (rerun) {
                CK(labels_write(L, wave_dist_at(wv), wave_masks_at(wv), w.nslots, lbase + c0, st));
            } else if ((wv + 1) % LG == 0 || wv == nwaves - 1) {
                const int g0 = wv / LG * LG;  // first wave of the group (ring slot 0 when staged)
                const int nc = std::min(C, (wv + 1) * P) - g0 * P;
                CK(labels_write(L, wave_dist_at(g0), wave_masks_at(g0), nc, lbase + g0 * P, st));
            }
        }
        ev = prof_begin(g, 0, st);
        k_check_sources<<<1, kThreads, 0, st>>>(w, g->seeds + wave_seed_off[wv], cnt, bound, g->wave_flags + wv);
        prof_end(g, ev, st);
        CK(cudaGetLastError());
        *rounds_out = rounds;
        return CBFS_OK;
    };
    int est = 0;
    bool any_optimistic = false;
    for (int wv = 0; wv < nwaves; ++wv) {
        const int bound = est > 0 ? std::min(est + 2, kMaxRounds - 1) : 0;
        int used = 0;
        rc = run_wave(wv, bound, false, &used);
        if (rc) return rc;
        if (bound == 0) est = used;
        else any_optimistic = true;
    }
    if (any_optimistic) {
        std::vector<int> flags((size_t)nwaves, 0);
        CK(cudaMemcpyAsync(flags.data(), g->wave_flags, sizeof(int) * (size_t)nwaves, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int wv = 0; wv < nwaves; ++wv) {
            if (!flags[wv]) continue;
            int used = 0;
            rc = run_wave(wv, 0, true, &used);
            if (rc) return rc;
        }
    }
    if (host_out)
        for (int b = 0; b < G; ++b) CK(cudaStreamWaitEvent(st, g->ev_copy[b], 0));
    // a blocking call returns (and clears) the status word, including an error
    // left by an earlier stream-ordered call that nobody has read yet
    int status = 0;
    CK(cudaMemcpyAsync(&status, g->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemsetAsync(g->status, 0, sizeof(int), st));
    CK(cudaStreamSynchronize(st));
    prof_collect(g);
    return status;
}

}  // namespace

extern "C" {

const char* cbfs_status_string(int status) {
    switch (status) {
        case CBFS_OK: return "CBFS_OK";
        case CBFS_E_INVALID: return "CBFS_E_INVALID: invalid argument";
        case CBFS_E_DIAMETER: return "CBFS_E_DIAMETER: cluster diameter exceeds d";
        case CBFS_E_DEPTH: return "CBFS_E_DEPTH: a distance does not fit one byte (>= 255)";
        case CBFS_E_NOMEM: return "CBFS_E_NOMEM: out of memory or over budget";
        case CBFS_E_TIMEOUT: return "CBFS_E_TIMEOUT: bounded device wait expired";
        case CBFS_E_CUDA: return "CBFS_E_CUDA: CUDA runtime error";
        case CBFS_E_GRAPH: return "CBFS_E_GRAPH: graph validation failed";
        default: return "CBFS: unknown status";
    }
}

int cbfs_graph_create(int64_t n, const void* off, int off_is_i64, const int32_t* adj, int64_t nnz,
                      int inputs_on_device, int validate, void* stream, cbfs_graph_t* out) {
    if (!out) return CBFS_E_INVALID;
    *out = nullptr;
    if (n < 0 || n >= (int64_t)0x7fffffff || nnz < 0 || nnz >= ((int64_t)1 << 40)) return CBFS_E_INVALID;
    if (!off || (nnz > 0 && !adj)) return CBFS_E_INVALID;
    if (!off_is_i64 && nnz > 0x7fffffffLL) return CBFS_E_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    cbfs_graph_s* g = new (std::nothrow) cbfs_graph_s();
    if (!g) return CBFS_E_NOMEM;
    int64_t* scratch = nullptr;
    int32_t* off32 = nullptr;
    DegreeStats* d_stats = nullptr;
    auto fail = [&](int code) {
        cudaStreamSynchronize(st);
        dev_free(scratch);
        dev_free(off32);
        dev_free(d_stats);
        cbfs_graph_destroy(g);
        return code;
    };
    cudaGetDevice(&g->device);
    g->n = n;
    g->nnz = nnz;
    int sms = 0, occ = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    sms = std::max(1, sms);
    int rc = dev_alloc(&g->off, n + 1);
    if (!rc) rc = dev_alloc(&g->adj, nnz);
    if (!rc) rc = dev_alloc(&g->ctl, kMaxRounds);
    if (!rc) rc = dev_alloc(&g->status, 1);
    if (!rc) rc = dev_alloc(&d_stats, 1);
    if (!rc) rc = dev_alloc(&scratch, std::max<int64_t>(rank_scratch_words(n), kMaxMidDeg + 2));
    if (!rc) rc = dev_alloc(&g->perm, n);
    if (!rc) rc = dev_alloc(&g->iperm_d, n);
    if (!rc) rc = dev_alloc(&g->off_r, n + 1);
    if (!rc) rc = dev_alloc(&g->adj_r, nnz);
    if (rc) return fail(rc);
    // the status word is sticky across calls: it starts at CBFS_OK and only a read clears it
    if (cudaMemsetAsync(g->status, 0, sizeof(int), st) != cudaSuccess) return fail(CBFS_E_CUDA);
    if (cudaMallocHost((void**)&g->h_q, sizeof(unsigned long long) * (kMaxRounds + 2)) != cudaSuccess) {
        g->h_q = nullptr;
        return fail(CBFS_E_NOMEM);
    }
    // the caller's CSR, offsets widened to int64 on the device
    cudaError_t e = cudaSuccess;
    const cudaMemcpyKind kind = inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (off_is_i64) {
        e = cudaMemcpyAsync(g->off, off, sizeof(int64_t) * (size_t)(n + 1), kind, st);
    } else if (inputs_on_device) {
        e = widen_offsets((const int32_t*)off, g->off, n + 1, sms, st);
    } else {
        if (dev_alloc(&off32, n + 1)) return fail(CBFS_E_NOMEM);
        e = cudaMemcpyAsync(off32, off, sizeof(int32_t) * (size_t)(n + 1), kind, st);
        if (e == cudaSuccess) e = widen_offsets(off32, g->off, n + 1, sms, st);
    }
    if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(g->adj, adj, sizeof(int32_t) * (size_t)nnz, kind, st);
    // offsets check, degree classes, sort keys
    if (e == cudaSuccess) e = degree_stats(n, nnz, g->off, d_stats, rank_keys(n, scratch), sms, st);
    DegreeStats hs;
    memset(&hs, 0, sizeof(hs));
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, d_stats, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(CBFS_E_CUDA);
    if (hs.bad) return fail(CBFS_E_GRAPH);
    dev_free(off32);
    g->n_small = (int64_t)hs.n_small;
    g->n_mid = (int64_t)hs.n_mid;
    g->n_big = (int64_t)hs.n_big;
    g->big_pieces = (int64_t)hs.big_pieces;
    const void* kb[4] = {(const void*)k_phase_b<1, false>, (const void*)k_phase_b<2, false>,
                         (const void*)k_phase_b<4, false>, (const void*)k_phase_b<8, false>};
    const void* ka[4] = {(const void*)k_phase_a<1>, (const void*)k_phase_a<2>, (const void*)k_phase_a<4>,
                         (const void*)k_phase_a<8>};
    for (int i = 0; i < 4; ++i) {
        // the default carveout: a larger shared-memory share would shrink the L1 these
        // gather-bound kernels depend on (measured slower)
        occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb[i], kThreads, 0);
        g->grid_p[i] = sms * std::max(1, std::min(occ, 8));
        occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ka[i], kThreads, 0);
        g->grid_a[i] = sms * std::max(1, std::min(occ, 8));
    }
    // internal order: ranks by degree (cbfs_relabel.cu); the degree classes are rank ranges
    e = rank_order_device(n, g->off, hs.maxdeg, scratch, g->perm, g->iperm_d, g->off_r, d_stats, sms, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, d_stats, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess || hs.order_bad) return fail(CBFS_E_CUDA);
    if (validate && n > 0) {
        // every arc has its reverse, no self-loops or repeats; lists of the
        // three degree classes are balanced separately (thread, warp, CTA per list)
        e = cudaMemsetAsync(g->status, 0, sizeof(int), st);
        if (e == cudaSuccess) {
            k_validate<<<sms * 8, kThreads, 0, st>>>(n, g->off, g->adj, g->iperm_d, g->perm + g->n_big + g->n_mid,
                                                     g->n_small, g->perm + g->n_big, g->n_mid, g->perm, g->n_big,
                                                     g->status, &d_stats->forward);
            e = cudaGetLastError();
        }
        int flag = 0;
        unsigned long long forward = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, g->status, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&forward, &d_stats->forward, sizeof(forward), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(CBFS_E_CUDA);
        if (flag || 2 * (int64_t)forward != nnz) return fail(CBFS_E_GRAPH);
    }
    if (e == cudaSuccess && nnz > 0)
        e = relabel_adjacency(n, g->n_big, g->n_mid, g->n_small, g->perm, g->iperm_d, g->off, g->adj, g->off_r, g->adj_r,
                              sms, st);
    // degree histogram: class sizes of other thresholds without another pass
    g->deg_count.assign(kMaxMidDeg + 2, 0ull);
    if (e == cudaSuccess) e = degree_hist(n, g->off, reinterpret_cast<unsigned long long*>(scratch), sms, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->deg_count.data(), scratch, sizeof(unsigned long long) * g->deg_count.size(),
                            cudaMemcpyDeviceToHost, st);
    // pieces of the high-degree lists for the dense edge phase (ranks [0, n_big)),
    // piece-major (every hub's first piece before any second piece): a later
    // piece usually finds its hub already complete and skips
    std::vector<int64_t> hub_off((size_t)g->n_big + 1, 0);
    if (e == cudaSuccess && g->n_big > 0)
        e = cudaMemcpyAsync(hub_off.data(), g->off_r, sizeof(int64_t) * hub_off.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(CBFS_E_CUDA);
    std::vector<uint64_t> pcs;
    pcs.reserve((size_t)g->big_pieces);
    static_assert(kBigDeg == kPullMid, "the push big list and the CTA pull class are the same vertices");
    g->big_vertices = g->n_big;
    for (int64_t k = 0; (int64_t)pcs.size() < g->big_pieces; ++k) {
        bool any = false;
        for (int64_t r = 0; r < g->n_big; ++r) {
            const int64_t dg = hub_off[(size_t)r + 1] - hub_off[(size_t)r];
            if (k * kBigDeg >= dg) break;  // ranks are sorted by degree: the rest are shorter
            pcs.push_back(((uint64_t)r << 32) | (uint64_t)k);
            any = true;
        }
        if (!any) break;
    }
    if ((int64_t)pcs.size() != g->big_pieces) return fail(CBFS_E_CUDA);
    if (dev_alloc(&g->pull_pieces, (int64_t)pcs.size()) != CBFS_OK) return fail(CBFS_E_NOMEM);
    if (!pcs.empty())
        e = cudaMemcpyAsync(g->pull_pieces, pcs.data(), sizeof(uint64_t) * pcs.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // pcs dies with this scope
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return fail(CBFS_E_CUDA);
    g->pieces.push_back({(int)kPullMid, g->pull_pieces, g->big_pieces});
    dev_free(scratch);
    dev_free(d_stats);
    dev_free(g->adj);  // the caller's adjacency is no longer needed
    *out = g;
    return CBFS_OK;
}

int cbfs_graph_destroy(cbfs_graph_t g) {
    if (!g) return CBFS_OK;
    status_forget(g);
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    free_scratch(g);
    dev_free(g->off);
    dev_free(g->adj);
    dev_free(g->off_r);
    dev_free(g->adj_r);
    dev_free(g->perm);
    dev_free(g->iperm_d);
    for (auto& hp : g->pieces)
        if (hp.d != g->pull_pieces) dev_free(hp.d);
    dev_free(g->pull_pieces);
    dev_free(g->masks_r);
    dev_free(g->hist);
    dev_free(g->fbh);
    dev_free(g->ctl);
    dev_free(g->status);
    dev_free(g->slots);
    dev_free(g->seeds);
    dev_free(g->members);
    dev_free(g->bitm);
    for (cudaEvent_t e : g->events) cudaEventDestroy(e);
    drop_graphs(g);
    dev_free(g->stage);
    if (g->copy_stream) cudaStreamDestroy(g->copy_stream);
    for (cudaEvent_t e : g->ev_emit) cudaEventDestroy(e);
    for (cudaEvent_t e : g->ev_copy) cudaEventDestroy(e);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    if (g->cap_stream2) cudaStreamDestroy(g->cap_stream2);
    dev_free(g->round_dev);
    dev_free(g->iters);
    dev_free(g->wave_flags);
    if (g->h_q) cudaFreeHost(g->h_q);
    for (auto& u : g->up) {
        if (u.slots) cudaFreeHost(u.slots);
        if (u.seeds) cudaFreeHost(u.seeds);
        if (u.members) cudaFreeHost(u.members);
        if (u.bitm) cudaFreeHost(u.bitm);
        if (u.done) cudaEventDestroy(u.done);
    }
    delete g;
    return CBFS_OK;
}

int cbfs_graph_info(cbfs_graph_t g, int64_t* host_n, int64_t* host_nnz) {
    if (!g) return CBFS_E_INVALID;
    if (host_n) *host_n = g->n;
    if (host_nnz) *host_nnz = g->nnz;
    return CBFS_OK;
}

int cbfs_run(cbfs_graph_t g, const int32_t* host_sources, int k, int d, uint8_t* dist, uint64_t* masks,
             void* stream) {
    if (!g || !host_sources || !dist || (d > 0 && !masks)) return CBFS_E_INVALID;
    if (k < 1 || k > 64) return CBFS_E_INVALID;
    const int32_t coff[2] = {0, k};
    cbfs_tune_t t;
    memset(&t, 0, sizeof(t));
    t.slots = 1;
    return run_clusters(g, host_sources, coff, 1, d, dist, masks, nullptr, &t, (cudaStream_t)stream);
}

int cbfs_run_batched(cbfs_graph_t g, const int32_t* host_sources_concat, const int32_t* host_cluster_off, int C,
                     int d, uint8_t* dist, uint64_t* masks, const cbfs_tune_t* tune, void* stream) {
    if (!g || C < 0 || !host_cluster_off) return CBFS_E_INVALID;
    if (C == 0) return CBFS_OK;
    if (!host_sources_concat || !dist || (d > 0 && !masks)) return CBFS_E_INVALID;
    return run_clusters(g, host_sources_concat, host_cluster_off, C, d, dist, masks, nullptr, tune,
                        (cudaStream_t)stream);
}

int cbfs_run_batched_labels(cbfs_graph_t g, const int32_t* host_sources_concat, const int32_t* host_cluster_off,
                            int C, int d, uint8_t* dist, uint64_t* masks, cbfs_labels_t labels,
                            const cbfs_tune_t* tune, void* stream) {
    if (!g || C < 0 || !host_cluster_off || !labels) return CBFS_E_INVALID;
    if (C == 0) return CBFS_OK;
    if (!host_sources_concat || (!dist && masks) || (dist && d > 0 && !masks)) return CBFS_E_INVALID;
    return run_clusters(g, host_sources_concat, host_cluster_off, C, d, dist, masks, labels, tune,
                        (cudaStream_t)stream);
}

int cbfs_graph_status(cbfs_graph_t g, void* stream) {
    if (!g) return CBFS_E_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    CK(cudaMemcpyAsync(&h, g->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemsetAsync(g->status, 0, sizeof(int), st));
    CK(cudaStreamSynchronize(st));
    return h;
}

int cbfs_sync_status(void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaStreamSynchronize(st));
    std::vector<PendingStatus> mine;
    {
        std::lock_guard<std::mutex> lock(g_pending_mu);
        for (size_t i = 0; i < g_pending.size();) {
            if (g_pending[i].stream == st) {
                mine.push_back(g_pending[i]);
                g_pending.erase(g_pending.begin() + (long)i);
            } else {
                ++i;
            }
        }
    }
    int first = CBFS_OK;
    for (const auto& p : mine) {
        int h = 0;
        CK(cudaMemcpyAsync(&h, p.word, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaMemsetAsync(p.word, 0, sizeof(int), st));
        CK(cudaStreamSynchronize(st));
        if (h != CBFS_OK && first == CBFS_OK) first = h;
    }
    return first;
}

int cbfs_host_alloc(size_t bytes, void** host_out) {
    if (!host_out) return CBFS_E_INVALID;
    *host_out = nullptr;
    if (cudaHostAlloc(host_out, std::max<size_t>(bytes, 1), cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        *host_out = nullptr;
        return CBFS_E_NOMEM;
    }
    return CBFS_OK;
}

int cbfs_host_free(void* host_ptr) {
    if (!host_ptr) return CBFS_OK;
    return cudaFreeHost(host_ptr) == cudaSuccess ? CBFS_OK : CBFS_E_CUDA;
}

int cbfs_profile(cbfs_graph_t g, int enable, cbfs_kernel_times_t* host_out) {
    if (!g) return CBFS_E_INVALID;
    if (g->iters) {
        // rounds run by graph-mode calls since the last read (three launches each, and
        // a k_flush launch each in waves with round records: bits 40 and up)
        unsigned long long it = 0;
        CK(cudaSetDevice(g->device));
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(&it, g->iters, sizeof(it), cudaMemcpyDeviceToHost));
        CK(cudaMemset(g->iters, 0, sizeof(it)));
        const unsigned long long rounds = it & ((1ull << 40) - 1), flushes = it >> 40;
        g->launches[0] += flushes;
        g->launches[1] += rounds;
        g->launches[2] += rounds;
        g->total_launches += 3ull * rounds + flushes;
    }
    if (host_out) {
        for (int i = 0; i < 3; ++i) {
            host_out->launches[i] = g->launches[i];
            host_out->ms[i] = g->ms[i];
        }
        host_out->total_launches = g->total_launches;
    }
    for (int i = 0; i < 3; ++i) {
        g->launches[i] = 0;
        g->ms[i] = 0.0;
    }
    g->total_launches = 0;
    g->timing = enable != 0;
    return CBFS_OK;
}

int cbfs_output_stats(cbfs_graph_t g, const uint8_t* dist, const uint64_t* masks, const int32_t* host_ks, int C,
                      int d, cbfs_cluster_stats_t* host_out, void* stream) {
    if (!g || C < 0 || d < 0 || d > 15 || !host_out || !host_ks) return CBFS_E_INVALID;
    if (C == 0) return CBFS_OK;
    if (!dist || (d > 0 && !masks)) return CBFS_E_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<uint64_t> alls((size_t)C);
    for (int c = 0; c < C; ++c) {
        if (host_ks[c] < 1 || host_ks[c] > 64) return CBFS_E_INVALID;
        alls[c] = host_ks[c] >= 64 ? ~0ull : ((1ull << host_ks[c]) - 1ull);
    }
    uint64_t* d_alls = nullptr;
    unsigned long long* d_out = nullptr;
    int rc = dev_alloc(&d_alls, C);
    if (!rc) rc = dev_alloc(&d_out, (int64_t)C * 4);
    if (rc) {
        dev_free(d_alls);
        return rc;
    }
    std::vector<unsigned long long> h((size_t)C * 4);
    cudaError_t e = cudaMemcpyAsync(d_alls, alls.data(), sizeof(uint64_t) * C, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_out, 0, sizeof(unsigned long long) * C * 4, st);
    if (e == cudaSuccess) {
        dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((g->n + kThreads - 1) / kThreads, 1024)), (unsigned)C);
        k_output_stats<<<grid, kThreads, 0, st>>>(g->n, d, g->off, dist, masks, d_alls, C, d_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d_out, sizeof(unsigned long long) * C * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(d_alls);
    dev_free(d_out);
    if (e != cudaSuccess) {
        g_last_cuda_error = e;
        return CBFS_E_CUDA;
    }
    for (int c = 0; c < C; ++c) {
        host_out[c].frontier_appearances = h[c * 4 + 0];
        host_out[c].arcs_scanned = h[c * 4 + 1];
        host_out[c].reached_arcs = h[c * 4 + 2];
        host_out[c].rounds = h[c * 4 + 3];
    }
    return CBFS_OK;
}

}  // extern "C"
