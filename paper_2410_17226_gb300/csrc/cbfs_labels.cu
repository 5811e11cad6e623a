// libcbfs.so, part 2: landmark labels and the distance query (Section 4.2).
//
// Label store: one row per vertex v (the L[v][.] of Algorithm "Framework of
// Landmark Labeling"), holding for every stored cluster c the byte
// Delta_v(c) and the subsets S_v[0..d-1](c) as w-bit words (w = 8, 16, 32 or
// 64: clusters of at most w sources, Section 5.3's word sizes):
//   [ dist: Ccap bytes | pad to P = round_up(Ccap, 8)
//     | d blocks of round_up(Ccap * w / 8, 8) bytes ]
// so one query reads two contiguous rows.  A cluster costs 1 + d * w / 8
// bytes per vertex (17 for w = 64, d = 2; 3 for w = 8).
//
// Query (Section 4.2, "Answering Queries with Clustered Landmarks"): for a
// cluster, the distance through its best landmark is Delta_u + Delta_v + t
// for the smallest t = i + j with S_u[i] & S_v[j] != 0 (i, j in 0..d, S_d
// implied as ALL minus the stored subsets); the answer is the minimum over
// clusters.  One warp handles one pair, lanes stride over clusters.
#include <algorithm>
#include <cstring>
#include <vector>

#include "cbfs_internal.cuh"

using namespace cbfs;

struct cbfs_labels_s {
    int64_t n = 0;
    int cap = 0;
    int d = 0;
    int wb = 8;  // bytes per subset word (w / 8)
    int count = 0;
    int64_t P = 0;      // offset of the first subset block
    int64_t block = 0;  // bytes per subset block
    int64_t stride = 0;
    uint8_t* rows = nullptr;
    uint64_t* alls = nullptr;  // [cap]
    // page-locked mirror of alls, the source of stream-ordered uploads: a
    // range below the high-water mark of uploads not yet known to be done is
    // rewritten only after alls_done (after cbfs_labels_reset)
    uint64_t* h_alls = nullptr;
    int64_t h_alls_hw = 0;
    cudaEvent_t alls_done = nullptr;
    int* status = nullptr;
    int device = 0;
};

namespace {

constexpr int kTV = 64;  // vertices per transpose tile
constexpr int kTC = 32;  // clusters per transpose tile

// Cluster-major outputs -> vertex-major rows for clusters [c0, c0 + C);
// subset words narrowed to T (their bits above the cluster size are zero).
template <class T>
__global__ void __launch_bounds__(256) k_labels_append(int64_t n, int d, int C, int c0, int64_t P, int64_t block,
                                                       int64_t stride, const uint8_t* dist, const uint64_t* masks,
                                                       uint8_t* rows) {
    __shared__ uint64_t tm[kTC][kTV + 1];
    __shared__ uint8_t td[kTC][kTV + 4];
    const int64_t v0 = (int64_t)blockIdx.x * kTV;
    const int cb = blockIdx.y * kTC;
    const int nc = min(kTC, C - cb);
    const int nv = (int)((n - v0) < (int64_t)kTV ? (n - v0) : (int64_t)kTV);
    // distances
    for (int i = threadIdx.x; i < kTC * kTV; i += blockDim.x) {
        const int c = i / kTV, vv = i % kTV;
        if (c < nc && vv < nv) td[c][vv] = dist[(size_t)(cb + c) * (size_t)n + v0 + vv];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kTC * kTV; i += blockDim.x) {
        const int vv = i / kTC, c = i % kTC;
        if (c < nc && vv < nv) rows[(v0 + vv) * stride + c0 + cb + c] = td[c][vv];
    }
    // subsets
    for (int s = 0; s < d; ++s) {
        __syncthreads();
        for (int i = threadIdx.x; i < kTC * kTV; i += blockDim.x) {
            const int c = i / kTV, vv = i % kTV;
            if (c < nc && vv < nv) tm[c][vv] = masks[((size_t)(cb + c) * (size_t)d + s) * (size_t)n + v0 + vv];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kTC * kTV; i += blockDim.x) {
            const int vv = i / kTC, c = i % kTC;
            if (c < nc && vv < nv) {
                T* dst = reinterpret_cast<T*>(rows + (v0 + vv) * stride + P + s * block) + c0 + cb + c;
                *dst = (T)tm[c][vv];
            }
        }
    }
}

// Rows of the few (<= 8) clusters of one traversal wave at position pos, from
// their cluster-major outputs: thread per (vertex, cluster), cluster fastest,
// so the lanes of a warp fill whole runs of each row while reading nc
// coalesced streams.  (The tile transpose above would leave most of its
// 32-cluster tile idle.)
template <class T>
__global__ void __launch_bounds__(256) k_labels_wave(int64_t n, int d, int nc, int pos, int64_t P, int64_t block,
                                                     int64_t stride, const uint8_t* dist, const uint64_t* masks,
                                                     uint8_t* rows) {
    const int64_t total = n * nc;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = t / nc;
        const int c = (int)(t - v * nc);
        uint8_t* row = rows + v * stride;
        row[pos + c] = dist[(size_t)c * (size_t)n + v];
        for (int s = 0; s < d; ++s)
            reinterpret_cast<T*>(row + P + s * block)[pos + c] = (T)masks[((size_t)c * (size_t)d + s) * (size_t)n + v];
    }
}

// Smallest t = i + j with Su[i] & Sv[j] != 0, or -1.
template <int D>
__device__ __forceinline__ int best_offset_fixed(const uint64_t* su, const uint64_t* sv) {
#pragma unroll
    for (int t = 0; t <= 2 * D; ++t) {
        uint64_t hit = 0;
#pragma unroll
        for (int i = 0; i <= D; ++i) {
            const int j = t - i;
            if (j >= 0 && j <= D) hit |= su[i] & sv[j];
        }
        if (hit) return t;
    }
    return -1;
}

__device__ __forceinline__ int best_offset_any(const uint64_t* su, const uint64_t* sv, int d) {
    for (int t = 0; t <= 2 * d; ++t) {
        uint64_t hit = 0;
        for (int i = max(0, t - d); i <= min(t, d); ++i) hit |= su[i] & sv[t - i];
        if (hit) return t;
    }
    return -1;
}

// Minimum over the stored clusters of Delta_u + Delta_v + (smallest i + j with
// S_u[i] & S_v[j] != 0), reduced over the calling warp (lanes stride over
// clusters); 0x7fffffff when no cluster reaches both.
template <int D, class T>
__device__ __forceinline__ int label_min(int d, int C, int64_t P, int64_t block, const uint8_t* ru, const uint8_t* rv,
                                         const uint64_t* alls, int lane) {
    constexpr int DM = (D > 0 ? D : 15) + 1;
    int best = 0x7fffffff;
    for (int c = lane; c < C; c += 32) {
        const int du = ru[c], dv = rv[c];
        if (du == 0xFF || dv == 0xFF) continue;
        uint64_t su[DM], sv[DM];
        uint64_t ou = 0, ov = 0;
        const int dd = D > 0 ? D : d;
#pragma unroll
        for (int i = 0; i < DM - 1; ++i) {
            if (i < dd) {
                su[i] = (uint64_t)__ldg(reinterpret_cast<const T*>(ru + P + i * block) + c);
                sv[i] = (uint64_t)__ldg(reinterpret_cast<const T*>(rv + P + i * block) + c);
                ou |= su[i];
                ov |= sv[i];
            }
        }
        const uint64_t all = __ldg(alls + c);
        su[dd] = all & ~ou;
        sv[dd] = all & ~ov;
        const int off = D > 0 ? best_offset_fixed<D>(su, sv) : best_offset_any(su, sv, dd);
        if (off >= 0) best = min(best, du + dv + off);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
    return best;
}

template <int D, class T>
__global__ void __launch_bounds__(256) k_query(int64_t n, int d, int C, int64_t P, int64_t block, int64_t stride,
                                               const uint8_t* rows, const uint64_t* alls, const int32_t* pairs,
                                               int64_t q, uint16_t* out, int* status) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp; t < q; t += nwarps) {
        const int32_t u = pairs[2 * t], v = pairs[2 * t + 1];
        if (u < 0 || v < 0 || (int64_t)u >= n || (int64_t)v >= n) {
            if (lane == 0) {
                out[t] = 0xFFFF;
                atomicCAS(status, 0, CBFS_E_INVALID);
            }
            continue;
        }
        if (u == v) {
            if (lane == 0) out[t] = 0;
            continue;
        }
        const int best = label_min<D, T>(d, C, P, block, rows + (int64_t)u * stride, rows + (int64_t)v * stride, alls,
                                         lane);
        if (lane == 0) out[t] = best == 0x7fffffff ? (uint16_t)0xFFFF : (uint16_t)min(best, 0xFFFE);
    }
}

// ------------------------------------------------ bounded bidirectional search
//
// Appendix B: before answering from the labels, a query searches a few
// vertices around both ends and takes the best meeting point.  Each side
// grows a BFS ball level by level and keeps a level only if the ball then
// holds at most tau vertices (a level that would overflow is dropped whole
// and the side stops), so the balls do not depend on the order in which a
// level's vertices are found.  The local answer is min over x in both balls
// of hops(u, x) + hops(v, x); the query returns the smaller of that and the
// label answer.  One CTA per pair; the two balls share one open-addressing
// table in shared memory: key = vertex rank, hop word = hops from u (bits
// 0-15) and from v (bits 16-31), 0xFFFF = not in that ball.

constexpr int kLocalThreads = 256;
constexpr int kMaxTau = 2048;  // the largest search size of Appendix B; 144 KB of shared memory
constexpr uint32_t kNoHop = 0xFFFFu;

struct LocalShared {
    int32_t* key;
    uint32_t* hop;
    int32_t* list[2];
    int hs_bits;
};

__device__ __forceinline__ uint32_t local_slot(int32_t x, int bits) {
    return ((uint32_t)x * 0x9E3779B1u) >> (32 - bits);
}

// Adds x to side `side`'s ball at hop h; true when x was not in that ball.
__device__ __forceinline__ bool local_insert(const LocalShared& sh, int32_t x, int side, uint32_t h) {
    const uint32_t mask = (1u << sh.hs_bits) - 1u;
    uint32_t s = local_slot(x, sh.hs_bits);
    for (uint32_t probe = 0; probe <= mask; ++probe, s = (s + 1) & mask) {
        int32_t k = sh.key[s];
        if (k == -1) {
            const int32_t prev = atomicCAS(&sh.key[s], -1, x);
            k = prev == -1 ? x : prev;
        }
        if (k != x) continue;
        const uint32_t shift = 16u * (uint32_t)side;
        uint32_t old = sh.hop[s];
        while (((old >> shift) & kNoHop) == kNoHop) {
            const uint32_t want = (old & ~(kNoHop << shift)) | (h << shift);
            const uint32_t got = atomicCAS(&sh.hop[s], old, want);
            if (got == old) return true;
            old = got;
        }
        return false;
    }
    return false;  // table full: cannot happen with the sizes below
}

// Grows one side's ball; returns its size (the list holds its vertices).
__device__ int local_ball(const LocalShared& sh, const int64_t* off, const int32_t* adj, int32_t c, int side, int tau,
                          int* s_cnt, int* s_over) {
    int32_t* list = sh.list[side];
    __syncthreads();  // every thread has read the previous ball's counters
    if (threadIdx.x == 0) {
        list[0] = c;
        *s_cnt = 1;
        *s_over = 0;
        local_insert(sh, c, side, 0);
    }
    __syncthreads();
    int lo = 0, size = 1;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = kLocalThreads / 32;
    for (uint32_t h = 1; h < kNoHop; ++h) {  // at most tau levels
        // one warp per frontier vertex, lanes over its arcs
        for (int i = lo + wp; i < size; i += nw) {
            const int32_t x = list[i];
            const int64_t e1 = off[x + 1];
            for (int64_t e = off[x] + lane; e < e1; e += 32) {
                if (*(volatile int*)s_over) break;
                const int32_t y = adj[e];
                if (local_insert(sh, y, side, h)) {
                    const int at = atomicAdd(s_cnt, 1);
                    if (at < tau) list[at] = y;
                    else *(volatile int*)s_over = 1;
                }
            }
        }
        __syncthreads();
        const int grown = *s_cnt, over = *s_over;
        if (over) {
            // drop the partial level h everywhere in the table
            const uint32_t shift = 16u * (uint32_t)side;
            for (int s = threadIdx.x; s < (1 << sh.hs_bits); s += kLocalThreads)
                if (((sh.hop[s] >> shift) & kNoHop) == h) atomicOr(&sh.hop[s], kNoHop << shift);
            __syncthreads();
            return size;
        }
        if (grown == size) return size;
        lo = size;
        size = grown;
        __syncthreads();
    }
    return size;
}

template <int D, class T>
__global__ void __launch_bounds__(kLocalThreads) k_query_local(int64_t n, int d, int C, int64_t P, int64_t block,
                                                               int64_t stride, const uint8_t* rows,
                                                               const uint64_t* alls, GraphView gv,
                                                               const int32_t* pairs, int64_t q, int tau,
                                                               int hs_bits, uint16_t* out, int* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    LocalShared sh;
    sh.hs_bits = hs_bits;
    const int hs = 1 << hs_bits;
    sh.key = reinterpret_cast<int32_t*>(smem);
    sh.hop = reinterpret_cast<uint32_t*>(smem + 4 * (size_t)hs);
    sh.list[0] = reinterpret_cast<int32_t*>(smem + 8 * (size_t)hs);
    sh.list[1] = sh.list[0] + tau;
    __shared__ int s_cnt, s_over, s_best, s_lab;
    const int lane = threadIdx.x & 31;
    for (int64_t t = blockIdx.x; t < q; t += gridDim.x) {
        const int32_t u = pairs[2 * t], v = pairs[2 * t + 1];
        if (u < 0 || v < 0 || (int64_t)u >= n || (int64_t)v >= n) {
            if (threadIdx.x == 0) {
                out[t] = 0xFFFF;
                atomicCAS(status, 0, CBFS_E_INVALID);
            }
            continue;
        }
        if (u == v) {
            if (threadIdx.x == 0) out[t] = 0;
            continue;
        }
        if (threadIdx.x < 32) {
            const int lab = C > 0 ? label_min<D, T>(d, C, P, block, rows + (int64_t)u * stride,
                                                    rows + (int64_t)v * stride, alls, lane)
                                  : 0x7fffffff;
            if (lane == 0) s_lab = lab;
        }
        for (int s = threadIdx.x; s < hs; s += kLocalThreads) {
            sh.key[s] = -1;
            sh.hop[s] = 0xFFFFFFFFu;
        }
        if (threadIdx.x == 0) s_best = 0x7fffffff;
        __syncthreads();
        const int32_t ru = gv.iperm[u], rv = gv.iperm[v];
        local_ball(sh, gv.off, gv.adj, ru, 0, tau, &s_cnt, &s_over);
        const int sv = local_ball(sh, gv.off, gv.adj, rv, 1, tau, &s_cnt, &s_over);
        // best meeting point over v's ball
        int best = 0x7fffffff;
        const uint32_t mask = (uint32_t)hs - 1u;
        for (int i = threadIdx.x; i < sv; i += kLocalThreads) {
            const int32_t x = sh.list[1][i];
            uint32_t s = local_slot(x, hs_bits);
            for (uint32_t probe = 0; probe <= mask; ++probe, s = (s + 1) & mask) {
                if (sh.key[s] != x) continue;
                const uint32_t w = sh.hop[s];
                const uint32_t a = w & kNoHop, b = w >> 16;
                if (a != kNoHop && b != kNoHop) best = min(best, (int)(a + b));
                break;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
        if (lane == 0 && best != 0x7fffffff) atomicMin(&s_best, best);
        __syncthreads();
        if (threadIdx.x == 0) {
            const int r = min(s_best, s_lab);
            out[t] = r == 0x7fffffff ? (uint16_t)0xFFFF : (uint16_t)min(r, 0xFFFE);
        }
        __syncthreads();
    }
}

// Launch helpers for the store's word width.
void append_rows(const cbfs_labels_s* L, const uint8_t* dist, const uint64_t* masks, int C, int pos, cudaStream_t st) {
    if (C <= 8) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, L->device);
        const unsigned blocks = (unsigned)std::min<int64_t>((L->n * C + 255) / 256, (int64_t)std::max(sms, 1) * 8);
#define CBFS_WAVE(T) k_labels_wave<T><<<blocks, 256, 0, st>>>(L->n, L->d, C, pos, L->P, L->block, L->stride, dist, masks, L->rows)
        switch (L->wb) {
            case 1: CBFS_WAVE(uint8_t); break;
            case 2: CBFS_WAVE(uint16_t); break;
            case 4: CBFS_WAVE(uint32_t); break;
            default: CBFS_WAVE(uint64_t); break;
        }
#undef CBFS_WAVE
    } else {
        dim3 grid((unsigned)((L->n + kTV - 1) / kTV), (unsigned)((C + kTC - 1) / kTC));
#define CBFS_TILE(T) k_labels_append<T><<<grid, 256, 0, st>>>(L->n, L->d, C, pos, L->P, L->block, L->stride, dist, masks, L->rows)
        switch (L->wb) {
            case 1: CBFS_TILE(uint8_t); break;
            case 2: CBFS_TILE(uint16_t); break;
            case 4: CBFS_TILE(uint32_t); break;
            default: CBFS_TILE(uint64_t); break;
        }
#undef CBFS_TILE
    }
}

template <int D, class T>
cudaError_t launch_local(const cbfs_labels_s* L, const GraphView& gv, const int32_t* pairs, int64_t q, int tau,
                         int hs_bits, uint16_t* out, int* status, cudaStream_t st) {
    const size_t smem = 8 * ((size_t)1 << hs_bits) + 8 * (size_t)tau;
    cudaError_t e = cudaFuncSetAttribute(k_query_local<D, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int sms = 0, occ = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, gv.device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_query_local<D, T>, kLocalThreads, smem);
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(q, (int64_t)std::max(sms, 1) * std::max(occ, 1)));
    if (L)
        k_query_local<D, T><<<(unsigned)blocks, kLocalThreads, smem, st>>>(
            L->n, L->d, L->count, L->P, L->block, L->stride, L->rows, L->alls, gv, pairs, q, tau, hs_bits, out, status);
    else
        k_query_local<D, T><<<(unsigned)blocks, kLocalThreads, smem, st>>>(gv.n, 0, 0, 0, 0, 0, nullptr, nullptr, gv,
                                                                           pairs, q, tau, hs_bits, out, status);
    return cudaGetLastError();
}

template <int D>
void query_rows(const cbfs_labels_s* L, unsigned blocks, const int32_t* pairs, int64_t q, uint16_t* out,
                cudaStream_t st) {
#define CBFS_QUERY(T)                                                                                              \
    k_query<D, T><<<blocks, 256, 0, st>>>(L->n, L->d, L->count, L->P, L->block, L->stride, L->rows, L->alls, pairs, \
                                          q, out, L->status)
    switch (L->wb) {
        case 1: CBFS_QUERY(uint8_t); break;
        case 2: CBFS_QUERY(uint16_t); break;
        case 4: CBFS_QUERY(uint32_t); break;
        default: CBFS_QUERY(uint64_t); break;
    }
#undef CBFS_QUERY
}

// Stream-ordered upload of the ALL words of clusters [L->count, L->count + C)
// with sizes ks[c] (already checked) from the page-locked mirror.  A range
// that an earlier upload may still be reading (after a reset) is rewritten
// only once that upload has run.
int put_alls(cbfs_labels_s* L, const int32_t* ks, int64_t ks_step, int C, cudaStream_t st) {
    if (C == 0) return CBFS_OK;
    if (L->count < L->h_alls_hw) {
        if (cudaEventSynchronize(L->alls_done) != cudaSuccess) return CBFS_E_CUDA;
        L->h_alls_hw = 0;
    }
    for (int c = 0; c < C; ++c) {
        const int k = ks[(int64_t)c * ks_step];
        L->h_alls[L->count + c] = k >= 64 ? ~0ull : ((1ull << k) - 1ull);
    }
    if (cudaMemcpyAsync(L->alls + L->count, L->h_alls + L->count, sizeof(uint64_t) * C, cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaEventRecord(L->alls_done, st) != cudaSuccess)
        return CBFS_E_CUDA;
    L->h_alls_hw = std::max<int64_t>(L->h_alls_hw, (int64_t)L->count + C);
    return CBFS_OK;
}

}  // namespace

namespace cbfs {

int labels_reserve(cbfs_labels_s* L, int64_t n, int d, const int32_t* coff, int C, int* base, cudaStream_t st) {
    if (L->n != n || L->d != d || C < 0) return CBFS_E_INVALID;
    if (L->count + C > L->cap) return CBFS_E_NOMEM;
    std::vector<int32_t> ks((size_t)std::max(C, 1));
    for (int c = 0; c < C; ++c) {
        ks[c] = coff[c + 1] - coff[c];
        if (ks[c] < 1 || ks[c] > 8 * L->wb) return CBFS_E_INVALID;
    }
    cudaSetDevice(L->device);
    const int rc = put_alls(L, ks.data(), 1, C, st);
    if (rc) return rc;
    *base = L->count;
    L->count += C;
    return CBFS_OK;
}

void labels_rollback(cbfs_labels_s* L, int base) { L->count = base; }

cudaError_t labels_write(cbfs_labels_s* L, const uint8_t* dist, const uint64_t* masks, int C, int pos,
                         cudaStream_t st) {
    if (L->n == 0 || C == 0) return cudaSuccess;
    append_rows(L, dist, masks, C, pos, st);
    return cudaGetLastError();
}

}  // namespace cbfs

extern "C" {

int cbfs_labels_create_w(int64_t n, int C_capacity, int d, int w, size_t hbm_budget_bytes, cbfs_labels_t* out) {
    if (!out || n < 0 || n >= (int64_t)0x7fffffff || C_capacity < 1 || d < 0 || d > 15) return CBFS_E_INVALID;
    if (w != 8 && w != 16 && w != 32 && w != 64) return CBFS_E_INVALID;
    *out = nullptr;
    cbfs_labels_s* L = new (std::nothrow) cbfs_labels_s();
    if (!L) return CBFS_E_NOMEM;
    cudaGetDevice(&L->device);
    L->n = n;
    L->cap = C_capacity;
    L->d = d;
    L->wb = w / 8;
    L->P = ((int64_t)C_capacity + 7) / 8 * 8;
    L->block = ((int64_t)C_capacity * L->wb + 7) / 8 * 8;
    L->stride = L->P + (int64_t)d * L->block;
    const size_t bytes = (size_t)std::max<int64_t>(n, 1) * (size_t)L->stride;
    if (hbm_budget_bytes && bytes > hbm_budget_bytes) {
        delete L;
        return CBFS_E_NOMEM;
    }
    if (cudaMalloc((void**)&L->rows, bytes) != cudaSuccess || cudaMalloc((void**)&L->alls, sizeof(uint64_t) * C_capacity) != cudaSuccess ||
        cudaMalloc((void**)&L->status, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cbfs_labels_destroy(L);
        return CBFS_E_NOMEM;
    }
    if (cudaMallocHost((void**)&L->h_alls, sizeof(uint64_t) * C_capacity) != cudaSuccess ||
        cudaEventCreateWithFlags(&L->alls_done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        L->h_alls = nullptr;
        cbfs_labels_destroy(L);
        return CBFS_E_NOMEM;
    }
    if (cudaMemset(L->rows, 0, bytes) != cudaSuccess || cudaMemset(L->status, 0, sizeof(int)) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        cbfs_labels_destroy(L);
        return CBFS_E_CUDA;
    }
    *out = L;
    return CBFS_OK;
}

int cbfs_labels_create(int64_t n, int C_capacity, int d, size_t hbm_budget_bytes, cbfs_labels_t* out) {
    return cbfs_labels_create_w(n, C_capacity, d, 64, hbm_budget_bytes, out);
}

int cbfs_labels_destroy(cbfs_labels_t L) {
    if (!L) return CBFS_OK;
    status_forget(L);
    cudaSetDevice(L->device);
    cudaDeviceSynchronize();
    if (L->rows) cudaFree(L->rows);
    if (L->alls) cudaFree(L->alls);
    if (L->status) cudaFree(L->status);
    if (L->h_alls) cudaFreeHost(L->h_alls);
    if (L->alls_done) cudaEventDestroy(L->alls_done);
    delete L;
    return CBFS_OK;
}

int cbfs_labels_append(cbfs_labels_t L, const uint8_t* dist, const uint64_t* masks, const int32_t* host_ks, int C,
                       void* stream) {
    if (!L || C < 0 || (C > 0 && (!dist || !host_ks || (L->d > 0 && !masks)))) return CBFS_E_INVALID;
    if (L->count + C > L->cap) return CBFS_E_INVALID;
    if (C == 0) return CBFS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    for (int c = 0; c < C; ++c)
        if (host_ks[c] < 1 || host_ks[c] > 8 * L->wb) return CBFS_E_INVALID;
    const int rc = put_alls(L, host_ks, 1, C, st);
    if (rc) return rc;
    if (L->n > 0) {
        append_rows(L, dist, masks, C, L->count, st);
        if (cudaGetLastError() != cudaSuccess) return CBFS_E_CUDA;
    }
    L->count += C;
    return CBFS_OK;
}

int cbfs_labels_reset(cbfs_labels_t L) {
    if (!L) return CBFS_E_INVALID;
    L->count = 0;
    return CBFS_OK;
}

int cbfs_labels_count(cbfs_labels_t L, int* host_count) {
    if (!L || !host_count) return CBFS_E_INVALID;
    *host_count = L->count;
    return CBFS_OK;
}

int cbfs_labels_rows(cbfs_labels_t L, const uint8_t** host_rows, int64_t* host_stride) {
    if (!L) return CBFS_E_INVALID;
    if (host_rows) *host_rows = L->rows;
    if (host_stride) *host_stride = L->stride;
    return CBFS_OK;
}

int cbfs_query_distance(cbfs_labels_t L, const int32_t* pairs, int64_t q, uint16_t* out, void* stream) {
    if (!L || q < 0 || (q > 0 && (!pairs || !out))) return CBFS_E_INVALID;
    if (q == 0) return CBFS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t warps_per_block = 8;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((q + warps_per_block - 1) / warps_per_block, 152 * 16));
    switch (L->d) {
        case 1: query_rows<1>(L, (unsigned)blocks, pairs, q, out, st); break;
        case 2: query_rows<2>(L, (unsigned)blocks, pairs, q, out, st); break;
        default: query_rows<0>(L, (unsigned)blocks, pairs, q, out, st); break;
    }
    if (cudaGetLastError() != cudaSuccess) return CBFS_E_CUDA;
    status_register(st, L->status, L);
    return CBFS_OK;
}

int cbfs_query_local(cbfs_labels_t L, cbfs_graph_t g, const int32_t* pairs, int64_t q, int tau, uint16_t* out,
                     void* stream) {
    if (!g || q < 0 || (q > 0 && (!pairs || !out)) || tau < 1 || tau > kMaxTau) return CBFS_E_INVALID;
    GraphView gv;
    if (graph_view(g, &gv) != CBFS_OK) return CBFS_E_INVALID;
    if (L && L->n != gv.n) return CBFS_E_INVALID;
    if (q == 0) return CBFS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // both balls' entries plus the inserts racing past an overflow, at load <= 1/2
    int hs_bits = 4;
    while ((1 << hs_bits) < 2 * (2 * tau + 2 * kLocalThreads)) hs_bits++;
    int* status = nullptr;
    if (L) {
        status = L->status;
    } else {
        status = graph_status(g);
    }
    cudaError_t e;
    if (!L) {
        e = launch_local<0, uint64_t>(nullptr, gv, pairs, q, tau, hs_bits, out, status, st);
    } else {
#define CBFS_LOCAL(DD)                                                                                    \
    switch (L->wb) {                                                                                      \
        case 1: e = launch_local<DD, uint8_t>(L, gv, pairs, q, tau, hs_bits, out, status, st); break;    \
        case 2: e = launch_local<DD, uint16_t>(L, gv, pairs, q, tau, hs_bits, out, status, st); break;   \
        case 4: e = launch_local<DD, uint32_t>(L, gv, pairs, q, tau, hs_bits, out, status, st); break;   \
        default: e = launch_local<DD, uint64_t>(L, gv, pairs, q, tau, hs_bits, out, status, st); break;  \
    }
        switch (L->d) {
            case 1: CBFS_LOCAL(1); break;
            case 2: CBFS_LOCAL(2); break;
            default: CBFS_LOCAL(0); break;
        }
#undef CBFS_LOCAL
    }
    if (e != cudaSuccess) return CBFS_E_CUDA;
    status_register(st, status, L ? (const void*)L : (const void*)g);
    return CBFS_OK;
}

int cbfs_labels_status(cbfs_labels_t L, void* stream) {
    if (!L) return CBFS_E_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    if (cudaMemcpyAsync(&h, L->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return CBFS_E_CUDA;
    if (cudaMemsetAsync(L->status, 0, sizeof(int), st) != cudaSuccess) return CBFS_E_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return CBFS_E_CUDA;
    return h;
}

}  // extern "C"
