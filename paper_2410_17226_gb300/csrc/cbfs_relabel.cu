// libcbfs.so, part 4: the internal vertex order of a resident graph.
//
// The traversal runs on a relabelled copy of the CSR: vertices are ranked by
// degree, highest first (ties to the smaller id), and every adjacency list is
// rewritten in ranks and ordered by rank.  High-degree vertices -- the
// neighbours most arcs of a power-law graph point to -- then have their state
// words side by side, so gathers of them hit in L1/L2, and every list starts
// with its best-connected neighbours, which are reached first, so the
// early exit of the dense edge phase comes sooner.  Lists of up to kPullMid
// arcs are fully sorted; longer lists are ordered by the top rank bits only
// (a one-pass bucket scatter), which keeps both effects.  Outputs are still
// written at the caller's vertex ids through the rank -> id map.
#include <algorithm>
#include <cstring>
#include <vector>

#include "cbfs_internal.cuh"

using namespace cbfs;

namespace {

constexpr int kBuckets = 256;

// Lists of degree <= kPullSmall: one thread maps and insertion-sorts in registers.
__global__ void k_relabel_small(int64_t r0, int64_t r1, const int32_t* perm, const int32_t* iperm, const int64_t* off,
                                const int32_t* adj, const int64_t* off_r, int32_t* adj_r) {
    for (int64_t r = r0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < r1; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = perm[r];
        const int64_t o0 = off[v];
        const int deg = (int)(off[v + 1] - o0);
        int32_t x[kPullSmall];
#pragma unroll
        for (int i = 0; i < kPullSmall; ++i) x[i] = i < deg ? iperm[adj[o0 + i]] : 0x7fffffff;
        // insertion sort (fixed trip counts keep x in registers)
#pragma unroll
        for (int i = 1; i < kPullSmall; ++i) {
#pragma unroll
            for (int j = i; j > 0; --j) {
                const int32_t a = x[j - 1], b = x[j];
                x[j - 1] = min(a, b);
                x[j] = max(a, b);
            }
        }
        int32_t* dst = adj_r + off_r[r];
#pragma unroll
        for (int i = 0; i < kPullSmall; ++i)
            if (i < deg) dst[i] = x[i];
    }
}

// Lists of degree in (kPullSmall, kPullMid]: one CTA maps and bitonic-sorts in shared memory.
__global__ void __launch_bounds__(kThreads) k_relabel_mid(int64_t r0, int64_t r1, const int32_t* perm, const int32_t* iperm,
                                                          const int64_t* off, const int32_t* adj, const int64_t* off_r,
                                                          int32_t* adj_r) {
    __shared__ int32_t s[kPullMid];
    for (int64_t r = r0 + blockIdx.x; r < r1; r += gridDim.x) {
        const int32_t v = perm[r];
        const int64_t o0 = off[v];
        const int deg = (int)(off[v + 1] - o0);
        int len = 1;
        while (len < deg) len <<= 1;
        for (int i = threadIdx.x; i < len; i += blockDim.x) s[i] = i < deg ? iperm[adj[o0 + i]] : 0x7fffffff;
        __syncthreads();
        for (int k = 2; k <= len; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < len; i += blockDim.x) {
                    const int p = i ^ j;
                    if (p > i) {
                        const bool up = (i & k) == 0;
                        const int32_t a = s[i], b = s[p];
                        if ((a > b) == up) {
                            s[i] = b;
                            s[p] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        int32_t* dst = adj_r + off_r[r];
        for (int i = threadIdx.x; i < deg; i += blockDim.x) dst[i] = s[i];
        __syncthreads();
    }
}

// Lists longer than kPullMid: one CTA maps and scatters by the top rank bits.
__global__ void __launch_bounds__(kThreads) k_relabel_big(int64_t r0, int64_t r1, int shift, const int32_t* perm,
                                                          const int32_t* iperm, const int64_t* off, const int32_t* adj,
                                                          const int64_t* off_r, int32_t* adj_r) {
    __shared__ unsigned int cnt[kBuckets];
    __shared__ unsigned int pos[kBuckets];
    for (int64_t r = r0 + blockIdx.x; r < r1; r += gridDim.x) {
        const int32_t v = perm[r];
        const int64_t o0 = off[v];
        const int64_t deg = off[v + 1] - o0;
        for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) cnt[i] = 0;
        __syncthreads();
        for (int64_t i = threadIdx.x; i < deg; i += blockDim.x) atomicAdd(&cnt[iperm[adj[o0 + i]] >> shift], 1u);
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned int sum = 0;
            for (int b = 0; b < kBuckets; ++b) {
                pos[b] = sum;
                sum += cnt[b];
            }
        }
        __syncthreads();
        int32_t* dst = adj_r + off_r[r];
        for (int64_t i = threadIdx.x; i < deg; i += blockDim.x) {
            const int32_t x = iperm[adj[o0 + i]];
            dst[atomicAdd(&pos[x >> shift], 1u)] = x;
        }
        __syncthreads();
    }
}

}  // namespace

namespace {

// ---------------------------------------------------------------- rank order
//
// Ranks are produced on the device: a stable LSD radix sort of the key
// 0xFFFFFFFF - order_deg(v) over the ids 0..n-1 (8-bit digits, only as many
// passes as the largest degree has bits).  order_deg is the degree above
// kPullSmall and the degree rounded up to a power of two at or below it, so
// ascending keys give descending degrees down to kPullSmall, then the
// buckets 32, 16, 8, 4, 2, 1 and finally the isolated vertices; stability
// keeps ascending ids within a degree or a bucket.  The buckets keep most of
// the input order of graphs whose vertices all have similar low degrees (a
// road grid's row-major order, where a vertex's neighbours are the ids next
// to it), while a warp's 32 consecutive vertices still differ in degree by
// less than 2x.
__device__ __forceinline__ uint32_t order_deg(int64_t dg) {
    if (dg > kPullSmall || dg <= 1) return (uint32_t)dg;
    uint32_t b = 2;
    while ((int64_t)b < dg) b <<= 1;
    return b;
}

constexpr int kSortItems = 16;                    // items per thread per tile
constexpr int kSortTile = kThreads * kSortItems;  // 4096 items per CTA

__global__ void k_widen_off(const int32_t* in, int64_t* out, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i];
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Offsets check, degree statistics and the sort keys.
__global__ void __launch_bounds__(kThreads) k_degree_stats(int64_t n, int64_t nnz, const int64_t* off, DegreeStats* st,
                                                           uint32_t* keys) {
    unsigned long long cls[4] = {0, 0, 0, 0};  // small, mid, big (> kPullMid), pieces of lists > kBigDeg
    unsigned long long mx = 0;
    int bad = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (off[0] != 0 || off[n] != nnz)) bad = 1;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t dg = off[v + 1] - off[v];
        if (dg < 0 || dg > 0x7fffffffLL) {
            bad = 1;
            keys[v] = 0;
            continue;
        }
        keys[v] = 0xFFFFFFFFu - order_deg(dg);
        mx = dg > (int64_t)mx ? (unsigned long long)dg : mx;
        if (dg == 0) continue;
        if (dg <= kPullSmall) cls[0]++;
        else if (dg <= kPullMid) cls[1]++;
        else cls[2]++;
        if (dg > kBigDeg) cls[3] += (unsigned long long)((dg + kBigDeg - 1) / kBigDeg);
    }
    __shared__ unsigned long long red[kWarps][5];
    __shared__ int sbad;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    if (bad) sbad = 1;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 4; ++i) cls[i] = warp_sum_u64(cls[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = y > mx ? y : mx;
    }
    if (lane == 0) {
        for (int i = 0; i < 4; ++i) red[wp][i] = cls[i];
        red[wp][4] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t[5] = {0, 0, 0, 0, 0};
        for (int k = 0; k < kWarps; ++k) {
            for (int i = 0; i < 4; ++i) t[i] += red[k][i];
            t[4] = red[k][4] > t[4] ? red[k][4] : t[4];
        }
        atomicAdd(&st->n_small, t[0]);
        atomicAdd(&st->n_mid, t[1]);
        atomicAdd(&st->n_big, t[2]);
        atomicAdd(&st->big_pieces, t[3]);
        atomicMax(&st->maxdeg, t[4]);
        if (sbad) atomicExch(&st->bad, 1ull);
    }
}

// Digit counts of one tile, stored digit-major: hist[digit * ntiles + tile].
__global__ void __launch_bounds__(kThreads) k_sort_hist(const uint32_t* keys, int64_t n, int shift, int64_t* hist,
                                                        int64_t ntiles) {
    __shared__ unsigned int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
    for (int i = 0; i < kSortItems; ++i) {
        const int64_t idx = base + i * kThreads + threadIdx.x;
        if (idx < n) atomicAdd(&cnt[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter of one tile: item order within a digit is kept by ranking
// the tile in 16 rounds of 256 consecutive items (warp match, then per-warp
// digit counts in shared memory, then a running count per digit).
__global__ void __launch_bounds__(kThreads) k_sort_scatter(const uint32_t* keys_in, const int32_t* vals_in, int64_t n,
                                                           int shift, const int64_t* start, int64_t ntiles,
                                                           uint32_t* keys_out, int32_t* vals_out) {
    __shared__ unsigned int wcnt[kWarps][256];
    __shared__ unsigned int run[256];
    __shared__ int64_t gbase[256];
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    run[t] = 0;
    gbase[t] = start[(int64_t)t * ntiles + blockIdx.x];
#pragma unroll
    for (int k = 0; k < kWarps; ++k) wcnt[k][t] = 0;
    __syncthreads();
    const unsigned int lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int i = 0; i < kSortItems; ++i) {
        const int64_t idx = base + i * kThreads + t;
        const bool valid = idx < n;
        const uint32_t key = valid ? keys_in[idx] : 0u;
        const int32_t val = valid ? (vals_in ? vals_in[idx] : (int32_t)idx) : 0;
        const unsigned int dg = valid ? ((key >> shift) & 255u) : 256u;
        const unsigned int peers = __match_any_sync(0xffffffffu, dg);
        const unsigned int wr = __popc(peers & lt);
        if (valid && wr == 0) wcnt[wp][dg] = __popc(peers);
        __syncthreads();
        if (valid) {
            unsigned int pos = run[dg] + wr;
            for (int k = 0; k < wp; ++k) pos += wcnt[k][dg];
            const int64_t at = gbase[dg] + pos;
            if (at < n) {  // always true for a consistent histogram
                keys_out[at] = key;
                vals_out[at] = val;
            }
        }
        __syncthreads();
        unsigned int sum = 0;
#pragma unroll
        for (int k = 0; k < kWarps; ++k) {
            sum += wcnt[k][t];
            wcnt[k][t] = 0;
        }
        run[t] += sum;
        __syncthreads();
    }
}

// Exclusive scan of int64 values in tiles of kSortTile: per-tile sums, a
// one-CTA scan of the sums, then per-tile prefixes.  out[count] = total.
__device__ __forceinline__ int64_t block_exclusive_i64(int64_t x, int64_t* total) {
    __shared__ int64_t ws[kWarps];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    int64_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) ws[wp] = inc;
    __syncthreads();
    int64_t before = 0, all = 0;
    for (int k = 0; k < kWarps; ++k) {
        if (k < wp) before += ws[k];
        all += ws[k];
    }
    __syncthreads();
    *total = all;
    return before + inc - x;
}

__global__ void __launch_bounds__(kThreads) k_scan_reduce(const int64_t* in, int64_t count, int64_t* sums) {
    const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)threadIdx.x * kSortItems;
    int64_t s = 0;
    for (int i = 0; i < kSortItems; ++i)
        if (base + i < count) s += in[base + i];
    int64_t total;
    block_exclusive_i64(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kThreads) k_scan_sums(int64_t* sums, int64_t ntiles) {
    int64_t carry = 0;
    for (int64_t b = 0; b < ntiles; b += kThreads) {
        const int64_t i = b + threadIdx.x;
        const int64_t x = i < ntiles ? sums[i] : 0;
        int64_t total;
        const int64_t ex = block_exclusive_i64(x, &total);
        if (i < ntiles) sums[i] = carry + ex;
        carry += total;
    }
}

__global__ void __launch_bounds__(kThreads) k_scan_apply(const int64_t* in, int64_t count, const int64_t* sums,
                                                         int64_t* out) {
    const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)threadIdx.x * kSortItems;
    int64_t v[kSortItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        v[i] = base + i < count ? in[base + i] : 0;
        s += v[i];
    }
    int64_t total;
    int64_t run = sums[blockIdx.x] + block_exclusive_i64(s, &total);
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        if (base + i < count) out[base + i] = run;
        run += v[i];
        if (base + i == count - 1) out[count] = run;
    }
}

__global__ void k_rank_finish(int64_t n, const int32_t* perm, const int64_t* off, int32_t* iperm, int64_t* deg_r) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = perm[r];
        iperm[v] = (int32_t)r;
        deg_r[r] = off[v + 1] - off[v];
    }
}

// The relabel kernels size their buffers by degree class, so the order is
// checked before they run: perm and iperm are inverse permutations and
// order_deg never increases along the ranks.
__global__ void k_check_rank(int64_t n, const int32_t* perm, const int32_t* iperm, const int64_t* deg_r,
                             DegreeStats* st) {
    bool bad = false;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = iperm[v];
        if (r < 0 || (int64_t)r >= n || perm[r] != (int32_t)v) bad = true;
        if (v + 1 < n && order_deg(deg_r[v]) < order_deg(deg_r[v + 1])) bad = true;
    }
    if (bad) atomicExch(&st->order_bad, 1ull);
}

// Degree histogram for the pull classes of any threshold pair: the common
// low degrees are counted per CTA in shared memory and merged with one atomic
// per non-empty bin; the rare higher ones go to the global bins directly.
constexpr int kHistShared = 4096;

__global__ void __launch_bounds__(kThreads) k_degree_hist(int64_t n, const int64_t* off, unsigned long long* hist) {
    __shared__ unsigned int bins[kHistShared + 1];
    for (int i = threadIdx.x; i <= kHistShared; i += kThreads) bins[i] = 0;
    __syncthreads();
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t dg = off[v + 1] - off[v];
        if (dg <= kHistShared) atomicAdd(&bins[(int)dg], 1u);
        else atomicAdd(&hist[dg > kMaxMidDeg ? kMaxMidDeg + 1 : (int)dg], 1ull);
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= kHistShared; i += kThreads)
        if (bins[i]) atomicAdd(&hist[i], (unsigned long long)bins[i]);
}

__global__ void k_map_seeds(uint64_t* seeds, int64_t count, const int32_t* iperm) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t e = seeds[i];
        seeds[i] = (e & 0xFFFFFFFF00000000ull) | (uint32_t)iperm[(uint32_t)e];
    }
}

int64_t tiles_of(int64_t count) { return (count + kSortTile - 1) / kSortTile; }

}  // namespace

namespace cbfs {

cudaError_t widen_offsets(const int32_t* in, int64_t* out, int64_t count, int sms, cudaStream_t st) {
    if (count > 0) k_widen_off<<<sms * 8, kThreads, 0, st>>>(in, out, count);
    return cudaGetLastError();
}

cudaError_t degree_stats(int64_t n, int64_t nnz, const int64_t* off, DegreeStats* st_dev, uint32_t* keys, int sms,
                         cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(st_dev, 0, sizeof(DegreeStats), st);
    if (e != cudaSuccess) return e;
    k_degree_stats<<<sms * 8, kThreads, 0, st>>>(n, nnz, off, st_dev, keys);
    return cudaGetLastError();
}

// Scratch of the rank order, in int64 words:
//   keys | keys2 | vals_a | vals_b (n 32-bit entries each) | hist (256 per tile, + 1)
//   | tile sums | deg_r (n)
struct RankScratch {
    uint32_t *keys, *keys2;
    int32_t *vals_a, *vals_b;
    int64_t *hist, *sums, *deg_r;
    int64_t words;
};

static RankScratch rank_layout(int64_t n, int64_t* base) {
    const int64_t half = n / 2 + 1;
    const int64_t nh = 256 * tiles_of(n);
    const int64_t o_hist = 4 * half, o_sums = o_hist + nh + 1;
    const int64_t o_deg = o_sums + tiles_of(nh + 1) + tiles_of(n) + 1;
    RankScratch r;
    r.words = o_deg + n + 1;
    r.keys = base ? (uint32_t*)base : nullptr;
    r.keys2 = base ? (uint32_t*)(base + half) : nullptr;
    r.vals_a = base ? (int32_t*)(base + 2 * half) : nullptr;
    r.vals_b = base ? (int32_t*)(base + 3 * half) : nullptr;
    r.hist = base ? base + o_hist : nullptr;
    r.sums = base ? base + o_sums : nullptr;
    r.deg_r = base ? base + o_deg : nullptr;
    return r;
}

int64_t rank_scratch_words(int64_t n) { return rank_layout(n, nullptr).words; }

uint32_t* rank_keys(int64_t n, int64_t* scratch) { return rank_layout(n, scratch).keys; }

cudaError_t exclusive_scan_i64(const int64_t* in, int64_t count, int64_t* out, int64_t* sums, cudaStream_t st) {
    if (count <= 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), st);
    const int64_t tiles = tiles_of(count);
    k_scan_reduce<<<(unsigned)tiles, kThreads, 0, st>>>(in, count, sums);
    k_scan_sums<<<1, kThreads, 0, st>>>(sums, tiles);
    k_scan_apply<<<(unsigned)tiles, kThreads, 0, st>>>(in, count, sums, out);
    return cudaGetLastError();
}

cudaError_t rank_order_device(int64_t n, const int64_t* off, uint64_t maxdeg, int64_t* scratch, int32_t* perm,
                              int32_t* iperm, int64_t* off_r, DegreeStats* st_dev, int sms, cudaStream_t st) {
    if (n == 0) return cudaMemsetAsync(off_r, 0, sizeof(int64_t), st);
    const RankScratch r = rank_layout(n, scratch);
    const int64_t tiles = tiles_of(n);
    const int64_t nh = 256 * tiles;
    int passes = 1;  // at least one pass: it also writes the identity values
    while (passes < 4 && (maxdeg >> (8 * passes)) != 0) passes++;
    uint32_t* kin = r.keys;
    uint32_t* kout = r.keys2;
    const int32_t* vin = nullptr;  // the ids themselves on the first pass
    int32_t* vout = r.vals_a;
    for (int p = 0; p < passes; ++p) {
        k_sort_hist<<<(unsigned)tiles, kThreads, 0, st>>>(kin, n, 8 * p, r.hist, tiles);
        // in place: every tile of the scan rewrites only the entries it read
        cudaError_t e = exclusive_scan_i64(r.hist, nh, r.hist, r.sums, st);
        if (e != cudaSuccess) return e;
        k_sort_scatter<<<(unsigned)tiles, kThreads, 0, st>>>(kin, vin, n, 8 * p, r.hist, tiles, kout, vout);
        std::swap(kin, kout);
        vin = vout;
        vout = (vout == r.vals_a) ? r.vals_b : r.vals_a;
    }
    cudaError_t e = cudaMemcpyAsync(perm, vin, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(iperm, 0xFF, sizeof(int32_t) * (size_t)n, st);
    if (e != cudaSuccess) return e;
    k_rank_finish<<<sms * 8, kThreads, 0, st>>>(n, perm, off, iperm, r.deg_r);
    k_check_rank<<<sms * 8, kThreads, 0, st>>>(n, perm, iperm, r.deg_r, st_dev);
    e = exclusive_scan_i64(r.deg_r, n, off_r, r.sums, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t degree_hist(int64_t n, const int64_t* off, unsigned long long* hist, int sms, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * (kMaxMidDeg + 2), st);
    if (e == cudaSuccess && n > 0) {
        k_degree_hist<<<sms * 4, kThreads, 0, st>>>(n, off, hist);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t map_seeds(uint64_t* seeds, int64_t count, const int32_t* iperm, cudaStream_t st) {
    if (count > 0)
        k_map_seeds<<<(unsigned)std::min<int64_t>((count + kThreads - 1) / kThreads, 1024), kThreads, 0, st>>>(seeds, count,
                                                                                                           iperm);
    return cudaGetLastError();
}

cudaError_t relabel_adjacency(int64_t n, int64_t n_big, int64_t n_mid, int64_t n_small, const int32_t* d_perm,
                              const int32_t* d_iperm, const int64_t* d_off, const int32_t* d_adj, const int64_t* d_off_r,
                              int32_t* d_adj_r, int sms, cudaStream_t st) {
    // ranks: [0, n_big) big, then mid, then small, then isolated
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) < n) bits++;
    const int shift = std::max(0, bits - 8);
    if (n_big > 0)
        k_relabel_big<<<(unsigned)std::min<int64_t>(n_big, (int64_t)sms * 8), kThreads, 0, st>>>(
            0, n_big, shift, d_perm, d_iperm, d_off, d_adj, d_off_r, d_adj_r);
    if (n_mid > 0)
        k_relabel_mid<<<(unsigned)std::min<int64_t>(n_mid, (int64_t)sms * 8), kThreads, 0, st>>>(
            n_big, n_big + n_mid, d_perm, d_iperm, d_off, d_adj, d_off_r, d_adj_r);
    if (n_small > 0) {
        const int64_t blocks = std::min<int64_t>((n_small + 127) / 128, (int64_t)sms * 16);
        k_relabel_small<<<(unsigned)blocks, 128, 0, st>>>(n_big + n_mid, n_big + n_mid + n_small, d_perm, d_iperm,
                                                          d_off, d_adj, d_off_r, d_adj_r);
    }
    (void)n;
    return cudaGetLastError();
}

}  // namespace cbfs
