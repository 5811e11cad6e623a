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

namespace cbfs {

void rank_order(int64_t n, const int64_t* h_off, std::vector<int32_t>& perm, std::vector<int32_t>& iperm,
                std::vector<int64_t>& off_r) {
    int64_t maxdeg = 0;
    for (int64_t v = 0; v < n; ++v) maxdeg = std::max(maxdeg, h_off[v + 1] - h_off[v]);
    // counting sort by degree, descending; ascending ids within a degree
    std::vector<int64_t> start((size_t)maxdeg + 2, 0);
    for (int64_t v = 0; v < n; ++v) start[(size_t)(maxdeg - (h_off[v + 1] - h_off[v])) + 1]++;
    for (size_t b = 1; b < start.size(); ++b) start[b] += start[b - 1];
    perm.assign((size_t)n, 0);
    iperm.assign((size_t)n, 0);
    for (int64_t v = 0; v < n; ++v) {
        const int64_t r = start[(size_t)(maxdeg - (h_off[v + 1] - h_off[v]))]++;
        perm[(size_t)r] = (int32_t)v;
        iperm[(size_t)v] = (int32_t)r;
    }
    off_r.assign((size_t)n + 1, 0);
    for (int64_t r = 0; r < n; ++r) off_r[(size_t)r + 1] = off_r[(size_t)r] + (h_off[perm[r] + 1] - h_off[perm[r]]);
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
