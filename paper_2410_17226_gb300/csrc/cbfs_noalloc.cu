// libcbfs.so, part 3: cbfs_run_noalloc, the C-BFS entry point that allocates
// nothing.
//
// Who needs it: callers that must not allocate device memory -- a process
// whose device memory is entirely held by another allocator (for instance a
// framework's caching pool sized to the whole GPU), or a latency-critical
// loop where cudaMalloc / cudaFree (which can block and synchronise the
// device) are not allowed.  Such callers pass the graph and the outputs in
// memory they already own; the traversal's scratch comes from one fixed
// array compiled into this file.
//
// The array below is a file-scope __device__ variable: every GPU that loads
// this module keeps it (kNoAllocBytes, about 7 MB) until the process exits.
// Host code must not use its name as a device address; the entry point looks
// the address up with cudaGetSymbolAddress once per device, on the first call
// made with that device current.  All calls share the array and it keeps the
// last call's contents, so every call clears what must start at zero, and
// calls that overlap on the GPU (other streams, other host threads) race.
#include <cstring>
#include <mutex>

#include "cbfs_internal.cuh"

using namespace cbfs;

namespace {

constexpr int64_t kNoAllocMaxN = (int64_t)1 << 17;    // 131,072 vertices
constexpr int64_t kNoAllocMaxNnz = (int64_t)1 << 22;  // 4,194,304 arcs
constexpr int64_t kListMax = kNoAllocMaxN + kTileMax;
constexpr int64_t kTilesMax = (kNoAllocMaxN + kTileMin - 1) / kTileMin + 1;
constexpr int64_t kBigMax = kNoAllocMaxNnz / (kBigDeg + 1) + 1;      // vertices of degree > kBigDeg
constexpr int64_t kPiecesMax = kNoAllocMaxNnz / kBigDeg + kBigMax;   // their kBigDeg-arc pieces
constexpr int kMaxDevices = 64;

constexpr int64_t al256(int64_t x) { return (x + 255) / 256 * 256; }

// byte offsets of the pieces of the scratch array (one cluster in flight)
constexpr int64_t kOffVis = 0;
constexpr int64_t kOffAcc = kOffVis + al256(8 * kNoAllocMaxN);
constexpr int64_t kOffRq = kOffAcc + al256(8 * kNoAllocMaxN);
constexpr int64_t kOffQ0 = kOffRq + al256(4 * kNoAllocMaxN);
constexpr int64_t kOffQ1 = kOffQ0 + al256(4 * kNoAllocMaxN);
constexpr int64_t kBitmapWords = (kNoAllocMaxN + 31) / 32 + 1;
constexpr int64_t kOffFb = kOffQ1 + al256(4 * kNoAllocMaxN);
constexpr int64_t kOffPre = kOffFb + al256(8 * kBitmapWords);
constexpr int64_t kOffOst = kOffPre + al256(4 * kListMax);
constexpr int64_t kOffFw = kOffOst + al256(8 * kListMax);
constexpr int64_t kOffTileCnt = kOffFw + al256(8 * kListMax);
constexpr int64_t kOffTileArcs = kOffTileCnt + al256(4 * kTilesMax);
constexpr int64_t kOffBig = kOffTileArcs + al256(4 * kTilesMax);
constexpr int64_t kOffBigFw = kOffBig + al256((int64_t)sizeof(BigEntry) * kBigMax);
constexpr int64_t kOffPieceEnt = kOffBigFw + al256(8 * kBigMax);
constexpr int64_t kOffPieceNo = kOffPieceEnt + al256(4 * kPiecesMax);
constexpr int64_t kOffCtl = kOffPieceNo + al256(4 * kPiecesMax);
constexpr int64_t kOffSlots = kOffCtl + al256((int64_t)sizeof(RoundCtl) * kMaxRounds);
constexpr int64_t kOffSeeds = kOffSlots + al256((int64_t)sizeof(SlotDesc));
constexpr int64_t kOffStatus = kOffSeeds + al256(8 * 64);
constexpr int64_t kNoAllocBytes = kOffStatus + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_setup_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {};
int g_grid[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once).
int scratch_for_device(int dev, unsigned char** out, int* grid) {
    if (dev < 0 || dev >= kMaxDevices) return CBFS_E_INVALID;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return CBFS_E_CUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return CBFS_E_CUDA;
        g_grid[dev] = sms * 4;
        g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[dev];
    *grid = g_grid[dev];
    return CBFS_OK;
}

// The caller's CSR is checked before any traversal kernel reads it through
// its offsets: off[0] = 0, off[n] = nnz, offsets never decrease, every id in
// [0, n).  Each read stays inside off[0..n] and adj[0..nnz), the sizes the
// caller states.  The first failure writes CBFS_E_GRAPH to the status word.
__global__ void k_noalloc_check(int64_t n, const int64_t* off, const int32_t* adj, int64_t nnz, int* status) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool ok = true;
    if (tid == 0) ok = off[0] == 0 && off[n] == nnz;
    for (int64_t v = tid; v < n; v += stride) ok &= off[v] <= off[v + 1];
    for (int64_t e = tid; e < nnz; e += stride) {
        const int32_t u = adj[e];
        ok &= u >= 0 && (int64_t)u < n;
    }
    if (!ok) set_status(status, CBFS_E_GRAPH);
}

}  // namespace

extern "C" int cbfs_run_noalloc(int64_t n, const int64_t* off, const int32_t* adj, int64_t nnz,
                                const int32_t* host_sources, int k, int d, uint8_t* dist, uint64_t* masks,
                                void* stream) {
    if (!off || !host_sources || !dist || (d > 0 && !masks) || (nnz > 0 && !adj)) return CBFS_E_INVALID;
    if (n < 1 || nnz < 0 || k < 1 || k > 64 || d < 0 || d > 15) return CBFS_E_INVALID;
    if (n > kNoAllocMaxN || nnz > kNoAllocMaxNnz) return CBFS_E_NOMEM;  // beyond the fixed scratch
    for (int j = 0; j < k; ++j) {
        if (host_sources[j] < 0 || (int64_t)host_sources[j] >= n) return CBFS_E_INVALID;
        for (int i = 0; i < j; ++i)
            if (host_sources[i] == host_sources[j]) return CBFS_E_INVALID;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CBFS_E_CUDA;
    unsigned char* base = nullptr;
    int grid = 0;
    int rc = scratch_for_device(dev, &base, &grid);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    Wave w;
    memset(&w, 0, sizeof(w));
    w.n_big_s = -1;  // push only: no pull classes
    w.n = n;
    w.nnz = nnz;
    w.off = off;
    w.adj = adj;
    w.d = d;
    w.P = 1;
    w.nslots = 1;
    w.slots = reinterpret_cast<const SlotDesc*>(base + kOffSlots);
    w.vis = reinterpret_cast<uint64_t*>(base + kOffVis);
    w.acc = reinterpret_cast<uint64_t*>(base + kOffAcc);
    w.rq = reinterpret_cast<uint32_t*>(base + kOffRq);
    w.q0 = reinterpret_cast<uint32_t*>(base + kOffQ0);
    w.q1 = reinterpret_cast<uint32_t*>(base + kOffQ1);
    w.fb0 = reinterpret_cast<uint32_t*>(base + kOffFb);
    w.fb1 = w.fb0 + kBitmapWords;
    w.ctl = reinterpret_cast<RoundCtl*>(base + kOffCtl);
    w.t_pre = reinterpret_cast<uint32_t*>(base + kOffPre);
    w.t_ost = reinterpret_cast<int64_t*>(base + kOffOst);
    w.t_fw = reinterpret_cast<uint64_t*>(base + kOffFw);
    w.tile_cnt = reinterpret_cast<uint32_t*>(base + kOffTileCnt);
    w.tile_arcs = reinterpret_cast<uint32_t*>(base + kOffTileArcs);
    w.big = reinterpret_cast<BigEntry*>(base + kOffBig);
    w.big_fw = reinterpret_cast<uint64_t*>(base + kOffBigFw);
    w.piece_ent = reinterpret_cast<uint32_t*>(base + kOffPieceEnt);
    w.piece_no = reinterpret_cast<uint32_t*>(base + kOffPieceNo);
    w.status = reinterpret_cast<int*>(base + kOffStatus);
    w.alpha = -1.f;  // push only: the dense edge phase needs degree-class lists this variant does not keep
    w.dist_r = nullptr;  // direct: the vertex phase writes the caller's arrays
    w.masks_r = nullptr;
    w.dense_div = 16;

    SlotDesc sd;
    memset(&sd, 0, sizeof(sd));
    sd.dist = dist;
    sd.masks = d ? masks : nullptr;
    sd.all = (k >= 64) ? ~0ull : ((1ull << k) - 1ull);
    uint64_t seeds[64];
    for (int j = 0; j < k; ++j) seeds[j] = ((uint64_t)j << 32) | (uint32_t)host_sources[j];
    uint64_t* d_seeds = reinterpret_cast<uint64_t*>(base + kOffSeeds);

#define NA_CK(call)                          \
    do {                                     \
        if ((call) != cudaSuccess) {         \
            cudaGetLastError();              \
            return CBFS_E_CUDA;              \
        }                                    \
    } while (0)
    // pageable sources: both copies are staged before the calls return
    NA_CK(cudaMemcpyAsync(base + kOffSlots, &sd, sizeof(sd), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(d_seeds, seeds, sizeof(uint64_t) * k, cudaMemcpyHostToDevice, st));
    // everything the traversal expects to start at zero (the array keeps the last call's data)
    NA_CK(cudaMemsetAsync(w.vis, 0, 8 * (size_t)n, st));
    NA_CK(cudaMemsetAsync(w.acc, 0, 8 * (size_t)n, st));
    NA_CK(cudaMemsetAsync(w.rq, 0, 4 * (size_t)n, st));
    NA_CK(cudaMemsetAsync(w.fb0, 0, 8 * (size_t)kBitmapWords, st));
    NA_CK(cudaMemsetAsync(w.ctl, 0, sizeof(RoundCtl) * kMaxRounds, st));
    NA_CK(cudaMemsetAsync(w.status, 0, sizeof(int), st));
    // the graph is checked before the traversal reads through its offsets and ids
    k_noalloc_check<<<grid, kThreads, 0, st>>>(n, off, adj, nnz, w.status);
    NA_CK(cudaGetLastError());
    int status = 0;
    // to pageable memory: returns once the copy (and the check before it) is done
    NA_CK(cudaMemcpyAsync(&status, w.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    if (status) return status;
    NA_CK(cudaMemsetAsync(dist, 0xFF, (size_t)n, st));
    if (d) NA_CK(cudaMemsetAsync(masks, 0, sizeof(uint64_t) * (size_t)d * (size_t)n, st));
    k_seed<<<1, kThreads, 0, st>>>(w, d_seeds, k);
    NA_CK(cudaGetLastError());
    // Rounds are enqueued two at a time and the host looks at the frontier
    // after each pair: a round whose frontier is empty returns at once, so the
    // second round of the last pair costs two empty launches, and the host
    // waits once per two levels instead of once per level.
    bool done = false;
    for (int r = 0; r + 1 < kMaxRounds - 1; r += 2) {
        NA_CK(launch_round(w, r, grid, st, 0));
        NA_CK(launch_round(w, r, grid, st, 1));
        NA_CK(launch_round(w, r + 1, grid, st, 0));
        NA_CK(launch_round(w, r + 1, grid, st, 1));
        unsigned long long qn = 0;
        NA_CK(cudaMemcpyAsync(&qn, &w.ctl[r + 2].qlen, sizeof(qn), cudaMemcpyDeviceToHost, st));
        NA_CK(cudaStreamSynchronize(st));
        if (qn == 0) {
            done = true;
            break;
        }
    }
    if (!done) return CBFS_E_DEPTH;
    k_check_sources<<<1, kThreads, 0, st>>>(w, d_seeds, k, 0, nullptr);
    NA_CK(cudaGetLastError());
    NA_CK(cudaMemcpyAsync(&status, w.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
#undef NA_CK
    return status;
}
