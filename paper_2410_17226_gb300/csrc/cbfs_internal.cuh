// Internal declarations shared by the CUDA translation units of libcbfs.so.
// Nothing here is part of the public C ABI (include/cbfs.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "cbfs.h"

namespace cbfs {

constexpr int kThreads = 256;       // threads per CTA of every traversal kernel
constexpr int kWarps = kThreads / 32;
constexpr int kMaxSlots = 8;        // clusters in flight per wave: P in {1, 2, 4, 8}
constexpr int kStageAuto = 96;      // round records kept by default (memory permitting)
constexpr int kMaxRounds = 288;     // > 254 + 15 + 1: Delta < 255, offsets <= 15
constexpr int64_t kBigDeg = 2048;   // push: longer lists are cut into pieces of this size
constexpr int64_t kPullSmall = 32;  // pull: thread per vertex up to this degree
constexpr int64_t kPullMid = 2048;  // pull: warp per vertex up to this degree, CTA above
                                    // (both are defaults: a call may set its own, see cbfs_tune_t)
constexpr int kMaxMidDeg = 65536;   // largest warp-per-vertex threshold a call may ask for
constexpr int kDefaultMidDeg = 16384;  // a call's default: warps beat 2048-arc CTA pieces up to
                                       // about this degree on power-law graphs (measured)
constexpr int kZeroWords = 4;       // a slot's subset words are zeroed at its first visit up to
                                    // this d (one 32-byte sector); above it a mask records the
                                    // words written
constexpr int kTileMin = kThreads;  // smallest phase-A tile (P >= 4)
constexpr int kTileMax = 4 * kThreads;

// Phase-A tiling for P clusters in flight: entries per thread and per tile.
template <int P>
struct Geo {
    static constexpr int kEpt = P >= 4 ? 1 : 4 / P;
    static constexpr int kTile = kThreads * kEpt;
};

// One cluster in flight: where its outputs go.
// One 64-bit slot word of a wave.  Unpacked: one cluster, its sources in the
// k low bits, its outputs here.  Packed (the wave's nmembers > 0): several
// clusters, described by the wave's member table; dist and masks are unused,
// cluster is the word's first member (wave-local index) and pad its count.
struct SlotDesc {
    uint8_t* dist;    // output Delta_v, doubles as the "first round" state
    uint64_t* masks;  // output S_v[0..d-1]
    uint64_t all;     // the word's source bits (packed: the union of its members' bits)
    int32_t cluster;
    int32_t pad;
};

// A cluster packed into a slot word with others (packed waves): its sources
// are bits [off, off + k) of word `word`; its outputs are dist / masks.
struct MemberDesc {
    uint8_t* dist;
    uint64_t* masks;
    uint64_t mask;  // its bits in the word: ((1 << k) - 1) << off
    int32_t off;
    int32_t word;
};
constexpr int kWordMembers = 31;  // clusters per slot word at most (a wave's members fit a byte index)

// Per-round control block, zeroed at the start of every wave.
struct RoundCtl {
    unsigned long long qlen;   // queue entries (vertices) of F_i, appended during round i-1
    unsigned long long nf;     // entries that carried new sources in some slot (phase A)
    unsigned long long sdeg;   // sum of deg(u) over the queue entries, added by their producers
    unsigned int npieces;      // big-list pieces written by phase A
    unsigned int nbig;         // big-list entries written by phase A
    unsigned int tile_ctr;     // phase-B work counters
    unsigned int piece_ctr;
    unsigned int slot_active;  // bit s: slot s has a non-empty frontier this round
    int mode;                  // 0 push, 1 pull: decided by phase A from qlen and sdeg
    int dense;                 // 1: F_i was produced by a pull round and is not in the queue;
                               //    phase A finds it by scanning every vertex's acc block
    int fused;                 // 1: that pull did F_i's vertex phase (new sources in nw[i & 1])
};

// A frontier vertex whose list is longer than kBigDeg (push mode).
struct BigEntry {
    int64_t ost;  // off[u]
    int64_t deg;
};

// Everything a traversal kernel needs, passed by value.
//
// Vertex-major state of the P clusters in flight:
//   vis[v*P + s] = sources of slot s seen at rounds <= the current one
//                  (Sseen of Algorithm 1);
//   acc[v*P + s] = sources pushed to v for the next round and not yet
//                  consumed (the part of Snext not in Sseen).
// One adjacency scan and one gathered vis block serve all P clusters.
struct Wave {
    int64_t n, nnz;
    const int64_t* off;
    const int32_t* adj;
    int d;
    int P;                  // slots per vertex block (template P of the phase kernels)
    int nslots;             // slot words in use in this wave (<= P)
    const SlotDesc* slots;  // device [nslots]
    uint64_t* vis;          // [n][P]
    uint64_t* acc;          // [n][P]
    uint64_t* nw0;          // [n][P] sources new at v in round i, for i even / odd: written by
    uint64_t* nw1;          //   the vertex phase of v (in phase A, or in the pull of round i-1)
                            //   and gathered by the pull of round i of a fused wave; cleared per
                            //   wave, except in waves with round records (hcap > 0), which
                            //   gather from the record of a recorded round and use nw only
                            //   past them, always through the frontier bitmap
    uint32_t* piece_cnt;    // [n] pull pieces of a hub done this round (the last one resets it)
    uint32_t* rq;           // [n] queue claim stamps: F_i holds v iff rq[v] was set to i+1
    uint32_t* q0;           // frontier queues of vertex ids
    uint32_t* q1;
    uint32_t* fb0;          // frontier bitmaps, F_i in fb[i & 1]: bit v set iff v carries new
    uint32_t* fb1;          //   sources in round i (pull gathers only from those neighbours)
    RoundCtl* ctl;          // [kMaxRounds]
    uint32_t* t_pre;        // tile lists (compacted per tile): tile-local arc prefix
    int64_t* t_ost;         //   off[u]
    uint64_t* t_fw;         //   [entry][P] sources new at u this round
    uint32_t* tile_cnt;     // entries per tile
    uint32_t* tile_arcs;    // arcs per tile
    BigEntry* big;
    uint64_t* big_fw;       // [entry][P]
    uint32_t* piece_ent;    // piece p covers arcs [piece_no*kBigDeg, ...) of big[piece_ent]
    uint32_t* piece_no;
    const uint64_t* pull_pieces;  // pull: (vertex << 32 | piece) for every kBigDeg-arc piece
    int64_t n_pull_pieces;        //   of every vertex above the warp class
    // pull rounds with a sparse frontier (qlen < n/32) use these classes instead when
    // n_big_s >= 0 (a call's sparse_mid_deg; off by default)
    int64_t n_small_s, n_mid_s, n_big_s;
    const uint64_t* pull_pieces_s;
    int64_t n_pull_pieces_s;
    int64_t n_small, n_mid, n_big;
    const int32_t* perm;    // internal vertex -> caller's id for the outputs (nullptr: identity)
    uint8_t* dist_r;        // [n][P] Delta rows of the wave in internal order, emitted to the
    uint64_t* masks_r;      // [n][P][d] caller's arrays after the wave; nullptr: the vertex
                            // phase writes each slot's output directly at perm[u] (waves with
                            // fused pulls, and the allocation-free entry point)
    uint16_t* wmask_r;      // [n][P] bit j: masks_r word j of the slot was written in this
                            // wave (started at the slot's first visit; never cleared)
    uint64_t* hist;         // [hcap][n][P] round records of waves without rows: hist[i][u] =
                            // the sources new at u in round i, valid iff bit u of fbh[i] is set
    uint32_t* fbh;          // [hcap][bitmap words] F_i's bitmap, copied by phase A of round i
    int hcap;               // rounds recorded (0: none, outputs written directly as they arise)
    const MemberDesc* members;  // packed waves: the clusters of the wave, word by word
    const uint8_t* bit_member;  // [P][64] member of each bit of each word (0xFF: none)
    int nmembers;           // 0: one cluster per slot word (the slot's own outputs)
    int dense_div;          // the vertex phase scans every vertex when qlen * dense_div > n
    int grid_a;             // CTAs of the vertex phase (0: the edge phase's grid)
    int fused_pull;         // 1: pull rounds do their vertices' vertex phase on the spot
                            //    (vis, rows, nw; nw cleared per wave); 0: plain pulls
    int* round_dev;         // graph mode: the current round lives here (nullptr: kernel argument)
    unsigned long long* iters;  // graph mode: rounds executed (for the launch accounting)
    int* status;
    float alpha;            // pull threshold factor (<= 0: push only)
};

// Scratch capacities for n vertices and P slots (entries of each array).
struct ScratchSizes {
    int64_t state, queue, list, tiles, bitmap;
};
inline ScratchSizes scratch_sizes(int64_t n, int P) {
    ScratchSizes z;
    z.state = n * P;
    z.queue = n;
    z.list = n + kTileMax;                   // tile slots: ntiles * tile <= n + tile - 1
    z.tiles = (n + kTileMin - 1) / kTileMin + 1;
    z.bitmap = (n + 31) / 32 + 1;
    return z;
}

__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, 0, code); }

// Traversal kernels (cbfs_core.cu).  seeds[i] = member << 48 | slot << 40 |
// j << 32 | vertex (j: the source's bit in the slot word; member: the index
// of its cluster in a packed wave's member table).
__global__ void k_seed(Wave w, const uint64_t* seeds, int count);
__global__ void k_check_sources(Wave w, const uint64_t* seeds, int count, int bound_round, int* unfinished);
template <int P>
__global__ void k_phase_a(Wave w, int round);
template <int P, bool FUSE>  // FUSE: the call's fused_pull
__global__ void k_phase_b(Wave w, int round);
// Writes the wave's internal rows to the caller's cluster-major outputs.
template <int P>
__global__ void k_emit(Wave w, const int32_t* iperm);
// Writes the outputs of a wave with round records (hcap > 0) from them:
// at_cap != 0 after phase A of round hcap - 1 (later rounds write their
// outputs directly), else after the wave when it ended before that round.
template <int P>
__global__ void k_flush(Wave w, const int32_t* iperm, int round, int at_cap, int bound_round);
// The same for packed waves (nmembers > 0): each member's outputs from its bits.
template <int P>
__global__ void k_flush_packed(Wave w, const int32_t* iperm, int round, int at_cap, int bound_round);

// Internal vertex order (cbfs_relabel.cu), computed on the device: ranks by
// degree, highest first, ties to the smaller id; perm[rank] = id,
// iperm[id] = rank, off_r = offsets of the relabelled CSR.
struct DegreeStats {
    unsigned long long n_small, n_mid, n_big;  // non-isolated vertices by degree class (kPullSmall, kPullMid)
    unsigned long long big_pieces;             // kBigDeg-arc pieces of the lists longer than kBigDeg
    unsigned long long maxdeg;
    unsigned long long bad;                    // offsets not starting at 0, not ending at nnz, or decreasing
    unsigned long long forward;                // graph check: arcs towards a later rank (half of all)
    unsigned long long order_bad;              // the rank order failed its check (never expected)
};
cudaError_t widen_offsets(const int32_t* in, int64_t* out, int64_t count, int sms, cudaStream_t st);
int64_t rank_scratch_words(int64_t n);
uint32_t* rank_keys(int64_t n, int64_t* scratch);
// Checks the offsets, fills st_dev and writes the sort keys into the scratch.
cudaError_t degree_stats(int64_t n, int64_t nnz, const int64_t* off, DegreeStats* st_dev, uint32_t* keys, int sms,
                         cudaStream_t st);
// Also checks its result into st_dev->order_bad.
cudaError_t rank_order_device(int64_t n, const int64_t* off, uint64_t maxdeg, int64_t* scratch, int32_t* perm,
                              int32_t* iperm, int64_t* off_r, DegreeStats* st_dev, int sms, cudaStream_t st);
// Exclusive scan of count int64 values into out[0..count] (out[count] = total);
// in == out is allowed.  sums: tile sums, (count + 4095) / 4096 entries.
cudaError_t exclusive_scan_i64(const int64_t* in, int64_t count, int64_t* out, int64_t* sums, cudaStream_t st);
// Vertices of each degree 0..kMaxMidDeg, and above it in hist[kMaxMidDeg + 1].
cudaError_t degree_hist(int64_t n, const int64_t* off, unsigned long long* hist, int sms, cudaStream_t st);
// Seeds hold callers' ids in their low 32 bits: rewrite them as ranks.
cudaError_t map_seeds(uint64_t* seeds, int64_t count, const int32_t* iperm, cudaStream_t st);
// Writes the relabelled adjacency (ranks, hubs first) of the ranks
// [0, n_big) (degree > kPullMid), then n_mid, then n_small vertices.
cudaError_t relabel_adjacency(int64_t n, int64_t n_big, int64_t n_mid, int64_t n_small, const int32_t* d_perm,
                              const int32_t* d_iperm, const int64_t* d_off, const int32_t* d_adj, const int64_t* d_off_r,
                              int32_t* d_adj_r, int sms, cudaStream_t st);

// Read-only view of a resident graph's relabelled CSR (cbfs_core.cu), for
// kernels outside the traversal (the local search of queries).
struct GraphView {
    int64_t n;
    const int64_t* off;   // relabelled offsets [n + 1]
    const int32_t* adj;   // relabelled adjacency (ranks)
    const int32_t* iperm; // caller's id -> rank
    int device;
};
int graph_view(const cbfs_graph_s* g, GraphView* out);
int* graph_status(cbfs_graph_s* g);  // the handle's device status word

// Label store (cbfs_labels.cu) fed by a batched run: reserve C rows' worth of
// clusters at the store's count (uploads their ALL words), write nc clusters
// of cluster-major outputs at position pos, or undo a reservation.
int labels_reserve(cbfs_labels_s* L, int64_t n, int d, const int32_t* coff, int C, int* base, cudaStream_t st);
cudaError_t labels_write(cbfs_labels_s* L, const uint8_t* dist, const uint64_t* masks, int nc, int pos,
                         cudaStream_t st);
void labels_rollback(cbfs_labels_s* L, int base);

// Launches phase A (which = 0), phase B (1) of one round, or the emit
// kernel (2) for w.P (1, 2, 4 or 8).
cudaError_t launch_round(const Wave& w, int round, int grid, cudaStream_t st, int which, const int32_t* iperm = nullptr);
// Launches k_flush for the wave (see there).
cudaError_t launch_flush(const Wave& w, int round, int grid, cudaStream_t st, int at_cap, int bound_round,
                         const int32_t* iperm);

// Stream-ordered calls leave device-detected errors in their owner's status
// word (a graph handle's or a label store's); cbfs_sync_status(stream) reads
// and clears the words registered for that stream.  status_forget drops an
// owner's entries when it is destroyed.  (cbfs_core.cu)
void status_register(cudaStream_t st, int* word, const void* owner);
void status_forget(const void* owner);

}  // namespace cbfs

// Implemented in cbfs_core.cu; used by cbfs_labels.cu.
extern "C" const char* cbfs_status_string(int status);
