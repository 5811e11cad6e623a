// Internal declarations shared by the CUDA translation units of libcbfs.so.
// Nothing here is part of the public C ABI (include/cbfs.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cbfs.h"

namespace cbfs {

constexpr int kThreads = 256;                  // threads per CTA of every traversal kernel
constexpr int kWarps = kThreads / 32;
constexpr int kTile = 1024;                    // frontier entries per phase-A tile
constexpr int kPerThread = kTile / kThreads;   // entries per thread in a tile
constexpr int kMaxSlots = 16;                  // clusters in flight per wave
constexpr int kMaxRounds = 288;                // > 254 + 15 + 1: Delta < 255, offsets <= 15
constexpr int64_t kBigDeg = 2048;              // push: longer lists are cut into pieces of this size
constexpr int64_t kPullSmall = 32;             // pull: thread per vertex up to this degree
constexpr int64_t kPullMid = 2048;             // pull: warp per vertex up to this degree, CTA above

// One cluster in flight.  va[v] = {visit, acc}: visit = sources seen at rounds
// <= the current one (Sseen of Algorithm 1), acc = sources pushed to v for
// the next round and not yet consumed (the part of Snext not in Sseen).
struct SlotDesc {
    ulonglong2* va;
    uint8_t* dist;    // output Delta_v, doubles as the "first round" state
    uint64_t* masks;  // output S_v[0..d-1]
    uint64_t all;     // the k low bits
    int32_t cluster;
    int32_t pad;
};

// Per-round control block, zeroed at the start of every wave.
struct RoundCtl {
    unsigned long long qlen;   // queue entries of F_i (appended during round i-1)
    unsigned long long nf;     // entries that carried new sources (|F_i| over all slots)
    unsigned long long sdeg;   // sum of deg(u) over those entries
    unsigned int npieces;      // big-list pieces written by phase A
    unsigned int nbig;         // big-list entries written by phase A
    unsigned int tile_ctr;     // phase-B work counters
    unsigned int piece_ctr;
    unsigned int slot_active;  // bit s: slot s has a non-empty frontier this round
    int mode;                  // 0 push, 1 pull (recorded by phase B)
    unsigned int pad[2];
};

// A frontier vertex whose list is longer than kBigDeg (push mode).
struct BigEntry {
    int64_t ost;  // off[u]
    int64_t deg;
    uint64_t fw;  // the sources new at u this round
    int32_t slot;
    int32_t pad;
};

// Everything a traversal kernel needs, passed by value.
struct Wave {
    int64_t n, nnz;
    const int64_t* off;
    const int32_t* adj;
    int d;
    int nslots;
    const SlotDesc* slots;  // device [nslots]
    uint64_t* q0;           // frontier queues, entry = slot << 32 | v
    uint64_t* q1;
    RoundCtl* ctl;          // [kMaxRounds]
    uint32_t* t_pre;        // tile lists (compacted per tile): tile-local arc prefix
    int64_t* t_ost;         //   off[u]
    uint64_t* t_fw;         //   new sources of u
    uint8_t* t_slot;        //   slot
    uint32_t* tile_cnt;     // entries per tile
    uint32_t* tile_arcs;    // arcs per tile
    BigEntry* big;
    uint32_t* piece_ent;    // piece p covers arcs [piece_no*kBigDeg, ...) of big[piece_ent]
    uint32_t* piece_no;
    const int32_t* pl_small;  // pull lists: vertices by degree class, ascending ids
    const int32_t* pl_mid;
    const int32_t* pl_big;
    int64_t n_small, n_mid, n_big;
    int* status;
    float alpha;            // pull threshold factor (<= 0: push only)
};

__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, 0, code); }

// Traversal kernels (cbfs_core.cu).  seeds[i] = slot << 40 | j << 32 | vertex.
__global__ void k_seed(Wave w, const uint64_t* seeds, int count);
__global__ void k_check_sources(Wave w, const uint64_t* seeds, int count);
__global__ void k_phase_a(Wave w, int round);
__global__ void k_phase_b(Wave w, int round);

}  // namespace cbfs

// Implemented in cbfs_core.cu; used by cbfs_labels.cu.
extern "C" const char* cbfs_status_string(int status);
