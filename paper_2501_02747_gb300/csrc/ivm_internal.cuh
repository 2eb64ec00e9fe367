// ivm_internal.cuh -- device data layouts and launcher declarations shared by
// the library's translation units.  Nothing here is part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ivm.h"

namespace ivm {

constexpr int kMaxSamplesPerSide = 8;
constexpr int kCoordLimit = 1 << 22;       // |scaled coordinate| < 2^22
constexpr int kStackDepth = 64;            // keys are unique 64-bit: depth <= 64

// Device error word values are the public IVM_ERR_* codes.  The first error
// raised in a call wins (atomicCAS from 0).
__device__ __forceinline__ void raise_error(int *err, int code) { atomicCAS(err, 0, code); }

// One facet as the traversal sees it (64 bytes, read by all lanes at once).
// All coordinates are scaled by 2s.  n is u x v divided by the gcd of its
// components (same direction, small magnitude): facing and plane-side tests
// only need its sign pattern.
struct __align__(16) Leaf {
    int ox, oy, oz, building;   // origin O = 2s o
    int ux, uy, uz, scene;      // edge U = 2s u
    int vx, vy, vz, dom;        // edge V = 2s v; dom: bits 0-1 the dominant axis of n,
                                // bit 2 set when U and V lie along two different axes
    int nx, ny, nz, pad;        // reduced outward normal; pad = Morton-sorted position
};

// Internal BVH node: the boxes of both children (closed, float holding exact
// integers) and their references.  A reference r >= 0 is an internal node
// (scene-local index + the scene's node offset); r < 0 is a leaf, facet ~r
// (global facet index).
struct __align__(16) Node {
    float4 a;   // lo_L.x lo_L.y lo_L.z hi_L.x
    float4 b;   // hi_L.y hi_L.z lo_R.x lo_R.y
    float4 c;   // lo_R.z hi_R.x hi_R.y hi_R.z
    int4 d;     // child_L child_R; first and last Morton-sorted position covered
};

// Per-scene descriptor (device copy).
struct SceneDesc {
    int facet0;       // first global facet index
    int n;            // facets
    int W;            // words per bit row
    int node0;        // first global internal-node index (n - 1 nodes)
    int root;         // node reference of the root
    int s;            // samples per side
    int sample0;      // first global sample index (n * s * s samples)
    int ntiles;       // table: tiles of consecutive snapshots, ceil(nsnap / tile)
    long long item0;  // table: first work item; the scene has 2 * W * ntiles items
    long long rw0;    // first (row, word) index of this scene: n * W of them
    long long los0;   // first 32-snapshot LoS chunk of this scene
    uint32_t *matrix; // output rows [n][W]
    const int *tx;    // [S][3] cm (table only)
    const int *rx;
    uint32_t *table;  // [S][2][W]
    uint8_t *los;     // [S]
    long long snap0;  // first index of this scene in the global snapshot space
    long long nsnap;
    int row_lo;       // matrix: only pairs (i, j), i < j, with row_lo <= i < row_hi
    int row_hi;
    int budget;       // steps of one BVH walk before IVM_ERR_TIMEOUT (>= 2n - 1 suffices)
};

// Device counters (u64), summed into ivm_stats.
enum Counter {
    C_SEGMENTS = 0,
    C_NODE_TESTS,
    C_LEAF_TESTS,
    C_UNDECIDED,
    C_EXACT_TESTS,
    C_RANKER_HITS,
    C_CAND_PAIRS,
    C_CACHE_HITS,
    C_DEDUP_ROWS,
    C_RANKER_HITS8,
    C_COUNT_
};

// Geometry of all scenes of a call, in the context's scratch.
struct DevScenes {
    int n_scenes;
    int total_facets;
    int total_nodes;         // sum of max(n - 1, 0)
    int total_samples;
    SceneDesc *desc;         // [n_scenes]
    const ivm_facet *facets; // [total_facets] raw input (device)
    Leaf *leaf;              // [total_facets]
    int *fscene;             // [total_facets] scene of each facet
    int *box;                // [total_facets][6] scaled int AABB lo xyz, hi xyz
    int *sx, *sy, *sz;       // [total_samples] scaled sample points
    int max_n;               // largest scene
    unsigned long long *keys;// [total_facets] sort keys
    unsigned long long *sorted; // [total_facets] keys in Morton order per scene
    int *bounds;             // [n_scenes][6] centroid bounds (lo + hi units)
    int *order;              // [total_facets] facet of each sorted key (global)
    Node *nodes;             // [total_nodes]
    int *parent;             // [total_facets + total_nodes] parent of leaf / node
    int *visits;             // [total_nodes] refit arrival counters
};

// ---------------------------------------------------------------- launchers
// Host-side count of kernels this library has launched (all threads).
void note_launches(int n);

// Each enqueues on `st` and returns cudaGetLastError().
cudaError_t launch_ingest(const DevScenes &g, int *err, cudaStream_t st);
cudaError_t launch_bvh(const DevScenes &g, cudaStream_t st);
cudaError_t launch_screen_count(const DevScenes &g, const SceneDesc *host_desc,
                                unsigned long long *count, cudaStream_t st);
cudaError_t launch_screen_emit(const DevScenes &g, const SceneDesc *host_desc, int2 *pairs,
                               unsigned long long *cursor, unsigned long long cap,
                               cudaStream_t st);

// Launch shape of the traversal kernels.
// Learned form: per candidate pair the top-8 proposed clusters (one byte
// each, best first), the per-scene cluster context and the cut-node marks.
struct LearnedDev {
    const unsigned long long *ranks = nullptr;
    const int *ctx = nullptr;
    const signed char *ncl = nullptr;
};

struct LaunchCfg {
    int mode;             // IVM_MODE_*
    int persistent;       // work queue over a grid of n_sm * blocks_per_sm blocks
    int warps_per_block;  // 1..16
    int tile;             // work items taken per queue pop (persistent)
    int n_sm;
    int cache;            // occluder cache in front of the BVH walk
    int dedup;            // table: compute one row per run of equal source positions
    int aligned = 0;      // filtered forms: exact test for axis-aligned rectangle facets
    int proof_tile = 32;  // table: snapshots per straight-stretch proof
    int corner = 1;       // matrix: try the corner proof before the packets
    const unsigned long long *count_dev = nullptr;  // matrix, persistent: device pair count
    LearnedDev learn;     // matrix, learned form (ranks == nullptr: off)
    void *steal = nullptr;// table, persistent: 16-byte slots, 64 per SM (nullptr: no splitting)
};

// Measured FP32 FMA lane operations per second (peak.cu).
cudaError_t ffma_peak(int n_sm, float *sink, cudaStream_t st, double *lane_ops_per_s);

cudaError_t launch_matrix(const DevScenes &g, const int2 *pairs, unsigned long long npairs,
                          const LaunchCfg &cfg, unsigned long long *work,
                          unsigned long long *ctr, int *err, cudaStream_t st);
cudaError_t launch_table(const DevScenes &g, long long total_snap, long long total_items,
                         long long total_los_chunks, int snap_tile, const LaunchCfg &cfg,
                         int *rep, unsigned long long *work, unsigned long long *ctr, int *err,
                         cudaStream_t st);

}  // namespace ivm
