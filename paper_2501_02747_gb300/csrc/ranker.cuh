// ranker.cuh -- learned occluder ranking (the learned form; not in the paper).
//
// A small MLP looks at a facet pair and proposes which of the scene's 64 BVH
// clusters to test first, so that blocked segments meet their occluder
// early.  It never decides a bit: a proposed cluster is walked with the same
// exact facet tests as every other, and the rest of the tree is walked after
// it.  Clusters are the subtrees of a cut through the scene's BVH: starting
// from the root, the node covering the most facets is replaced by its two
// children until there are 64 (or only leaves are left).  Each cluster is a
// contiguous range of the Morton-sorted facet order (every node's range is in
// Node.d.z / d.w); clusters are numbered by that order.  A proposal is walked
// from its own subtree root, so trying it costs no descent from the scene
// root, and the walk of the rest skips the subtrees already walked.
//
// Network: 76 inputs -> 128 -> 128 -> 128 (ReLU) -> 64 logits.  Inputs: the
// pair's two facet centroids normalised to the scene box (6), both unit
// normals (6), and per cluster the entry depth of the centroid-to-centroid
// segment into the cluster's box (1 - t_entry if it meets the box, else 0;
// 64).  Inference runs BF16 weights with FP32 accumulation on the 5th-generation
// tensor cores (tcgen05.mma, 128 pairs per tile, operands in shared memory,
// accumulators in tensor memory); training keeps FP32 master weights.
#pragma once

#include <cuda_bf16.h>

#include "traverse.cuh"

namespace ivm {

constexpr int kRIn = 76, kRInPad = 80, kRH = 128, kROut = 64, kRTop = 8;
constexpr int kRClusters = 64;

// FP32 master weights, row-major W[in][out], in one array (floats)
constexpr int kRW1 = 0, kRB1 = kRW1 + kRIn * kRH;
constexpr int kRW2 = kRB1 + kRH, kRB2 = kRW2 + kRH * kRH;
constexpr int kRW3 = kRB2 + kRH, kRB3 = kRW3 + kRH * kRH;
constexpr int kRW4 = kRB3 + kRH, kRB4 = kRW4 + kRH * kROut;
constexpr int kRParams = kRB4 + kROut;   // 51,136

// BF16 inference copy for the tensor cores: each layer's W^T[out][in] (the
// B operand, N = out rows, K = in columns) in the canonical K-major layout of
// tcgen05.mma without swizzling: 8 x 8 core matrices of 128 contiguous bytes
// (8 rows of 16 bytes), core matrices along K 128 bytes apart, 8-row groups
// K / 8 core matrices apart.  Layer 1's K is the 76 inputs padded to 80.
// FP32 biases are read from the master weights.
constexpr int kRK1 = 80;
constexpr int kRT1 = 0, kRT2 = kRT1 + kRH * kRK1, kRT3 = kRT2 + kRH * kRH,
              kRT4 = kRT3 + kRH * kRH, kRTEnd = kRT4 + kROut * kRH;   // bf16 elements

// Element offset of (row, k) in a canonical K-major operand with K columns.
__host__ __device__ constexpr int canon_off(int row, int k, int K)
{
    return (row >> 3) * (K >> 3) * 64 + (k >> 3) * 64 + (row & 7) * 8 + (k & 7);
}

struct RankerDev {
    const __nv_bfloat16 *wt;   // kRTEnd elements
    const float *master;       // kRParams (biases are read from here)
};

// Per-scene cluster context (ints): 64 cluster boxes (lo xyz, hi xyz; empty
// clusters lo > hi), the 64 cut nodes (node index, or ~facet for a leaf) and
// 65 sorted-range starts (cluster c = positions [start[c], start[c + 1]);
// unused clusters are empty ranges at n).
// The boxes are also kept as floats of twice their value (the features work
// in 2x scaled units; exact below 2^23), so that the features need no
// integer conversions.
constexpr int kRCBox = 0, kRCut = 6 * kRClusters, kRCStart = kRCut + kRClusters;
constexpr int kRCFBox = 516;   // >= kRCStart + kRClusters + 1, a multiple of 4
constexpr int kRCtx = kRCFBox + 6 * kRClusters;
static_assert(kRCStart + kRClusters + 1 <= kRCFBox, "cluster context");

// Cluster holding sorted position pos (starts ascending, start[0] = 0).
__device__ __forceinline__ int cluster_at(const int *start, int pos)
{
    int lo = 0, hi = kRClusters - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= pos) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Walk of the rest of the tree: skip the cut subtrees already walked.
// ncl[node] = the cluster a cut node roots, -1 for every other node.
struct CutFilter {
    const signed char *ncl;
    unsigned long long done;
    __device__ __forceinline__ bool node(int id) const
    {
        const int c = __ldg(ncl + id);
        return c < 0 || !((done >> c) & 1ull);
    }
    __device__ __forceinline__ void grow(float &, float &, float &, float &, float &,
                                         float &) const {}
};

// The pair's centroid segment in 2x scaled units (2 o + u + v is twice a
// parallelogram's centroid): start p, direction d = q - p, and 1/d.
struct PairGeom {
    float p[3], d[3], r[3];
    __device__ __forceinline__ PairGeom(const Leaf &Li, const Leaf &Lj)
    {
        p[0] = (float)(2 * Li.ox + Li.ux + Li.vx);
        p[1] = (float)(2 * Li.oy + Li.uy + Li.vy);
        p[2] = (float)(2 * Li.oz + Li.uz + Li.vz);
        d[0] = (float)(2 * Lj.ox + Lj.ux + Lj.vx) - p[0];
        d[1] = (float)(2 * Lj.oy + Lj.uy + Lj.vy) - p[1];
        d[2] = (float)(2 * Lj.oz + Lj.uz + Lj.vz) - p[2];
        for (int a = 0; a < 3; a++) r[a] = d[a] != 0.f ? __frcp_rn(d[a]) : 0.f;
    }
};

// Feature f (0..79) of the pair (Li, Lj); bounds are the scene's centroid
// bounds (lo + hi units), C the scene's cluster context (its float boxes).
__device__ __forceinline__ float pair_feature(int f, const PairGeom &G, const Leaf &Li,
                                              const Leaf &Lj, const int *bounds, const int *C)
{
    if (f < 6) {   // centroids, normalised to the scene's centroid box
        const int a = f % 3;
        const float v = f < 3 ? G.p[a] : G.p[a] + G.d[a];
        const float lo = (float)__ldg(bounds + a),
                    span = fmaxf(1.f, (float)__ldg(bounds + 3 + a) - lo);
        return fminf(fmaxf((v - lo) / span, 0.f), 1.f);
    }
    if (f < 12) {   // unit normals
        const Leaf &L = f < 9 ? Li : Lj;
        const float nx = (float)L.nx, ny = (float)L.ny, nz = (float)L.nz;
        const float inv = rsqrtf(fmaxf(nx * nx + ny * ny + nz * nz, 1e-30f));
        const int a = (f - 6) % 3;
        return (a == 0 ? nx : a == 1 ? ny : nz) * inv;
    }
    if (f >= kRIn) return 0.f;
    // entry depth of the centroid segment into cluster box c: 1 - t_entry
    const float *b = reinterpret_cast<const float *>(C + kRCFBox) + 6 * (f - 12);
    const float b0 = __ldg(b), b3 = __ldg(b + 3);
    if (b0 > b3) return 0.f;   // empty cluster
    float tn = 0.f, tf = 1.f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float lo = a == 0 ? b0 : __ldg(b + a);
        const float hi = a == 0 ? b3 : __ldg(b + 3 + a);
        if (G.d[a] == 0.f) {
            if (G.p[a] < lo || G.p[a] > hi) return 0.f;
            continue;
        }
        const float t0 = (lo - G.p[a]) * G.r[a], t1 = (hi - G.p[a]) * G.r[a];
        tn = fmaxf(tn, fminf(t0, t1));
        tf = fminf(tf, fmaxf(t0, t1));
    }
    return tn <= tf ? 1.f - tn : 0.f;
}

// ---------------------------------------------------------------- launchers
// The cut, cluster boxes and starts of every scene into ctx [n_scenes][kRCtx],
// and ncl [total_nodes] (after the BVH is built).
cudaError_t ranker_clusters(const DevScenes &g, int *ctx, signed char *ncl, cudaStream_t st);
// Top-8 clusters of every candidate pair (tensor cores; one CTA per SM, 135 KB
// of shared memory and 128 TMEM columns each); IVM_ERR_TIMEOUT into err if a
// wait for the tensor cores runs out.
cudaError_t ranker_rank_pairs(const DevScenes &g, const int2 *pairs, unsigned long long npairs,
                              const unsigned long long *count_dev, const int *ctx,
                              const RankerDev &r, unsigned long long *ranks, int n_sm, int *err,
                              cudaStream_t st);
// The same network over precomputed feature rows [n][76]: logits [n][64]
// and packed top-8 cluster indices [n].
cudaError_t ranker_infer(const float *feat, unsigned long long n, const RankerDev &r,
                         float *logits, unsigned long long *ranks, int n_sm, int *err,
                         cudaStream_t st);
cudaError_t ranker_log_hits(const DevScenes &g, const int2 *pairs, unsigned long long npairs,
                            const int *ctx, float *feat, int *label,
                            unsigned long long *cursor, unsigned long long cap, int *err,
                            cudaStream_t st);
cudaError_t ranker_pack(const float *master, __nv_bfloat16 *wt, cudaStream_t st);
// loss and gradients of a batch (all device pointers); grads has kRParams
cudaError_t ranker_grad(const float *master, const float *x, const int *y, int batch,
                        float *act, float *grads, float *loss, cudaStream_t st);
cudaError_t ranker_adam(float *master, const float *grads, float *m, float *v, float lr,
                        int step, cudaStream_t st);
size_t ranker_act_floats(int batch);
cudaError_t ranker_gather(const float *feat, const int *label, const int *idx, int B, float *x,
                          int *y, cudaStream_t st);

}  // namespace ivm
