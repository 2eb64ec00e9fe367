// matrix.cu -- the 3D inter-visibility matrix (Sec. II of the paper).
//
// M_ij = 1 when some sample p of facet i and some sample q of facet j see
// each other: q strictly in front of i, p strictly in front of j (Sec. II-B,
// Eq. (2)), and no facet meets the open segment p-q (the intersection
// judgment moved into pre-processing, Abstract and Sec. I).  The Tx plays no
// part (Sec. II-B: Tx-to-reference-face visibility is assumed).
//
// One warp decides one candidate pair (i < j).  Its lanes take the s^4 sample
// pairs 32 at a time as a packet; a packet ends as soon as every lane is
// blocked, and the pair ends at the first packet with a free lane.  The bit
// is written to row i and, by symmetry, row j.
#include "ivm_internal.cuh"
#include "traverse.cuh"
#include "filter.cuh"

namespace ivm {

template <bool CACHE, class LeafFn>
__device__ __forceinline__ void decide_pair(const DevScenes &g, int gi, int gj, int *err,
                                            WalkCounters &wc, LeafFn leaf, OccluderCache &cache)
{
    const int lane = threadIdx.x & 31;
    const Leaf Li = load_leaf(g.leaf, gi), Lj = load_leaf(g.leaf, gj);
    const SceneDesc &D = g.desc[Li.scene];
    if (CACHE) cache.enter_scene(Li.scene);
    const int s = D.s, s2 = s * s, total = s2 * s2;
    const int i = gi - D.facet0, j = gj - D.facet0;
    const int baseI = D.sample0 + i * s2, baseJ = D.sample0 + j * s2;
    const float dirx = (float)(2 * (Lj.ox - Li.ox) + Lj.ux + Lj.vx - Li.ux - Li.vx);
    const float diry = (float)(2 * (Lj.oy - Li.oy) + Lj.uy + Lj.vy - Li.uy - Li.vy);
    const float dirz = (float)(2 * (Lj.oz - Li.oz) + Lj.uz + Lj.vz - Li.uz - Li.vz);
    const int budget = 4 * D.n + 16;
    bool visible = false;
    for (int b0 = 0; b0 < total; b0 += 32) {
        const int idx = b0 + lane;
        const bool valid = idx < total;
        const int a = valid ? idx / s2 : 0, b = valid ? idx - a * s2 : 0;
        int px = 0, py = 0, pz = 0, qx = 0, qy = 0, qz = 0;
        if (valid) {
            px = __ldg(g.sx + baseI + a); py = __ldg(g.sy + baseI + a); pz = __ldg(g.sz + baseI + a);
            qx = __ldg(g.sx + baseJ + b); qy = __ldg(g.sy + baseJ + b); qz = __ldg(g.sz + baseJ + b);
        }
        const bool face = valid && front_of(Lj, px, py, pz) && front_of(Li, qx, qy, qz);
        unsigned alive = __ballot_sync(kFull, face);
        if (!alive) continue;
        wc.segments += face;
        Seg sg = make_seg(px, py, pz, qx, qy, qz);
        int myblk = -1;
        alive = occlude<CACHE>(sg, alive, g.nodes, g.leaf, D.root, dirx, diry, dirz, budget, err,
                               wc, leaf, cache, myblk);
        if (alive) {
            visible = true;
            break;
        }
    }
    if (visible && lane == 0) {
        atomicOr(D.matrix + (size_t)i * D.W + (j >> 5), 1u << (j & 31));
        atomicOr(D.matrix + (size_t)j * D.W + (i >> 5), 1u << (i & 31));
    }
}

template <bool PERSIST, bool CACHE, class LeafFn>
__global__ void __launch_bounds__(kTravThreads, IVM_MIN_BLOCKS)
k_matrix(DevScenes g, const int2 *pairs, unsigned long long npairs, int tile,
         const unsigned long long *count_dev, unsigned long long *work, unsigned long long *ctr,
         int *err)
{
    WalkCounters wc;
    LeafFn leaf;
    OccluderCache cache;
    const int lane = threadIdx.x & 31;
    // persistent launches may take the pair count from the screen's device
    // counter (written by an earlier kernel on the same stream)
    if (PERSIST && count_dev) npairs = min(npairs, *count_dev);
    if (!PERSIST) {
        unsigned long long w = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        if (w < npairs) {
            const int2 p = pairs[w];
            decide_pair<CACHE>(g, p.x, p.y, err, wc, leaf, cache);
        }
    } else {
        for (;;) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(work, (unsigned long long)tile);
            base = __shfl_sync(kFull, base, 0);
            if (base >= npairs) break;
            unsigned long long end = min(base + (unsigned long long)tile, npairs);
            for (unsigned long long w = base; w < end; w++) {
                const int2 p = pairs[w];
                decide_pair<CACHE>(g, p.x, p.y, err, wc, leaf, cache);
            }
        }
    }
    flush_counters(wc, ctr);
}

template <bool PERSIST, bool CACHE, class LeafFn>
static void launch_one(const DevScenes &g, const int2 *pairs, unsigned long long npairs,
                       const LaunchCfg &cfg, unsigned long long *work, unsigned long long *ctr,
                       int *err, cudaStream_t st)
{
    const int threads = 32 * cfg.warps_per_block;
    auto kern = k_matrix<PERSIST, CACHE, LeafFn>;
    if (PERSIST) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
        int blocks = cfg.n_sm * (per_sm > 0 ? per_sm : 1);
        cudaMemsetAsync(work, 0, sizeof(unsigned long long), st);
        kern<<<blocks, threads, 0, st>>>(g, pairs, npairs, cfg.tile, cfg.count_dev, work, ctr,
                                         err);
    } else {
        unsigned long long blocks = (npairs + cfg.warps_per_block - 1) / cfg.warps_per_block;
        kern<<<(unsigned)blocks, threads, 0, st>>>(g, pairs, npairs, 1, nullptr, work, ctr, err);
    }
}

template <class LeafFn>
static void launch_leaf(const DevScenes &g, const int2 *pairs, unsigned long long npairs,
                        const LaunchCfg &cfg, unsigned long long *work, unsigned long long *ctr,
                        int *err, cudaStream_t st)
{
    if (cfg.persistent) {
        if (cfg.cache) launch_one<true, true, LeafFn>(g, pairs, npairs, cfg, work, ctr, err, st);
        else launch_one<true, false, LeafFn>(g, pairs, npairs, cfg, work, ctr, err, st);
    } else {
        if (cfg.cache) launch_one<false, true, LeafFn>(g, pairs, npairs, cfg, work, ctr, err, st);
        else launch_one<false, false, LeafFn>(g, pairs, npairs, cfg, work, ctr, err, st);
    }
}

cudaError_t launch_matrix(const DevScenes &g, const int2 *pairs, unsigned long long npairs,
                          const LaunchCfg &cfg, unsigned long long *work,
                          unsigned long long *ctr, int *err, cudaStream_t st)
{
    if (npairs == 0) return cudaSuccess;
    if (cfg.mode == IVM_MODE_EXACT) launch_leaf<ExactLeaf>(g, pairs, npairs, cfg, work, ctr, err, st);
    else launch_leaf<FilteredLeaf>(g, pairs, npairs, cfg, work, ctr, err, st);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace ivm
