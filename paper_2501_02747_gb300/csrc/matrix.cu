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
//
// Learned form: the pair's ranked clusters (ranker.cu) are walked first, in
// order, while they keep blocking lanes; then the rest of the tree without
// them.  The set of facets tested is the same as in a full walk, so the bit
// is the same.
#include "ivm_internal.cuh"
#include "traverse.cuh"
#include "filter.cuh"
#include "ranker.cuh"

namespace ivm {

// Proposals walked at most before the rest of the tree.
constexpr int kRankedWalks = 8;

// Box-test form of the matrix walks (seg_box): the absolute form, one FMA
// per plane (city, fast form: matrix 286 ms against 304 ms with the relative
// form, the same box tests to 0.03%).
#ifndef IVM_MATRIX_ABS_BOX
#define IVM_MATRIX_ABS_BOX 1
#endif
constexpr bool kMatrixAbsBox = IVM_MATRIX_ABS_BOX != 0;

// Cluster-first walk of a packet; same contract as occlude().
template <bool CACHE, class LeafFn>
__device__ __forceinline__ unsigned occlude_ranked(Seg &s, unsigned alive, const Node *nodes,
                                                   const Leaf *leaves, int root,
                                                   const int *C, const signed char *ncl,
                                                   unsigned long long rk, float dirx, float diry,
                                                   float dirz, int budget, int *err,
                                                   WalkCounters &wc, LeafFn leaf_hit,
                                                   OccluderCache &cache, int &myblk)
{
    const int lane = threadIdx.x & 31;
    if (CACHE) {
        alive = cache_tests(s, alive, leaves, wc, leaf_hit, cache, myblk);
        if (!alive) return 0;
    }
    if (s.ix == 0.f) finish_seg<kMatrixAbsBox>(s);
    unsigned long long done = 0;
    int blocker, last = -1;
    for (int k = 0; k < kRankedWalks && k < kRTop; k++) {
        const int c = (int)((rk >> (8 * k)) & 0xff);
        if (c >= kRClusters || ((done >> c) & 1ull)) continue;
        if (__ldg(C + kRCStart + c + 1) <= __ldg(C + kRCStart + c)) continue;   // empty
        const unsigned before = alive;
        alive = walk_packet<LeafFn, NoFilter, kMatrixAbsBox>(s, alive, nodes, leaves,
                                                             __ldg(C + kRCut + c), dirx, diry,
                                                             dirz, budget, err, wc, leaf_hit,
                                                             blocker, myblk);
        done |= 1ull << c;
        if (blocker >= 0) last = blocker;
        if (k == 0) wc.ranker_hits += ((before & ~alive) >> lane) & 1u;
        wc.ranker_hits8 += ((before & ~alive) >> lane) & 1u;
        if (!alive) {
            if (CACHE) cache.put(last);
            return 0;
        }
        if (alive == before) break;   // the proposal blocked nothing: stop trusting it
    }
    alive = walk_packet<LeafFn, CutFilter, kMatrixAbsBox>(s, alive, nodes, leaves, root, dirx,
                                                          diry, dirz, budget, err, wc, leaf_hit,
                                                          blocker, myblk, CutFilter{ncl, done});
    if (blocker >= 0) last = blocker;
    if (CACHE) cache.put(last);
    return alive;
}

// Blocked sets are convex: for a convex facet F and a fixed end q, the
// points p from which the open segment p-q meets F form a convex set
// ({q + L (f - q) : f in F, L > 1}), and so do the points q for a fixed p.
// A facet's samples lie in the convex hull of its four corner samples.  So
// if F blocks the 16 segments between the corner samples of facets i and j,
// it blocks every sample segment between them and M_ij = 0: for each corner
// p_c the q-set contains j's corners, hence all of j's samples; then for
// each sample q the p-set contains i's corners, hence all of i's samples.
// Candidates F are the warp's recent occluders; lanes 0-15 test one, 16-31
// another, with the same exact facet test as everywhere else.
// The proof is tried unless IVM_FLAG_NO_CORNER_PROOF is given: it pays where
// one facet often hides a whole pair (district: matrix 1.18 ms with it, 1.21
// without; degenerate district 1.26 / 1.31) and costs more than it settles
// on the 25k-facet city (315 / 296 ms); the autotuner chooses.

template <class LeafFn>
__device__ __noinline__ bool corners_blocked(const DevScenes &g, int baseI, int baseJ, int s,
                                             int f0, int f1, int f2, int f3, WalkCounters &wc,
                                             LeafFn leaf)
{
    const int lane = threadIdx.x & 31;
    const int l = s - 1;   // corner samples: a, b in {0, s - 1}, index a s + b
    const int ka = ((lane & 1) ? l * s : 0) + ((lane & 2) ? l : 0);
    const int kb = ((lane & 4) ? l * s : 0) + ((lane & 8) ? l : 0);
    const Seg sg = make_seg(__ldg(g.sx + baseI + ka), __ldg(g.sy + baseI + ka),
                            __ldg(g.sz + baseI + ka), __ldg(g.sx + baseJ + kb),
                            __ldg(g.sy + baseJ + kb), __ldg(g.sz + baseJ + kb));
    for (int pass = 0; pass < 2; pass++) {
        const int F = (lane >> 4) ? (pass ? f3 : f1) : (pass ? f2 : f0);
        bool hit = false;
        if (F >= 0) {
            wc.leaf_tests++;
            hit = leaf(sg, load_leaf(g.leaf, F), wc);
        }
        const unsigned hm = __ballot_sync(kFull, hit);
        if ((hm & 0xFFFFu) == 0xFFFFu || (hm >> 16) == 0xFFFFu) return true;
        if ((pass ? f2 : f0) < 0) break;
    }
    return false;
}

template <bool CACHE, bool LEARN, class LeafFn>
__device__ __forceinline__ void decide_pair(const DevScenes &g, int gi, int gj,
                                            const LearnedDev &lrn, unsigned long long rk,
                                            int *err, WalkCounters &wc, LeafFn leaf,
                                            OccluderCache &cache, bool corner)
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
    const int budget = D.budget;
    if (CACHE && corner && cache.f[0] >= 0 &&
        corners_blocked(g, baseI, baseJ, s, cache.f[0], cache.f[1], cache.f[2], cache.f[3], wc,
                        leaf))
        return;
    bool visible = false;
    bool retried = false;
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
        if (LEARN)
            alive = occlude_ranked<CACHE>(sg, alive, g.nodes, g.leaf, D.root,
                                          lrn.ctx + (size_t)kRCtx * Li.scene, lrn.ncl, rk, dirx,
                                          diry, dirz, budget, err, wc, leaf, cache, myblk);
        else
            alive = occlude<CACHE, LeafFn, CACHE, kMatrixAbsBox>(sg, alive, g.nodes, g.leaf,
                                                                 D.root, dirx, diry, dirz,
                                                                 budget, err, wc, leaf, cache,
                                                                 myblk);
        if (alive) {
            visible = true;
            break;
        }
        // the first blocked packet may have brought a new occluder to the front
        if (CACHE && corner && !retried && b0 + 32 < total) {
            retried = true;
            const int f = cache.f[0];
            if (f >= 0 && corners_blocked(g, baseI, baseJ, s, f, -1, -1, -1, wc, leaf)) return;
        }
    }
    if (visible && lane == 0) {
        atomicOr(D.matrix + (size_t)i * D.W + (j >> 5), 1u << (j & 31));
        atomicOr(D.matrix + (size_t)j * D.W + (i >> 5), 1u << (i & 31));
    }
}

// Register cap of the matrix kernel: 7 resident blocks of 128 threads (72
// registers).  With the absolute-form box test, 7 beat 8 and 6 (city, fast
// form: 266 ms against 286 and 277 ms; district 1.19 against 1.29 ms): more
// warps hide the dependent box-test latency, fewer registers spill more.
// The learned walk holds more state: 6 (city, learned form: 417 ms against
// 445 ms with 4 and 449 ms with 8).
#ifndef IVM_MATRIX_MIN_BLOCKS
#define IVM_MATRIX_MIN_BLOCKS 7
#endif
#ifndef IVM_MATRIX_MIN_BLOCKS_LEARNED
#define IVM_MATRIX_MIN_BLOCKS_LEARNED 6
#endif
constexpr int kMatrixMinBlocks = IVM_MATRIX_MIN_BLOCKS,
              kMatrixMinBlocksLearned = IVM_MATRIX_MIN_BLOCKS_LEARNED;

template <bool PERSIST, bool CACHE, bool LEARN, class LeafFn>
__global__ void __launch_bounds__(kTravThreads, LEARN ? kMatrixMinBlocksLearned : kMatrixMinBlocks)
k_matrix(DevScenes g, const int2 *pairs, unsigned long long npairs, int tile, int corner,
         const unsigned long long *count_dev, LearnedDev lrn, unsigned long long *work,
         unsigned long long *ctr, int *err)
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
            decide_pair<CACHE, LEARN>(g, p.x, p.y, lrn, LEARN ? lrn.ranks[w] : 0ull, err, wc,
                                      leaf, cache, corner != 0);
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
                decide_pair<CACHE, LEARN>(g, p.x, p.y, lrn, LEARN ? lrn.ranks[w] : 0ull, err,
                                          wc, leaf, cache, corner != 0);
            }
        }
    }
    flush_counters(wc, ctr);
}

template <bool PERSIST, bool CACHE, bool LEARN, class LeafFn>
static void launch_one(const DevScenes &g, const int2 *pairs, unsigned long long npairs,
                       const LaunchCfg &cfg, unsigned long long *work, unsigned long long *ctr,
                       int *err, cudaStream_t st)
{
    const int threads = 32 * cfg.warps_per_block;
    auto kern = k_matrix<PERSIST, CACHE, LEARN, LeafFn>;
    if (PERSIST) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
        int blocks = cfg.n_sm * (per_sm > 0 ? per_sm : 1);
        cudaMemsetAsync(work, 0, sizeof(unsigned long long), st);
        kern<<<blocks, threads, 0, st>>>(g, pairs, npairs, cfg.tile, cfg.corner, cfg.count_dev,
                                         cfg.learn, work, ctr, err);
    } else {
        unsigned long long blocks = (npairs + cfg.warps_per_block - 1) / cfg.warps_per_block;
        kern<<<(unsigned)blocks, threads, 0, st>>>(g, pairs, npairs, 1, cfg.corner, nullptr,
                                                   cfg.learn, work, ctr, err);
    }
}

template <class LeafFn, bool LEARN>
static void launch_leaf(const DevScenes &g, const int2 *pairs, unsigned long long npairs,
                        const LaunchCfg &cfg, unsigned long long *work, unsigned long long *ctr,
                        int *err, cudaStream_t st)
{
    if (cfg.persistent) {
        if (cfg.cache) launch_one<true, true, LEARN, LeafFn>(g, pairs, npairs, cfg, work, ctr, err, st);
        else launch_one<true, false, LEARN, LeafFn>(g, pairs, npairs, cfg, work, ctr, err, st);
    } else {
        if (cfg.cache) launch_one<false, true, LEARN, LeafFn>(g, pairs, npairs, cfg, work, ctr, err, st);
        else launch_one<false, false, LEARN, LeafFn>(g, pairs, npairs, cfg, work, ctr, err, st);
    }
}

cudaError_t launch_matrix(const DevScenes &g, const int2 *pairs, unsigned long long npairs,
                          const LaunchCfg &cfg, unsigned long long *work,
                          unsigned long long *ctr, int *err, cudaStream_t st)
{
    if (npairs == 0) return cudaSuccess;
    if (cfg.mode == IVM_MODE_EXACT)
        launch_leaf<ExactLeaf, false>(g, pairs, npairs, cfg, work, ctr, err, st);
    else if (cfg.learn.ranks && cfg.aligned)
        launch_leaf<AlignedLeafCall, true>(g, pairs, npairs, cfg, work, ctr, err, st);
    else if (cfg.learn.ranks)
        launch_leaf<FilteredLeaf, true>(g, pairs, npairs, cfg, work, ctr, err, st);
    else if (cfg.aligned)
        // out of line: one copy of the test instead of one per cache slot and
        // walk (city, fast form: 327 ms against 367 ms inlined, 362 ms with the
        // inlined four-edge filter)
        launch_leaf<AlignedLeafCall, false>(g, pairs, npairs, cfg, work, ctr, err, st);
    else
        launch_leaf<FilteredLeaf, false>(g, pairs, npairs, cfg, work, ctr, err, st);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace ivm
