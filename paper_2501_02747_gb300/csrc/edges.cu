// edges.cu -- edges as visible nodes (the matrix and table list visible faces
// and edges: Sec. I-II) and the edge nearest a source (first-order
// diffraction by the edge closest to the receiver: Sec. III-B).
//
// Edge e = segment A -> B (cm) carries s samples at the cell centres
// p_a = 2s A + (2a+1)(B - A).  vis_X[t][e] = some sample has not
// blocked(X_t, p_a).  The nearest visible edge of X_t is the visible edge
// with the sample closest to X_t (squared distance over all of its samples,
// ties to the lower edge index).
//
// Work item = (side, 32-edge word, run of consecutive snapshots); per
// snapshot the word's edges go floor(32 / s) at a time into a packet of
// sample segments (a lane keeps the same edge sample at every snapshot of
// the item).  Consecutive snapshots see nearly the same picture, so a lane
// first re-walks only if its sample was the reachable one of its edge last
// time (an edge found visible that way needs no other walk), then tests the
// facet that blocked its sample last time, and only then goes to the warp's
// recent occluders and the BVH; every test is the same exact facet test, so
// the rows never depend on these guesses.  The samples of visible edges give
// (squared distance << 16 | edge), and one 64-bit atomicMin per (snapshot,
// side) keeps the smallest: squared distances of in-range points stay below
// 2^48 and edges are fewer than 2^16.
#include <type_traits>

#include "edges.cuh"
#include "traverse.cuh"
#include "filter.cuh"

namespace ivm {

constexpr int kEdgeWarps = kTravThreads / 32;

template <bool FILTERED>
__global__ void __launch_bounds__(kTravThreads)
k_edge_table(DevScenes g, EdgeArgs a, int *err)
{
    // per warp and packet of the word: each lane's last blocker, and the
    // lanes whose sample was the reachable one at the last snapshot
    __shared__ int s_blk[kEdgeWarps][32][32];
    __shared__ unsigned s_free[kEdgeWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long per_side = (long long)a.WE * a.ntiles;
    if (w >= 2 * per_side) return;   // uniform per warp
    const SceneDesc &D = g.desc[0];
    const int side = w >= per_side ? 1 : 0;
    const long long rem = w - side * per_side;
    const int c = (int)(rem / a.ntiles);
    const long long t0 = (rem - (long long)c * a.ntiles) * a.tile;
    const long long t1 = min(t0 + a.tile, a.S);
    const int s = D.s;
    const long long k = 2LL * s;
    const int *pos = side ? a.rx : a.tx;
    WalkCounters wc;
    OccluderCache cache;
    cache.enter_scene(0);
    typename std::conditional<FILTERED, FilteredLeafCall, ExactLeaf>::type leaf;
    const int G = 32 / s;
    const int gi = lane / s, smp = lane - gi * s;
    for (int q = 0; q < 32; q++) s_blk[warp][q][lane] = -1;
    s_free[warp][lane] = 0u;
    __syncwarp();
    const unsigned smask = s == 32 ? kFull : ((1u << s) - 1u);
    long long L0 = 0, L1 = 0, L2 = 0;   // the last traced position
    bool have_last = false;
    uint32_t word = 0;
    unsigned long long best = ~0ull;
    for (long long t = t0; t < t1; t++) {
        const long long X0 = k * pos[3 * t], X1 = k * pos[3 * t + 1], X2 = k * pos[3 * t + 2];
        const bool xin = X0 > -kCoordLimit && X0 < kCoordLimit && X1 > -kCoordLimit &&
                         X1 < kCoordLimit && X2 > -kCoordLimit && X2 < kCoordLimit;
        if (!xin) {
            if (lane == 0) raise_error(err, IVM_ERR_RANGE);
            continue;
        }
        if (have_last && X0 == L0 && X1 == L1 && X2 == L2) {   // same position: same row
            if (lane == 0) {
                a.table[((size_t)t * 2 + side) * a.WE + c] = word;
                if (best != ~0ull) atomicMin(a.nearest_key + 2 * t + side, best);
            }
            continue;
        }
        have_last = true;
        L0 = X0; L1 = X1; L2 = X2;
        word = 0;
        best = ~0ull;
        for (int e0 = 32 * c, grp = 0; e0 < min(32 * c + 32, a.ne); e0 += G, grp++) {
            const int e = e0 + gi;
            const bool mine = gi < G && e < min(32 * c + 32, a.ne);
            long long px = 0, py = 0, pz = 0;
            bool ok = mine;
            if (mine) {
                const int *E = a.edges + 6 * (size_t)e;
                px = k * E[0] + (2 * smp + 1) * (long long)(E[3] - E[0]);
                py = k * E[1] + (2 * smp + 1) * (long long)(E[4] - E[1]);
                pz = k * E[2] + (2 * smp + 1) * (long long)(E[5] - E[2]);
                ok = px > -kCoordLimit && px < kCoordLimit && py > -kCoordLimit &&
                     py < kCoordLimit && pz > -kCoordLimit && pz < kCoordLimit;
                if (!ok) raise_error(err, IVM_ERR_RANGE);
            }
            unsigned alive = __ballot_sync(kFull, ok);
            if (!alive) continue;
            wc.segments += ok;
            Seg sg = make_seg((int)X0, (int)X1, (int)X2, (int)px, (int)py, (int)pz);
            const int lead = __ffs(alive) - 1;
            const float dx = (float)__shfl_sync(kFull, sg.dx, lead);
            const float dy = (float)__shfl_sync(kFull, sg.dy, lead);
            const float dz = (float)__shfl_sync(kFull, sg.dz, lead);
            int myblk = -1;
            unsigned freem = 0;
            // 1. lanes whose sample was reachable last time walk first
            const unsigned pm = alive & s_free[warp][grp];
            if (pm) {
                freem = pm & occlude<true, decltype(leaf), false>(sg, pm, g.nodes, g.leaf, D.root,
                                                                  dx, dy, dz, D.budget, err, wc,
                                                                  leaf, cache, myblk);
                // an edge seen through one sample needs no other walk
                const bool seen = mine && ((freem >> (gi * s)) & smask) != 0u;
                alive &= ~(__ballot_sync(kFull, seen) | pm);
            }
            // 2. each remaining lane tests the facet that blocked its sample last time
            if (alive) {
                const int tb = s_blk[warp][grp][lane];
                bool hit = false;
                if (((alive >> lane) & 1u) && tb >= 0) {
                    wc.leaf_tests++;
                    hit = leaf(sg, load_leaf(g.leaf, tb), wc);
                    if (hit) { myblk = tb; wc.cache_hits++; }
                }
                alive &= ~__ballot_sync(kFull, hit);
            }
            // 3. the rest: recent occluders, then the BVH
            if (alive)
                freem |= alive & occlude<true>(sg, alive, g.nodes, g.leaf, D.root, dx, dy, dz,
                                               D.budget, err, wc, leaf, cache, myblk);
            if (mine && myblk >= 0) s_blk[warp][grp][lane] = myblk;
            __syncwarp();
            if (lane == 0) s_free[warp][grp] = freem;
            __syncwarp();
            const bool free_lane = (freem >> lane) & 1u;
            word |= __reduce_or_sync(kFull, free_lane ? 1u << (e & 31) : 0u);
            const bool vis_edge = mine && ((freem >> (gi * s)) & smask) != 0u;
            if (vis_edge) {
                const long long rx_ = px - X0, ry_ = py - X1, rz_ = pz - X2;
                const unsigned long long d2 =
                    (unsigned long long)(rx_ * rx_ + ry_ * ry_ + rz_ * rz_);
                const unsigned long long key = (d2 << 16) | (unsigned long long)e;
                if (key < best) best = key;
            }
        }
        for (int o = 16; o; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(kFull, best, o);
            if (v < best) best = v;
        }
        if (lane == 0) {
            a.table[((size_t)t * 2 + side) * a.WE + c] = word;
            if (best != ~0ull) atomicMin(a.nearest_key + 2 * t + side, best);
        }
    }
    flush_counters(wc, a.ctr);
}

__global__ void k_edge_key_init(unsigned long long *key, long long n)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) key[i] = ~0ull;
}

__global__ void k_edge_nearest(const unsigned long long *key, long long n, int *nearest)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) nearest[i] = key[i] == ~0ull ? -1 : (int)(key[i] & 0xffffu);
}

cudaError_t edges_table(const DevScenes &g, const EdgeArgs &a, bool filtered, int *err,
                        cudaStream_t st)
{
    const long long n = 2 * a.S;
    if (n == 0) return cudaSuccess;
    k_edge_key_init<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a.nearest_key, n);
    const long long warps = 2LL * a.WE * a.ntiles;
    const unsigned blocks = (unsigned)((warps * 32 + kTravThreads - 1) / kTravThreads);
    if (warps > 0) {
        if (filtered) k_edge_table<true><<<blocks, kTravThreads, 0, st>>>(g, a, err);
        else k_edge_table<false><<<blocks, kTravThreads, 0, st>>>(g, a, err);
    }
    k_edge_nearest<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a.nearest_key, n, a.nearest);
    note_launches(warps > 0 ? 3 : 2);
    return cudaGetLastError();
}

}  // namespace ivm
