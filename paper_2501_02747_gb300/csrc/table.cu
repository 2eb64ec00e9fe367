// table.cu -- the 3D inter-visibility table for the mobile Tx and Rx at the
// specific points of their routes (Sec. III-B/C, Table II of the paper).
//
// vis_X[t][j] = 1 when facet j faces X_t strictly and some sample of j is
// reachable from X_t by a segment no facet blocks; los[t] = 1 when the direct
// Tx_t - Rx_t segment is free (Sec. III-B: the transmitter is the parent node
// that searches its reference faces).
//
// Work item = (side, 32-facet word c, tile of consecutive snapshots).  Lane l
// owns facet 32c + l: it does the facing test, and the warp then takes the
// front-facing facets a packet at a time -- with s*s <= 32 samples,
// floor(32 / (s*s)) facets share a packet; with more samples a facet takes
// several packets and stops at the first free one.  Lane 0 writes the word.
//
// Along a trajectory the table changes only at ray creation and suppression
// points (Sec. III-C); between them consecutive snapshots see the same
// facets through the same gaps.  With the occluder cache on, lane l also
// keeps the facet that blocked facet 32c + l at the previous snapshot of the
// tile and tests it first: a blocked facet usually stays blocked by the same
// building, so one exact facet test replaces the BVH walk.  The cached facet
// is only tested, never trusted: a lane it does not block goes on to the walk.
//
// Runs of equal positions (a static Tx, a receiver that pauses) have equal
// rows: with deduplication on, a pre-pass finds the first snapshot of each
// run, only that row is traced, and a post-pass copies it over the run.
//
// Hidden facets are settled for a whole tile at once when the tile's
// positions lie on the segment between its first and last position (a
// straight stretch of route).  For a convex facet F and a sample q, the
// positions a from which the open segment a-q meets F form the convex set
// {q + L (f - q) : f in F, L > 1}; so if F blocks every sample segment of
// facet j from both end positions, it blocks them from every position of
// the tile, and j is hidden at all of the tile's snapshots.  F is the facet
// that hid j at the tile's first traced snapshot; the two end tests per
// sample are the same exact facet tests as everywhere else.
//
// Lazy splitting (persistent launches).  A work item is a long dependent
// chain, and a few long items decide the kernel's span.  Each warp publishes
// the snapshot range it still has to do, [cur, end), in a 16-byte slot; a
// warp that finds the queue empty takes the back half of the largest
// remaining range by one 128-bit compare-and-swap that lowers the owner's
// end (only while both halves keep at least one straight stretch).  The
// owner republishes cur by compare-and-swap at each stretch and never runs
// past the end it reads there; the split point is at least one stretch past
// the published cur, so no snapshot is done twice and none is left out.
// Nobody waits: an owner never depends on a thief, and a thief that finds
// nothing worth taking exits.
#include "ivm_internal.cuh"
#include "traverse.cuh"
#include "filter.cuh"

namespace ivm {

// Box-test form of the table walks (seg_box): the relative form (city, fast
// form: table 176 ms against 180 ms with the absolute form, the same box
// tests to 0.1%).
#ifndef IVM_TABLE_ABS_BOX
#define IVM_TABLE_ABS_BOX 0
#endif
constexpr bool kTableAbsBox = IVM_TABLE_ABS_BOX != 0;

// Table packet strategy: probe the previously seen sample first; test the
// warp's recently used occluders before a walk.
constexpr bool kTableProbe = true;
constexpr bool kTableLru = true;
constexpr bool kTableTileProof = true;
constexpr bool kTableSweep = true;   // also settle visible facets by a swept walk
constexpr bool kTableBatchProbe = true;
// Per-sample temporal blockers (shared memory, 32 facets x 32 samples per warp).
constexpr bool kTableSampleBlockers = true;
constexpr int kSampleSlots = 32 * 32;
// Snapshots per straight-stretch proof (a work item may hold several) come
// from the launch (PT, ivm_params.proof_tile).

// ------------------------------------------------------------ lazy splitting

// a = work item + 1 (0: never used); b = cur | end << 32 (local snapshots)
struct __align__(16) StealSlot {
    unsigned long long a, b;
};

__device__ __forceinline__ bool same(const StealSlot &x, const StealSlot &y)
{
    return x.a == y.a && x.b == y.b;
}

__device__ __forceinline__ StealSlot slot_read(StealSlot *p)
{
    return atomicCAS(p, StealSlot{0ull, 0ull}, StealSlot{0ull, 0ull});   // atomic 128-bit load
}

__device__ __forceinline__ unsigned long long pack_range(long long cur, long long end)
{
    return (unsigned long long)(unsigned)cur | ((unsigned long long)(unsigned)end << 32);
}

// Sets the owner's cur and returns its current end.  Thieves only ever lower
// end, so the loop ends after at most one retry per successful split.
__device__ __noinline__ long long slot_publish(StealSlot *p, long long cur)
{
    StealSlot old = slot_read(p);
    for (int k = 0; k < 64; k++) {
        const StealSlot want{old.a, pack_range(cur, (long long)(old.b >> 32))};
        const StealSlot got = atomicCAS(p, old, want);
        if (same(got, old)) return (long long)(old.b >> 32);
        old = got;
    }
    // never reached in practice; the range read last is still a valid bound
    // (a thief that split after it redoes at most the same snapshots)
    return (long long)(old.b >> 32);
}

__device__ __forceinline__ void slot_start(StealSlot *p, long long item, long long cur,
                                           long long end)
{
    StealSlot old = slot_read(p);
    const StealSlot want{(unsigned long long)item + 1ull, pack_range(cur, end)};
    for (int k = 0; k < 64; k++) {
        const StealSlot got = atomicCAS(p, old, want);
        if (same(got, old)) return;
        old = got;
    }
}

__device__ __forceinline__ int scene_of_snap(const SceneDesc *desc, int n_scenes, long long T)
{
    int lo = 0, hi = n_scenes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (desc[mid].snap0 <= T) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int scene_of_item(const SceneDesc *desc, int n_scenes, long long it)
{
    int lo = 0, hi = n_scenes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (desc[mid].item0 <= it) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int scene_of_los(const SceneDesc *desc, int n_scenes, long long c)
{
    int lo = 0, hi = n_scenes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (desc[mid].los0 <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ bool in_range(long long x, long long y, long long z)
{
    return (x > -kCoordLimit) & (x < kCoordLimit) & (y > -kCoordLimit) & (y < kCoordLimit) &
           (z > -kCoordLimit) & (z < kCoordLimit);
}

// Packet of segments from (x, y, z) to samples of facets of word c.  Lane
// takes sample b of the packet's group gi (lanes gi*s2 .. gi*s2 + s2 - 1).
// Returns a lane mask in which a group has a set bit iff some segment of
// that group is unblocked (its facet is visible); bits of unblocked lanes
// are exact, a group settled by its probe keeps only the probe's bit.
// With the caches on, each lane first tests `tb`, the facet that hid its
// facet at the previous snapshot; then each group whose facet was visible
// at the previous snapshot through sample pf walks that one segment first,
// and if it is free the rest of the group is skipped.
template <bool CACHE, class LeafFn>
__device__ __forceinline__ unsigned table_packet(const DevScenes &g, const SceneDesc &D, bool mine,
                                                 int sidx, int lead, int x, int y, int z,
                                                 int tb, int pf, int gi, int b, int s2, int *err,
                                                 WalkCounters &wc, LeafFn leaf,
                                                 OccluderCache &cache, int &myblk)
{
    const int lane = threadIdx.x & 31;
    int qx = 0, qy = 0, qz = 0;
    if (mine) { qx = __ldg(g.sx + sidx); qy = __ldg(g.sy + sidx); qz = __ldg(g.sz + sidx); }
    unsigned alive = __ballot_sync(kFull, mine);
    wc.segments += mine;
    Seg sg = make_seg(x, y, z, qx, qy, qz);
    myblk = -1;
    const Leaf Lf = load_leaf(g.leaf, lead);
    const float dirx = (float)(2 * Lf.ox + Lf.ux + Lf.vx - 2 * x);
    const float diry = (float)(2 * Lf.oy + Lf.uy + Lf.vy - 2 * y);
    const float dirz = (float)(2 * Lf.oz + Lf.uz + Lf.vz - 2 * z);
    const int budget = D.budget;
    unsigned shown = 0;   // probe lanes found free
    if (CACHE) {
        bool hit = false;
        if (mine && tb >= 0) {
            wc.leaf_tests++;
            hit = leaf(sg, load_leaf(g.leaf, tb), wc);
        }
        if (hit) { myblk = tb; wc.cache_hits++; }
        alive &= ~__ballot_sync(kFull, hit);
        if (!alive) return 0;
        const bool probe = kTableProbe && mine && pf >= 0 && b == pf && ((alive >> lane) & 1u);
        const unsigned pm = __ballot_sync(kFull, probe);
        if (pm) {
            shown = pm & occlude<CACHE, LeafFn, false, kTableAbsBox>(
                             sg, pm, g.nodes, g.leaf, D.root, dirx, diry, dirz, budget, err, wc,
                             leaf, cache, myblk);
            // groups whose probe is free are visible: their other lanes need no walk
            const bool done = mine && pf >= 0 && ((shown >> (gi * s2 + pf)) & 1u);
            alive &= ~(__ballot_sync(kFull, done) | pm);
            if (!alive) return shown;
        }
    }
    return shown | occlude<CACHE, LeafFn, CACHE && kTableLru, kTableAbsBox>(
                       sg, alive, g.nodes, g.leaf, D.root, dirx, diry, dirz, budget, err, wc, leaf,
                       cache, myblk);
}

// Facets of word c (lanes with blk >= 0 hold a candidate blocker) that the
// blocker hides from both a = (ax, ay, az) and e = (ex, ey, ez), at every
// sample: their bits are set in the returned (warp-uniform) mask.
template <class LeafFn>
__device__ __noinline__ unsigned tile_hidden(const DevScenes &g, const SceneDesc &D, int c,
                                             int blk, const int *pa, const int *pe, int k,
                                             const int *sblk, WalkCounters &wc, LeafFn leaf)
{
    const int lane = threadIdx.x & 31;
    const int s2 = D.s * D.s;
    const int ax = k * pa[0], ay = k * pa[1], az = k * pa[2];   // in range: checked
    const int ex = k * pe[0], ey = k * pe[1], ez = k * pe[2];
    unsigned cm = __ballot_sync(kFull, blk >= 0);
    unsigned hidden = 0;
    while (cm) {
        if (s2 <= 32) {   // floor(32 / s2) facets per packet, lane = sample
            const int G = 32 / s2;
            const int cnt = min(G, __popc(cm));
            const int gi = lane / s2, b = lane - gi * s2;
            const bool mine = gi < cnt;
            unsigned m = cm;
            for (int q = 0; q < gi && q < 31; q++) m &= m - 1;
            const int jbit = mine ? __ffs(m) - 1 : 0;
            int tb = __shfl_sync(kFull, blk, jbit);
            if (sblk && mine && sblk[32 * jbit + b] >= 0) tb = sblk[32 * jbit + b];
            bool hit = true;
            if (mine) {
                const int si = D.sample0 + (32 * c + jbit) * s2 + b;
                const int qx = __ldg(g.sx + si), qy = __ldg(g.sy + si), qz = __ldg(g.sz + si);
                const Leaf F = load_leaf(g.leaf, tb);
                wc.leaf_tests += 2;
                hit = leaf(make_seg(ax, ay, az, qx, qy, qz), F, wc) &&
                      leaf(make_seg(ex, ey, ez, qx, qy, qz), F, wc);
            }
            const unsigned hm = __ballot_sync(kFull, hit);
            const unsigned smask = (s2 == 32) ? kFull : ((1u << s2) - 1u);
            const bool all = mine && ((hm >> (gi * s2)) & smask) == smask;
            hidden |= __reduce_or_sync(kFull, (all && b == 0) ? (1u << jbit) : 0u);
            for (int q = 0; q < cnt; q++) cm &= cm - 1;
        } else {          // one facet, 32 samples at a time
            const int jbit = __ffs(cm) - 1;
            cm &= cm - 1;
            const int tb = __shfl_sync(kFull, blk, jbit);
            const Leaf F = load_leaf(g.leaf, tb);
            bool all = true;
            for (int b0 = 0; b0 < s2 && all; b0 += 32) {
                const int b = b0 + lane;
                bool hit = true;
                if (b < s2) {
                    const int si = D.sample0 + (32 * c + jbit) * s2 + b;
                    const int qx = __ldg(g.sx + si), qy = __ldg(g.sy + si), qz = __ldg(g.sz + si);
                    wc.leaf_tests += 2;
                    hit = leaf(make_seg(ax, ay, az, qx, qy, qz), F, wc) &&
                          leaf(make_seg(ex, ey, ez, qx, qy, qz), F, wc);
                }
                all = __all_sync(kFull, hit);
            }
            if (all) hidden |= 1u << jbit;
        }
    }
    return hidden;
}

// Swept walk: the segments from the points a of [A, E] to q fill the
// triangle T = conv(A, E, q), and T lies in the segment [A, q] moved by
// every vector between 0 and E - A (per axis); so a box meets some open
// segment a-q only if segment A-q meets the box widened by that range.
struct SweepFilter {
    float lx, ly, lz, hx, hy, hz;   // lo -= max(0, E - A), hi -= min(0, E - A)
    __device__ __forceinline__ bool node(int) const { return true; }
    __device__ __forceinline__ void grow(float &ax, float &ay, float &az, float &bx, float &by,
                                         float &bz) const
    {
        // directed rounding keeps the widened box a superset
        ax = __fsub_rd(ax, lx); ay = __fsub_rd(ay, ly); az = __fsub_rd(az, lz);
        bx = __fadd_ru(bx, hx); by = __fadd_ru(by, hy); bz = __fadd_ru(bz, hz);
    }
};

// Leaf test of the swept walk: false only when facet F provably blocks no
// open segment a-q, a in [A, E] (the Seg holds A and q - A, the functor E).
// Along [A, E] the plane side n.(a - o) and the four edge orientations
// orient(a, f_k, f_k+1, q) are affine in a, so a sign shared by both ends
// holds all along.  F blocks a-q only if a is strictly on the other side of
// F's plane from q (or, with q on the plane, the segment lies in it) and the
// four edge orientations are all >= 0 or all <= 0.
struct SweepLeaf {
    int ex, ey, ez;
    __device__ __forceinline__ bool operator()(const Seg &s, const Leaf &L, WalkCounters &wc) const
    {
        const int qx = s.px + s.dx, qy = s.py + s.dy, qz = s.pz + s.dz;
        const long long sq = (long long)L.nx * (qx - L.ox) + (long long)L.ny * (qy - L.oy) +
                             (long long)L.nz * (qz - L.oz);
        const long long sa = (long long)L.nx * (s.px - L.ox) + (long long)L.ny * (s.py - L.oy) +
                             (long long)L.nz * (s.pz - L.oz);
        const long long se = (long long)L.nx * (ex - L.ox) + (long long)L.ny * (ey - L.oy) +
                             (long long)L.nz * (ez - L.oz);
        if (sq == 0) return !((sa > 0 && se > 0) || (sa < 0 && se < 0));
        if (sq > 0 ? (sa >= 0 && se >= 0) : (sa <= 0 && se <= 0)) return false;
        unsigned neg = 0xF, pos = 0xF;   // edges strictly negative / positive at both ends
        for (int end = 0; end < 2; end++) {
            const int px = end ? ex : s.px, py = end ? ey : s.py, pz = end ? ez : s.pz;
            const float dx = (float)(qx - px), dy = (float)(qy - py), dz = (float)(qz - pz);
            const float f0x = (float)(L.ox - px), f0y = (float)(L.oy - py), f0z = (float)(L.oz - pz);
            const float f1x = f0x + (float)L.ux, f1y = f0y + (float)L.uy, f1z = f0z + (float)L.uz;
            const float f2x = f1x + (float)L.vx, f2y = f1y + (float)L.vy, f2z = f1z + (float)L.vz;
            const float f3x = f0x + (float)L.vx, f3y = f0y + (float)L.vy, f3z = f0z + (float)L.vz;
            const int e0 = orient_filtered(f0x, f0y, f0z, f1x, f1y, f1z, dx, dy, dz);
            const int e1 = orient_filtered(f1x, f1y, f1z, f2x, f2y, f2z, dx, dy, dz);
            const int e2 = orient_filtered(f2x, f2y, f2z, f3x, f3y, f3z, dx, dy, dz);
            const int e3 = orient_filtered(f3x, f3y, f3z, f0x, f0y, f0z, dx, dy, dz);
            neg &= (e0 < 0) | ((e1 < 0) << 1) | ((e2 < 0) << 2) | ((e3 < 0) << 3);
            pos &= (e0 > 0) | ((e1 > 0) << 1) | ((e2 > 0) << 2) | ((e3 > 0) << 3);
        }
        (void)wc;
        return !(neg && pos);   // undecided signs (0) never rule a case out
    }
};

// Facets of word c (lanes with pf >= 0: seen through sample pf) that face
// both A = k pa and E = k pe strictly and whose segment to sample pf no facet
// can block from any point of [A, E]: visible at every snapshot of the
// stretch (facing is affine along [A, E] too).  One swept walk for the word.
__device__ __noinline__ unsigned tile_shown(const DevScenes &g, const SceneDesc &D, int c,
                                            int pf, const int *pa, const int *pe, int k, int *err,
                                            WalkCounters &wc)
{
    const int lane = threadIdx.x & 31;
    const int jl = 32 * c + lane;
    const int ax = k * pa[0], ay = k * pa[1], az = k * pa[2];   // in range: checked
    const int ex = k * pe[0], ey = k * pe[1], ez = k * pe[2];
    bool cand = false;
    int qx = 0, qy = 0, qz = 0;
    if (jl < D.n && pf >= 0) {
        const Leaf L = load_leaf(g.leaf, D.facet0 + jl);
        cand = front_of(L, ax, ay, az) && front_of(L, ex, ey, ez);
        const int si = D.sample0 + jl * D.s * D.s + pf;
        qx = __ldg(g.sx + si); qy = __ldg(g.sy + si); qz = __ldg(g.sz + si);
    }
    const unsigned pm = __ballot_sync(kFull, cand);
    if (!pm) return 0;
    Seg sg = make_seg(ax, ay, az, qx, qy, qz);
    finish_seg<kTableAbsBox>(sg);
    const int lead = __ffs(pm) - 1;
    const float dirx = (float)__shfl_sync(kFull, sg.dx, lead);
    const float diry = (float)__shfl_sync(kFull, sg.dy, lead);
    const float dirz = (float)__shfl_sync(kFull, sg.dz, lead);
    const int gx = ex - ax, gy = ey - ay, gz = ez - az;
    const SweepFilter f{(float)max(gx, 0), (float)max(gy, 0), (float)max(gz, 0),
                        (float)-min(gx, 0), (float)-min(gy, 0), (float)-min(gz, 0)};
    int blocker, myblk = -1;
    wc.segments += cand;
    return walk_packet<SweepLeaf, SweepFilter, kTableAbsBox>(sg, pm, g.nodes, g.leaf, D.root,
                                                             dirx, diry, dirz, D.budget, err, wc,
                                                             SweepLeaf{ex, ey, ez}, blocker,
                                                             myblk, f);
}

// True (warp-uniform) when every position of snapshots [t0, t1) is in range
// and lies on the segment from position t0 to position t1 - 1 (scaled by k).
__device__ __noinline__ bool tile_on_segment(const int *pos, long long t0, long long t1,
                                             long long k)
{
    const int lane = threadIdx.x & 31;
    const long long te = t1 - 1;
    const long long A0 = k * pos[3 * t0], A1 = k * pos[3 * t0 + 1], A2 = k * pos[3 * t0 + 2];
    const long long E0 = k * pos[3 * te], E1 = k * pos[3 * te + 1], E2 = k * pos[3 * te + 2];
    bool ok = in_range(A0, A1, A2) && in_range(E0, E1, E2);
    if (ok) {
        const long long d0 = E0 - A0, d1 = E1 - A1, d2 = E2 - A2;
        const long long dd = d0 * d0 + d1 * d1 + d2 * d2;
        for (long long t = t0 + lane; t < t1 && ok; t += 32) {
            const long long P0 = k * pos[3 * t], P1 = k * pos[3 * t + 1], P2 = k * pos[3 * t + 2];
            if (!in_range(P0, P1, P2)) {
                ok = false;
                break;
            }
            const long long p0 = P0 - A0, p1 = P1 - A1, p2 = P2 - A2;
            if (dd == 0) {
                ok = p0 == 0 && p1 == 0 && p2 == 0;
            } else {
                const long long dot = p0 * d0 + p1 * d1 + p2 * d2;
                ok = p1 * d2 == p2 * d1 && p2 * d0 == p0 * d2 && p0 * d1 == p1 * d0 &&
                     dot >= 0 && dot <= dd;
            }
        }
    }
    return __all_sync(kFull, ok);
}

// Snapshots [tb, te) of work item `item` (tb < 0: the item's whole tile).
// With a slot, the range's end is re-read from it at every stretch.
template <bool CACHE, class LeafFn>
__device__ __noinline__ void table_tile(const DevScenes &g, long long item, int TT, int PT,
                                           long long tb, long long te, StealSlot *slot,
                                           const int *rep, int *err, WalkCounters &wc,
                                           LeafFn leaf, OccluderCache &cache, int *sblk)
{
    const int lane = threadIdx.x & 31;
    const int sc = scene_of_item(g.desc, g.n_scenes, item);
    const SceneDesc &D = g.desc[sc];
    const long long local = item - D.item0;
    const long long per_side = (long long)D.W * D.ntiles;
    const int side = local >= per_side ? 1 : 0;
    const long long rem = local - side * per_side;
    const int c = (int)(rem / D.ntiles);
    long long t0 = (rem - (long long)c * D.ntiles) * TT;
    long long t1 = min(t0 + TT, D.nsnap);
    if (tb >= 0) {
        t0 = tb;
        t1 = te;
    } else if (slot && lane == 0) {
        slot_start(slot, item, t0, t1);
    }
    if (CACHE) cache.enter_scene(sc);
    const int *pos = side ? D.rx : D.tx;
    const int jl = 32 * c + lane;
    const bool has = jl < D.n;
    int fnx = 0, fny = 0, fnz = 0, fox = 0, foy = 0, foz = 0;
    if (has) {
        const Leaf L = load_leaf(g.leaf, D.facet0 + jl);
        fnx = L.nx; fny = L.ny; fnz = L.nz; fox = L.ox; foy = L.oy; foz = L.oz;
    }
    const int s2 = D.s * D.s;
    const long long k = 2LL * D.s;
    int prev_blk = -1;   // lane l: facet that last blocked facet 32c + l
    int prev_free = -1;  // lane l: sample of facet 32c + l seen at the previous snapshot
    // sblk[32 f + b]: the facet that last blocked sample b of facet 32c + f
    const bool per_sample = CACHE && kTableSampleBlockers && s2 <= 32;
    if (per_sample) {
        for (int i = lane; i < kSampleSlots; i += 32) sblk[i] = -1;
        __syncwarp();
    }
    for (long long u0 = t0; u0 < t1; u0 += PT) {   // straight-stretch proofs
        if (slot) {
            long long end = 0;
            if (lane == 0) end = slot_publish(slot, u0);
            t1 = min(t1, __shfl_sync(kFull, end, 0));
            if (u0 >= t1) break;
        }
        const long long u1 = min(u0 + (long long)PT, t1);
        if (rep) {   // a stretch whose rows are all copied later needs nothing
            bool traced = false;
            for (long long t = u0 + lane; t < u1; t += 32)
                traced |= rep[2 * (D.snap0 + t) + side] == t;
            if (!__any_sync(kFull, traced)) continue;
        }
        bool proof = CACHE && kTableTileProof && u1 - u0 >= 3 &&
                     tile_on_segment(pos, u0, u1, k);
        unsigned hidden = 0;   // facets settled hidden for snapshots [u0, u1)
        unsigned shown = 0;    // facets settled visible for snapshots [u0, u1)
        if (proof && u0 > t0) {
            // what the previous stretch left (each facet's blockers or free
            // sample) is tried first; the facets it settles need no snapshot
            hidden = tile_hidden(g, D, c, prev_free < 0 ? prev_blk : -1, pos + 3 * u0,
                                 pos + 3 * (u1 - 1), (int)k, per_sample ? sblk : nullptr, wc,
                                 leaf);
            if (kTableSweep)
                shown = tile_shown(g, D, c, prev_free, pos + 3 * u0, pos + 3 * (u1 - 1), (int)k,
                                   err, wc);
        }
        for (long long t = u0; t < u1; t++) {
            if (rep && rep[2 * (D.snap0 + t) + side] != t) continue;   // copied later
            uint32_t *row = D.table + ((size_t)t * 2 + side) * D.W;
            const long long X0 = k * pos[3 * t], X1 = k * pos[3 * t + 1], X2 = k * pos[3 * t + 2];
            if (!in_range(X0, X1, X2)) {
                if (lane == 0) {
                    raise_error(err, IVM_ERR_RANGE);
                    row[c] = 0u;
                }
                continue;
            }
            const int x = (int)X0, y = (int)X1, z = (int)X2;
            const bool fr = has && ((long long)fnx * (x - fox) + (long long)fny * (y - foy) +
                                    (long long)fnz * (z - foz)) > 0;
            unsigned fm = __ballot_sync(kFull, fr) & ~hidden & ~shown;
            unsigned word = shown;
            if (CACHE && kTableBatchProbe) {
                // one packet for the whole word: each facet seen at the previous
                // snapshot walks the segment to the sample it was seen through;
                // free ones are visible, the rest go on to their own packets
                const bool pr = ((fm >> lane) & 1u) && prev_free >= 0;
                const unsigned pm = __ballot_sync(kFull, pr);
                if (pm) {
                    int qx = 0, qy = 0, qz = 0;
                    if (pr) {
                        const int si = D.sample0 + jl * s2 + prev_free;
                        qx = __ldg(g.sx + si); qy = __ldg(g.sy + si); qz = __ldg(g.sz + si);
                    }
                    wc.segments += pr;
                    Seg sg = make_seg(x, y, z, qx, qy, qz);
                    const int lead = __ffs(pm) - 1;
                    const float dirx = (float)__shfl_sync(kFull, sg.dx, lead);
                    const float diry = (float)__shfl_sync(kFull, sg.dy, lead);
                    const float dirz = (float)__shfl_sync(kFull, sg.dz, lead);
                    int myblk = -1;
                    const unsigned freem = pm & occlude<CACHE, LeafFn, false, kTableAbsBox>(
                        sg, pm, g.nodes, g.leaf, D.root, dirx, diry, dirz, D.budget, err, wc,
                        leaf, cache, myblk);
                    word |= freem;
                    fm &= ~freem;
                    if (pr && !((freem >> lane) & 1u)) {
                        if (myblk >= 0) {
                            prev_blk = myblk;
                            if (per_sample) sblk[32 * lane + prev_free] = myblk;
                        }
                        prev_free = -1;
                    }
                    if (per_sample) __syncwarp();
                }
            }
            while (fm) {
                if (s2 <= 32) {
                    const int G = 32 / s2;
                    const int cnt = min(G, __popc(fm));
                    const int gi = lane / s2, b = lane - gi * s2;
                    const bool mine = gi < cnt;
                    unsigned m = fm;
                    for (int q = 0; q < gi && q < 31; q++) m &= m - 1;
                    const int jbit = mine ? __ffs(m) - 1 : 0;
                    const int sidx = D.sample0 + (32 * c + jbit) * s2 + b;
                    int tb = __shfl_sync(kFull, prev_blk, jbit);
                    if (per_sample && mine) {
                        const int v = sblk[32 * jbit + b];
                        if (v >= 0) tb = v;
                    }
                    const int pf = __shfl_sync(kFull, prev_free, jbit);
                    const int lead = D.facet0 + 32 * c + __shfl_sync(kFull, jbit, 0);
                    int myblk;
                    const unsigned alive = table_packet<CACHE>(g, D, mine, sidx, lead, x, y, z, tb,
                                                               pf, gi, b, s2, err, wc, leaf, cache,
                                                               myblk);
                    if (per_sample) {
                        if (mine && myblk >= 0) sblk[32 * jbit + b] = myblk;
                        __syncwarp();
                    }
                    const unsigned smask = (s2 == 32) ? kFull : ((1u << s2) - 1u);
                    const unsigned gbits = (alive >> (gi * s2)) & smask;
                    const bool gvis = mine && gbits != 0u;
                    word |= __reduce_or_sync(kFull, (gvis && b == 0) ? (1u << jbit) : 0u);
                    if (CACHE) {
                        // per facet: the blocker that hid it, or the sample it was seen through
                        const int fs = gvis ? __ffs(gbits) - 1 : -1;
                        for (int q = 0; q < cnt; q++) {
                            const int jb = __shfl_sync(kFull, jbit, q * s2);
                            const int nb = __shfl_sync(kFull, myblk, q * s2);
                            const int f1 = __shfl_sync(kFull, fs, q * s2);
                            if (lane == jb) {
                                prev_free = f1;
                                if (f1 < 0 && nb >= 0) prev_blk = nb;
                            }
                        }
                    }
                    for (int q = 0; q < cnt; q++) fm &= fm - 1;
                } else {
                    const int jbit = __ffs(fm) - 1;
                    fm &= fm - 1;
                    const int jlocal = 32 * c + jbit;
                    const int tb = __shfl_sync(kFull, prev_blk, jbit);
                    int last = -1;
                    bool vis = false;
                    for (int b0 = 0; b0 < s2; b0 += 32) {
                        const int b = b0 + lane;
                        int myblk;
                        const unsigned alive = table_packet<CACHE>(
                            g, D, b < s2, D.sample0 + jlocal * s2 + b, D.facet0 + jlocal, x, y, z,
                            tb, -1, 0, b, 32, err, wc, leaf, cache, myblk);
                        if (alive) {
                            vis = true;
                            break;
                        }
                        last = __shfl_sync(kFull, myblk, 0);
                    }
                    if (vis) word |= 1u << jbit;
                    else if (CACHE && lane == jbit && last >= 0) prev_blk = last;
                }
            }
            if (lane == 0) row[c] = word;
            if (proof && t + 2 < u1) {   // once, after the first traced snapshot
                proof = false;
                const bool open = !(((hidden | shown) >> lane) & 1u);   // not settled yet
                hidden |= tile_hidden(g, D, c, open && prev_free < 0 ? prev_blk : -1,
                                      pos + 3 * u0, pos + 3 * (u1 - 1), (int)k,
                                      per_sample ? sblk : nullptr, wc, leaf);
                if (kTableSweep)
                    shown |= tile_shown(g, D, c, open ? prev_free : -1, pos + 3 * u0,
                                        pos + 3 * (u1 - 1), (int)k, err, wc);
            }
        }
    }
    if (slot && lane == 0) slot_publish(slot, t1);   // done: nothing left to take
}

template <bool CACHE, class LeafFn>
__device__ __forceinline__ void los_item(const DevScenes &g, long long chunk, int *err,
                                         WalkCounters &wc, LeafFn leaf, OccluderCache &cache)
{
    const int lane = threadIdx.x & 31;
    const int sc = scene_of_los(g.desc, g.n_scenes, chunk);
    const SceneDesc &D = g.desc[sc];
    if (CACHE) cache.enter_scene(sc);
    const long long t = (chunk - D.los0) * 32 + lane;
    const bool valid = t < D.nsnap;
    const long long k = 2LL * D.s;
    long long a0 = 0, a1 = 0, a2 = 0, b0 = 0, b1 = 0, b2 = 0;
    if (valid) {
        a0 = k * D.tx[3 * t]; a1 = k * D.tx[3 * t + 1]; a2 = k * D.tx[3 * t + 2];
        b0 = k * D.rx[3 * t]; b1 = k * D.rx[3 * t + 1]; b2 = k * D.rx[3 * t + 2];
    }
    const bool ok = in_range(a0, a1, a2) & in_range(b0, b1, b2);
    if (valid && !ok) raise_error(err, IVM_ERR_RANGE);
    const bool same = (a0 == b0) & (a1 == b1) & (a2 == b2);
    const bool test = valid && ok && !same;
    unsigned alive = __ballot_sync(kFull, test);
    wc.segments += test;
    Seg sg = make_seg((int)a0, (int)a1, (int)a2, (int)b0, (int)b1, (int)b2);
    const int lead = __ffs(alive | 1u) - 1;
    const float dirx = (float)__shfl_sync(kFull, sg.dx, lead);
    const float diry = (float)__shfl_sync(kFull, sg.dy, lead);
    const float dirz = (float)__shfl_sync(kFull, sg.dz, lead);
    int myblk = -1;
    if (alive)
        alive = occlude<CACHE, LeafFn, CACHE, kTableAbsBox>(sg, alive, g.nodes, g.leaf, D.root,
                                                            dirx, diry, dirz, D.budget, err, wc,
                                                            leaf, cache, myblk);
    if (valid) D.los[t] = (uint8_t)((ok && same) || ((alive >> lane) & 1u));
}

// Items [0, total_items) are table tiles; the next total_los_chunks are LoS.
// Register cap of the table kernel: 4 resident blocks of 128 threads.  A
// sweep of 4-8 on the district gave the same times at fixed launch shapes
// (the kernel is bound by its work items' latency, not by resident warps),
// and 4 keeps the per-snapshot state in registers (8 spills 1.5 KB a thread).
#ifndef IVM_TABLE_MIN_BLOCKS
#define IVM_TABLE_MIN_BLOCKS 4
#endif
constexpr int kTableMinBlocks = IVM_TABLE_MIN_BLOCKS;

// A warp whose queue is empty: take the back half of the largest remaining
// range (at least two stretches) in a window of slots, do it, and look again;
// exit when a full scan finds no range worth splitting.  Windows start at a
// pseudo-random slot per warp and round, so that idle warps spread over the
// busy ones instead of all racing for the same range.  The scan's plain
// loads may be stale or torn: they only propose the compare value of the
// swap, which then fails.
constexpr int kStealWindow = 256;
// The smallest remaining range worth splitting is two stretches (2 PT).

template <bool CACHE, class LeafFn>
__device__ __forceinline__ void steal_loop(const DevScenes &g, int TT, int PT, StealSlot *slots,
                                           StealSlot *mine, const int *rep, int *err,
                                           WalkCounters &wc, LeafFn leaf, OccluderCache &cache,
                                           int *sblk)
{
    const int lane = threadIdx.x & 31;
    const int nslots = (int)(gridDim.x * (blockDim.x >> 5));
    const unsigned me = (unsigned)(mine - slots);
    bool full = nslots <= kStealWindow;   // the next scan covers every slot
    for (int round = 0; round < (1 << 20); round++) {
        long long best_rem = 0;
        int best = -1;
        unsigned long long sa = 0, sb = 0;
        unsigned h = (me + 1u) * 0x9E3779B1u ^ (unsigned)round * 0x85EBCA77u;
        h ^= h >> 15;
        h *= 0x2C1B3C6Du;
        h ^= h >> 12;
        const int start = full ? 0 : (int)(h % (unsigned)nslots);
        const int span = full ? nslots : kStealWindow;
        for (int k = lane; k < span; k += 32) {
            int i = start + k;
            if (i >= nslots) i -= nslots;
            const unsigned long long a = __ldcg(&slots[i].a), b = __ldcg(&slots[i].b);
            const long long rem = (long long)(b >> 32) - (long long)(unsigned)b;
            if (a != 0ull && rem > best_rem) {
                best_rem = rem;
                best = i;
                sa = a;
                sb = b;
            }
        }
        for (int o = 16; o; o >>= 1) {   // largest remaining range over the warp
            const long long r2 = __shfl_xor_sync(kFull, best_rem, o);
            const int i2 = __shfl_xor_sync(kFull, best, o);
            const unsigned long long a2 = __shfl_xor_sync(kFull, sa, o);
            const unsigned long long b2 = __shfl_xor_sync(kFull, sb, o);
            if (r2 > best_rem || (r2 == best_rem && i2 > best)) {
                best_rem = r2; best = i2; sa = a2; sb = b2;
            }
        }
        if (best_rem < 2LL * PT) {
            if (full) return;
            full = true;   // nothing in this window: look at all slots once
            continue;
        }
        full = nslots <= kStealWindow;
        const long long cur = (long long)(unsigned)sb, end = (long long)(sb >> 32);
        const long long half = best_rem / 2;
        const long long mid = cur + (half + PT - 1) / PT * PT;
        bool ok = false;
        if (lane == 0) {
            const StealSlot seen{sa, sb};
            ok = same(atomicCAS(&slots[best], seen, StealSlot{sa, pack_range(cur, mid)}), seen);
            if (ok) slot_start(mine, (long long)sa - 1, mid, end);
        }
        if (!__shfl_sync(kFull, ok, 0)) continue;
        table_tile<CACHE>(g, (long long)sa - 1, TT, PT, mid, end, mine, rep, err, wc, leaf,
                          cache, sblk);
    }
}

template <bool PERSIST, bool CACHE, class LeafFn>
__global__ void __launch_bounds__(kTravThreads, kTableMinBlocks)
k_table(DevScenes g, long long total_items, long long all_items, int TT, int PT,
                        const int *rep, unsigned long long *work, StealSlot *slots,
                        unsigned long long *ctr, int *err)
{
    extern __shared__ int smem_blk[];
    WalkCounters wc;
    LeafFn leaf;
    OccluderCache cache;
    const int lane = threadIdx.x & 31;
    int *sblk = CACHE ? smem_blk + (threadIdx.x >> 5) * kSampleSlots : nullptr;
    StealSlot *mine = (PERSIST && slots)
                          ? slots + (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)
                          : nullptr;
    auto run = [&](long long it) {
        if (it < total_items)
            table_tile<CACHE>(g, it, TT, PT, -1, -1, mine, rep, err, wc, leaf, cache, sblk);
        else los_item<CACHE>(g, it - total_items, err, wc, leaf, cache);
    };
    if (!PERSIST) {
        long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        if (w < all_items) run(w);
    } else {
        for (;;) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(work, 1ull);
            base = __shfl_sync(kFull, base, 0);
            if ((long long)base >= all_items) break;
            run((long long)base);
        }
        if (mine) steal_loop<CACHE>(g, TT, PT, slots, mine, rep, err, wc, leaf, cache, sblk);
    }
    flush_counters(wc, ctr);
}

// ------------------------------------------------------------ deduplication

// One block of 1024 threads per (scene, side): rep[2 T + side] = local index
// of the first snapshot of the run of equal positions containing t.  Each
// thread scans a contiguous chunk; a block max-scan joins the chunks.
__global__ void k_runs(DevScenes g, int *rep)
{
    __shared__ long long carry[1024];
    const SceneDesc D = g.desc[blockIdx.x];
    const int side = blockIdx.y;
    const long long S = D.nsnap;
    if (S == 0) return;
    const int *X = side ? D.rx : D.tx;
    const long long per = (S + 1023) / 1024;
    const long long b = threadIdx.x * per, e = min(b + per, S);
    long long last = -1;
    for (long long t = b; t < e; t++) {
        bool start = t == 0 || X[3 * t] != X[3 * t - 3] || X[3 * t + 1] != X[3 * t - 2] ||
                     X[3 * t + 2] != X[3 * t - 1];
        if (start) last = t;
    }
    carry[threadIdx.x] = last;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {   // inclusive max-scan of chunk results
        long long v = threadIdx.x >= o ? carry[threadIdx.x - o] : -1;
        __syncthreads();
        if (v > carry[threadIdx.x]) carry[threadIdx.x] = v;
        __syncthreads();
    }
    long long run = threadIdx.x > 0 ? carry[threadIdx.x - 1] : -1;
    for (long long t = b; t < e; t++) {
        bool start = t == 0 || X[3 * t] != X[3 * t - 3] || X[3 * t + 1] != X[3 * t - 2] ||
                     X[3 * t + 2] != X[3 * t - 1];
        if (start) run = t;
        rep[2 * (D.snap0 + t) + side] = (int)run;
    }
}

// Warp per (snapshot, side): copy the run's first row when this row is a copy.
__global__ void k_copy_rows(DevScenes g, long long total_snap, const int *rep,
                            unsigned long long *ctr)
{
    const long long item = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (item >= 2 * total_snap) return;
    const long long T = item >> 1;
    const int side = (int)(item & 1);
    const SceneDesc &D = g.desc[scene_of_snap(g.desc, g.n_scenes, T)];
    const long long t = T - D.snap0;
    const long long r = rep[item];
    if (r == t) return;
    const uint32_t *srcrow = D.table + ((size_t)r * 2 + side) * D.W;
    uint32_t *dst = D.table + ((size_t)t * 2 + side) * D.W;
    for (int c = lane; c < D.W; c += 32) dst[c] = srcrow[c];
    if (lane == 0) atomicAdd(ctr + C_DEDUP_ROWS, 1ull);
}

// ------------------------------------------------------------ launchers

template <bool PERSIST, bool CACHE, class LeafFn>
static void launch_one(const DevScenes &g, long long items, long long all, int TT,
                       const LaunchCfg &cfg, const int *rep, unsigned long long *work,
                       unsigned long long *ctr, int *err, cudaStream_t st)
{
    const int threads = 32 * cfg.warps_per_block;
    auto kern = k_table<PERSIST, CACHE, LeafFn>;
    const size_t smem = CACHE ? sizeof(int) * kSampleSlots * cfg.warps_per_block : 0;
    if (PERSIST) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
        int blocks = cfg.n_sm * (per_sm > 0 ? per_sm : 1);
        cudaMemsetAsync(work, 0, sizeof(unsigned long long), st);
        // one slot per warp of the grid (the context holds 64 per SM)
        StealSlot *slots = nullptr;
        const long long warps = (long long)blocks * cfg.warps_per_block;
        if (cfg.steal && warps <= 64LL * cfg.n_sm) {
            slots = static_cast<StealSlot *>(cfg.steal);
            cudaMemsetAsync(slots, 0, sizeof(StealSlot) * (size_t)warps, st);
        }
        kern<<<blocks, threads, smem, st>>>(g, items, all, TT, cfg.proof_tile, rep, work, slots,
                                            ctr, err);
    } else {
        long long blocks = (all + cfg.warps_per_block - 1) / cfg.warps_per_block;
        kern<<<(unsigned)blocks, threads, smem, st>>>(g, items, all, TT, cfg.proof_tile, rep, work,
                                                      nullptr, ctr, err);
    }
}

template <class LeafFn>
static void launch_leaf(const DevScenes &g, long long items, long long all, int TT,
                        const LaunchCfg &cfg, const int *rep, unsigned long long *work,
                        unsigned long long *ctr, int *err, cudaStream_t st)
{
    if (cfg.persistent) {
        if (cfg.cache) launch_one<true, true, LeafFn>(g, items, all, TT, cfg, rep, work, ctr, err, st);
        else launch_one<true, false, LeafFn>(g, items, all, TT, cfg, rep, work, ctr, err, st);
    } else {
        if (cfg.cache) launch_one<false, true, LeafFn>(g, items, all, TT, cfg, rep, work, ctr, err, st);
        else launch_one<false, false, LeafFn>(g, items, all, TT, cfg, rep, work, ctr, err, st);
    }
}

cudaError_t launch_table(const DevScenes &g, long long total_snap, long long total_items,
                         long long total_los_chunks, int snap_tile, const LaunchCfg &cfg,
                         int *rep, unsigned long long *work, unsigned long long *ctr, int *err,
                         cudaStream_t st)
{
    const long long all = total_items + total_los_chunks;
    if (all == 0) return cudaSuccess;
    int launched = 1;
    if (cfg.dedup) {
        k_runs<<<dim3(g.n_scenes, 2), 1024, 0, st>>>(g, rep);
        launched++;
    }
    const int *r = cfg.dedup ? rep : nullptr;
    if (cfg.mode == IVM_MODE_EXACT)
        launch_leaf<ExactLeaf>(g, total_items, all, snap_tile, cfg, r, work, ctr, err, st);
    else if (cfg.aligned)
        launch_leaf<AlignedLeafCall>(g, total_items, all, snap_tile, cfg, r, work, ctr, err, st);
    else
        launch_leaf<FilteredLeafCall>(g, total_items, all, snap_tile, cfg, r, work, ctr, err, st);
    if (cfg.dedup && total_snap > 0) {
        long long warps = 2 * total_snap;
        k_copy_rows<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(g, total_snap, rep, ctr);
        launched++;
    }
    note_launches(launched);
    return cudaGetLastError();
}

}  // namespace ivm
