// traverse.cuh -- the occlusion test ("intersection judgment", Abstract and
// Sec. II-B of the paper) on the GPU: a segment against the closed facets of
// a scene, through its BVH, one warp at a time.
//
// A warp holds a packet of up to 32 segments (one per lane) that start and end
// near each other (sample pairs of one facet pair, or samples of one facet
// seen from one point).  The warp walks the BVH together: a node is entered
// when any still-unblocked lane's segment touches the node's box, and a lane
// drops out of the packet at the first facet that blocks it.  The walk stops
// early when every lane is blocked.
//
// Exactness.  Box tests only cull: they are conservative (a box the segment
// touches is never culled; a near miss may be kept).  Every facet decision is
// exact: integer plane sides and edge orientations (int64 / int128), or the
// FP32 filter of filter.cuh that falls back to them when it cannot decide.
#pragma once

#include "ivm_internal.cuh"

namespace ivm {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kBig = 3.0e38f;

// One lane's segment P -> Q = P + d (scaled integer coordinates).
struct Seg {
    int px, py, pz;
    int dx, dy, dz;
    float ix, iy, iz;     // round-to-nearest reciprocal of d; 2^100 where d == 0
    float fx, fy, fz;     // box-test offsets: P as float (relative form), rn(-P i) (absolute)
    float w;              // absolute form: widening of the box test
};

// The reciprocals are only needed by box tests; finish_seg computes them
// right before a BVH walk, so segments settled by cached occluders skip it.
__device__ __forceinline__ Seg make_seg(int px, int py, int pz, int qx, int qy, int qz)
{
    Seg s;
    s.px = px; s.py = py; s.pz = pz;
    s.dx = qx - px; s.dy = qy - py; s.dz = qz - pz;
    s.ix = s.iy = s.iz = 0.f;
    s.fx = s.fy = s.fz = 0.f;
    s.w = 0.f;
    return s;
}

template <bool ABS = false>
__device__ __forceinline__ void finish_seg(Seg &s)
{
    s.ix = s.dx ? __frcp_rn((float)s.dx) : 0x1p100f;
    s.iy = s.dy ? __frcp_rn((float)s.dy) : 0x1p100f;
    s.iz = s.dz ? __frcp_rn((float)s.dz) : 0x1p100f;
    if (ABS) {
        s.fx = __fmul_rn(-(float)s.px, s.ix);
        s.fy = __fmul_rn(-(float)s.py, s.iy);
        s.fz = __fmul_rn(-(float)s.pz, s.iz);
        // an axis with d == 0 has an exact offset (p times a power of two)
        const float e = fmaxf(fmaxf(s.dx ? fabsf(s.fx) : 0.f, s.dy ? fabsf(s.fy) : 0.f),
                              s.dz ? fabsf(s.fz) : 0.f);
        s.w = __fmaf_rn(e, 0x1p-22f, 0x1p-19f);
    } else {
        s.fx = (float)s.px; s.fy = (float)s.py; s.fz = (float)s.pz;
    }
}

// Conservative segment-box test: true whenever the open segment touches the
// closed box.  Boxes are stored enlarged by half a unit (integer bound -/+
// 0.5; exact in float below 2^23) and only ever widened further, so no box
// plane equals a coordinate of P.  That gives the d = 0 axes their answer
// without a branch: with 1/d replaced by 2^100, an axis where the segment
// lies inside the slab gives (-huge, +huge) and one where it lies outside
// gives an entry above 1 or an exit below 0.
//
// Relative form: for d != 0, (l - p) is exact and the product with the
// rounded reciprocal has relative error below 2^-23; widening entry and exit
// by 2^-20 of their magnitude makes the test a superset of the exact one.
//
// Absolute form: one FMA per plane, a = rn(l i + o) with o = rn(-p i).  With
// t = (l - p) / d, a differs from t by at most 2^-23 |t| + 2^-24 |p i| (both
// to first order; o is exact on d = 0 axes).  If the exact segment meets the
// box at some t in (0, 1), every axis's entry is at most t + e1 and every
// exit at least t - e1, with e1 = 2^-23 + 2^-24 max |p i| (entries below 0
// and exits above 1 only move further away, and the clamps to [0, 1] keep
// t inside), so entry <= exit + 2 e1; w = 2^-19 + 2^-22 max |o| covers 2 e1,
// the rounding of o and the rounding of exit + w.
template <bool ABS = false>
__device__ __forceinline__ bool seg_box(const Seg &s, float lx, float ly, float lz, float hx,
                                        float hy, float hz)
{
    if (ABS) {
        float ax = __fmaf_rn(lx, s.ix, s.fx), bx = __fmaf_rn(hx, s.ix, s.fx);
        float ay = __fmaf_rn(ly, s.iy, s.fy), by = __fmaf_rn(hy, s.iy, s.fy);
        float az = __fmaf_rn(lz, s.iz, s.fz), bz = __fmaf_rn(hz, s.iz, s.fz);
        float tn = fmaxf(fmaxf(fminf(ax, bx), fminf(ay, by)), fmaxf(fminf(az, bz), 0.f));
        float tf = fminf(fminf(fmaxf(ax, bx), fmaxf(ay, by)), fminf(fmaxf(az, bz), 1.f));
        return tn <= __fadd_rn(tf, s.w);
    }
    float ax = __fmul_rn(lx - s.fx, s.ix), bx = __fmul_rn(hx - s.fx, s.ix);
    float ay = __fmul_rn(ly - s.fy, s.iy), by = __fmul_rn(hy - s.fy, s.iy);
    float az = __fmul_rn(lz - s.fz, s.iz), bz = __fmul_rn(hz - s.fz, s.iz);
    float tn = fmaxf(fmaxf(fminf(ax, bx), fminf(ay, by)), fminf(az, bz));
    float tf = fminf(fminf(fmaxf(ax, bx), fmaxf(ay, by)), fmaxf(az, bz));
    float tnw = tn - fabsf(tn) * 0x1p-20f;
    float tfw = tf + fabsf(tf) * 0x1p-20f;
    return (tnw <= tfw) & (tnw < 1.f) & (tfw > 0.f);
}

// ------------------------------------------------------------ exact facet test

__device__ __forceinline__ int sgn_ll(long long v) { return (v > 0) - (v < 0); }

// sign(d . (a x b)); a, b, d have int32 components below 2^23 in magnitude,
// so a x b fits int64 (< 2^47) and the dot needs int128 (< 2^72).
__device__ __forceinline__ int orient_sign(int ax, int ay, int az, int bx, int by, int bz,
                                           int dx, int dy, int dz)
{
    long long cx = (long long)ay * bz - (long long)az * by;
    long long cy = (long long)az * bx - (long long)ax * bz;
    long long cz = (long long)ax * by - (long long)ay * bx;
    __int128 r = (__int128)cx * dx + (__int128)cy * dy + (__int128)cz * dz;
    return (r > 0) - (r < 0);
}

// Segment lying in the facet's plane: clip l in [0,1] against the four edge
// half-planes of the parallelogram, projected along its normal's dominant
// axis; bounds are kept as exact fractions.  Open segment meets the closed
// facet iff lo <= hi, lo < 1 and hi > 0.
// (Arguments by value: the segment and the facet stay in registers in the
// caller; only this rare path pays for the call.)
// Also gives the clip interval's lower end lo = lon / lod (lod > 0, lo >= 0):
// the first parameter at which the segment is inside the facet.
static __device__ __noinline__ bool coplanar_clip_v(int px, int py, int pz, int dx, int dy, int dz,
                                                    int ox, int oy, int oz, int ux, int uy, int uz,
                                                    int vx, int vy, int vz, int dom,
                                                    long long *lo_num, long long *lo_den)
{
    dom &= 3;   // bit 2 marks axis-aligned rectangles
    int a0 = dom == 0 ? 1 : 0;
    int a1 = dom == 2 ? 1 : 2;
    auto pick = [](int x, int y, int z, int a) { return a == 0 ? x : (a == 1 ? y : z); };
    long long P0 = pick(px, py, pz, a0), P1 = pick(px, py, pz, a1);
    long long D0 = pick(dx, dy, dz, a0), D1 = pick(dx, dy, dz, a1);
    long long O0 = pick(ox, oy, oz, a0), O1 = pick(ox, oy, oz, a1);
    long long U0 = pick(ux, uy, uz, a0), U1 = pick(ux, uy, uz, a1);
    long long V0 = pick(vx, vy, vz, a0), V1 = pick(vx, vy, vz, a1);
    int sig = sgn_ll(U0 * V1 - U1 * V0);      // != 0: the dominant normal component
    long long cx[4] = {O0, O0 + U0, O0 + U0 + V0, O0 + V0};
    long long cy[4] = {O1, O1 + U1, O1 + U1 + V1, O1 + V1};
    long long ex[4] = {U0, V0, -U0, -V0};
    long long ey[4] = {U1, V1, -U1, -V1};
    long long lon = 0, lod = 1, hin = 1, hid = 1;
    for (int k = 0; k < 4; k++) {
        long long al = sig * (ex[k] * (P1 - cy[k]) - ey[k] * (P0 - cx[k]));
        long long be = sig * (ex[k] * D1 - ey[k] * D0);
        if (be > 0) {            // l >= -al / be
            if ((__int128)(-al) * lod > (__int128)lon * be) { lon = -al; lod = be; }
        } else if (be < 0) {     // l <= al / (-be)
            if ((__int128)al * hid < (__int128)hin * (-be)) { hin = al; hid = -be; }
        } else if (al < 0) {
            return false;
        }
    }
    *lo_num = lon;
    *lo_den = lod;
    return ((__int128)lon * hid <= (__int128)hin * lod) && (lon < lod) && (hin > 0);
}

static __device__ __noinline__ bool coplanar_hit_v(int px, int py, int pz, int dx, int dy, int dz,
                                                   int ox, int oy, int oz, int ux, int uy, int uz,
                                                   int vx, int vy, int vz, int dom)
{
    long long n, d;
    return coplanar_clip_v(px, py, pz, dx, dy, dz, ox, oy, oz, ux, uy, uz, vx, vy, vz, dom, &n,
                           &d);
}

__device__ __forceinline__ bool coplanar_hit(const Seg &s, const Leaf &L)
{
    return coplanar_hit_v(s.px, s.py, s.pz, s.dx, s.dy, s.dz, L.ox, L.oy, L.oz, L.ux, L.uy, L.uz,
                          L.vx, L.vy, L.vz, L.dom);
}

// Exact: does the open segment s meet the closed facet L?
__device__ __forceinline__ bool facet_hit_exact(const Seg &s, const Leaf &L)
{
    long long rx = s.px - L.ox, ry = s.py - L.oy, rz = s.pz - L.oz;
    long long sp = (long long)L.nx * rx + (long long)L.ny * ry + (long long)L.nz * rz;
    long long sd = (long long)L.nx * s.dx + (long long)L.ny * s.dy + (long long)L.nz * s.dz;
    int a = sgn_ll(sp), b = sgn_ll(sp + sd);
    if (a == b) return a == 0 ? coplanar_hit(s, L) : false;
    if (a == 0 || b == 0) return false;      // touches the plane only at an endpoint
    // corners relative to P, in cyclic order O, O+U, O+U+V, O+V
    int c0x = L.ox - s.px, c0y = L.oy - s.py, c0z = L.oz - s.pz;
    int c1x = c0x + L.ux, c1y = c0y + L.uy, c1z = c0z + L.uz;
    int c2x = c1x + L.vx, c2y = c1y + L.vy, c2z = c1z + L.vz;
    int c3x = c0x + L.vx, c3y = c0y + L.vy, c3z = c0z + L.vz;
    int e0 = orient_sign(c0x, c0y, c0z, c1x, c1y, c1z, s.dx, s.dy, s.dz);
    int e1 = orient_sign(c1x, c1y, c1z, c2x, c2y, c2z, s.dx, s.dy, s.dz);
    int e2 = orient_sign(c2x, c2y, c2z, c3x, c3y, c3z, s.dx, s.dy, s.dz);
    int e3 = orient_sign(c3x, c3y, c3z, c0x, c0y, c0z, s.dx, s.dy, s.dz);
    bool nonneg = (e0 >= 0) & (e1 >= 0) & (e2 >= 0) & (e3 >= 0);
    bool nonpos = (e0 <= 0) & (e1 <= 0) & (e2 <= 0) & (e3 <= 0);
    return nonneg | nonpos;
}

// Exact test for an axis-aligned rectangle facet (normal along axis K, U and V
// along the other two axes): the same answer as facet_hit_exact.  The open
// segment P -> P + d meets the closed rectangle when P and P + d lie strictly
// on opposite sides of the plane x_K = O_K and the crossing point lies in the
// rectangle's closed range on both other axes; with sp = P_K - O_K the
// crossing is at P + (|sp| / |d_K|) d, so on axis m the condition is
//   (lo_m - P_m) |d_K| <= |sp| d_m <= (hi_m - P_m) |d_K|,
// products of integers below 2^23 in magnitude, exact in int64.  A segment
// in the plane goes to the coplanar clip; touching the plane at one end only
// is no hit (open segment).
template <int K>
__device__ __forceinline__ bool aligned_hit_k(const Seg &s, const Leaf &L)
{
    constexpr int K1 = (K + 1) % 3, K2 = (K + 2) % 3;
    const int P[3] = {s.px, s.py, s.pz}, D[3] = {s.dx, s.dy, s.dz};
    const int O[3] = {L.ox, L.oy, L.oz};
    const int E[3] = {L.ux + L.vx, L.uy + L.vy, L.uz + L.vz};   // far corner - O
    const int sp = P[K] - O[K], sq = sp + D[K];
    if ((sp > 0 && sq > 0) || (sp < 0 && sq < 0)) return false;
    if (sp == 0 || sq == 0) return (sp == 0 && sq == 0) ? coplanar_hit(s, L) : false;
    const long long a = sp < 0 ? -sp : sp, b = D[K] < 0 ? -D[K] : D[K];
    const int lo1 = min(O[K1], O[K1] + E[K1]) - P[K1], hi1 = max(O[K1], O[K1] + E[K1]) - P[K1];
    const int lo2 = min(O[K2], O[K2] + E[K2]) - P[K2], hi2 = max(O[K2], O[K2] + E[K2]) - P[K2];
    const long long t1 = a * D[K1], t2 = a * D[K2];
    return ((long long)lo1 * b <= t1) & (t1 <= (long long)hi1 * b) & ((long long)lo2 * b <= t2) &
           (t2 <= (long long)hi2 * b);
}

// The facet test for facets marked axis-aligned (Leaf.dom bit 2).
__device__ __forceinline__ bool aligned_hit(const Seg &s, const Leaf &L)
{
    const int k = L.dom & 3;
    if (k == 0) return aligned_hit_k<0>(s, L);
    if (k == 1) return aligned_hit_k<1>(s, L);
    return aligned_hit_k<2>(s, L);
}

// Strict facing test: (u x v) . (x - O) > 0, exact in int64 (|n| < 2^31).
__device__ __forceinline__ bool front_of(const Leaf &L, int x, int y, int z)
{
    long long v = (long long)L.nx * (x - L.ox) + (long long)L.ny * (y - L.oy) +
                  (long long)L.nz * (z - L.oz);
    return v > 0;
}

__device__ __forceinline__ Leaf load_leaf(const Leaf *leaves, int g)
{
    const int4 *p = reinterpret_cast<const int4 *>(leaves + g);
    int4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2), d = __ldg(p + 3);
    Leaf L;
    L.ox = a.x; L.oy = a.y; L.oz = a.z; L.building = a.w;
    L.ux = b.x; L.uy = b.y; L.uz = b.z; L.scene = b.w;
    L.vx = c.x; L.vy = c.y; L.vz = c.z; L.dom = c.w;
    L.nx = d.x; L.ny = d.y; L.nz = d.z; L.pad = d.w;
    return L;
}

// ------------------------------------------------------------ packet walk

// Per-lane test counts, summed over the warp and flushed once per kernel.
// A lane does far fewer than 2^32 tests in one launch.
struct WalkCounters {
    unsigned node_tests = 0, leaf_tests = 0, undecided = 0, exact = 0, segments = 0,
             cache_hits = 0, ranker_hits = 0, ranker_hits8 = 0;
};

// Traversal kernels run 128-thread blocks; the minimum-blocks hint caps
// registers so that more warps per scheduler hide the latency of the
// dependent box-test chains.
constexpr int kTravThreads = 128;
#ifndef IVM_MIN_BLOCKS
#define IVM_MIN_BLOCKS 4
#endif

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ void flush_counters(const WalkCounters &wc, unsigned long long *ctr)
{
    unsigned long long a = warp_sum(wc.node_tests), b = warp_sum(wc.leaf_tests),
                       c = warp_sum(wc.undecided), d = warp_sum(wc.exact),
                       e = warp_sum(wc.segments), f = warp_sum(wc.cache_hits),
                       h = warp_sum(wc.ranker_hits), h8 = warp_sum(wc.ranker_hits8);
    if ((threadIdx.x & 31) == 0) {
        if (f) atomicAdd(ctr + C_CACHE_HITS, f);
        if (h) atomicAdd(ctr + C_RANKER_HITS, h);
        if (h8) atomicAdd(ctr + C_RANKER_HITS8, h8);
        if (a) atomicAdd(ctr + C_NODE_TESTS, a);
        if (b) atomicAdd(ctr + C_LEAF_TESTS, b);
        if (c) atomicAdd(ctr + C_UNDECIDED, c);
        if (d) atomicAdd(ctr + C_EXACT_TESTS, d);
        if (e) atomicAdd(ctr + C_SEGMENTS, e);
    }
}

// Walks the BVH for the packet.  Must be called by all 32 lanes with the
// same `alive` (lanes whose segment takes part).  Returns the lanes whose
// segment no facet blocks.  LeafFn(seg, leaf, counters) -> bool hit.
// (dirx, diry, dirz) is a packet direction used to visit the nearer child
// first.  `budget` bounds the number of steps (a valid tree needs at most
// 2 * nodes + 2); when it runs out, IVM_ERR_TIMEOUT is raised.
// `root` may be any node (or ~facet), so a walk can cover one subtree.
// Walk filters: filt.node(index) says whether the walk enters an internal
// node, filt.grow widens each child box before its test; NoFilter enters
// every node and keeps the boxes.
struct NoFilter {
    __device__ __forceinline__ bool node(int) const { return true; }
    // widen a child box before it is tested (swept walks)
    __device__ __forceinline__ void grow(float &, float &, float &, float &, float &,
                                         float &) const {}
};

template <class LeafFn, class Filter = NoFilter, bool ABS = false>
__device__ __forceinline__ unsigned walk_packet(const Seg &s, unsigned alive, const Node *nodes,
                                                const Leaf *leaves, int root, float dirx,
                                                float diry, float dirz, int budget, int *err,
                                                WalkCounters &wc, LeafFn leaf_hit, int &blocker,
                                                int &myblk, Filter filt = Filter())
{
    const int lane = threadIdx.x & 31;
    int s0 = 0, s1 = 0, sp = 0;   // stack: entry k lives in lane k&31 of s0 / s1
    int node = root;
    blocker = -1;                 // warp-uniform: the last facet that blocked any lane
    while (alive) {
        if (--budget < 0) {
            if (lane == 0) raise_error(err, IVM_ERR_TIMEOUT);
            return 0;
        }
        bool have_next = false;
        if (node < 0) {
            const Leaf L = load_leaf(leaves, ~node);
            bool me = (alive >> lane) & 1u;
            bool hit = me && leaf_hit(s, L, wc);
            wc.leaf_tests += me;
            const unsigned hm = __ballot_sync(kFull, hit);
            if (hm) blocker = ~node;
            if (hit) myblk = ~node;   // per lane: the facet that blocked this segment
            alive &= ~hm;
        } else {
            const float4 *np = reinterpret_cast<const float4 *>(nodes + node);
            float4 A = __ldg(np), B = __ldg(np + 1), C = __ldg(np + 2);
            int4 D = __ldg(reinterpret_cast<const int4 *>(np + 3));
            bool me = ((alive >> lane) & 1u) && filt.node(node);
            filt.grow(A.x, A.y, A.z, A.w, B.x, B.y);
            filt.grow(B.z, B.w, C.x, C.y, C.z, C.w);
            bool hl = me && seg_box<ABS>(s, A.x, A.y, A.z, A.w, B.x, B.y);
            bool hr = me && seg_box<ABS>(s, B.z, B.w, C.x, C.y, C.z, C.w);
            wc.node_tests += 2 * me;
            unsigned ml = __ballot_sync(kFull, hl), mr = __ballot_sync(kFull, hr);
            if (ml && mr) {
                // nearer child first along the packet direction
                float kl = (A.x + A.w) * dirx + (A.y + B.x) * diry + (A.z + B.y) * dirz;
                float kr = (B.z + C.y) * dirx + (B.w + C.z) * diry + (C.x + C.w) * dirz;
                int first = kl <= kr ? D.x : D.y, second = kl <= kr ? D.y : D.x;
                if (sp >= kStackDepth) {
                    if (lane == 0) raise_error(err, IVM_ERR_INTERNAL);
                    return 0;
                }
                if (lane == (sp & 31)) {
                    if (sp < 32) s0 = second; else s1 = second;
                }
                sp++;
                node = first;
                have_next = true;
            } else if (ml) {
                node = D.x;
                have_next = true;
            } else if (mr) {
                node = D.y;
                have_next = true;
            }
        }
        if (!have_next) {
            if (sp == 0) break;
            sp--;
            int v0 = __shfl_sync(kFull, s0, sp & 31), v1 = __shfl_sync(kFull, s1, sp & 31);
            node = sp < 32 ? v0 : v1;
        }
    }
    return alive;
}

// Occluder cache: the facets that most recently blocked a segment of this
// warp (warp-uniform, most recent first).  Neighbouring packets -- the next
// sample pairs of the same facet pair, the next facet of the same row -- are
// often blocked by the same building, so testing these few facets first
// settles most blocked lanes without a BVH walk.  A cached facet is tested
// with the same exact leaf test, so the result never depends on the cache.
constexpr int kCacheSize = 4;

struct OccluderCache {
    int f[kCacheSize];
    int scene = -1;   // facets are global indices: the cache belongs to one scene
    __device__ __forceinline__ OccluderCache()
    {
        for (int k = 0; k < kCacheSize; k++) f[k] = -1;
    }
    // Call at the start of every work item (warp-uniform).
    __device__ __forceinline__ void enter_scene(int sc)
    {
        if (sc == scene) return;
        scene = sc;
        for (int k = 0; k < kCacheSize; k++) f[k] = -1;
    }
    __device__ __forceinline__ void put(int g)
    {
        if (g < 0 || g == f[0]) return;
        int prev = g;
        for (int k = 0; k < kCacheSize; k++) {   // move-to-front, dropping the oldest
            int cur = f[k];
            f[k] = prev;
            if (cur == g) break;
            prev = cur;
        }
    }
};

// Lanes of the packet left unblocked: cached occluders first (when `cache`),
// then the BVH walk.  Same contract as walk_packet; `myblk` receives, in each
// lane that gets blocked, the facet that blocked it.
// The warp's recently used occluders, tested before any walk.
template <class LeafFn>
__device__ __forceinline__ unsigned cache_tests(const Seg &s, unsigned alive, const Leaf *leaves,
                                                WalkCounters &wc, LeafFn leaf_hit,
                                                OccluderCache &cache, int &myblk)
{
    const int lane = threadIdx.x & 31;
    int promote = -1;
#pragma unroll
    for (int k = 0; k < kCacheSize; k++) {
        const int g = cache.f[k];
        if (!alive || g < 0) break;
        const Leaf L = load_leaf(leaves, g);
        bool me = (alive >> lane) & 1u;
        bool hit = me && leaf_hit(s, L, wc);
        wc.leaf_tests += me;
        wc.cache_hits += hit;
        if (hit) myblk = g;
        const unsigned hm = __ballot_sync(kFull, hit);
        alive &= ~hm;
        if (hm && k > 0 && promote < 0) promote = g;
    }
    if (promote >= 0) cache.put(promote);   // the facet that worked moves to the front
    return alive;
}

template <bool CACHE, class LeafFn, bool LRU = CACHE, bool ABS = false>
__device__ __forceinline__ unsigned occlude(Seg &s, unsigned alive, const Node *nodes,
                                            const Leaf *leaves, int root, float dirx, float diry,
                                            float dirz, int budget, int *err, WalkCounters &wc,
                                            LeafFn leaf_hit, OccluderCache &cache, int &myblk)
{
    if (CACHE && LRU) {
        alive = cache_tests(s, alive, leaves, wc, leaf_hit, cache, myblk);
        if (!alive) return 0;
    }
    int blocker;
    if (s.ix == 0.f) finish_seg<ABS>(s);   // reciprocals only when walking
    alive = walk_packet<LeafFn, NoFilter, ABS>(s, alive, nodes, leaves, root, dirx, diry, dirz,
                                               budget, err, wc, leaf_hit, blocker, myblk);
    if (CACHE) cache.put(blocker);
    return alive;
}

struct ExactLeaf {
    __device__ __forceinline__ bool operator()(const Seg &s, const Leaf &L, WalkCounters &wc) const
    {
        wc.exact++;
        return facet_hit_exact(s, L);
    }
};

}  // namespace ivm
