// edge_matrix.cu -- edges as rows and columns of the matrix (the matrix lists,
// per face or edge, the visible faces and edges: Sec. I-II; edges are the
// nodes of first-order diffraction, Sec. III-B).
//
// Edge e (A -> B, cm) carries s samples q_b = 2s A + (2b+1)(B - A) and the two
// facets f1(e), f2(e) that meet at it.  A point P reaches the edge from
// outside its building only when it is strictly in front of f1 or f2
// (ext(P, e)); otherwise the segment would leave through the building's
// inside, which holds no facet of its own between two boundary points.
//   fe[i][e] = some facet sample p of i and edge sample q of e with
//              front(q, i), ext(p, e) and the open segment p-q unblocked;
//   ee[e][g] = e != g and some q on e, r on g with ext(r, e), ext(q, g) and
//              q-r unblocked (symmetric: both bits are set by one decision).
// The edge -> facet block of the full matrix is the transpose of fe.
//
// One warp per pair, pairs from a persistent work queue: one launch over the
// N * ne facet-edge pairs, one over the ne^2 ordered edge pairs of which e < g
// are decided.  A
// pair passes a necessary screen on its endpoints and corners first (every
// sample is a strict convex combination of them, and the front tests are
// affine), then packets of 32 sample segments go through the occluder cache
// and the BVH walk; the first packet with a free segment decides the pair.
#include <type_traits>

#include "edges.cuh"
#include "traverse.cuh"
#include "filter.cuh"

namespace ivm {

namespace {

// n . (X - O) > 0 for X given in 64-bit (endpoints may sit just outside the
// sample range): |n| < 2^31 and |X - O| < 2^25, so the sum fits in int64.
__device__ __forceinline__ bool front_ll(const Leaf &L, long long x, long long y, long long z)
{
    return (long long)L.nx * (x - L.ox) + (long long)L.ny * (y - L.oy) +
           (long long)L.nz * (z - L.oz) > 0;
}

__device__ __forceinline__ bool in_range(long long x, long long y, long long z)
{
    return x > -kCoordLimit && x < kCoordLimit && y > -kCoordLimit && y < kCoordLimit &&
           z > -kCoordLimit && z < kCoordLimit;
}

// the plane of one facet: reduced outward normal and origin (scaled)
struct Plane {
    int nx, ny, nz, ox, oy, oz;
};

__device__ __forceinline__ Plane plane_of(const Leaf &L)
{
    return Plane{L.nx, L.ny, L.nz, L.ox, L.oy, L.oz};
}

__device__ __forceinline__ bool front_ll(const Plane &P, long long x, long long y, long long z)
{
    return (long long)P.nx * (x - P.ox) + (long long)P.ny * (y - P.oy) +
           (long long)P.nz * (z - P.oz) > 0;
}

struct EdgeGeom {
    long long ax, ay, az, bx, by, bz;   // scaled endpoints 2s A, 2s B
    int dx, dy, dz;                     // B - A (cm)
    Plane F1, F2;                       // the two facets meeting at the edge
    bool ok;
};

__device__ __forceinline__ EdgeGeom edge_geom(const DevScenes &g, const SceneDesc &D,
                                              const EdgeMatrixArgs &a, int e, int *err)
{
    EdgeGeom E;
    const int *r = a.edges + 6 * (size_t)e;
    const long long k = 2LL * D.s;
    E.ax = k * r[0]; E.ay = k * r[1]; E.az = k * r[2];
    E.bx = k * r[3]; E.by = k * r[4]; E.bz = k * r[5];
    E.dx = r[3] - r[0]; E.dy = r[4] - r[1]; E.dz = r[5] - r[2];
    const int f1 = a.faces[2 * e], f2 = a.faces[2 * e + 1];
    E.ok = f1 >= 0 && f1 < D.n && f2 >= 0 && f2 < D.n;
    if (!E.ok) {
        raise_error(err, IVM_ERR_ARG);
        return E;
    }
    // the first and last samples in range: the ones between lie on the segment
    // joining them, inside the same box
    const long long m = 2LL * D.s - 1;
    E.ok = in_range(E.ax + E.dx, E.ay + E.dy, E.az + E.dz) &&
           in_range(E.ax + m * E.dx, E.ay + m * E.dy, E.az + m * E.dz);
    if (!E.ok) {
        raise_error(err, IVM_ERR_RANGE);
        return E;
    }
    E.F1 = plane_of(load_leaf(g.leaf, D.facet0 + f1));
    E.F2 = plane_of(load_leaf(g.leaf, D.facet0 + f2));
    return E;
}

// sample b of the edge (in range: checked by edge_geom)
__device__ __forceinline__ void edge_sample(const EdgeGeom &E, int b, int &x, int &y, int &z)
{
    const long long m = 2 * b + 1;
    x = (int)(E.ax + m * E.dx);
    y = (int)(E.ay + m * E.dy);
    z = (int)(E.az + m * E.dz);
}

__device__ __forceinline__ bool ext_of(const EdgeGeom &E, long long x, long long y, long long z)
{
    return front_ll(E.F1, x, y, z) || front_ll(E.F2, x, y, z);
}

// some endpoint of E strictly in front of one of G's two facets
__device__ __forceinline__ bool ends_ext(const EdgeGeom &E, const EdgeGeom &G)
{
    return ext_of(G, E.ax, E.ay, E.az) || ext_of(G, E.bx, E.by, E.bz);
}

}  // namespace

// facet i against edge e: one bit of fe
template <class LeafFn>
__device__ __forceinline__ void decide_fe(const DevScenes &g, const SceneDesc &D,
                                          const EdgeMatrixArgs &a, int i, int e, int *err,
                                          WalkCounters &wc, LeafFn leaf, OccluderCache &cache)
{
    const int lane = threadIdx.x & 31;
    const int s = D.s, s2 = s * s;
    const Leaf Li = load_leaf(g.leaf, D.facet0 + i);
    const EdgeGeom E = edge_geom(g, D, a, e, err);
    if (!E.ok) return;
    if (!front_ll(Li, E.ax, E.ay, E.az) && !front_ll(Li, E.bx, E.by, E.bz)) return;
    const long long c0x = Li.ox, c0y = Li.oy, c0z = Li.oz;
    if (!ext_of(E, c0x, c0y, c0z) && !ext_of(E, c0x + Li.ux, c0y + Li.uy, c0z + Li.uz) &&
        !ext_of(E, c0x + Li.vx, c0y + Li.vy, c0z + Li.vz) &&
        !ext_of(E, c0x + Li.ux + Li.vx, c0y + Li.uy + Li.vy, c0z + Li.uz + Li.vz))
        return;
    const float dirx = (float)((E.ax + E.bx) - (2LL * Li.ox + Li.ux + Li.vx));
    const float diry = (float)((E.ay + E.by) - (2LL * Li.oy + Li.uy + Li.vy));
    const float dirz = (float)((E.az + E.bz) - (2LL * Li.oz + Li.uz + Li.vz));
    const int baseI = D.sample0 + i * s2;
    const int total_seg = s2 * s;
    for (int b0 = 0; b0 < total_seg; b0 += 32) {
        const int idx = b0 + lane;
        bool cond = idx < total_seg;
        int px = 0, py = 0, pz = 0, qx = 0, qy = 0, qz = 0;
        if (cond) {
            const int ap = idx / s, bq = idx - ap * s;
            px = __ldg(g.sx + baseI + ap);
            py = __ldg(g.sy + baseI + ap);
            pz = __ldg(g.sz + baseI + ap);
            edge_sample(E, bq, qx, qy, qz);
            cond = front_of(Li, qx, qy, qz) && ext_of(E, px, py, pz);
        }
        const unsigned alive = __ballot_sync(kFull, cond);
        if (!alive) continue;
        wc.segments += cond;
        Seg sg = make_seg(px, py, pz, qx, qy, qz);
        int myblk = -1;
        if (occlude<true>(sg, alive, g.nodes, g.leaf, D.root, dirx, diry, dirz, D.budget, err, wc,
                          leaf, cache, myblk)) {
            if (lane == 0) atomicOr(a.fe + (size_t)i * a.WE + (e >> 5), 1u << (e & 31));
            return;
        }
    }
}

// edges e < h: the two symmetric bits of ee
template <class LeafFn>
__device__ __forceinline__ void decide_ee(const DevScenes &g, const SceneDesc &D,
                                          const EdgeMatrixArgs &a, int e, int h, int *err,
                                          WalkCounters &wc, LeafFn leaf, OccluderCache &cache)
{
    const int lane = threadIdx.x & 31;
    const int s = D.s;
    const EdgeGeom E = edge_geom(g, D, a, e, err);
    const EdgeGeom H = edge_geom(g, D, a, h, err);
    if (!E.ok || !H.ok) return;
    if (!ends_ext(H, E) || !ends_ext(E, H)) return;
    const float dirx = (float)((H.ax + H.bx) - (E.ax + E.bx));
    const float diry = (float)((H.ay + H.by) - (E.ay + E.by));
    const float dirz = (float)((H.az + H.bz) - (E.az + E.bz));
    const int total_seg = s * s;
    for (int b0 = 0; b0 < total_seg; b0 += 32) {
        const int idx = b0 + lane;
        bool cond = idx < total_seg;
        int qx = 0, qy = 0, qz = 0, rx = 0, ry = 0, rz = 0;
        if (cond) {
            const int bq = idx / s, cr = idx - bq * s;
            edge_sample(E, bq, qx, qy, qz);
            edge_sample(H, cr, rx, ry, rz);
            cond = ext_of(E, rx, ry, rz) && ext_of(H, qx, qy, qz);
        }
        const unsigned alive = __ballot_sync(kFull, cond);
        if (!alive) continue;
        wc.segments += cond;
        Seg sg = make_seg(qx, qy, qz, rx, ry, rz);
        int myblk = -1;
        if (occlude<true>(sg, alive, g.nodes, g.leaf, D.root, dirx, diry, dirz, D.budget, err, wc,
                          leaf, cache, myblk)) {
            if (lane == 0) {
                atomicOr(a.ee + (size_t)e * a.WE + (h >> 5), 1u << (h & 31));
                atomicOr(a.ee + (size_t)h * a.WE + (e >> 5), 1u << (e & 31));
            }
            return;
        }
    }
}

// EE = false: the N * ne facet-edge pairs (i-major); EE = true: the ne^2
// ordered edge pairs, of which e < h are decided.
template <class LeafFn, bool EE>
__global__ void __launch_bounds__(kTravThreads, 4)
k_edge_matrix(DevScenes g, EdgeMatrixArgs a, unsigned long long total, int *err)
{
    const int lane = threadIdx.x & 31;
    const SceneDesc &D = g.desc[0];
    WalkCounters wc;
    LeafFn leaf;
    OccluderCache cache;
    cache.enter_scene(0);
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(a.work, (unsigned long long)a.tile);
        base = __shfl_sync(kFull, base, 0);
        if (base >= total) break;
        const unsigned long long end = min(base + (unsigned long long)a.tile, total);
        for (unsigned long long w = base; w < end; w++) {
            const int r = (int)(w / a.ne), c = (int)(w - (unsigned long long)r * a.ne);
            if (!EE) decide_fe(g, D, a, r, c, err, wc, leaf, cache);
            else if (c > r) decide_ee(g, D, a, r, c, err, wc, leaf, cache);
        }
    }
    flush_counters(wc, a.ctr);
}

template <class LeafFn, bool EE>
static void launch_em(const DevScenes &g, const EdgeMatrixArgs &a, unsigned long long total,
                      int n_sm, int *err, cudaStream_t st)
{
    if (total == 0) return;
    auto kern = k_edge_matrix<LeafFn, EE>;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTravThreads, 0);
    const int blocks = n_sm * (per_sm > 0 ? per_sm : 1);
    cudaMemsetAsync(a.work, 0, sizeof(unsigned long long), st);
    kern<<<blocks, kTravThreads, 0, st>>>(g, a, total, err);
    note_launches(1);
}

cudaError_t edges_matrix(const DevScenes &g, const EdgeMatrixArgs &a, bool filtered, int n_sm,
                         int *err, cudaStream_t st)
{
    const unsigned long long nfe = (unsigned long long)a.n * a.ne;
    const unsigned long long nee = (unsigned long long)a.ne * a.ne;
    if (filtered) {
        launch_em<FilteredLeaf, false>(g, a, nfe, n_sm, err, st);
        launch_em<FilteredLeaf, true>(g, a, nee, n_sm, err, st);
    } else {
        launch_em<ExactLeaf, false>(g, a, nfe, n_sm, err, st);
        launch_em<ExactLeaf, true>(g, a, nee, n_sm, err, st);
    }
    return cudaGetLastError();
}

}  // namespace ivm
