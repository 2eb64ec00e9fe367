// filter.cuh -- FP32 facet test with a proven error bound (the precision
// form).  It returns exactly what facet_hit_exact returns; the integer
// arithmetic runs only for edge orientations the float value cannot decide.
//
// Plane sides stay exact in int64 (three 32x32->64 products, cheap).  The four
// edge orientations e = d . (a x b), with a, b, d integer vectors below 2^23
// (exact in float), are evaluated as
//   c_i = fl(fl(p_i) - fl(q_i))          (p_i, q_i the two products of a x b)
//   e~  = fl(fl(fl(c_x d_x) + fl(c_y d_y)) + fl(c_z d_z))
// with round-to-nearest intrinsics (never contracted into FMAs).  With
// u = 2^-24 and m_i = |p_i| + |q_i|, standard rounding-error analysis gives
//   |fl(c_i) - c_i| <= (2u + u^2) m_i,
//   |e~ - sum d_i fl(c_i)| <= gamma_3 sum |d_i| |fl(c_i)|,
// so |e~ - e| <= (5u + O(u^2)) M with M = sum_i |d_i| m_i.  M' is M computed
// from |fl(p_i)|, |fl(q_i)| with round-up additions and products, so
// M <= M' / (1 - u), and |e~ - e| < 6u M' < 2^-21 M'.  When |e~| > 2^-21 M',
// sign(e~) = sign(e).  Inputs are integers, so no product underflows; all
// magnitudes stay below 2^75, far from overflow.
#pragma once

#include "traverse.cuh"

namespace ivm {

// +1 / -1 when the float value decides the sign, 0 when it cannot.
__device__ __forceinline__ int orient_filtered(float ax, float ay, float az, float bx, float by,
                                               float bz, float dx, float dy, float dz)
{
    float p1 = __fmul_rn(ay, bz), q1 = __fmul_rn(az, by);
    float p2 = __fmul_rn(az, bx), q2 = __fmul_rn(ax, bz);
    float p3 = __fmul_rn(ax, by), q3 = __fmul_rn(ay, bx);
    float cx = __fsub_rn(p1, q1), cy = __fsub_rn(p2, q2), cz = __fsub_rn(p3, q3);
    float e = __fadd_rn(__fadd_rn(__fmul_rn(cx, dx), __fmul_rn(cy, dy)), __fmul_rn(cz, dz));
    float m1 = __fadd_ru(fabsf(p1), fabsf(q1));
    float m2 = __fadd_ru(fabsf(p2), fabsf(q2));
    float m3 = __fadd_ru(fabsf(p3), fabsf(q3));
    float M = __fadd_ru(__fadd_ru(__fmul_ru(fabsf(dx), m1), __fmul_ru(fabsf(dy), m2)),
                        __fmul_ru(fabsf(dz), m3));
    float bound = M * 0x1p-21f;   // exact: power-of-two scaling of a value >= 1 or 0
    return e > bound ? 1 : (e < -bound ? -1 : 0);
}

// The rare path: some edge orientation was undecided and the decided ones
// agree; recompute the undecided ones exactly.  Out of line so that its
// int128 registers do not count against the traversal loop.
// Arguments by value (corner O - P, edges U and V, direction d, the four
// float verdicts packed as 2-bit fields) so nothing is spilled to the stack.
static __device__ __noinline__ bool settle_exact(int c0x, int c0y, int c0z, int ux, int uy,
                                                 int uz, int vx, int vy, int vz, int dx, int dy,
                                                 int dz, int packed)
{
    int e0 = ((packed >> 0) & 3) - 1, e1 = ((packed >> 2) & 3) - 1;
    int e2 = ((packed >> 4) & 3) - 1, e3 = ((packed >> 6) & 3) - 1;
    int c1x = c0x + ux, c1y = c0y + uy, c1z = c0z + uz;
    int c2x = c1x + vx, c2y = c1y + vy, c2z = c1z + vz;
    int c3x = c0x + vx, c3y = c0y + vy, c3z = c0z + vz;
    if (e0 == 0) e0 = orient_sign(c0x, c0y, c0z, c1x, c1y, c1z, dx, dy, dz);
    if (e1 == 0) e1 = orient_sign(c1x, c1y, c1z, c2x, c2y, c2z, dx, dy, dz);
    if (e2 == 0) e2 = orient_sign(c2x, c2y, c2z, c3x, c3y, c3z, dx, dy, dz);
    if (e3 == 0) e3 = orient_sign(c3x, c3y, c3z, c0x, c0y, c0z, dx, dy, dz);
    bool nonneg = (e0 >= 0) & (e1 >= 0) & (e2 >= 0) & (e3 >= 0);
    bool nonpos = (e0 <= 0) & (e1 <= 0) & (e2 <= 0) & (e3 <= 0);
    return nonneg | nonpos;
}

__device__ __forceinline__ bool facet_hit_filtered(const Seg &s, const Leaf &L, WalkCounters &wc)
{
    long long rx = s.px - L.ox, ry = s.py - L.oy, rz = s.pz - L.oz;
    long long sp = (long long)L.nx * rx + (long long)L.ny * ry + (long long)L.nz * rz;
    long long sd = (long long)L.nx * s.dx + (long long)L.ny * s.dy + (long long)L.nz * s.dz;
    int a = sgn_ll(sp), b = sgn_ll(sp + sd);
    if (a == b) {
        if (a != 0) return false;
        wc.exact++;
        return coplanar_hit(s, L);
    }
    if (a == 0 || b == 0) return false;
    // corners relative to P: integers below 2^23, exact in float
    float f0x = (float)(L.ox - s.px), f0y = (float)(L.oy - s.py), f0z = (float)(L.oz - s.pz);
    float f1x = f0x + (float)L.ux, f1y = f0y + (float)L.uy, f1z = f0z + (float)L.uz;
    float f2x = f1x + (float)L.vx, f2y = f1y + (float)L.vy, f2z = f1z + (float)L.vz;
    float f3x = f0x + (float)L.vx, f3y = f0y + (float)L.vy, f3z = f0z + (float)L.vz;
    float dx = (float)s.dx, dy = (float)s.dy, dz = (float)s.dz;
    int e0 = orient_filtered(f0x, f0y, f0z, f1x, f1y, f1z, dx, dy, dz);
    int e1 = orient_filtered(f1x, f1y, f1z, f2x, f2y, f2z, dx, dy, dz);
    int e2 = orient_filtered(f2x, f2y, f2z, f3x, f3y, f3z, dx, dy, dz);
    int e3 = orient_filtered(f3x, f3y, f3z, f0x, f0y, f0z, dx, dy, dz);
    bool pos = (e0 > 0) | (e1 > 0) | (e2 > 0) | (e3 > 0);
    bool neg = (e0 < 0) | (e1 < 0) | (e2 < 0) | (e3 < 0);
    if (pos & neg) return false;
    if ((e0 != 0) & (e1 != 0) & (e2 != 0) & (e3 != 0)) return true;
    // some edge is undecided and the decided ones agree: settle it exactly
    wc.undecided++;
    wc.exact++;
    const int packed = (e0 + 1) | ((e1 + 1) << 2) | ((e2 + 1) << 4) | ((e3 + 1) << 6);
    return settle_exact(L.ox - s.px, L.oy - s.py, L.oz - s.pz, L.ux, L.uy, L.uz, L.vx, L.vy, L.vz,
                        s.dx, s.dy, s.dz, packed);
}

// The same test out of line, for kernels whose hot loop holds several walks:
// one copy of the test instead of one per walk keeps the code small enough
// for the instruction cache when many warps run different parts of it.  A
// register-only interface (coordinates in, flags out: bit 0 = hit, bit 1 =
// an exact test was used, bit 2 = the filter was undecided) keeps the call
// free of local-memory traffic.
static __device__ __noinline__ int facet_hit_filtered_call(int px, int py, int pz, int dx,
                                                           int dy, int dz, int ox, int oy, int oz,
                                                           int ux, int uy, int uz, int vx, int vy,
                                                           int vz, int nx, int ny, int nz,
                                                           int dom)
{
    const Seg s = make_seg(px, py, pz, px + dx, py + dy, pz + dz);
    Leaf L;
    L.ox = ox; L.oy = oy; L.oz = oz; L.building = 0;
    L.ux = ux; L.uy = uy; L.uz = uz; L.scene = 0;
    L.vx = vx; L.vy = vy; L.vz = vz; L.dom = dom;
    L.nx = nx; L.ny = ny; L.nz = nz; L.pad = 0;
    WalkCounters wc;
    const bool hit = facet_hit_filtered(s, L, wc);
    return (int)hit | ((wc.exact != 0) << 1) | ((wc.undecided != 0) << 2);
}

struct FilteredLeafCall {
    __device__ __forceinline__ bool operator()(const Seg &s, const Leaf &L, WalkCounters &wc) const
    {
        const int r = facet_hit_filtered_call(s.px, s.py, s.pz, s.dx, s.dy, s.dz, L.ox, L.oy,
                                              L.oz, L.ux, L.uy, L.uz, L.vx, L.vy, L.vz, L.nx,
                                              L.ny, L.nz, L.dom);
        wc.exact += (r >> 1) & 1;
        wc.undecided += (r >> 2) & 1;
        return r & 1;
    }
};

struct FilteredLeaf {
    __device__ __forceinline__ bool operator()(const Seg &s, const Leaf &L, WalkCounters &wc) const
    {
        return facet_hit_filtered(s, L, wc);
    }
};

// ------------------------------------------------ axis-aligned rectangles
//
// For a facet whose normal lies along axis K and whose edges lie along the
// other two axes (Leaf.dom bit 2), the open segment P -> P + d meets the
// closed rectangle iff it crosses the plane x_K = O_K strictly between its
// ends (an exact int32 sign test on sp = P_K - O_K and sp + d_K) at a point
// inside the rectangle's closed range on both other axes m:
//   c_lo = |sp| d_m - (lo_m - P_m) |d_K| >= 0  and  c_hi = (hi_m - P_m) |d_K| - |sp| d_m >= 0
// (traverse.cuh, aligned_hit_k).  Each c = x - y is a difference of two
// products of integers below 2^23, exact in float as factors.  With
// x~ = fl(x), y~ = fl(y) (one rounding each, u = 2^-24) and c~ = fl(x~ - y~),
//   |c~ - c| <= u |x~ - y~| + u (|x| + |y|) <= (2u + O(u^2)) (|x~| + |y~|),
// so B = fl_up(|x~| + |y~|) 2^-22 (a power-of-two scaling, exact) bounds the
// error with room to spare: c~ > B proves c > 0, c~ < -B proves c < 0.  When
// some condition is not proven and none is proven false, the exact int64
// test decides.  The products are round-to-nearest intrinsics, never
// contracted into FMAs.

// Exact int64 decision of the four conditions (the rare path), out of line.
static __device__ __noinline__ bool aligned_settle(int a, int b, int d1, int d2, int lo1, int hi1,
                                                   int lo2, int hi2)
{
    const long long t1 = (long long)a * d1, t2 = (long long)a * d2;
    return ((long long)lo1 * b <= t1) & (t1 <= (long long)hi1 * b) & ((long long)lo2 * b <= t2) &
           (t2 <= (long long)hi2 * b);
}

// 1 when x - y > 0 is proven, -1 when x - y < 0 is proven, 0 otherwise.
__device__ __forceinline__ int diff_sign(float x, float y)
{
    const float c = __fsub_rn(x, y);
    const float B = __fmul_rn(__fadd_ru(fabsf(x), fabsf(y)), 0x1p-22f);
    return c > B ? 1 : (c < -B ? -1 : 0);
}

template <int K>
__device__ __forceinline__ bool aligned_filtered_k(const Seg &s, const Leaf &L, WalkCounters &wc)
{
    constexpr int K1 = (K + 1) % 3, K2 = (K + 2) % 3;
    const int P[3] = {s.px, s.py, s.pz}, D[3] = {s.dx, s.dy, s.dz};
    const int O[3] = {L.ox, L.oy, L.oz};
    const int E[3] = {L.ux + L.vx, L.uy + L.vy, L.uz + L.vz};   // far corner - O
    const int sp = P[K] - O[K], sq = sp + D[K];
    if ((sp > 0 && sq > 0) || (sp < 0 && sq < 0)) return false;
    if (sp == 0 || sq == 0) {
        if (sp != 0 || sq != 0) return false;   // touches the plane only at an endpoint
        wc.exact++;
        return coplanar_hit(s, L);
    }
    const int a = sp < 0 ? -sp : sp, b = D[K] < 0 ? -D[K] : D[K];
    const int lo1 = min(O[K1], O[K1] + E[K1]) - P[K1], hi1 = max(O[K1], O[K1] + E[K1]) - P[K1];
    const int lo2 = min(O[K2], O[K2] + E[K2]) - P[K2], hi2 = max(O[K2], O[K2] + E[K2]) - P[K2];
    const float fa = (float)a, fb = (float)b;
    const float x1 = __fmul_rn(fa, (float)D[K1]), x2 = __fmul_rn(fa, (float)D[K2]);
    const int c0 = diff_sign(x1, __fmul_rn((float)lo1, fb));
    const int c1 = diff_sign(__fmul_rn((float)hi1, fb), x1);
    const int c2 = diff_sign(x2, __fmul_rn((float)lo2, fb));
    const int c3 = diff_sign(__fmul_rn((float)hi2, fb), x2);
    if ((c0 < 0) | (c1 < 0) | (c2 < 0) | (c3 < 0)) return false;
    if ((c0 > 0) & (c1 > 0) & (c2 > 0) & (c3 > 0)) return true;
    wc.undecided++;
    wc.exact++;
    return aligned_settle(a, b, D[K1], D[K2], lo1, hi1, lo2, hi2);
}

__device__ __forceinline__ bool aligned_filtered(const Seg &s, const Leaf &L, WalkCounters &wc)
{
    const int k = L.dom & 3;
    if (k == 0) return aligned_filtered_k<0>(s, L, wc);
    if (k == 1) return aligned_filtered_k<1>(s, L, wc);
    return aligned_filtered_k<2>(s, L, wc);
}

// The filtered test with the rectangle form for axis-aligned facets
// (IVM_FLAG_ALIGNED_FACETS), out of line with the register interface of
// facet_hit_filtered_call: both tests give facet_hit_exact's answer.
static __device__ __noinline__ int facet_hit_aligned_call(int px, int py, int pz, int dx, int dy,
                                                          int dz, int ox, int oy, int oz, int ux,
                                                          int uy, int uz, int vx, int vy, int vz,
                                                          int nx, int ny, int nz, int dom)
{
    const Seg s = make_seg(px, py, pz, px + dx, py + dy, pz + dz);
    Leaf L;
    L.ox = ox; L.oy = oy; L.oz = oz; L.building = 0;
    L.ux = ux; L.uy = uy; L.uz = uz; L.scene = 0;
    L.vx = vx; L.vy = vy; L.vz = vz; L.dom = dom;
    L.nx = nx; L.ny = ny; L.nz = nz; L.pad = 0;
    WalkCounters wc;
    const bool hit = (dom & 4) ? aligned_filtered(s, L, wc) : facet_hit_filtered(s, L, wc);
    return (int)hit | ((wc.exact != 0) << 1) | ((wc.undecided != 0) << 2);
}

struct AlignedLeafCall {
    __device__ __forceinline__ bool operator()(const Seg &s, const Leaf &L, WalkCounters &wc) const
    {
        const int r = facet_hit_aligned_call(s.px, s.py, s.pz, s.dx, s.dy, s.dz, L.ox, L.oy, L.oz,
                                             L.ux, L.uy, L.uz, L.vx, L.vy, L.vz, L.nx, L.ny,
                                             L.nz, L.dom);
        wc.exact += (r >> 1) & 1;
        wc.undecided += (r >> 2) & 1;
        return r & 1;
    }
};

}  // namespace ivm
