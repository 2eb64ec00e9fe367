// relations.cu -- interface relations and angular bouncing ranges of the
// visible ordered pairs (Sec. II-B, Table I, Eq. (1)-(2)).
//
// For every set bit M_ij (reference face i, aim face j), in row-major order:
// the relation is PAR (1) when the normals are parallel, PER (2) when they
// are perpendicular, else 0; exact on the integer normals.  Angles follow
// Sec. II-B's 2D views: for edge k of face i (O -> O+U -> O+U+V -> O+V) the
// view is the plane through the edge's midpoint B perpendicular to the edge,
// the reference line runs from B to the opposite edge's midpoint (the
// paper's BA), and the angle turns from it towards face i's outward normal.
// Each corner F of face j, projected into the view, gives Eq. (1) when it
// lies in front (below 180 degrees), and 0 when it lies behind the face's
// plane, straight beyond the edge (180) or on the edge's line (Eq. (2));
// the cases are decided exactly on integers, the value in double.  The
// edge's range is (min, max) over j's corners.  Coordinates are the input
// records' centimetres.
//
// Warp per row: a count pass (popcounts), an exclusive scan over rows, and a
// write pass in which lanes take the row's words 32 at a time and place
// their bits by a warp prefix of popcounts.
#include "relations.cuh"
#include "traverse.cuh"

namespace ivm {

__global__ void k_rel_count(const uint32_t *M, int n, int W, long long *deg)
{
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;   // uniform per warp
    const uint32_t *row = M + (size_t)w * W;
    unsigned cnt = 0;
    for (int c = lane; c < W; c += 32) {
        uint32_t v = row[c];
        const int k = n - 32 * c;
        if (k < 32) v &= (1u << k) - 1u;   // padding bits are not facets
        cnt += __popc(v);
    }
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
    if (lane == 0) deg[w] = cnt;
}

namespace {

typedef __int128 i128;

// Correctly rounded (to nearest, ties to even) conversion of a 128-bit
// integer to double, so that both sides of a comparison convert the same
// exact integer to the same double.
__device__ double to_double(i128 x)
{
    if (x == 0) return 0.0;
    const bool neg = x < 0;
    unsigned __int128 m = neg ? (unsigned __int128)0 - (unsigned __int128)x : (unsigned __int128)x;
    const unsigned long long hi = (unsigned long long)(m >> 64), lo = (unsigned long long)m;
    const int p = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
    double r;
    if (p <= 52) {
        r = (double)lo;                                   // exact
    } else {
        const int sh = p - 52;
        unsigned __int128 q = m >> sh;                    // 53 bits
        const unsigned __int128 rem = m - (q << sh), half = (unsigned __int128)1 << (sh - 1);
        if (rem > half || (rem == half && (q & 1))) q += 1;   // at most 2^53: exact
        r = ldexp((double)(unsigned long long)q, sh);
    }
    return neg ? -r : r;
}

__device__ i128 dot3(const long long *a, const long long *b)
{
    return (i128)a[0] * b[0] + (i128)a[1] * b[1] + (i128)a[2] * b[2];
}

// Angle of the aim-face corner at 2 B + bf2 (doubled coordinates) seen from
// edge e (direction) of the reference face, whose doubled reference vector
// is ba2 and outward normal n: the clockwise angle in the view perpendicular
// to the edge, from the reference line towards the normal; 0 when it is at
// least 180 degrees or the corner lies on the edge's line (Eq. (2)).  With
// ee = |e|^2, the projections w, ref of bf2, ba2 satisfy
//   w . ref = A / ee,  |w|^2 = Bw / ee,  |ref|^2 = Br / ee,  sign(w . n) = sign(bf2 . n),
// A = ee (bf2 . ba2) - (bf2 . e)(ba2 . e), Bw = ee |bf2|^2 - (bf2 . e)^2,
// Br = ee |ba2|^2 - (ba2 . e)^2 (e lies in the face, so e . n = 0).
__device__ double corner_angle(const long long *e, const long long *ba2, const long long *bf2,
                               const long long *n)
{
    const i128 ee = dot3(e, e), be = dot3(bf2, e), ae = dot3(ba2, e);
    const i128 A = ee * dot3(bf2, ba2) - be * ae;
    const i128 Bw = ee * dot3(bf2, bf2) - be * be;
    const i128 Br = ee * dot3(ba2, ba2) - ae * ae;
    const i128 side = dot3(bf2, n);
    if (Bw == 0 || side < 0 || (side == 0 && A < 0)) return 0.0;
    double c = to_double(A) / (sqrt(to_double(Bw)) * sqrt(to_double(Br)));
    c = fmin(1.0, fmax(-1.0, c));
    return acos(c) * (180.0 / 3.14159265358979323846);
}

// Relation and the 4 edges' ranges of reference face I towards aim face J,
// from the input records (cm).
__device__ void annotate(const ivm_facet &I, const ivm_facet &J, uint8_t &rel, double *rng)
{
    long long ci[4][3], cj[4][3], ni[3], nj[3];
    for (int a = 0; a < 3; a++) {
        ci[0][a] = I.o[a];
        ci[1][a] = (long long)I.o[a] + I.u[a];
        ci[2][a] = (long long)I.o[a] + I.u[a] + I.v[a];
        ci[3][a] = (long long)I.o[a] + I.v[a];
        cj[0][a] = J.o[a];
        cj[1][a] = (long long)J.o[a] + J.u[a];
        cj[2][a] = (long long)J.o[a] + J.u[a] + J.v[a];
        cj[3][a] = (long long)J.o[a] + J.v[a];
    }
    ni[0] = (long long)I.u[1] * I.v[2] - (long long)I.u[2] * I.v[1];
    ni[1] = (long long)I.u[2] * I.v[0] - (long long)I.u[0] * I.v[2];
    ni[2] = (long long)I.u[0] * I.v[1] - (long long)I.u[1] * I.v[0];
    nj[0] = (long long)J.u[1] * J.v[2] - (long long)J.u[2] * J.v[1];
    nj[1] = (long long)J.u[2] * J.v[0] - (long long)J.u[0] * J.v[2];
    nj[2] = (long long)J.u[0] * J.v[1] - (long long)J.u[1] * J.v[0];
    const bool par = (i128)ni[1] * nj[2] - (i128)ni[2] * nj[1] == 0 &&
                     (i128)ni[2] * nj[0] - (i128)ni[0] * nj[2] == 0 &&
                     (i128)ni[0] * nj[1] - (i128)ni[1] * nj[0] == 0;
    const bool per = dot3(ni, nj) == 0;
    rel = par ? 1 : (per ? 2 : 0);
    for (int k = 0; k < 4; k++) {
        long long e[3], mid2[3], ba2[3];
        for (int a = 0; a < 3; a++) {
            e[a] = ci[(k + 1) & 3][a] - ci[k][a];
            mid2[a] = ci[k][a] + ci[(k + 1) & 3][a];
            ba2[a] = ci[(k + 2) & 3][a] + ci[(k + 3) & 3][a] - mid2[a];
        }
        double lo = 0.0, hi = 0.0;
        for (int q = 0; q < 4; q++) {
            long long bf2[3];
            for (int a = 0; a < 3; a++) bf2[a] = 2 * cj[q][a] - mid2[a];
            const double w = corner_angle(e, ba2, bf2, ni);
            if (q == 0 || w < lo) lo = w;
            if (q == 0 || w > hi) hi = w;
        }
        rng[2 * k] = lo;
        rng[2 * k + 1] = hi;
    }
}

}  // namespace

__global__ void k_rel_write(DevScenes g, RelArgs a)
{
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= a.n) return;   // uniform per warp
    const SceneDesc &D = g.desc[0];
    const uint32_t *row = a.M + (size_t)w * a.W;
    long long base = a.off[w];
    const ivm_facet I = g.facets[D.facet0 + (int)w];
    for (int c0 = 0; c0 < a.W; c0 += 32) {
        const int c = c0 + lane;
        uint32_t v = c < a.W ? row[c] : 0u;
        const int k = a.n - 32 * c;
        if (c < a.W && k < 32) v &= (1u << k) - 1u;
        const unsigned cnt = __popc(v);
        unsigned incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned u = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += u;
        }
        long long idx = base + incl - cnt;
        while (v) {
            const int b = __ffs(v) - 1;
            v &= v - 1;
            const int j = 32 * c + b;
            a.pairs[2 * idx] = (int)w;
            a.pairs[2 * idx + 1] = j;
            uint8_t rel;
            annotate(I, g.facets[D.facet0 + j], rel, a.ranges + 8 * idx);
            a.relation[idx] = rel;
            idx++;
        }
        base += __shfl_sync(kFull, incl, 31);
    }
}

cudaError_t relations_count(const uint32_t *M, int n, int W, long long *deg, cudaStream_t st)
{
    k_rel_count<<<(unsigned)(((long long)n * 32 + 127) / 128), 128, 0, st>>>(M, n, W, deg);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t relations_write(const DevScenes &g, const RelArgs &a, cudaStream_t st)
{
    k_rel_write<<<(unsigned)(((long long)a.n * 32 + 127) / 128), 128, 0, st>>>(g, a);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace ivm
