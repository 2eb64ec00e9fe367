// relations.cu -- interface relations and angular bouncing ranges of the
// visible ordered pairs (Sec. II-B, Table I, Eq. (1)-(2)).
//
// For every set bit M_ij (reference face i, aim face j), in row-major order:
// the relation is PAR (1) when the normals are parallel, PER (2) when they
// are perpendicular, else 0; exact on the gcd-reduced integer normals.  For
// edge k of face i (O -> O+U -> O+U+V -> O+V), B_k is the edge's midpoint and
// the reference vector runs from B_k to the opposite edge's midpoint (along
// the face, the paper's BA); each corner F of face j gives the Eq. (1) angle
// arccos(ref . (F - B_k) / |ref| |F - B_k|) in degrees, 180 recorded as 0
// (Eq. (2)) and decided exactly on the doubled integer vectors; the edge's
// range is (min, max) over j's corners.  Angles are computed in double from
// the scaled coordinates (angles do not depend on the scale).
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

__device__ double angle_deg(long long rx, long long ry, long long rz, long long dx, long long dy,
                            long long dz)
{
    const long long cx = ry * dz - rz * dy, cy = rz * dx - rx * dz, cz = rx * dy - ry * dx;
    const long long dot = rx * dx + ry * dy + rz * dz;
    if (cx == 0 && cy == 0 && cz == 0 && dot < 0) return 0.0;   // exactly 180: Eq. (2)
    const double rr = (double)(rx * rx + ry * ry + rz * rz), dd = (double)(dx * dx + dy * dy + dz * dz);
    double c = (double)dot / (sqrt(rr) * sqrt(dd));
    c = fmin(1.0, fmax(-1.0, c));
    return acos(c) * (180.0 / 3.14159265358979323846);
}

__device__ void annotate(const Leaf &I, const Leaf &J, uint8_t &rel, double *rng)
{
    const long long nix = I.nx, niy = I.ny, niz = I.nz, njx = J.nx, njy = J.ny, njz = J.nz;
    const bool par = niy * njz - niz * njy == 0 && niz * njx - nix * njz == 0 &&
                     nix * njy - niy * njx == 0;
    const bool per = nix * njx + niy * njy + niz * njz == 0;
    rel = par ? 1 : (per ? 2 : 0);
    // corners of i and j (scaled), doubled where midpoints are needed
    const long long ci[4][3] = {{I.ox, I.oy, I.oz},
                                {I.ox + I.ux, I.oy + I.uy, I.oz + I.uz},
                                {I.ox + I.ux + I.vx, I.oy + I.uy + I.vy, I.oz + I.uz + I.vz},
                                {I.ox + I.vx, I.oy + I.vy, I.oz + I.vz}};
    const long long cj[4][3] = {{J.ox, J.oy, J.oz},
                                {J.ox + J.ux, J.oy + J.uy, J.oz + J.uz},
                                {J.ox + J.ux + J.vx, J.oy + J.uy + J.vy, J.oz + J.uz + J.vz},
                                {J.ox + J.vx, J.oy + J.vy, J.oz + J.vz}};
    for (int k = 0; k < 4; k++) {
        long long m[3], r[3];
        for (int a = 0; a < 3; a++) {
            m[a] = ci[k][a] + ci[(k + 1) & 3][a];
            r[a] = ci[(k + 2) & 3][a] + ci[(k + 3) & 3][a] - m[a];
        }
        double lo = 0.0, hi = 0.0;
        for (int q = 0; q < 4; q++) {
            const double w = angle_deg(r[0], r[1], r[2], 2 * cj[q][0] - m[0], 2 * cj[q][1] - m[1],
                                       2 * cj[q][2] - m[2]);
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
    const Leaf I = load_leaf(g.leaf, D.facet0 + (int)w);
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
            annotate(I, load_leaf(g.leaf, D.facet0 + j), rel, a.ranges + 8 * idx);
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
