// ingest.cu -- scenario database to device geometry (the flow chart's first
// stage, Sec. III-C: vertex positions and face IDs of every building).
//
// Per facet: check the range contract, scale by 2s, reduce the outward
// normal u x v by the gcd of its components, mark axis-aligned rectangles,
// record its bounding box, and write the s x s cell-centre samples
// p_ab = 2s o + (2a+1) u + (2b+1) v.
#include "ivm_internal.cuh"

namespace ivm {

__device__ __forceinline__ long long llabs_(long long v) { return v < 0 ? -v : v; }

__device__ long long gcd_ll(long long a, long long b)
{
    a = llabs_(a);
    b = llabs_(b);
    while (b) {   // at most ~92 steps for 64-bit operands
        long long t = a % b;
        a = b;
        b = t;
    }
    return a;
}

__global__ void k_facet_scene(const SceneDesc *desc, int n_scenes, int total, int *fscene)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    int lo = 0, hi = n_scenes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (desc[mid].facet0 <= g) lo = mid; else hi = mid - 1;
    }
    fscene[g] = lo;
}

__global__ void k_ingest(DevScenes g, int *err)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= g.total_facets) return;
    const int sc = g.fscene[f];
    const SceneDesc D = g.desc[sc];
    const ivm_facet r = g.facets[f];
    const long long k = 2LL * D.s;
    long long o[3] = {r.o[0], r.o[1], r.o[2]};
    long long u[3] = {r.u[0], r.u[1], r.u[2]};
    long long v[3] = {r.v[0], r.v[1], r.v[2]};
    bool ok = true;
    long long lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
        long long c0 = k * o[a], c1 = k * (o[a] + u[a]), c2 = k * (o[a] + u[a] + v[a]),
                  c3 = k * (o[a] + v[a]);
        lo[a] = min(min(c0, c1), min(c2, c3));
        hi[a] = max(max(c0, c1), max(c2, c3));
        ok &= (llabs_(lo[a]) < kCoordLimit) & (llabs_(hi[a]) < kCoordLimit);
    }
    long long n[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2],
                      u[0] * v[1] - u[1] * v[0]};
    long long gg = gcd_ll(gcd_ll(n[0], n[1]), n[2]);
    if (gg == 0) ok = false;
    long long nr[3] = {0, 0, 0};
    if (ok) {
        for (int a = 0; a < 3; a++) {
            nr[a] = n[a] / gg;
            ok &= llabs_(nr[a]) < 2147483647LL;
        }
    }
    if (!ok) {
        raise_error(err, IVM_ERR_RANGE);
        return;
    }
    int dom = 0;
    if (llabs_(nr[1]) > llabs_(nr[dom])) dom = 1;
    if (llabs_(nr[2]) > llabs_(nr[dom])) dom = 2;
    // axis-aligned rectangle: U and V each along one coordinate axis, not the same one
    int nu = 0, nv = 0, au = -1, av = -1;
    for (int a = 0; a < 3; a++) {
        if (u[a]) { nu++; au = a; }
        if (v[a]) { nv++; av = a; }
    }
    if (nu == 1 && nv == 1 && au != av) dom |= 4;
    Leaf L;
    L.ox = (int)(k * o[0]); L.oy = (int)(k * o[1]); L.oz = (int)(k * o[2]);
    L.building = r.building;
    L.ux = (int)(k * u[0]); L.uy = (int)(k * u[1]); L.uz = (int)(k * u[2]);
    L.scene = sc;
    L.vx = (int)(k * v[0]); L.vy = (int)(k * v[1]); L.vz = (int)(k * v[2]);
    L.dom = dom;
    L.nx = (int)nr[0]; L.ny = (int)nr[1]; L.nz = (int)nr[2];
    L.pad = 0;
    g.leaf[f] = L;
    int *b = g.box + 6 * (size_t)f;
    b[0] = (int)lo[0]; b[1] = (int)lo[1]; b[2] = (int)lo[2];
    b[3] = (int)hi[0]; b[4] = (int)hi[1]; b[5] = (int)hi[2];
    const int s = D.s;
    size_t base = (size_t)D.sample0 + (size_t)(f - D.facet0) * s * s;
    for (int a = 0; a < s; a++)
        for (int c = 0; c < s; c++) {
            size_t idx = base + a * s + c;
            g.sx[idx] = (int)(k * o[0] + (2 * a + 1) * u[0] + (2 * c + 1) * v[0]);
            g.sy[idx] = (int)(k * o[1] + (2 * a + 1) * u[1] + (2 * c + 1) * v[1]);
            g.sz[idx] = (int)(k * o[2] + (2 * a + 1) * u[2] + (2 * c + 1) * v[2]);
        }
}

cudaError_t launch_ingest(const DevScenes &g, int *err, cudaStream_t st)
{
    int nb = (g.total_facets + 255) / 256;
    k_facet_scene<<<nb, 256, 0, st>>>(g.desc, g.n_scenes, g.total_facets, g.fscene);
    k_ingest<<<nb, 256, 0, st>>>(g, err);
    note_launches(2);
    return cudaGetLastError();
}

}  // namespace ivm
