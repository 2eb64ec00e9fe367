// screen.cu -- candidate facet pairs for the matrix (the facing rule of
// Sec. II-B, Eq. (2), applied to whole facets before any sample is tested).
//
// A pair (i, j), i < j, is kept when some corner of j is strictly in front of
// i and some corner of i is strictly in front of j.  This is necessary for
// M_ij = 1: samples are convex combinations of the corners, and the facing
// value n . (x - O) is linear in x, so its maximum over a facet is at a
// corner: max = n.(O_j - O_i) + max(0, n.U_j) + max(0, n.V_j).
//
// One warp handles one (scene, row i, word c): lanes are j = 32c + lane.
#include "ivm_internal.cuh"
#include "traverse.cuh"

namespace ivm {

__device__ __forceinline__ bool corner_in_front(const Leaf &A, const Leaf &B)
{
    long long base = (long long)A.nx * (B.ox - A.ox) + (long long)A.ny * (B.oy - A.oy) +
                     (long long)A.nz * (B.oz - A.oz);
    long long du = (long long)A.nx * B.ux + (long long)A.ny * B.uy + (long long)A.nz * B.uz;
    long long dv = (long long)A.nx * B.vx + (long long)A.ny * B.vy + (long long)A.nz * B.vz;
    return base + max(du, 0LL) + max(dv, 0LL) > 0;
}

__device__ __forceinline__ int scene_of_rw(const SceneDesc *desc, int n_scenes, long long w)
{
    int lo = 0, hi = n_scenes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (desc[mid].rw0 <= w) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Returns this lane's candidate bit for the warp's (scene, i, c); all lanes
// of a warp share (scene, i, c).
__device__ __forceinline__ bool screen_lane(const DevScenes &g, long long w, int &i, int &j,
                                            const SceneDesc *&Dp, int &sc)
{
    sc = scene_of_rw(g.desc, g.n_scenes, w);
    Dp = g.desc + sc;
    const SceneDesc &D = *Dp;
    long long local = w - D.rw0;
    i = (int)(local / D.W);
    int c = (int)(local - (long long)i * D.W);
    j = 32 * c + (threadIdx.x & 31);
    if (i < D.row_lo || i >= D.row_hi) return false;   // another part's rows (warp-uniform)
    if (j <= i || j >= D.n) return false;
    const Leaf Li = load_leaf(g.leaf, D.facet0 + i);
    const Leaf Lj = load_leaf(g.leaf, D.facet0 + j);
    return corner_in_front(Li, Lj) && corner_in_front(Lj, Li);
}

__global__ void k_screen_count(DevScenes g, long long total_rw, unsigned long long *count)
{
    long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= total_rw) return;   // uniform per warp
    int i, j, sc;
    const SceneDesc *D;
    bool cand = screen_lane(g, w, i, j, D, sc);
    unsigned m = __ballot_sync(kFull, cand);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(count, (unsigned long long)__popc(m));
}

__global__ void k_screen_emit(DevScenes g, long long total_rw, int2 *pairs,
                              unsigned long long *cursor, unsigned long long cap)
{
    long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= total_rw) return;
    int i, j, sc;
    const SceneDesc *D;
    bool cand = screen_lane(g, w, i, j, D, sc);
    unsigned m = __ballot_sync(kFull, cand);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(cursor, (unsigned long long)__popc(m));
    base = __shfl_sync(kFull, base, 0);
    if (cand) {
        unsigned long long k = base + __popc(m & ((1u << lane) - 1));
        if (k < cap) pairs[k] = make_int2(D->facet0 + i, D->facet0 + j);
    }
}

static long long total_row_words(const DevScenes &g, const SceneDesc *host_desc)
{
    const SceneDesc &L = host_desc[g.n_scenes - 1];
    return L.rw0 + (long long)L.n * L.W;
}

cudaError_t launch_screen_count(const DevScenes &g, const SceneDesc *host_desc,
                                unsigned long long *count, cudaStream_t st)
{
    long long rw = total_row_words(g, host_desc);
    long long blocks = (rw * 32 + 255) / 256;
    k_screen_count<<<(unsigned)blocks, 256, 0, st>>>(g, rw, count);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_screen_emit(const DevScenes &g, const SceneDesc *host_desc, int2 *pairs,
                               unsigned long long *cursor, unsigned long long cap,
                               cudaStream_t st)
{
    long long rw = total_row_words(g, host_desc);
    long long blocks = (rw * 32 + 255) / 256;
    k_screen_emit<<<(unsigned)blocks, 256, 0, st>>>(g, rw, pairs, cursor, cap);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace ivm
