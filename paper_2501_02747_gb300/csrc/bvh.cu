// bvh.cu -- linear BVH over the facets of every scene, built on the GPU.
//
// The paper's related work names bounding volume hierarchies as the usual
// accelerator for ray-object tests (Sec. I); here the BVH only speeds up the
// occlusion test and never decides a bit: its boxes are exact integer
// bounds, tested conservatively.
//
// Build: per-scene bounds of the facet centroids -> 30-bit Morton code per
// facet (one cubic grid over the bounds) -> sort keys (Morton << 32 | local index, unique) -> binary radix
// tree over the sorted keys (each internal node finds its key range and split
// from common-prefix lengths, after T. Karras, "Maximizing parallelism in the
// construction of BVHs, octrees, and k-d trees", HPG 2012) -> bottom-up box
// refit with one arrival counter per node.
//
// The sort is a rank sort: each key's position is the number of smaller keys
// of its scene, counted through shared-memory tiles.  It costs N^2 / 2
// comparisons per scene, well under a millisecond up to a few 1e4 facets.
#include <climits>

#include "ivm_internal.cuh"

namespace ivm {

__global__ void k_bounds_init(int *bounds, int n_scenes)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 6 * n_scenes) bounds[i] = (i % 6) < 3 ? INT_MAX : INT_MIN;
}

// centroid * 2 = lo + hi (stays an exact integer)
__global__ void k_bounds(DevScenes g, int *bounds)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= g.total_facets) return;
    const int *b = g.box + 6 * (size_t)f;
    int *B = bounds + 6 * g.fscene[f];
    for (int a = 0; a < 3; a++) {
        int c = b[a] + b[3 + a];
        atomicMin(B + a, c);
        atomicMax(B + 3 + a, c);
    }
}

__device__ __forceinline__ unsigned long long spread10(unsigned v)
{
    unsigned long long x = v & 0x3ffu;
    x = (x | (x << 16)) & 0x30000ffull;
    x = (x | (x << 8)) & 0x300f00full;
    x = (x | (x << 4)) & 0x30c30c3ull;
    x = (x | (x << 2)) & 0x9249249ull;
    return x;
}

__global__ void k_morton(DevScenes g, const int *bounds)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= g.total_facets) return;
    const int sc = g.fscene[f];
    const int *b = g.box + 6 * (size_t)f;
    const int *B = bounds + 6 * sc;
    // One scale for all three axes (the largest centroid span): a city is far
    // wider than it is tall, and stretching each axis to its own span would
    // give a few metres of height as many Morton levels as a kilometre of
    // ground, scattering neighbours along the curve.
    long long span = 0;
    for (int a = 0; a < 3; a++) span = max(span, (long long)B[3 + a] - B[a]);
    unsigned q[3];
    for (int a = 0; a < 3; a++) {
        long long c = (long long)b[a] + b[3 + a];
        q[a] = span > 0 ? (unsigned)(((c - B[a]) * 1023) / span) : 0u;
    }
    unsigned long long code = spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2);
    // A facet spanning more than 1/4 of the scene in x or y (the ground) would
    // give every ancestor in the Morton order a scene-sized box; its key gets
    // the top bit so the root splits such facets off into their own subtree.
    bool large = false;
    for (int a = 0; a < 2; a++) {
        long long ext = 2LL * ((long long)b[3 + a] - b[a]);   // in centroid (lo + hi) units
        long long span = (long long)B[3 + a] - B[a];
        large |= span > 0 && 4 * ext > span;
    }
    g.keys[f] = (large ? (1ull << 63) : 0ull) | (code << 32) | (unsigned)(f - g.desc[sc].facet0);
}

// grid (ceil(maxN / 256), n_scenes): thread = one key of scene blockIdx.y
__global__ void k_rank_sort(DevScenes g, unsigned long long *sorted)
{
    __shared__ unsigned long long tile[256];
    const SceneDesc D = g.desc[blockIdx.y];
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (blockIdx.x * 256 >= D.n) return;   // whole block idle (uniform)
    unsigned long long mine = i < D.n ? g.keys[D.facet0 + i] : 0ull;
    int rank = 0;
    for (int t0 = 0; t0 < D.n; t0 += 256) {
        int j = t0 + threadIdx.x;
        tile[threadIdx.x] = j < D.n ? g.keys[D.facet0 + j] : ~0ull;
        __syncthreads();
        int m = min(256, D.n - t0);
        for (int k = 0; k < m; k++) rank += tile[k] < mine;
        __syncthreads();
    }
    if (i < D.n) {
        sorted[D.facet0 + rank] = mine;
        g.order[D.facet0 + rank] = D.facet0 + (int)(mine & 0xffffffffu);
        g.leaf[D.facet0 + (int)(mine & 0xffffffffu)].pad = rank;   // sorted position
    }
}

__device__ __forceinline__ int delta(const unsigned long long *k, int n, int i, int j)
{
    if (j < 0 || j >= n) return -1;
    return __clzll(k[i] ^ k[j]);
}

// Parent links: parent[leaf facet] and parent[total_facets + node] hold
// (parent node << 1) | side, or -1 for a root.
__global__ void k_karras(DevScenes g, const unsigned long long *sorted)
{
    const SceneDesc D = g.desc[blockIdx.y];
    const int i = blockIdx.x * 256 + threadIdx.x;
    const int n = D.n;
    if (i == 0 && n == 1) g.parent[D.facet0] = -1;
    if (i >= n - 1) return;
    const unsigned long long *k = sorted + D.facet0;
    const int d = (delta(k, n, i, i + 1) - delta(k, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = delta(k, n, i, i - d);
    int lmax = 2;
    while (delta(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(k, n, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = delta(k, n, i, j);
    int s = 0;
    for (int div = 2;; div <<= 1) {
        int t = (l + div - 1) / div;
        if (delta(k, n, i, i + (s + t) * d) > dnode) s += t;
        if (t == 1) break;
    }
    const int gam = i + s * d + min(d, 0);
    const int lo = min(i, j), hi = max(i, j);
    const int node = D.node0 + i;
    int left, right;
    if (lo == gam) {
        int f = g.order[D.facet0 + gam];
        left = ~f;
        g.parent[f] = (node << 1) | 0;
    } else {
        left = D.node0 + gam;
        g.parent[g.total_facets + left] = (node << 1) | 0;
    }
    if (hi == gam + 1) {
        int f = g.order[D.facet0 + gam + 1];
        right = ~f;
        g.parent[f] = (node << 1) | 1;
    } else {
        right = D.node0 + gam + 1;
        g.parent[g.total_facets + right] = (node << 1) | 1;
    }
    g.nodes[node].d = make_int4(left, right, lo, hi);   // + the node's sorted range
    if (i == 0) g.parent[g.total_facets + node] = -1;
}

__device__ __forceinline__ void write_slot(Node *nodes, int parent_side, const float *bx)
{
    float *p = reinterpret_cast<float *>(nodes + (parent_side >> 1)) + 6 * (parent_side & 1);
    for (int a = 0; a < 6; a++) p[a] = bx[a];
}

// Thread per facet walks towards the root; the second child to arrive at a
// node merges both slots and continues.  No thread waits on another.
__global__ void k_refit(DevScenes g)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= g.total_facets) return;
    // boxes are stored enlarged by half a unit (see seg_box in traverse.cuh)
    float bx[6];
    const int *b = g.box + 6 * (size_t)f;
    for (int a = 0; a < 3; a++) {
        bx[a] = (float)b[a] - 0.5f;
        bx[3 + a] = (float)b[3 + a] + 0.5f;
    }
    int ps = g.parent[f];
    int guard = 0;
    while (ps >= 0 && guard++ < 128) {
        write_slot(g.nodes, ps, bx);
        __threadfence();
        const int node = ps >> 1;
        if (atomicAdd(g.visits + node, 1) == 0) return;   // sibling not there yet
        __threadfence();
        const float *q = reinterpret_cast<const float *>(g.nodes + node);
        float L[6], R[6];
        for (int a = 0; a < 6; a++) { L[a] = __ldcg(q + a); R[a] = __ldcg(q + 6 + a); }
        for (int a = 0; a < 3; a++) {
            bx[a] = fminf(L[a], R[a]);
            bx[3 + a] = fmaxf(L[3 + a], R[3 + a]);
        }
        ps = __ldcg(g.parent + g.total_facets + node);
    }
}

cudaError_t launch_bvh(const DevScenes &g, cudaStream_t st)
{
    int nb = (g.total_facets + 255) / 256;
    k_bounds_init<<<(6 * g.n_scenes + 255) / 256, 256, 0, st>>>(g.bounds, g.n_scenes);
    k_bounds<<<nb, 256, 0, st>>>(g, g.bounds);
    k_morton<<<nb, 256, 0, st>>>(g, g.bounds);
    dim3 grid((g.max_n + 255) / 256, g.n_scenes);
    k_rank_sort<<<grid, 256, 0, st>>>(g, g.sorted);
    k_karras<<<grid, 256, 0, st>>>(g, g.sorted);
    if (g.total_nodes > 0) {
        // the refit's arrival counters must start at zero: a failed clear
        // would leave the previous call's counts, so it ends the build here
        cudaError_t e = cudaMemsetAsync(g.visits, 0, sizeof(int) * (size_t)g.total_nodes, st);
        if (e != cudaSuccess) {
            note_launches(5);
            return e;
        }
    }
    k_refit<<<nb, 256, 0, st>>>(g);
    note_launches(7);
    return cudaGetLastError();
}

}  // namespace ivm
