// ranker.cu -- the learned occluder ranking: cluster boxes, tensor-core
// inference over candidate pairs, hit logging for training labels, and the
// FP32 training kernels (forward, backward, softmax cross-entropy, Adam).
// See ranker.cuh for what the network sees and why it can never change a bit.
#include <climits>

#include "ranker.cuh"

namespace ivm {

// ------------------------------------------------------------ clusters

// Warp per scene: the cut of at most 64 subtrees.  Starting from the root,
// each round splits every frontier node covering at least half as many
// facets as the largest one (the largest first, while the count allows), so
// big subtrees are split before small ones in a few dependent rounds.  The
// cut is sorted by range start into the scene's context block, and ncl marks
// its internal nodes.  Lane k holds frontier entries k and k + 32.
__global__ void k_cut(DevScenes g, int *ctx, signed char *ncl)
{
    __shared__ int s_ref[4][kRClusters], s_lo[4][kRClusters], s_hi[4][kRClusters];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sc = blockIdx.x * 4 + warp;
    if (sc >= g.n_scenes) return;
    const SceneDesc D = g.desc[sc];
    int *C = ctx + (size_t)kRCtx * sc;
    int *ref = s_ref[warp], *lo = s_lo[warp], *hi = s_hi[warp];
    auto range_of = [&](int r, int &a, int &b) {
        if (r >= 0) {
            const int4 d = g.nodes[r].d;
            a = d.z;
            b = d.w;
        } else {
            a = b = g.leaf[~r].pad;
        }
    };
    int cnt = 0;
    if (D.n > 0) {
        if (lane == 0) {
            ref[0] = D.root;
            range_of(D.root, lo[0], hi[0]);
        }
        cnt = 1;
    }
    __syncwarp();
    for (int round = 0; round < kRClusters && cnt < kRClusters; round++) {
        // widest internal entry
        int wmax = 0;
        for (int k = lane; k < cnt; k += 32)
            if (ref[k] >= 0) wmax = max(wmax, hi[k] - lo[k] + 1);
        for (int o = 16; o; o >>= 1) wmax = max(wmax, __shfl_xor_sync(kFull, wmax, o));
        if (wmax == 0) break;   // only leaves left
        // candidates: internal, at least half the widest; keep the widest
        // kRClusters - cnt of them (ties to the lower range start)
        const int budget = kRClusters - cnt;
        bool split[2] = {false, false};
        for (int h = 0; h < 2; h++) {
            const int k = lane + 32 * h;
            if (k >= cnt || ref[k] < 0) continue;
            const int w = hi[k] - lo[k] + 1;
            if (2 * w < wmax) continue;
            int better = 0;
            for (int m = 0; m < cnt; m++) {
                if (ref[m] < 0) continue;
                const int wm = hi[m] - lo[m] + 1;
                if (2 * wm >= wmax && (wm > w || (wm == w && lo[m] < lo[k]))) better++;
            }
            split[h] = better < budget;
        }
        // children of the split entries: left in place, right appended
        const unsigned b0 = __ballot_sync(kFull, split[0]), b1 = __ballot_sync(kFull, split[1]);
        const unsigned below = (1u << lane) - 1u;
        int nl[2], nr[2], la[2], lb[2], ra[2], rb[2];
        for (int h = 0; h < 2; h++) {
            if (!split[h]) continue;
            const int4 d = g.nodes[ref[lane + 32 * h]].d;
            nl[h] = d.x;
            nr[h] = d.y;
            range_of(nl[h], la[h], lb[h]);
            range_of(nr[h], ra[h], rb[h]);
        }
        __syncwarp();
        for (int h = 0; h < 2; h++) {
            if (!split[h]) continue;
            const int k = lane + 32 * h;
            const int slot = cnt + (h == 0 ? __popc(b0 & below) : __popc(b0) + __popc(b1 & below));
            ref[k] = nl[h]; lo[k] = la[h]; hi[k] = lb[h];
            ref[slot] = nr[h]; lo[slot] = ra[h]; hi[slot] = rb[h];
        }
        cnt += __popc(b0) + __popc(b1);
        __syncwarp();
    }
    // sort by range start: the ranges partition [0, n), so the rank of an
    // entry is the number of entries that start before it
    for (int h = 0; h < 2; h++) {
        const int k = lane + 32 * h;
        int r = 0, myref = 0, mylo = 0;
        if (k < cnt) {
            myref = ref[k];
            mylo = lo[k];
            for (int m = 0; m < cnt; m++) r += lo[m] < mylo;
            C[kRCut + r] = myref;
            C[kRCStart + r] = mylo;
            if (myref >= 0) ncl[myref] = (signed char)r;
        } else if (k < kRClusters) {
            C[kRCut + k] = D.root;
            C[kRCStart + k] = D.n;
        }
    }
    if (lane == 0) C[kRCStart + kRClusters] = D.n;
}

__global__ void k_cbox_init(int *ctx, int n_scenes)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_scenes * 6 * kRClusters) return;
    const int sc = i / (6 * kRClusters), k = i % (6 * kRClusters);
    ctx[(size_t)kRCtx * sc + kRCBox + k] = (k % 6) < 3 ? INT_MAX : INT_MIN;
}

__global__ void k_cbox(DevScenes g, int *ctx)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= g.total_facets) return;
    int *C = ctx + (size_t)kRCtx * g.fscene[f];
    const int c = cluster_at(C + kRCStart, g.leaf[f].pad);
    int *B = C + kRCBox + 6 * c;
    const int *b = g.box + 6 * (size_t)f;
    for (int a = 0; a < 3; a++) {
        atomicMin(B + a, b[a]);
        atomicMax(B + 3 + a, b[3 + a]);
    }
}

cudaError_t ranker_clusters(const DevScenes &g, int *ctx, signed char *ncl, cudaStream_t st)
{
    cudaError_t e;
    if (g.total_nodes > 0 &&
        (e = cudaMemsetAsync(ncl, 0xff, (size_t)g.total_nodes, st)) != cudaSuccess)
        return e;
    k_cut<<<(g.n_scenes + 3) / 4, 128, 0, st>>>(g, ctx, ncl);
    const int n = 6 * kRClusters * g.n_scenes;
    k_cbox_init<<<(n + 255) / 256, 256, 0, st>>>(ctx, g.n_scenes);
    k_cbox<<<(g.total_facets + 255) / 256, 256, 0, st>>>(g, ctx);
    note_launches(3);
    return cudaGetLastError();
}

// ------------------------------------------------------------ inference

__device__ __forceinline__ void mma_bf16(float *c, unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned pack_relu(float lo, float hi)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(lo, 0.f), fmaxf(hi, 0.f));
    return *reinterpret_cast<unsigned *>(&h);
}

__device__ __forceinline__ unsigned lds32(const __nv_bfloat16 *p)
{
    return *reinterpret_cast<const unsigned *>(p);
}

// One hidden layer 128 -> 128 from A fragments `a` (8 k-steps); result in acc.
__device__ __forceinline__ void layer128(const unsigned (&a)[8][4], const __nv_bfloat16 *Wt,
                                         const float *bias, float (&acc)[16][4], int r0, int q)
{
#pragma unroll
    for (int t = 0; t < 16; t++) {
        const float b0 = bias[8 * t + 2 * q], b1 = bias[8 * t + 2 * q + 1];
        acc[t][0] = b0; acc[t][1] = b1; acc[t][2] = b0; acc[t][3] = b1;
    }
#pragma unroll
    for (int s = 0; s < 8; s++)
#pragma unroll
        for (int t = 0; t < 16; t++) {
            const __nv_bfloat16 *w = Wt + (8 * t + r0) * kRS2 + 16 * s + 2 * q;
            mma_bf16(acc[t], a[s][0], a[s][1], a[s][2], a[s][3], lds32(w), lds32(w + 8));
        }
}

__device__ __forceinline__ void to_frags(const float (&acc)[16][4], unsigned (&a)[8][4])
{
#pragma unroll
    for (int s = 0; s < 8; s++) {
        a[s][0] = pack_relu(acc[2 * s][0], acc[2 * s][1]);
        a[s][1] = pack_relu(acc[2 * s][2], acc[2 * s][3]);
        a[s][2] = pack_relu(acc[2 * s + 1][0], acc[2 * s + 1][1]);
        a[s][3] = pack_relu(acc[2 * s + 1][2], acc[2 * s + 1][3]);
    }
}

constexpr int kRankWarps = 12;   // one block per SM (the weights fill most of shared memory)
constexpr size_t kRankSmem = sizeof(__nv_bfloat16) * (kRTEnd + kRankWarps * 16 * kRS1);

// Warp per 16 candidate pairs: features into shared memory, four layers on
// the tensor cores with the activations kept in registers, then the top 8
// logits per pair (ties to the lower cluster) packed one byte each.
__global__ void __launch_bounds__(32 * kRankWarps, 1)
k_rank_pairs(DevScenes g, const int2 *pairs, unsigned long long npairs,
             const unsigned long long *count_dev, const int *ctx, RankerDev r,
             unsigned long long *ranks, const float *feat, float *logits)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16 *W = reinterpret_cast<__nv_bfloat16 *>(smem);
    __nv_bfloat16 *F = W + kRTEnd;
    for (int i = threadIdx.x; i < kRTEnd / 8; i += blockDim.x)
        reinterpret_cast<uint4 *>(W)[i] = reinterpret_cast<const uint4 *>(r.wt)[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = lane >> 2, q = lane & 3;
    unsigned long long total = npairs;
    if (count_dev && *count_dev < total) total = *count_dev;
    __nv_bfloat16 *Fw = F + warp * 16 * kRS1;
    const float *bias = r.master;
    for (unsigned long long base = ((unsigned long long)blockIdx.x * kRankWarps + warp) * 16;
         base < total; base += (unsigned long long)gridDim.x * kRankWarps * 16) {
        {   // features: lane -> pair (lane & 15), half (lane >> 4) of the 80
            const int row = lane & 15;
            const unsigned long long p = base + row;
            const bool ok = p < total;
            const int f0 = (lane >> 4) * 40;
            if (feat) {   // precomputed feature rows [n][76]
                for (int f = f0; f < f0 + 40; f++)
                    Fw[row * kRS1 + f] = __float2bfloat16(ok && f < kRIn ? feat[p * kRIn + f] : 0.f);
            } else {
                Leaf Li = {}, Lj = {};
                int sc = 0;
                if (ok) {
                    const int2 pr = pairs[p];
                    Li = load_leaf(g.leaf, pr.x);
                    Lj = load_leaf(g.leaf, pr.y);
                    sc = Li.scene;
                }
                const int *bounds = g.bounds + 6 * sc;
                const int *cb = ctx + (size_t)kRCtx * sc + kRCBox;
                const PairGeom G(Li, Lj);
                for (int f = f0; f < f0 + 40; f += 2) {
                    const float v0 = ok ? pair_feature(f, G, Li, Lj, bounds, cb) : 0.f;
                    const float v1 = ok ? pair_feature(f + 1, G, Li, Lj, bounds, cb) : 0.f;
                    *reinterpret_cast<__nv_bfloat162 *>(Fw + row * kRS1 + f) =
                        __floats2bfloat162_rn(v0, v1);
                }
            }
        }
        __syncwarp();
        float acc[16][4];
        unsigned a[8][4];
        // layer 1: 80 -> 128
#pragma unroll
        for (int t = 0; t < 16; t++) {
            const float b0 = bias[kRB1 + 8 * t + 2 * q], b1 = bias[kRB1 + 8 * t + 2 * q + 1];
            acc[t][0] = b0; acc[t][1] = b1; acc[t][2] = b0; acc[t][3] = b1;
        }
#pragma unroll
        for (int s = 0; s < kRInPad / 16; s++) {
            const __nv_bfloat16 *x = Fw + r0 * kRS1 + 16 * s + 2 * q;
            const unsigned a0 = lds32(x), a1 = lds32(x + 8 * kRS1), a2 = lds32(x + 8),
                           a3 = lds32(x + 8 * kRS1 + 8);
#pragma unroll
            for (int t = 0; t < 16; t++) {
                const __nv_bfloat16 *w = W + kRT1 + (8 * t + r0) * kRS1 + 16 * s + 2 * q;
                mma_bf16(acc[t], a0, a1, a2, a3, lds32(w), lds32(w + 8));
            }
        }
        __syncwarp();   // features of this tile are consumed
        to_frags(acc, a);
        layer128(a, W + kRT2, bias + kRB2, acc, r0, q);
        to_frags(acc, a);
        layer128(a, W + kRT3, bias + kRB3, acc, r0, q);
        to_frags(acc, a);
        // layer 4: 128 -> 64
        float z[8][4];
#pragma unroll
        for (int t = 0; t < 8; t++) {
            const float b0 = bias[kRB4 + 8 * t + 2 * q], b1 = bias[kRB4 + 8 * t + 2 * q + 1];
            z[t][0] = b0; z[t][1] = b1; z[t][2] = b0; z[t][3] = b1;
        }
#pragma unroll
        for (int s = 0; s < 8; s++)
#pragma unroll
            for (int t = 0; t < 8; t++) {
                const __nv_bfloat16 *w = W + kRT4 + (8 * t + r0) * kRS2 + 16 * s + 2 * q;
                mma_bf16(z[t], a[s][0], a[s][1], a[s][2], a[s][3], lds32(w), lds32(w + 8));
            }
        if (logits) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const unsigned long long p = base + r0 + 8 * h;
                if (p < total)
#pragma unroll
                    for (int t = 0; t < 8; t++) {
                        logits[p * kROut + 8 * t + 2 * q] = z[t][2 * h];
                        logits[p * kROut + 8 * t + 2 * q + 1] = z[t][2 * h + 1];
                    }
            }
        }
        // top 8 of the 64 logits of rows r0 and r0 + 8 (a quad of lanes holds a row)
#pragma unroll
        for (int h = 0; h < 2; h++) {
            unsigned long long packed = 0;
            float v[16];
#pragma unroll
            for (int t = 0; t < 8; t++) {
                v[2 * t] = z[t][2 * h];
                v[2 * t + 1] = z[t][2 * h + 1];
            }
#pragma unroll
            for (int k = 0; k < kRTop; k++) {
                float bv = -INFINITY;
                int bc = 255;
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    const int col = 8 * (i >> 1) + 2 * q + (i & 1);
                    if (v[i] > bv || (v[i] == bv && col < bc)) { bv = v[i]; bc = col; }
                }
#pragma unroll
                for (int off = 1; off <= 2; off <<= 1) {
                    const float ov = __shfl_xor_sync(kFull, bv, off);
                    const int oc = __shfl_xor_sync(kFull, bc, off);
                    if (ov > bv || (ov == bv && oc < bc)) { bv = ov; bc = oc; }
                }
#pragma unroll
                for (int i = 0; i < 16; i++)
                    if (8 * (i >> 1) + 2 * q + (i & 1) == bc) v[i] = -INFINITY;
                packed |= (unsigned long long)(bc & 0xff) << (8 * k);
            }
            const unsigned long long p = base + r0 + 8 * h;
            if (q == 0 && p < total) ranks[p] = packed;
        }
    }
}

cudaError_t ranker_rank_pairs(const DevScenes &g, const int2 *pairs, unsigned long long npairs,
                              const unsigned long long *count_dev, const int *ctx,
                              const RankerDev &r, unsigned long long *ranks, int n_sm,
                              cudaStream_t st)
{
    if (npairs == 0) return cudaSuccess;
    cudaFuncSetAttribute(k_rank_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kRankSmem);
    const unsigned long long tiles = (npairs + 15) / 16;
    unsigned long long blocks = (tiles + kRankWarps - 1) / kRankWarps;
    if (blocks > (unsigned long long)n_sm) blocks = (unsigned long long)n_sm;
    k_rank_pairs<<<(unsigned)blocks, 32 * kRankWarps, kRankSmem, st>>>(
        g, pairs, npairs, count_dev, ctx, r, ranks, nullptr, nullptr);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t ranker_infer(const float *feat, unsigned long long n, const RankerDev &r,
                         float *logits, unsigned long long *ranks, int n_sm, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    cudaFuncSetAttribute(k_rank_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kRankSmem);
    const unsigned long long tiles = (n + 15) / 16;
    unsigned long long blocks = (tiles + kRankWarps - 1) / kRankWarps;
    if (blocks > (unsigned long long)n_sm) blocks = (unsigned long long)n_sm;
    k_rank_pairs<<<(unsigned)blocks, 32 * kRankWarps, kRankSmem, st>>>(
        DevScenes{}, nullptr, n, nullptr, nullptr, r, ranks, feat, logits);
    note_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------ hit logging

// Leaf test that never stops the walk but remembers the nearest facet the
// segment meets (by the plane parameter, for ordering only).
struct NearestHit {
    float *best_t;
    int *best_pos;
    __device__ __forceinline__ bool operator()(const Seg &s, const Leaf &L, WalkCounters &wc) const
    {
        if (facet_hit_exact(s, L)) {
            const double num = (double)L.nx * (L.ox - s.px) + (double)L.ny * (L.oy - s.py) +
                               (double)L.nz * (L.oz - s.pz);
            const double den = (double)L.nx * s.dx + (double)L.ny * s.dy + (double)L.nz * s.dz;
            const float t = den != 0.0 ? (float)(num / den) : 0.5f;
            if (t < *best_t) { *best_t = t; *best_pos = L.pad; }
        }
        return false;
    }
};

// Warp per candidate pair: the segment between the facets' central samples
// (the centroids for odd s); label = cluster of the nearest facet it meets,
// -1 when it is free or the central samples do not face each other.
__global__ void k_log_hits(DevScenes g, const int2 *pairs, unsigned long long npairs,
                           const int *ctx, float *feat, int *label, int *err)
{
    const unsigned long long w = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= npairs) return;
    const int2 pr = pairs[w];
    const Leaf Li = load_leaf(g.leaf, pr.x), Lj = load_leaf(g.leaf, pr.y);
    const SceneDesc &D = g.desc[Li.scene];
    const int s = D.s, mid = (s / 2) * s + s / 2;
    const int ia = D.sample0 + (pr.x - D.facet0) * s * s + mid;
    const int ib = D.sample0 + (pr.y - D.facet0) * s * s + mid;
    const int px = g.sx[ia], py = g.sy[ia], pz = g.sz[ia];
    const int qx = g.sx[ib], qy = g.sy[ib], qz = g.sz[ib];
    const int *C = ctx + (size_t)kRCtx * Li.scene;
    const PairGeom G(Li, Lj);
    for (int f = lane; f < kRInPad; f += 32)
        feat[w * kRInPad + f] = pair_feature(f, G, Li, Lj, g.bounds + 6 * Li.scene, C + kRCBox);
    const bool facing = front_of(Lj, px, py, pz) && front_of(Li, qx, qy, qz);
    float best_t = 2.f;
    int best_pos = -1;
    if (facing) {
        Seg sg = make_seg(px, py, pz, qx, qy, qz);
        finish_seg(sg);
        WalkCounters wc;
        int blocker, myblk = -1;
        NearestHit nh{&best_t, &best_pos};
        walk_packet(sg, 1u, g.nodes, g.leaf, D.root, (float)sg.dx, (float)sg.dy, (float)sg.dz,
                    D.budget, err, wc, nh, blocker, myblk);
    }
    if (lane == 0) label[w] = best_pos >= 0 ? cluster_at(C + kRCStart, best_pos) : -1;
}

cudaError_t ranker_log_hits(const DevScenes &g, const int2 *pairs, unsigned long long npairs,
                            const int *ctx, float *feat, int *label,
                            unsigned long long *cursor, unsigned long long cap, int *err,
                            cudaStream_t st)
{
    (void)cursor;
    (void)cap;
    if (npairs == 0) return cudaSuccess;
    k_log_hits<<<(unsigned)((npairs * 32 + 127) / 128), 128, 0, st>>>(g, pairs, npairs, ctx, feat,
                                                                    label, err);
    note_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------ weights

__global__ void k_pack(const float *m, __nv_bfloat16 *wt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kRTEnd) return;
    float v = 0.f;
    if (i < kRT2) {                        // W1^T [128][88]
        const int n = i / kRS1, k = i % kRS1;
        if (k < kRIn) v = m[kRW1 + k * kRH + n];
    } else if (i < kRT3) {
        const int j = i - kRT2, n = j / kRS2, k = j % kRS2;
        if (k < kRH) v = m[kRW2 + k * kRH + n];
    } else if (i < kRT4) {
        const int j = i - kRT3, n = j / kRS2, k = j % kRS2;
        if (k < kRH) v = m[kRW3 + k * kRH + n];
    } else {
        const int j = i - kRT4, n = j / kRS2, k = j % kRS2;
        if (k < kRH) v = m[kRW4 + k * kROut + n];
    }
    wt[i] = __float2bfloat16(v);
}

cudaError_t ranker_pack(const float *master, __nv_bfloat16 *wt, cudaStream_t st)
{
    k_pack<<<(kRTEnd + 255) / 256, 256, 0, st>>>(master, wt);
    note_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------ training (FP32)

// activations of a batch: x (B x 76 from the caller), h1, h2, h3 (B x 128),
// z (B x 64), and the gradients dz, dh3, dh2, dh1
size_t ranker_act_floats(int B) { return (size_t)B * (3 * kRH + 2 * kROut + 3 * kRH + 1); }

__global__ void k_fwd(const float *in, int in_dim, const float *Wm, const float *b, float *out,
                      int out_dim, int relu, int B)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * out_dim) return;
    const int r = i / out_dim, o = i % out_dim;
    float acc = b[o];
    for (int k = 0; k < in_dim; k++) acc += in[r * in_dim + k] * Wm[k * out_dim + o];
    out[i] = relu ? fmaxf(acc, 0.f) : acc;
}

// softmax cross-entropy per row: rowloss[r], dz = (p - onehot) / B
__global__ void k_softmax_ce(const float *z, const int *y, int B, float *dz, float *rowloss)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= B) return;
    const float *zr = z + r * kROut;
    float m = zr[0];
    for (int o = 1; o < kROut; o++) m = fmaxf(m, zr[o]);
    float sum = 0.f;
    for (int o = 0; o < kROut; o++) sum += expf(zr[o] - m);
    const float lse = m + logf(sum);
    rowloss[r] = lse - zr[y[r]];
    for (int o = 0; o < kROut; o++) dz[r * kROut + o] = (expf(zr[o] - lse) - (o == y[r])) / B;
}

__global__ void k_sum(const float *v, int n, float scale, float *out)
{
    __shared__ float sh[256];
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += 256) s += v[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] * scale;
}

// din[r][k] = sum_o dout[r][o] W[k][o], times [act[r][k] > 0] (ReLU)
__global__ void k_bwd_data(const float *dout, int out_dim, const float *Wm, float *din,
                           const float *act, int in_dim, int B)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * in_dim) return;
    const int r = i / in_dim, k = i % in_dim;
    float acc = 0.f;
    for (int o = 0; o < out_dim; o++) acc += dout[r * out_dim + o] * Wm[k * out_dim + o];
    din[i] = act[i] > 0.f ? acc : 0.f;
}

// gW[k][o] = sum_r in[r][k] dout[r][o]; gb[o] = sum_r dout[r][o]
__global__ void k_bwd_weight(const float *in, int in_dim, const float *dout, int out_dim,
                             float *gW, float *gb, int B)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (in_dim + 1) * out_dim) return;
    const int k = i / out_dim, o = i % out_dim;
    float acc = 0.f;
    if (k < in_dim) {
        for (int r = 0; r < B; r++) acc += in[r * in_dim + k] * dout[r * out_dim + o];
        gW[k * out_dim + o] = acc;
    } else {
        for (int r = 0; r < B; r++) acc += dout[r * out_dim + o];
        gb[o] = acc;
    }
}

static inline unsigned nb(long long n) { return (unsigned)((n + 255) / 256); }

cudaError_t ranker_grad(const float *m, const float *x, const int *y, int B, float *act,
                        float *grads, float *loss, cudaStream_t st)
{
    float *h1 = act, *h2 = h1 + (size_t)B * kRH, *h3 = h2 + (size_t)B * kRH;
    float *z = h3 + (size_t)B * kRH, *dz = z + (size_t)B * kROut;
    float *dh3 = dz + (size_t)B * kROut, *dh2 = dh3 + (size_t)B * kRH, *dh1 = dh2 + (size_t)B * kRH;
    float *rowloss = dh1 + (size_t)B * kRH;
    k_fwd<<<nb((long long)B * kRH), 256, 0, st>>>(x, kRIn, m + kRW1, m + kRB1, h1, kRH, 1, B);
    k_fwd<<<nb((long long)B * kRH), 256, 0, st>>>(h1, kRH, m + kRW2, m + kRB2, h2, kRH, 1, B);
    k_fwd<<<nb((long long)B * kRH), 256, 0, st>>>(h2, kRH, m + kRW3, m + kRB3, h3, kRH, 1, B);
    k_fwd<<<nb((long long)B * kROut), 256, 0, st>>>(h3, kRH, m + kRW4, m + kRB4, z, kROut, 0, B);
    k_softmax_ce<<<nb(B), 256, 0, st>>>(z, y, B, dz, rowloss);
    k_sum<<<1, 256, 0, st>>>(rowloss, B, 1.f / B, loss);
    k_bwd_weight<<<nb((long long)(kRH + 1) * kROut), 256, 0, st>>>(h3, kRH, dz, kROut,
                                                                   grads + kRW4, grads + kRB4, B);
    k_bwd_data<<<nb((long long)B * kRH), 256, 0, st>>>(dz, kROut, m + kRW4, dh3, h3, kRH, B);
    k_bwd_weight<<<nb((long long)(kRH + 1) * kRH), 256, 0, st>>>(h2, kRH, dh3, kRH, grads + kRW3,
                                                                 grads + kRB3, B);
    k_bwd_data<<<nb((long long)B * kRH), 256, 0, st>>>(dh3, kRH, m + kRW3, dh2, h2, kRH, B);
    k_bwd_weight<<<nb((long long)(kRH + 1) * kRH), 256, 0, st>>>(h1, kRH, dh2, kRH, grads + kRW2,
                                                                 grads + kRB2, B);
    k_bwd_data<<<nb((long long)B * kRH), 256, 0, st>>>(dh2, kRH, m + kRW2, dh1, h1, kRH, B);
    k_bwd_weight<<<nb((long long)(kRIn + 1) * kRH), 256, 0, st>>>(x, kRIn, dh1, kRH, grads + kRW1,
                                                                  grads + kRB1, B);
    note_launches(13);
    return cudaGetLastError();
}

// x[b][0..75] = feat[idx[b]][0..75], y[b] = label[idx[b]]
__global__ void k_gather(const float *feat, const int *label, const int *idx, int B, float *x,
                         int *y)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * kRIn) return;
    const int b = i / kRIn, f = i % kRIn;
    x[i] = feat[(size_t)idx[b] * kRInPad + f];
    if (f == 0) y[b] = label[idx[b]];
}

cudaError_t ranker_gather(const float *feat, const int *label, const int *idx, int B, float *x,
                          int *y, cudaStream_t st)
{
    k_gather<<<nb((long long)B * kRIn), 256, 0, st>>>(feat, label, idx, B, x, y);
    note_launches(1);
    return cudaGetLastError();
}

__global__ void k_adam(float *w, const float *g, float *m, float *v, float lr, float c1, float c2)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kRParams) return;
    const float gi = g[i];
    m[i] = 0.9f * m[i] + 0.1f * gi;
    v[i] = 0.999f * v[i] + 0.001f * gi * gi;
    w[i] -= lr * (m[i] * c1) / (sqrtf(v[i] * c2) + 1e-8f);
}

cudaError_t ranker_adam(float *master, const float *grads, float *m, float *v, float lr, int step,
                        cudaStream_t st)
{
    const float c1 = 1.f / (1.f - powf(0.9f, (float)step));
    const float c2 = 1.f / (1.f - powf(0.999f, (float)step));
    k_adam<<<nb(kRParams), 256, 0, st>>>(master, grads, m, v, lr, c1, c2);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace ivm
