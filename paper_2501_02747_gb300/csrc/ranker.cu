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

__global__ void k_cbox_float(int *ctx, int n_scenes)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_scenes * 6 * kRClusters) return;
    int *C = ctx + (size_t)kRCtx * (i / (6 * kRClusters));
    const int k = i % (6 * kRClusters);
    C[kRCFBox + k] = __float_as_int(2.f * (float)C[kRCBox + k]);
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
    k_cbox_float<<<(n + 255) / 256, 256, 0, st>>>(ctx, g.n_scenes);
    note_launches(4);
    return cudaGetLastError();
}

// ------------------------------------------------------------ inference

// tcgen05 (5th-generation tensor cores) in inline PTX.  One CTA per SM holds
// the BF16 weights of all four layers in shared memory (100 KB) and 128
// columns of tensor memory (TMEM) for the accumulator; it takes tiles of 128
// candidate pairs (M = 128, one TMEM lane per pair).  Per tile: the features
// go to shared memory as the A operand of layer 1; thread 0 issues the
// layer's MMAs (K = 16 each) and commits them to an mbarrier; all threads
// wait on it, read their rows of the accumulator with tcgen05.ld, add the
// bias, apply ReLU, and write BF16 activations back to shared memory as the
// next layer's A operand.  After layer 4, the top 8 of each row's 64 logits
// are packed one byte each.  Operands use the canonical K-major layout with
// no swizzling (canon_off): the shared-memory descriptors carry the start
// address, the 128-byte stride between core matrices along K and the stride
// between 8-row groups.  Every wait on the mbarrier has an iteration limit;
// a wait that runs out raises IVM_ERR_TIMEOUT, and the CTA still releases
// its tensor memory before it returns.

constexpr int kTcThreads = 512;          // two warpgroups of 8 warps, one tile in flight each
constexpr int kTcGroup = 256;            // threads per warpgroup
constexpr int kTcParts = 2;              // threads of a warpgroup per pair (row)
constexpr int kTcRows = 128;             // pairs per tile (MMA M)
constexpr size_t kTcABytes = sizeof(__nv_bfloat16) * kTcRows * kRH;        // one A buffer
constexpr size_t kTcOffA = sizeof(__nv_bfloat16) * kRTEnd;                  // after the weights
constexpr size_t kTcOffBar = kTcOffA + 2 * kTcABytes;
constexpr size_t kTcSmem = kTcOffBar + 64;
constexpr uint32_t kTcCols = 256;        // TMEM columns: 128 fp32 per warpgroup
constexpr int kTcWaitLimit = 1 << 20;   // try_wait rounds before IVM_ERR_TIMEOUT

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading (along K) and
// stride (between 8-row groups) byte offsets, descriptor version 1, no
// swizzling, base offset 0.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N / 8 and M / 16 in their fields.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                 "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Waits for the mbarrier phase of parity `ph`; false when the limit ran out.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t ph)
{
    uint32_t done = 0;
    for (int it = 0; it < kTcWaitLimit && !done; it++)
        asm volatile("{\n\t.reg .pred P1;\n\tmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
                     "selp.b32 %0, 1, 0, P1;\n\t}"
                     : "=r"(done)
                     : "r"(mbar), "r"(ph));
    return done != 0;
}

// 16 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[j]);
}

// One layer: K / 16 MMAs from the A buffer and weight block w (B operand,
// N rows), into TMEM; issued by thread 0, completion on the mbarrier.
__device__ __forceinline__ void tc_layer(uint32_t tmem, uint32_t a_addr, uint32_t w_addr, int K,
                                         int N, uint32_t mbar)
{
    const uint32_t sbo = (uint32_t)(K / 8) * 128u, idesc = tc_idesc(kTcRows, N);
    for (int ks = 0; ks < K / 16; ks++)
        tc_mma(tmem, tc_desc(a_addr + 256u * ks, 128u, sbo), tc_desc(w_addr + 256u * ks, 128u, sbo),
               idesc, ks > 0);
    tc_commit(mbar);
}

// Bias and ReLU of this thread's 64 accumulator columns [c0, c0 + 64) of
// TMEM lane `row`, written as BF16 to the A buffer (K = 128 layout).
__device__ __forceinline__ void tc_hidden(uint32_t trow, int row, int c0, const float *bias,
                                          __nv_bfloat16 *A)
{
#pragma unroll
    for (int c = 0; c < 64; c += 16) {
        float v[16];
        tc_ld16(trow + (uint32_t)(c0 + c), v);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            __align__(16) __nv_bfloat162 q[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int k = 8 * h + 2 * j;
                q[j] = __floats2bfloat162_rn(fmaxf(v[k] + __ldg(bias + c0 + c + k), 0.f),
                                             fmaxf(v[k + 1] + __ldg(bias + c0 + c + k + 1), 0.f));
            }
            *reinterpret_cast<uint4 *>(A + canon_off(row, c0 + c + 8 * h, kRH)) =
                *reinterpret_cast<const uint4 *>(q);
        }
    }
}

// Barrier of one warpgroup (named barrier 1 + group, 256 threads).
__device__ __forceinline__ void group_sync(int group)
{
    asm volatile("bar.sync %0, %1;" ::"r"(1 + group), "r"(kTcGroup) : "memory");
}

// The k best of a thread's 32 logits, best first (ties to the lower column).
__device__ __forceinline__ void top_of32(const float (&z)[32], int c0, float (&bv)[kRTop],
                                         int (&bc)[kRTop])
{
    unsigned taken = 0;
#pragma unroll
    for (int k = 0; k < kRTop; k++) {
        float v = -INFINITY;
        int c = 255;
#pragma unroll
        for (int j = 0; j < 32; j++) {
            const bool free = !((taken >> j) & 1u);
            if (free && (z[j] > v || (z[j] == v && c0 + j < c))) { v = z[j]; c = c0 + j; }
        }
        if (c < 255) taken |= 1u << (c - c0);
        bv[k] = v;
        bc[k] = c;
    }
}

// Tiles of 128 candidate pairs (or precomputed feature rows when `feat` is
// given): 76 features, four layers on the tensor cores, then the top 8 of
// the 64 logits per pair (ties to the lower cluster) packed one byte each.
// The two warpgroups take alternate tiles, each with its own A buffer, TMEM
// columns and mbarrier, so that one group's MMAs run while the other works.
__global__ void __launch_bounds__(kTcThreads, 1)
k_rank_pairs(DevScenes g, const int2 *pairs, unsigned long long npairs,
             const unsigned long long *count_dev, const int *ctx, RankerDev r,
             unsigned long long *ranks, const float *feat, float *logits, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int group = tid / kTcGroup, gtid = tid % kTcGroup, gwarp = warp & 7;
    __nv_bfloat16 *W = reinterpret_cast<__nv_bfloat16 *>(smem);
    __nv_bfloat16 *A = reinterpret_cast<__nv_bfloat16 *>(smem + kTcOffA + group * kTcABytes);
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem + kTcOffBar);
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + kTcOffBar + 16);
    int *stop = reinterpret_cast<int *>(smem + kTcOffBar + 24);   // [2] per group
    // after layer 4 a group's A buffer holds each row's candidates: [row][part][k]
    float *cv = reinterpret_cast<float *>(A);
    int *ci = reinterpret_cast<int *>(A) + kTcRows * kTcParts * kRTop;
    for (int i = tid; i < kRTEnd / 8; i += kTcThreads)
        reinterpret_cast<uint4 *>(W)[i] = __ldg(reinterpret_cast<const uint4 *>(r.wt) + i);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar + 1)));
        stop[0] = stop[1] = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(slot)),
                     "r"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    async_proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot + 128u * group;
    const uint32_t mbar = smem_u32(bar + group), a_addr = smem_u32(A), w_addr = smem_u32(W);
    unsigned long long total = npairs;
    if (count_dev && *count_dev < total) total = *count_dev;
    const unsigned long long ntiles = (total + kTcRows - 1) / kTcRows;
    // features: thread -> (row, half of the 80 columns); accumulator: warp
    // w reads TMEM lanes 32 (w % 4) .. + 31, two warps of the group per lane
    // quarter, each with half of the columns
    const int row = gtid & (kTcRows - 1), part = gtid >> 7;
    const int arow = 32 * (gwarp & 3) + lane, apart = gwarp >> 2;
    const uint32_t trow = tmem + ((uint32_t)(32 * (gwarp & 3)) << 16);
    const float *bias = r.master;
    const int k0 = 40 * part;
    uint32_t ph = 0;
    for (unsigned long long tile = 2ull * blockIdx.x + group; tile < ntiles;
         tile += 2ull * gridDim.x) {
        const unsigned long long base = tile * kTcRows;
        {
            const unsigned long long p = base + row;
            const bool in = p < total;
            Leaf Li = {}, Lj = {};
            int sc = 0;
            if (in && !feat) {
                const int2 pr = pairs[p];
                Li = load_leaf(g.leaf, pr.x);
                Lj = load_leaf(g.leaf, pr.y);
                sc = Li.scene;
            }
            const int *bounds = feat ? nullptr : g.bounds + 6 * sc;
            const int *cb = feat ? nullptr : ctx + (size_t)kRCtx * sc;
            const PairGeom G(Li, Lj);
            for (int c = k0; c < k0 + 40; c += 8) {
                float v[8];
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const int f = c + j;
                    v[j] = !in || f >= kRIn ? 0.f
                         : (feat ? __ldg(feat + p * kRIn + f) : pair_feature(f, G, Li, Lj, bounds, cb));
                }
                __align__(16) __nv_bfloat162 q[4];
#pragma unroll
                for (int j = 0; j < 4; j++) q[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                *reinterpret_cast<uint4 *>(A + canon_off(row, c, kRK1)) =
                    *reinterpret_cast<const uint4 *>(q);
            }
        }
        async_proxy_fence();
        tc_fence_before();
        group_sync(group);
        bool ok = true;
        // layers 1-4: 80 -> 128, 128 -> 128, 128 -> 128 (ReLU), 128 -> 64
#pragma unroll
        for (int l = 0; l < 4; l++) {
            const int K = l == 0 ? kRK1 : kRH, N = l == 3 ? kROut : kRH;
            const int wbase = l == 0 ? kRT1 : (l == 1 ? kRT2 : (l == 2 ? kRT3 : kRT4));
            if (gtid == 0) {
                tc_fence_after();
                tc_layer(tmem, a_addr, w_addr + 2u * wbase, K, N, mbar);
            }
            if (!tc_wait(mbar, ph)) stop[group] = 1;
            ph ^= 1u;
            group_sync(group);
            if (stop[group]) { ok = false; break; }
            tc_fence_after();
            if (l < 3) {
                const int bbase = l == 0 ? kRB1 : (l == 1 ? kRB2 : kRB3);
                tc_hidden(trow, arow, 64 * apart, bias + bbase, A);
                async_proxy_fence();
                tc_fence_before();
                group_sync(group);
            }
        }
        if (!ok) break;
        {   // each thread: 32 of its row's logits, their best 8 as candidates
            const int c0 = 32 * apart;
            float z[32];
            {
                float v[16];
                tc_ld16(trow + (uint32_t)c0, v);
#pragma unroll
                for (int j = 0; j < 16; j++) z[j] = v[j];
                tc_ld16(trow + (uint32_t)(c0 + 16), v);
#pragma unroll
                for (int j = 0; j < 16; j++) z[16 + j] = v[j];
            }
#pragma unroll
            for (int j = 0; j < 32; j++) z[j] += __ldg(bias + kRB4 + c0 + j);
            const unsigned long long p = base + arow;
            if (logits && p < total) {
#pragma unroll
                for (int j = 0; j < 32; j++) logits[p * kROut + c0 + j] = z[j];
            }
            float bv[kRTop];
            int bc[kRTop];
            top_of32(z, c0, bv, bc);
            const int o = (arow * kTcParts + apart) * kRTop;
#pragma unroll
            for (int k = 0; k < kRTop; k++) { cv[o + k] = bv[k]; ci[o + k] = bc[k]; }
        }
        tc_fence_before();
        group_sync(group);
        if (gtid < kTcRows) {   // merge the two sorted candidate lists of row `gtid`
            const unsigned long long p = base + gtid;
            int ha = 0, hb = 0;
            unsigned long long packed = 0;
            const int o = gtid * kTcParts * kRTop;
#pragma unroll
            for (int k = 0; k < kRTop; k++) {
                // a list holds 8 and 8 are taken in all, so a head past its
                // list is never compared
                const float va = ha < kRTop ? cv[o + ha] : -INFINITY;
                const int ca = ha < kRTop ? ci[o + ha] : 256;
                const float vb = hb < kRTop ? cv[o + kRTop + hb] : -INFINITY;
                const int cb2 = hb < kRTop ? ci[o + kRTop + hb] : 256;
                const bool take_a = va > vb || (va == vb && ca < cb2);
                packed |= (unsigned long long)((take_a ? ca : cb2) & 0xff) << (8 * k);
                ha += take_a;
                hb += !take_a;
            }
            if (p < total) ranks[p] = packed;
        }
        group_sync(group);   // the accumulator and the A buffer are free for the next tile
    }
    if (gtid == 0 && stop[group]) raise_error(err, IVM_ERR_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*slot),
                     "r"(kTcCols));
    }
}

cudaError_t ranker_rank_pairs(const DevScenes &g, const int2 *pairs, unsigned long long npairs,
                              const unsigned long long *count_dev, const int *ctx,
                              const RankerDev &r, unsigned long long *ranks, int n_sm, int *err,
                              cudaStream_t st)
{
    if (npairs == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_rank_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTcSmem);
    if (e != cudaSuccess) return e;
    const unsigned long long tiles = (npairs + 2 * kTcRows - 1) / (2 * kTcRows);   // tile pairs
    const unsigned blocks = (unsigned)(tiles < (unsigned long long)n_sm ? tiles : n_sm);
    k_rank_pairs<<<blocks, kTcThreads, kTcSmem, st>>>(g, pairs, npairs, count_dev, ctx, r, ranks,
                                                      nullptr, nullptr, err);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t ranker_infer(const float *feat, unsigned long long n, const RankerDev &r,
                         float *logits, unsigned long long *ranks, int n_sm, int *err,
                         cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_rank_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTcSmem);
    if (e != cudaSuccess) return e;
    const unsigned long long tiles = (n + 2 * kTcRows - 1) / (2 * kTcRows);   // tile pairs
    const unsigned blocks = (unsigned)(tiles < (unsigned long long)n_sm ? tiles : n_sm);
    k_rank_pairs<<<blocks, kTcThreads, kTcSmem, st>>>(DevScenes{}, nullptr, n, nullptr, nullptr, r,
                                                      ranks, feat, logits, err);
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
        feat[w * kRInPad + f] = pair_feature(f, G, Li, Lj, g.bounds + 6 * Li.scene, C);
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

// Thread per (n, k) of the four W^T blocks in natural order; writes the BF16
// value to its place in the canonical layout (zero in layer 1's padding).
__global__ void k_pack(const float *m, __nv_bfloat16 *wt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kRTEnd) return;
    int base, K, n, k;
    float v = 0.f;
    if (i < kRT2) {                        // W1^T [128][80]
        base = kRT1; K = kRK1; n = i / kRK1; k = i % kRK1;
        if (k < kRIn) v = m[kRW1 + k * kRH + n];
    } else if (i < kRT3) {                 // W2^T [128][128]
        const int j = i - kRT2;
        base = kRT2; K = kRH; n = j / kRH; k = j % kRH;
        v = m[kRW2 + k * kRH + n];
    } else if (i < kRT4) {                 // W3^T [128][128]
        const int j = i - kRT3;
        base = kRT3; K = kRH; n = j / kRH; k = j % kRH;
        v = m[kRW3 + k * kRH + n];
    } else {                               // W4^T [64][128]
        const int j = i - kRT4;
        base = kRT4; K = kRH; n = j / kRH; k = j % kRH;
        v = m[kRW4 + k * kROut + n];
    }
    wt[base + canon_off(n, k, K)] = __float2bfloat16(v);
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
