// ranges.cu -- visibility ranges along the route (Sec. III-C, Tables III-IV),
// the Blockage column, and the coherence-time sums (Sec. III-D, Eq. (8)-(9)).
//
// A range is a maximal run [begin, end) of snapshots in which bit j of one
// side's table row is set: facet j is visible from the transmitter (side 0)
// or from the receiver (side 1) all along, and begin / end are the ray
// creation / suppression points.  Records are ordered by (side, facet, begin).
//
// Pass 1: warp per (side, word c, chunk of kRngChunk snapshots).  Lane l takes
// row t0 + 32 k + l; the row above it arrives by a shuffle, and a run starts
// where a bit is set that was clear one row before.  Ballots count the starts
// of each of the word's 32 facets.  Pass 2, after an exclusive scan over
// (side, facet, chunk): the same walk writes each start at its index and each
// end -- a bit set one row before and clear now, with an empty row after the
// route -- into the range of the last start above it.  Pass 3: at the
// snapshot before a range and at its end, the first facet on the segment from
// the source to facet j's centre sample (exact; smallest segment parameter,
// ties to the lower facet index), found by a BVH walk that never stops early.
#include "ranges.cuh"
#include "traverse.cuh"

namespace ivm {

// Facets of word c that exist (padding bits beyond n are ignored).
__device__ __forceinline__ uint32_t word_mask(int c, int n)
{
    const int k = n - 32 * c;
    return k >= 32 ? 0xffffffffu : ((1u << k) - 1u);
}

__global__ void k_rng_count(RangeArgs a)
{
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= 2LL * a.W * a.nchunks) return;   // uniform per warp
    const int chunk = (int)(w % a.nchunks);
    const long long sc = w / a.nchunks;
    const int c = (int)(sc % a.W), side = (int)(sc / a.W);
    const long long t0 = (long long)chunk * kRngChunk, t1 = min(t0 + kRngChunk, a.S);
    const uint32_t vm = word_mask(c, a.n);
    uint32_t carry = t0 > 0 ? (__ldg(a.table + ((size_t)(t0 - 1) * 2 + side) * a.W + c) & vm) : 0u;
    unsigned cnt = 0;
    unsigned long long set = 0;   // set bits: the summed lengths of the ranges
    for (long long tb = t0; tb < t1; tb += 32) {
        const long long t = tb + lane;
        const uint32_t cur = t < t1 ? (__ldg(a.table + ((size_t)t * 2 + side) * a.W + c) & vm) : 0u;
        uint32_t prev = __shfl_up_sync(kFull, cur, 1);
        if (lane == 0) prev = carry;
        carry = __shfl_sync(kFull, cur, 31);
        set += __popc(cur);
        const uint32_t starts = cur & ~prev;
        for (int b = 0; b < 32; b++) {
            const unsigned m = __ballot_sync(kFull, (starts >> b) & 1u);
            if (lane == b) cnt += __popc(m);
        }
    }
    const int j = 32 * c + lane;
    if (j < a.n) a.count[((long long)side * a.n + j) * a.nchunks + chunk] = cnt;
    for (int o = 16; o; o >>= 1) set += __shfl_xor_sync(kFull, set, o);
    if (lane == 0 && set) atomicAdd(a.sums + side, set);
}

__global__ void k_rng_write(RangeArgs a)
{
    __shared__ uint32_t s_ms[4][32];
    __shared__ long long s_base[4][32];
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w >= 2LL * a.W * a.nchunks) return;   // uniform per warp
    const int chunk = (int)(w % a.nchunks);
    const long long sc = w / a.nchunks;
    const int c = (int)(sc % a.W), side = (int)(sc / a.W);
    const long long t0 = (long long)chunk * kRngChunk, t1 = min(t0 + kRngChunk, a.S);
    // the last chunk also looks at the empty row after the route (ends at S)
    const long long tend = t1 == a.S ? a.S + 1 : t1;
    const uint32_t vm = word_mask(c, a.n);
    const int j = 32 * c + lane;
    s_base[warp][lane] = j < a.n ? a.off[((long long)side * a.n + j) * a.nchunks + chunk] : 0;
    uint32_t carry = t0 > 0 ? (__ldg(a.table + ((size_t)(t0 - 1) * 2 + side) * a.W + c) & vm) : 0u;
    __syncwarp();
    for (long long tb = t0; tb < tend; tb += 32) {
        const long long t = tb + lane;
        const uint32_t cur = t < t1 ? (__ldg(a.table + ((size_t)t * 2 + side) * a.W + c) & vm) : 0u;
        uint32_t prev = __shfl_up_sync(kFull, cur, 1);
        if (lane == 0) prev = carry;
        carry = __shfl_sync(kFull, cur, 31);
        const bool row = t < tend;
        const uint32_t starts = row ? (cur & ~prev) : 0u;
        const uint32_t ends = row ? (prev & ~cur) : 0u;
        for (int b = 0; b < 32; b++) {
            const unsigned m = __ballot_sync(kFull, (starts >> b) & 1u);
            if (lane == b) s_ms[warp][b] = m;
        }
        __syncwarp();
        const unsigned below = (1u << lane) - 1u;
        uint32_t todo = starts | ends;
        while (todo) {
            const int b = __ffs(todo) - 1;
            todo &= todo - 1;
            const long long idx = s_base[warp][b] + __popc(s_ms[warp][b] & below);
            if ((starts >> b) & 1u) {
                ivm_range &r = a.rec[idx];
                r.side = side;
                r.facet = 32 * c + b;
                r.begin = t;
            } else {   // the range of the last start above this row
                a.rec[idx - 1].end = t;
            }
        }
        __syncwarp();
        s_base[warp][lane] += __popc(s_ms[warp][lane]);
        __syncwarp();
    }
}

// Leaf test of the blocker walk: never stops the walk, keeps the first hit
// (smallest parameter l = ln / ld, then the lower facet index).
struct FirstHit {
    long long *ln, *ld;
    int *best;
    const int *order;   // sorted position -> global facet
    __device__ __forceinline__ bool operator()(const Seg &s, const Leaf &L, WalkCounters &wc) const
    {
        if (!facet_hit_exact(s, L)) return false;
        const long long sp = (long long)L.nx * (s.px - L.ox) + (long long)L.ny * (s.py - L.oy) +
                             (long long)L.nz * (s.pz - L.oz);
        const long long sq = sp + (long long)L.nx * s.dx + (long long)L.ny * s.dy +
                             (long long)L.nz * s.dz;
        long long n, d;
        if (sp == 0 && sq == 0) {
            coplanar_clip_v(s.px, s.py, s.pz, s.dx, s.dy, s.dz, L.ox, L.oy, L.oz, L.ux, L.uy, L.uz,
                            L.vx, L.vy, L.vz, L.dom, &n, &d);
        } else {
            n = sp;
            d = sp - sq;
            if (d < 0) { n = -n; d = -d; }
        }
        const int f = __ldg(order + L.pad);
        const __int128 lhs = (__int128)n * *ld, rhs = (__int128)*ln * d;
        if (*best < 0 || lhs < rhs || (lhs == rhs && f < *best)) {
            *ln = n;
            *ld = d;
            *best = f;
        }
        (void)wc;
        return false;
    }
};

// Item k: the snapshot before range k / 2 (k even) or its end (k odd).
__global__ void k_rng_blockers(DevScenes g, RangeArgs a, long long R, int *err)
{
    const int lane = threadIdx.x & 31;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long k0 = k - lane;
    if (k0 >= 2 * R) return;   // uniform per warp
    const SceneDesc &D = g.desc[0];
    const bool valid = k < 2 * R;
    int result = -1;
    bool walk = false;
    int px = 0, py = 0, pz = 0, qx = 0, qy = 0, qz = 0, j = 0;
    if (valid) {
        const ivm_range &r = a.rec[k >> 1];
        const long long t = (k & 1) ? r.end : r.begin - 1;
        j = r.facet;
        if (t >= 0 && t < a.S) {
            const int *pos = r.side ? a.rx : a.tx;
            const long long k2 = 2LL * D.s;
            const long long X0 = k2 * pos[3 * t], X1 = k2 * pos[3 * t + 1], X2 = k2 * pos[3 * t + 2];
            px = (int)X0; py = (int)X1; pz = (int)X2;
            const Leaf L = load_leaf(g.leaf, D.facet0 + j);
            if (X0 <= -kCoordLimit || X0 >= kCoordLimit || X1 <= -kCoordLimit ||
                X1 >= kCoordLimit || X2 <= -kCoordLimit || X2 >= kCoordLimit) {
                raise_error(err, IVM_ERR_RANGE);
                result = -1;
            } else if (!front_of(L, px, py, pz)) {
                result = -2;
            } else {
                const int si = D.sample0 + (j * D.s + D.s / 2) * D.s + D.s / 2;
                qx = g.sx[si]; qy = g.sy[si]; qz = g.sz[si];
                walk = true;
            }
        }
    }
    const unsigned alive = __ballot_sync(kFull, walk);
    if (alive) {
        Seg sg = make_seg(px, py, pz, qx, qy, qz);
        finish_seg(sg);
        const int lead = __ffs(alive) - 1;
        const float dx = (float)__shfl_sync(kFull, sg.dx, lead);
        const float dy = (float)__shfl_sync(kFull, sg.dy, lead);
        const float dz = (float)__shfl_sync(kFull, sg.dz, lead);
        long long ln = 1, ld = 1;
        int best = -1;
        WalkCounters wc;
        int blocker, myblk = -1;
        walk_packet(sg, alive, g.nodes, g.leaf, D.root, dx, dy, dz, D.budget, err, wc,
                    FirstHit{&ln, &ld, &best, g.order + D.facet0}, blocker, myblk);
        if (walk) result = best >= 0 ? best - D.facet0 : -3;   // -3: a facing hidden facet is blocked
    }
    if (valid) {
        ivm_range &r = a.rec[k >> 1];
        if (k & 1) r.block_after = result;
        else r.block_before = result;
    }
}

cudaError_t ranges_count(const RangeArgs &a, cudaStream_t st)
{
    const long long warps = 2LL * a.W * a.nchunks;
    k_rng_count<<<(unsigned)((warps * 32 + 127) / 128), 128, 0, st>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t ranges_write(const RangeArgs &a, cudaStream_t st)
{
    const long long warps = 2LL * a.W * a.nchunks;
    k_rng_write<<<(unsigned)((warps * 32 + 127) / 128), 128, 0, st>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t ranges_blockers(const DevScenes &g, const RangeArgs &a, long long R, int *err,
                            cudaStream_t st)
{
    if (R == 0) return cudaSuccess;
    k_rng_blockers<<<(unsigned)((2 * R + 127) / 128), 128, 0, st>>>(g, a, R, err);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace ivm
