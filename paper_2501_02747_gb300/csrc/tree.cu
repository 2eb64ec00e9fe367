// tree.cu -- image-tree expansion from the matrix and the table (Sec. II
// intro: the image tree is the costly step of the image method; Sec. III-B,
// Table II: order-k rows are transmitter -> reference face -> ... -> aim face).
//
// Path sets are summarised per (snapshot t, order k) by their count and two
// fingerprints sum_paths prod_m h_c(m, f_m) mod 2^64.  All three are chains of
// vector-matrix products over the ring Z / 2^64:
//   x_1[f] = w(1, f) vis_Tx[t][f],
//   x_k[g] = w(k, g) sum_{f : M[g][f]} x_{k-1}[f]       (M is symmetric),
//   summary[t][k] = sum_g x_k[g] vis_Rx[t][g],
// with w = 1 for counts and w = h_c for fingerprint c.  Ring arithmetic makes
// the order of summation irrelevant, so every result is exact.  M is sparse in
// city scenes, so a hop walks each row's adjacency list (CSR built from the
// bit rows) instead of a dense product.
//
// Snapshots are processed in chunks; vectors are stored [c][f][t] so the 32
// lanes of a warp (32 snapshots) read 256 contiguous bytes per facet.
//
// Optional enumeration: one item per (t, k, f1) in lexicographic order; a
// counting pass, an exclusive scan and a writing pass give records in order
// (t, k, f1, ..., fk) since adjacency lists are ascending.
#include "ivm_internal.cuh"
#include "tree.cuh"

namespace ivm {

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x)
{
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__constant__ unsigned long long c_fp_seed[2] = {0x243F6A8885A308D3ull, 0x13198A2E03707344ull};

// ---------------------------------------------------------------- adjacency

__global__ void k_degree(const uint32_t *M, int n, int W, long long *deg)
{
    int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (g >= n) return;
    long long d = 0;
    for (int w = lane; w < W; w += 32) d += __popc(M[(size_t)g * W + w]);
    for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (lane == 0) deg[g] = d;
}

// Exclusive scan of n values by one block of 1024 threads (n up to ~1e6).
__global__ void k_scan_single(const long long *in, long long n, long long *out)
{
    __shared__ long long part[1024];
    const long long per = (n + 1023) / 1024;
    const long long b = threadIdx.x * per, e = min(b + per, n);
    long long s = 0;
    for (long long i = b; i < e; i++) s += in[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        long long v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    long long run = part[threadIdx.x] - s;
    for (long long i = b; i < e; i++) {
        long long v = in[i];
        out[i] = run;
        run += v;
    }
    if (threadIdx.x == 1023) out[n] = part[1023];
}

__global__ void k_fill(const uint32_t *M, int n, int W, const long long *rowptr, int *col)
{
    int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (g >= n) return;
    long long base = rowptr[g];
    for (int w0 = 0; w0 < W; w0 += 32) {
        int w = w0 + lane;
        uint32_t word = w < W ? M[(size_t)g * W + w] : 0u;
        int c = __popc(word), incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        long long pos = base + incl - c;
        while (word) {
            int b = __ffs(word) - 1;
            word &= word - 1;
            col[pos++] = 32 * w + b;
        }
        base += __shfl_sync(0xffffffffu, incl, 31);
    }
}

__global__ void k_weights(int n, int K, unsigned long long *wt)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long per = (long long)(K + 1) * n;
    if (i >= 2 * per) return;
    int c = (int)(i / per);
    long long r = i - c * per;
    int m = (int)(r / n), f = (int)(r - (long long)m * n);
    wt[i] = splitmix64(c_fp_seed[c] ^ ((unsigned long long)(unsigned)m << 32) ^
                       (unsigned long long)(unsigned)f) | 1ull;
}

// ---------------------------------------------------------------- chains

__device__ __forceinline__ bool row_bit(const uint32_t *table, int W, long long t, int side, int f)
{
    return (table[((size_t)t * 2 + side) * W + (f >> 5)] >> (f & 31)) & 1u;
}

// The Tx-side chain x_1 .. x_K depends on the snapshot only through its Tx
// row, so it is computed once per run of consecutive equal Tx rows (a
// static Tx is one run); each snapshot then only takes the dot products
// with its own Rx row.

// flag[t] = 1 when Tx row t differs from Tx row t-1 (warp per snapshot)
__global__ void k_tx_run_flags(TreeArgs a, long long *flag)
{
    const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= a.S) return;
    bool diff = t == 0;
    if (t > 0) {
        const uint32_t *r0 = a.table + (size_t)t * 2 * a.W;
        const uint32_t *r1 = a.table + (size_t)(t - 1) * 2 * a.W;
        for (int w = lane; w < a.W && !diff; w += 32) diff = r0[w] != r1[w];
    }
    diff = __any_sync(0xffffffffu, diff);
    if (lane == 0) flag[t] = diff ? 1 : 0;
}

// run_of[t] from the exclusive scan of the flags; start[u] = first t of run u
__global__ void k_tx_runs(TreeArgs a, const long long *flag, const long long *excl,
                          int *run_of, long long *start)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.S) return;
    const long long u = excl[t] + flag[t] - 1;
    run_of[t] = (int)u;
    if (flag[t]) start[u] = t;
}

// x_1[c][f][ul] for the runs u0 .. u0 + C - 1
__global__ void k_init_runs(TreeArgs a, const long long *start, long long u0, int C,
                            unsigned long long *x)
{
    int ul = blockIdx.x * blockDim.x + threadIdx.x;
    int f = blockIdx.y;
    if (ul >= C) return;
    bool v = row_bit(a.table, a.W, start[u0 + ul], 0, f);
    size_t plane = (size_t)a.n * C;
    size_t o = (size_t)f * C + ul;
    x[o] = v ? 1ull : 0ull;
    x[plane + o] = v ? a.wt[(size_t)1 * a.n + f] : 0ull;
    x[2 * plane + o] = v ? a.wt[(size_t)(a.K + 1) * a.n + (size_t)1 * a.n + f] : 0ull;
}

// For snapshots [t0, t1) (all in runs u0 .. u0 + C - 1): summary[t][k] =
// sum_g x_k[c][g][run(t) - u0] vis_Rx[t][g] for k = 1..K, and order 0.
// xs holds x_1 .. x_K, 3 n C words each.
// Warp per snapshot: lanes take the Rx row's words, sum x over its set bits,
// and the warp adds the lanes' sums (exact: arithmetic mod 2^64).
__global__ void k_dot_runs(TreeArgs a, const int *run_of, long long t0, long long t1,
                           long long u0, int C, const unsigned long long *xs)
{
    const int lane = threadIdx.x & 31;
    const long long t = t0 + (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (t >= t1) return;   // uniform per warp
    const int ul = (int)(run_of[t] - u0);
    const size_t plane = (size_t)a.n * C;
    const uint32_t *rx = a.table + ((size_t)t * 2 + 1) * a.W;
    ivm_tree_summary *out = a.summary + (size_t)t * (a.K + 1);
    if (lane == 0) {
        const unsigned long long l = a.los[t] ? 1ull : 0ull;
        out[0].count = l;
        out[0].fp0 = l;
        out[0].fp1 = l;
    }
    for (int k = 1; k <= a.K; k++) {
        const unsigned long long *x = xs + (size_t)(k - 1) * 3 * plane;
        unsigned long long s0 = 0, s1 = 0, s2 = 0;
        for (int w = lane; w < a.W; w += 32) {
            uint32_t word = rx[w];
            while (word) {
                const int b = __ffs(word) - 1;
                word &= word - 1;
                const size_t o = (size_t)(32 * w + b) * C + ul;
                s0 += x[o];
                s1 += x[plane + o];
                s2 += x[2 * plane + o];
            }
        }
        for (int o = 16; o; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) {
            out[k].count = s0;
            out[k].fp0 = s1;
            out[k].fp1 = s2;
        }
    }
}

// x_new[c][g][t] = w_c(k, g) * sum_{f in adj(g)} x_old[c][f][t].  Warp =
// (row g, Cp consecutive runs t), Cp a power of two <= 32: lane = (group q,
// run r), the 32 / Cp groups stride over the row's nonzeros and their sums
// are added over the warp (exact: mod 2^64).  With few runs (a static
// transmitter has one) the lanes still share the row's work.
__global__ void k_hop(TreeArgs a, int C, int Cp, int k, const unsigned long long *xo,
                      unsigned long long *xn)
{
    const int lane = threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int tiles = (C + Cp - 1) / Cp;
    const long long g = wid / tiles;
    if (g >= a.n) return;   // uniform per warp
    const int G = 32 / Cp;
    const int r = lane & (Cp - 1), q = lane / Cp;
    const int tl = (int)(wid - g * tiles) * Cp + r;
    const bool ok = tl < C;
    const size_t plane = (size_t)a.n * C;
    unsigned long long s0 = 0, s1 = 0, s2 = 0;
    const long long e = a.rowptr[g + 1];
    for (long long p = a.rowptr[g] + q; p < e; p += G) {
        const int f = __ldg(a.col + p);
        if (ok) {
            const size_t o = (size_t)f * C + tl;
            s0 += xo[o];
            s1 += xo[plane + o];
            s2 += xo[2 * plane + o];
        }
    }
    for (int o = Cp; o < 32; o <<= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (ok && q == 0) {
        const size_t o = (size_t)g * C + tl;
        xn[o] = s0;
        xn[plane + o] = s1 * a.wt[(size_t)k * a.n + g];
        xn[2 * plane + o] = s2 * a.wt[(size_t)(a.K + 1) * a.n + (size_t)k * a.n + g];
    }
}

// ---------------------------------------------------------------- enumeration

// Item i of snapshot t: 0 is the direct path, 1 + (k-1) n + f1 is (k, f1).
__device__ __forceinline__ void item_of(const TreeArgs &a, long long it, long long &t, int &k,
                                        int &f1)
{
    const long long per = 1 + (long long)a.K * a.n;
    t = it / per;
    long long r = it - t * per;
    if (r == 0) { k = 0; f1 = -1; return; }
    r -= 1;
    k = 1 + (int)(r / a.n);
    f1 = (int)(r - (long long)(k - 1) * a.n);
}

// Depth-first walk of the paths of one item; writes records when out != null.
__device__ long long walk_paths(const TreeArgs &a, long long t, int k, int f1, int *out,
                                long long start, long long cap)
{
    if (k == 0) {
        if (!a.los[t]) return 0;
        if (out && start < cap) {
            int *r = out + (size_t)start * (a.K + 2);
            r[0] = (int)t; r[1] = 0;
            for (int m = 0; m < a.K; m++) r[2 + m] = -1;
        }
        return 1;
    }
    if (!row_bit(a.table, a.W, t, 0, f1)) return 0;
    int path[8];
    long long pos[8];
    path[0] = f1;
    long long count = 0;
    int depth = 0;   // path[0..depth] fixed
    pos[0] = a.rowptr[f1];
    for (;;) {
        if (depth == k - 1) {
            if (row_bit(a.table, a.W, t, 1, path[depth])) {
                if (out && start + count < cap) {
                    int *r = out + (size_t)(start + count) * (a.K + 2);
                    r[0] = (int)t; r[1] = k;
                    for (int m = 0; m < a.K; m++) r[2 + m] = m < k ? path[m] : -1;
                }
                count++;
            }
            depth--;
            if (depth < 0) break;
            continue;
        }
        if (pos[depth] < a.rowptr[path[depth] + 1]) {
            int nxt = a.col[pos[depth]++];
            path[depth + 1] = nxt;
            depth++;
            if (depth < k - 1) pos[depth] = a.rowptr[nxt];
        } else {
            depth--;
            if (depth < 0) break;
        }
    }
    return count;
}

__global__ void k_path_count(TreeArgs a, long long items, long long *cnt)
{
    long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= items) return;
    long long t; int k, f1;
    item_of(a, it, t, k, f1);
    cnt[it] = walk_paths(a, t, k, f1, nullptr, 0, 0);
}

__global__ void k_path_write(TreeArgs a, long long items, const long long *off, int *out,
                             long long cap)
{
    long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= items) return;
    long long t; int k, f1;
    item_of(a, it, t, k, f1);
    if (off[it] < cap && off[it + 1] > off[it]) walk_paths(a, t, k, f1, out, off[it], cap);
}

// Multi-block exclusive scan: per-block sums, a single-block scan of them,
// then a second pass that rescans each block from its offset.
__global__ void k_block_sums(const long long *in, long long n, long long *sums)
{
    __shared__ long long sh[256];
    long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    sh[threadIdx.x] = i < n ? in[i] : 0;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = sh[0];
}

__global__ void k_block_scan(const long long *in, long long n, const long long *boff,
                             long long *out)
{
    __shared__ long long sh[256];
    long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    long long v = i < n ? in[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
        long long u = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += u;
        __syncthreads();
    }
    long long excl = sh[threadIdx.x] - v + boff[blockIdx.x];
    if (i < n) out[i] = excl;
    if (i == n - 1) out[n] = excl + v;
}

// ---------------------------------------------------------------- launchers

cudaError_t tree_adjacency(TreeArgs &a, long long *deg, cudaStream_t st)
{
    int nb = (a.n * 32 + 255) / 256;
    k_degree<<<nb, 256, 0, st>>>(a.matrix, a.n, a.W, deg);
    k_scan_single<<<1, 1024, 0, st>>>(deg, a.n, a.rowptr);
    note_launches(2);
    return cudaGetLastError();
}

cudaError_t tree_fill(TreeArgs &a, cudaStream_t st)
{
    int nb = (a.n * 32 + 255) / 256;
    k_fill<<<nb, 256, 0, st>>>(a.matrix, a.n, a.W, a.rowptr, a.col);
    long long nw = 2LL * (a.K + 1) * a.n;
    k_weights<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(a.n, a.K, a.wt);
    note_launches(2);
    return cudaGetLastError();
}

cudaError_t tree_tx_runs(TreeArgs &a, long long *flag, long long *excl, long long *bsum,
                         long long *boff, int *run_of, long long *start, cudaStream_t st)
{
    k_tx_run_flags<<<(unsigned)((a.S * 32 + 255) / 256), 256, 0, st>>>(a, flag);
    cudaError_t e = tree_scan(flag, a.S, bsum, boff, excl, st);
    if (e != cudaSuccess) return e;
    k_tx_runs<<<(unsigned)((a.S + 255) / 256), 256, 0, st>>>(a, flag, excl, run_of, start);
    note_launches(2);
    return cudaGetLastError();
}

// Runs [u0, u0 + C) covering snapshots [t0, t1): chains x_1..x_K into xs
// (K blocks of 3 n C words), then the dots of every snapshot of those runs.
cudaError_t tree_run_chunk(TreeArgs &a, const long long *start, const int *run_of, long long u0,
                           int C, long long t0, long long t1, unsigned long long *xs,
                           cudaStream_t st)
{
    const size_t block = (size_t)3 * a.n * C;
    dim3 gi((C + 127) / 128, a.n);
    k_init_runs<<<gi, 128, 0, st>>>(a, start, u0, C, xs);
    int Cp = 1;
    while (Cp < C && Cp < 32) Cp <<= 1;
    const long long warps = (long long)a.n * ((C + Cp - 1) / Cp);
    for (int k = 2; k <= a.K; k++)
        k_hop<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(
            a, C, Cp, k, xs + (k - 2) * block, xs + (k - 1) * block);
    k_dot_runs<<<(unsigned)((t1 - t0 + 3) / 4), 128, 0, st>>>(a, run_of, t0, t1, u0, C, xs);
    note_launches(2 + (a.K - 1));
    return cudaGetLastError();
}

__global__ void k_order0(TreeArgs a)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.S) return;
    unsigned long long l = a.los[t] ? 1ull : 0ull;
    ivm_tree_summary *o = a.summary + (size_t)t * (a.K + 1);
    o[0].count = l; o[0].fp0 = l; o[0].fp1 = l;
}

cudaError_t tree_order0(TreeArgs &a, cudaStream_t st)
{
    k_order0<<<(unsigned)((a.S + 255) / 256), 256, 0, st>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t tree_paths_count(TreeArgs &a, long long items, long long *cnt, cudaStream_t st)
{
    k_path_count<<<(unsigned)((items + 127) / 128), 128, 0, st>>>(a, items, cnt);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t tree_scan(const long long *in, long long n, long long *sums, long long *sums_off,
                      long long *out, cudaStream_t st)
{
    long long nb = (n + 255) / 256;
    k_block_sums<<<(unsigned)nb, 256, 0, st>>>(in, n, sums);
    k_scan_single<<<1, 1024, 0, st>>>(sums, nb, sums_off);
    k_block_scan<<<(unsigned)nb, 256, 0, st>>>(in, n, sums_off, out);
    note_launches(3);
    return cudaGetLastError();
}

cudaError_t tree_paths_write(TreeArgs &a, long long items, const long long *off, int *out,
                             long long cap, cudaStream_t st)
{
    k_path_write<<<(unsigned)((items + 127) / 128), 128, 0, st>>>(a, items, off, out, cap);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace ivm
