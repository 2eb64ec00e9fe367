// ivm_api.cu -- the C ABI declared in include/ivm.h: context, scratch arena,
// host/device argument staging, and the launch sequences of the three calls.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <vector>

#include "ivm_internal.cuh"
#include "tree.cuh"

using namespace ivm;

static std::atomic<unsigned long long> g_launches{0};

void ivm::note_launches(int n) { g_launches.fetch_add((unsigned long long)n); }

namespace {

enum Slot {
    S_FACETS, S_DESC, S_LEAF, S_FSCENE, S_BOX, S_SX, S_SY, S_SZ, S_KEYS, S_SORTED, S_BOUNDS,
    S_ORDER, S_NODES, S_PARENT, S_VISITS, S_PAIRS, S_OUT, S_TX, S_RX, S_LOS, S_REP,
    S_T_MAT, S_T_TAB, S_T_LOS, S_T_SUM, S_T_DEG, S_T_ROW, S_T_COL, S_T_WT, S_T_XA, S_T_XB,
    S_T_CNT, S_T_OFF, S_T_BS, S_T_BO, S_T_PATHS,
    S_COUNT
};

struct Buf {
    void *p = nullptr;
    size_t cap = 0;
};

}  // namespace

struct ivm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int n_sm = 0;
    Buf buf[S_COUNT];
    int *d_err = nullptr;                 // device error word
    unsigned long long *d_ctr = nullptr;  // C_COUNT_ counters
    unsigned long long *d_misc = nullptr; // [0] count, [1] cursor, [2] work queue
    int *h_err = nullptr;
    unsigned long long *h_ctr = nullptr, *h_misc = nullptr;
    cudaEvent_t ev[8] = {};
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d)
    {
        cudaGetDevice(&prev);
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

#define CK(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            fprintf(stderr, "ivm: %s failed: %s (%s:%d)\n", #call, cudaGetErrorString(e_), \
                    __FILE__, __LINE__);                                                   \
            return IVM_ERR_CUDA;                                                           \
        }                                                                                  \
    } while (0)

int ensure(ivm_ctx *c, int slot, size_t bytes)
{
    Buf &b = c->buf[slot];
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) return IVM_OK;
    if (b.p) CK(cudaFree(b.p));
    b.p = nullptr;
    b.cap = 0;
    size_t want = bytes + bytes / 4 + 256;
    CK(cudaMalloc(&b.p, want));
    b.cap = want;
    return IVM_OK;
}

template <class T>
T *ptr(ivm_ctx *c, int slot)
{
    return static_cast<T *>(c->buf[slot].p);
}

bool is_device(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int words(int n) { return (n + 31) / 32; }

int check_params(const ivm_params *p)
{
    if (!p) return IVM_ERR_ARG;
    if (p->samples_per_side < 1 || p->samples_per_side > kMaxSamplesPerSide) return IVM_ERR_ARG;
    if (p->mode < IVM_MODE_EXACT || p->mode > IVM_MODE_LEARNED) return IVM_ERR_ARG;
    if (p->tile < 0 || p->warps_per_block < 0 || p->warps_per_block > 4) return IVM_ERR_ARG;
    return IVM_OK;
}

LaunchCfg launch_cfg(const ivm_ctx *c, const ivm_params *p)
{
    LaunchCfg L;
    L.mode = p->mode == IVM_MODE_EXACT ? IVM_MODE_EXACT : IVM_MODE_FILTERED;
    L.persistent = (p->flags & IVM_FLAG_PERSISTENT) != 0;
    L.warps_per_block = p->warps_per_block > 0 ? p->warps_per_block : 4;
    L.tile = p->tile > 0 ? p->tile : (L.persistent ? 4 : 1);
    L.n_sm = c->n_sm;
    L.cache = (p->flags & IVM_FLAG_OCCLUDER_CACHE) != 0;
    L.dedup = (p->flags & IVM_FLAG_DEDUP_SOURCES) != 0;
    return L;
}

// Copies the scenes' facets into the arena, lays out the per-scene
// descriptors, and points the geometry arrays into the arena.
int setup_geometry(ivm_ctx *c, const ivm_scene *scenes, int n_scenes, int s, DevScenes &g,
                   std::vector<SceneDesc> &hd)
{
    if (!scenes || n_scenes < 1) return IVM_ERR_ARG;
    hd.assign(n_scenes, SceneDesc());
    long long facets = 0, nodes = 0, samples = 0, rw = 0, maxn = 0;
    for (int k = 0; k < n_scenes; k++) {
        const ivm_scene &S = scenes[k];
        if (!S.facets || S.n_facets < 1) return IVM_ERR_ARG;
        SceneDesc &D = hd[k];
        D.facet0 = (int)facets;
        D.n = S.n_facets;
        D.W = words(S.n_facets);
        D.node0 = (int)nodes;
        D.root = S.n_facets >= 2 ? (int)nodes : ~(int)facets;
        D.s = s;
        D.sample0 = (int)samples;
        D.rw0 = rw;
        facets += S.n_facets;
        nodes += S.n_facets - 1;
        samples += (long long)S.n_facets * s * s;
        rw += (long long)S.n_facets * D.W;
        if (S.n_facets > maxn) maxn = S.n_facets;
    }
    if (facets >= (1LL << 30) || samples >= (1LL << 31)) return IVM_ERR_ARG;
    int r;
    if ((r = ensure(c, S_FACETS, sizeof(ivm_facet) * facets))) return r;
    if ((r = ensure(c, S_DESC, sizeof(SceneDesc) * n_scenes))) return r;
    if ((r = ensure(c, S_LEAF, sizeof(Leaf) * facets))) return r;
    if ((r = ensure(c, S_FSCENE, sizeof(int) * facets))) return r;
    if ((r = ensure(c, S_BOX, sizeof(int) * 6 * facets))) return r;
    if ((r = ensure(c, S_SX, sizeof(int) * samples))) return r;
    if ((r = ensure(c, S_SY, sizeof(int) * samples))) return r;
    if ((r = ensure(c, S_SZ, sizeof(int) * samples))) return r;
    if ((r = ensure(c, S_KEYS, sizeof(unsigned long long) * facets))) return r;
    if ((r = ensure(c, S_SORTED, sizeof(unsigned long long) * facets))) return r;
    if ((r = ensure(c, S_BOUNDS, sizeof(int) * 6 * n_scenes))) return r;
    if ((r = ensure(c, S_ORDER, sizeof(int) * facets))) return r;
    if ((r = ensure(c, S_NODES, sizeof(Node) * (nodes > 0 ? nodes : 1)))) return r;
    if ((r = ensure(c, S_PARENT, sizeof(int) * (facets + nodes)))) return r;
    if ((r = ensure(c, S_VISITS, sizeof(int) * (nodes > 0 ? nodes : 1)))) return r;
    ivm_facet *df = ptr<ivm_facet>(c, S_FACETS);
    for (int k = 0; k < n_scenes; k++)
        CK(cudaMemcpyAsync(df + hd[k].facet0, scenes[k].facets,
                           sizeof(ivm_facet) * scenes[k].n_facets, cudaMemcpyDefault, c->stream));
    g.n_scenes = n_scenes;
    g.total_facets = (int)facets;
    g.total_nodes = (int)nodes;
    g.total_samples = (int)samples;
    g.max_n = (int)maxn;
    g.desc = ptr<SceneDesc>(c, S_DESC);
    g.facets = df;
    g.leaf = ptr<Leaf>(c, S_LEAF);
    g.fscene = ptr<int>(c, S_FSCENE);
    g.box = ptr<int>(c, S_BOX);
    g.sx = ptr<int>(c, S_SX);
    g.sy = ptr<int>(c, S_SY);
    g.sz = ptr<int>(c, S_SZ);
    g.keys = ptr<unsigned long long>(c, S_KEYS);
    g.sorted = ptr<unsigned long long>(c, S_SORTED);
    g.bounds = ptr<int>(c, S_BOUNDS);
    g.order = ptr<int>(c, S_ORDER);
    g.nodes = ptr<Node>(c, S_NODES);
    g.parent = ptr<int>(c, S_PARENT);
    g.visits = ptr<int>(c, S_VISITS);
    return IVM_OK;
}

int read_error(ivm_ctx *c)
{
    CK(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return *c->h_err;
}

int reset_counters(ivm_ctx *c)
{
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    CK(cudaMemsetAsync(c->d_ctr, 0, sizeof(unsigned long long) * C_COUNT_, c->stream));
    return IVM_OK;
}

// Ingest + BVH for a call's scenes; leaves the geometry on the device.
int build_geometry(ivm_ctx *c, const DevScenes &g)
{
    CK(launch_ingest(g, c->d_err, c->stream));
    int e = read_error(c);
    if (e) return e;
    CK(cudaEventRecord(c->ev[1], c->stream));
    CK(launch_bvh(g, c->stream));
    CK(cudaEventRecord(c->ev[2], c->stream));
    return IVM_OK;
}

float elapsed(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        return 0.f;
    }
    return ms;
}

int fill_stats(ivm_ctx *c, ivm_stats *st, unsigned long long pairs, int phases)
{
    if (!st) return IVM_OK;
    CK(cudaMemcpy(c->h_ctr, c->d_ctr, sizeof(unsigned long long) * C_COUNT_,
                  cudaMemcpyDeviceToHost));
    memset(st, 0, sizeof(*st));
    st->pairs = pairs;
    st->cand_pairs = c->h_ctr[C_CAND_PAIRS];
    st->segments = c->h_ctr[C_SEGMENTS];
    st->node_tests = c->h_ctr[C_NODE_TESTS];
    st->leaf_tests = c->h_ctr[C_LEAF_TESTS];
    st->undecided = c->h_ctr[C_UNDECIDED];
    st->exact_tests = c->h_ctr[C_EXACT_TESTS];
    st->ranker_hits = c->h_ctr[C_RANKER_HITS];
    st->cache_hits = c->h_ctr[C_CACHE_HITS];
    st->dedup_rows = c->h_ctr[C_DEDUP_ROWS];
    st->ms_ingest = elapsed(c->ev[0], c->ev[1]);
    st->ms_bvh = elapsed(c->ev[1], c->ev[2]);
    if (phases >= 3) st->ms_screen = elapsed(c->ev[2], c->ev[3]);
    st->ms_traverse = elapsed(c->ev[phases >= 3 ? 3 : 2], c->ev[4]);
    st->ms_total = elapsed(c->ev[0], c->ev[4]);
    return IVM_OK;
}

}  // namespace

// ============================================================================ ABI

extern "C" const char *ivm_strerror(int code)
{
    switch (code) {
    case IVM_OK: return "ok";
    case IVM_ERR_ARG: return "invalid argument";
    case IVM_ERR_RANGE: return "geometry outside the supported coordinate range";
    case IVM_ERR_CAPACITY: return "path buffer too small";
    case IVM_ERR_TIMEOUT: return "device iteration budget exhausted";
    case IVM_ERR_CUDA: return "CUDA runtime error";
    case IVM_ERR_INTERNAL: return "internal invariant violated";
    default: return "unknown error";
    }
}

extern "C" uint64_t ivm_kernel_launches(void) { return g_launches.load(); }

extern "C" int ivm_create(ivm_ctx **out, int device, void *cuda_stream)
{
    if (!out) return IVM_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return device < 0 ? IVM_ERR_ARG : IVM_ERR_CUDA;
    }
    DeviceGuard dg(device);
    ivm_ctx *c = new ivm_ctx();
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    CK(cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device));
    CK(cudaMalloc(&c->d_err, sizeof(int)));
    CK(cudaMalloc(&c->d_ctr, sizeof(unsigned long long) * C_COUNT_));
    CK(cudaMalloc(&c->d_misc, sizeof(unsigned long long) * 4));
    CK(cudaMallocHost(&c->h_err, sizeof(int)));
    CK(cudaMallocHost(&c->h_ctr, sizeof(unsigned long long) * C_COUNT_));
    CK(cudaMallocHost(&c->h_misc, sizeof(unsigned long long) * 4));
    for (auto &e : c->ev) CK(cudaEventCreate(&e));
    *out = c;
    return IVM_OK;
}

extern "C" int ivm_destroy(ivm_ctx *c)
{
    if (!c) return IVM_OK;
    DeviceGuard dg(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto &b : c->buf)
        if (b.p) cudaFree(b.p);
    cudaFree(c->d_err);
    cudaFree(c->d_ctr);
    cudaFree(c->d_misc);
    cudaFreeHost(c->h_err);
    cudaFreeHost(c->h_ctr);
    cudaFreeHost(c->h_misc);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    delete c;
    return IVM_OK;
}

extern "C" int ivm_build_matrix(ivm_ctx *c, const ivm_scene *scenes, int32_t n_scenes,
                                const ivm_params *params, uint32_t *const *matrix,
                                ivm_stats *stats)
{
    if (!c || !matrix) return IVM_ERR_ARG;
    int r = check_params(params);
    if (r) return r;
    DeviceGuard dg(c->device);
    DevScenes g;
    std::vector<SceneDesc> hd;
    if ((r = setup_geometry(c, scenes, n_scenes, params->samples_per_side, g, hd))) return r;
    // outputs: device pointers are written in place; host ones go via the arena
    std::vector<char> on_host(n_scenes);
    size_t host_words = 0;
    for (int k = 0; k < n_scenes; k++) {
        if (!matrix[k]) return IVM_ERR_ARG;
        on_host[k] = !is_device(matrix[k]);
        if (on_host[k]) host_words += (size_t)hd[k].n * hd[k].W;
    }
    if ((r = ensure(c, S_OUT, sizeof(uint32_t) * host_words))) return r;
    size_t off = 0;
    unsigned long long pairs_total = 0;
    for (int k = 0; k < n_scenes; k++) {
        size_t nw = (size_t)hd[k].n * hd[k].W;
        hd[k].matrix = on_host[k] ? ptr<uint32_t>(c, S_OUT) + off : matrix[k];
        if (on_host[k]) off += nw;
        pairs_total += (unsigned long long)hd[k].n * hd[k].n;
    }
    CK(cudaMemcpyAsync(g.desc, hd.data(), sizeof(SceneDesc) * n_scenes, cudaMemcpyHostToDevice,
                       c->stream));
    if ((r = reset_counters(c))) return r;
    CK(cudaEventRecord(c->ev[0], c->stream));
    if ((r = build_geometry(c, g))) return r;
    // facing screen -> candidate pair list
    CK(cudaMemsetAsync(c->d_misc, 0, sizeof(unsigned long long) * 2, c->stream));
    CK(launch_screen_count(g, hd.data(), c->d_misc, c->stream));
    CK(cudaMemcpyAsync(c->h_misc, c->d_misc, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const unsigned long long npairs = c->h_misc[0];
    if ((r = ensure(c, S_PAIRS, sizeof(int2) * npairs))) return r;
    CK(launch_screen_emit(g, hd.data(), ptr<int2>(c, S_PAIRS), c->d_misc + 1, npairs, c->stream));
    CK(cudaMemcpyAsync(c->d_ctr + C_CAND_PAIRS, c->d_misc, sizeof(unsigned long long),
                       cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaEventRecord(c->ev[3], c->stream));
    for (int k = 0; k < n_scenes; k++)
        CK(cudaMemsetAsync(hd[k].matrix, 0, sizeof(uint32_t) * hd[k].n * hd[k].W, c->stream));
    const LaunchCfg cfg = launch_cfg(c, params);
    CK(launch_matrix(g, ptr<int2>(c, S_PAIRS), npairs, cfg, c->d_misc + 2, c->d_ctr, c->d_err,
                     c->stream));
    CK(cudaEventRecord(c->ev[4], c->stream));
    if ((r = read_error(c))) return r;
    for (int k = 0; k < n_scenes; k++)
        if (on_host[k])
            CK(cudaMemcpyAsync(matrix[k], hd[k].matrix, sizeof(uint32_t) * hd[k].n * hd[k].W,
                               cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return fill_stats(c, stats, pairs_total, 3);
}

extern "C" int ivm_build_table(ivm_ctx *c, const ivm_scene *scenes, int32_t n_scenes,
                               const ivm_params *params, const int32_t *const *tx,
                               const int32_t *const *rx, const int64_t *n_snap,
                               uint32_t *const *table, uint8_t *const *los, ivm_stats *stats)
{
    if (!c || !tx || !rx || !n_snap || !table || !los) return IVM_ERR_ARG;
    int r = check_params(params);
    if (r) return r;
    DeviceGuard dg(c->device);
    DevScenes g;
    std::vector<SceneDesc> hd;
    if ((r = setup_geometry(c, scenes, n_scenes, params->samples_per_side, g, hd))) return r;
    long long snaps = 0, chunks = 0, items = 0;
    const int snap_tile = params->tile > 0 ? params->tile : 16;
    size_t host_tab = 0, host_los = 0, pos_tx = 0, pos_rx = 0;
    std::vector<char> tab_host(n_scenes), los_host(n_scenes), tx_host(n_scenes),
        rx_host(n_scenes);
    for (int k = 0; k < n_scenes; k++) {
        if (n_snap[k] < 0) return IVM_ERR_ARG;
        if (n_snap[k] > 0 && (!table[k] || !los[k] || !tx[k] || !rx[k])) return IVM_ERR_ARG;
        hd[k].snap0 = snaps;
        hd[k].nsnap = n_snap[k];
        hd[k].los0 = chunks;
        hd[k].item0 = items;
        hd[k].ntiles = (int)((n_snap[k] + snap_tile - 1) / snap_tile);
        snaps += n_snap[k];
        chunks += (n_snap[k] + 31) / 32;
        items += 2LL * hd[k].W * hd[k].ntiles;
        const size_t S = (size_t)n_snap[k];
        if (S == 0) continue;
        tab_host[k] = !is_device(table[k]);
        los_host[k] = !is_device(los[k]);
        tx_host[k] = !is_device(tx[k]);
        rx_host[k] = !is_device(rx[k]);
        if (tab_host[k]) host_tab += S * 2 * hd[k].W;
        if (los_host[k]) host_los += S;
        if (tx_host[k]) pos_tx += 3 * S;
        if (rx_host[k]) pos_rx += 3 * S;
    }
    if ((r = ensure(c, S_OUT, sizeof(uint32_t) * host_tab))) return r;
    if ((r = ensure(c, S_LOS, host_los))) return r;
    if ((r = ensure(c, S_TX, sizeof(int) * pos_tx))) return r;
    if ((r = ensure(c, S_RX, sizeof(int) * pos_rx))) return r;
    size_t o_tab = 0, o_los = 0, o_tx = 0, o_rx = 0;
    for (int k = 0; k < n_scenes; k++) {
        const size_t S = (size_t)n_snap[k];
        if (S == 0) continue;
        hd[k].table = tab_host[k] ? ptr<uint32_t>(c, S_OUT) + o_tab : table[k];
        if (tab_host[k]) o_tab += S * 2 * hd[k].W;
        hd[k].los = los_host[k] ? ptr<uint8_t>(c, S_LOS) + o_los : los[k];
        if (los_host[k]) o_los += S;
        if (tx_host[k]) {
            int *d = ptr<int>(c, S_TX) + o_tx;
            CK(cudaMemcpyAsync(d, tx[k], sizeof(int) * 3 * S, cudaMemcpyHostToDevice, c->stream));
            hd[k].tx = d;
            o_tx += 3 * S;
        } else {
            hd[k].tx = tx[k];
        }
        if (rx_host[k]) {
            int *d = ptr<int>(c, S_RX) + o_rx;
            CK(cudaMemcpyAsync(d, rx[k], sizeof(int) * 3 * S, cudaMemcpyHostToDevice, c->stream));
            hd[k].rx = d;
            o_rx += 3 * S;
        } else {
            hd[k].rx = rx[k];
        }
    }
    CK(cudaMemcpyAsync(g.desc, hd.data(), sizeof(SceneDesc) * n_scenes, cudaMemcpyHostToDevice,
                       c->stream));
    if ((r = reset_counters(c))) return r;
    CK(cudaEventRecord(c->ev[0], c->stream));
    if ((r = build_geometry(c, g))) return r;
    const LaunchCfg cfg = launch_cfg(c, params);
    if (cfg.dedup && (r = ensure(c, S_REP, sizeof(int) * 2 * (size_t)snaps))) return r;
    CK(launch_table(g, snaps, items, chunks, snap_tile, cfg, ptr<int>(c, S_REP), c->d_misc + 2,
                    c->d_ctr, c->d_err, c->stream));
    CK(cudaEventRecord(c->ev[4], c->stream));
    if ((r = read_error(c))) return r;
    for (int k = 0; k < n_scenes; k++) {
        const size_t S = (size_t)n_snap[k];
        if (S == 0) continue;
        if (tab_host[k])
            CK(cudaMemcpyAsync(table[k], hd[k].table, sizeof(uint32_t) * S * 2 * hd[k].W,
                               cudaMemcpyDeviceToHost, c->stream));
        if (los_host[k])
            CK(cudaMemcpyAsync(los[k], hd[k].los, S, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    unsigned long long pairs = 0;
    for (int k = 0; k < n_scenes; k++) pairs += 2ull * hd[k].n * (unsigned long long)n_snap[k];
    return fill_stats(c, stats, pairs, 2);
}

extern "C" int ivm_expand_image_tree(ivm_ctx *c, const uint32_t *matrix, const uint32_t *table,
                                     const uint8_t *los, int32_t n_facets, int64_t n_snap,
                                     int32_t max_order, ivm_tree_summary *summary,
                                     int32_t *paths, int64_t path_capacity,
                                     int64_t *n_paths_out)
{
    if (!c || n_facets < 1 || n_snap < 0 || max_order < 0 || max_order > 8) return IVM_ERR_ARG;
    if (n_snap > 0 && (!matrix || !table || !los || !summary)) return IVM_ERR_ARG;
    if (paths && path_capacity < 0) return IVM_ERR_ARG;
    if (n_paths_out) *n_paths_out = 0;
    if (n_snap == 0) return IVM_OK;
    DeviceGuard dg(c->device);
    int r;
    const int n = n_facets, W = words(n_facets), K = max_order;
    const long long S = n_snap;
    TreeArgs a;
    a.n = n; a.W = W; a.K = K; a.S = S;
    // stage inputs that live on the host
    if (is_device(matrix)) {
        a.matrix = matrix;
    } else {
        if ((r = ensure(c, S_T_MAT, sizeof(uint32_t) * (size_t)n * W))) return r;
        CK(cudaMemcpyAsync(c->buf[S_T_MAT].p, matrix, sizeof(uint32_t) * (size_t)n * W,
                           cudaMemcpyHostToDevice, c->stream));
        a.matrix = ptr<uint32_t>(c, S_T_MAT);
    }
    if (is_device(table)) {
        a.table = table;
    } else {
        if ((r = ensure(c, S_T_TAB, sizeof(uint32_t) * (size_t)S * 2 * W))) return r;
        CK(cudaMemcpyAsync(c->buf[S_T_TAB].p, table, sizeof(uint32_t) * (size_t)S * 2 * W,
                           cudaMemcpyHostToDevice, c->stream));
        a.table = ptr<uint32_t>(c, S_T_TAB);
    }
    if (is_device(los)) {
        a.los = los;
    } else {
        if ((r = ensure(c, S_T_LOS, (size_t)S))) return r;
        CK(cudaMemcpyAsync(c->buf[S_T_LOS].p, los, (size_t)S, cudaMemcpyHostToDevice, c->stream));
        a.los = ptr<uint8_t>(c, S_T_LOS);
    }
    const bool sum_host = !is_device(summary);
    if (sum_host) {
        if ((r = ensure(c, S_T_SUM, sizeof(ivm_tree_summary) * (size_t)S * (K + 1)))) return r;
        a.summary = ptr<ivm_tree_summary>(c, S_T_SUM);
    } else {
        a.summary = summary;
    }
    CK(cudaEventRecord(c->ev[0], c->stream));
    // adjacency lists of the matrix rows
    if ((r = ensure(c, S_T_DEG, sizeof(long long) * (size_t)n))) return r;
    if ((r = ensure(c, S_T_ROW, sizeof(long long) * ((size_t)n + 1)))) return r;
    a.rowptr = ptr<long long>(c, S_T_ROW);
    CK(tree_adjacency(a, ptr<long long>(c, S_T_DEG), c->stream));
    long long nnz = 0;
    CK(cudaMemcpyAsync(&nnz, a.rowptr + n, sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if ((r = ensure(c, S_T_COL, sizeof(int) * (size_t)nnz))) return r;
    if ((r = ensure(c, S_T_WT, sizeof(unsigned long long) * 2 * (size_t)(K + 1) * n))) return r;
    a.col = ptr<int>(c, S_T_COL);
    a.wt = ptr<unsigned long long>(c, S_T_WT);
    CK(tree_fill(a, c->stream));
    // snapshot chunks: three vectors of n x C u64, twice, within ~768 MB
    long long C = (768LL << 20) / (48LL * n);
    C = C / 32 * 32;
    if (C < 32) C = 32;
    if (C > 8192) C = 8192;
    if (C > S) C = (S + 31) / 32 * 32;
    if (K >= 1) {
        const size_t xbytes = sizeof(unsigned long long) * 3 * (size_t)n * C;
        if ((r = ensure(c, S_T_XA, xbytes))) return r;
        if ((r = ensure(c, S_T_XB, K >= 2 ? xbytes : 16))) return r;
        for (long long t0 = 0; t0 < S; t0 += C) {
            int Cc = (int)(S - t0 < C ? S - t0 : C);
            CK(tree_chunk(a, t0, Cc, ptr<unsigned long long>(c, S_T_XA),
                          ptr<unsigned long long>(c, S_T_XB), c->stream));
        }
    } else {
        CK(tree_order0(a, c->stream));
    }
    int status = IVM_OK;
    if (paths || n_paths_out) {
        const long long items = S * (1 + (long long)K * n);
        if (paths) {
            if ((r = ensure(c, S_T_CNT, sizeof(long long) * (size_t)items))) return r;
            if ((r = ensure(c, S_T_OFF, sizeof(long long) * ((size_t)items + 1)))) return r;
            const long long nb = (items + 255) / 256;
            if ((r = ensure(c, S_T_BS, sizeof(long long) * (size_t)nb))) return r;
            if ((r = ensure(c, S_T_BO, sizeof(long long) * ((size_t)nb + 1)))) return r;
            CK(tree_paths_count(a, items, ptr<long long>(c, S_T_CNT), c->stream));
            CK(tree_scan(ptr<long long>(c, S_T_CNT), items, ptr<long long>(c, S_T_BS),
                         ptr<long long>(c, S_T_BO), ptr<long long>(c, S_T_OFF), c->stream));
            long long total = 0;
            CK(cudaMemcpyAsync(&total, ptr<long long>(c, S_T_OFF) + items, sizeof(long long),
                               cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            const bool paths_host = path_capacity > 0 && !is_device(paths);
            int *dst = paths;
            const long long wrote = total < path_capacity ? total : path_capacity;
            if (paths_host) {
                if ((r = ensure(c, S_T_PATHS, sizeof(int) * (size_t)wrote * (K + 2)))) return r;
                dst = ptr<int>(c, S_T_PATHS);
            }
            if (wrote > 0)
                CK(tree_paths_write(a, items, ptr<long long>(c, S_T_OFF), dst, path_capacity,
                                    c->stream));
            if (paths_host && wrote > 0)
                CK(cudaMemcpyAsync(paths, dst, sizeof(int) * (size_t)wrote * (K + 2),
                                   cudaMemcpyDeviceToHost, c->stream));
            if (n_paths_out) *n_paths_out = total;
            if (total > path_capacity) status = IVM_ERR_CAPACITY;
        }
    }
    if (sum_host)
        CK(cudaMemcpyAsync(summary, a.summary, sizeof(ivm_tree_summary) * (size_t)S * (K + 1),
                           cudaMemcpyDeviceToHost, c->stream));
    CK(cudaEventRecord(c->ev[4], c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (n_paths_out && !paths) {
        // total path count from the summaries: sum over t and k of count
        std::vector<ivm_tree_summary> hs;
        const ivm_tree_summary *src = summary;
        if (!sum_host) {
            hs.resize((size_t)S * (K + 1));
            CK(cudaMemcpy(hs.data(), summary, sizeof(ivm_tree_summary) * hs.size(),
                          cudaMemcpyDeviceToHost));
            src = hs.data();
        }
        long long tot = 0;
        for (size_t i = 0; i < (size_t)S * (K + 1); i++) tot += (long long)src[i].count;
        *n_paths_out = tot;
    }
    return status;
}
