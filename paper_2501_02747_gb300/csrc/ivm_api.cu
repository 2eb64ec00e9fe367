// ivm_api.cu -- the C ABI declared in include/ivm.h: context, scratch arena,
// host/device argument staging, and the launch sequences of the three calls.
//
// Each build call runs in four stages: plan (lay out the scenes and grow the
// arena -- the only place that allocates), enqueue (copies, memsets and
// kernels on the context's stream), execute (directly, or by replaying a
// CUDA graph captured from the enqueue stage), finalize (one
// synchronisation, the device error word, copies back to host buffers,
// stats).  The persistent form enqueues without any host synchronisation:
// the matrix kernel reads the candidate-pair count from device memory and
// the ingest range check is reported at the end.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <vector>

#include "ivm_internal.cuh"
#include "ranker.cuh"
#include "edges.cuh"
#include "relations.cuh"
#include "ranges.cuh"
#include "rays.cuh"
#include "tree.cuh"

using namespace ivm;

static std::atomic<unsigned long long> g_launches{0};

void ivm::note_launches(int n) { g_launches.fetch_add((unsigned long long)n); }

namespace {

enum Slot {
    S_FACETS, S_DESC, S_LEAF, S_FSCENE, S_BOX, S_SX, S_SY, S_SZ, S_KEYS, S_SORTED, S_BOUNDS,
    S_ORDER, S_NODES, S_PARENT, S_VISITS, S_PAIRS, S_OUT, S_TX, S_RX, S_LOS, S_REP,
    S_T_MAT, S_T_TAB, S_T_LOS, S_T_SUM, S_T_DEG, S_T_ROW, S_T_COL, S_T_WT, S_T_XA, S_T_XB,
    S_T_CNT, S_T_OFF, S_T_BS, S_T_BO, S_T_PATHS, S_T_FLAG, S_T_EXCL, S_T_RUN, S_T_START,
    S_TUNE_M, S_TUNE_T, S_TUNE_L,
    S_REL_M, S_REL_DEG, S_REL_OFF, S_REL_BS, S_REL_BO, S_REL_PAIRS, S_REL_REL, S_REL_RNG,
    S_PEAK,
    S_EM_EDGES, S_EM_FACES, S_EM_FE, S_EM_EE, S_EM_WORK,
    S_EDGES, S_EDGE_TAB, S_EDGE_KEY, S_EDGE_NEAR,
    S_RAY_PATHS, S_RAY_VALID,
    S_RNG_CNT, S_RNG_OFF, S_RNG_BS, S_RNG_BO, S_RNG_SUM, S_RNG_REC, S_RNG_TAB,
    S_CBOX, S_NCL, S_RANKS, S_RFEAT, S_RLAB, S_RIDX, S_RXB, S_RYB, S_RACT, S_RLOSS, S_RWT, S_RGT,
    S_COUNT
};

struct Buf {
    void *p = nullptr;
    size_t cap = 0;
};

// A captured launch sequence, replayed while the call's shape and buffers
// are unchanged.
struct GraphEntry {
    std::vector<unsigned long long> key;
    cudaGraphExec_t exec = nullptr;
    SceneDesc *h_desc = nullptr;   // pinned copy the graph's first node reads
    unsigned long long gen = 0;    // arena generation at capture
    unsigned long long last_use = 0;
    int kernels = 0;               // kernels per replay (launch accounting)
};

constexpr int kMaxGraphs = 8;
// Host-resident tables of one scene of at least 2 kOutChunkMin snapshots
// leave in at most kMaxOutChunks snapshot chunks (ivm_build_table).
constexpr int kMaxOutChunks = 8;
constexpr long long kOutChunkMin = 8192;
constexpr long long kDevCountMaxPairs = 1LL << 31;   // upper-bound pair list cap (16 GB)

}  // namespace

struct ivm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int n_sm = 0;
    Buf buf[S_COUNT];
    unsigned long long arena_gen = 1;     // bumps whenever a buffer moves
    int *d_err = nullptr;                 // device error word
    unsigned long long *d_ctr = nullptr;  // C_COUNT_ counters
    unsigned long long *d_misc = nullptr; // [0] pair count, [1] emit cursor (the count when the
                                          // list holds every pair), [2] work queue
    void *d_steal = nullptr;              // table: lazy-splitting slots, 64 x 16 B per SM
    int *h_err = nullptr;
    unsigned long long *h_ctr = nullptr, *h_misc = nullptr;
    cudaEvent_t ev[8] = {};
    std::vector<GraphEntry> graphs;
    unsigned long long uses = 0;
    cudaStream_t cap = nullptr;           // private stream used only for capture
    cudaStream_t out = nullptr;           // device-to-host copies of table chunks
    cudaEvent_t out_ev[kMaxOutChunks] = {};
    // learned ranking: FP32 master weights, Adam moments, BF16 inference copy
    float *r_master = nullptr, *r_m = nullptr, *r_v = nullptr, *r_grads = nullptr;
    __nv_bfloat16 *r_wt = nullptr;
    bool has_ranker = false;
    int walk_budget = 0;   // 0: automatic (see ivm_set_walk_budget)
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
    c->arena_gen++;
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
    if (p->table_tile < 0) return IVM_ERR_ARG;
    if (p->proof_tile < 0 || p->proof_tile > (1 << 16)) return IVM_ERR_ARG;
    return IVM_OK;
}

LaunchCfg launch_cfg(const ivm_ctx *c, const ivm_params *p)
{
    LaunchCfg L;
    L.mode = p->mode == IVM_MODE_EXACT ? IVM_MODE_EXACT : IVM_MODE_FILTERED;
    // graph replay needs the synchronisation-free (persistent) sequence
    L.persistent = (p->flags & (IVM_FLAG_PERSISTENT | IVM_FLAG_GRAPH)) != 0;
    L.warps_per_block = p->warps_per_block > 0 ? p->warps_per_block : 4;
    L.tile = p->tile > 0 ? p->tile : (L.persistent ? 4 : 1);
    L.n_sm = c->n_sm;
    L.cache = (p->flags & IVM_FLAG_OCCLUDER_CACHE) != 0;
    L.dedup = (p->flags & IVM_FLAG_DEDUP_SOURCES) != 0;
    L.aligned = (p->flags & IVM_FLAG_ALIGNED_FACETS) != 0;
    L.proof_tile = p->proof_tile > 0 ? p->proof_tile : 32;
    L.corner = (p->flags & IVM_FLAG_NO_CORNER_PROOF) == 0;
    return L;
}

// Lays out the per-scene descriptors and grows the geometry buffers.
int plan_geometry(ivm_ctx *c, const ivm_scene *scenes, int n_scenes, int s, DevScenes &g,
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
        D.row_lo = 0;
        D.row_hi = S.n_facets;
        D.budget = 4 * S.n_facets + 16;   // a walk visits at most 2n - 1 nodes and leaves
        if (c->walk_budget > 0 && c->walk_budget < D.budget) D.budget = c->walk_budget;
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
    g.n_scenes = n_scenes;
    g.total_facets = (int)facets;
    g.total_nodes = (int)nodes;
    g.total_samples = (int)samples;
    g.max_n = (int)maxn;
    return IVM_OK;
}

// Arena pointers (call after every ensure of the call is done).
void bind_geometry(ivm_ctx *c, DevScenes &g)
{
    g.desc = ptr<SceneDesc>(c, S_DESC);
    g.facets = ptr<ivm_facet>(c, S_FACETS);
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
}

// Phase events.  Inside a capture they are recorded as "external" event
// nodes, so that a replay records them too (a plain record inside a capture
// only orders the graph's nodes); the flag is refused outside a capture.
cudaError_t record(ivm_ctx *c, int i)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(c->stream, &cs);
    if (e != cudaSuccess) return e;
    if (cs == cudaStreamCaptureStatusActive)
        return cudaEventRecordWithFlags(c->ev[i], c->stream, cudaEventRecordExternal);
    return cudaEventRecord(c->ev[i], c->stream);
}

int read_error(ivm_ctx *c)
{
    CK(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return *c->h_err;
}

// Facet copies, descriptors, zeroed counters, ingest and BVH.  With
// `check` the ingest range check is read back before the BVH is built.
int enqueue_geometry(ivm_ctx *c, const DevScenes &g, const ivm_scene *scenes,
                     const std::vector<SceneDesc> &hd, const SceneDesc *desc_src, bool check)
{
    ivm_facet *df = ptr<ivm_facet>(c, S_FACETS);
    for (int k = 0; k < g.n_scenes; k++)
        CK(cudaMemcpyAsync(df + hd[k].facet0, scenes[k].facets,
                           sizeof(ivm_facet) * scenes[k].n_facets, cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(g.desc, desc_src, sizeof(SceneDesc) * g.n_scenes, cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    CK(cudaMemsetAsync(c->d_ctr, 0, sizeof(unsigned long long) * C_COUNT_, c->stream));
    CK(record(c, 0));
    CK(launch_ingest(g, c->d_err, c->stream));
    if (check) {
        int e = read_error(c);
        if (e) return e;
    }
    CK(record(c, 1));
    CK(launch_bvh(g, c->stream));
    CK(record(c, 2));
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
    st->ranker_hits8 = c->h_ctr[C_RANKER_HITS8];
    st->cache_hits = c->h_ctr[C_CACHE_HITS];
    st->dedup_rows = c->h_ctr[C_DEDUP_ROWS];
    st->ms_ingest = elapsed(c->ev[0], c->ev[1]);
    st->ms_bvh = elapsed(c->ev[1], c->ev[2]);
    if (phases >= 3) st->ms_screen = elapsed(c->ev[2], c->ev[3]);
    st->ms_traverse = elapsed(c->ev[phases >= 3 ? 3 : 2], c->ev[4]);
    st->ms_total = elapsed(c->ev[0], c->ev[4]);
    return IVM_OK;
}

// ------------------------------------------------------------------ graphs

void drop_graph(GraphEntry &e)
{
    if (e.exec) cudaGraphExecDestroy(e.exec);
    if (e.h_desc) cudaFreeHost(e.h_desc);
    e = GraphEntry();
}

GraphEntry *find_graph(ivm_ctx *c, const std::vector<unsigned long long> &key)
{
    for (auto &e : c->graphs)
        if (e.exec && e.gen == c->arena_gen && e.key == key) {
            e.last_use = ++c->uses;
            return &e;
        }
    return nullptr;
}

// Captures `enqueue` (a callable returning an IVM code) into a new entry.
template <class F>
int capture_graph(ivm_ctx *c, const std::vector<unsigned long long> &key, size_t desc_bytes,
                  const SceneDesc *desc, F &&enqueue, GraphEntry **out)
{
    // evict stale entries, then the least recently used one if full
    for (auto &e : c->graphs)
        if (e.exec && e.gen != c->arena_gen) drop_graph(e);
    GraphEntry *slot = nullptr;
    for (auto &e : c->graphs)
        if (!e.exec) { slot = &e; break; }
    if (!slot) {
        if ((int)c->graphs.size() < kMaxGraphs) {
            c->graphs.emplace_back();
            slot = &c->graphs.back();
        } else {
            slot = &c->graphs[0];
            for (auto &e : c->graphs)
                if (e.last_use < slot->last_use) slot = &e;
            drop_graph(*slot);
        }
    }
    CK(cudaMallocHost(&slot->h_desc, desc_bytes));
    memcpy(slot->h_desc, desc, desc_bytes);
    // The caller's stream may be the legacy default stream, which cannot be
    // captured: record on a private stream; the graph is launched on the
    // caller's stream afterwards.
    if (!c->cap) CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    const unsigned long long l0 = g_launches.load();
    cudaStream_t user = c->stream;
    c->stream = c->cap;
    cudaError_t eb = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    int r = eb == cudaSuccess ? enqueue(slot->h_desc) : IVM_ERR_CUDA;
    cudaGraph_t graph = nullptr;
    cudaError_t ec = eb == cudaSuccess ? cudaStreamEndCapture(c->stream, &graph) : eb;
    c->stream = user;
    if (r || ec != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        drop_graph(*slot);
        return r ? r : IVM_ERR_CUDA;
    }
    cudaError_t ei = cudaGraphInstantiate(&slot->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        drop_graph(*slot);
        return IVM_ERR_CUDA;
    }
    slot->kernels = (int)(g_launches.load() - l0);
    g_launches.fetch_sub((unsigned long long)slot->kernels);   // counted when replayed
    slot->key = key;
    slot->gen = c->arena_gen;
    slot->last_use = ++c->uses;
    *out = slot;
    return IVM_OK;
}

int replay(ivm_ctx *c, GraphEntry *e)
{
    CK(cudaGraphLaunch(e->exec, c->stream));
    note_launches(e->kernels);
    return IVM_OK;
}

void key_params(std::vector<unsigned long long> &k, const ivm_params *p)
{
    k.push_back((unsigned long long)p->samples_per_side);
    k.push_back((unsigned long long)p->mode);
    k.push_back((unsigned long long)p->tile);
    k.push_back((unsigned long long)p->warps_per_block);
    k.push_back((unsigned long long)p->flags);
    k.push_back((unsigned long long)p->table_tile);
    k.push_back((unsigned long long)p->proof_tile);
}

// Table of one scene whose table or LoS lives on the host, traversed in
// n_out snapshot chunks [cut[q], cut[q + 1]): the rows of chunk q are copied
// out on the context's second stream while chunk q + 1 is traversed.  Every
// copy has landed when this returns, whatever the outcome.
int table_in_chunks(ivm_ctx *c, DevScenes &g, const ivm_scene *scenes,
                    const std::vector<SceneDesc> &hd, const LaunchCfg &cfg, const int32_t *tx,
                    const int32_t *rx, bool tx_staged, bool rx_staged, uint32_t *table,
                    uint8_t *los, bool tab_host, bool los_host, int snap_tile,
                    const std::vector<long long> &cut, int n_out, ivm_stats *stats)
{
    const SceneDesc &F = hd[0];
    const long long S = F.nsnap;
    std::vector<SceneDesc> dq(1 + n_out, F);
    for (int q = 0; q < n_out; q++) {
        const long long a = cut[q];
        SceneDesc &D = dq[1 + q];
        D.snap0 = 0;
        D.los0 = 0;
        D.item0 = 0;
        D.nsnap = cut[q + 1] - a;
        D.ntiles = (int)((D.nsnap + snap_tile - 1) / snap_tile);
        D.tx = F.tx + 3 * a;
        D.rx = F.rx + 3 * a;
        D.table = F.table + (size_t)a * 2 * F.W;
        D.los = F.los + a;
    }
    if (!c->out) CK(cudaStreamCreateWithFlags(&c->out, cudaStreamNonBlocking));
    for (int q = 0; q < n_out; q++)
        if (!c->out_ev[q]) CK(cudaEventCreateWithFlags(&c->out_ev[q], cudaEventDisableTiming));
    bind_geometry(c, g);
    auto enqueue = [&]() -> int {
        const size_t bytes3 = sizeof(int) * 3 * (size_t)S;
        if (tx_staged)
            CK(cudaMemcpyAsync(ptr<int>(c, S_TX), tx, bytes3, cudaMemcpyHostToDevice, c->stream));
        if (rx_staged)
            CK(cudaMemcpyAsync(ptr<int>(c, S_RX), rx, bytes3, cudaMemcpyHostToDevice, c->stream));
        int e;
        if ((e = enqueue_geometry(c, g, scenes, hd, hd.data(), !cfg.persistent))) return e;
        CK(cudaMemcpyAsync(g.desc + 1, dq.data() + 1, sizeof(SceneDesc) * n_out,
                           cudaMemcpyHostToDevice, c->stream));
        for (int q = 0; q < n_out; q++) {
            const SceneDesc &D = dq[1 + q];
            const long long a = cut[q];
            DevScenes gq = g;
            gq.desc = g.desc + 1 + q;
            CK(launch_table(gq, D.nsnap, 2LL * D.W * D.ntiles, (D.nsnap + 31) / 32, snap_tile,
                            cfg, ptr<int>(c, S_REP), c->d_misc + 2, c->d_ctr, c->d_err,
                            c->stream));
            CK(cudaEventRecord(c->out_ev[q], c->stream));
            CK(cudaStreamWaitEvent(c->out, c->out_ev[q], 0));
            if (tab_host)
                CK(cudaMemcpyAsync(table + (size_t)a * 2 * F.W, D.table,
                                   sizeof(uint32_t) * 2 * F.W * (size_t)D.nsnap,
                                   cudaMemcpyDeviceToHost, c->out));
            if (los_host)
                CK(cudaMemcpyAsync(los + a, D.los, (size_t)D.nsnap, cudaMemcpyDeviceToHost,
                                   c->out));
        }
        CK(record(c, 4));
        return IVM_OK;
    };
    int r = enqueue();
    // the copies wait only for chunks that were enqueued, so this ends
    const cudaError_t e_out = cudaStreamSynchronize(c->out);
    if (r) {
        cudaStreamSynchronize(c->stream);
        return r;
    }
    if ((r = read_error(c))) return r;
    if (e_out != cudaSuccess) return IVM_ERR_CUDA;
    return fill_stats(c, stats, 2ull * F.n * (unsigned long long)S, 2);
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
    CK(cudaMalloc(&c->d_steal, 16 * 64 * (size_t)c->n_sm));
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
    for (auto &e : c->graphs) drop_graph(e);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->out) cudaStreamDestroy(c->out);
    for (auto &e : c->out_ev)
        if (e) cudaEventDestroy(e);
    for (void *p : {(void *)c->r_master, (void *)c->r_m, (void *)c->r_v, (void *)c->r_grads,
                    (void *)c->r_wt})
        if (p) cudaFree(p);
    for (auto &b : c->buf)
        if (b.p) cudaFree(b.p);
    cudaFree(c->d_err);
    cudaFree(c->d_ctr);
    cudaFree(c->d_misc);
    cudaFree(c->d_steal);
    cudaFreeHost(c->h_err);
    cudaFreeHost(c->h_ctr);
    cudaFreeHost(c->h_misc);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    delete c;
    return IVM_OK;
}

namespace {

int build_matrix(ivm_ctx *c, const ivm_scene *scenes, int32_t n_scenes, const ivm_params *params,
                 const int32_t *row_begin, const int32_t *row_end, uint32_t *const *matrix,
                 ivm_stats *stats)
{
    if (!c || !matrix || (!row_begin != !row_end)) return IVM_ERR_ARG;
    int r = check_params(params);
    if (r) return r;
    DeviceGuard dg(c->device);
    DevScenes g;
    std::vector<SceneDesc> hd;
    // ---- plan
    if ((r = plan_geometry(c, scenes, n_scenes, params->samples_per_side, g, hd))) return r;
    std::vector<char> on_host(n_scenes);
    bool all_device = true;
    size_t host_words = 0;
    long long upper = 0;
    unsigned long long pairs_total = 0;
    for (int k = 0; k < n_scenes; k++) {
        if (!matrix[k]) return IVM_ERR_ARG;
        const long long n = hd[k].n;
        if (row_begin) {
            if (row_begin[k] < 0 || row_begin[k] > row_end[k] || row_end[k] > n) return IVM_ERR_ARG;
            hd[k].row_lo = row_begin[k];
            hd[k].row_hi = row_end[k];
        }
        on_host[k] = !is_device(matrix[k]);
        all_device &= !on_host[k] && is_device(scenes[k].facets);
        if (on_host[k]) host_words += (size_t)hd[k].n * hd[k].W;
        // unordered pairs (i < j) with row_lo <= i < row_hi, and the ordered
        // pairs they decide (both bits, plus the diagonal of those rows)
        const long long lo = hd[k].row_lo, hi = hd[k].row_hi;
        const long long part = (hi - lo) * (n - 1) - (lo + hi - 1) * (hi - lo) / 2;
        upper += part;
        pairs_total += (unsigned long long)(2 * part + (hi - lo));
    }
    const LaunchCfg cfg0 = launch_cfg(c, params);
    const bool dev_count = cfg0.persistent && upper <= kDevCountMaxPairs;
    const bool use_graph = (params->flags & IVM_FLAG_GRAPH) && dev_count && all_device;
    const bool learned = params->mode == IVM_MODE_LEARNED && c->has_ranker;
    if (learned) {
        if ((r = ensure(c, S_CBOX, sizeof(int) * kRCtx * (size_t)n_scenes))) return r;
        if ((r = ensure(c, S_NCL, (size_t)g.total_nodes + 1))) return r;
        if (dev_count && (r = ensure(c, S_RANKS, sizeof(unsigned long long) * (size_t)upper)))
            return r;
    }
    if ((r = ensure(c, S_OUT, sizeof(uint32_t) * host_words))) return r;
    if (dev_count && (r = ensure(c, S_PAIRS, sizeof(int2) * (size_t)upper))) return r;
    size_t off = 0;
    for (int k = 0; k < n_scenes; k++) {
        hd[k].matrix = on_host[k] ? ptr<uint32_t>(c, S_OUT) + off : matrix[k];
        if (on_host[k]) off += (size_t)hd[k].n * hd[k].W;
    }
    // ---- enqueue
    auto enqueue = [&](const SceneDesc *desc_src) -> int {
        int e;
        bind_geometry(c, g);
        if ((e = enqueue_geometry(c, g, scenes, hd, desc_src, !dev_count))) return e;
        CK(cudaMemsetAsync(c->d_misc, 0, sizeof(unsigned long long) * 2, c->stream));
        unsigned long long npairs = (unsigned long long)upper;
        if (!dev_count) {   // size the pair list from a count pass
            CK(launch_screen_count(g, hd.data(), c->d_misc, c->stream));
            CK(cudaMemcpyAsync(c->h_misc, c->d_misc, sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            npairs = c->h_misc[0];
            if ((e = ensure(c, S_PAIRS, sizeof(int2) * npairs))) return e;
        }
        // with the list sized for every pair (dev_count), the emit pass's final
        // cursor is the count, and the traversal reads it from device memory
        CK(launch_screen_emit(g, hd.data(), ptr<int2>(c, S_PAIRS), c->d_misc + 1, npairs,
                              c->stream));
        CK(cudaMemcpyAsync(c->d_ctr + C_CAND_PAIRS, c->d_misc + 1, sizeof(unsigned long long),
                           cudaMemcpyDeviceToDevice, c->stream));
        CK(record(c, 3));
        for (int k = 0; k < n_scenes; k++)
            CK(cudaMemsetAsync(hd[k].matrix, 0, sizeof(uint32_t) * hd[k].n * hd[k].W, c->stream));
        LaunchCfg cfg = cfg0;
        cfg.count_dev = dev_count ? c->d_misc + 1 : nullptr;
        if (learned) {   // rank the clusters of every candidate pair
            if (!dev_count && (e = ensure(c, S_RANKS, sizeof(unsigned long long) * npairs)))
                return e;
            CK(ranker_clusters(g, ptr<int>(c, S_CBOX), ptr<signed char>(c, S_NCL), c->stream));
            CK(ranker_rank_pairs(g, ptr<int2>(c, S_PAIRS), npairs, cfg.count_dev,
                                 ptr<int>(c, S_CBOX), RankerDev{c->r_wt, c->r_master},
                                 ptr<unsigned long long>(c, S_RANKS), c->n_sm, c->d_err,
                                 c->stream));
            cfg.learn.ranks = ptr<unsigned long long>(c, S_RANKS);
            cfg.learn.ctx = ptr<int>(c, S_CBOX);
            cfg.learn.ncl = ptr<signed char>(c, S_NCL);
        }
        CK(launch_matrix(g, ptr<int2>(c, S_PAIRS), npairs, cfg, c->d_misc + 2, c->d_ctr,
                         c->d_err, c->stream));
        CK(record(c, 4));
        return IVM_OK;
    };
    // ---- execute
    if (use_graph) {
        std::vector<unsigned long long> key = {0ull, (unsigned long long)n_scenes,
                                               (unsigned long long)learned};
        key_params(key, params);
        key.push_back((unsigned long long)c->walk_budget);
        for (int k = 0; k < n_scenes; k++) {
            key.push_back((unsigned long long)(uintptr_t)scenes[k].facets);
            key.push_back((unsigned long long)scenes[k].n_facets);
            key.push_back((unsigned long long)(uintptr_t)matrix[k]);
            key.push_back(((unsigned long long)(unsigned)hd[k].row_lo << 32) |
                          (unsigned)hd[k].row_hi);
        }
        GraphEntry *ge = find_graph(c, key);
        if (!ge && (r = capture_graph(c, key, sizeof(SceneDesc) * n_scenes, hd.data(), enqueue,
                                      &ge)))
            return r;
        if ((r = replay(c, ge))) return r;
    } else {
        if ((r = enqueue(hd.data()))) return r;
    }
    // ---- finalize
    if ((r = read_error(c))) return r;
    for (int k = 0; k < n_scenes; k++)
        if (on_host[k])
            CK(cudaMemcpyAsync(matrix[k], hd[k].matrix, sizeof(uint32_t) * hd[k].n * hd[k].W,
                               cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return fill_stats(c, stats, pairs_total, 3);
}

}  // namespace

extern "C" int ivm_build_matrix(ivm_ctx *c, const ivm_scene *scenes, int32_t n_scenes,
                                const ivm_params *params, uint32_t *const *matrix,
                                ivm_stats *stats)
{
    return build_matrix(c, scenes, n_scenes, params, nullptr, nullptr, matrix, stats);
}

extern "C" int ivm_build_matrix_rows(ivm_ctx *c, const ivm_scene *scenes, int32_t n_scenes,
                                     const ivm_params *params, const int32_t *row_begin,
                                     const int32_t *row_end, uint32_t *const *matrix,
                                     ivm_stats *stats)
{
    if (!row_begin || !row_end) return IVM_ERR_ARG;
    return build_matrix(c, scenes, n_scenes, params, row_begin, row_end, matrix, stats);
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
    // ---- plan
    if ((r = plan_geometry(c, scenes, n_scenes, params->samples_per_side, g, hd))) return r;
    long long snaps = 0, chunks = 0, items = 0;
    const int snap_tile = params->table_tile > 0 ? params->table_tile : 32;
    size_t host_tab = 0, host_los = 0, pos_tx = 0, pos_rx = 0;
    std::vector<char> tab_host(n_scenes), los_host(n_scenes), tx_host(n_scenes),
        rx_host(n_scenes);
    bool all_device = true;
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
        all_device &= is_device(scenes[k].facets);
        const size_t S = (size_t)n_snap[k];
        if (S == 0) continue;
        tab_host[k] = !is_device(table[k]);
        los_host[k] = !is_device(los[k]);
        tx_host[k] = !is_device(tx[k]);
        rx_host[k] = !is_device(rx[k]);
        all_device &= !tab_host[k] && !los_host[k] && !tx_host[k] && !rx_host[k];
        if (tab_host[k]) host_tab += S * 2 * hd[k].W;
        if (los_host[k]) host_los += S;
        if (tx_host[k]) pos_tx += 3 * S;
        if (rx_host[k]) pos_rx += 3 * S;
    }
    LaunchCfg cfg = launch_cfg(c, params);
    // lazy splitting keeps snapshot indices in 32 bits and work items below 2^32
    bool splittable = !(params->flags & IVM_FLAG_NO_SPLIT) && items < (1LL << 32) - 2;
    for (int k = 0; k < n_scenes; k++) splittable &= n_snap[k] < (1LL << 31);
    if (cfg.persistent && splittable) cfg.steal = c->d_steal;
    const bool sync_free = cfg.persistent;
    const bool use_graph = (params->flags & IVM_FLAG_GRAPH) && all_device;
    // One scene whose table or LoS goes to the host: traverse it in snapshot
    // chunks and copy each chunk out on a second stream while the next one is
    // traversed.  Each chunk is half of what is left (rounded up to the
    // snapshot tile, itself rounded up to 32 snapshots) while both parts keep
    // at least kOutChunkMin / 2 snapshots: a chunk's copy then overlaps a
    // traversal about as long, and only the last, small copy and one tail
    // per chunk remain exposed.  The device holds one descriptor per chunk
    // after the scene's own.
    int n_out = 1;
    std::vector<long long> cut;
    if (n_scenes == 1 && (tab_host[0] || los_host[0]) && n_snap[0] >= 2 * kOutChunkMin) {
        const long long unit = (snap_tile + 31LL) / 32 * 32, S = n_snap[0];
        cut.push_back(0);
        while ((int)cut.size() < kMaxOutChunks && S - cut.back() >= kOutChunkMin) {
            const long long len = ((S - cut.back()) / 2 + unit - 1) / unit * unit;
            if (S - cut.back() - len < kOutChunkMin / 2) break;
            cut.push_back(cut.back() + len);
        }
        cut.push_back(S);
        n_out = (int)cut.size() - 1;
    }
    if (n_out > 1 && (r = ensure(c, S_DESC, sizeof(SceneDesc) * (1 + n_out)))) return r;
    if ((r = ensure(c, S_OUT, sizeof(uint32_t) * host_tab))) return r;
    if ((r = ensure(c, S_LOS, host_los))) return r;
    if ((r = ensure(c, S_TX, sizeof(int) * pos_tx))) return r;
    if ((r = ensure(c, S_RX, sizeof(int) * pos_rx))) return r;
    if (cfg.dedup && (r = ensure(c, S_REP, sizeof(int) * 2 * (size_t)snaps))) return r;
    size_t o_tab = 0, o_los = 0, o_tx = 0, o_rx = 0;
    std::vector<int> tx_off(n_scenes, -1), rx_off(n_scenes, -1);
    for (int k = 0; k < n_scenes; k++) {
        const size_t S = (size_t)n_snap[k];
        if (S == 0) continue;
        hd[k].table = tab_host[k] ? ptr<uint32_t>(c, S_OUT) + o_tab : table[k];
        if (tab_host[k]) o_tab += S * 2 * hd[k].W;
        hd[k].los = los_host[k] ? ptr<uint8_t>(c, S_LOS) + o_los : los[k];
        if (los_host[k]) o_los += S;
        if (tx_host[k]) {
            hd[k].tx = ptr<int>(c, S_TX) + o_tx;
            tx_off[k] = (int)o_tx;
            o_tx += 3 * S;
        } else {
            hd[k].tx = tx[k];
        }
        if (rx_host[k]) {
            hd[k].rx = ptr<int>(c, S_RX) + o_rx;
            rx_off[k] = (int)o_rx;
            o_rx += 3 * S;
        } else {
            hd[k].rx = rx[k];
        }
    }
    // ---- enqueue
    auto enqueue = [&](const SceneDesc *desc_src) -> int {
        int e;
        bind_geometry(c, g);
        for (int k = 0; k < n_scenes; k++) {
            const size_t S = (size_t)n_snap[k];
            if (tx_off[k] >= 0)
                CK(cudaMemcpyAsync(ptr<int>(c, S_TX) + tx_off[k], tx[k], sizeof(int) * 3 * S,
                                   cudaMemcpyHostToDevice, c->stream));
            if (rx_off[k] >= 0)
                CK(cudaMemcpyAsync(ptr<int>(c, S_RX) + rx_off[k], rx[k], sizeof(int) * 3 * S,
                                   cudaMemcpyHostToDevice, c->stream));
        }
        if ((e = enqueue_geometry(c, g, scenes, hd, desc_src, !sync_free))) return e;
        CK(launch_table(g, snaps, items, chunks, snap_tile, cfg, ptr<int>(c, S_REP),
                        c->d_misc + 2, c->d_ctr, c->d_err, c->stream));
        CK(record(c, 4));
        return IVM_OK;
    };
    // ---- execute
    if (use_graph) {
        std::vector<unsigned long long> key = {1ull, (unsigned long long)n_scenes};
        key_params(key, params);
        key.push_back((unsigned long long)c->walk_budget);
        for (int k = 0; k < n_scenes; k++) {
            key.push_back((unsigned long long)(uintptr_t)scenes[k].facets);
            key.push_back((unsigned long long)scenes[k].n_facets);
            key.push_back((unsigned long long)n_snap[k]);
            key.push_back((unsigned long long)(uintptr_t)tx[k]);
            key.push_back((unsigned long long)(uintptr_t)rx[k]);
            key.push_back((unsigned long long)(uintptr_t)table[k]);
            key.push_back((unsigned long long)(uintptr_t)los[k]);
        }
        GraphEntry *ge = find_graph(c, key);
        if (!ge && (r = capture_graph(c, key, sizeof(SceneDesc) * n_scenes, hd.data(), enqueue,
                                      &ge)))
            return r;
        if ((r = replay(c, ge))) return r;
    } else if (n_out > 1) {
        return table_in_chunks(c, g, scenes, hd, cfg, tx[0], rx[0], tx_off[0] >= 0,
                               rx_off[0] >= 0, table[0], los[0], tab_host[0], los_host[0],
                               snap_tile, cut, n_out, stats);
    } else {
        if ((r = enqueue(hd.data()))) return r;
    }
    // ---- finalize
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

extern "C" int ivm_interface_relations(ivm_ctx *c, const ivm_scene *scene,
                                       const ivm_params *params, const uint32_t *matrix,
                                       int32_t *pairs, uint8_t *relation, double *ranges,
                                       int64_t capacity, int64_t *n_pairs)
{
    if (!c || !scene || !matrix || !n_pairs || capacity < 0) return IVM_ERR_ARG;
    if (pairs && (!relation || !ranges)) return IVM_ERR_ARG;
    int r = check_params(params);
    if (r) return r;
    DeviceGuard dg(c->device);
    DevScenes g;
    std::vector<SceneDesc> hd;
    if ((r = plan_geometry(c, scene, 1, params->samples_per_side, g, hd))) return r;
    const int n = hd[0].n, W = hd[0].W;
    const bool m_host = !is_device(matrix);
    const long long nb = (n + 255) / 256;
    if ((r = ensure(c, S_REL_M, m_host ? sizeof(uint32_t) * (size_t)n * W : 0))) return r;
    if ((r = ensure(c, S_REL_DEG, sizeof(long long) * (size_t)(n + 1)))) return r;
    if ((r = ensure(c, S_REL_OFF, sizeof(long long) * (size_t)(n + 1)))) return r;
    if ((r = ensure(c, S_REL_BS, sizeof(long long) * (size_t)(nb + 1)))) return r;
    if ((r = ensure(c, S_REL_BO, sizeof(long long) * (size_t)(nb + 1)))) return r;
    bind_geometry(c, g);
    const uint32_t *M = m_host ? ptr<uint32_t>(c, S_REL_M) : matrix;
    if (m_host)
        CK(cudaMemcpyAsync(ptr<uint32_t>(c, S_REL_M), matrix, sizeof(uint32_t) * (size_t)n * W,
                           cudaMemcpyHostToDevice, c->stream));
    long long *off = ptr<long long>(c, S_REL_OFF);
    CK(relations_count(M, n, W, ptr<long long>(c, S_REL_DEG), c->stream));
    CK(tree_scan(ptr<long long>(c, S_REL_DEG), n, ptr<long long>(c, S_REL_BS),
                 ptr<long long>(c, S_REL_BO), off, c->stream));
    CK(cudaMemcpyAsync(&c->h_misc[0], off + n, sizeof(long long), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const long long P = (long long)c->h_misc[0];
    *n_pairs = P;
    if (!pairs || P == 0) return IVM_OK;
    if (P > capacity) return IVM_ERR_CAPACITY;
    const bool p_host = !is_device(pairs), r_host = !is_device(relation),
               g_host = !is_device(ranges);
    if ((r = ensure(c, S_REL_PAIRS, p_host ? sizeof(int) * 2 * (size_t)P : 0))) return r;
    if ((r = ensure(c, S_REL_REL, r_host ? (size_t)P : 0))) return r;
    if ((r = ensure(c, S_REL_RNG, g_host ? sizeof(double) * 8 * (size_t)P : 0))) return r;
    bind_geometry(c, g);
    RelArgs a;
    a.M = m_host ? ptr<uint32_t>(c, S_REL_M) : matrix;
    a.n = n;
    a.W = W;
    a.off = ptr<long long>(c, S_REL_OFF);
    a.pairs = p_host ? ptr<int>(c, S_REL_PAIRS) : pairs;
    a.relation = r_host ? ptr<uint8_t>(c, S_REL_REL) : relation;
    a.ranges = g_host ? ptr<double>(c, S_REL_RNG) : ranges;
    if ((r = enqueue_geometry(c, g, scene, hd, hd.data(), true))) return r;   // the leaves
    CK(relations_write(g, a, c->stream));
    if ((r = read_error(c))) return r;
    if (p_host)
        CK(cudaMemcpyAsync(pairs, a.pairs, sizeof(int) * 2 * (size_t)P, cudaMemcpyDeviceToHost,
                           c->stream));
    if (r_host)
        CK(cudaMemcpyAsync(relation, a.relation, (size_t)P, cudaMemcpyDeviceToHost, c->stream));
    if (g_host)
        CK(cudaMemcpyAsync(ranges, a.ranges, sizeof(double) * 8 * (size_t)P,
                           cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return IVM_OK;
}

extern "C" int ivm_build_edge_table(ivm_ctx *c, const ivm_scene *scene, const ivm_params *params,
                                    const int32_t *edges, int32_t n_edges, const int32_t *tx,
                                    const int32_t *rx, int64_t n_snap, uint32_t *table,
                                    int32_t *nearest)
{
    if (!c || !scene || n_edges < 0 || n_edges > 0xffff || n_snap < 0) return IVM_ERR_ARG;
    if (n_snap > 0 && (!tx || !rx || !table || !nearest)) return IVM_ERR_ARG;
    if (n_edges > 0 && !edges) return IVM_ERR_ARG;
    int r = check_params(params);
    if (r) return r;
    DeviceGuard dg(c->device);
    DevScenes g;
    std::vector<SceneDesc> hd;
    if ((r = plan_geometry(c, scene, 1, params->samples_per_side, g, hd))) return r;
    if (n_snap == 0) return IVM_OK;
    const int WE = words(n_edges);
    const size_t S = (size_t)n_snap;
    const bool e_host = n_edges > 0 && !is_device(edges);
    const bool tx_host = !is_device(tx), rx_host = !is_device(rx);
    const bool t_host = !is_device(table), n_host = !is_device(nearest);
    if ((r = ensure(c, S_EDGES, e_host ? sizeof(int) * 6 * (size_t)n_edges : 0))) return r;
    if ((r = ensure(c, S_EDGE_TAB, t_host ? sizeof(uint32_t) * S * 2 * WE : 0))) return r;
    if ((r = ensure(c, S_EDGE_KEY, sizeof(unsigned long long) * 2 * S))) return r;
    if ((r = ensure(c, S_EDGE_NEAR, n_host ? sizeof(int) * 2 * S : 0))) return r;
    if ((r = ensure(c, S_TX, tx_host ? sizeof(int) * 3 * S : 0))) return r;
    if ((r = ensure(c, S_RX, rx_host ? sizeof(int) * 3 * S : 0))) return r;
    bind_geometry(c, g);
    EdgeArgs a;
    a.edges = e_host ? ptr<int>(c, S_EDGES) : edges;
    a.ne = n_edges;
    a.WE = WE;
    a.tx = tx_host ? ptr<int>(c, S_TX) : tx;
    a.rx = rx_host ? ptr<int>(c, S_RX) : rx;
    a.S = n_snap;
    a.tile = params->table_tile > 0 ? params->table_tile : 32;
    a.ntiles = (n_snap + a.tile - 1) / a.tile;
    a.table = t_host ? ptr<uint32_t>(c, S_EDGE_TAB) : table;
    a.nearest_key = ptr<unsigned long long>(c, S_EDGE_KEY);
    a.nearest = n_host ? ptr<int>(c, S_EDGE_NEAR) : nearest;
    a.ctr = c->d_ctr;
    if (e_host)
        CK(cudaMemcpyAsync(ptr<int>(c, S_EDGES), edges, sizeof(int) * 6 * (size_t)n_edges,
                           cudaMemcpyHostToDevice, c->stream));
    if (tx_host)
        CK(cudaMemcpyAsync(ptr<int>(c, S_TX), tx, sizeof(int) * 3 * S, cudaMemcpyHostToDevice,
                           c->stream));
    if (rx_host)
        CK(cudaMemcpyAsync(ptr<int>(c, S_RX), rx, sizeof(int) * 3 * S, cudaMemcpyHostToDevice,
                           c->stream));
    if ((r = enqueue_geometry(c, g, scene, hd, hd.data(), true))) return r;
    if (WE > 0)
        CK(cudaMemsetAsync(a.table, 0, sizeof(uint32_t) * S * 2 * WE, c->stream));
    CK(edges_table(g, a, params->mode != IVM_MODE_EXACT, c->d_err, c->stream));
    if ((r = read_error(c))) return r;
    if (t_host && WE > 0)
        CK(cudaMemcpyAsync(table, a.table, sizeof(uint32_t) * S * 2 * WE, cudaMemcpyDeviceToHost,
                           c->stream));
    if (n_host)
        CK(cudaMemcpyAsync(nearest, a.nearest, sizeof(int) * 2 * S, cudaMemcpyDeviceToHost,
                           c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return IVM_OK;
}

extern "C" int ivm_fp32_peak(ivm_ctx *c, double *lane_ops_per_s)
{
    if (!c || !lane_ops_per_s) return IVM_ERR_ARG;
    DeviceGuard dg(c->device);
    int r;
    if ((r = ensure(c, S_PEAK, sizeof(float)))) return r;
    CK(ffma_peak(c->n_sm, ptr<float>(c, S_PEAK), c->stream, lane_ops_per_s));
    CK(cudaStreamSynchronize(c->stream));
    return IVM_OK;
}

extern "C" int ivm_build_edge_matrix(ivm_ctx *c, const ivm_scene *scene,
                                     const ivm_params *params, const int32_t *edges,
                                     const int32_t *edge_faces, int32_t n_edges, uint32_t *fe,
                                     uint32_t *ee)
{
    if (!c || !scene || n_edges < 0) return IVM_ERR_ARG;
    if (n_edges > 0 && (!edges || !edge_faces || !fe || !ee)) return IVM_ERR_ARG;
    int r = check_params(params);
    if (r) return r;
    DeviceGuard dg(c->device);
    DevScenes g;
    std::vector<SceneDesc> hd;
    if ((r = plan_geometry(c, scene, 1, params->samples_per_side, g, hd))) return r;
    if (n_edges == 0) return IVM_OK;
    const int n = hd[0].n, WE = words(n_edges);
    const size_t ne = (size_t)n_edges;
    const bool e_host = !is_device(edges), f_host = !is_device(edge_faces);
    const bool fe_host = !is_device(fe), ee_host = !is_device(ee);
    if ((r = ensure(c, S_EM_EDGES, e_host ? sizeof(int) * 6 * ne : 0))) return r;
    if ((r = ensure(c, S_EM_FACES, f_host ? sizeof(int) * 2 * ne : 0))) return r;
    if ((r = ensure(c, S_EM_FE, fe_host ? sizeof(uint32_t) * (size_t)n * WE : 0))) return r;
    if ((r = ensure(c, S_EM_EE, ee_host ? sizeof(uint32_t) * ne * WE : 0))) return r;
    if ((r = ensure(c, S_EM_WORK, sizeof(unsigned long long)))) return r;
    bind_geometry(c, g);
    EdgeMatrixArgs a;
    a.edges = e_host ? ptr<int>(c, S_EM_EDGES) : edges;
    a.faces = f_host ? ptr<int>(c, S_EM_FACES) : edge_faces;
    a.n = n;
    a.ne = n_edges;
    a.WE = WE;
    a.fe = fe_host ? ptr<uint32_t>(c, S_EM_FE) : fe;
    a.ee = ee_host ? ptr<uint32_t>(c, S_EM_EE) : ee;
    a.tile = 4;
    a.work = ptr<unsigned long long>(c, S_EM_WORK);
    a.ctr = c->d_ctr;
    if (e_host)
        CK(cudaMemcpyAsync(ptr<int>(c, S_EM_EDGES), edges, sizeof(int) * 6 * ne,
                           cudaMemcpyHostToDevice, c->stream));
    if (f_host)
        CK(cudaMemcpyAsync(ptr<int>(c, S_EM_FACES), edge_faces, sizeof(int) * 2 * ne,
                           cudaMemcpyHostToDevice, c->stream));
    if ((r = enqueue_geometry(c, g, scene, hd, hd.data(), true))) return r;
    CK(cudaMemsetAsync(a.fe, 0, sizeof(uint32_t) * (size_t)n * WE, c->stream));
    CK(cudaMemsetAsync(a.ee, 0, sizeof(uint32_t) * ne * WE, c->stream));
    CK(edges_matrix(g, a, params->mode != IVM_MODE_EXACT, c->n_sm, c->d_err, c->stream));
    if ((r = read_error(c))) return r;
    if (fe_host)
        CK(cudaMemcpyAsync(fe, a.fe, sizeof(uint32_t) * (size_t)n * WE, cudaMemcpyDeviceToHost,
                           c->stream));
    if (ee_host)
        CK(cudaMemcpyAsync(ee, a.ee, sizeof(uint32_t) * ne * WE, cudaMemcpyDeviceToHost,
                           c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return IVM_OK;
}

extern "C" int ivm_validate_paths(ivm_ctx *c, const ivm_scene *scene, const ivm_params *params,
                                  const int32_t *tx, const int32_t *rx, int64_t n_snap,
                                  const int32_t *paths, int64_t n_paths, int32_t max_order,
                                  uint8_t *valid)
{
    if (!c || !scene || n_snap < 0 || n_paths < 0 || max_order < 0 || max_order > kRayMaxOrder)
        return IVM_ERR_ARG;
    if (n_paths > 0 && (!paths || !valid || !tx || !rx)) return IVM_ERR_ARG;
    int r = check_params(params);
    if (r) return r;
    if (!scene->facets || scene->n_facets < 1) return IVM_ERR_ARG;
    DeviceGuard dg(c->device);
    // every facet an axis-aligned rectangle: u and v along two different axes
    {
        std::vector<ivm_facet> hf(scene->n_facets);
        CK(cudaMemcpy(hf.data(), scene->facets, sizeof(ivm_facet) * hf.size(), cudaMemcpyDefault));
        for (const ivm_facet &f : hf) {
            int nu = 0, nv = 0, au = -1, av = -1;
            for (int i = 0; i < 3; i++) {
                if (f.u[i]) { nu++; au = i; }
                if (f.v[i]) { nv++; av = i; }
            }
            if (nu != 1 || nv != 1 || au == av) return IVM_ERR_ARG;
        }
    }
    DevScenes g;
    std::vector<SceneDesc> hd;
    if ((r = plan_geometry(c, scene, 1, params->samples_per_side, g, hd))) return r;
    if (n_paths == 0) return IVM_OK;
    const bool p_host = !is_device(paths), v_host = !is_device(valid);
    const bool tx_host = !is_device(tx), rx_host = !is_device(rx);
    const size_t rec = (size_t)max_order + 2;
    if ((r = ensure(c, S_RAY_PATHS, p_host ? sizeof(int) * rec * (size_t)n_paths : 0))) return r;
    if ((r = ensure(c, S_RAY_VALID, v_host ? (size_t)n_paths : 0))) return r;
    if ((r = ensure(c, S_TX, tx_host ? sizeof(int) * 3 * (size_t)n_snap : 0))) return r;
    if ((r = ensure(c, S_RX, rx_host ? sizeof(int) * 3 * (size_t)n_snap : 0))) return r;
    bind_geometry(c, g);
    RayArgs a;
    a.tx = tx_host ? ptr<int>(c, S_TX) : tx;
    a.rx = rx_host ? ptr<int>(c, S_RX) : rx;
    a.n_snap = n_snap;
    a.paths = p_host ? ptr<int>(c, S_RAY_PATHS) : paths;
    a.n_paths = n_paths;
    a.max_order = max_order;
    a.valid = v_host ? ptr<uint8_t>(c, S_RAY_VALID) : valid;
    if (tx_host)
        CK(cudaMemcpyAsync(ptr<int>(c, S_TX), tx, sizeof(int) * 3 * (size_t)n_snap,
                           cudaMemcpyHostToDevice, c->stream));
    if (rx_host)
        CK(cudaMemcpyAsync(ptr<int>(c, S_RX), rx, sizeof(int) * 3 * (size_t)n_snap,
                           cudaMemcpyHostToDevice, c->stream));
    if (p_host)
        CK(cudaMemcpyAsync(ptr<int>(c, S_RAY_PATHS), paths, sizeof(int) * rec * (size_t)n_paths,
                           cudaMemcpyHostToDevice, c->stream));
    if ((r = enqueue_geometry(c, g, scene, hd, hd.data(), true))) return r;
    CK(rays_validate(g, a, c->d_err, c->stream));
    if ((r = read_error(c))) return r;
    if (v_host)
        CK(cudaMemcpyAsync(valid, a.valid, (size_t)n_paths, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return IVM_OK;
}

extern "C" int ivm_set_walk_budget(ivm_ctx *c, int32_t steps)
{
    if (!c || steps < 0) return IVM_ERR_ARG;
    c->walk_budget = steps;
    return IVM_OK;
}

extern "C" int ivm_visibility_ranges(ivm_ctx *c, const ivm_scene *scene, const ivm_params *params,
                                     const int32_t *tx, const int32_t *rx, int64_t n_snap,
                                     const uint32_t *table, ivm_range *ranges, int64_t capacity,
                                     int64_t *n_ranges, ivm_range_summary *summary)
{
    if (!c || !scene || !n_ranges || n_snap < 0 || capacity < 0) return IVM_ERR_ARG;
    if (n_snap > 0 && (!tx || !rx || !table)) return IVM_ERR_ARG;
    int r = check_params(params);
    if (r) return r;
    DeviceGuard dg(c->device);
    DevScenes g;
    std::vector<SceneDesc> hd;
    if ((r = plan_geometry(c, scene, 1, params->samples_per_side, g, hd))) return r;
    const int n = hd[0].n, W = hd[0].W;
    const long long S = n_snap;
    const int nchunks = (int)((S + kRngChunk - 1) / kRngChunk);
    const long long items = 2LL * n * nchunks;
    const bool tab_host = S > 0 && !is_device(table);
    const bool tx_host = S > 0 && !is_device(tx), rx_host = S > 0 && !is_device(rx);
    const long long nb = (items + 255) / 256;
    if ((r = ensure(c, S_RNG_CNT, sizeof(long long) * (size_t)(items + 1)))) return r;
    if ((r = ensure(c, S_RNG_OFF, sizeof(long long) * (size_t)(items + 1)))) return r;
    if ((r = ensure(c, S_RNG_BS, sizeof(long long) * (size_t)(nb + 1)))) return r;
    if ((r = ensure(c, S_RNG_BO, sizeof(long long) * (size_t)(nb + 1)))) return r;
    if ((r = ensure(c, S_RNG_SUM, sizeof(unsigned long long) * 2))) return r;
    if ((r = ensure(c, S_RNG_TAB, tab_host ? sizeof(uint32_t) * (size_t)S * 2 * W : 0))) return r;
    if ((r = ensure(c, S_TX, tx_host ? sizeof(int) * 3 * (size_t)S : 0))) return r;
    if ((r = ensure(c, S_RX, rx_host ? sizeof(int) * 3 * (size_t)S : 0))) return r;
    bind_geometry(c, g);
    RangeArgs a;
    a.table = tab_host ? ptr<uint32_t>(c, S_RNG_TAB) : table;
    a.n = n;
    a.W = W;
    a.S = S;
    a.nchunks = nchunks;
    a.tx = tx_host ? ptr<int>(c, S_TX) : tx;
    a.rx = rx_host ? ptr<int>(c, S_RX) : rx;
    a.count = ptr<long long>(c, S_RNG_CNT);
    a.off = ptr<long long>(c, S_RNG_OFF);
    a.rec = nullptr;
    a.sums = ptr<unsigned long long>(c, S_RNG_SUM);
    if (tab_host)
        CK(cudaMemcpyAsync(ptr<uint32_t>(c, S_RNG_TAB), table, sizeof(uint32_t) * (size_t)S * 2 * W,
                           cudaMemcpyHostToDevice, c->stream));
    if (tx_host)
        CK(cudaMemcpyAsync(ptr<int>(c, S_TX), tx, sizeof(int) * 3 * (size_t)S,
                           cudaMemcpyHostToDevice, c->stream));
    if (rx_host)
        CK(cudaMemcpyAsync(ptr<int>(c, S_RX), rx, sizeof(int) * 3 * (size_t)S,
                           cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(a.sums, 0, sizeof(unsigned long long) * 2, c->stream));
    long long R = 0, side0 = 0;
    unsigned long long sums[2] = {0, 0};
    if (items > 0) {
        CK(ranges_count(a, c->stream));
        CK(tree_scan(a.count, items, ptr<long long>(c, S_RNG_BS), ptr<long long>(c, S_RNG_BO),
                     a.off, c->stream));
        CK(cudaMemcpyAsync(&c->h_misc[0], a.off + items, sizeof(long long), cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaMemcpyAsync(&c->h_misc[1], a.off + (long long)n * nchunks, sizeof(long long),
                           cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(sums, a.sums, sizeof(sums), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        R = (long long)c->h_misc[0];
        side0 = (long long)c->h_misc[1];
    }
    *n_ranges = R;
    if (summary) {
        summary->ranges[0] = side0;
        summary->ranges[1] = R - side0;
        summary->snapshots[0] = (int64_t)sums[0];
        summary->snapshots[1] = (int64_t)sums[1];
    }
    if (!ranges || R == 0) return IVM_OK;
    if (R > capacity) return IVM_ERR_CAPACITY;
    const bool rec_host = !is_device(ranges);
    if ((r = ensure(c, S_RNG_REC, rec_host ? sizeof(ivm_range) * (size_t)R : 0))) return r;
    bind_geometry(c, g);
    a.rec = rec_host ? ptr<ivm_range>(c, S_RNG_REC) : ranges;
    // the scene's BVH for the Blockage walks
    if ((r = enqueue_geometry(c, g, scene, hd, hd.data(), true))) return r;
    CK(ranges_write(a, c->stream));
    CK(ranges_blockers(g, a, R, c->d_err, c->stream));
    if ((r = read_error(c))) return r;
    if (rec_host)
        CK(cudaMemcpyAsync(ranges, a.rec, sizeof(ivm_range) * (size_t)R, cudaMemcpyDeviceToHost,
                           c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return IVM_OK;
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
    CK(record(c, 0));
    // adjacency lists of the matrix rows; the column array is sized for a
    // full matrix when that is small, so no count has to be read back
    if ((r = ensure(c, S_T_DEG, sizeof(long long) * (size_t)n))) return r;
    if ((r = ensure(c, S_T_ROW, sizeof(long long) * ((size_t)n + 1)))) return r;
    a.rowptr = ptr<long long>(c, S_T_ROW);
    const long long full = (long long)n * n;
    long long nnz = full;
    if (full > (1LL << 26)) {
        CK(tree_adjacency(a, ptr<long long>(c, S_T_DEG), c->stream));
        CK(cudaMemcpyAsync(&nnz, a.rowptr + n, sizeof(long long), cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    if ((r = ensure(c, S_T_COL, sizeof(int) * (size_t)(nnz > 0 ? nnz : 1)))) return r;
    if ((r = ensure(c, S_T_WT, sizeof(unsigned long long) * 2 * (size_t)(K + 1) * n))) return r;
    a.rowptr = ptr<long long>(c, S_T_ROW);
    a.col = ptr<int>(c, S_T_COL);
    a.wt = ptr<unsigned long long>(c, S_T_WT);
    if (full <= (1LL << 26)) CK(tree_adjacency(a, ptr<long long>(c, S_T_DEG), c->stream));
    CK(tree_fill(a, c->stream));
    if (K >= 1) {
        // runs of consecutive equal Tx rows: one chain per run
        const long long nb = (S + 255) / 256;
        if ((r = ensure(c, S_T_FLAG, sizeof(long long) * (size_t)S))) return r;
        if ((r = ensure(c, S_T_EXCL, sizeof(long long) * ((size_t)S + 1)))) return r;
        if ((r = ensure(c, S_T_BS, sizeof(long long) * (size_t)nb))) return r;
        if ((r = ensure(c, S_T_BO, sizeof(long long) * ((size_t)nb + 1)))) return r;
        if ((r = ensure(c, S_T_RUN, sizeof(int) * (size_t)S))) return r;
        if ((r = ensure(c, S_T_START, sizeof(long long) * (size_t)S))) return r;
        CK(tree_tx_runs(a, ptr<long long>(c, S_T_FLAG), ptr<long long>(c, S_T_EXCL),
                        ptr<long long>(c, S_T_BS), ptr<long long>(c, S_T_BO), ptr<int>(c, S_T_RUN),
                        ptr<long long>(c, S_T_START), c->stream));
        long long U = 0;
        CK(cudaMemcpyAsync(&U, ptr<long long>(c, S_T_EXCL) + S, sizeof(long long),
                           cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        std::vector<long long> start((size_t)U);
        CK(cudaMemcpy(start.data(), ptr<long long>(c, S_T_START), sizeof(long long) * U,
                      cudaMemcpyDeviceToHost));
        // run chunks: K chains of three n x C u64 vectors within ~768 MB
        long long C = (768LL << 20) / (24LL * K * n);
        if (C < 1) C = 1;
        if (C > 8192) C = 8192;
        if (C > U) C = U;
        const size_t xbytes = sizeof(unsigned long long) * 3 * (size_t)n * C * K;
        if ((r = ensure(c, S_T_XA, xbytes))) return r;
        for (long long u0 = 0; u0 < U; u0 += C) {
            const int Cc = (int)(U - u0 < C ? U - u0 : C);
            const long long t0 = start[u0], t1 = u0 + Cc < U ? start[u0 + Cc] : S;
            CK(tree_run_chunk(a, ptr<long long>(c, S_T_START), ptr<int>(c, S_T_RUN), u0, Cc, t0,
                              t1, ptr<unsigned long long>(c, S_T_XA), c->stream));
        }
    } else {
        CK(tree_order0(a, c->stream));
    }
    int status = IVM_OK;
    if (paths) {
        const long long items = S * (1 + (long long)K * n);
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
    if (sum_host)
        CK(cudaMemcpyAsync(summary, a.summary, sizeof(ivm_tree_summary) * (size_t)S * (K + 1),
                           cudaMemcpyDeviceToHost, c->stream));
    CK(record(c, 4));
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

// ============================================================================ ranker

namespace {

struct RankerHeader {
    uint32_t magic, version, in, hidden, out, params;
};
constexpr uint32_t kRankerMagic = 0x524d5649u;   // "IVMR"

int ranker_alloc(ivm_ctx *c)
{
    if (c->r_master) return IVM_OK;
    CK(cudaMalloc(&c->r_master, sizeof(float) * kRParams));
    CK(cudaMalloc(&c->r_m, sizeof(float) * kRParams));
    CK(cudaMalloc(&c->r_v, sizeof(float) * kRParams));
    CK(cudaMalloc(&c->r_grads, sizeof(float) * kRParams));
    CK(cudaMalloc(&c->r_wt, sizeof(__nv_bfloat16) * kRTEnd));
    return IVM_OK;
}

uint64_t sm64(uint64_t &state)
{
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// He-uniform initial weights from a fixed SplitMix64 stream, zero biases
void ranker_init(std::vector<float> &w)
{
    w.assign(kRParams, 0.f);
    uint64_t st = 0x1D0E5EEDull;
    const int lay[4][3] = {{kRIn, kRH, kRW1}, {kRH, kRH, kRW2}, {kRH, kRH, kRW3}, {kRH, kROut, kRW4}};
    for (auto &L : lay) {
        const float bound = sqrtf(6.f / L[0]);
        for (int i = 0; i < L[0] * L[1]; i++) {
            const float u = (float)(sm64(st) >> 11) * (1.f / 9007199254740992.f);
            w[L[2] + i] = (2.f * u - 1.f) * bound;
        }
    }
}

}  // namespace

extern "C" int ivm_ranker_train(ivm_ctx *c, const ivm_scene *scenes, int32_t n_scenes,
                                const ivm_params *params, int32_t epochs, float lr,
                                float *final_loss)
{
    if (!c || epochs < 1 || !(lr > 0.f)) return IVM_ERR_ARG;
    int r = check_params(params);
    if (r) return r;
    DeviceGuard dg(c->device);
    // candidate pairs and their logged nearest occluders
    DevScenes g;
    std::vector<SceneDesc> hd;
    if ((r = plan_geometry(c, scenes, n_scenes, params->samples_per_side, g, hd))) return r;
    if ((r = ensure(c, S_CBOX, sizeof(int) * kRCtx * (size_t)n_scenes))) return r;
    if ((r = ensure(c, S_NCL, (size_t)g.total_nodes + 1))) return r;
    bind_geometry(c, g);
    if ((r = enqueue_geometry(c, g, scenes, hd, hd.data(), true))) return r;
    CK(cudaMemsetAsync(c->d_misc, 0, sizeof(unsigned long long) * 2, c->stream));
    CK(launch_screen_count(g, hd.data(), c->d_misc, c->stream));
    CK(cudaMemcpyAsync(c->h_misc, c->d_misc, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const unsigned long long npairs = c->h_misc[0];
    if (npairs == 0) return IVM_ERR_ARG;
    if ((r = ensure(c, S_PAIRS, sizeof(int2) * npairs))) return r;
    if ((r = ensure(c, S_RFEAT, sizeof(float) * kRInPad * npairs))) return r;
    if ((r = ensure(c, S_RLAB, sizeof(int) * npairs))) return r;
    bind_geometry(c, g);
    CK(launch_screen_emit(g, hd.data(), ptr<int2>(c, S_PAIRS), c->d_misc + 1, npairs, c->stream));
    CK(ranker_clusters(g, ptr<int>(c, S_CBOX), ptr<signed char>(c, S_NCL), c->stream));
    CK(ranker_log_hits(g, ptr<int2>(c, S_PAIRS), npairs, ptr<int>(c, S_CBOX),
                       ptr<float>(c, S_RFEAT), ptr<int>(c, S_RLAB), nullptr, npairs, c->d_err,
                       c->stream));
    if ((r = read_error(c))) return r;
    std::vector<int> lab(npairs);
    std::vector<int2> prs(npairs);
    CK(cudaMemcpy(lab.data(), ptr<int>(c, S_RLAB), sizeof(int) * npairs, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(prs.data(), ptr<int2>(c, S_PAIRS), sizeof(int2) * npairs,
                  cudaMemcpyDeviceToHost));
    std::vector<int> idx;
    for (unsigned long long i = 0; i < npairs; i++)
        if (lab[i] >= 0) idx.push_back((int)i);
    if (idx.empty()) return IVM_ERR_ARG;
    // the screen emits pairs in atomic order: sort by pair so that the
    // shuffled batches, and so the trained weights, are reproducible
    std::sort(idx.begin(), idx.end(), [&](int a, int b) {
        return prs[a].x != prs[b].x ? prs[a].x < prs[b].x : prs[a].y < prs[b].y;
    });
    // weights and optimiser state
    if ((r = ranker_alloc(c))) return r;
    std::vector<float> w;
    ranker_init(w);
    CK(cudaMemcpy(c->r_master, w.data(), sizeof(float) * kRParams, cudaMemcpyHostToDevice));
    CK(cudaMemset(c->r_m, 0, sizeof(float) * kRParams));
    CK(cudaMemset(c->r_v, 0, sizeof(float) * kRParams));
    const int B = 512;
    const int n = (int)idx.size();
    const int steps = (n + B - 1) / B;
    if ((r = ensure(c, S_RIDX, sizeof(int) * (size_t)n))) return r;
    if ((r = ensure(c, S_RXB, sizeof(float) * B * kRIn))) return r;
    if ((r = ensure(c, S_RYB, sizeof(int) * B))) return r;
    if ((r = ensure(c, S_RACT, sizeof(float) * ranker_act_floats(B)))) return r;
    if ((r = ensure(c, S_RLOSS, sizeof(float) * (size_t)steps))) return r;
    uint64_t shuffle = 0xC0FFEEull;
    int step = 0;
    for (int ep = 0; ep < epochs; ep++) {
        for (int i = n - 1; i > 0; i--) {   // Fisher-Yates with a fixed stream
            const int j = (int)(sm64(shuffle) % (uint64_t)(i + 1));
            std::swap(idx[i], idx[j]);
        }
        CK(cudaMemcpyAsync(ptr<int>(c, S_RIDX), idx.data(), sizeof(int) * n,
                           cudaMemcpyHostToDevice, c->stream));
        for (int b = 0; b < steps; b++) {
            const int bb = b * B + B <= n ? B : n - b * B;
            CK(ranker_gather(ptr<float>(c, S_RFEAT), ptr<int>(c, S_RLAB), ptr<int>(c, S_RIDX) + b * B,
                             bb, ptr<float>(c, S_RXB), ptr<int>(c, S_RYB), c->stream));
            CK(ranker_grad(c->r_master, ptr<float>(c, S_RXB), ptr<int>(c, S_RYB), bb,
                           ptr<float>(c, S_RACT), c->r_grads, ptr<float>(c, S_RLOSS) + b, c->stream));
            CK(ranker_adam(c->r_master, c->r_grads, c->r_m, c->r_v, lr, ++step, c->stream));
        }
        CK(cudaStreamSynchronize(c->stream));   // the index buffer is rewritten next epoch
    }
    std::vector<float> losses(steps);
    CK(cudaMemcpy(losses.data(), ptr<float>(c, S_RLOSS), sizeof(float) * steps,
                  cudaMemcpyDeviceToHost));
    double sum = 0.0;
    for (float l : losses) sum += l;
    if (final_loss) *final_loss = (float)(sum / steps);
    CK(ranker_pack(c->r_master, c->r_wt, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->has_ranker = true;
    return IVM_OK;
}

extern "C" int ivm_ranker_save(ivm_ctx *c, void *blob, size_t *bytes)
{
    if (!c || !bytes || !c->has_ranker) return IVM_ERR_ARG;
    const size_t need = sizeof(RankerHeader) + sizeof(float) * kRParams;
    if (!blob) {
        *bytes = need;
        return IVM_OK;
    }
    if (*bytes < need) return IVM_ERR_ARG;
    DeviceGuard dg(c->device);
    RankerHeader h = {kRankerMagic, 1u, (uint32_t)kRIn, (uint32_t)kRH, (uint32_t)kROut,
                      (uint32_t)kRParams};
    memcpy(blob, &h, sizeof h);
    CK(cudaMemcpy(static_cast<char *>(blob) + sizeof h, c->r_master, sizeof(float) * kRParams,
                  cudaMemcpyDeviceToHost));
    *bytes = need;
    return IVM_OK;
}

extern "C" int ivm_ranker_load(ivm_ctx *c, const void *blob, size_t bytes)
{
    if (!c || !blob || bytes != sizeof(RankerHeader) + sizeof(float) * kRParams) return IVM_ERR_ARG;
    RankerHeader h;
    memcpy(&h, blob, sizeof h);
    if (h.magic != kRankerMagic || h.version != 1u || h.in != (uint32_t)kRIn ||
        h.hidden != (uint32_t)kRH || h.out != (uint32_t)kROut || h.params != (uint32_t)kRParams)
        return IVM_ERR_ARG;
    DeviceGuard dg(c->device);
    int r;
    if ((r = ranker_alloc(c))) return r;
    CK(cudaMemcpy(c->r_master, static_cast<const char *>(blob) + sizeof h,
                  sizeof(float) * kRParams, cudaMemcpyHostToDevice));
    CK(ranker_pack(c->r_master, c->r_wt, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->has_ranker = true;
    return IVM_OK;
}

extern "C" int ivm_ranker_infer(ivm_ctx *c, const float *x, int32_t batch, float *logits,
                                uint8_t *top)
{
    if (!c || !x || batch < 1 || (!logits && !top) || !c->has_ranker) return IVM_ERR_ARG;
    DeviceGuard dg(c->device);
    int r;
    if ((r = ensure(c, S_RXB, sizeof(float) * (size_t)batch * kRIn))) return r;
    if ((r = ensure(c, S_RACT, sizeof(float) * (size_t)batch * kROut))) return r;
    if ((r = ensure(c, S_RANKS, sizeof(unsigned long long) * (size_t)batch))) return r;
    CK(cudaMemcpyAsync(ptr<float>(c, S_RXB), x, sizeof(float) * (size_t)batch * kRIn,
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    CK(ranker_infer(ptr<float>(c, S_RXB), (unsigned long long)batch, RankerDev{c->r_wt, c->r_master},
                    ptr<float>(c, S_RACT), ptr<unsigned long long>(c, S_RANKS), c->n_sm, c->d_err,
                    c->stream));
    if ((r = read_error(c))) return r;
    if (logits)
        CK(cudaMemcpyAsync(logits, ptr<float>(c, S_RACT), sizeof(float) * (size_t)batch * kROut,
                           cudaMemcpyDeviceToHost, c->stream));
    if (top)
        CK(cudaMemcpyAsync(top, ptr<unsigned long long>(c, S_RANKS),
                           sizeof(unsigned long long) * (size_t)batch, cudaMemcpyDeviceToHost,
                           c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return IVM_OK;
}

extern "C" int ivm_ranker_gradients(ivm_ctx *c, const float *weights, const float *x,
                                    const int32_t *y, int32_t batch, float *grads, float *loss)
{
    if (!c || !weights || !x || !y || !grads || !loss || batch < 1) return IVM_ERR_ARG;
    for (int i = 0; i < batch; i++)
        if (y[i] < 0 || y[i] >= kROut) return IVM_ERR_ARG;
    DeviceGuard dg(c->device);
    int r;
    if ((r = ensure(c, S_RWT, sizeof(float) * kRParams))) return r;
    if ((r = ensure(c, S_RGT, sizeof(float) * (kRParams + 1)))) return r;
    if ((r = ensure(c, S_RXB, sizeof(float) * (size_t)batch * kRIn))) return r;
    if ((r = ensure(c, S_RYB, sizeof(int) * (size_t)batch))) return r;
    if ((r = ensure(c, S_RACT, sizeof(float) * ranker_act_floats(batch)))) return r;
    CK(cudaMemcpyAsync(ptr<float>(c, S_RWT), weights, sizeof(float) * kRParams,
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(ptr<float>(c, S_RXB), x, sizeof(float) * (size_t)batch * kRIn,
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(ptr<int>(c, S_RYB), y, sizeof(int) * (size_t)batch, cudaMemcpyHostToDevice,
                       c->stream));
    float *g = ptr<float>(c, S_RGT);
    CK(ranker_grad(ptr<float>(c, S_RWT), ptr<float>(c, S_RXB), ptr<int>(c, S_RYB), batch,
                   ptr<float>(c, S_RACT), g, g + kRParams, c->stream));
    CK(cudaMemcpyAsync(grads, g, sizeof(float) * kRParams, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(loss, g + kRParams, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return IVM_OK;
}

// ============================================================================ autotuner

extern "C" int ivm_autotune(ivm_ctx *c, const ivm_scene *scenes, int32_t n_scenes,
                            const int32_t *const *tx, const int32_t *const *rx,
                            const int64_t *n_snap, ivm_params *params)
{
    if (!c || !scenes || n_scenes < 1 || !params) return IVM_ERR_ARG;
    int r = check_params(params);
    if (r) return r;
    DeviceGuard dg(c->device);
    const int ns = n_scenes < 8 ? n_scenes : 8;
    const bool with_table = tx && rx && n_snap;
    // trial outputs in the context's scratch
    std::vector<int64_t> snaps(ns, 0);
    size_t mwords = 0, twords = 0, lbytes = 0;
    for (int k = 0; k < ns; k++) {
        if (!scenes[k].facets || scenes[k].n_facets < 1) return IVM_ERR_ARG;
        const size_t W = (size_t)words(scenes[k].n_facets);
        mwords += (size_t)scenes[k].n_facets * W;
        if (with_table) {
            if (n_snap[k] < 0) return IVM_ERR_ARG;
            // enough snapshots that the sample has the full run's parallelism
            snaps[k] = n_snap[k] < 16384 ? n_snap[k] : 16384;
            twords += (size_t)snaps[k] * 2 * W;
            lbytes += (size_t)snaps[k];
        }
    }
    if ((r = ensure(c, S_TUNE_M, sizeof(uint32_t) * mwords))) return r;
    if ((r = ensure(c, S_TUNE_T, sizeof(uint32_t) * twords))) return r;
    if ((r = ensure(c, S_TUNE_L, lbytes))) return r;
    std::vector<uint32_t *> mout(ns), tout(ns);
    std::vector<uint8_t *> lout(ns);
    size_t om = 0, ot = 0, ol = 0;
    for (int k = 0; k < ns; k++) {
        const size_t W = (size_t)words(scenes[k].n_facets);
        mout[k] = ptr<uint32_t>(c, S_TUNE_M) + om;
        om += (size_t)scenes[k].n_facets * W;
        tout[k] = ptr<uint32_t>(c, S_TUNE_T) + ot;
        ot += (size_t)snaps[k] * 2 * W;
        lout[k] = ptr<uint8_t>(c, S_TUNE_L) + ol;
        ol += (size_t)snaps[k];
    }
    ivm_params base = *params;
    base.flags &= ~IVM_FLAG_GRAPH;
    const int wpbs[] = {2, 4};
    const int mtiles[] = {1, 2, 4, 8, 16, 32, 64};
    const int ttiles[] = {8, 16, 32, 64, 128, 256, 512, 1024, 2048};
    const int ptiles[] = {16, 64, 128};   // stretch lengths tried besides the default 32
    float best_total = 1e30f;
    ivm_params best = *params;
    for (int wpb : wpbs) {
        ivm_params p = base;
        p.warps_per_block = wpb;
        float bm = 0.f, bt = 0.f;
        int mt = mtiles[0], tt = ttiles[0];
        bool first = true;
        for (int tile : mtiles) {
            p.tile = tile;
            ivm_stats st;
            float ms = 1e30f;
            for (int rep = 0; rep < 3; rep++) {   // the first run warms the arena up
                if ((r = ivm_build_matrix(c, scenes, ns, &p, mout.data(), &st))) return r;
                if (rep == 1 || (rep > 1 && st.ms_traverse > ms)) ms = st.ms_traverse;
            }
            if (first || ms < bm) { bm = ms; mt = tile; }
            first = false;
        }
        p.tile = mt;
        // then the corner proof the other way at that tile (same bits either way)
        {
            ivm_params q = p;
            q.flags ^= IVM_FLAG_NO_CORNER_PROOF;
            ivm_stats st;
            float ms = 1e30f;
            for (int rep = 0; rep < 3; rep++) {
                if ((r = ivm_build_matrix(c, scenes, ns, &q, mout.data(), &st))) return r;
                if (rep == 1 || (rep > 1 && st.ms_traverse > ms)) ms = st.ms_traverse;
            }
            if (ms < bm) { bm = ms; p.flags = q.flags; }
        }
        if (with_table) {
            first = true;
            for (int tile : ttiles) {
                p.table_tile = tile;
                ivm_stats st;
                float ms = 1e30f;
                for (int rep = 0; rep < 3; rep++) {   // warm-up, then the slower of two
                    if ((r = ivm_build_table(c, scenes, ns, &p, tx, rx, snaps.data(), tout.data(),
                                             lout.data(), &st)))
                        return r;
                    if (rep == 1 || (rep > 1 && st.ms_traverse > ms)) ms = st.ms_traverse;
                }
                if (first || ms < bt) { bt = ms; tt = tile; }
                first = false;
            }
            p.table_tile = tt;
            // then the stretch length at that item size
            int pt = base.proof_tile > 0 ? base.proof_tile : 32;
            for (int ptile : ptiles) {
                p.proof_tile = ptile;
                ivm_stats st;
                float ms = 1e30f;
                for (int rep = 0; rep < 3; rep++) {
                    if ((r = ivm_build_table(c, scenes, ns, &p, tx, rx, snaps.data(), tout.data(),
                                             lout.data(), &st)))
                        return r;
                    if (rep == 1 || (rep > 1 && st.ms_traverse > ms)) ms = st.ms_traverse;
                }
                if (ms < bt) { bt = ms; pt = ptile; }
            }
            p.proof_tile = pt;
        }
        if (bm + bt < best_total) {
            best_total = bm + bt;
            best = *params;
            best.warps_per_block = wpb;
            best.tile = mt;
            best.flags = (params->flags & ~IVM_FLAG_NO_CORNER_PROOF) |
                         (p.flags & IVM_FLAG_NO_CORNER_PROOF);
            if (with_table) {
                best.table_tile = tt;
                best.proof_tile = p.proof_tile;
            }
        }
    }
    *params = best;
    return IVM_OK;
}
