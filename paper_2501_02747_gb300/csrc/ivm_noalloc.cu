// ivm_noalloc.cu -- ivm_build_matrix_noalloc: the matrix build of one scene
// with every scratch buffer in a fixed device array, so that the call itself
// allocates no memory.
//
// Who needs it: callers that must not allocate device memory at the time of
// the call -- code running inside a memory pool or allocator that forbids
// cudaMalloc, real-time loops that must not hit the allocator's
// synchronisation, or hosts that own all device memory themselves.  The
// regular entry points grow a per-context scratch arena with cudaMalloc.
//
// The scratch is one file-scope __device__ array sized for the limits below
// (about 5 MB); every GPU that loads the library holds it until the process
// exits.  In host code the array's name is only a host-side stand-in, so its
// device address is looked up with cudaGetSymbolAddress, once per device, on
// the first call made with that device current (that first call should
// therefore come before any stream capture).  The address is kept for the
// life of the process: after cudaDeviceReset on that device it is stale, and
// the entry point must not be called again on that device.  All calls share the array and
// it keeps the last call's contents: everything that must start at zero is
// cleared by each call, and two calls that overlap on the GPU (on different
// streams, or from different host threads) race on it.
#include <mutex>

#include "ivm_internal.cuh"

using namespace ivm;

namespace {

constexpr int kMaxN = IVM_NOALLOC_MAX_FACETS;
constexpr int kMaxS = IVM_NOALLOC_MAX_SAMPLES_PER_SIDE;
constexpr long long kMaxPairs = (long long)kMaxN * (kMaxN - 1) / 2;

constexpr size_t al(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t OFF_DESC = 0;
constexpr size_t OFF_ERR = OFF_DESC + al(sizeof(SceneDesc));
constexpr size_t OFF_CTR = OFF_ERR + al(sizeof(int));
constexpr size_t OFF_MISC = OFF_CTR + al(sizeof(unsigned long long) * C_COUNT_);
constexpr size_t OFF_LEAF = OFF_MISC + al(sizeof(unsigned long long) * 4);
constexpr size_t OFF_FSCENE = OFF_LEAF + al(sizeof(Leaf) * kMaxN);
constexpr size_t OFF_BOX = OFF_FSCENE + al(sizeof(int) * kMaxN);
constexpr size_t OFF_SX = OFF_BOX + al(sizeof(int) * 6 * kMaxN);
constexpr size_t OFF_SY = OFF_SX + al(sizeof(int) * kMaxN * kMaxS * kMaxS);
constexpr size_t OFF_SZ = OFF_SY + al(sizeof(int) * kMaxN * kMaxS * kMaxS);
constexpr size_t OFF_KEYS = OFF_SZ + al(sizeof(int) * kMaxN * kMaxS * kMaxS);
constexpr size_t OFF_SORTED = OFF_KEYS + al(sizeof(unsigned long long) * kMaxN);
constexpr size_t OFF_BOUNDS = OFF_SORTED + al(sizeof(unsigned long long) * kMaxN);
constexpr size_t OFF_ORDER = OFF_BOUNDS + al(sizeof(int) * 6);
constexpr size_t OFF_NODES = OFF_ORDER + al(sizeof(int) * kMaxN);
constexpr size_t OFF_PARENT = OFF_NODES + al(sizeof(Node) * kMaxN);
constexpr size_t OFF_VISITS = OFF_PARENT + al(sizeof(int) * 2 * kMaxN);
constexpr size_t OFF_PAIRS = OFF_VISITS + al(sizeof(int) * kMaxN);
constexpr size_t kScratchBytes = OFF_PAIRS + al(sizeof(int2) * kMaxPairs);

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

}  // namespace

// The scratch array.  Device code could name it directly; host code must
// use the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array on the current device (looked up once).
static int scratch_base(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return IVM_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return IVM_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[dev]);
    return IVM_OK;
}

#define NA_CK(call)                             \
    do {                                        \
        if ((call) != cudaSuccess) {            \
            cudaGetLastError();                 \
            return IVM_ERR_CUDA;                \
        }                                       \
    } while (0)

// True when p is device (or managed) memory that the current device dev can
// use.  A host pointer or another GPU's memory would make the kernels read an
// address they cannot reach, so such arguments are refused before anything is
// enqueued.
static bool on_device(const void *p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

static int noalloc_error(unsigned char *base, cudaStream_t st)
{
    int h = 0;
    NA_CK(cudaMemcpyAsync(&h, base + OFF_ERR, sizeof(int), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    return h;
}

extern "C" int ivm_build_matrix_noalloc(const ivm_facet *facets, int32_t n_facets,
                                        const ivm_params *params, uint32_t *matrix,
                                        void *cuda_stream)
{
    if (!facets || !matrix || !params) return IVM_ERR_ARG;
    if (n_facets < 1 || n_facets > kMaxN) return IVM_ERR_ARG;
    const int s = params->samples_per_side;
    if (s < 1 || s > kMaxS) return IVM_ERR_ARG;
    // no context, hence no ranker: the learned form is refused rather than
    // silently run as the filtered one
    if (params->mode != IVM_MODE_EXACT && params->mode != IVM_MODE_FILTERED) return IVM_ERR_ARG;
    if (params->tile < 0 || params->warps_per_block < 0 || params->warps_per_block > 4)
        return IVM_ERR_ARG;
    int dev = 0;
    NA_CK(cudaGetDevice(&dev));
    if (!on_device(facets, dev) || !on_device(matrix, dev)) return IVM_ERR_ARG;
    unsigned char *base = nullptr;
    int r = scratch_base(dev, &base);
    if (r) return r;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int n_sm = 0;
    NA_CK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));

    SceneDesc hd = {};
    hd.facet0 = 0;
    hd.n = n_facets;
    hd.W = (n_facets + 31) / 32;
    hd.node0 = 0;
    hd.root = n_facets >= 2 ? 0 : ~0;
    hd.s = s;
    hd.sample0 = 0;
    hd.rw0 = 0;
    hd.matrix = matrix;
    hd.row_lo = 0;
    hd.row_hi = n_facets;
    hd.budget = 4 * n_facets + 16;

    DevScenes g = {};
    g.n_scenes = 1;
    g.total_facets = n_facets;
    g.total_nodes = n_facets - 1;
    g.total_samples = n_facets * s * s;
    g.max_n = n_facets;
    g.desc = reinterpret_cast<SceneDesc *>(base + OFF_DESC);
    g.facets = facets;
    g.leaf = reinterpret_cast<Leaf *>(base + OFF_LEAF);
    g.fscene = reinterpret_cast<int *>(base + OFF_FSCENE);
    g.box = reinterpret_cast<int *>(base + OFF_BOX);
    g.sx = reinterpret_cast<int *>(base + OFF_SX);
    g.sy = reinterpret_cast<int *>(base + OFF_SY);
    g.sz = reinterpret_cast<int *>(base + OFF_SZ);
    g.keys = reinterpret_cast<unsigned long long *>(base + OFF_KEYS);
    g.sorted = reinterpret_cast<unsigned long long *>(base + OFF_SORTED);
    g.bounds = reinterpret_cast<int *>(base + OFF_BOUNDS);
    g.order = reinterpret_cast<int *>(base + OFF_ORDER);
    g.nodes = reinterpret_cast<Node *>(base + OFF_NODES);
    g.parent = reinterpret_cast<int *>(base + OFF_PARENT);
    g.visits = reinterpret_cast<int *>(base + OFF_VISITS);
    int *err = reinterpret_cast<int *>(base + OFF_ERR);
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(base + OFF_CTR);
    unsigned long long *misc = reinterpret_cast<unsigned long long *>(base + OFF_MISC);
    int2 *pairs = reinterpret_cast<int2 *>(base + OFF_PAIRS);

    // state left by the previous call is cleared here
    NA_CK(cudaMemcpyAsync(g.desc, &hd, sizeof(SceneDesc), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
    NA_CK(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long) * C_COUNT_, st));
    NA_CK(cudaMemsetAsync(misc, 0, sizeof(unsigned long long) * 4, st));
    NA_CK(launch_ingest(g, err, st));
    if ((r = noalloc_error(base, st))) return r;
    NA_CK(launch_bvh(g, st));
    NA_CK(launch_screen_count(g, &hd, misc, st));
    unsigned long long npairs = 0;
    NA_CK(cudaMemcpyAsync(&npairs, misc, sizeof(npairs), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    if ((long long)npairs > kMaxPairs) return IVM_ERR_INTERNAL;
    NA_CK(launch_screen_emit(g, &hd, pairs, misc + 1, npairs, st));
    NA_CK(cudaMemsetAsync(matrix, 0, sizeof(uint32_t) * (size_t)hd.n * hd.W, st));
    LaunchCfg cfg;
    cfg.mode = params->mode == IVM_MODE_EXACT ? IVM_MODE_EXACT : IVM_MODE_FILTERED;
    cfg.persistent = (params->flags & IVM_FLAG_PERSISTENT) != 0;
    cfg.warps_per_block = params->warps_per_block > 0 ? params->warps_per_block : 4;
    cfg.tile = params->tile > 0 ? params->tile : (cfg.persistent ? 4 : 1);
    cfg.n_sm = n_sm;
    cfg.cache = (params->flags & IVM_FLAG_OCCLUDER_CACHE) != 0;
    cfg.dedup = 0;
    cfg.aligned = (params->flags & IVM_FLAG_ALIGNED_FACETS) != 0;
    cfg.corner = (params->flags & IVM_FLAG_NO_CORNER_PROOF) == 0;
    NA_CK(launch_matrix(g, pairs, npairs, cfg, misc + 2, ctr, err, st));
    return noalloc_error(base, st);
}
