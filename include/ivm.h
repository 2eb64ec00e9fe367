/*
 * ivm.h -- C ABI of the GB300 inter-visibility library.
 *
 * The library builds, on one GPU, the three products of the pre-processing
 * method of Yang et al., "An Efficient Pre-Processing Method for 6G Dynamic
 * Ray-Tracing Channel Modeling" (arXiv 2501.02747):
 *
 *   ivm_build_matrix       the static inter-visibility matrix over building
 *                          facets (Sec. II: the intersection judgment between
 *                          static objects is done once, in pre-processing);
 *   ivm_build_table        the per-snapshot inter-visibility table of the
 *                          mobile Tx and Rx (Sec. III-B/C, Table II);
 *   ivm_expand_image_tree  the image-tree path sets read off the matrix and
 *                          the table (Sec. II intro, Sec. III-B, Table II).
 *
 * Geometry.  Coordinates are int32 centimetres.  A facet is the
 * parallelogram {o + a u + b v : a, b in [0,1]} with outward normal u x v.
 * Internally every coordinate is multiplied by 2s (s = samples per side) so
 * that the s x s cell-centre samples p_ab = 2s o + (2a+1) u + (2b+1) v are
 * integers.  Range contract (else IVM_ERR_RANGE): every scaled corner
 * coordinate and every scaled Tx/Rx coordinate has magnitude < 2^22; u x v is
 * not zero; u x v divided by the gcd of its components fits in int32.
 *
 * Visibility rules (exact; no tolerance):
 *   front(x, f)   <=> (u x v) . (x - 2s o) > 0, strict (Sec. II-B, Eq. (2):
 *                     180 degrees or more counts as not visible);
 *   blocked(P, Q) <=> some facet of the scene (closed) meets the open
 *                     segment {P + l (Q - P) : 0 < l < 1};
 *   M_ij = [i != j] and exists samples p of i, q of j: front(q, i) and
 *          front(p, j) and not blocked(p, q)  (any free sample pair suffices:
 *          partial visibility is visibility, Sec. III-A);
 *   vis_X[t][j] = front(X_t, j) and exists sample q of j: not blocked(X_t, q)
 *          for X in {Tx, Rx}; los[t] = not blocked(Tx_t, Rx_t).
 *
 * Bit rows.  A row of N bits is W = ceil(N / 32) uint32 words; bit j is word
 * j >> 5, bit j & 31 (LSB first); padding bits are written as 0.
 *
 * Memory.  Every pointer argument may be host memory or device memory of the
 * context's device; the library tells them apart with
 * cudaPointerGetAttributes.  Host inputs are copied to the device and host
 * outputs copied back inside the call.  The caller owns every buffer it
 * passes; the context owns its scratch (scaled facets, BVH, pair lists,
 * counters), which grows on demand and is freed by ivm_destroy.
 *
 * Streams and errors.  Work is enqueued on the stream given to ivm_create;
 * every call synchronises that stream before it returns, so that device-side
 * error words can be reported.  Calls return IVM_OK or a negative-free error
 * code below; no exception crosses the ABI.  A context is used by one host
 * thread at a time.
 */
#ifndef IVM_H
#define IVM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ error codes */
#define IVM_OK 0
#define IVM_ERR_ARG 1        /* null pointer, bad size or bad parameter */
#define IVM_ERR_RANGE 2      /* geometry outside the range contract above */
#define IVM_ERR_CAPACITY 3   /* path buffer too small; *n_paths_out = needed */
#define IVM_ERR_TIMEOUT 4    /* a device-side iteration budget ran out */
#define IVM_ERR_CUDA 5       /* a CUDA runtime call failed */
#define IVM_ERR_INTERNAL 6   /* an internal invariant failed (stack depth) */

/* ----------------------------------------------------------- forms (mode) */
#define IVM_MODE_EXACT 0     /* exact integer facet tests */
#define IVM_MODE_FILTERED 1  /* FP32 facet tests with a proven error bound,
                                exact integer tests only when undecided */
#define IVM_MODE_LEARNED 2   /* FILTERED + learned order of BVH clusters */

/* ------------------------------------------------------------ flag bits */
#define IVM_FLAG_PERSISTENT 1  /* persistent kernels over a work queue */
#define IVM_FLAG_GRAPH 2       /* replay the call's launches as a CUDA graph */
#define IVM_FLAG_OCCLUDER_CACHE 4 /* test each warp's last blockers before the BVH */
#define IVM_FLAG_DEDUP_SOURCES 8  /* table: trace one row per run of equal positions */
#define IVM_FLAG_NO_SPLIT 16      /* table, persistent: no lazy splitting of snapshot ranges
                                     (idle warps otherwise take half of a busy warp's rest) */
#define IVM_FLAG_ALIGNED_FACETS 32 /* FILTERED / LEARNED: facets that are axis-aligned
                                     rectangles (u and v along two different coordinate
                                     axes) take a plane-crossing test, FP32 with a proven
                                     error bound and exact int64 where it cannot decide,
                                     in place of the four-edge FP32 filter; other facets
                                     keep the filter.  Same bits; not in the paper */
#define IVM_FLAG_NO_CORNER_PROOF 64 /* matrix, with OCCLUDER_CACHE: do not try to settle a
                                     hidden pair from its 16 corner-sample segments before
                                     its packets (a schedule choice: same bits; the
                                     autotuner sets or clears it); not in the paper */

typedef struct ivm_facet {
    int32_t o[3], u[3], v[3]; /* cm; u x v points outward */
    int32_t building;         /* id carried through; -1 for the ground */
} ivm_facet;                  /* 40 bytes */

typedef struct ivm_scene {
    const ivm_facet *facets;  /* host or device, n_facets records */
    int32_t n_facets;         /* >= 1 */
} ivm_scene;

typedef struct ivm_params {
    int32_t samples_per_side; /* s, 1..8 */
    int32_t max_order;        /* K for ivm_expand_image_tree, 0..8 */
    int32_t mode;             /* IVM_MODE_* */
    int32_t tile;             /* matrix: candidate pairs per queue pop (0 = default) */
    int32_t warps_per_block;  /* 1..4 (0 = default 4) */
    int32_t flags;            /* IVM_FLAG_* */
    int32_t table_tile;       /* table: consecutive snapshots per work item (0 = 32) */
    int32_t proof_tile;       /* table: snapshots per straight-stretch proof, 1..65536
                                 (0 = 32); a launch-shape choice, same bits */
} ivm_params;

typedef struct ivm_stats {
    uint64_t pairs;           /* ordered facet pairs decided (sum of N^2) */
    uint64_t cand_pairs;      /* unordered pairs passing the facing screen */
    uint64_t segments;        /* segments whose occlusion was tested */
    uint64_t node_tests;      /* segment-vs-box tests */
    uint64_t leaf_tests;      /* segment-vs-facet tests */
    uint64_t undecided;       /* FP32 facet tests left undecided (FILTERED) */
    uint64_t exact_tests;     /* facet tests decided by integer arithmetic */
    uint64_t ranker_hits;     /* blocked segments whose occluder lay in the
                                 ranker's first proposed cluster (LEARNED) */
    uint64_t cache_hits;      /* segments blocked by an occluder-cache facet */
    uint64_t dedup_rows;      /* table rows copied from an equal-position row */
    float ms_ingest, ms_bvh, ms_screen, ms_traverse, ms_tree, ms_total;
    uint64_t ranker_hits8;    /* blocked segments whose occluder lay in one of the
                                 ranker's proposed clusters walked first (LEARNED;
                                 up to 8 per pair: hits at 8) */
} ivm_stats;

typedef struct ivm_tree_summary {
    uint64_t count;           /* number of order-k paths */
    uint64_t fp0, fp1;        /* sum over paths of prod_m h_c(m, f_m), mod 2^64 */
} ivm_tree_summary;

typedef struct ivm_ctx ivm_ctx;

/* Create a context on `device`; `cuda_stream` is a cudaStream_t (NULL for
 * the legacy default stream).  Errors: IVM_ERR_ARG, IVM_ERR_CUDA. */
int ivm_create(ivm_ctx **out, int device, void *cuda_stream);

/* Free the context and its scratch.  Accepts NULL. */
int ivm_destroy(ivm_ctx *ctx);

/* Inter-visibility matrix (Sec. II; the intersection judgment moved into
 * pre-processing, Abstract and Sec. I).  For each scene k, matrix[k] receives
 * N_k rows of W_k words, row i = facets visible from facet i; the matrix is
 * symmetric with a zero diagonal.  n_scenes > 1 runs all scenes in one
 * launch sequence (the batched form).  stats may be NULL.
 * Errors: IVM_ERR_ARG (null pointers, n_scenes < 1, s outside 1..8),
 * IVM_ERR_RANGE, IVM_ERR_TIMEOUT, IVM_ERR_INTERNAL, IVM_ERR_CUDA. */
int ivm_build_matrix(ivm_ctx *ctx, const ivm_scene *scenes, int32_t n_scenes,
                     const ivm_params *params, uint32_t *const *matrix, ivm_stats *stats);

/* One part of the matrix, for splitting the work across devices (rows are
 * independent given the scene).  Decides only the unordered pairs (i, j),
 * i < j, with row_begin[k] <= i < row_end[k], and writes both of their bits
 * (row i and row j); every other bit of matrix[k] is 0.  Over a partition of
 * [0, N_k) into row ranges, the bitwise OR -- or, the bit sets being
 * disjoint, the integer sum -- of the parts is the ivm_build_matrix result.
 * stats->pairs counts the ordered pairs the part decides.  Errors: as
 * ivm_build_matrix; IVM_ERR_ARG if a range is not 0 <= begin <= end <= N_k. */
int ivm_build_matrix_rows(ivm_ctx *ctx, const ivm_scene *scenes, int32_t n_scenes,
                          const ivm_params *params, const int32_t *row_begin,
                          const int32_t *row_end, uint32_t *const *matrix, ivm_stats *stats);

/* Inter-visibility table for specific points along the route (Sec. III-B/C,
 * Table II).  For scene k: tx[k], rx[k] are [n_snap[k]][3] int32 cm;
 * table[k] receives [n_snap[k]][2][W_k] words (row 0 the Tx's visible
 * facets, row 1 the Rx's); los[k] receives n_snap[k] bytes, 1 if the direct
 * Tx-Rx segment is free (1 when Tx_t = Rx_t).  The matrix is not an input:
 * the table is defined by geometry, and the image tree combines the two.
 * One scene of at least 16,384 snapshots whose table or los is host memory
 * is traversed in up to 8 snapshot chunks, each copied to the host on a
 * second stream of the context while the next is traversed; the call returns
 * once every copy has landed.  After an error return the output buffers hold
 * unspecified contents.
 * Errors: as ivm_build_matrix (IVM_ERR_RANGE also for a Tx/Rx position). */
int ivm_build_table(ivm_ctx *ctx, const ivm_scene *scenes, int32_t n_scenes,
                    const ivm_params *params, const int32_t *const *tx,
                    const int32_t *const *rx, const int64_t *n_snap,
                    uint32_t *const *table, uint8_t *const *los, ivm_stats *stats);

/* Image-tree expansion (Sec. II intro; Sec. III-B, Table II: a path is
 * transmitter -> reference face -> ... -> aim face).  For every snapshot t
 * and order k = 0..max_order: summary[t][k] = {count, fp0, fp1} over the
 * paths (f1..fk) with vis_Tx[t][f1], M[f_m][f_m+1] for each hop, and
 * vis_Rx[t][fk]; order 0 is the direct path (count = fp0 = fp1 = los[t]).
 * Fingerprint weights: h_c(m, f) = splitmix64(seed_c ^ (m << 32) ^ f) | 1
 * with seed_0 = 0x243F6A8885A308D3, seed_1 = 0x13198A2E03707344 and
 * splitmix64 the SplitMix64 output function (Steele, Lea, Flood 2014).
 * matrix is [n_facets][W], table [n_snap][2][W], los [n_snap],
 * summary [n_snap][max_order + 1].
 * If paths is not NULL, path records int32 [path_capacity][max_order + 2] =
 * (t, k, f1..fk, -1 padding) are written in lexicographic order of
 * (t, k, f1, ..., fk); *n_paths_out (may be NULL) receives the total number
 * of paths, whether or not they fit.  Errors: IVM_ERR_ARG,
 * IVM_ERR_CAPACITY (the first path_capacity records are written),
 * IVM_ERR_CUDA. */
int ivm_expand_image_tree(ivm_ctx *ctx, const uint32_t *matrix, const uint32_t *table,
                          const uint8_t *los, int32_t n_facets, int64_t n_snap,
                          int32_t max_order, ivm_tree_summary *summary, int32_t *paths,
                          int64_t path_capacity, int64_t *n_paths_out);

/* Cap on the steps of every BVH walk of this context's later calls (0: the
 * automatic 4 N + 16, more than any valid tree needs).  A walk that runs out
 * stops, the call returns IVM_ERR_TIMEOUT, and the context stays usable: the
 * device-side watchdog every traversal carries, made testable.
 * Errors: IVM_ERR_ARG (steps < 0). */
int ivm_set_walk_budget(ivm_ctx *ctx, int32_t steps);

/* ------------------------------------------------------- visibility ranges
 * Sec. III-C, Tables III-IV: along the route, a visibility range of facet j
 * seen from a side's source (the transmitter, side 0, or the receiver, side
 * 1) is a maximal run of consecutive snapshots [begin, end) in which bit j of
 * that side's table row is set; begin and end are the ray creation and
 * suppression points.  The Blockage column: at snapshot begin - 1 and at
 * snapshot end, the first facet (smallest segment parameter, ties to the
 * lower facet index) on the segment from the source to facet j's centre
 * sample (a = b = floor(s / 2)); -1 where the route starts or ends, -2 where
 * facet j does not face the source there, -3 when no facet blocks it (only
 * for a table that does not match the geometry).  The facet's building, the
 * paper's column, is its ivm_facet.building. */
typedef struct ivm_range {
    int32_t side;             /* 0: Tx row, 1: Rx row */
    int32_t facet;            /* the visible node j */
    int64_t begin, end;       /* snapshots [begin, end) */
    int32_t block_before;     /* first facet on the segment at begin - 1 (or -1/-2/-3) */
    int32_t block_after;      /* the same at end */
} ivm_range;

/* Sec. III-D, Eq. (8)-(9): with snapshots dt apart, range l lasts
 * T_c,l = d_l / v_l = (end - begin) dt, and the mean over a side's L ranges is
 * T_c = dt snapshots[side] / ranges[side]; with both ends moving, the smaller
 * of the two sides' values is the scenario's. */
typedef struct ivm_range_summary {
    int64_t ranges[2];        /* number of ranges per side */
    int64_t snapshots[2];     /* summed range lengths per side (= set bits) */
} ivm_range_summary;

/* Visibility ranges of one scene's table [n_snap][2][W] (as written by
 * ivm_build_table for the same scene, params and positions tx, rx [n_snap][3]
 * cm; host or device pointers).  ranges (host or device) receives the records
 * ordered by side, facet, begin; *n_ranges the count.  ranges NULL: count
 * and summary only.  Errors: IVM_ERR_ARG, IVM_ERR_RANGE (a position out of
 * range), IVM_ERR_CAPACITY (capacity < *n_ranges; nothing written but the
 * count and summary), IVM_ERR_TIMEOUT, IVM_ERR_CUDA. */
int ivm_visibility_ranges(ivm_ctx *ctx, const ivm_scene *scene, const ivm_params *params,
                          const int32_t *tx, const int32_t *rx, int64_t n_snap,
                          const uint32_t *table, ivm_range *ranges, int64_t capacity,
                          int64_t *n_ranges, ivm_range_summary *summary);

/* ---------------------------------------------------- interface relations
 * Sec. II-B, Table I, Eq. (1)-(2), for every visible ordered pair M_ij = 1
 * (reference face i, aim face j), row-major: relation 1 = PAR (parallel
 * normals), 2 = PER (perpendicular normals), 0 = neither; and per edge k of
 * face i (O -> O+U -> O+U+V -> O+V), the range (min, max) over face j's
 * corners F of the angle, in degrees, between the reference vector from the
 * edge's midpoint B to the opposite edge's midpoint and F - B (Eq. (1)), an
 * angle of 180 recorded as 0 (Eq. (2)).
 *
 * matrix [N][W] as written by ivm_build_matrix (host or device); pairs
 * [capacity][2] int32, relation [capacity], ranges [capacity][4][2] double
 * (host or device; pairs NULL: count only, *n_pairs gets the count).
 * Errors: IVM_ERR_ARG, IVM_ERR_CAPACITY (capacity < *n_pairs; nothing
 * written but the count), IVM_ERR_CUDA. */
int ivm_interface_relations(ivm_ctx *ctx, const ivm_scene *scene, const ivm_params *params,
                            const uint32_t *matrix, int32_t *pairs, uint8_t *relation,
                            double *ranges, int64_t capacity, int64_t *n_pairs);

/* ---------------------------------------------------------------- edges
 * Edges as visible nodes (the matrix and table list visible faces and edges:
 * Sec. I-II) and the edge nearest a source (first-order diffraction by the
 * edge closest to the receiver: Sec. III-B).  Edge e is the segment from
 * (edges[6e], edges[6e+1], edges[6e+2]) to (edges[6e+3..6e+5]), cm, with s
 * samples at the cell centres A + (2a+1)/(2s) (B - A).  For each snapshot
 * and side (0: Tx, 1: Rx), bit e of the row is 1 when some sample of e is
 * reachable from the source by a segment no facet blocks (open segment,
 * closed facets), and nearest holds the visible edge with the sample
 * closest to the source (squared distance over all of its samples, ties to
 * the lower index), -1 if none.
 *
 * table [n_snap][2][WE] (WE = ceil(n_edges / 32)) and nearest [n_snap][2]:
 * host or device.  Errors: IVM_ERR_ARG (n_edges outside 0..65535),
 * IVM_ERR_RANGE (a source or an edge sample out of range), IVM_ERR_TIMEOUT,
 * IVM_ERR_CUDA. */
int ivm_build_edge_table(ivm_ctx *ctx, const ivm_scene *scene, const ivm_params *params,
                         const int32_t *edges, int32_t n_edges, const int32_t *tx,
                         const int32_t *rx, int64_t n_snap, uint32_t *table, int32_t *nearest);

/* Measured FP32 FMA issue rate of the context's GPU, in FMA lane operations
 * per second (one per lane per FMA; FLOP/s is twice this): eight independent
 * FMA chains per thread on a full-occupancy grid, best of three timed runs
 * after one warm-up.  The denominator of the traversal kernels' "alu"
 * roofline, which no library GEMM peak measures.  Errors: IVM_ERR_ARG,
 * IVM_ERR_CUDA. */
int ivm_fp32_peak(ivm_ctx *ctx, double *lane_ops_per_s);

/* Edges as rows and columns of the matrix (Sec. I-II: per face or edge, the
 * visible faces and edges; the nodes of first-order diffraction, Sec. III-B).
 * Edge e is edges[6e..6e+5] as above, with s samples, and edge_faces[2e],
 * edge_faces[2e+1] are the two facets (scene indices) that meet at it; a
 * point P reaches the edge from outside only when P is strictly in front of
 * one of them (ext).  fe[i][e] = 1 when some sample p of facet i and some
 * sample q of edge e have q strictly in front of i, ext(p, e) and the open
 * segment p-q meets no closed facet; ee[e][g] = 1 (e != g) when some samples
 * q of e and r of g have ext(r, e), ext(q, g) and q-r unblocked (ee is
 * symmetric).  The edge -> facet block of the full matrix is fe transposed.
 *
 * edges [n_edges][6], edge_faces [n_edges][2], fe [N][WE], ee [n_edges][WE]
 * (WE = ceil(n_edges / 32), padding bits 0): host or device.  params:
 * samples_per_side and mode (IVM_MODE_EXACT or IVM_MODE_FILTERED, the same
 * bits).  Errors: IVM_ERR_ARG (n_edges < 0, a null buffer, an adjacent facet
 * index outside 0..N-1), IVM_ERR_RANGE (an edge sample out of range),
 * IVM_ERR_TIMEOUT, IVM_ERR_CUDA. */
int ivm_build_edge_matrix(ivm_ctx *ctx, const ivm_scene *scene, const ivm_params *params,
                          const int32_t *edges, const int32_t *edge_faces, int32_t n_edges,
                          uint32_t *fe, uint32_t *ee);

/* ------------------------------------------------- ray validation
 * The image method on image-tree candidates (Sec. IV-B: the pre-processed
 * image tree and the brute-force method give the same valid rays).  For path
 * record (t, k, f1..fk), source T = tx[t] and receiver R = rx[t]: images I_0
 * = T, I_m = the mirror image of I_(m-1) in the plane of f_m; reflection
 * points from the receiver back, P_(k+1) = R and P_m where the segment from
 * P_(m+1) to I_m crosses the plane of f_m strictly inside it; the candidate is
 * a valid ray when every P_m lies in the closed face f_m, I_(m-1) and P_(m+1)
 * are strictly in front of f_m, and no facet meets any open leg P_m -> P_(m+1)
 * (P_0 = T).  Order 0 is the direct segment.  Exact integer arithmetic;
 * every facet of the scene must be an axis-aligned rectangle.
 *
 * paths [n_paths][max_order + 2] as written by ivm_expand_image_tree (host or
 * device); valid [n_paths] receives 1 or 0 (host or device); max_order <= 8.
 * Errors: IVM_ERR_ARG (a facet not axis-aligned, a record with t or k or a
 * facet index out of range), IVM_ERR_RANGE, IVM_ERR_TIMEOUT, IVM_ERR_CUDA. */
int ivm_validate_paths(ivm_ctx *ctx, const ivm_scene *scene, const ivm_params *params,
                       const int32_t *tx, const int32_t *rx, int64_t n_snap,
                       const int32_t *paths, int64_t n_paths, int32_t max_order,
                       uint8_t *valid);

/* ------------------------------------------------------------ learned form
 * Not in the paper: a small MLP proposes, for each candidate facet pair, the
 * order in which to walk the scene's 64 BVH clusters (64 contiguous ranges
 * of the Morton-sorted facets), so that blocked sample segments meet their
 * occluder early.  Inputs: the two facet centroids normalised to the scene
 * box (6), both unit normals (6), and per cluster the entry depth of the
 * centroid segment into the cluster's box (64).  Layers 76 -> 128 -> 128 ->
 * 128 -> 64 with ReLU; inference in BF16 with FP32 accumulation on the
 * tensor cores, training in FP32.  With IVM_MODE_LEARNED and a trained or
 * loaded ranker, ivm_build_matrix walks the top proposals first (while they
 * keep blocking lanes) and then the rest of the tree; every bit is still
 * decided by the same exact facet tests, so results never depend on the
 * weights.  Without weights IVM_MODE_LEARNED behaves as IVM_MODE_FILTERED.
 *
 * Master weights: IVM_RANKER_PARAMS floats, row-major W1[76][128], b1[128],
 * W2[128][128], b2, W3[128][128], b3, W4[128][64], b4[64]. */
#define IVM_RANKER_PARAMS 51136

/* Train the ranker on the given scenes: for every candidate pair whose
 * central-sample segment is blocked, the label is the cluster of the nearest
 * facet it meets (logged by the exact traversal); weights are initialised
 * from a fixed seed and trained by Adam (batch 512) for `epochs` epochs with
 * step `lr`.  *final_loss (may be NULL) receives the mean cross-entropy of the
 * last epoch.  Errors: as ivm_build_matrix; IVM_ERR_ARG if no pair is
 * labelled. */
int ivm_ranker_train(ivm_ctx *ctx, const ivm_scene *scenes, int32_t n_scenes,
                     const ivm_params *params, int32_t epochs, float lr, float *final_loss);

/* Serialise the ranker (header + master weights).  blob NULL: *bytes gets the
 * size.  Errors: IVM_ERR_ARG (no ranker, or *bytes too small). */
int ivm_ranker_save(ivm_ctx *ctx, void *blob, size_t *bytes);

/* Load a ranker saved by ivm_ranker_save.  Errors: IVM_ERR_ARG (bad blob). */
int ivm_ranker_load(ivm_ctx *ctx, const void *blob, size_t bytes);

/* Run the loaded ranker's inference kernel (BF16 tensor cores, FP32
 * accumulation) on feature rows x [batch][76] (host): logits [batch][64] and
 * top [batch][8], the eight highest-scoring clusters per row in order (ties
 * to the lower index); either output may be NULL.  For checking the kernel.
 * Errors: IVM_ERR_ARG (no ranker, batch < 1, both outputs NULL). */
int ivm_ranker_infer(ivm_ctx *ctx, const float *x, int32_t batch, float *logits, uint8_t *top);

/* Mean softmax cross-entropy of a batch and its gradient with respect to the
 * master weights, computed by the training kernels (host pointers): weights
 * [IVM_RANKER_PARAMS], x [batch][76], y [batch] (0..63), grads
 * [IVM_RANKER_PARAMS].  For checking the training kernels. */
int ivm_ranker_gradients(ivm_ctx *ctx, const float *weights, const float *x, const int32_t *y,
                         int32_t batch, float *grads, float *loss);

/* Autotuner for the batched / persistent form (not in the paper: a launch
 * schedule choice).  Times candidate launch shapes on a sample of the given
 * workload -- the first 8 scenes at most and the first 16,384 snapshots of
 * each -- with params' samples_per_side, mode and flags (graph replay is
 * switched off while timing), and writes the fastest warps_per_block, tile,
 * table_tile and proof_tile into *params, and sets or clears
 * IVM_FLAG_NO_CORNER_PROOF in params->flags (the other flags are kept).  Inputs as for ivm_build_table (host or
 * device; tx, rx, n_snap may be NULL to tune the matrix only).  The outputs
 * of the trial runs go to the context's scratch.  Errors: as
 * ivm_build_table. */
int ivm_autotune(ivm_ctx *ctx, const ivm_scene *scenes, int32_t n_scenes,
                 const int32_t *const *tx, const int32_t *const *rx, const int64_t *n_snap,
                 ivm_params *params);

/* Message for an error code (static string). */
const char *ivm_strerror(int code);

/* Matrix build that allocates no memory (the paper has no counterpart).
 * For callers that cannot allocate device memory during the call: code
 * running inside an allocator or memory pool that forbids cudaMalloc,
 * real-time loops that must not take the allocator's synchronisation, hosts
 * that own all device memory.  Computes the same matrix as ivm_build_matrix
 * for one scene, without a context: every scratch buffer lives in one fixed
 * device array of the library (about 5 MB, held on every GPU that loads the
 * library until the process exits).
 *   facets  device pointer, n_facets records (1..IVM_NOALLOC_MAX_FACETS);
 *   params  samples_per_side 1..IVM_NOALLOC_MAX_SAMPLES_PER_SIDE; mode
 *           IVM_MODE_EXACT or IVM_MODE_FILTERED (there is no ranker without a
 *           context, so IVM_MODE_LEARNED is refused); the PERSISTENT and
 *           OCCLUDER_CACHE flags, warps_per_block and tile as for
 *           ivm_build_matrix (0 = default); IVM_FLAG_GRAPH and
 *           IVM_FLAG_DEDUP_SOURCES have no effect here;
 *   matrix  device pointer, [n_facets][W] words, written as ivm_build_matrix;
 *   cuda_stream  cudaStream_t of the current device (NULL: legacy stream).
 * facets and matrix must be memory of the current device (or managed
 * memory); anything else is refused with IVM_ERR_ARG before any work is
 * enqueued.  Runs on the current device.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) and keeps it for the
 * life of the process; make that first call before any stream capture, and
 * do not call the entry point on a device after cudaDeviceReset of that
 * device (the kept address is stale then).  Calls share the array: each
 * call clears what must start at zero, and calls that overlap on the GPU
 * race on it.  It synchronises the stream before returning.  Errors:
 * IVM_ERR_ARG (null or non-device pointer, learned mode, n_facets /
 * samples_per_side above the limits), IVM_ERR_RANGE, IVM_ERR_TIMEOUT,
 * IVM_ERR_INTERNAL, IVM_ERR_CUDA. */
#define IVM_NOALLOC_MAX_FACETS 1024
#define IVM_NOALLOC_MAX_SAMPLES_PER_SIDE 5
int ivm_build_matrix_noalloc(const ivm_facet *facets, int32_t n_facets, const ivm_params *params,
                             uint32_t *matrix, void *cuda_stream);

/* Diagnostic, not from the paper: number of CUDA kernels this library has
 * launched in this process so far (all contexts and threads).  Lets a caller
 * count the launches of a timed region without a profiler. */
uint64_t ivm_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* IVM_H */
