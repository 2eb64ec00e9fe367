// edges.cuh -- arguments and launcher of the edge rows (edges.cu).
#pragma once

#include "ivm_internal.cuh"

namespace ivm {

struct EdgeArgs {
    const int *edges;                 // [ne][6] endpoints, cm (device)
    int ne, WE;                       // edges, words per row
    const int *tx, *rx;               // [S][3] cm (device)
    long long S;
    int tile;                         // snapshots per work item
    long long ntiles;
    uint32_t *table;                  // [S][2][WE]
    unsigned long long *nearest_key;  // [S][2] scratch
    int *nearest;                     // [S][2]
    unsigned long long *ctr;          // test counters
};

cudaError_t edges_table(const DevScenes &g, const EdgeArgs &a, bool filtered, int *err,
                        cudaStream_t st);

// Edges as rows and columns of the matrix (edge_matrix.cu).
struct EdgeMatrixArgs {
    const int *edges;        // [ne][6] endpoints, cm (device)
    const int *faces;        // [ne][2] the two facets meeting at each edge (scene-local)
    int n, ne, WE;           // facets, edges, words per row
    uint32_t *fe;            // [N][WE]: facet rows' edge bits
    uint32_t *ee;            // [ne][WE]: edge rows' edge bits
    int tile;                // pairs per queue pop
    unsigned long long *work;// queue cursor (device)
    unsigned long long *ctr; // test counters
};

cudaError_t edges_matrix(const DevScenes &g, const EdgeMatrixArgs &a, bool filtered, int n_sm,
                         int *err, cudaStream_t st);

}  // namespace ivm
