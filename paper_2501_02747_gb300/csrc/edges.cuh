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

}  // namespace ivm
