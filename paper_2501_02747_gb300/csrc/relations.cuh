// relations.cuh -- arguments and launchers of the interface relations (relations.cu).
#pragma once

#include "ivm_internal.cuh"

namespace ivm {

struct RelArgs {
    const uint32_t *M;     // [n][W] matrix bit rows (device)
    int n, W;
    const long long *off;  // [n + 1] exclusive scan of the rows' bit counts
    int *pairs;            // [P][2]
    uint8_t *relation;     // [P]
    double *ranges;        // [P][4][2]
};

cudaError_t relations_count(const uint32_t *M, int n, int W, long long *deg, cudaStream_t st);
cudaError_t relations_write(const DevScenes &g, const RelArgs &a, cudaStream_t st);

}  // namespace ivm
