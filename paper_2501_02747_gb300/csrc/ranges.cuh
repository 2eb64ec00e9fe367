// ranges.cuh -- arguments and launchers of the visibility ranges (ranges.cu).
#pragma once

#include "ivm_internal.cuh"

namespace ivm {

constexpr int kRngChunk = 256;   // snapshots per counting item

struct RangeArgs {
    const uint32_t *table;       // [S][2][W]
    int n, W;
    long long S;
    int nchunks;                 // ceil(S / kRngChunk)
    const int *tx, *rx;          // [S][3] cm, device
    long long *count;            // [2][n][nchunks] starts per (side, facet, chunk)
    long long *off;              // exclusive scan of count, [2 n nchunks + 1]
    ivm_range *rec;              // [R] output records
    unsigned long long *sums;    // [2] summed range lengths per side
};

cudaError_t ranges_count(const RangeArgs &a, cudaStream_t st);
cudaError_t ranges_write(const RangeArgs &a, cudaStream_t st);
cudaError_t ranges_blockers(const DevScenes &g, const RangeArgs &a, long long R, int *err,
                            cudaStream_t st);

}  // namespace ivm
