// rays.cuh -- arguments and launcher of the ray validation (rays.cu).
#pragma once

#include "ivm_internal.cuh"

namespace ivm {

constexpr int kRayMaxOrder = 8;

struct RayArgs {
    const int *tx, *rx;     // [n_snap][3] cm, device
    long long n_snap;
    const int *paths;       // [n_paths][max_order + 2]: t, k, f1..fK (-1 padded)
    long long n_paths;
    int max_order;          // <= kRayMaxOrder
    uint8_t *valid;         // [n_paths]
};

cudaError_t rays_validate(const DevScenes &g, const RayArgs &a, int *err, cudaStream_t st);

}  // namespace ivm
