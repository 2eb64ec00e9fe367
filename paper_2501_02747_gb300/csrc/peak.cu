// peak.cu -- measured FP32 FMA issue rate of this GPU, the denominator of the
// traversal kernels' "alu" roofline (their work is FP32 and integer box and
// facet tests; no contraction, no HBM stream).
//
// Every thread runs eight independent FMA chains (enough to cover the FMA
// latency), a full-occupancy grid of 256-thread blocks on every SM; the rate
// is FMA lane operations per second (FLOP/s is twice this).
#include "ivm_internal.cuh"

namespace ivm {

__global__ void __launch_bounds__(256) k_ffma(float *sink, int iters, float b, float c)
{
    float a0 = threadIdx.x * 1e-3f, a1 = a0 + 1.f, a2 = a0 + 2.f, a3 = a0 + 3.f;
    float a4 = a0 + 4.f, a5 = a0 + 5.f, a6 = a0 + 6.f, a7 = a0 + 7.f;
#pragma unroll 4
    for (int i = 0; i < iters; i++) {
        a0 = fmaf(a0, b, c); a1 = fmaf(a1, b, c); a2 = fmaf(a2, b, c); a3 = fmaf(a3, b, c);
        a4 = fmaf(a4, b, c); a5 = fmaf(a5, b, c); a6 = fmaf(a6, b, c); a7 = fmaf(a7, b, c);
    }
    const float s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
    if (s == -1.f) sink[0] = s;   // never true; keeps the chains alive
}

cudaError_t ffma_peak(int n_sm, float *sink, cudaStream_t st, double *lane_ops_per_s)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ffma, 256, 0);
    const int blocks = n_sm * (per_sm > 0 ? per_sm : 1);
    const int iters = 1 << 15;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 0.f;
    for (int rep = 0; rep < 4; rep++) {   // the first run warms the clocks up
        cudaEventRecord(e0, st);
        k_ffma<<<blocks, 256, 0, st>>>(sink, iters, 0.99999994f, 1e-7f);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    note_launches(4);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double ops = 8.0 * iters * 256.0 * blocks;
    *lane_ops_per_s = best > 0.f ? ops / (best * 1e-3) : 0.0;
    return cudaGetLastError();
}

}  // namespace ivm
