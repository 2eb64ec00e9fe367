// tree.cuh -- arguments and launchers of the image-tree expansion (tree.cu).
#pragma once

#include "ivm_internal.cuh"

namespace ivm {

struct TreeArgs {
    const uint32_t *matrix;    // [n][W]
    const uint32_t *table;     // [S][2][W]
    const uint8_t *los;        // [S]
    int n, W, K;
    long long S;
    long long *rowptr;         // [n + 1] CSR of the matrix rows
    int *col;                  // [nnz] ascending within each row
    unsigned long long *wt;    // [2][K + 1][n] fingerprint weights h_c(m, f)
    ivm_tree_summary *summary; // [S][K + 1]
};

cudaError_t tree_adjacency(TreeArgs &a, long long *deg, cudaStream_t st);
cudaError_t tree_fill(TreeArgs &a, cudaStream_t st);
cudaError_t tree_tx_runs(TreeArgs &a, long long *flag, long long *excl, long long *bsum,
                         long long *boff, int *run_of, long long *start, cudaStream_t st);
cudaError_t tree_run_chunk(TreeArgs &a, const long long *start, const int *run_of, long long u0,
                           int C, long long t0, long long t1, unsigned long long *xs,
                           cudaStream_t st);
cudaError_t tree_order0(TreeArgs &a, cudaStream_t st);
cudaError_t tree_paths_count(TreeArgs &a, long long items, long long *cnt, cudaStream_t st);
cudaError_t tree_scan(const long long *in, long long n, long long *sums, long long *sums_off,
                      long long *out, cudaStream_t st);
cudaError_t tree_paths_write(TreeArgs &a, long long items, const long long *off, int *out,
                             long long cap, cudaStream_t st);

}  // namespace ivm
