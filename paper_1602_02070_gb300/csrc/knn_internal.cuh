// knn_internal.cuh - interface between the generic kNN pass (knn.cu) and the
// tensor-core candidate pass (knn_tc.cu).
#pragma once
#include <cuda_fp16.h>

#include "common.cuh"

namespace cpca {

// Tensor-core candidate pass on H, the points scaled by hsc[0] (a power of
// two) and rounded to half precision (N x d, row stride ldh halves,
// knn_half_ld(d)); hsc[1] = 1 / hsc[0]^2. Fills cand_i/cand_d ([S][N][M],
// lists sorted by approximate distance, -1/inf padded) and sets *done =
// true, or leaves *done = false when the shapes are not supported (the SIMT
// pass then runs on the FP32 points).
bool knn_tc_supported(int N, int d, int M);
int64_t knn_half_ld(int d);
cpca_status knn_candidates_tc(const __half* H, int N, int d, int64_t ldh, const float* hsc, int M, int S,
                              const float* nrm, int32_t* cand_i, float* cand_d, int* err, bool* done,
                              cudaStream_t st);
size_t knn_tc_smem(int M);
// Relative error bound of the tensor-core distances (times |a|^2 + |b|^2).
float knn_tc_err_rel(int d);
// k-steps (of 64 dimensions) per tensor-core accumulation, 0 for one
// accumulation over all d.
int knn_tc_chunk_ksteps(int d);

}  // namespace cpca
