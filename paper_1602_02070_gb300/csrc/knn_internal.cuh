// knn_internal.cuh - interface between the generic kNN pass (knn.cu) and the
// tensor-core candidate pass (knn_tc.cu).
#pragma once
#include "common.cuh"

namespace cpca {

// Tensor-core candidate pass. Fills cand_i/cand_d ([S][N][M], lists sorted
// by approximate distance, -1/inf padded) and sets *done = true, or leaves
// *done = false when the shapes are not supported (the SIMT pass then runs).
cpca_status knn_candidates_tc(const float* P, int N, int d, int64_t ld, int M, int S,
                              const float* nrm, int32_t* cand_i, float* cand_d, int* err, bool* done,
                              cudaStream_t st);
size_t knn_tc_smem(int M);
// Relative error bound of the tensor-core distances (times |a|^2 + |b|^2).
float knn_tc_err_rel(int d);

}  // namespace cpca
