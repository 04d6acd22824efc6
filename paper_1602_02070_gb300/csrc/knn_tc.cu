// knn_tc.cu - tensor-core candidate pass for the kNN graph (placeholder:
// reports "not handled" so the SIMT pass runs).
#include "knn_internal.cuh"

namespace cpca {

cpca_status knn_candidates_tc(const float*, int, int, int64_t, int, int, const float*, int32_t*,
                              float*, bool* done, cudaStream_t) {
  *done = false;
  return CPCA_OK;
}
float knn_tc_err_rel(int) { return 0.f; }

}  // namespace cpca
