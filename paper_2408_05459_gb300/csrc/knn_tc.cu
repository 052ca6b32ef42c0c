// tcgen05 BF16 candidate search (filled in by the tensor-core kernel).
#include "common.cuh"

namespace ancka {

bool knn_tc_available() { return false; }

ancka_status knn_candidates_bf16(const PrepOut&, int64_t, float*, int32_t*, cudaStream_t) {
  set_error("BF16 tensor-core contraction is not available in this build");
  return ANCKA_ERR_UNSUPPORTED;
}

}  // namespace ancka
