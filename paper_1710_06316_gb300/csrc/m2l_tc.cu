// m2l_tc.cu -- list-2 translations (M2L) on the tensor cores (precision mode 1).
#include "internal.cuh"

namespace afmpb {

Err build_m2l_tc(afmpb_t *h) {
  (void)h;
  return make_err(AFMPB_EINVAL, "precision 1 (tensor-core M2L) is not available in this build");
}

Err enqueue_m2l_tc(afmpb_t *h, cudaStream_t s) {
  (void)h;
  (void)s;
  return make_err(AFMPB_EINVAL, "precision 1 (tensor-core M2L) is not available in this build");
}

}  // namespace afmpb
