// sk_tc.cu -- tensor-core forms (BF16 split-A with tcgen05 / TMEM / TMA).
// Placeholder entry points until the kernels land.
#include "sk_internal.h"

namespace sk {

size_t tc_workspace_bytes(const GemmShape&) { return 0; }

sk_status tc_check(const GemmShape&, const float*, int64_t, const float*, int64_t) {
  return SK_EUNSUPPORTED;
}

cudaError_t tc_sketch(const sk_sketch*, const GemmShape&, const float*, int64_t, float*, int64_t,
                      void*, size_t, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace sk
