// tf32_path.cu -- placeholder until the tensor-core path lands.
#include "internal.cuh"
#include "plan.h"

namespace cs {
cs_status run_tf32(const void*, int64_t, cs_prec, void*, void*, char*, const Layout&, int, int, cudaStream_t) {
  return fail(CS_EINVAL, "precision not available in this build");
}
}  // namespace cs
