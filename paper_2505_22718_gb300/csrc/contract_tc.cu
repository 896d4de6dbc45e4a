// a3 on the 5th-generation tensor cores (tcgen05): placeholder until the kernels land.
#include "swcl_internal.h"

namespace swcl {

int compute_delta_tc(swcl_ctx* c, int precision) {
  (void)precision;
  return fail(c, SWCL_ERR_UNSUPPORTED, "tensor-core contraction not built yet");
}

int contract_adj_tc(swcl_ctx* c, int precision) {
  (void)precision;
  return fail(c, SWCL_ERR_UNSUPPORTED, "tensor-core contraction not built yet");
}

}  // namespace swcl
