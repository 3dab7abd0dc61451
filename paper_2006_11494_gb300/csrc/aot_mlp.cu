// aot_mlp.cu - learned router (placeholder until the MLP kernels land).
#include "aot_internal.cuh"

namespace aot {
aot_status learned_routes(aot_graph* g, cudaStream_t) {
  return g->model ? AOT_ERR_NOT_READY : AOT_ERR_NOT_READY;
}
}  // namespace aot
