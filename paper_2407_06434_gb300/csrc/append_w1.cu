// The append/update kernels with one warp per signal (the code is in append.cuh; each warp
// count is a translation unit of its own, so the build compiles them in parallel).
#include "append.cuh"

namespace ompk {

cudaError_t configure_update_w1(const Ws& ws) { return set_attr_w<1>(ws); }

void launch_update_w1(const Ws& ws, int V, int k, int B, int S, float eps, int eps_rel, cudaStream_t s) {
  launch_w<1>(ws, V, k, B, S, eps, eps_rel, s);
}

}  // namespace ompk
