// Tensor-core correlation (tcgen05): placeholder until the kernel lands.
#include "common.cuh"

namespace ompk {
struct TcPlan {
  int dummy;
};
int tc_pieces(int, int, int, int) { return 1; }
cudaError_t tc_setup(const Ws&, int, TcPlan** plan) {
  *plan = nullptr;
  return cudaErrorNotSupported;
}
void tc_destroy(TcPlan* plan) { delete plan; }
void launch_corr_tc(const Ws&, const TcPlan*, int, int, cudaStream_t) {}
}  // namespace ompk
