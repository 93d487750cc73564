// Dispatch of the append/update step (the kernels are in append.cuh, compiled per warp count
// in append_w1.cu .. append_w8.cu): shared-memory limits, slots per lane, the launch.
#include "append.cuh"

namespace ompk {

cudaError_t configure_update_kernels(const Ws& ws) {
  if (ws.Mp > 8192 || ws.Smax > 32 * kMaxBlk) return cudaErrorInvalidValue;
  cudaError_t e = configure_update_w1(ws);
  if (e == cudaSuccess) e = configure_update_w2(ws);
  if (e == cudaSuccess) e = configure_update_w4(ws);
  if (e == cudaSuccess) e = configure_update_w8(ws);
  return e;
}

// float4 slots per lane for W warps per signal (a power of two, 0 if more than 8 are needed)
int update_slots(int Mp, int W) {
  const int need = (Mp + 128 * W - 1) / (128 * W);
  int V = 1;
  while (V < need) V <<= 1;
  return V <= 8 ? V : 0;
}

int update_default_warps(int Mp) {
  for (int W = 1; W <= 8; W <<= 1)
    if (update_slots(Mp, W)) return W;
  return 0;
}

void launch_update(const Ws& ws, int k, int B, int S, float eps, int eps_rel, cudaStream_t s) {
  const int W = ws.upd_w;
  const int V = update_slots(ws.Mp, W);
  if (W == 1) launch_update_w1(ws, V, k, B, S, eps, eps_rel, s);
  else if (W == 2) launch_update_w2(ws, V, k, B, S, eps, eps_rel, s);
  else if (W == 4) launch_update_w4(ws, V, k, B, S, eps, eps_rel, s);
  else launch_update_w8(ws, V, k, B, S, eps, eps_rel, s);
}

}  // namespace ompk
