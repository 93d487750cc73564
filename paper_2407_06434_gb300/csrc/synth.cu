// Signal synthesis for generated training data: y_b = sum_j coef[b, j] a_{sup[b, j]} + noise_b.
// This is the input model of the problem statement (Sec. 1), run on the device so that large
// training sets need no host-side matrix products.
#include "common.cuh"

namespace ompk {
namespace {

// one warp per signal, lanes over the signal length
__global__ void __launch_bounds__(256) synth_kernel(const float* __restrict__ A, int M, const int* __restrict__ sup,
                                                    const float* __restrict__ coef, const float* __restrict__ noise,
                                                    int B, int s, float* __restrict__ Y) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (b >= B) return;
  const int* sb = sup + static_cast<size_t>(b) * s;
  const float* cb = coef + static_cast<size_t>(b) * s;
  float* y = Y + static_cast<size_t>(b) * M;
  for (int m = lane; m < M; m += 32) {
    float acc = noise ? noise[static_cast<size_t>(b) * M + m] : 0.f;
    for (int j = 0; j < s; ++j) {
      const int n = sb[j];
      if (n >= 0) acc = fmaf(cb[j], A[static_cast<size_t>(n) * M + m], acc);
    }
    y[m] = acc;
  }
}

}  // namespace
}  // namespace ompk

extern "C" omp_status omp_synthesize_signals(const float* A, int64_t M, int64_t N, const int32_t* sup,
                                             const float* coef, const float* noise, int64_t B, int32_t s,
                                             float* Y_out, void* stream) {
  (void)N;
  if (!A || !sup || !coef || !Y_out || M < 1 || B < 1 || s < 1) return OMP_ERR_INVALID_ARGUMENT;
  ompk::synth_kernel<<<static_cast<unsigned>((B + 7) / 8), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      A, static_cast<int>(M), sup, coef, noise, static_cast<int>(B), s, Y_out);
  return cudaGetLastError() == cudaSuccess ? OMP_OK : OMP_ERR_CUDA;
}
