// Streaming-read bandwidth probe: the denominator of the update kernel's roofline when the FP32
// dictionary fits in L2 (the kernel's atom-row gathers then come from L2, not HBM).
//
// Every thread reads 16-byte words with ld.global.cg (cached in L2 only, so repeated passes do
// not hit L1) over the caller's buffer, `reps` times, and each block writes one float so the
// loads stay live. With a buffer well inside the 129 MB L2 the time per pass measures the
// L2-to-SM read bandwidth.
#include "common.cuh"

namespace ompk {
namespace {

__global__ void __launch_bounds__(512) l2_read_kernel(const float4* __restrict__ src, size_t n4,
                                                      int reps, float* __restrict__ out) {
  float acc = 0.f;
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  for (int r = 0; r < reps; ++r)
    for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldcg(src + i);
      acc += (v.x + v.y) + (v.z + v.w);
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ float red[16];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) s += red[w];
    out[blockIdx.x] = s;
  }
}

}  // namespace
}  // namespace ompk

extern "C" omp_status omp_read_bandwidth_probe(const void* buf, int64_t bytes, int32_t reps,
                                               float* block_out, int32_t blocks, void* stream) {
  if (!buf || !block_out || bytes < 16 || (bytes & 15) || reps < 1 || blocks < 1 ||
      (reinterpret_cast<uintptr_t>(buf) & 15))
    return OMP_ERR_INVALID_ARGUMENT;
  ompk::l2_read_kernel<<<blocks, 512, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const float4*>(buf), static_cast<size_t>(bytes / 16), reps, block_out);
  return cudaGetLastError() == cudaSuccess ? OMP_OK : OMP_ERR_CUDA;
}
