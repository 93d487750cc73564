// Allocation-free correlate-and-select: omp_correlate_argmax_noalloc.
//
// This is a variant of the FP32 correlation kernel for callers that must not allocate device
// memory: code running under a fixed device-memory budget or inside a framework that owns every
// device allocation (cudaMalloc synchronises the device and can fail at run time), and callers
// that only need one scoring pass and cannot create a handle (omp_create allocates all of a
// solver's workspaces up front).
//
// The only scratch it needs -- one packed (score, ~index) key per signal, merged across atom
// tiles with a 64-bit atomicMax -- lives in a file-scope device array of fixed size that every
// GPU loading this library holds until the process exits. Atom norms are accumulated inside the
// kernel from the same tiles it multiplies, so no prepared dictionary is needed either.
//
// Sharing rules: every call on a device uses the same array. Each call clears the keys it uses
// before scoring, but two calls whose kernels overlap on the GPU (different streams, no
// ordering between them) race on the array and may return each other's results.
#include <mutex>

#include "common.cuh"

namespace ompk {

// The scratch: one key per signal, 512 KiB per GPU for the whole life of the process. Host code
// must not take its address directly (that is a host-side stand-in); the device address comes
// from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned long long g_noalloc_keys[OMP_NOALLOC_MAX_SIGNALS];

namespace {

constexpr int NA_BM = 128, NA_BN = 128, NA_BK = 16, NA_PAD = 4;
constexpr int kMaxDevices = 64;

std::mutex g_setup_mu;
unsigned long long* g_keys_dev[kMaxDevices] = {};

__global__ void na_clear_kernel(unsigned long long* keys, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) keys[b] = 0ull;
}

// C[b, n] = <r_b, a_n> for a 128-signal x 128-atom tile, K (= M) in chunks of 16 through
// double-buffered shared memory; ||a_n||^2 accumulated from the same chunks. The epilogue forms
// |c| / ||a_n|| and merges each signal's best atom (lowest index on ties) with atomicMax.
template <bool VEC>
__global__ void __launch_bounds__(256, 2)
    na_corr_kernel(const float* __restrict__ A, const float* __restrict__ R, int M, int N, int B,
                   unsigned long long* __restrict__ keys) {
  __shared__ __align__(16) float Xs[2][NA_BK][NA_BM + NA_PAD];
  __shared__ __align__(16) float As[2][NA_BK][NA_BN + NA_PAD];
  const int tid = threadIdx.x;
  const int n0 = blockIdx.x * NA_BN;
  const int p0 = blockIdx.y * NA_BM;
  const int lrow = tid >> 2, lk = (tid & 3) * 4;
  bool xv[2], av[2];
  const float* xsrc[2];
  const float* asrc[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int p = p0 + lrow + 64 * i;
    xv[i] = p < B;
    xsrc[i] = R + static_cast<size_t>(xv[i] ? p : 0) * M;
    const int n = n0 + lrow + 64 * i;
    av[i] = n < N;
    asrc[i] = A + static_cast<size_t>(av[i] ? n : 0) * M;
  }
  float4 xr[2], ar[2];
  auto ld4 = [&](const float* row, bool valid, int m) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!valid) return v;
    if (VEC) {
      if (m < M) v = __ldg(reinterpret_cast<const float4*>(row + m));
    } else {
      if (m < M) v.x = __ldg(row + m);
      if (m + 1 < M) v.y = __ldg(row + m + 1);
      if (m + 2 < M) v.z = __ldg(row + m + 2);
      if (m + 3 < M) v.w = __ldg(row + m + 3);
    }
    return v;
  };
  auto gload = [&](int kc) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      xr[i] = ld4(xsrc[i], xv[i], kc + lk);
      ar[i] = ld4(asrc[i], av[i], kc + lk);
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int r = lrow + 64 * i;
      Xs[buf][lk + 0][r] = xr[i].x;
      Xs[buf][lk + 1][r] = xr[i].y;
      Xs[buf][lk + 2][r] = xr[i].z;
      Xs[buf][lk + 3][r] = xr[i].w;
      As[buf][lk + 0][r] = ar[i].x;
      As[buf][lk + 1][r] = ar[i].y;
      As[buf][lk + 2][r] = ar[i].z;
      As[buf][lk + 3][r] = ar[i].w;
    }
  };
  float acc[8][8];
  float nrm[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    nrm[i] = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  }
  const int tx = tid & 15, ty = tid >> 4;
  const int nk = (M + NA_BK - 1) / NA_BK;
  gload(0);
  sstore(0);
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nk) gload((kt + 1) * NA_BK);
#pragma unroll
    for (int kk = 0; kk < NA_BK; ++kk) {
      const float4 x0 = *reinterpret_cast<const float4*>(&Xs[buf][kk][ty * 4]);
      const float4 x1 = *reinterpret_cast<const float4*>(&Xs[buf][kk][64 + ty * 4]);
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][tx * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + tx * 4]);
      const float xf[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
      const float af[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
      for (int j = 0; j < 8; ++j) nrm[j] = fmaf(af[j], af[j], nrm[j]);
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(xf[i], af[j], acc[i][j]);
    }
    if (kt + 1 < nk) sstore(buf ^ 1);
    __syncthreads();
  }
  int ncol[8];
  float inv[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    ncol[j] = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
    inv[j] = nrm[j] > 0.f ? 1.f / sqrtf(nrm[j]) : 0.f;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int prow = p0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    float best = -1.f;
    int bidx = 0x7fffffff;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (ncol[j] < N) {
        const float s = fabsf(acc[i][j]) * inv[j];
        if (s > best) {
          best = s;
          bidx = ncol[j];
        }
      }
    }
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
      if (better(ob, oi, best, bidx)) {
        best = ob;
        bidx = oi;
      }
    }
    if (tx == 0 && prow < B && bidx < N) atomicMax(keys + prow, pack_key(best, bidx));
  }
}

__global__ void na_unpack_kernel(const unsigned long long* keys, int B, int* idx, float* score) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const unsigned long long k = keys[b];
  idx[b] = k ? key_index(k) : -1;
  score[b] = k ? key_score(k) : -1.f;
}

}  // namespace
}  // namespace ompk

using namespace ompk;

extern "C" omp_status omp_correlate_argmax_noalloc(const float* A, const float* R, int64_t M,
                                                   int64_t N, int64_t B, int32_t* idx_out,
                                                   float* score_out, void* stream) {
  if (!A || !R || !idx_out || !score_out) return OMP_ERR_INVALID_ARGUMENT;
  if (M < 1 || M > (1 << 24) || N < 1 || N > (1 << 30) || B < 1 || B > OMP_NOALLOC_MAX_SIGNALS)
    return OMP_ERR_INVALID_ARGUMENT;
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(R) |
       reinterpret_cast<uintptr_t>(idx_out) | reinterpret_cast<uintptr_t>(score_out)) & 3u)
    return OMP_ERR_INVALID_ARGUMENT;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return OMP_ERR_CUDA;
  unsigned long long* keys = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_keys_dev[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_keys) != cudaSuccess || !p) {
        cudaGetLastError();
        return OMP_ERR_CUDA;
      }
      g_keys_dev[dev] = static_cast<unsigned long long*>(p);
    }
    keys = g_keys_dev[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int b = static_cast<int>(B), m = static_cast<int>(M), n = static_cast<int>(N);
  na_clear_kernel<<<(b + 255) / 256, 256, 0, s>>>(keys, b);
  const dim3 grid((n + NA_BN - 1) / NA_BN, (b + NA_BM - 1) / NA_BM);
  const bool vec = (m % 4 == 0) && !((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(R)) & 15u);
  if (vec)
    na_corr_kernel<true><<<grid, 256, 0, s>>>(A, R, m, n, b, keys);
  else
    na_corr_kernel<false><<<grid, 256, 0, s>>>(A, R, m, n, b, keys);
  na_unpack_kernel<<<(b + 255) / 256, 256, 0, s>>>(keys, b, idx_out, score_out);
  return cudaGetLastError() == cudaSuccess ? OMP_OK : OMP_ERR_CUDA;
}
