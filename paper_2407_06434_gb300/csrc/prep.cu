// Dictionary preparation (once per A): FP64 column norms (the ||a_n|| of Alg. 1's score, App. A),
// the zero-padded FP32 atom rows used by the update, the optional 24-bit split copy of them for
// the update's q gather, and the quantised copies used by the tensor-core correlation (BF16
// round-to-nearest-even; E4M3 with a per-atom scale amax_n / 448, satfinite
// round-to-nearest-even).
#include "common.cuh"

namespace ompk {

// One warp per atom; grid-stride over atoms. Reads column n of the caller's A (M contiguous
// floats at A + n*M) with coalesced scalar loads, so any M and any 4-byte alignment works.
__global__ void __launch_bounds__(256) prep_kernel(Ws ws, const float* __restrict__ A) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int n = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; n < ws.N; n += warps) {
    const float* a = A + static_cast<size_t>(n) * ws.M;
    float* a32 = ws.A32 + static_cast<size_t>(n) * ws.Mp;
    double s = 0.0;
    float amax = 0.f;
    for (int m = lane; m < ws.Mp; m += 32) {
      const float v = m < ws.M ? a[m] : 0.f;
      a32[m] = v;
      s += static_cast<double>(v) * static_cast<double>(v);
      amax = fmaxf(amax, fabsf(v));
    }
    s = warp_sum(s);
    amax = warp_max(amax);
    if (lane == 0) {
      ws.norm2[n] = s;
      ws.inv_norm[n] = s > 0.0 ? static_cast<float>(1.0 / sqrt(s)) : 0.f;
    }
    if (lane == 0 && ws.escale) {
      const float in = s > 0.0 ? static_cast<float>(1.0 / sqrt(s)) : 0.f;
      ws.escale[n] = ws.prec == OMP_PREC_FP8_E4M3 ? (amax > 0.f ? amax / 448.f : 0.f) * in : in;
    }
    if (ws.A24h) {
      // round to nearest (ties to even) at the 8th bit, then split: the value rebuilt from the two
      // planes is a with its mantissa rounded to 15 bits (relative error <= 2^-16)
      uint16_t* h = ws.A24h + static_cast<size_t>(n) * ws.Mp;
      uint8_t* l = ws.A24l + static_cast<size_t>(n) * ws.Mp;
      for (int m = lane; m < ws.Mp; m += 32) {
        const uint32_t u = __float_as_uint(a32[m]);
        const uint32_t r = u + 0x7Fu + ((u >> 8) & 1u);
        h[m] = static_cast<uint16_t>(r >> 16);
        l[m] = static_cast<uint8_t>(r >> 8);
      }
    }
    // e2: squared norm of the quantisation error of the atom as the correlation sees it (the E4M3
    // code times the atom's scale), for the data-driven score bound of the E4M3 path
    double e2 = 0.0;
    if (ws.prec == OMP_PREC_BF16) {
      __nv_bfloat16* a16 = ws.A16 + static_cast<size_t>(n) * ws.Mp;
      for (int m = lane; m < ws.Mp; m += 32) a16[m] = __float2bfloat16_rn(a32[m]);
    } else if (ws.prec == OMP_PREC_FP8_E4M3) {
      const float inv = amax > 0.f ? 448.f / amax : 0.f;
      const float sa = amax > 0.f ? amax / 448.f : 0.f;
      if (lane == 0) ws.sa[n] = sa;
      uint8_t* a8 = ws.A8 + static_cast<size_t>(n) * ws.Mp;
      for (int m = lane; m < ws.Mp; m += 32) {
        const __nv_fp8_storage_t c = __nv_cvt_float_to_fp8(a32[m] * inv, __NV_SATFINITE, __NV_E4M3);
        a8[m] = static_cast<uint8_t>(c);
        const double d = static_cast<double>(e4m3_to_float(c)) * sa - static_cast<double>(a32[m]);
        e2 += d * d;
      }
    }
    if (ws.ea) {
      e2 = warp_sum(e2);
      if (lane == 0 && s > 0.0) {
        const float rel = static_cast<float>(sqrt(e2 / s)) * (1.f + 0x1p-20f);
        atomicMax(reinterpret_cast<unsigned int*>(ws.ea), __float_as_uint(rel));
      }
    }
  }
}

void launch_prep(const Ws& ws, const float* A, cudaStream_t s) {
  const int blocks = (ws.N + 7) / 8;
  prep_kernel<<<blocks < 65535 ? blocks : 65535, 256, 0, s>>>(ws, A);
}

}  // namespace ompk
