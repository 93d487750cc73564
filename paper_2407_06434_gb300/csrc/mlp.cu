// Learned proposal network: kernels and the C ABI of the omp_proposal object.
//
// The network maps the first correlation of a signal to per-atom logits:
//   x = (A^T y)_n / (||a_n|| ||y||)              features, BF16 (the first OMP correlation)
//   h = GELU(W1 x + b1)                          W1: hidden x N, exact GELU x Phi(x) via erff
//   o = W2 h + b2 + beta |x|                     W2: N x hidden, beta a learned scalar (skip term:
//                                                the hidden width is far below N, so the
//                                                per-atom magnitude |x_n| enters directly)
// and proposes, per signal, the `topk` atoms with the largest logits (lowest index on ties).
// Training minimises the mean binary cross-entropy with logits against the support that plain
// OMP picked, with a positive-class weight, using AdamW on FP32 master weights.
//
// Every GEMM runs on the tcgen05 mainloop of tcgemm.cuh with BF16 operands and FP32
// accumulation; operands are K-major, so the epilogues also write the transposed copies the
// backward GEMMs need (Xt, Ht, dOt, dZ1t):
//   features  X   = Yq A16^T            (rows: signals, K = Mp)
//   fwd1      H   = GELU(X W1^T + b1)   (K = N)          also Z1 (FP32) and Ht for training
//   fwd2      O   = H W2^T + b2         (K = hidden)     inference: FP32 logits;
//                                                         training: dO = dBCE/dO, and dOt
//   bwd       dH  = dO W2 = dO (W2t)^T  (K = N)          dZ1t = (dH * GELU'(Z1))^T
//   grads     dW2 = dOt (Ht)^T          (K = batch)      dW1 = dZ1t (Xt)^T
//   biases    db2 = row sums of dOt,    db1 = row sums of dZ1t
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "tcgemm.cuh"

namespace ompk {
namespace {

using namespace tcg;

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
  const float cdf = 0.5f * (1.f + erff(x * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
  return cdf + x * pdf;
}
// log(1 + exp(x)) without overflow
__device__ __forceinline__ float softplus_f(float x) { return x > 0.f ? x + log1pf(expf(-x)) : log1pf(expf(x)); }

// ---------------------------------------------------------------------------- epilogues
// value = acc * rowscale[r] * colscale[c] + bias[c], optional GELU; BF16 store (row-major and
// optionally transposed into a matrix with leading dimension ldT) and optional FP32 store of the
// pre-activation.
struct EpiAct {
  int rows, cols, ldT, gelu;
  const float* rowscale;
  const float* colscale;
  const float* bias;
  float* pre;
  __nv_bfloat16* out;
  __nv_bfloat16* outT;
  int row;
  __device__ void begin(int, int, int, int row_, int, float*, unsigned long long*) { row = row_; }
  __device__ void unit(int, int) {}
  __device__ void chunk(int s, int t, int c0, const uint32_t (&v)[32]) {
    const int r = s * BM + row;
    const int cb = t * BN + c0;
    const bool rok = r < rows;
    const float rs = (rok && rowscale) ? rowscale[r] : 1.f;
    uint32_t ow[16];  // the 32 BF16 results, two per word (kept in registers)
#pragma unroll
    for (int j = 0; j < 32; j += 2) {
      float y2[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int c = cb + j + e;
        float x = __uint_as_float(v[j + e]) * rs;
        if (c < cols) {
          if (colscale) x *= __ldg(colscale + c);
          if (bias) x += __ldg(bias + c);
        }
        if (rok && c < cols && pre) pre[static_cast<size_t>(r) * cols + c] = x;
        y2[e] = gelu ? gelu_f(x) : x;
        if (outT && c < cols && rok) outT[static_cast<size_t>(c) * ldT + r] = __float2bfloat16_rn(y2[e]);
      }
      const __nv_bfloat162 h = __floats2bfloat162_rn(y2[0], y2[1]);
      ow[j >> 1] = *reinterpret_cast<const uint32_t*>(&h);
    }
    if (!rok) return;
    __nv_bfloat16* dst = out + static_cast<size_t>(r) * cols + cb;
    if (cb + 32 <= cols && (cols & 7) == 0) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        reinterpret_cast<uint4*>(dst)[q] = make_uint4(ow[4 * q], ow[4 * q + 1], ow[4 * q + 2], ow[4 * q + 3]);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (cb + j < cols) dst[j] = __ushort_as_bfloat16(static_cast<unsigned short>((j & 1) ? (ow[j >> 1] >> 16) : (ow[j >> 1] & 0xFFFFu)));
    }
  }
  __device__ void end(bool) {}
};

// FP32 store of acc (+ bias): logits at inference, weight gradients in training.
struct EpiF32 {
  int rows, cols;
  const float* bias;
  const __nv_bfloat16* skipX;  // optional skip term beta * |x| (x: rows x cols features)
  const float* beta;
  float* out;
  int row;
  __device__ void begin(int, int, int, int row_, int, float*, unsigned long long*) { row = row_; }
  __device__ void unit(int, int) {}
  __device__ float val(const uint32_t (&v)[32], int j, int r, int c, float bt) const {
    float o = __uint_as_float(v[j]) + (bias ? __ldg(bias + c) : 0.f);
    if (skipX) o = fmaf(bt, fabsf(__bfloat162float(skipX[static_cast<size_t>(r) * cols + c])), o);
    return o;
  }
  __device__ void chunk(int s, int t, int c0, const uint32_t (&v)[32]) {
    const int r = s * BM + row;
    if (r >= rows) return;
    const int cb = t * BN + c0;
    const float bt = skipX ? *beta : 0.f;
    float* dst = out + static_cast<size_t>(r) * cols + cb;
    if (cb + 32 <= cols && (cols & 7) == 0) {
      // the row's 32 skip features in four 16-byte loads (cols a multiple of 8 keeps them
      // aligned), the bias once per column
      uint32_t xw[16];  // 32 BF16 values, two per word (a BF16 is the top half of an FP32)
      if (skipX) {
        const uint4* src = reinterpret_cast<const uint4*>(skipX + static_cast<size_t>(r) * cols + cb);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint4 u = __ldg(src + q);
          xw[4 * q] = u.x;
          xw[4 * q + 1] = u.y;
          xw[4 * q + 2] = u.z;
          xw[4 * q + 3] = u.w;
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float ov[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = 4 * q + e;
          float o = __uint_as_float(v[j]) + (bias ? __ldg(bias + cb + j) : 0.f);
          if (skipX) {
            const uint32_t wd = xw[j >> 1];
            const float xf = __uint_as_float((j & 1) ? (wd & 0xFFFF0000u) : (wd << 16));
            o = fmaf(bt, fabsf(xf), o);
          }
          ov[e] = o;
        }
        reinterpret_cast<float4*>(dst)[q] = make_float4(ov[0], ov[1], ov[2], ov[3]);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (cb + j < cols) dst[j] = val(v, j, r, cb + j, bt);
    }
  }
  __device__ void end(bool) {}
};

// Gradient of the mean weighted BCE with logits o = acc + b2 and labels from a bit matrix
// (row r, column c at bit c % 32 of word r * (cols / 32) + c / 32):
//   loss = pw y softplus(-o) + (1 - y) softplus(o),  dloss/do = sigma(o) (1 - y + pw y) - pw y,
// both divided by rows * cols. Stores dO (row-major) and dOt (transposed, leading dim ldT) in
// BF16 and adds the loss to *loss.
struct EpiBCE {
  int rows, cols, ldT;
  float pos_weight, inv_count;
  const float* bias;
  const uint32_t* labels;
  const __nv_bfloat16* skipX;  // features x: the logit has the skip term beta * |x|
  const float* beta;
  float* dbeta;                // accumulates sum dO * |x|
  __nv_bfloat16* dO;
  __nv_bfloat16* dOT;
  float* loss;
  int row;
  float lsum, bsum;
  __device__ void begin(int, int, int, int row_, int, float*, unsigned long long*) {
    row = row_;
    lsum = 0.f;
    bsum = 0.f;
  }
  __device__ void unit(int, int) {}
  __device__ void chunk(int s, int t, int c0, const uint32_t (&v)[32]) {
    const int r = s * BM + row;
    const bool rok = r < rows;
    const int cb = t * BN + c0;
    const uint32_t bits = (rok && cb < cols) ? labels[static_cast<size_t>(r) * (cols >> 5) + (cb >> 5)] : 0u;
    const float bt = *beta;
    uint32_t ow[16];  // the 32 BF16 gradients, two per word (kept in registers)
#pragma unroll
    for (int j = 0; j < 32; j += 2) {
      float g2[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int c = cb + j + e;
        const bool ok = rok && c < cols;
        const float ax = ok ? fabsf(__bfloat162float(skipX[static_cast<size_t>(r) * cols + c])) : 0.f;
        const float o = fmaf(bt, ax, __uint_as_float(v[j + e]) + (c < cols ? __ldg(bias + c) : 0.f));
        const float y = ((bits >> (j + e)) & 1u) ? 1.f : 0.f;
        const float sg = 1.f / (1.f + expf(-o));
        const float g = (sg * (1.f - y + pos_weight * y) - pos_weight * y) * inv_count;
        if (ok) {
          lsum += (pos_weight * y * softplus_f(-o) + (1.f - y) * softplus_f(o)) * inv_count;
          bsum = fmaf(g, ax, bsum);
        }
        g2[e] = ok ? g : 0.f;
        if (ok) dOT[static_cast<size_t>(c) * ldT + r] = __float2bfloat16_rn(g2[e]);
      }
      const __nv_bfloat162 h = __floats2bfloat162_rn(g2[0], g2[1]);
      ow[j >> 1] = *reinterpret_cast<const uint32_t*>(&h);
    }
    if (!rok) return;
    __nv_bfloat16* dst = dO + static_cast<size_t>(r) * cols + cb;
    if (cb + 32 <= cols) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        reinterpret_cast<uint4*>(dst)[q] = make_uint4(ow[4 * q], ow[4 * q + 1], ow[4 * q + 2], ow[4 * q + 3]);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (cb + j < cols) dst[j] = __ushort_as_bfloat16(static_cast<unsigned short>((j & 1) ? (ow[j >> 1] >> 16) : (ow[j >> 1] & 0xFFFFu)));
    }
  }
  __device__ void end(bool) {
    float v = lsum, w = bsum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v += __shfl_xor_sync(0xffffffffu, v, o);
      w += __shfl_xor_sync(0xffffffffu, w, o);
    }
    if ((threadIdx.x & 31) == 0) {
      if (loss) atomicAdd(loss, v);
      atomicAdd(dbeta, w);
    }
  }
};

// dZ1 = dH * GELU'(Z1), stored transposed (hidden x batch, leading dim ldT) in BF16.
struct EpiGeluBwd {
  int rows, cols, ldT;
  const float* Z1;
  __nv_bfloat16* dZT;
  int row;
  __device__ void begin(int, int, int, int row_, int, float*, unsigned long long*) { row = row_; }
  __device__ void unit(int, int) {}
  __device__ void chunk(int s, int t, int c0, const uint32_t (&v)[32]) {
    const int r = s * BM + row;
    if (r >= rows) return;
    const int cb = t * BN + c0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int c = cb + j;
      if (c < cols) {
        const float z = Z1[static_cast<size_t>(r) * cols + c];
        dZT[static_cast<size_t>(c) * ldT + r] = __float2bfloat16_rn(__uint_as_float(v[j]) * gelu_grad_f(z));
      }
    }
  }
  __device__ void end(bool) {}
};

template <class Epi>
__global__ void __launch_bounds__(THREADS, 1)
    mlp_gemm_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                    int rows, int cols, int K, unsigned int* err, Epi epi) {
  gemm_body<OMP_PREC_BF16>(&ta, &tb, (rows + BM - 1) / BM, (cols + BN - 1) / BN, K / 64, 1, err, epi);
}

// ------------------------------------------------------------------------ small kernels
// Feature input: y in BF16 (zero padded to Mp) and 1/||y|| (0 for y == 0 or non-finite y).
__global__ void __launch_bounds__(256) feat_prep_kernel(const float* __restrict__ Y, int M, int Mp, int B,
                                                        __nv_bfloat16* Yq, float* inv_ynorm, float* ynorm) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (b >= B) return;
  const float* y = Y + static_cast<size_t>(b) * M;
  double s = 0.0;
  bool finite = true;
  for (int m = lane; m < Mp; m += 32) {
    const float v = m < M ? y[m] : 0.f;
    finite = finite && isfinite(v);
    s += static_cast<double>(v) * v;
  }
  s = warp_sum(s);
  finite = __all_sync(0xffffffffu, finite);
  __nv_bfloat16* q = Yq + static_cast<size_t>(b) * Mp;
  for (int m = lane; m < Mp; m += 32) q[m] = __float2bfloat16_rn((finite && m < M) ? y[m] : 0.f);
  if (lane == 0) {
    const bool ok = finite && s > 0.0;
    inv_ynorm[b] = ok ? static_cast<float>(1.0 / sqrt(s)) : 0.f;
    if (ynorm) ynorm[b] = ok ? static_cast<float>(sqrt(s)) : 0.f;
  }
}

// Label bit matrix from supports (B x S, -1 padded): bit c of row b is set if c is in the row.
__global__ void labels_kernel(const int* __restrict__ sup, int B, int S, int N, uint32_t* bits) {
  const int b = blockIdx.x;
  uint32_t* row = bits + static_cast<size_t>(b) * (N >> 5);
  for (int w = threadIdx.x; w < (N >> 5); w += blockDim.x) row[w] = 0u;
  __syncthreads();
  for (int j = threadIdx.x; j < S; j += blockDim.x) {
    const int c = sup[static_cast<size_t>(b) * S + j];
    if (c >= 0 && c < N) atomicOr(row + (c >> 5), 1u << (c & 31));
  }
}

// out[i] = sum_j in[i * ld + j], j < n (one warp per row, FP32 accumulation)
__global__ void row_sum_kernel(const __nv_bfloat16* __restrict__ in, int rows, int n, int ld, float* out) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= rows) return;
  const __nv_bfloat16* p = in + static_cast<size_t>(r) * ld;
  float s = 0.f;
  for (int j = lane; j < n; j += 32) s += __bfloat162float(p[j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[r] = s;
}

struct AdamParams {
  float lr, beta1, beta2, eps, wd, c1, c2;  // c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t)
};

// AdamW step on FP32 master weights; also writes the BF16 copy (if given).
__global__ void adamw_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                             const float* __restrict__ g, size_t n, AdamParams a, __nv_bfloat16* wb) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = a.beta1 * m[i] + (1.f - a.beta1) * gi;
    const float vi = a.beta2 * v[i] + (1.f - a.beta2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float upd = (mi * a.c1) / (sqrtf(vi * a.c2) + a.eps) + a.wd * w[i];
    const float wi = w[i] - a.lr * upd;
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16_rn(wi);
  }
}

__global__ void abs_bf16_kernel(const __nv_bfloat16* __restrict__ x, size_t n, float* out) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    out[i] = fabsf(__bfloat162float(x[i]));
}

__global__ void to_bf16_kernel(const float* __restrict__ w, size_t n, __nv_bfloat16* wb) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    wb[i] = __float2bfloat16_rn(w[i]);
}

// out (cols x rows, BF16) = transpose of in (rows x cols, FP32), 32 x 32 tiles through smem
__global__ void transpose_bf16_kernel(const float* __restrict__ in, int rows, int cols, __nv_bfloat16* out) {
  __shared__ float tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? in[static_cast<size_t>(r) * cols + c] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows) out[static_cast<size_t>(c) * rows + r] = __float2bfloat16_rn(tile[threadIdx.x][i]);
  }
}

// Per row of logits (N values): the K largest, lowest index first among equal values, written
// in ascending index order. One 256-thread block per row: a bitwise search over the
// order-preserving integer image of the floats finds the K-th largest value t, then every
// element > t is kept and the elements == t fill the remaining slots in index order.
__device__ __forceinline__ uint32_t orderable(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// SMEM: the row's orderable keys are staged in dynamic shared memory once (N x 4 bytes), so the 33
// counting passes read shared memory instead of the row in global memory.
template <bool SMEM>
__global__ void __launch_bounds__(256) topk_rows_kernel(const float* __restrict__ logits, int N, int K,
                                                         int* __restrict__ out) {
  __shared__ int red[8];
  __shared__ int wcnt_gt[8], wcnt_eq[8];
  extern __shared__ uint32_t keys_s[];
  const int row = blockIdx.x;
  const float* x = logits + static_cast<size_t>(row) * N;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (SMEM) {
    for (int i = tid; i < N; i += 256) keys_s[i] = orderable(x[i]);
    __syncthreads();
  }
  auto key = [&](int i) -> uint32_t { return SMEM ? keys_s[i] : orderable(x[i]); };
  // T = the K-th largest key: the largest threshold with count(key >= T) >= K
  uint32_t T = 0;
  if (SMEM) {
    // radix select, 8 bits a pass from the top: a 256-bin histogram of the keys that share the
    // bits fixed so far (warp-aggregated shared-memory atomics), then the bin that holds the
    // K-th largest of them
    __shared__ int hist[256];
    __shared__ uint32_t sel_s[2];  // the bin found, the rank still to find within it
    uint32_t fixed = 0;            // mask of the bits of T fixed so far
    int rem = K;
    for (int shift = 24; shift >= 0; shift -= 8) {
      hist[tid] = 0;
      __syncthreads();
      for (int i0 = 0; i0 < N; i0 += 256) {
        const int i = i0 + tid;
        const uint32_t kv = i < N ? keys_s[i] : 0u;
        const bool in = i < N && (kv & fixed) == T;
        const int bin = in ? static_cast<int>((kv >> shift) & 255u) : 256;
        const unsigned same = __match_any_sync(0xffffffffu, bin);
        if (in && lane == __ffs(same) - 1) atomicAdd(&hist[bin], __popc(same));
      }
      __syncthreads();
      if (warp == 0) {
        // lane l owns bins 8l .. 8l + 7; counts above a bin come from the higher lanes
        int cnt[8], tot = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          cnt[j] = hist[8 * lane + j];
          tot += cnt[j];
        }
        int above = 0;  // keys in the bins of the lanes above this one
        for (int l2 = 31; l2 > 0; --l2) {
          const int t2 = __shfl_sync(0xffffffffu, tot, l2);
          if (l2 > lane) above += t2;
        }
#pragma unroll
        for (int j = 7; j >= 0; --j) {
          if (above < rem && above + cnt[j] >= rem) {
            sel_s[0] = static_cast<uint32_t>(8 * lane + j);
            sel_s[1] = static_cast<uint32_t>(rem - above);
          }
          above += cnt[j];
        }
      }
      __syncthreads();
      T |= sel_s[0] << shift;
      fixed |= 255u << shift;
      rem = static_cast<int>(sel_s[1]);
      __syncthreads();
    }
  } else {
    // bitwise search over the row in global memory
    for (int bit = 31; bit >= 0; --bit) {
      const uint32_t cand = T | (1u << bit);
      int c = 0;
      for (int i = tid; i < N; i += 256) c += key(i) >= cand ? 1 : 0;
      c = warp_sum_int(c);
      if (lane == 0) red[warp] = c;
      __syncthreads();
      int tot = 0;
#pragma unroll
      for (int w = 0; w < 8; ++w) tot += red[w];
      __syncthreads();
      if (tot >= K) T = cand;
    }
  }
  // Output: the > T elements and the first K - count(> T) elements == T, in index order. Each
  // warp owns a contiguous index range: one pass counts its > T and == T elements, one barrier
  // gives every warp the counts of the ranges before it, and each warp then writes its selected
  // indices in order (ballots within the warp, no further barriers).
  const int per = (N + 7) / 8;
  const int lo = min(N, warp * per), hi = min(N, lo + per);
  int cg = 0, ce = 0;
  for (int i = lo + lane; i < hi; i += 32) {
    const uint32_t kv = key(i);
    cg += kv > T ? 1 : 0;
    ce += kv == T ? 1 : 0;
  }
  cg = warp_sum_int(cg);
  ce = warp_sum_int(ce);
  if (lane == 0) {
    wcnt_gt[warp] = cg;
    wcnt_eq[warp] = ce;
  }
  __syncthreads();
  int total_gt = 0, base_gt = 0, base_eq = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    total_gt += wcnt_gt[w];
    if (w < warp) {
      base_gt += wcnt_gt[w];
      base_eq += wcnt_eq[w];
    }
  }
  const int need_eq = K - total_gt;
  int* o = out + static_cast<size_t>(row) * K;
  const unsigned below = (1u << lane) - 1u;
  for (int i0 = lo; i0 < hi; i0 += 32) {
    const int i = i0 + lane;
    const uint32_t kv = i < hi ? key(i) : 0u;
    const bool gt = i < hi && kv > T;
    const bool eq = i < hi && kv == T;
    const unsigned mg = __ballot_sync(0xffffffffu, gt);
    const unsigned me = __ballot_sync(0xffffffffu, eq);
    const int rg = base_gt + __popc(mg & below);
    const int re = base_eq + __popc(me & below);
    if (gt || (eq && re < need_eq)) {
      const int slot = rg + min(re, need_eq);
      if (slot < K) o[slot] = i;
    }
    base_gt += __popc(mg);
    base_eq += __popc(me);
  }
}

// The rows' K largest entries (see topk_rows_kernel); shared-memory keys when a row fits.
bool launch_topk_rows(const float* logits, int rows, int N, int K, int* out, cudaStream_t s) {
  const size_t bytes = static_cast<size_t>(N) * 4;
  if (bytes <= 160 * 1024 &&
      raise_smem_limit(reinterpret_cast<const void*>(topk_rows_kernel<true>), bytes) == cudaSuccess) {
    topk_rows_kernel<true><<<rows, 256, bytes, s>>>(logits, N, K, out);
  } else {
    cudaGetLastError();
    topk_rows_kernel<false><<<rows, 256, 0, s>>>(logits, N, K, out);
  }
  return cudaGetLastError() == cudaSuccess;
}

// tau[k] = the q-quantile (the floor(q * n)-th smallest, 0-based) of the positive entries of
// column k of a B x S matrix; 0 if the column has none. One block per column; a bitwise search
// over the IEEE bits of the (positive) values.
__global__ void __launch_bounds__(256) quantile_cols_kernel(const float* __restrict__ v, int B, int S, float q,
                                                            float* __restrict__ tau) {
  __shared__ int red[8];
  const int k = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  auto block_count = [&](auto pred) {
    int c = 0;
    for (int b = tid; b < B; b += 256) {
      const float x = v[static_cast<size_t>(b) * S + k];
      c += (x > 0.f && pred(__float_as_uint(x))) ? 1 : 0;
    }
    c = warp_sum_int(c);
    if (lane == 0) red[warp] = c;
    __syncthreads();
    int t = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w];
    __syncthreads();
    return t;
  };
  const int n = block_count([](uint32_t) { return true; });
  if (n == 0) {
    if (tid == 0) tau[k] = 0.f;
    return;
  }
  int m = static_cast<int>(q * static_cast<float>(n));
  if (m > n - 1) m = n - 1;
  uint32_t T = 0;
  for (int bit = 30; bit >= 0; --bit) {
    const uint32_t cand = T | (1u << bit);
    const int below = block_count([cand](uint32_t u) { return u < cand; });
    if (below <= m) T = cand;
  }
  if (tid == 0) tau[k] = __uint_as_float(T);
}

}  // namespace
}  // namespace ompk

// =============================================================================== C ABI
using namespace ompk;

struct omp_proposal_s {
  omp_proposal_desc d{};
  int dev = 0;
  int N = 0, M = 0, Mp = 0, H = 0, Bi = 0, Bt = 0;
  int grid = 0;
  long long step = 0;
  std::vector<void*> allocs;
  // parameters (FP32 masters, Adam moments, BF16 copies)
  float *W1 = nullptr, *b1 = nullptr, *W2 = nullptr, *b2 = nullptr;
  float *beta = nullptr, *mbeta = nullptr, *vbeta = nullptr, *dbeta = nullptr;  // skip-term scale
  float *mW1 = nullptr, *vW1 = nullptr, *mb1 = nullptr, *vb1 = nullptr;
  float *mW2 = nullptr, *vW2 = nullptr, *mb2 = nullptr, *vb2 = nullptr;
  __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W2Tb = nullptr;
  // dictionary copy (BF16) and scales used by the feature GEMM
  __nv_bfloat16* A16 = nullptr;
  float* escale = nullptr;
  const float* prepared_A = nullptr;
  // activations
  __nv_bfloat16 *Yq = nullptr, *X = nullptr, *XT = nullptr, *Hh = nullptr, *HT = nullptr;
  float *inv_yn = nullptr, *Z1 = nullptr, *logits = nullptr;
  __nv_bfloat16 *dO = nullptr, *dOT = nullptr, *dZT = nullptr;
  float *dW1 = nullptr, *db1 = nullptr, *dW2 = nullptr, *db2 = nullptr;
  uint32_t* labels = nullptr;
  float* loss = nullptr;
  float* tau = nullptr;
  int* cand = nullptr;
  int Smax_tau = 0;
  unsigned int* err = nullptr;
};

namespace ompk {
namespace mlpd {

using namespace tcg;

template <class T>
bool palloc(omp_proposal_s* p, T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) return true;
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  p->allocs.push_back(q);
  *ptr = static_cast<T*>(q);
  return true;
}

void pfree(omp_proposal_s* p) {
  for (void* q : p->allocs) cudaFree(q);
  p->allocs.clear();
}

int blocks_for(size_t n) {
  const size_t b = (n + 255) / 256;
  return static_cast<int>(b < 4096 ? b : 4096);
}

template <class Epi>
bool gemm(const omp_proposal_s* p, const void* a, int a_rows, const void* b, int b_rows, int K,
          const Epi& epi, cudaStream_t s, int ld = 0) {
  CUtensorMap ta, tb;
  if (!make_kmajor_map(&ta, a, OMP_PREC_BF16, a_rows, K, BM, ld) ||
      !make_kmajor_map(&tb, b, OMP_PREC_BF16, b_rows, K, BN, ld))
    return false;
  static bool attr_done = false;  // per epilogue type
  if (!attr_done) {
    if (set_smem_attr(reinterpret_cast<const void*>(mlp_gemm_kernel<Epi>)) != cudaSuccess) return false;
    attr_done = true;
  }
  mlp_gemm_kernel<Epi><<<p->grid, THREADS, SMEM_BYTES, s>>>(ta, tb, a_rows, b_rows, K, p->err, epi);
  return cudaGetLastError() == cudaSuccess;
}

// Dictionary copy for the feature GEMM: BF16 rows zero-padded to Mp and escale = 1/||a_n||.
__global__ void dict_bf16_kernel(const float* __restrict__ A, int M, int Mp, int N, __nv_bfloat16* A16,
                                 float* escale) {
  const int lane = threadIdx.x & 31;
  const int n = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (n >= N) return;
  const float* a = A + static_cast<size_t>(n) * M;
  double s = 0.0;
  for (int m = lane; m < Mp; m += 32) {
    const float v = m < M ? a[m] : 0.f;
    A16[static_cast<size_t>(n) * Mp + m] = __float2bfloat16_rn(v);
    s += static_cast<double>(v) * v;
  }
  s = warp_sum(s);
  if (lane == 0) escale[n] = s > 0.0 ? static_cast<float>(1.0 / sqrt(s)) : 0.f;
}

bool features(omp_proposal_s* p, const float* A, const float* Y, int B, bool transposed,
              cudaStream_t s) {
  if (A != p->prepared_A) {
    dict_bf16_kernel<<<(p->N + 7) / 8, 256, 0, s>>>(A, p->M, p->Mp, p->N, p->A16, p->escale);
    p->prepared_A = A;
  }
  feat_prep_kernel<<<(B + 7) / 8, 256, 0, s>>>(Y, p->M, p->Mp, B, p->Yq, p->inv_yn, nullptr);
  EpiAct e{};
  e.rows = B;
  e.cols = p->N;
  e.ldT = p->Bt;
  e.gelu = 0;
  e.rowscale = p->inv_yn;
  e.colscale = p->escale;
  e.out = p->X;
  e.outT = transposed ? p->XT : nullptr;
  return gemm(p, p->Yq, B, p->A16, p->N, p->Mp, e, s);
}

bool forward_hidden(omp_proposal_s* p, int B, bool training, cudaStream_t s) {
  EpiAct e{};
  e.rows = B;
  e.cols = p->H;
  e.ldT = p->Bt;
  e.gelu = 1;
  e.bias = p->b1;
  e.pre = training ? p->Z1 : nullptr;
  e.out = p->Hh;
  e.outT = training ? p->HT : nullptr;
  return gemm(p, p->X, B, p->W1b, p->H, p->N, e, s);
}

bool gradients(omp_proposal_s* p, const float* A, const float* Y, const int* labels_sup, int B, int S,
               cudaStream_t s) {
  if (!features(p, A, Y, B, true, s)) return false;
  if (!forward_hidden(p, B, true, s)) return false;
  labels_kernel<<<B, 256, 0, s>>>(labels_sup, B, S, p->N, p->labels);
  cudaMemsetAsync(p->loss, 0, sizeof(float), s);
  cudaMemsetAsync(p->dbeta, 0, sizeof(float), s);
  EpiBCE eb{};
  eb.skipX = p->X;
  eb.beta = p->beta;
  eb.dbeta = p->dbeta;
  eb.rows = B;
  eb.cols = p->N;
  eb.ldT = p->Bt;
  eb.pos_weight = p->d.pos_weight;
  eb.inv_count = 1.f / (static_cast<float>(B) * static_cast<float>(p->N));
  eb.bias = p->b2;
  eb.labels = p->labels;
  eb.dO = p->dO;
  eb.dOT = p->dOT;
  eb.loss = p->loss;
  if (!gemm(p, p->Hh, B, p->W2b, p->N, p->H, eb, s)) return false;
  EpiGeluBwd eg{};
  eg.rows = B;
  eg.cols = p->H;
  eg.ldT = p->Bt;
  eg.Z1 = p->Z1;
  eg.dZT = p->dZT;
  if (!gemm(p, p->dO, B, p->W2Tb, p->H, p->N, eg, s)) return false;
  EpiF32 e2{};
  e2.rows = p->N;
  e2.cols = p->H;
  e2.out = p->dW2;
  if (!gemm(p, p->dOT, p->N, p->HT, p->H, B, e2, s, p->Bt)) return false;
  EpiF32 e1{};
  e1.rows = p->H;
  e1.cols = p->N;
  e1.out = p->dW1;
  if (!gemm(p, p->dZT, p->H, p->XT, p->N, B, e1, s, p->Bt)) return false;
  row_sum_kernel<<<(p->N + 7) / 8, 256, 0, s>>>(p->dOT, p->N, B, p->Bt, p->db2);
  row_sum_kernel<<<(p->H + 7) / 8, 256, 0, s>>>(p->dZT, p->H, B, p->Bt, p->db1);
  return cudaGetLastError() == cudaSuccess;
}

void refresh_bf16(omp_proposal_s* p, cudaStream_t s) {
  const size_t n1 = static_cast<size_t>(p->H) * p->N;
  to_bf16_kernel<<<blocks_for(n1), 256, 0, s>>>(p->W1, n1, p->W1b);
  to_bf16_kernel<<<blocks_for(n1), 256, 0, s>>>(p->W2, n1, p->W2b);
  dim3 grid((p->H + 31) / 32, (p->N + 31) / 32);
  transpose_bf16_kernel<<<grid, dim3(32, 8), 0, s>>>(p->W2, p->N, p->H, p->W2Tb);
}

}  // namespace mlpd
}  // namespace ompk

using namespace ompk::mlpd;

extern "C" {

void omp_proposal_desc_default(omp_proposal_desc* d) {
  if (!d) return;
  std::memset(d, 0, sizeof(*d));
  d->hidden = 1024;
  d->topk = 256;
  d->max_batch = 16384;
  d->train_batch = 4096;
  d->lr = 1e-3f;
  d->beta1 = 0.9f;
  d->beta2 = 0.999f;
  d->weight_decay = 0.f;
  d->adam_eps = 1e-8f;
  d->pos_weight = 1.f;
}

omp_status omp_proposal_create(omp_handle h, const omp_proposal_desc* desc, omp_proposal* out) {
  if (!h || !desc || !out) return OMP_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  omp_desc hd{};
  int dev = 0, sms = 0;
  if (omp_handle_info(h, &hd, &sms) != OMP_OK) return OMP_ERR_INVALID_ARGUMENT;
  dev = hd.device;
  const omp_proposal_desc d = *desc;
  if (d.hidden < 64 || d.hidden % 64 || hd.N % 64 || d.topk < 1 || d.topk > hd.N || d.max_batch < 1 ||
      d.max_batch > hd.max_batch || d.train_batch < 64 || d.train_batch % 64 || d.topk > 256)
    return OMP_ERR_INVALID_ARGUMENT;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(dev);
  omp_proposal_s* p = new (std::nothrow) omp_proposal_s();
  if (!p) return OMP_ERR_OUT_OF_MEMORY;
  p->d = d;
  p->dev = dev;
  p->N = static_cast<int>(hd.N);
  p->M = static_cast<int>(hd.M);
  p->Mp = static_cast<int>((hd.M + 63) / 64 * 64);
  p->H = d.hidden;
  p->Bi = (d.max_batch + 127) / 128 * 128;
  p->Bt = d.train_batch;
  p->grid = sms;
  p->Smax_tau = hd.max_iters;
  const size_t N = p->N, H = p->H, Bx = p->Bi > p->Bt ? p->Bi : p->Bt, Bt = p->Bt, Mp = p->Mp;
  bool ok = palloc(p, &p->W1, H * N) && palloc(p, &p->b1, H) && palloc(p, &p->W2, N * H) && palloc(p, &p->b2, N);
  ok = ok && palloc(p, &p->beta, 1) && palloc(p, &p->mbeta, 1) && palloc(p, &p->vbeta, 1) && palloc(p, &p->dbeta, 1);
  ok = ok && palloc(p, &p->mW1, H * N) && palloc(p, &p->vW1, H * N) && palloc(p, &p->mb1, H) && palloc(p, &p->vb1, H);
  ok = ok && palloc(p, &p->mW2, N * H) && palloc(p, &p->vW2, N * H) && palloc(p, &p->mb2, N) && palloc(p, &p->vb2, N);
  ok = ok && palloc(p, &p->W1b, H * N) && palloc(p, &p->W2b, N * H) && palloc(p, &p->W2Tb, H * N);
  ok = ok && palloc(p, &p->A16, N * Mp) && palloc(p, &p->escale, N);
  ok = ok && palloc(p, &p->Yq, Bx * Mp) && palloc(p, &p->inv_yn, Bx) && palloc(p, &p->X, Bx * N) &&
       palloc(p, &p->Hh, Bx * H) && palloc(p, &p->logits, static_cast<size_t>(p->Bi) * N) &&
       palloc(p, &p->cand, static_cast<size_t>(p->Bi) * d.topk);
  ok = ok && palloc(p, &p->XT, N * Bt) && palloc(p, &p->HT, H * Bt) && palloc(p, &p->Z1, Bt * H) &&
       palloc(p, &p->dO, Bt * N) && palloc(p, &p->dOT, N * Bt) && palloc(p, &p->dZT, H * Bt) &&
       palloc(p, &p->dW1, H * N) && palloc(p, &p->db1, H) && palloc(p, &p->dW2, N * H) &&
       palloc(p, &p->db2, N) && palloc(p, &p->labels, Bt * (N / 32)) && palloc(p, &p->loss, 1) &&
       palloc(p, &p->tau, static_cast<size_t>(p->Smax_tau)) && palloc(p, &p->err, 1);
  bool cuda_ok = ok;
  if (ok) {
    const size_t n1 = H * N;
    cuda_ok = cudaMemset(p->W1, 0, n1 * 4) == cudaSuccess && cudaMemset(p->W2, 0, n1 * 4) == cudaSuccess &&
              cudaMemset(p->b1, 0, H * 4) == cudaSuccess && cudaMemset(p->b2, 0, N * 4) == cudaSuccess &&
              cudaMemset(p->mW1, 0, n1 * 4) == cudaSuccess && cudaMemset(p->vW1, 0, n1 * 4) == cudaSuccess &&
              cudaMemset(p->mW2, 0, n1 * 4) == cudaSuccess && cudaMemset(p->vW2, 0, n1 * 4) == cudaSuccess &&
              cudaMemset(p->mb1, 0, H * 4) == cudaSuccess && cudaMemset(p->vb1, 0, H * 4) == cudaSuccess &&
              cudaMemset(p->mb2, 0, N * 4) == cudaSuccess && cudaMemset(p->vb2, 0, N * 4) == cudaSuccess &&
              cudaMemset(p->tau, 0, p->Smax_tau * 4) == cudaSuccess && cudaMemset(p->err, 0, 4) == cudaSuccess &&
              cudaMemset(p->beta, 0, 4) == cudaSuccess && cudaMemset(p->mbeta, 0, 4) == cudaSuccess &&
              cudaMemset(p->vbeta, 0, 4) == cudaSuccess &&
              cudaDeviceSynchronize() == cudaSuccess;
  }
  if (prev >= 0) cudaSetDevice(prev);
  if (!ok || !cuda_ok) {
    pfree(p);
    delete p;
    return ok ? OMP_ERR_CUDA : OMP_ERR_OUT_OF_MEMORY;
  }
  *out = p;
  return OMP_OK;
}

omp_status omp_proposal_destroy(omp_proposal p) {
  if (!p) return OMP_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(p->dev);
  cudaDeviceSynchronize();
  pfree(p);
  if (prev >= 0) cudaSetDevice(prev);
  delete p;
  return OMP_OK;
}

omp_status omp_proposal_set_weights(omp_proposal p, const float* W1, const float* b1, const float* W2,
                                    const float* b2, const float* beta, void* stream) {
  if (!p || !W1 || !b1 || !W2 || !b2 || !beta) return OMP_ERR_INVALID_ARGUMENT;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t n1 = static_cast<size_t>(p->H) * p->N;
  bool ok = cudaMemcpyAsync(p->beta, beta, 4, cudaMemcpyDefault, s) == cudaSuccess &&
            cudaMemsetAsync(p->mbeta, 0, 4, s) == cudaSuccess && cudaMemsetAsync(p->vbeta, 0, 4, s) == cudaSuccess &&
            cudaMemcpyAsync(p->W1, W1, n1 * 4, cudaMemcpyDefault, s) == cudaSuccess &&
            cudaMemcpyAsync(p->W2, W2, n1 * 4, cudaMemcpyDefault, s) == cudaSuccess &&
            cudaMemcpyAsync(p->b1, b1, p->H * 4, cudaMemcpyDefault, s) == cudaSuccess &&
            cudaMemcpyAsync(p->b2, b2, p->N * 4, cudaMemcpyDefault, s) == cudaSuccess;
  if (!ok) return OMP_ERR_CUDA;
  refresh_bf16(p, s);
  p->step = 0;
  const size_t z1 = n1 * 4;
  ok = cudaMemsetAsync(p->mW1, 0, z1, s) == cudaSuccess && cudaMemsetAsync(p->vW1, 0, z1, s) == cudaSuccess &&
       cudaMemsetAsync(p->mW2, 0, z1, s) == cudaSuccess && cudaMemsetAsync(p->vW2, 0, z1, s) == cudaSuccess &&
       cudaMemsetAsync(p->mb1, 0, p->H * 4, s) == cudaSuccess && cudaMemsetAsync(p->vb1, 0, p->H * 4, s) == cudaSuccess &&
       cudaMemsetAsync(p->mb2, 0, p->N * 4, s) == cudaSuccess && cudaMemsetAsync(p->vb2, 0, p->N * 4, s) == cudaSuccess;
  return ok && cudaGetLastError() == cudaSuccess ? OMP_OK : OMP_ERR_CUDA;
}

omp_status omp_proposal_get_weights(omp_proposal p, float* W1, float* b1, float* W2, float* b2, float* beta,
                                    void* stream) {
  if (!p || !W1 || !b1 || !W2 || !b2 || !beta) return OMP_ERR_INVALID_ARGUMENT;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t n1 = static_cast<size_t>(p->H) * p->N;
  const bool ok = cudaMemcpyAsync(beta, p->beta, 4, cudaMemcpyDefault, s) == cudaSuccess &&
                  cudaMemcpyAsync(W1, p->W1, n1 * 4, cudaMemcpyDefault, s) == cudaSuccess &&
                  cudaMemcpyAsync(W2, p->W2, n1 * 4, cudaMemcpyDefault, s) == cudaSuccess &&
                  cudaMemcpyAsync(b1, p->b1, p->H * 4, cudaMemcpyDefault, s) == cudaSuccess &&
                  cudaMemcpyAsync(b2, p->b2, p->N * 4, cudaMemcpyDefault, s) == cudaSuccess &&
                  cudaStreamSynchronize(s) == cudaSuccess;
  return ok ? OMP_OK : OMP_ERR_CUDA;
}

omp_status omp_proposal_gradients(omp_proposal p, const float* A, const float* Y, const int32_t* labels,
                                  int64_t B, int32_t S, float* dW1, float* db1, float* dW2, float* db2,
                                  float* dbeta, float* loss_out, void* stream) {
  if (!p || !A || !Y || !labels || B < 64 || B % 64 || B > p->Bt || S < 1) return OMP_ERR_INVALID_ARGUMENT;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!gradients(p, A, Y, labels, static_cast<int>(B), S, s)) return OMP_ERR_CUDA;
  const size_t n1 = static_cast<size_t>(p->H) * p->N;
  bool ok = true;
  if (dW1) ok = ok && cudaMemcpyAsync(dW1, p->dW1, n1 * 4, cudaMemcpyDefault, s) == cudaSuccess;
  if (dW2) ok = ok && cudaMemcpyAsync(dW2, p->dW2, n1 * 4, cudaMemcpyDefault, s) == cudaSuccess;
  if (db1) ok = ok && cudaMemcpyAsync(db1, p->db1, p->H * 4, cudaMemcpyDefault, s) == cudaSuccess;
  if (db2) ok = ok && cudaMemcpyAsync(db2, p->db2, p->N * 4, cudaMemcpyDefault, s) == cudaSuccess;
  if (dbeta) ok = ok && cudaMemcpyAsync(dbeta, p->dbeta, 4, cudaMemcpyDefault, s) == cudaSuccess;
  if (loss_out) ok = ok && cudaMemcpyAsync(loss_out, p->loss, 4, cudaMemcpyDefault, s) == cudaSuccess;
  return ok ? OMP_OK : OMP_ERR_CUDA;
}

omp_status omp_proposal_train_step(omp_proposal p, const float* A, const float* Y, const int32_t* labels,
                                   int64_t B, int32_t S, float* loss_out, void* stream) {
  if (!p || !A || !Y || !labels || B < 64 || B % 64 || B > p->Bt || S < 1) return OMP_ERR_INVALID_ARGUMENT;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!gradients(p, A, Y, labels, static_cast<int>(B), S, s)) return OMP_ERR_CUDA;
  p->step += 1;
  AdamParams a;
  a.lr = p->d.lr;
  a.beta1 = p->d.beta1;
  a.beta2 = p->d.beta2;
  a.eps = p->d.adam_eps;
  a.wd = p->d.weight_decay;
  a.c1 = static_cast<float>(1.0 / (1.0 - std::pow(static_cast<double>(a.beta1), static_cast<double>(p->step))));
  a.c2 = static_cast<float>(1.0 / (1.0 - std::pow(static_cast<double>(a.beta2), static_cast<double>(p->step))));
  const size_t n1 = static_cast<size_t>(p->H) * p->N;
  adamw_kernel<<<blocks_for(n1), 256, 0, s>>>(p->W1, p->mW1, p->vW1, p->dW1, n1, a, p->W1b);
  adamw_kernel<<<blocks_for(n1), 256, 0, s>>>(p->W2, p->mW2, p->vW2, p->dW2, n1, a, p->W2b);
  adamw_kernel<<<blocks_for(p->H), 256, 0, s>>>(p->b1, p->mb1, p->vb1, p->db1, p->H, a, nullptr);
  adamw_kernel<<<blocks_for(p->N), 256, 0, s>>>(p->b2, p->mb2, p->vb2, p->db2, p->N, a, nullptr);
  adamw_kernel<<<1, 32, 0, s>>>(p->beta, p->mbeta, p->vbeta, p->dbeta, 1, a, nullptr);
  dim3 grid((p->H + 31) / 32, (p->N + 31) / 32);
  transpose_bf16_kernel<<<grid, dim3(32, 8), 0, s>>>(p->W2, p->N, p->H, p->W2Tb);
  if (loss_out && cudaMemcpyAsync(loss_out, p->loss, 4, cudaMemcpyDefault, s) != cudaSuccess) return OMP_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? OMP_OK : OMP_ERR_CUDA;
}

omp_status omp_proposal_infer(omp_proposal p, const float* A, const float* Y, int64_t B, int32_t* cand_out,
                              float* logits_out, void* stream) {
  if (!p || !A || !Y || B < 1 || B > p->d.max_batch) return OMP_ERR_INVALID_ARGUMENT;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int b = static_cast<int>(B);
  if (!features(p, A, Y, b, false, s) || !forward_hidden(p, b, false, s)) return OMP_ERR_CUDA;
  EpiF32 e{};
  e.rows = b;
  e.cols = p->N;
  e.bias = p->b2;
  e.skipX = p->X;
  e.beta = p->beta;
  e.out = p->logits;
  if (!gemm(p, p->Hh, b, p->W2b, p->N, p->H, e, s)) return OMP_ERR_CUDA;
  bool ok = launch_topk_rows(p->logits, b, p->N, p->d.topk, p->cand, s);
  if (cand_out)
    ok = ok && cudaMemcpyAsync(cand_out, p->cand, static_cast<size_t>(b) * p->d.topk * 4, cudaMemcpyDefault, s) == cudaSuccess;
  if (logits_out)
    ok = ok && cudaMemcpyAsync(logits_out, p->logits, static_cast<size_t>(b) * p->N * 4, cudaMemcpyDefault, s) == cudaSuccess;
  return ok && cudaGetLastError() == cudaSuccess ? OMP_OK : OMP_ERR_CUDA;
}

// Candidates of the method without the network: the top-K atoms of |x| = |A^T y| / (||a|| ||y||).
omp_status omp_proposal_baseline_candidates(omp_proposal p, const float* A, const float* Y, int64_t B,
                                            int32_t* cand_out, void* stream) {
  if (!p || !A || !Y || !cand_out || B < 1 || B > p->d.max_batch) return OMP_ERR_INVALID_ARGUMENT;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int b = static_cast<int>(B);
  if (!features(p, A, Y, b, false, s)) return OMP_ERR_CUDA;
  const size_t n = static_cast<size_t>(b) * p->N;
  abs_bf16_kernel<<<blocks_for(n), 256, 0, s>>>(p->X, n, p->logits);
  return launch_topk_rows(p->logits, b, p->N, p->d.topk, cand_out, s) ? OMP_OK : OMP_ERR_CUDA;
}

omp_status omp_proposal_set_thresholds(omp_proposal p, const float* tau_host, int32_t S) {
  if (!p || !tau_host || S < 1 || S > p->Smax_tau) return OMP_ERR_INVALID_ARGUMENT;
  return cudaMemcpy(p->tau, tau_host, static_cast<size_t>(S) * 4, cudaMemcpyHostToDevice) == cudaSuccess
             ? OMP_OK
             : OMP_ERR_CUDA;
}

omp_status omp_proposal_get_thresholds(omp_proposal p, float* tau_host, int32_t S) {
  if (!p || !tau_host || S < 1 || S > p->Smax_tau) return OMP_ERR_INVALID_ARGUMENT;
  return cudaMemcpy(tau_host, p->tau, static_cast<size_t>(S) * 4, cudaMemcpyDeviceToHost) == cudaSuccess
             ? OMP_OK
             : OMP_ERR_CUDA;
}

// ------------------------------------------------------------------------------ save / load
// File layout (little-endian): the 8 bytes "OMPPROP1"; int32 N, hidden, topk, S (thresholds);
// FP32 W1 (hidden x N), b1 (hidden), W2 (N x hidden), b2 (N), beta (1), tau (S); then a 64-bit
// FNV-1a hash of every byte before it, so a truncated or altered file is refused.
namespace {
constexpr char kPropMagic[8] = {'O', 'M', 'P', 'P', 'R', 'O', 'P', '1'};

uint64_t fnv1a(const unsigned char* data, size_t n, uint64_t h = 1469598103934665603ull) {
  for (size_t i = 0; i < n; ++i) {
    h ^= data[i];
    h *= 1099511628211ull;
  }
  return h;
}

struct PropFile {
  int32_t hdr[4];  // N, hidden, topk, S
  std::vector<float> W1, b1, W2, b2, beta, tau;
};

size_t prop_payload_floats(const int32_t* hdr) {
  const size_t N = static_cast<size_t>(hdr[0]), H = static_cast<size_t>(hdr[1]);
  return 2 * N * H + H + N + 1 + static_cast<size_t>(hdr[3]);
}
}  // namespace

omp_status omp_proposal_save(omp_proposal p, const char* path) {
  if (!p || !path) return OMP_ERR_INVALID_ARGUMENT;
  const int32_t hdr[4] = {p->N, p->H, p->d.topk, p->Smax_tau};
  const size_t n1 = static_cast<size_t>(p->H) * p->N;
  std::vector<float> buf(prop_payload_floats(hdr));
  float* W1 = buf.data();
  float* W2 = W1 + n1;
  float* b1 = W2 + n1;
  float* b2 = b1 + p->H;
  float* beta = b2 + p->N;
  float* tau = beta + 1;
  omp_status st = omp_proposal_get_weights(p, W1, b1, W2, b2, beta, nullptr);
  if (st == OMP_OK) st = omp_proposal_get_thresholds(p, tau, p->Smax_tau);
  if (st != OMP_OK) return st;
  // written in the file's order: W1, b1, W2, b2, beta, tau
  std::vector<unsigned char> out(sizeof(kPropMagic) + sizeof(hdr) + buf.size() * 4);
  unsigned char* o = out.data();
  std::memcpy(o, kPropMagic, sizeof(kPropMagic));
  o += sizeof(kPropMagic);
  std::memcpy(o, hdr, sizeof(hdr));
  o += sizeof(hdr);
  const std::pair<const float*, size_t> parts[] = {{W1, n1}, {b1, static_cast<size_t>(p->H)}, {W2, n1},
                                                   {b2, static_cast<size_t>(p->N)}, {beta, 1},
                                                   {tau, static_cast<size_t>(p->Smax_tau)}};
  for (const auto& part : parts) {
    std::memcpy(o, part.first, part.second * 4);
    o += part.second * 4;
  }
  const uint64_t h = fnv1a(out.data(), out.size());
  FILE* f = std::fopen(path, "wb");
  if (!f) return OMP_ERR_INVALID_ARGUMENT;
  const bool ok = std::fwrite(out.data(), 1, out.size(), f) == out.size() &&
                  std::fwrite(&h, sizeof(h), 1, f) == 1;
  return (std::fclose(f) == 0 && ok) ? OMP_OK : OMP_ERR_INVALID_ARGUMENT;
}

omp_status omp_proposal_load(omp_proposal p, const char* path) {
  if (!p || !path) return OMP_ERR_INVALID_ARGUMENT;
  FILE* f = std::fopen(path, "rb");
  if (!f) return OMP_ERR_INVALID_ARGUMENT;
  std::vector<unsigned char> in;
  unsigned char chunk[1 << 16];
  size_t got;
  while ((got = std::fread(chunk, 1, sizeof(chunk), f)) > 0) in.insert(in.end(), chunk, chunk + got);
  std::fclose(f);
  const size_t head = sizeof(kPropMagic) + 4 * sizeof(int32_t);
  if (in.size() < head + sizeof(uint64_t) || std::memcmp(in.data(), kPropMagic, sizeof(kPropMagic)) != 0)
    return OMP_ERR_INVALID_ARGUMENT;
  int32_t hdr[4];
  std::memcpy(hdr, in.data() + sizeof(kPropMagic), sizeof(hdr));
  if (hdr[0] != p->N || hdr[1] != p->H || hdr[3] < 1 || hdr[3] > 4096) return OMP_ERR_INVALID_ARGUMENT;
  const size_t nf = prop_payload_floats(hdr);
  if (in.size() != head + nf * 4 + sizeof(uint64_t)) return OMP_ERR_INVALID_ARGUMENT;
  uint64_t h = 0;
  std::memcpy(&h, in.data() + head + nf * 4, sizeof(h));
  if (h != fnv1a(in.data(), head + nf * 4)) return OMP_ERR_INVALID_ARGUMENT;
  std::vector<float> buf(nf);
  std::memcpy(buf.data(), in.data() + head, nf * 4);
  const size_t n1 = static_cast<size_t>(p->H) * p->N;
  const float* W1 = buf.data();
  const float* b1 = W1 + n1;
  const float* W2 = b1 + p->H;
  const float* b2 = W2 + n1;
  const float* beta = b2 + p->N;
  const float* tau = beta + 1;
  omp_status st = omp_proposal_set_weights(p, W1, b1, W2, b2, beta, nullptr);
  if (st == OMP_OK && cudaDeviceSynchronize() != cudaSuccess) st = OMP_ERR_CUDA;
  // thresholds: as many as both the file and the proposal hold; the rest accept every step
  const int S = hdr[3] < p->Smax_tau ? hdr[3] : p->Smax_tau;
  std::vector<float> t(static_cast<size_t>(p->Smax_tau), 0.f);
  std::memcpy(t.data(), tau, static_cast<size_t>(S) * 4);
  if (st == OMP_OK) st = omp_proposal_set_thresholds(p, t.data(), p->Smax_tau);
  return st;
}

omp_status omp_proposal_calibrate(omp_proposal p, const float* drops, int64_t B, int32_t S, float quantile,
                                  void* stream) {
  if (!p || !drops || B < 1 || S < 1 || S > p->Smax_tau || !(quantile >= 0.f && quantile <= 1.f))
    return OMP_ERR_INVALID_ARGUMENT;
  quantile_cols_kernel<<<S, 256, 0, static_cast<cudaStream_t>(stream)>>>(drops, static_cast<int>(B), S,
                                                                           quantile, p->tau);
  return cudaGetLastError() == cudaSuccess ? OMP_OK : OMP_ERR_CUDA;
}

omp_status omp_topk_rows(const float* logits, int64_t rows, int64_t N, int32_t K, int32_t* idx_out, void* stream) {
  if (!logits || !idx_out || rows < 1 || N < 1 || K < 1 || K > N || N > (1 << 30)) return OMP_ERR_INVALID_ARGUMENT;
  return launch_topk_rows(logits, static_cast<int>(rows), static_cast<int>(N), K, idx_out,
                          static_cast<cudaStream_t>(stream))
             ? OMP_OK
             : OMP_ERR_CUDA;
}

}  // extern "C"

namespace ompk {
bool proposal_run_inference(omp_proposal p, const float* A, const float* Y, int B, cudaStream_t s) {
  if (B > p->d.max_batch) return false;
  if (!features(p, A, Y, B, false, s) || !forward_hidden(p, B, false, s)) return false;
  EpiF32 e{};
  e.rows = B;
  e.cols = p->N;
  e.bias = p->b2;
  e.skipX = p->X;
  e.beta = p->beta;
  e.out = p->logits;
  if (!gemm(p, p->Hh, B, p->W2b, p->N, p->H, e, s)) return false;
  return launch_topk_rows(p->logits, B, p->N, p->d.topk, p->cand, s);
}

// accessors used by the learned solve (runtime.cu)
const int* proposal_candidates(omp_proposal p) { return p->cand; }
int proposal_topk(omp_proposal p) { return p->d.topk; }
const float* proposal_tau(omp_proposal p) { return p->tau; }
int proposal_tau_len(omp_proposal p) { return p->Smax_tau; }
float* proposal_tau_mut(omp_proposal p) { return p->tau; }
}  // namespace ompk
