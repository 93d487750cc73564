// FP32 correlation on the CUDA cores (the plain-FP32 path) and the FP32 Gram matrix.
//
// Both are the contraction C = X A^T over the padded signal length Mp with both operands stored
// K-major (rows of Mp contiguous floats): for the correlation X holds the live residuals
// (batched as one GEMM, Sec. 3.2 eq:bmm), for the Gram matrix X = A^T itself (Sec. 2.2).
// A 128 x 128 output tile per 256-thread block, 8 x 8 outputs per thread, K chunks of 16 staged
// through double-buffered shared memory.
//
// A third form stores C = Y A^T for signals 0..B-1 (rows of R32 in signal order) into the c0
// workspace: the exact first correlation the Gram-space solve starts from.
//
// The correlation never writes C: the epilogue forms the score |c| / ||a_n|| (Alg. 1), takes
// each thread's best atom in ascending index order (strict '>', so the lowest index keeps a
// tie), reduces across the 16 threads that share a signal with warp shuffles, and merges the
// tile's winner into the signal's packed (score, ~index) key with one 64-bit atomicMax: the
// maximum key is the highest score and, among equal scores, the lowest index, whatever order
// the tiles finish in.
#include "common.cuh"

namespace ompk {

namespace {
constexpr int BM = 128, BN = 128, BK = 16, PAD = 4;

constexpr int kCorrelate = 0, kGram = 1, kStoreC = 2;

// MODE kCorrelate: k is the iteration; kGram: k unused; kStoreC: k is the number of signals
template <int MODE>
__global__ void __launch_bounds__(256, 2) simt_tile_kernel(Ws ws, int k) {
  constexpr bool GRAM = MODE == kGram;
  __shared__ __align__(16) float Xs[2][BK][BM + PAD];
  __shared__ __align__(16) float As[2][BK][BN + PAD];
  const int tid = threadIdx.x;
  const int n0 = blockIdx.x * BN;
  const int p0 = blockIdx.y * BM;
  int L;
  const int* live = nullptr;
  if (GRAM) {
    L = ws.N;
  } else if (MODE == kStoreC) {
    L = k;
  } else {
    k = iter_of(ws, k);
    L = ws.cnt[k + 1];
    live = ws.live[k & 1];
  }
  if (p0 >= L) return;

  const int lrow = tid >> 2, lk = (tid & 3) * 4;
  const float* xsrc[2];
  const float* asrc[2];
  bool xv[2], av[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int p = p0 + lrow + 64 * i;
    xv[i] = p < L;
    const int row = xv[i] ? ((GRAM || MODE == kStoreC) ? p : live[p]) : 0;
    xsrc[i] = (GRAM ? ws.A32 : ws.R32) + static_cast<size_t>(row) * ws.Mp + lk;
    const int n = n0 + lrow + 64 * i;
    av[i] = n < ws.N;
    asrc[i] = ws.A32 + static_cast<size_t>(av[i] ? n : 0) * ws.Mp + lk;
  }
  float4 xr[2], ar[2];
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  auto gload = [&](int kc) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      xr[i] = xv[i] ? __ldg(reinterpret_cast<const float4*>(xsrc[i] + kc)) : zero;
      ar[i] = av[i] ? __ldg(reinterpret_cast<const float4*>(asrc[i] + kc)) : zero;
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
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  const int tx = tid & 15, ty = tid >> 4;
  const int nk = ws.Mp / BK;
  gload(0);
  sstore(0);
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nk) gload((kt + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 x0 = *reinterpret_cast<const float4*>(&Xs[buf][kk][ty * 4]);
      const float4 x1 = *reinterpret_cast<const float4*>(&Xs[buf][kk][64 + ty * 4]);
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][tx * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + tx * 4]);
      const float xf[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
      const float af[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(xf[i], af[j], acc[i][j]);
    }
    if (kt + 1 < nk) sstore(buf ^ 1);
    __syncthreads();
  }

  // atoms of this thread, ascending: n0 + tx*4 + {0..3}, then n0 + 64 + tx*4 + {0..3}
  int ncol[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) ncol[j] = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));

  if (GRAM) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int row = p0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
      if (row >= ws.N) continue;
      float* g = ws.gram + static_cast<size_t>(row) * ws.N;
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (ncol[j] < ws.N) g[ncol[j]] = acc[i][j];
    }
    return;
  }
  if (MODE == kStoreC) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int row = p0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
      if (row >= L) continue;
      float* c = ws.c0 + static_cast<size_t>(row) * ws.N;
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (ncol[j] < ws.N) c[ncol[j]] = acc[i][j];
    }
    return;
  }

  float inv[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) inv[j] = ncol[j] < ws.N ? __ldg(ws.inv_norm + ncol[j]) : 0.f;
  if (ws.cand2) {
    // Margins recorded: each row's best two atoms of the tile (same scan and ties), then
    // cand1 keeps the global best as before and cand2 receives every key that loses a merge
    // (the smaller of the old and the new key of each atomicMax) and each tile's second best,
    // so that it ends with the largest key other than the best: the runner-up.
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int prow = p0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
      float b1 = -1.f, b2 = -1.f;
      int i1 = 0x7fffffff, i2 = 0x7fffffff;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (ncol[j] < ws.N) {
          const float sc = fabsf(acc[i][j]) * inv[j];
          if (better(sc, ncol[j], b1, i1)) {
            b2 = b1;
            i2 = i1;
            b1 = sc;
            i1 = ncol[j];
          } else if (better(sc, ncol[j], b2, i2)) {
            b2 = sc;
            i2 = ncol[j];
          }
        }
      }
#pragma unroll
      for (int o = 1; o < 16; o <<= 1) {
        const float o1 = __shfl_xor_sync(0xffffffffu, b1, o);
        const int oi1 = __shfl_xor_sync(0xffffffffu, i1, o);
        const float o2 = __shfl_xor_sync(0xffffffffu, b2, o);
        const int oi2 = __shfl_xor_sync(0xffffffffu, i2, o);
        if (better(o1, oi1, b1, i1)) {
          if (!better(b1, i1, o2, oi2)) {
            b1 = o2;  // the partner holds both: (o1, o2)
            i1 = oi2;
          }
          b2 = b1;
          i2 = i1;
          b1 = o1;
          i1 = oi1;
        } else if (better(o1, oi1, b2, i2)) {
          b2 = o1;
          i2 = oi1;
        }
      }
      if (tx == 0 && prow < L && i1 < ws.N) {
        const unsigned long long k1 = pack_key(b1, i1);
        const unsigned long long old = atomicMax(ws.cand1 + prow, k1);
        atomicMax(ws.cand2 + prow, old < k1 ? old : k1);
        if (i2 < ws.N) atomicMax(ws.cand2 + prow, pack_key(b2, i2));
      }
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int prow = p0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    float best = -1.f;
    int bidx = 0x7fffffff;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (ncol[j] < ws.N) {
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
    if (tx == 0 && prow < L && bidx < ws.N) atomicMax(ws.cand1 + prow, pack_key(best, bidx));
  }
}
}  // namespace

void launch_corr_simt(const Ws& ws, int k, int B, cudaStream_t s) {
  dim3 grid((ws.N + BN - 1) / BN, (B + BM - 1) / BM);
  simt_tile_kernel<kCorrelate><<<grid, 256, 0, s>>>(ws, k);
}

void launch_c0_simt(const Ws& ws, int B, cudaStream_t s) {
  dim3 grid((ws.N + BN - 1) / BN, (B + BM - 1) / BM);
  simt_tile_kernel<kStoreC><<<grid, 256, 0, s>>>(ws, B);
}

void launch_gram_simt(const Ws& ws, cudaStream_t s) {
  dim3 grid((ws.N + BN - 1) / BN, (ws.N + BM - 1) / BM);
  simt_tile_kernel<kGram><<<grid, 256, 0, s>>>(ws, 0);
}

}  // namespace ompk
