// Candidate-restricted OMP iteration for the learned proposal (one warp per signal).
//
// Given K candidate atoms per signal (from the proposal network), the iteration runs the paper's
// v0 scheme (Sec. 2.3: "D_k = A^T A_k F_k", projections updated by one vector per step)
// restricted to the candidates, so no per-step correlation with the whole dictionary is needed:
//   c      = A_K^T y                        exact FP32 dot products of the K candidate rows
//   per step k:
//     n*   = argmax_i |c_i| / ||a_i||        lowest atom index on ties
//     z    = Q^T a_{n*}, read from D        (D column j = A_K^T q_j, so z_j = D[j][n*])
//     delta = ||a_{n*}||^2 - ||z||^2 (FP64), gamma = 1 / sqrt(delta)
//     D[k] = gamma (G[K, n*] - sum_j z_j D[j])    G row of n* gathered at the candidates
//     b_k  = gamma c_{n*},  c <- c - b_k D[k],  ||r_k||^2 = ||r_{k-1}||^2 - b_k^2
//     F column k = [-gamma F z ; gamma]   (for x = F b)
//   residual-drop check: step k is accepted only if b_k^2 / ||r_{k-1}||^2 >= tau_k; a signal
//   that fails (or whose best candidate is dependent or scores 0) leaves the restricted phase
//   with steps 0..k-1, its residual r = y - A_S F b materialised, and continues in the dense
//   loop from iteration k (flag = 1).
// At the end every signal's F (FP64 and FP32 copies), b, support and iteration count are in the
// same state arrays the dense loop uses, and its residual is recomputed from the support.
#include "common.cuh"

namespace ompk {
namespace {

struct RSmem {
  float* D;     // S x K: D[j * K + i]
  float* Fs;    // S (S + 1) / 2, packed by columns
  float* c;     // K
  float* y;     // Mp
  float* z;     // S
  int* pos;     // S: candidate slot of the j-th pick
};

__host__ __device__ __forceinline__ size_t rs_bytes(int S, int K, int Mp) {
  size_t b = static_cast<size_t>(S) * K * 4 + static_cast<size_t>(S) * (S + 1) / 2 * 4 +
             static_cast<size_t>(K) * 4 + static_cast<size_t>(Mp) * 4 + static_cast<size_t>(S) * 8;
  return (b + 15) / 16 * 16;
}

__device__ __forceinline__ RSmem rs_smem(unsigned char* base, int w, int S, int K, int Mp) {
  unsigned char* g = base + static_cast<size_t>(w) * rs_bytes(S, K, Mp);
  RSmem s;
  s.y = reinterpret_cast<float*>(g);
  s.D = s.y + Mp;
  s.Fs = s.D + static_cast<size_t>(S) * K;
  s.c = s.Fs + static_cast<size_t>(S) * (S + 1) / 2;
  s.z = s.c + K;
  s.pos = reinterpret_cast<int*>(s.z + S);
  return s;
}

constexpr int kMaxCandPerLane = 8;  // K <= 256

__global__ void restricted_kernel(Ws ws, const CallArgs* args, const int* __restrict__ cand, int K,
                                  const float* __restrict__ tau, int B, int S, float eps, int eps_rel,
                                  int* __restrict__ fallback) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = blockIdx.x * (blockDim.x >> 5) + w;
  if (b >= B) return;
  RSmem sm = rs_smem(smem, w, S, K, ws.Mp);
  const float yn = ws.ynorm[b];
  const int* cb = cand + static_cast<size_t>(b) * K;
  int* supg = ws.sup + static_cast<size_t>(b) * ws.Smax;
  double* bvg = ws.bv + static_cast<size_t>(b) * ws.Smax;
  if (!(yn > 0.f)) {  // y == 0 or non-finite: handled by init (empty support, not live)
    if (lane == 0) {
      ws.flag[b] = 0;
      fallback[b] = -1;
    }
    return;
  }
  // y into shared memory
  const float* yg = args->Y + static_cast<size_t>(b) * ws.M;
  for (int m = lane; m < ws.Mp; m += 32) sm.y[m] = m < ws.M ? yg[m] : 0.f;
  __syncwarp();
  // c_i = a_i^T y for the candidates (FP32, lanes over the signal, one candidate at a time)
  const int M4 = ws.Mp >> 2;
  for (int i = 0; i < K; ++i) {
    const float4* a4 = reinterpret_cast<const float4*>(ws.A32 + static_cast<size_t>(cb[i]) * ws.Mp);
    float acc = 0.f;
    for (int q = lane; q < M4; q += 32) {
      const float4 a = __ldg(a4 + q);
      const float4 y = reinterpret_cast<const float4*>(sm.y)[q];
      acc += a.x * y.x + a.y * y.y + a.z * y.z + a.w * y.w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) sm.c[i] = acc;
  }
  __syncwarp();
  // per-lane candidate slots i = lane + 32 t
  int atom[kMaxCandPerLane];
  float inv[kMaxCandPerLane];
#pragma unroll
  for (int t = 0; t < kMaxCandPerLane; ++t) {
    const int i = lane + 32 * t;
    atom[t] = i < K ? cb[i] : -1;
    inv[t] = i < K ? __ldg(ws.inv_norm + atom[t]) : 0.f;
  }
  double r2 = static_cast<double>(yn) * static_cast<double>(yn);
  const double thr = eps_rel ? static_cast<double>(eps) * yn : static_cast<double>(eps);
  int k = 0;
  int fb = -1;
  int stop = kStopIters;
  for (; k < S; ++k) {
    // ---- pick: argmax |c_i| / ||a_i||, lowest atom index on ties
    float bs = -1.f;
    int bi = 0x7fffffff, bslot = -1;
#pragma unroll
    for (int t = 0; t < kMaxCandPerLane; ++t) {
      const int i = lane + 32 * t;
      if (i < K) {
        const float sc = fabsf(sm.c[i]) * inv[t];
        if (better(sc, atom[t], bs, bi)) {
          bs = sc;
          bi = atom[t];
          bslot = i;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float os = __shfl_xor_sync(0xffffffffu, bs, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      const int osl = __shfl_xor_sync(0xffffffffu, bslot, o);
      if (better(os, oi, bs, bi)) {
        bs = os;
        bi = oi;
        bslot = osl;
      }
    }
    const int ns = bi, slot = bslot;
    if (!(bs > 0.f) || ns < 0 || ns >= ws.N) {
      fb = k;
      break;
    }
    // ---- z_j = D[j][slot], delta, gamma
    double zz = 0.0;
    for (int j = lane; j < k; j += 32) {
      const float zj = sm.D[static_cast<size_t>(j) * K + slot];
      sm.z[j] = zj;
      zz += static_cast<double>(zj) * zj;
    }
    zz = warp_sum(zz);
    const double nrm2 = ws.norm2[ns];
    const double delta = nrm2 - zz;
    if (!(delta > kDepRtol * nrm2)) {
      fb = k;
      break;
    }
    const double gamma = 1.0 / sqrt(delta);
    const float gf = static_cast<float>(gamma);
    const float cn = sm.c[slot];
    const double bk = gamma * static_cast<double>(cn);
    // ---- residual-drop check
    const double drop = (bk * bk) / r2;
    if (drop < static_cast<double>(tau[k])) {
      fb = k;
      break;
    }
    __syncwarp();
    // ---- new D column: gamma (G[n*, K] - sum_j z_j D[j])
    const float* grow = ws.gram + static_cast<size_t>(ns) * ws.N;
    float* Dk = sm.D + static_cast<size_t>(k) * K;
#pragma unroll
    for (int t = 0; t < kMaxCandPerLane; ++t) {
      const int i = lane + 32 * t;
      if (i < K) {
        float acc = __ldg(grow + atom[t]);
        for (int j = 0; j < k; ++j) acc = fmaf(-sm.z[j], sm.D[static_cast<size_t>(j) * K + i], acc);
        const float d = gf * acc;
        Dk[i] = d;
        sm.c[i] = fmaf(-static_cast<float>(bk), d, sm.c[i]);
      }
    }
    // ---- F column k = [-gamma F z ; gamma] (FP32 products, FP64 scaling)
    float* Fcol = sm.Fs + static_cast<size_t>(k) * (k + 1) / 2;
    double* Fg = ws.F + static_cast<size_t>(b) * ws.Fstride + static_cast<size_t>(k) * (k + 1) / 2;
    float* Ff = ws.F32 + static_cast<size_t>(b) * ws.Fstride + static_cast<size_t>(k) * (k + 1) / 2;
    for (int j = lane; j < k; j += 32) {
      float u = 0.f;
      for (int l = j; l < k; ++l) u = fmaf(sm.Fs[static_cast<size_t>(l) * (l + 1) / 2 + j], sm.z[l], u);
      const double fv = -gamma * static_cast<double>(u);
      Fcol[j] = static_cast<float>(fv);
      Fg[j] = fv;
      Ff[j] = static_cast<float>(fv);
    }
    if (lane == 0) {
      Fcol[k] = gf;
      Fg[k] = gamma;
      Ff[k] = gf;
      sm.pos[k] = slot;
      supg[k] = ns;
      bvg[k] = bk;
      ws.drop[static_cast<size_t>(b) * ws.Smax + k] = static_cast<float>(drop);
    }
    r2 -= bk * bk;
    __syncwarp();
    if (r2 <= thr * thr) {
      stop = kStopEps;
      ++k;
      break;
    }
  }
  // ---- materialise the residual r = y - A_S x with x = F b (FP64), and its norm
  const int n = k;
  __syncwarp();
  // x into shared z (float) after an FP64 back-substitution; lanes over i
  const double* Fb = ws.F + static_cast<size_t>(b) * ws.Fstride;
  for (int i = lane; i < n; i += 32) {
    double acc = 0.0;
    for (int j = i; j < n; ++j) acc += Fb[static_cast<size_t>(j) * (j + 1) / 2 + i] * bvg[j];
    sm.z[i] = static_cast<float>(acc);
  }
  __syncwarp();
  float rr = 0.f;
  float4* rg = reinterpret_cast<float4*>(ws.R32 + static_cast<size_t>(b) * ws.Mp);
  for (int q = lane; q < M4; q += 32) {
    float4 r = reinterpret_cast<const float4*>(sm.y)[q];
    for (int i = 0; i < n; ++i) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(ws.A32 + static_cast<size_t>(supg[i]) * ws.Mp) + q);
      const float xi = sm.z[i];
      r.x = fmaf(-xi, a.x, r.x);
      r.y = fmaf(-xi, a.y, r.y);
      r.z = fmaf(-xi, a.z, r.z);
      r.w = fmaf(-xi, a.w, r.w);
    }
    rg[q] = r;
    rr += r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rr += __shfl_xor_sync(0xffffffffu, rr, o);
  if (lane == 0) {
    ws.niter[b] = n;
    ws.rnorm[b] = sqrtf(rr);
    fallback[b] = fb;
    const bool cont = fb >= 0 && n < S;
    ws.flag[b] = cont ? 1 : 0;
    ws.stop[b] = fb >= 0 ? kStopIters : stop;
  }
}

}  // namespace

size_t restricted_smem_per_signal(int S, int K, int Mp) { return rs_bytes(S, K, Mp); }

bool launch_restricted(const Ws& ws, const CallArgs* args, const int* cand, int K, const float* tau,
                       int B, int S, float eps, int eps_rel, int* fallback, cudaStream_t s) {
  if (K > 32 * kMaxCandPerLane) return false;
  const size_t per = rs_bytes(S, K, ws.Mp);
  int per_cta = static_cast<int>((200 * 1024) / per);
  if (per_cta < 1) return false;
  if (per_cta > 8) per_cta = 8;
  const size_t smem = per * per_cta;
  if (raise_smem_limit(reinterpret_cast<const void*>(restricted_kernel), smem) != cudaSuccess) return false;
  restricted_kernel<<<(B + per_cta - 1) / per_cta, 32 * per_cta, smem, s>>>(ws, args, cand, K, tau, B, S, eps,
                                                                             eps_rel, fallback);
  return cudaGetLastError() == cudaSuccess;
}

}  // namespace ompk
