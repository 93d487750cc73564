// Candidate-restricted OMP iteration for the learned proposal: one 256-thread block per signal,
// one candidate per thread.
//
// Given K <= 256 candidate atoms per signal (from the proposal network), the iteration runs the
// paper's v0 scheme (Sec. 2.3: "D_k = A^T A_k F_k", projections updated by one vector per step)
// restricted to the candidates, so no per-step correlation with the whole dictionary is needed:
//   c      = A_K^T y                        exact FP32 dot products of the K candidate rows
//   per step k:
//     n*   = argmax_i |c_i| / ||a_i||        lowest atom index on ties
//     z    = Q^T a_{n*}, read from D        (D row j = A_K^T q_j, so z_j = D[j][n*])
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
//
// Layout: thread i owns candidate slot i (its atom, inverse norm and correlation c_i in
// registers); D (S x K FP32), the FP32 factor, y and the step's scalars are in shared memory.
// A block per signal (rather than a warp) spreads the K-wide work of a step over 8 warps and
// keeps the per-signal shared memory (S K floats) the only limit on residency.
#include "common.cuh"

namespace ompk {
namespace {

constexpr int kRThreads = 256;  // = the largest K
constexpr int kRWarps = kRThreads / 32;

struct RSmem {
  float* D;      // S x K: D[j * K + i]
  float* Fs;     // S (S + 1) / 2, packed by columns
  float* y;      // Mp
  float* z;      // S
  float* xs;     // S: coefficients for the final residual
  float* wred;   // kRWarps: per-warp scores
  float* wc;     // kRWarps: per-warp correlations of those
  int* wati;     // kRWarps: per-warp atoms
  int* wslot;    // kRWarps: per-warp slots
  double* dred;  // kRWarps: per-warp FP64 partials
  int* ctl;      // 4: picked slot, picked atom, stop flag
  double* bk;    // 1: b_k of the step
};

// Floats first (y at the 16-byte aligned base: Mp is a multiple of 64, so every float array
// after it stays 4-byte aligned and y keeps its float4 alignment), then the ints, then the
// doubles at the next 8-byte boundary.
__host__ __device__ __forceinline__ size_t rs_float_words(int S, int K, int Mp) {
  return static_cast<size_t>(Mp) + static_cast<size_t>(S) * K +
         static_cast<size_t>(S) * (S + 1) / 2 + 2 * static_cast<size_t>(S) + 2 * kRWarps;
}

__host__ __device__ __forceinline__ size_t rs_bytes(int S, int K, int Mp) {
  const size_t ints = (rs_float_words(S, K, Mp) + 2 * kRWarps + 4) * 4;
  return (ints + 7) / 8 * 8 + (kRWarps + 1) * 8;
}

__device__ __forceinline__ RSmem rs_smem(unsigned char* base, int S, int K, int Mp) {
  RSmem s;
  s.y = reinterpret_cast<float*>(base);
  s.D = s.y + Mp;
  s.Fs = s.D + static_cast<size_t>(S) * K;
  s.z = s.Fs + static_cast<size_t>(S) * (S + 1) / 2;
  s.xs = s.z + S;
  s.wred = s.xs + S;
  s.wc = s.wred + kRWarps;
  s.wati = reinterpret_cast<int*>(s.wc + kRWarps);
  s.wslot = s.wati + kRWarps;
  s.ctl = s.wslot + kRWarps;
  const size_t ints = (rs_float_words(S, K, Mp) + 2 * kRWarps + 4) * 4;
  s.dred = reinterpret_cast<double*>(base + (ints + 7) / 8 * 8);
  s.bk = s.dred + kRWarps;
  return s;
}

__global__ void __launch_bounds__(kRThreads)
    restricted_kernel(Ws ws, const CallArgs* args, const int* __restrict__ cand, int K,
                      const float* __restrict__ tau, int B, int S, float eps, int eps_rel,
                      int* __restrict__ fallback) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = blockIdx.x;
  if (b >= B) return;
  RSmem sm = rs_smem(smem, S, K, ws.Mp);
  const float yn = ws.ynorm[b];
  const int* cb = cand + static_cast<size_t>(b) * K;
  int* supg = ws.sup + static_cast<size_t>(b) * ws.Smax;
  double* bvg = ws.bv + static_cast<size_t>(b) * ws.Smax;
  if (!(yn > 0.f)) {  // y == 0 or non-finite: handled by init (empty support, not live)
    if (tid == 0) {
      ws.flag[b] = 0;
      fallback[b] = -1;
    }
    return;
  }
  const int M4 = ws.Mp >> 2;
  const float* yg = args->Y + static_cast<size_t>(b) * ws.M;
  for (int m = tid; m < ws.Mp; m += kRThreads) sm.y[m] = m < ws.M ? yg[m] : 0.f;
  // this thread's candidate
  const bool has = tid < K;
  const int atom = has ? cb[tid] : -1;
  const bool valid = has && atom >= 0 && atom < ws.N;
  const float inv = valid ? __ldg(ws.inv_norm + atom) : 0.f;
  __syncthreads();
  // c_i = a_i^T y (FP32): each warp takes every 8th candidate, lanes over the signal; four
  // candidates' rows, four float4 slots of each, in flight at a time
  for (int i0 = warp; i0 < K; i0 += 4 * kRWarps) {
    const float4* ar[4];
    bool okr[4];
#pragma unroll
    for (int c4 = 0; c4 < 4; ++c4) {
      const int i = i0 + c4 * kRWarps;
      const int n = i < K ? cb[i] : -1;
      okr[c4] = n >= 0 && n < ws.N;
      ar[c4] = reinterpret_cast<const float4*>(ws.A32 + static_cast<size_t>(okr[c4] ? n : 0) * ws.Mp);
    }
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int q0 = lane; q0 < M4; q0 += 128) {
      float4 av[4][4];
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = q0 + 32 * u;
          av[c4][u] = okr[c4] && q < M4 ? __ldg(ar[c4] + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = q0 + 32 * u;
        const float4 y4 = q < M4 ? reinterpret_cast<const float4*>(sm.y)[q] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4)
          acc[c4] += av[c4][u].x * y4.x + av[c4][u].y * y4.y + av[c4][u].z * y4.z + av[c4][u].w * y4.w;
      }
    }
#pragma unroll
    for (int c4 = 0; c4 < 4; ++c4) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[c4] += __shfl_xor_sync(0xffffffffu, acc[c4], o);
      const int i = i0 + c4 * kRWarps;
      if (lane == 0 && i < K) sm.D[i] = acc[c4];  // staged in D's first row until the loop starts
    }
  }
  __syncthreads();
  float c = has ? sm.D[tid] : 0.f;
  __syncthreads();

  double r2 = static_cast<double>(yn) * static_cast<double>(yn);
  const double thr = eps_rel ? static_cast<double>(eps) * yn : static_cast<double>(eps);
  int k = 0;
  int fb = -1;
  int stop = kStopIters;
  for (; k < S; ++k) {
    // ---- pick: argmax |c_i| / ||a_i||, lowest atom index on ties
    float bs = valid ? fabsf(c) * inv : -1.f;
    float bc = c;  // the best's correlation travels with it (b_k = gamma c_{n*})
    int bi = valid ? atom : 0x7fffffff, bslot = valid ? tid : -1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float os = __shfl_xor_sync(0xffffffffu, bs, o);
      const float oc = __shfl_xor_sync(0xffffffffu, bc, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      const int osl = __shfl_xor_sync(0xffffffffu, bslot, o);
      if (better(os, oi, bs, bi)) {
        bs = os;
        bc = oc;
        bi = oi;
        bslot = osl;
      }
    }
    if (lane == 0) {
      sm.wred[warp] = bs;
      sm.wc[warp] = bc;
      sm.wati[warp] = bi;
      sm.wslot[warp] = bslot;
    }
    __syncthreads();
    if (warp == 0) {
      float s2 = lane < kRWarps ? sm.wred[lane] : -1.f;
      float c2 = lane < kRWarps ? sm.wc[lane] : 0.f;
      int i2 = lane < kRWarps ? sm.wati[lane] : 0x7fffffff;
      int l2 = lane < kRWarps ? sm.wslot[lane] : -1;
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        const float os = __shfl_xor_sync(0xffffffffu, s2, o);
        const float oc = __shfl_xor_sync(0xffffffffu, c2, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i2, o);
        const int osl = __shfl_xor_sync(0xffffffffu, l2, o);
        if (better(os, oi, s2, i2)) {
          s2 = os;
          c2 = oc;
          i2 = oi;
          l2 = osl;
        }
      }
      // lanes 0..7 now hold the winner; every lane of the warp needs it for the z loop
      s2 = __shfl_sync(0xffffffffu, s2, 0);
      c2 = __shfl_sync(0xffffffffu, c2, 0);
      i2 = __shfl_sync(0xffffffffu, i2, 0);
      l2 = __shfl_sync(0xffffffffu, l2, 0);
      // ---- z_j = D[j][slot], delta, gamma, the drop check (warp 0; lanes over j)
      const bool ok = s2 > 0.f && i2 >= 0 && i2 < ws.N && l2 >= 0;
      double zz = 0.0;
      if (ok)
        for (int j = lane; j < k; j += 32) {
          const float zj = sm.D[static_cast<size_t>(j) * K + l2];
          sm.z[j] = zj;
          zz += static_cast<double>(zj) * zj;
        }
      zz = warp_sum(zz);
      if (lane == 0) {
        int verdict = 0;  // 0: accept, 1: fall back (no positive score, or a dependent atom)
        if (!ok) {
          verdict = 1;
        } else {
          const double nrm2 = ws.norm2[i2];
          const double delta = nrm2 - zz;
          if (!(delta > kDepRtol * nrm2)) {
            verdict = 1;
          } else {
            const double gamma = 1.0 / sqrt(delta);
            sm.dred[0] = gamma;
            sm.bk[0] = gamma * static_cast<double>(c2);  // b_k = gamma c_{n*}
          }
        }
        sm.ctl[0] = l2;
        sm.ctl[1] = i2;
        sm.ctl[2] = verdict;
      }
    }
    __syncthreads();
    if (sm.ctl[2]) {
      fb = k;
      break;
    }
    const int ns = sm.ctl[1];
    const double gamma = sm.dred[0];
    const double bk = sm.bk[0];
    const double drop = (bk * bk) / r2;
    if (drop < static_cast<double>(tau[k])) {
      fb = k;
      break;
    }
    const float gf = static_cast<float>(gamma);
    // ---- new D row and the correlations: thread i, D[k][i] = gamma (G[n*, a_i] - sum_j z_j D[j][i])
    float* Dk = sm.D + static_cast<size_t>(k) * K;
    if (has) {
      float acc = valid ? __ldg(ws.gram + static_cast<size_t>(ns) * ws.N + atom) : 0.f;
      for (int j = 0; j < k; ++j) acc = fmaf(-sm.z[j], sm.D[static_cast<size_t>(j) * K + tid], acc);
      const float d = gf * acc;
      Dk[tid] = d;
      c = fmaf(-static_cast<float>(bk), d, c);
    }
    // ---- F column k = [-gamma F z ; gamma] (FP32 products, FP64 scaling), warp 1
    if (warp == 1) {
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
        supg[k] = ns;
        bvg[k] = bk;
        ws.drop[static_cast<size_t>(b) * ws.Smax + k] = static_cast<float>(drop);
      }
    }
    r2 -= bk * bk;
    __syncthreads();  // D row k, the factor and z are complete before the next step reads them
    if (r2 <= thr * thr) {
      stop = kStopEps;
      ++k;
      break;
    }
  }
  // ---- materialise the residual r = y - A_S x with x = F b (FP64), and its norm
  const int n = k;
  __syncthreads();
  const double* Fb = ws.F + static_cast<size_t>(b) * ws.Fstride;
  if (warp == 0)
    for (int i = lane; i < n; i += 32) {
      double acc = 0.0;
      for (int j = i; j < n; ++j) acc += Fb[static_cast<size_t>(j) * (j + 1) / 2 + i] * bvg[j];
      sm.xs[i] = static_cast<float>(acc);
    }
  __syncthreads();
  float rr = 0.f;
  float4* rg = reinterpret_cast<float4*>(ws.R32 + static_cast<size_t>(b) * ws.Mp);
  for (int q = tid; q < M4; q += kRThreads) {
    float4 r = reinterpret_cast<const float4*>(sm.y)[q];
#pragma unroll 8
    for (int i = 0; i < n; ++i) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(ws.A32 + static_cast<size_t>(supg[i]) * ws.Mp) + q);
      const float xi = sm.xs[i];
      r.x = fmaf(-xi, a.x, r.x);
      r.y = fmaf(-xi, a.y, r.y);
      r.z = fmaf(-xi, a.z, r.z);
      r.w = fmaf(-xi, a.w, r.w);
    }
    rg[q] = r;
    rr += r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w;
  }
  double rd = warp_sum(static_cast<double>(rr));
  if (lane == 0) sm.dred[warp] = rd;
  __syncthreads();
  if (tid == 0) {
    double tot = 0.0;
    for (int w = 0; w < kRWarps; ++w) tot += sm.dred[w];
    ws.niter[b] = n;
    ws.rnorm[b] = static_cast<float>(sqrt(tot));
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
  if (K < 1 || K > kRThreads) return false;
  const size_t smem = rs_bytes(S, K, ws.Mp);
  if (smem > 227 * 1024) return false;
  if (raise_smem_limit(reinterpret_cast<const void*>(restricted_kernel), smem) != cudaSuccess) return false;
  restricted_kernel<<<B, kRThreads, smem, s>>>(ws, args, cand, K, tau, B, S, eps, eps_rel, fallback);
  return cudaGetLastError() == cudaSuccess;
}

}  // namespace ompk
