// Gram-space OMP over the whole dictionary: the paper's v0 family (Sec. 2.3, projections
// updated through the Gram matrix instead of a correlation GEMM per step), for dictionaries
// whose Gram matrix is small (N up to a few thousand atoms, so G = A^T A stays in L2).
//
// One warp runs all iterations of one signal:
//   c      = A^T y                           FP32, from one batched SIMT GEMM before the loop
//   per step k (0-based; the paper's k+1):
//     n*   = argmax_n |c_n| / ||a_n||        lowest atom index on ties (Alg. 1)
//     w    = G[n*, S]                        the Gram row of n* at the support (Sec. 2.2)
//     z    = F^T w,  delta = ||a_{n*}||^2 - ||z||^2 (FP64); dependent if delta <= 1e-10 ||a||^2
//     gamma = 1 / sqrt(delta),  F[:,k] = [-gamma F z ; gamma]        (Sec. 2.3)
//     b_k  = q_k^T r_{k-1} = gamma c_{n*}    (c on the old support is 0: r is orthogonal to it)
//     c   <- c - b_k A^T q_k,  A^T q_k = sum_j F[j,k] G[:, s_j]   ((k+1) Gram rows, G symmetric)
//     ||r_k||^2 = ||r_{k-1}||^2 - b_k^2 (FP64), eps stop after the update
// so no step touches A or the residual, except that near the eps threshold the stop test forms
// the residual from the support (the running ||r||^2 carries the FP32 error of the b_k). At the
// end x = F b (FP64) and the residual r = y - A_S x is materialised for the reported norm.
// c lives in shared memory, and so does the support's FP32 factor (the triangular products z
// and F z read it there); the FP64 factor and b go to the same per-signal arrays the dense loop
// uses, so finalize is shared.
//
// Per signal and step the work is (k+1) N FMAs on Gram rows read from L2 (shared by all
// signals), against the dense loop's 2 M N tensor-core FLOPs, 8 rescoring rows and k+1 gathered
// atom rows of M floats: the Gram form wins when N is small next to M. A warp per signal keeps
// about 32 signals resident per SM (shared memory permitting), which the Gram-row reads need to
// reach L2 bandwidth: one signal's chain of dependent steps leaves its warp mostly waiting.
#include "common.cuh"

namespace ompk {
namespace {

constexpr int kWarpsPerBlock = 1;  // one signal per block: residency is set by registers and smem
constexpr int kPanel = 512;        // atoms per pass of the c update: 4 float4 per lane

struct GSmem {
  float* c;    // Np4: current correlations (N rounded up to 4, tail zero)
  float* Fs;   // S (S + 1) / 2: FP32 copy of the packed factor, column j at j (j + 1) / 2
  float* w;    // S: Gram row of n* at the support
  float* z;    // S: F^T w, then x
  float* f;    // S + 1: the new factor column
  int* sup;    // S: support in selection order
};

__host__ __device__ __forceinline__ int np4(int N) { return (N + 3) / 4 * 4; }

__host__ __device__ __forceinline__ size_t gs_bytes(int N, int S) {
  size_t b = static_cast<size_t>(np4(N)) * 4 + static_cast<size_t>(S) * (S + 1) / 2 * 4 +
             static_cast<size_t>(S) * 4 * 2 + static_cast<size_t>(S + 1) * 4 + static_cast<size_t>(S) * 4;
  return (b + 15) / 16 * 16;
}

__device__ __forceinline__ GSmem gs_layout(unsigned char* base, int N, int S) {
  GSmem g;
  g.c = reinterpret_cast<float*>(base);
  g.Fs = g.c + np4(N);
  g.w = g.Fs + static_cast<size_t>(S) * (S + 1) / 2;
  g.z = g.w + S;
  g.f = g.z + S;
  g.sup = reinterpret_cast<int*>(g.f + S + 1);
  return g;
}

// ||y - A_S x||^2 for the first n picks, x = F b (FP64 back-substitution into g.z); with `store`
// the residual replaces y in R32. Called by the whole warp.
__device__ double residual_norm2(const Ws& ws, const GSmem& g, const double* Fg, const double* bvg,
                                 int b, int n, bool store, int lane) {
  for (int i = lane; i < n; i += 32) {
    double acc = 0.0;
    for (int j = i; j < n; ++j) acc += Fg[static_cast<size_t>(j) * (j + 1) / 2 + i] * bvg[j];
    g.z[i] = static_cast<float>(acc);
  }
  __syncwarp();
  const int M4 = ws.Mp >> 2;
  float4* rg = reinterpret_cast<float4*>(ws.R32 + static_cast<size_t>(b) * ws.Mp);  // holds y
  double rr = 0.0;
  for (int q = lane; q < M4; q += 32) {
    float4 r = rg[q];
    for (int i = 0; i < n; ++i) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(ws.A32 + static_cast<size_t>(g.sup[i]) * ws.Mp) + q);
      const float xi = g.z[i];
      r.x = fmaf(-xi, a.x, r.x);
      r.y = fmaf(-xi, a.y, r.y);
      r.z = fmaf(-xi, a.z, r.z);
      r.w = fmaf(-xi, a.w, r.w);
    }
    if (store) rg[q] = r;
    rr += static_cast<double>(r.x) * r.x + static_cast<double>(r.y) * r.y +
          static_cast<double>(r.z) * r.z + static_cast<double>(r.w) * r.w;
  }
  __syncwarp();
  return warp_sum(rr);
}

__global__ void __launch_bounds__(32 * kWarpsPerBlock) gram_solve_kernel(Ws ws, int B, int S, float eps,
                                                                        int eps_rel) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int b = blockIdx.x * kWarpsPerBlock + wib;
  if (b >= B) return;  // the whole warp leaves; warps of a block never wait on each other
  const int N = ws.N;
  GSmem g = gs_layout(smem + static_cast<size_t>(wib) * gs_bytes(N, S), N, S);
  const float yn = ws.ynorm[b];
  // y == 0 or non-finite: the init kernel left an empty support (stop code 3)
  if (!(yn > 0.f) || ws.flag[b] == 0) return;
  int* supg = ws.sup + static_cast<size_t>(b) * ws.Smax;
  double* bvg = ws.bv + static_cast<size_t>(b) * ws.Smax;
  double* Fg = ws.F + static_cast<size_t>(b) * ws.Fstride;
  float* Ff = ws.F32 + static_cast<size_t>(b) * ws.Fstride;
  const float* c0 = ws.c0 + static_cast<size_t>(b) * N;
  for (int n = lane; n < np4(N); n += 32) g.c[n] = n < N ? c0[n] : 0.f;
  __syncwarp();
  const bool vec = (N & 3) == 0;  // Gram rows start 16-byte aligned

  double r2 = static_cast<double>(yn) * static_cast<double>(yn);
  const double thr = eps_rel ? static_cast<double>(eps) * static_cast<double>(yn) : static_cast<double>(eps);
  int k = 0;
  int stop = kStopIters;
  for (; k < S; ++k) {
    // ---- n* = argmax |c_n| / ||a_n||: lane l scans atoms 4l + 128p + {0..3}, ascending with a
    // strict '>' (lowest index first), then the warp reduction keeps the lower index on ties
    float bs = -1.f;
    int bi = 0x7fffffff;
    for (int n0 = 4 * lane; n0 < N; n0 += 128) {
      const float4 cv = *reinterpret_cast<const float4*>(g.c + n0);
      const float cq[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int n = n0 + q;
        if (n < N) {
          const float sc = fabsf(cq[q]) * __ldg(ws.inv_norm + n);
          if (sc > bs) {
            bs = sc;
            bi = n;
          }
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float os = __shfl_xor_sync(0xffffffffu, bs, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (better(os, oi, bs, bi)) {
        bs = os;
        bi = oi;
      }
    }
    const int ns = bi;
    if (ns < 0 || ns >= N) {  // no finite score
      if (lane == 0) atomicOr(ws.err, OMP_DEVERR_BAD_STATE);
      break;
    }
    // ---- w_i = G[n*, s_i]
    const float* grow = ws.gram + static_cast<size_t>(ns) * N;
    for (int i = lane; i < k; i += 32) g.w[i] = __ldg(grow + g.sup[i]);
    const double nrm2 = ws.norm2[ns];
    const float cn = g.c[ns];
    __syncwarp();
    // ---- z_j = sum_{i<=j} F[i,j] w_i (lane j, j + 32, ...), ||z||^2 in FP64
    double zz = 0.0;
    for (int j = lane; j < k; j += 32) {
      const float* col = g.Fs + static_cast<size_t>(j) * (j + 1) / 2;
      float zj = 0.f;
      for (int i = 0; i <= j; ++i) zj = fmaf(col[i], g.w[i], zj);
      g.z[j] = zj;
      zz += static_cast<double>(zj) * zj;
    }
    zz = warp_sum(zz);
    const double delta = nrm2 - zz;
    if (!(delta > kDepRtol * nrm2)) {
      stop = kStopDependent;
      break;
    }
    const double gamma = 1.0 / sqrt(delta);
    __syncwarp();
    // ---- F[:,k] = [-gamma F z ; gamma]: u_i = sum_{j>=i} F[i,j] z_j (lane i, i + 32, ...)
    const size_t off = static_cast<size_t>(k) * (k + 1) / 2;
    for (int i = lane; i < k; i += 32) {
      float u = 0.f;
      for (int j = i; j < k; ++j) u = fmaf(g.Fs[static_cast<size_t>(j) * (j + 1) / 2 + i], g.z[j], u);
      const double fv = -gamma * static_cast<double>(u);
      const float f32 = static_cast<float>(fv);
      g.f[i] = f32;
      g.Fs[off + i] = f32;
      Fg[off + i] = fv;
      Ff[off + i] = f32;
    }
    if (lane == 0) {
      const float gf = static_cast<float>(gamma);
      g.f[k] = gf;
      g.Fs[off + k] = gf;
      Fg[off + k] = gamma;
      Ff[off + k] = gf;
      g.sup[k] = ns;
      supg[k] = ns;
    }
    __syncwarp();
    const double bk = gamma * static_cast<double>(cn);
    // ---- c <- c - b_k sum_j f_j G[s_j, :], in panels of kPanel atoms: lane l takes 4 atoms
    // per 128, 16-byte Gram loads (scalar ones when N is not a multiple of 4)
    const float bf = static_cast<float>(bk);
    for (int p0 = 0; p0 < N; p0 += kPanel) {
      float4 acc[kPanel / 128];
#pragma unroll
      for (int t = 0; t < kPanel / 128; ++t) acc[t] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 2
      for (int a = 0; a <= k; ++a) {
        const float fa = g.f[a];
        const float* gr = ws.gram + static_cast<size_t>(g.sup[a]) * N;
#pragma unroll
        for (int t = 0; t < kPanel / 128; ++t) {
          const int n0 = p0 + 128 * t + 4 * lane;
          if (n0 < N) {
            float4 gv;
            if (vec) {
              gv = __ldg(reinterpret_cast<const float4*>(gr + n0));
            } else {
              gv.x = __ldg(gr + n0);
              gv.y = n0 + 1 < N ? __ldg(gr + n0 + 1) : 0.f;
              gv.z = n0 + 2 < N ? __ldg(gr + n0 + 2) : 0.f;
              gv.w = n0 + 3 < N ? __ldg(gr + n0 + 3) : 0.f;
            }
            acc[t].x = fmaf(fa, gv.x, acc[t].x);
            acc[t].y = fmaf(fa, gv.y, acc[t].y);
            acc[t].z = fmaf(fa, gv.z, acc[t].z);
            acc[t].w = fmaf(fa, gv.w, acc[t].w);
          }
        }
      }
#pragma unroll
      for (int t = 0; t < kPanel / 128; ++t) {
        const int n0 = p0 + 128 * t + 4 * lane;
        if (n0 < N) {
          float4* cp = reinterpret_cast<float4*>(g.c + n0);
          float4 cv = *cp;
          cv.x = fmaf(-bf, acc[t].x, cv.x);
          cv.y = fmaf(-bf, acc[t].y, cv.y);
          cv.z = fmaf(-bf, acc[t].z, cv.z);
          cv.w = fmaf(-bf, acc[t].w, cv.w);
          *cp = cv;  // the tail beyond N only ever holds zeros times zeros
        }
      }
    }
    const double r2prev = r2;
    r2 -= bk * bk;
    if (lane == 0) {
      bvg[k] = bk;
      ws.drop[static_cast<size_t>(b) * ws.Smax + k] = r2prev > 0.0 ? static_cast<float>((bk * bk) / r2prev) : 0.f;
    }
    __syncwarp();  // c updated before the next selection
    // The running ||r||^2 carries the FP32 error of the b_k (about k 2^-24 ||y||^2), so near
    // the threshold the stop test uses the residual itself, formed from the support.
    if (thr > 0.0 && r2 <= 4.0 * thr * thr + 2e-5 * static_cast<double>(yn) * yn) {
      const double rr = residual_norm2(ws, g, Fg, bvg, b, k + 1, false, lane);
      if (rr <= thr * thr) {
        stop = kStopEps;
        ++k;
        break;
      }
    }
  }

  // ---- x = F b, r = y - A_S x (stored) and its norm
  const int n_it = k;
  const double rr = residual_norm2(ws, g, Fg, bvg, b, n_it, true, lane);
  if (lane == 0) {
    ws.niter[b] = n_it;
    ws.rnorm[b] = static_cast<float>(sqrt(rr));
    ws.stop[b] = stop;
    ws.flag[b] = 0;
  }
}

}  // namespace

cudaError_t configure_gram_solve(const Ws& ws) {
  const size_t bytes = gs_bytes(ws.N, ws.Smax) * kWarpsPerBlock;
  if (bytes > 227 * 1024) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(gram_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(bytes));
}

void launch_gram_solve(const Ws& ws, const CallArgs*, int B, int S, float eps, int eps_rel,
                       cudaStream_t s) {
  gram_solve_kernel<<<(B + kWarpsPerBlock - 1) / kWarpsPerBlock, 32 * kWarpsPerBlock,
                      gs_bytes(ws.N, S) * kWarpsPerBlock, s>>>(ws, B, S, eps, eps_rel);
}

}  // namespace ompk
