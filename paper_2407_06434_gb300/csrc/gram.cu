// Gram-space OMP over the whole dictionary: the paper's v0 family (Sec. 2.3, projections
// updated through the Gram matrix instead of a correlation GEMM per step), for dictionaries
// whose Gram matrix is small (N up to a few thousand atoms, so G = A^T A stays in L2).
//
// One block of W warps (W = 1 for up to 1536 atoms and a batch of at least 32 signals per SM,
// 8 otherwise) runs all iterations of one
// signal:
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
// atom rows of M floats: the Gram form wins when N is small next to M. Small blocks keep many
// signals resident per SM (shared memory permitting), which the Gram-row reads need to reach L2
// bandwidth, since one signal's chain of dependent steps leaves its warps mostly waiting; a
// larger N shortens each signal's argmax and c update with more warps.
#include "common.cuh"

namespace ompk {
namespace {


struct GSmem {
  double* rd;  // 12: block reduction scratch [0, 8); the step's gamma [8], b_k [9], and whether
               // the running ||r||^2 is near the threshold [10], formed by thread 0
  float* rs;   // 8: per-warp best scores
  int* ri;     // 9: per-warp best atoms, then the block's
  float* c;    // Np4: current correlations (N rounded up to 4, tail zero)
  float* Fs;   // S (S + 1) / 2: FP32 copy of the packed factor, column j at j (j + 1) / 2
  float* w;    // S: Gram row of n* at the support
  float* z;    // S: F^T w, then x
  float* f;    // S + 1: the new factor column
  int* sup;    // S: support in selection order
};

__host__ __device__ __forceinline__ int np4(int N) { return (N + 3) / 4 * 4; }

__host__ __device__ __forceinline__ size_t gs_bytes(int N, int S) {
  size_t b = 12 * 8 + 8 * 4 + 9 * 4 + 12 + static_cast<size_t>(np4(N)) * 4 +
             static_cast<size_t>(S) * (S + 1) / 2 * 4 + static_cast<size_t>(S) * 4 * 2 +
             static_cast<size_t>(S + 1) * 4 + static_cast<size_t>(S) * 4;
  return (b + 15) / 16 * 16;
}

__device__ __forceinline__ GSmem gs_layout(unsigned char* base, int N, int S) {
  GSmem g;
  g.rd = reinterpret_cast<double*>(base);
  g.rs = reinterpret_cast<float*>(base + 12 * 8);
  g.ri = reinterpret_cast<int*>(g.rs + 8);
  g.c = reinterpret_cast<float*>(base + 12 * 8 + 8 * 4 + 9 * 4 + 12);  // 16-byte aligned
  g.Fs = g.c + np4(N);
  g.w = g.Fs + static_cast<size_t>(S) * (S + 1) / 2;
  g.z = g.w + S;
  g.f = g.z + S;
  g.sup = reinterpret_cast<int*>(g.f + S + 1);
  return g;
}

template <int W>
__device__ __forceinline__ void bsync() {
  if (W == 1)
    __syncwarp();
  else
    __syncthreads();
}

// Sum over the block's W warps; every thread gets the total.
template <int W>
__device__ __forceinline__ double bsum(double v, double* red) {
  v = warp_sum(v);
  if (W == 1) return v;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int i = 0; i < W; ++i) t += red[i];
  __syncthreads();
  return t;
}

// Sum of the block's (hi, lo) pairs (each an unevaluated FP32 sum), as a double; every thread
// gets the total.
template <int W>
__device__ __forceinline__ double bsum2(float hi, float lo, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
    lo = __fadd_rn(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    two_sum(hi, lo, oh);
  }
  if (W > 1) {
    float* rf = reinterpret_cast<float*>(red);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
      rf[2 * warp] = hi;
      rf[2 * warp + 1] = lo;
    }
    __syncthreads();
    hi = rf[0];
    lo = rf[1];
#pragma unroll
    for (int i = 1; i < W; ++i) {
      lo = __fadd_rn(lo, rf[2 * i + 1]);
      two_sum(hi, lo, rf[2 * i]);
    }
    __syncthreads();
  }
  return static_cast<double>(hi) + static_cast<double>(lo);
}

// ||y - A_S x||^2 for the first n picks, x = F b (FP64 back-substitution into g.z); with `store`
// the residual replaces y in R32. Called by the whole block.
template <int W>
__device__ double residual_norm2(const Ws& ws, const GSmem& g, const double* Fg, const double* bvg,
                                 int b, int n, bool store) {
  const int tid = threadIdx.x;
  for (int i = tid; i < n; i += 32 * W) {
    double acc = 0.0;
    for (int j = i; j < n; ++j) acc += Fg[static_cast<size_t>(j) * (j + 1) / 2 + i] * bvg[j];
    g.z[i] = static_cast<float>(acc);
  }
  bsync<W>();
  const int M4 = ws.Mp >> 2;
  float4* rg = reinterpret_cast<float4*>(ws.R32 + static_cast<size_t>(b) * ws.Mp);  // holds y
  double rr = 0.0;
  for (int q = tid; q < M4; q += 32 * W) {
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
  bsync<W>();
  return bsum<W>(rr, g.rd);
}

template <int W>
__global__ void __launch_bounds__(32 * W) gram_solve_kernel(Ws ws, int B, int S, float eps, int eps_rel) {
  constexpr int T = 32 * W;
  // c update shape: a lone warp keeps 4 float4 accumulators and 2 Gram rows in flight; wider
  // blocks spread the atoms thinner (one float4 per thread) and keep 8 rows in flight
  constexpr int VP = W == 1 ? 4 : 1;
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = blockIdx.x;
  if (b >= B) return;  // the whole block leaves
  const int N = ws.N;
  GSmem g = gs_layout(smem, N, S);
  const float yn = ws.ynorm[b];
  // y == 0 or non-finite: the init kernel left an empty support (stop code 3)
  if (!(yn > 0.f) || ws.flag[b] == 0) return;
  int* supg = ws.sup + static_cast<size_t>(b) * ws.Smax;
  double* bvg = ws.bv + static_cast<size_t>(b) * ws.Smax;
  double* Fg = ws.F + static_cast<size_t>(b) * ws.Fstride;
  float* Ff = ws.F32 + static_cast<size_t>(b) * ws.Fstride;
  const float* c0 = ws.c0 + static_cast<size_t>(b) * N;
  for (int n = tid; n < np4(N); n += T) g.c[n] = n < N ? c0[n] : 0.f;
  bsync<W>();
  const bool vec = (N & 3) == 0;  // Gram rows start 16-byte aligned

  double r2 = static_cast<double>(yn) * static_cast<double>(yn);
  const double thr = eps_rel ? static_cast<double>(eps) * static_cast<double>(yn) : static_cast<double>(eps);
  int k = 0;
  int stop = kStopIters;
  for (; k < S; ++k) {
    // ---- n* = argmax |c_n| / ||a_n||: thread t scans atoms 4t + 4Tp + {0..3}, ascending with a
    // strict '>' (lowest index first), then the reductions keep the lower index on ties
    float bs = -1.f;
    int bi = 0x7fffffff;
    for (int n0 = 4 * tid; n0 < N; n0 += 4 * T) {
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
    if (W > 1) {
      if (lane == 0) {
        g.rs[warp] = bs;
        g.ri[warp] = bi;
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < W; ++i)
        if (better(g.rs[i], g.ri[i], bs, bi)) {
          bs = g.rs[i];
          bi = g.ri[i];
        }
      __syncthreads();
    }
    const int ns = bi;
    if (ns < 0 || ns >= N) {  // no finite score
      if (tid == 0) atomicOr(ws.err, OMP_DEVERR_BAD_STATE);
      break;
    }
    // ---- w_i = G[n*, s_i]
    const float* grow = ws.gram + static_cast<size_t>(ns) * N;
    for (int i = tid; i < k; i += T) g.w[i] = __ldg(grow + g.sup[i]);
    const double nrm2 = ws.norm2[ns];
    const float cn = g.c[ns];
    bsync<W>();
    // ---- z_j = sum_{i<=j} F[i,j] w_i (thread j, j + T, ...); ||z||^2 as an exact FP32
    // double-float sum (squares split by an FMA, two-sum additions), which carries it far
    // beyond the FP32 accuracy of z without FP64 arithmetic per thread
    float zh = 0.f, zlo = 0.f;
    for (int j = tid; j < k; j += T) {
      const float* col = g.Fs + static_cast<size_t>(j) * (j + 1) / 2;
      float zj = 0.f;
      for (int i = 0; i <= j; ++i) zj = fmaf(col[i], g.w[i], zj);
      g.z[j] = zj;
      const float p = __fmul_rn(zj, zj);
      zlo = __fadd_rn(zlo, fmaf(zj, zj, -p));
      two_sum(zh, zlo, p);
    }
    const double zz = bsum2<W>(zh, zlo, g.rd);  // (its barrier also publishes z)
    // The step's scalars, formed once by thread 0 (GB300 issues FP64 at a small fraction of
    // its FP32 rate, so the block does not repeat it): gamma = 1/sqrt(delta) from an FP32
    // reciprocal square root seed and one FP64 Newton-Raphson step (0 for a dependent atom),
    // b_k = gamma c_n*, the running ||r||^2 and whether it has come near the threshold.
    if (tid == 0) {
      const double delta = nrm2 - zz;
      double gamma = 0.0, bk = 0.0;
      if (delta > kDepRtol * nrm2) {
        if (delta > 1e-36 && delta < 1e36) {
          const double y0 = static_cast<double>(rsqrtf(static_cast<float>(delta)));
          gamma = y0 * (1.5 - 0.5 * delta * y0 * y0);
        } else {
          gamma = 1.0 / sqrt(delta);
        }
        bk = gamma * static_cast<double>(cn);
        const double r2prev = r2;
        r2 -= bk * bk;
        bvg[k] = bk;
        ws.drop[static_cast<size_t>(b) * ws.Smax + k] = r2prev > 0.0 ? static_cast<float>((bk * bk) / r2prev) : 0.f;
      }
      g.rd[8] = gamma;
      g.rd[9] = bk;
      g.rd[10] = thr > 0.0 && r2 <= 4.0 * thr * thr + 2e-5 * static_cast<double>(yn) * yn ? 1.0 : 0.0;
    }
    bsync<W>();
    const double gamma = g.rd[8];
    if (!(gamma > 0.0)) {
      stop = kStopDependent;
      break;
    }
    // ---- F[:,k] = [-gamma F z ; gamma]: u_i = sum_{j>=i} F[i,j] z_j (thread i, i + T, ...)
    const size_t off = static_cast<size_t>(k) * (k + 1) / 2;
    for (int i = tid; i < k; i += T) {
      float u = 0.f;
      for (int j = i; j < k; ++j) u = fmaf(g.Fs[static_cast<size_t>(j) * (j + 1) / 2 + i], g.z[j], u);
      const double fv = -gamma * static_cast<double>(u);
      const float f32 = static_cast<float>(fv);
      g.f[i] = f32;
      g.Fs[off + i] = f32;
      Fg[off + i] = fv;
      Ff[off + i] = f32;
    }
    if (tid == 0) {
      const float gf = static_cast<float>(gamma);
      g.f[k] = gf;
      g.Fs[off + k] = gf;
      Fg[off + k] = gamma;
      Ff[off + k] = gf;
      g.sup[k] = ns;
      supg[k] = ns;
    }
    bsync<W>();
    // ---- c <- c - b_k sum_j f_j G[s_j, :], in panels: thread t takes 4 atoms per 4T, 16-byte
    // Gram loads (scalar ones when N is not a multiple of 4)
    const float bf = static_cast<float>(g.rd[9]);
    for (int p0 = 0; p0 < N; p0 += 4 * T * VP) {
      float4 acc[VP];
#pragma unroll
      for (int t = 0; t < VP; ++t) acc[t] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll (W == 1 ? 2 : 8)
      for (int a = 0; a <= k; ++a) {
        const float fa = g.f[a];
        const float* gr = ws.gram + static_cast<size_t>(g.sup[a]) * N;
#pragma unroll
        for (int t = 0; t < VP; ++t) {
          const int n0 = p0 + 4 * T * t + 4 * tid;
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
      for (int t = 0; t < VP; ++t) {
        const int n0 = p0 + 4 * T * t + 4 * tid;
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
    bsync<W>();  // c updated before the next selection
    // The running ||r||^2 carries the FP32 error of the b_k (about k 2^-24 ||y||^2), so near
    // the threshold the stop test uses the residual itself, formed from the support.
    if (g.rd[10] != 0.0) {
      const double rr = residual_norm2<W>(ws, g, Fg, bvg, b, k + 1, false);
      if (rr <= thr * thr) {
        stop = kStopEps;
        ++k;
        break;
      }
    }
  }

  // ---- x = F b, r = y - A_S x (stored) and its norm
  const int n_it = k;
  const double rr = residual_norm2<W>(ws, g, Fg, bvg, b, n_it, true);
  if (tid == 0) {
    ws.niter[b] = n_it;
    ws.rnorm[b] = static_cast<float>(sqrt(rr));
    ws.stop[b] = stop;
    ws.flag[b] = 0;
  }
}

// warps per signal: one for small dictionaries when the batch fills the GPU with one-warp
// signals (16 per SM), eight otherwise (a larger N shortens each signal's argmax and c update;
// a small batch needs the parallelism within each signal)
int gram_warps(int N, int B, int sms) { return (N <= 1536 && B >= 2 * 16 * sms) ? 1 : 8; }

template <int W>
cudaError_t set_attr(size_t bytes) {
  return raise_smem_limit(reinterpret_cast<const void*>(gram_solve_kernel<W>), bytes);
}

}  // namespace

cudaError_t configure_gram_solve(const Ws& ws) {
  const size_t bytes = gs_bytes(ws.N, ws.Smax);
  if (bytes > 227 * 1024) return cudaErrorInvalidValue;
  const cudaError_t e = set_attr<1>(bytes);
  return e == cudaSuccess ? set_attr<8>(bytes) : e;
}

void launch_gram_solve(const Ws& ws, const CallArgs*, int B, int S, float eps, int eps_rel,
                       cudaStream_t s) {
  const size_t smem = gs_bytes(ws.N, S);
  if (gram_warps(ws.N, B, ws.tc_grid > 0 ? ws.tc_grid : 152) == 1)
    gram_solve_kernel<1><<<B, 32, smem, s>>>(ws, B, S, eps, eps_rel);
  else
    gram_solve_kernel<8><<<B, 256, smem, s>>>(ws, B, S, eps, eps_rel);
}

}  // namespace ompk
