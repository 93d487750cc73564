// Per-signal kernels around the OMP iteration: initialisation, live-set compaction, the final
// back-substitution x = F b (FP64), and the top-k output of omp_correlate_topk. The per-iteration
// append and residual update is in append.cuh.
#include <mutex>

#include "common.cuh"

namespace ompk {

cudaError_t raise_smem_limit(const void* kernel, size_t bytes) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  if (static_cast<size_t>(fa.maxDynamicSharedSizeBytes) >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
}

// ------------------------------------------------------------------------------------ args
__global__ void set_args_kernel(CallArgs* dst, CallArgs v) { *dst = v; }

void launch_set_args(CallArgs* dst, const CallArgs& v, cudaStream_t s) {
  set_args_kernel<<<1, 1, 0, s>>>(dst, v);
}

// ------------------------------------------------------------------------------------ init
// One warp per signal: r = y (zero padded to Mp), ||y|| in FP64, non-finite check. The signal
// enters the live set unless y == 0 or y has a NaN/Inf. Writes the identity list as the
// "previous" list (live[1], cnt[0] = B) for compaction step 0.
__global__ void __launch_bounds__(256) init_kernel(Ws ws, const CallArgs* args, int B) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (blockIdx.x == 0 && threadIdx.x == 0) *ws.kdev = 0;
  if (blockIdx.x == 0 && ws.upd_ctr)
    for (int i = threadIdx.x; i <= ws.Smax; i += blockDim.x) ws.upd_ctr[i] = 0;
  if (b >= B) return;
  const float* y = args->Y + static_cast<size_t>(b) * ws.M;
  float* r = ws.R32 + static_cast<size_t>(b) * ws.Mp;
  double s = 0.0;
  bool finite = true;
  for (int m = lane; m < ws.Mp; m += 32) {
    const float v = m < ws.M ? y[m] : 0.f;
    finite = finite && isfinite(v);
    r[m] = v;
    s += static_cast<double>(v) * static_cast<double>(v);
  }
  s = warp_sum(s);
  finite = __all_sync(0xffffffffu, finite);
  if (!finite)
    for (int m = lane; m < ws.Mp; m += 32) r[m] = 0.f;
  if (lane == 0) {
    const bool alive = finite && s > 0.0;
    ws.ynorm[b] = finite ? static_cast<float>(sqrt(s)) : 0.f;
    ws.rnorm[b] = ws.ynorm[b];
    ws.niter[b] = 0;
    ws.stop[b] = alive ? kStopIters : kStopZero;
    ws.flag[b] = alive ? 1 : 0;
    ws.fb[b] = -1;
    ws.live[1][b] = b;
    ws.livek[1][b] = 0;
    if (ws.tau) ws.tau[b] = TauRec{0.f, 0.f, -1, 0};
    if (!finite) atomicOr(ws.err, OMP_DEVERR_NONFINITE);
    if (b == 0) ws.cnt[0] = B;
  }
}

void launch_init(const Ws& ws, const CallArgs* args, int B, cudaStream_t s) {
  init_kernel<<<(B + 7) / 8, 256, 0, s>>>(ws, args, B);
}

// Residual rows given directly (omp_correlate_topk): every row is live.
__global__ void __launch_bounds__(256) load_rows_kernel(Ws ws, const float* __restrict__ R, int B) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (b >= B) return;
  const float* x = R + static_cast<size_t>(b) * ws.M;
  float* r = ws.R32 + static_cast<size_t>(b) * ws.Mp;
  for (int m = lane; m < ws.Mp; m += 32) r[m] = m < ws.M ? x[m] : 0.f;
  if (lane == 0) {
    ws.flag[b] = 1;
    ws.live[1][b] = b;
    ws.livek[1][b] = 0;
    if (b == 0) ws.cnt[0] = B;
  }
}

void launch_load_rows(const Ws& ws, const float* R, int B, cudaStream_t s) {
  load_rows_kernel<<<(B + 7) / 8, 256, 0, s>>>(ws, R, B);
}

// ------------------------------------------------------------------------------ compaction
// Compaction step j: keeps the positions of list live[(j+1)&1] (count cnt[j]) whose flag is
// set, in order, into live[j&1] (and each kept signal's iteration count into livek[j&1]); writes
// cnt[j+1]. Each block owns kCompactChunk positions and
// counts the kept flags before its range itself (16 flags per load), so the compaction is
// stable and needs no inter-block communication. Kept signals get their candidate key cleared
// and, on the tensor-core paths, their residual row quantised into position order (Rq[j&1],
// sr[j&1]); one warp per row, the row's loads issued together in batches of 8 per lane.
constexpr int kCompactChunk = 16;

__global__ void __launch_bounds__(256) compact_kernel(Ws ws, int j, int S, int reuse) {
  j = j >= 0 ? j : *ws.kdev + 1;  // -1: the step after the loop's current iteration
  if (j >= S) return;           // no further iteration reads this list
  __shared__ int dest_s[kCompactChunk];
  __shared__ int red_i[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Lin = ws.cnt[j];
  const int* in = ws.live[(j + 1) & 1];
  int* out = ws.live[j & 1];
  const int p0 = blockIdx.x * kCompactChunk;
  if (p0 >= Lin) {
    if (blockIdx.x == 0 && tid == 0) ws.cnt[j + 1] = 0;
    return;
  }
  // The signals at this warp's two positions and their records (iteration count, threshold
  // record, residual norm) do not depend on the kept flags, so their loads go out first and land
  // while the flags are counted
  static_assert(kCompactChunk == 16, "two positions per warp of eight");
  int pid[2], pnk[2];
  float prn[2];
  TauRec ptr[2];
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const int p = p0 + warp + 8 * m;
    pid[m] = p < Lin ? in[p] : 0;
  }
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    pnk[m] = ws.niter[pid[m]];
    prn[m] = ws.tau_pos ? ws.rnorm[pid[m]] : 0.f;
    ptr[m] = ws.tau_pos && j > 0 ? ws.tau[pid[m]] : TauRec{0.f, 0.f, -1, 0};
  }
  // kept flags before p0 (a multiple of 16; flags are 0 or 1 bytes, so a word's bit count is
  // its number of kept positions)
  int c = 0;
  const uint4* fl4 = reinterpret_cast<const uint4*>(ws.flag);
  for (int i = tid; i < p0 / 16; i += 256) {
    const uint4 v = fl4[i];
    c += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
  }
  c = warp_sum_int(c);
  if (lane == 0) red_i[warp] = c;
  if (warp == 0) {
    const int p = p0 + lane;
    const bool keep = lane < kCompactChunk && p < Lin && ws.flag[p] != 0;
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (lane < kCompactChunk) dest_s[lane] = keep ? __popc(m & ((1u << lane) - 1u)) : -1;
  }
  __syncthreads();
  int before = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) before += red_i[w];
  if (tid == 0 && p0 + kCompactChunk >= Lin) {
    int total = 0;
    for (int i = 0; i < kCompactChunk; ++i) total += dest_s[i] >= 0 ? 1 : 0;
    ws.cnt[j + 1] = before + total;
  }
  const int M4 = ws.Mp / 4;
  // Positions that do not move (nothing before them retired) keep the quantised rows the
  // one-warp update kernel wrote for them; other blocks quantise from the FP32 residuals.
  int keep_all = 1;
  for (int i = 0; i < kCompactChunk; ++i)
    if (p0 + i < Lin && dest_s[i] != i) keep_all = 0;
  const bool rows_in_place = reuse && ws.upd_w == 1 && ws.prec != OMP_PREC_FP32 && before == p0 &&
                             keep_all;
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const int i = warp + 8 * m;
    const int r = dest_s[i];
    if (r < 0) continue;
    const int dest = before + r;
    const int id = pid[m];
    // For the correlation (FP8: in the units of the scores, which leave out the row's scale):
    // the threshold the update kernel of step j - 1 wrote for this signal, and three score error
    // bounds at its residual, the same bound and norm the update of step j will use (rounded up)
    float tau = 0.f, win = 0.f;
    if (ws.tau_pos) {
      float eps_j = ws.rescore_eps;
      if (j > 0) {
        const TauRec t = ptr[m];
        if (t.step == j) {
          tau = t.tau > 0.f ? t.tau : 0.f;
          if (t.eps > 0.f) eps_j = fminf(t.eps, ws.rescore_eps);
        }
      }
      win = 3.f * eps_j * prn[m];
      win = win > 0.f ? win * (1.f + 0x1p-20f) : 0.f;
    }
    const bool fp8_pos = ws.tau_pos && ws.prec == OMP_PREC_FP8_E4M3;
    if (lane == 0) {
      out[dest] = id;
      ws.livek[j & 1][dest] = pnk[m];
      ws.cand1[dest] = 0ull;
      if (ws.cand2) ws.cand2[dest] = 0ull;
      if (ws.tau_pos && !fp8_pos) {
        ws.tau_pos[dest] = tau;
        ws.win_pos[dest] = win;
      }
    }
    if (rows_in_place) {
      if (lane == 0 && fp8_pos) {  // the row's scale was written with it by the update kernel
        const float sr = ws.sr[j & 1][dest];
        ws.tau_pos[dest] = sr > 0.f ? tau / sr : 0.f;
        ws.win_pos[dest] = sr > 0.f ? win / sr * (1.f + 0x1p-20f) : 0.f;
      }
      continue;
    }
    const float4* src = reinterpret_cast<const float4*>(ws.R32 + static_cast<size_t>(id) * ws.Mp);
    if (ws.prec == OMP_PREC_BF16) {
      __nv_bfloat162* dst = reinterpret_cast<__nv_bfloat162*>(
          static_cast<__nv_bfloat16*>(ws.Rq[j & 1]) + static_cast<size_t>(dest) * ws.Mp);
      for (int m0 = 0; m0 < M4; m0 += 256) {
        float4 v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int m = m0 + t * 32 + lane;
          v[t] = m < M4 ? src[m] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int m = m0 + t * 32 + lane;
          if (m < M4) {
            dst[2 * m] = __floats2bfloat162_rn(v[t].x, v[t].y);
            dst[2 * m + 1] = __floats2bfloat162_rn(v[t].z, v[t].w);
          }
        }
      }
    } else if (ws.prec == OMP_PREC_FP8_E4M3) {
      float amax = 0.f;
      for (int m0 = 0; m0 < M4; m0 += 256) {
        float4 v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int m = m0 + t * 32 + lane;
          v[t] = m < M4 ? src[m] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int t = 0; t < 8; ++t)
          amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v[t].x), fabsf(v[t].y)), fmaxf(fabsf(v[t].z), fabsf(v[t].w))));
      }
      amax = warp_max(amax);
      const float inv = amax > 0.f ? 448.f / amax : 0.f;
      const float sr = amax > 0.f ? amax / 448.f : 0.f;
      if (lane == 0) {
        ws.sr[j & 1][dest] = sr;
        if (fp8_pos) {
          ws.tau_pos[dest] = sr > 0.f ? tau / sr : 0.f;
          ws.win_pos[dest] = sr > 0.f ? win / sr * (1.f + 0x1p-20f) : 0.f;
        }
      }
      uint32_t* dst = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(ws.Rq[j & 1]) +
                                                  static_cast<size_t>(dest) * ws.Mp);
      for (int m0 = 0; m0 < M4; m0 += 256) {
        float4 v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int m = m0 + t * 32 + lane;
          v[t] = m < M4 ? src[m] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int m = m0 + t * 32 + lane;
          if (m < M4) {
            const uint32_t b0 = __nv_cvt_float_to_fp8(v[t].x * inv, __NV_SATFINITE, __NV_E4M3);
            const uint32_t b1 = __nv_cvt_float_to_fp8(v[t].y * inv, __NV_SATFINITE, __NV_E4M3);
            const uint32_t b2 = __nv_cvt_float_to_fp8(v[t].z * inv, __NV_SATFINITE, __NV_E4M3);
            const uint32_t b3 = __nv_cvt_float_to_fp8(v[t].w * inv, __NV_SATFINITE, __NV_E4M3);
            dst[m] = b0 | (b1 << 8) | (b2 << 16) | (b3 << 24);
          }
        }
      }
    }
  }
}

void launch_compact(const Ws& ws, int j, int B, int S, bool reuse, cudaStream_t s) {
  compact_kernel<<<(B + kCompactChunk - 1) / kCompactChunk, 256, 0, s>>>(ws, j, S, reuse ? 1 : 0);
}

// End of one pass of the graph's while loop: advance the iteration counter and keep looping
// while iterations remain and some signal is live for the next one (its count was just written
// by the compaction).
__global__ void advance_kernel(Ws ws, int S, cudaGraphConditionalHandle cond) {
  const int k1 = *ws.kdev + 1;
  *ws.kdev = k1;
  cudaGraphSetConditional(cond, (k1 < S && ws.cnt[k1 + 1] > 0) ? 1u : 0u);
}

void launch_advance(const Ws& ws, int S, cudaGraphConditionalHandle cond, cudaStream_t s) {
  advance_kernel<<<1, 1, 0, s>>>(ws, S, cond);
}

// ---------------------------------------------------------------------------------- finalize
// One warp per signal: x = F b (x_i = sum_{j>=i} F[i,j] b_j, FP64 back-substitution with the
// inverse factor), written in selection order with the support; padding 0 / -1.
__global__ void __launch_bounds__(256) finalize_kernel(Ws ws, const CallArgs* args, int B, int S) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (b >= B) return;
  const int n = ws.niter[b];
  const double* Fg = ws.F + static_cast<size_t>(b) * ws.Fstride;
  const double* bv = ws.bv + static_cast<size_t>(b) * ws.Smax;
  const int* sup = ws.sup + static_cast<size_t>(b) * ws.Smax;
  float* X = args->X + static_cast<size_t>(b) * S;
  int* so = args->support + static_cast<size_t>(b) * S;
  for (int i = lane; i < S; i += 32) {
    float x = 0.f;
    int s = -1;
    if (i < n) {
      double acc = 0.0;
      for (int j = i; j < n; ++j) acc += Fg[static_cast<size_t>(j) * (j + 1) / 2 + i] * bv[j];
      x = static_cast<float>(acc);
      s = sup[i];
    }
    X[i] = x;
    so[i] = s;
  }
  if (args->drop) {
    const float* dg = ws.drop + static_cast<size_t>(b) * ws.Smax;
    float* dd = args->drop + static_cast<size_t>(b) * S;
    for (int i = lane; i < S; i += 32) dd[i] = i < n ? dg[i] : 0.f;
  }
  if (args->margin && ws.margin) {
    const float* mg = ws.margin + static_cast<size_t>(b) * ws.Smax;
    float* md = args->margin + static_cast<size_t>(b) * S;
    for (int i = lane; i < S; i += 32) md[i] = i < n ? mg[i] : -1.f;
  }
  if (lane == 0) {
    if (args->n_iter) args->n_iter[b] = n;
    if (args->resid) args->resid[b] = ws.rnorm[b];
    if (args->stop) args->stop[b] = ws.stop[b];
    if (args->fallback) args->fallback[b] = ws.fb[b];
  }
}

void launch_finalize(const Ws& ws, const CallArgs* args, int B, int S, cudaStream_t s) {
  finalize_kernel<<<(B + 7) / 8, 256, 0, s>>>(ws, args, B, S);
}

// ------------------------------------------------------------------------------ top-k output
// omp_correlate_topk: per signal, the best `topk` candidates of the correlation (no rescoring),
// decreasing score, ties to the lower index. Position p holds signal p (all rows live).
__global__ void __launch_bounds__(32) topk_out_kernel(Ws ws, const CallArgs* args, int B, int topk) {
  const int p = blockIdx.x;
  const int lane = threadIdx.x;
  if (p >= B) return;
  int* io = args->topk_idx + static_cast<size_t>(p) * topk;
  float* so = args->topk_score + static_cast<size_t>(p) * topk;
  if (ws.prec == OMP_PREC_FP32) {
    if (lane == 0) {
      const unsigned long long key = ws.cand1[p];
      io[0] = key ? key_index(key) : -1;
      so[0] = key ? key_score(key) : -1.f;
    }
    return;
  }
  const int total = tc_piece_count(ws, ws.cnt[1], p) * kMaxTopk;
  const float* cs = ws.cand_s + static_cast<size_t>(p) * ws.pieces * kMaxTopk;
  const int* ci = ws.cand_i + static_cast<size_t>(p) * ws.pieces * kMaxTopk;
  float vs[8];
  int vi[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int e = lane + 32 * t;
    const bool ok = e < total;
    vs[t] = ok ? cs[e] : -1.f;
    vi[t] = ok ? ci[e] : 0x7fffffff;
    if (vi[t] < 0) { vs[t] = -1.f; vi[t] = 0x7fffffff; }
  }
  for (int sel = 0; sel < topk; ++sel) {
    float bs = -2.f;
    int bi = 0x7fffffff, bt = -1;
#pragma unroll
    for (int t = 0; t < 8; ++t)
      if (better(vs[t], vi[t], bs, bi)) { bs = vs[t]; bi = vi[t]; bt = t; }
    float gs = bs;
    int gi = bi;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float os = __shfl_xor_sync(0xffffffffu, gs, o);
      const int oi = __shfl_xor_sync(0xffffffffu, gi, o);
      if (better(os, oi, gs, gi)) { gs = os; gi = oi; }
    }
    if (bt >= 0 && bi == gi && bs == gs) {
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (t == bt) { vs[t] = -2.f; vi[t] = 0x7fffffff; }
    }
    if (lane == 0) {
      const bool ok = gi >= 0 && gi < ws.N && gs >= 0.f;
      io[sel] = ok ? gi : -1;
      so[sel] = ok ? gs : -1.f;
    }
  }
}

void launch_topk_out(const Ws& ws, const CallArgs* args, int B, int topk, cudaStream_t s) {
  topk_out_kernel<<<B, 32, 0, s>>>(ws, args, B, topk);
}

}  // namespace ompk
