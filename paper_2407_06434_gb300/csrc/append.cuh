// Per-iteration selection, inverse-Cholesky append and residual update, one block of W warps
// per live signal (W = 1 for padded lengths up to 1024, up to 8 for 8192; the autotuner picks).
// The kernels and their launch templates; each warp count is compiled in its own translation
// unit (append_w1.cu .. append_w8.cu), the dispatch is in append.cu.
//
// Iteration k (0-based; the paper's k+1), following Sec. 2.3:
//   n*    the correlation's pick (FP32 path), or the best of the merged top-8 rescored in FP32
//         (quantised paths; only the candidates within twice a rigorous score error bound of the
//         quantised best are rescored, none when the best leads by more)
//   w     = A_S^T a_{n*}          read from the Gram matrix row n* (Sec. 2.2 precompute)
//   z     = F_k^T w               FP32, on an FP32 copy of F staged in shared memory
//   delta = ||a_{n*}||^2 - ||z||^2 in FP64; the atom is dependent if delta <= 1e-10 ||a_{n*}||^2
//   gamma = 1 / sqrt(delta)       FP64: the diagonal of the new inverse-Cholesky column
//   F[:,k] = [-gamma F_k z ; gamma]  (stored in FP64 and FP32)
//   q     = A_{S+n*} F[:,k]       the new orthonormal direction (gather of k+1 atom rows: FP32, or
//                                  with the handle's 24-bit option the rows rounded to a 15-bit
//                                  mantissa, read as 3 bytes per element)
//   b_k   = q^T r,  r <- r - b_k q (y_hat = A_k F_k (A_k F_k)^T y built one term at a time)
// and, with one warp per signal, the next step's quantised operand row at this position, and
// (BF16) the next correlation's pruning threshold from the exact FP32 correlation of the new
// residual with the best candidate that was not picked.
//
// Layout of the work: the residual and q live in registers, sliced over the block's lanes in
// float4 slots (slot s of a row belongs to lane s mod 32 of warp (s / 32) mod W). The small
// triangular work runs in the first warp, lane-parallel over rows or columns of F. GB300 issues
// FP64 at a small fraction of its FP32 rate, so only the Schur complement, gamma (an FP32
// seed and one Newton step) and the stored factor are FP64; their FP32 inputs (w from the FP32
// Gram matrix) carry no more precision, and ||z||^2, b and ||r|| are FP32 sums.
#pragma once
#include "common.cuh"

namespace ompk {
namespace {

// One block per signal (W warps): a block's slot on the SM frees as soon as its own signal is
// done, so signals that skip the rescoring or retire early are not held back by slower ones of
// the same block. W * 32 threads x (16 / W) blocks keep 128 registers a thread and 16 warps per
// SM.
constexpr int kMaxBlk = 8;  // lane slots of 32 rows/columns of F: Smax <= 256
constexpr int kTriMax = 64;  // the packed FP32 factor is staged in shared memory for Smax <= 64

__device__ __forceinline__ void group_sync(int W, int grp) {
  if (W == 1)
    __syncwarp();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(W * 32) : "memory");
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 16-byte global -> shared copy (L2 only) that holds no register while in flight
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// wait until at most one of this thread's committed groups is still in flight
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }


struct GroupSmem {
  float* w;      // Smax: A_S^T a_{n*} (Gram row entries)
  float* z;      // Smax: F^T w
  float* f;      // Smax + 1: new F column (FP32 copy used by the gather)
  int* sup;      // Smax + 1: support including n*
  float* cpart;  // 8 x 8: rescoring partial dot products [candidate][warp]
  int* cidx;     // 8
  float* part;   // 16: per-warp partials of b [0, 8) and of ||r||^2 [8, 16)
  int* scal;     // 4: n*, dependent flag, rescoring skipped, candidates to rescore
  float* top2;   // 2: the merged lists' best and second-best quantised scores
  float* rinv;   // 2: inverse norms of the two best merged candidates (threshold on)
  float* cq;     // 8: the merged candidates' quantised scores, best first
  float* rows;   // 2 x Mp when the threshold is on: FP32 rows of the two best merged candidates
  float* tri;    // Smax (Smax + 1) / 2 when Smax <= kTriMax: staged copy of the packed FP32 F
};

__host__ __device__ __forceinline__ size_t tri_floats(int Smax) {
  return Smax <= kTriMax ? static_cast<size_t>(Smax) * (Smax + 1) / 2 : 0;
}

// rows of the two best merged candidates, staged for the next step's threshold
__host__ __device__ __forceinline__ size_t row_floats(const Ws& ws) {
  return ws.tau ? 2 * static_cast<size_t>(ws.Mp) : 0;
}

__host__ __device__ __forceinline__ size_t group_bytes(const Ws& ws) {
  const int Smax = ws.Smax;
  const size_t b = static_cast<size_t>(Smax + 1) * 8 + static_cast<size_t>(Smax) * 8 + 64 * 4 +
                   8 * 4 + 16 * 4 + 16 + 8 + 8 + 8 * 4 + row_floats(ws) * 4 +
                   (tri_floats(Smax) * 4 + 15) / 16 * 16;
  return (b + 15) / 16 * 16;
}

__device__ __forceinline__ GroupSmem group_smem(unsigned char* base, int grp, const Ws& ws) {
  const int Smax = ws.Smax;
  unsigned char* g = base + grp * group_bytes(ws);
  GroupSmem s;
  s.tri = reinterpret_cast<float*>(g);  // first, so it is 16-byte aligned
  g += (tri_floats(Smax) * 4 + 15) / 16 * 16;
  s.rows = reinterpret_cast<float*>(g);  // 16-byte aligned too
  g += row_floats(ws) * 4;
  s.part = reinterpret_cast<float*>(g);
  s.f = s.part + 16;
  s.sup = reinterpret_cast<int*>(s.f + Smax + 1);
  s.cpart = reinterpret_cast<float*>(s.sup + Smax + 1);
  s.cidx = reinterpret_cast<int*>(s.cpart + 64);
  s.scal = s.cidx + 8;
  s.w = reinterpret_cast<float*>(s.scal + 4);
  s.z = s.w + Smax;
  s.top2 = s.z + Smax;
  s.rinv = s.top2 + 2;
  s.cq = s.rinv + 2;
  return s;
}

// New inverse-Cholesky column for a support of kk atoms, run by one warp: lane slot j = lane + 32 t
// for t < NB covers the kk <= 32 NB rows/columns of F (NB is the smallest power of two that fits,
// so early iterations issue no predicated-off work). Fr is where the current factor is read (a
// shared-memory copy or F itself); the new column goes to Ff (FP32) and Fg (FP64).
template <int NB>
__device__ __forceinline__ void append_column(const Ws& ws, const GroupSmem& gs, const float* Fr,
                                              float* Ff, double* Fg, int kk, int ns, int lane) {
  // z_j = sum_{i<=j} F[i,j] w_i
  float zl[NB];
#pragma unroll
  for (int t = 0; t < NB; ++t) zl[t] = 0.f;
  for (int i = 0; i < kk; ++i) {
    const float wi = gs.w[i];
#pragma unroll
    for (int t = 0; t < NB; ++t) {
      const int j = lane + 32 * t;
      if (j < kk && i <= j) zl[t] = fmaf(Fr[static_cast<size_t>(j) * (j + 1) / 2 + i], wi, zl[t]);
    }
  }
  // ||z||^2 as an unevaluated sum hi + lo of FP32 numbers: each square is split exactly by an
  // FMA and the sums are error-free (Knuth's two-sum), so the FP64 Schur complement below gets
  // ||z||^2 to about 2^-42 relative (far inside the FP32 error of z itself) without FP64 work
  // per lane, which GB300 issues at a small fraction of its FP32 rate.
  float zh = 0.f, zlo = 0.f;
#pragma unroll
  for (int t = 0; t < NB; ++t) {
    const int j = lane + 32 * t;
    if (j < kk) {
      gs.z[j] = zl[t];
      const float p = __fmul_rn(zl[t], zl[t]);
      zlo = __fadd_rn(zlo, fmaf(zl[t], zl[t], -p));
      two_sum(zh, zlo, p);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, zh, o);
    zlo = __fadd_rn(zlo, __shfl_xor_sync(0xffffffffu, zlo, o));
    two_sum(zh, zlo, oh);
  }
  const double zz = static_cast<double>(zh) + static_cast<double>(zlo);
  const double nrm2 = ws.norm2[ns];
  const double delta = nrm2 - zz;
  const bool dep = !(delta > kDepRtol * nrm2);
  if (lane == 0) gs.scal[1] = dep ? 1 : 0;
  __syncwarp();
  if (dep) return;
  // gamma = 1/sqrt(delta): the FP32 reciprocal square root as a seed, then one Newton-Raphson
  // step y <- y (3 - delta y^2) / 2 in FP64 (the error squares: about 2^-42 relative with a 2-ulp seed)
  double gamma;
  if (delta > 1e-36 && delta < 1e36) {
    const double y0 = static_cast<double>(rsqrtf(static_cast<float>(delta)));
    gamma = y0 * (1.5 - 0.5 * delta * y0 * y0);
  } else {
    gamma = 1.0 / sqrt(delta);
  }
  // u_i = sum_{j>=i} F[i,j] z_j, lane slot i; one coalesced column per j
  float ul[NB];
#pragma unroll
  for (int t = 0; t < NB; ++t) ul[t] = 0.f;
  for (int j = 0; j < kk; ++j) {
    const float zj = gs.z[j];
    const float* col = Fr + static_cast<size_t>(j) * (j + 1) / 2;
#pragma unroll
    for (int t = 0; t < NB; ++t) {
      const int i = lane + 32 * t;
      if (i <= j) ul[t] = fmaf(col[i], zj, ul[t]);
    }
  }
  const size_t off = static_cast<size_t>(kk) * (kk + 1) / 2;
#pragma unroll
  for (int t = 0; t < NB; ++t) {
    const int i = lane + 32 * t;
    if (i < kk) {
      const double fv = -gamma * static_cast<double>(ul[t]);
      const float f32 = static_cast<float>(fv);
      Fg[off + i] = fv;
      Ff[off + i] = f32;
      gs.f[i] = f32;
    }
  }
  if (lane == 0) {
    Fg[off + kk] = gamma;
    Ff[off + kk] = static_cast<float>(gamma);
    gs.f[kk] = static_cast<float>(gamma);
    gs.sup[kk] = ns;
  }
}

// Four consecutive elements of an atom row (float4 slot s) for the q gather: from the FP32 rows,
// or (G24) rebuilt from the 24-bit split copy -- 8 bytes of high halves and 4 bytes of the next
// 8 bits, i.e. the element rounded to a 15-bit mantissa, three quarters of the FP32 bytes.
// The loaded words stay in their raw form (3 registers for G24) while the rows are in flight and
// are widened only where they are multiplied.
template <bool G24>
struct Slot4 {
  float4 v;
};
template <>
struct Slot4<true> {
  uint2 h;
  uint32_t l;
};

template <bool G24>
__device__ __forceinline__ Slot4<G24> gather4(const Ws& ws, int n, int s) {
  Slot4<G24> r;
  if constexpr (G24) {
    r.h = __ldg(reinterpret_cast<const uint2*>(ws.A24h + static_cast<size_t>(n) * ws.Mp) + s);
    r.l = __ldg(reinterpret_cast<const uint32_t*>(ws.A24l + static_cast<size_t>(n) * ws.Mp) + s);
  } else {
    r.v = __ldg(reinterpret_cast<const float4*>(ws.A32 + static_cast<size_t>(n) * ws.Mp) + s);
  }
  return r;
}
template <bool G24>
__device__ __forceinline__ Slot4<G24> zero4() {
  Slot4<G24> r;
  if constexpr (G24) {
    r.h = make_uint2(0u, 0u);
    r.l = 0u;
  } else {
    r.v = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  return r;
}
template <bool G24>
__device__ __forceinline__ float4 widen(const Slot4<G24>& r) {
  if constexpr (G24) {
    float4 v;
    v.x = __uint_as_float((r.h.x << 16) | ((r.l & 0xFFu) << 8));
    v.y = __uint_as_float((r.h.x & 0xFFFF0000u) | (((r.l >> 8) & 0xFFu) << 8));
    v.z = __uint_as_float((r.h.y << 16) | (((r.l >> 16) & 0xFFu) << 8));
    v.w = __uint_as_float((r.h.y & 0xFFFF0000u) | ((r.l >> 24) << 8));
    return v;
  } else {
    return r.v;
  }
}

// One step of the signal at live position p (p < L), by the block's W warps; every return is
// taken by the whole block.
template <int W, int V, bool G24>
__device__ __forceinline__ void update_position(const Ws& ws, int k, int L, int p, int S, float eps,
                                                int eps_rel, unsigned char* smem) {
  const bool top1 = ws.prec == OMP_PREC_FP32;
  const int lane = threadIdx.x & 31;
  const int grp = 0, wig = threadIdx.x >> 5;
  // the signal at this position and its own iteration (signals may join the loop late), from two
  // arrays the compaction wrote side by side, so both arrive in one round trip
  const int id = ws.live[k & 1][p];
  const int kk = ws.livek[k & 1][p];
  GroupSmem gs = group_smem(smem, grp, ws);

  // The candidate lists head the critical path (merge, rescoring, append), so their loads are
  // issued first; they are only read at the merge below.
  float vs[8];
  int vi[8];
  if (!top1 && wig == 0) {
    const int total = tc_piece_count(ws, L, p) * kMaxTopk;
    const float* cs = ws.cand_s + static_cast<size_t>(p) * ws.pieces * kMaxTopk;
    const int* ci = ws.cand_i + static_cast<size_t>(p) * ws.pieces * kMaxTopk;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int e = lane + 32 * t;
      const bool ok = e < total;
      vs[t] = ok ? cs[e] : -1.f;
      vi[t] = ok ? ci[e] : 0x7fffffff;
    }
  }

  // Loads that do not depend on the selection go out next. The packed FP32 factor (so that the
  // serial z and F z loops wait on no global load) and the support are copied into shared memory
  // by cp.async, which holds no register and does not stall the warp: they land while the merge
  // and the rescoring run, and the append waits for them (the first group this warp commits).
  float* Ff = ws.F32 + static_cast<size_t>(id) * ws.Fstride;
  const bool staged = ws.Smax <= kTriMax;
  if (wig == 0) {
    if (staged) {
      const int tn4 = (kk * (kk + 1) / 2 + 3) >> 2;  // within the padded stride
      for (int e = lane; e < tn4; e += 32) cp_async16(gs.tri + 4 * e, Ff + 4 * e);
    }
    const int* supg = ws.sup + static_cast<size_t>(id) * ws.Smax;
    for (int i = lane; i < kk; i += 32) cp_async4(gs.sup + i, supg + i);
    cp_async_commit();
  }
  bool rows_group = false;  // a second cp.async group (the threshold's candidate rows) follows
  const float rprev = ws.rnorm[id];
  const float ynorm = ws.ynorm[id];
  // the pruning threshold the correlation used for this position (0: none; in the units of the
  // quantised scores) and this step's score error bound per unit of ||r||: the one the previous
  // step derived from this residual row's actual quantisation error, else the worst case
  const float tau_used = ws.tau_pos ? ws.tau_pos[p] : 0.f;
  float eps_k = ws.rescore_eps;
  if (ws.tau && ws.rescore_eps > 0.f) {
    const TauRec tr = ws.tau[id];
    if (tr.step == k && tr.eps > 0.f) eps_k = fminf(tr.eps, ws.rescore_eps);
  }

  const int M4 = ws.Mp >> 2;
  const float4* rrow = reinterpret_cast<const float4*>(ws.R32 + static_cast<size_t>(id) * ws.Mp);
  float4 r[V];
#pragma unroll
  for (int t = 0; t < V; ++t) {
    const int s = t * (W * 32) + wig * 32 + lane;
    r[t] = s < M4 ? rrow[s] : make_float4(0.f, 0.f, 0.f, 0.f);
  }

  // ---------------------------------------------------------------- selection
  int ns;
  if (top1) {
    ns = key_index(ws.cand1[p]);
  } else {
    if (wig == 0) {
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (vi[t] < 0) {  // an unfilled list entry
          vs[t] = -1.f;
          vi[t] = 0x7fffffff;
        }
      // Candidates come out best first; one more than 2 rescore_eps ||r|| below the best has an
      // FP32 score strictly below the best one's, so the rescoring stops before it. FP8 scores
      // leave out the residual's scale qs, so the window is taken in their units.
      const float qs = ws.prec == OMP_PREC_FP8_E4M3 ? ws.sr[k & 1][p] : 1.f;
      const bool bound = ws.rescore_eps > 0.f && rprev > 1e-30f && qs > 0.f;
      const float win = bound ? 2.f * eps_k * rprev / qs : 0.f;
      float s_first = 0.f;
      int nres = ws.topk;
      for (int sel = 0; sel < ws.topk; ++sel) {
        float bs = -2.f;
        int bi = 0x7fffffff, bt = -1;
#pragma unroll
        for (int t = 0; t < 8; ++t)
          if (better(vs[t], vi[t], bs, bi)) {
            bs = vs[t];
            bi = vi[t];
            bt = t;
          }
        float g_s = bs;
        int g_i = bi;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float os = __shfl_xor_sync(0xffffffffu, g_s, o);
          const int oi = __shfl_xor_sync(0xffffffffu, g_i, o);
          if (better(os, oi, g_s, g_i)) {
            g_s = os;
            g_i = oi;
          }
        }
        if (bt >= 0 && bi == g_i && bs == g_s) {
#pragma unroll
          for (int t = 0; t < 8; ++t)
            if (t == bt) {
              vs[t] = -2.f;
              vi[t] = 0x7fffffff;
            }
        }
        if (lane == 0) gs.cidx[sel] = (g_i >= 0 && g_i < ws.N) ? g_i : -1;
        if (lane == 0) gs.cq[sel] = g_s;
        if (lane == 0 && sel < 2) gs.top2[sel] = g_s;
        if (sel == 0)
          s_first = g_s;
        else if (bound && nres == ws.topk && !(g_s >= s_first - win))
          nres = sel;
        if (nres < ws.topk) {  // the window is closed and the two best are known
          if (lane == 0)
            for (int c = sel + 1; c < ws.topk; ++c) gs.cidx[c] = -1;
          break;
        }
      }
      // margins recorded: at least the two best are rescored (the handle then runs without
      // the score bound, so nothing is skipped or trimmed)
      if (ws.margin && nres < 2 && ws.topk >= 2) nres = 2;
      if (lane == 0) gs.scal[3] = nres;
      // The rescoring can only confirm the quantised best when its lead over the second is
      // more than twice the bound on |quantised - FP32| score (rescore_eps ||r||, from the
      // quantisation and both accumulations, with ||a|| inv_norm = 1): every other candidate's
      // FP32 score is then strictly below the best one's, so the rescoring is skipped. Columns
      // that the correlation pruned scored at most tau_used, so tau_used stands in for a
      // missing second.
      if (lane == 0) {
        const float lead = gs.top2[0] - fmaxf(gs.top2[1], tau_used);
        gs.scal[2] = (bound && gs.cidx[0] >= 0 && lead > win) ? 1 : 0;
      }
    }
    group_sync(W, grp);
    const bool skip = gs.scal[2] != 0;
    int nres = gs.scal[3];
    if (ws.tau) {
      // the two best merged candidates' FP32 rows and inverse norms, for the next step's
      // threshold: copied to shared memory in the background (each warp its own slots), read at
      // the end of the kernel
      for (int c = 0; c < 2 && c < ws.topk; ++c) {
        const int n = gs.cidx[c];
        if (n < 0) continue;
        const float4* src = reinterpret_cast<const float4*>(ws.A32 + static_cast<size_t>(n) * ws.Mp);
        float4* dst = reinterpret_cast<float4*>(gs.rows + static_cast<size_t>(c) * ws.Mp);
#pragma unroll
        for (int t = 0; t < V; ++t) {
          const int s = t * (W * 32) + wig * 32 + lane;
          if (s < M4) cp_async16(dst + s, src + s);
        }
        if (wig == 0 && lane == c) cp_async4(gs.rinv + c, ws.inv_norm + n);
      }
      cp_async_commit();
      rows_group = true;
    }
    // FP32 rescoring: every warp dots its residual slice with each candidate's FP32 row, two
    // candidates per pass so their row loads are in flight together. With the bound, a pass
    // starts only if its first candidate (they come best first) could still beat the best FP32
    // score found so far: one whose quantised score is more than eps_k ||r|| below that has an
    // FP32 score strictly below it, and so have all that follow.
    const float qsr = ws.prec == OMP_PREC_FP8_E4M3 ? ws.sr[k & 1][p] : 1.f;
    const bool adapt = ws.rescore_eps > 0.f && rprev > 1e-30f && qsr > 0.f;
    float tmax = -1.f;
    int ndone = 0;
    for (int c = 0; !skip && c < nres; c += 2) {
      if (adapt && c > 0 && !(gs.cq[c] >= (tmax - eps_k * rprev) / qsr)) break;
      const int n0 = gs.cidx[c];
      const int n1 = c + 1 < nres ? gs.cidx[c + 1] : -1;
      const float4* a0 = reinterpret_cast<const float4*>(ws.A32 + static_cast<size_t>(n0 < 0 ? 0 : n0) * ws.Mp);
      const float4* a1 = reinterpret_cast<const float4*>(ws.A32 + static_cast<size_t>(n1 < 0 ? 0 : n1) * ws.Mp);
      float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
      for (int t = 0; t < V; ++t) {
        const int s = t * (W * 32) + wig * 32 + lane;
        if (s < M4) {
          const float4 x0 = n0 >= 0 ? __ldg(a0 + s) : make_float4(0.f, 0.f, 0.f, 0.f);
          const float4 x1 = n1 >= 0 ? __ldg(a1 + s) : make_float4(0.f, 0.f, 0.f, 0.f);
          acc0 += x0.x * r[t].x + x0.y * r[t].y + x0.z * r[t].z + x0.w * r[t].w;
          acc1 += x1.x * r[t].x + x1.y * r[t].y + x1.z * r[t].z + x1.w * r[t].w;
        }
      }
      acc0 = warp_sum_f(acc0);
      acc1 = warp_sum_f(acc1);
      if (lane == 0) {
        gs.cpart[c * 8 + wig] = acc0;
        if (c + 1 < nres) gs.cpart[(c + 1) * 8 + wig] = acc1;
      }
      ndone = c + 2 < nres ? c + 2 : nres;
      if (adapt && ndone < nres) {  // the pass's FP32 scores (every thread, from the partials)
        group_sync(W, grp);
        for (int cc = c; cc < ndone; ++cc) {
          const int n = gs.cidx[cc];
          if (n < 0) continue;
          float v = 0.f;
          for (int w = 0; w < W; ++w) v += gs.cpart[cc * 8 + w];
          tmax = fmaxf(tmax, fabsf(v) * __ldg(ws.inv_norm + n));
        }
      }
    }
    if (!skip) nres = ndone;  // the candidates not rescored cannot beat the best that was
    group_sync(W, grp);
    if (wig == 0 && skip) {
      if (lane == 0) gs.scal[0] = gs.cidx[0];
    } else if (wig == 0) {
      float sc = -2.f;
      int ix = 0x7fffffff;
      if (lane < nres && gs.cidx[lane] >= 0) {
        float v = 0.f;
        for (int w = 0; w < W; ++w) v += gs.cpart[lane * 8 + w];
        ix = gs.cidx[lane];
        sc = fabsf(v) * __ldg(ws.inv_norm + ix);
      }
      const float own_s = sc;
      const int own_i = ix;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float os = __shfl_xor_sync(0xffffffffu, sc, o);
        const int oi = __shfl_xor_sync(0xffffffffu, ix, o);
        if (better(os, oi, sc, ix)) {
          sc = os;
          ix = oi;
        }
      }
      if (lane == 0) gs.scal[0] = ix;
      if (ws.margin) {  // (s1 - s2) / s1 over the FP32 scores of the rescored candidates
        const float s2 = warp_max(own_i != ix ? own_s : -2.f);
        if (lane == 0) gs.top2[1] = sc > 0.f ? (s2 > 0.f ? (sc - s2) / sc : 1.f) : 0.f;
      }
    }
    group_sync(W, grp);
    ns = gs.scal[0];
  }
  if (ns < 0 || ns >= ws.N) {
    cp_async_wait_all();  // no copy outlives the block
    if (wig == 0 && lane == 0) {
      atomicOr(ws.err, OMP_DEVERR_BAD_STATE);
      ws.flag[p] = 0;
    }
    return;
  }

  // ---------------------------------------------------------------- append (first warp)
  // z and F z run in FP32 on the FP32 copy of F: their input w comes from the FP32 Gram matrix,
  // so FP64 arithmetic there would add no accuracy. The Schur complement delta, gamma and the
  // stored factor (used by the back-substitution) are FP64.
  double* Fg = ws.F + static_cast<size_t>(id) * ws.Fstride;
  if (wig == 0) {
    // the staged factor and the support have landed (the candidate rows of the threshold,
    // committed after them, may still be in flight) and are visible to the whole warp
    if (rows_group)
      cp_async_wait_one();
    else
      cp_async_wait_all();
    __syncwarp();
    const float* grow = ws.gram + static_cast<size_t>(ns) * ws.N;
    for (int i = lane; i < kk; i += 32) gs.w[i] = __ldg(grow + gs.sup[i]);
    __syncwarp();
    const float* Fr = staged ? gs.tri : Ff;
    const int nb = (kk + 31) >> 5;
    if (nb <= 1) append_column<1>(ws, gs, Fr, Ff, Fg, kk, ns, lane);
    else if (nb <= 2) append_column<2>(ws, gs, Fr, Ff, Fg, kk, ns, lane);
    else if (nb <= 4) append_column<4>(ws, gs, Fr, Ff, Fg, kk, ns, lane);
    else append_column<8>(ws, gs, Fr, Ff, Fg, kk, ns, lane);
  }
  group_sync(W, grp);
  if (gs.scal[1]) {
    if (ws.tau) cp_async_wait_all();  // no copy outlives the block
    if (wig == 0 && lane == 0) {
      ws.flag[p] = 0;
      ws.stop[id] = kStopDependent;
    }
    return;
  }

  // ---------------------------------------------------------------- q, b, residual update
  float4 q[V];
#pragma unroll
  for (int t = 0; t < V; ++t) q[t] = make_float4(0.f, 0.f, 0.f, 0.f);
  const int na = kk + 1;
  int a = 0;
  // r is not needed during the gather (it is read again below), so its registers carry a third
  // row in flight
  for (; a + 3 <= na; a += 3) {
    const float f0 = gs.f[a], f1 = gs.f[a + 1], f2 = gs.f[a + 2];
    const int n0 = gs.sup[a], n1 = gs.sup[a + 1], n2 = gs.sup[a + 2];
    Slot4<G24> w0[V], w1[V], w2[V];
#pragma unroll
    for (int t = 0; t < V; ++t) {
      const int s = t * (W * 32) + wig * 32 + lane;
      w0[t] = s < M4 ? gather4<G24>(ws, n0, s) : zero4<G24>();
      w1[t] = s < M4 ? gather4<G24>(ws, n1, s) : zero4<G24>();
      w2[t] = s < M4 ? gather4<G24>(ws, n2, s) : zero4<G24>();
    }
#pragma unroll
    for (int t = 0; t < V; ++t) {
      const float4 v0 = widen<G24>(w0[t]), v1 = widen<G24>(w1[t]), v2 = widen<G24>(w2[t]);
      q[t].x = fmaf(f2, v2.x, fmaf(f1, v1.x, fmaf(f0, v0.x, q[t].x)));
      q[t].y = fmaf(f2, v2.y, fmaf(f1, v1.y, fmaf(f0, v0.y, q[t].y)));
      q[t].z = fmaf(f2, v2.z, fmaf(f1, v1.z, fmaf(f0, v0.z, q[t].z)));
      q[t].w = fmaf(f2, v2.w, fmaf(f1, v1.w, fmaf(f0, v0.w, q[t].w)));
    }
  }
  for (; a + 2 <= na; a += 2) {
    const float f0 = gs.f[a], f1 = gs.f[a + 1];
    const int n0 = gs.sup[a], n1 = gs.sup[a + 1];
    Slot4<G24> w0[V], w1[V];
#pragma unroll
    for (int t = 0; t < V; ++t) {
      const int s = t * (W * 32) + wig * 32 + lane;
      w0[t] = s < M4 ? gather4<G24>(ws, n0, s) : zero4<G24>();
      w1[t] = s < M4 ? gather4<G24>(ws, n1, s) : zero4<G24>();
    }
#pragma unroll
    for (int t = 0; t < V; ++t) {
      const float4 v0 = widen<G24>(w0[t]), v1 = widen<G24>(w1[t]);
      q[t].x = fmaf(f1, v1.x, fmaf(f0, v0.x, q[t].x));
      q[t].y = fmaf(f1, v1.y, fmaf(f0, v0.y, q[t].y));
      q[t].z = fmaf(f1, v1.z, fmaf(f0, v0.z, q[t].z));
      q[t].w = fmaf(f1, v1.w, fmaf(f0, v0.w, q[t].w));
    }
  }
  if (a < na) {
    const float f0 = gs.f[a];
    const int n0 = gs.sup[a];
#pragma unroll
    for (int t = 0; t < V; ++t) {
      const int s = t * (W * 32) + wig * 32 + lane;
      const float4 v = widen<G24>(s < M4 ? gather4<G24>(ws, n0, s) : zero4<G24>());
      q[t].x = fmaf(f0, v.x, q[t].x);
      q[t].y = fmaf(f0, v.y, q[t].y);
      q[t].z = fmaf(f0, v.z, q[t].z);
      q[t].w = fmaf(f0, v.w, q[t].w);
    }
  }
#pragma unroll
  for (int t = 0; t < V; ++t) {
    const int s = t * (W * 32) + wig * 32 + lane;
    r[t] = s < M4 ? rrow[s] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  float bp = 0.f;
#pragma unroll
  for (int t = 0; t < V; ++t) bp += q[t].x * r[t].x + q[t].y * r[t].y + q[t].z * r[t].z + q[t].w * r[t].w;
  bp = warp_sum_f(bp);
  // per-warp partials of b and ||r||^2 (FP32 sums of FP32 products: no FP64 needed here)
  float* pf = gs.part;
  if (lane == 0) pf[wig] = bp;
  group_sync(W, grp);
  float bf = 0.f;
  for (int w = 0; w < W; ++w) bf += pf[w];  // W <= 8 partials
  float4* rw = reinterpret_cast<float4*>(ws.R32 + static_cast<size_t>(id) * ws.Mp);
  float rr = 0.f;
#pragma unroll
  for (int t = 0; t < V; ++t) {
    const int s = t * (W * 32) + wig * 32 + lane;
    r[t].x = fmaf(-bf, q[t].x, r[t].x);
    r[t].y = fmaf(-bf, q[t].y, r[t].y);
    r[t].z = fmaf(-bf, q[t].z, r[t].z);
    r[t].w = fmaf(-bf, q[t].w, r[t].w);
    if (s < M4) rw[s] = r[t];
    rr += r[t].x * r[t].x + r[t].y * r[t].y + r[t].z * r[t].z + r[t].w * r[t].w;
  }
  rr = warp_sum_f(rr);
  if (ws.tau) {
    // this warp's part of a_c^T r_k for the two staged candidate rows
    cp_async_wait_all();
    __syncwarp();
    const float4* x0 = reinterpret_cast<const float4*>(gs.rows);
    const float4* x1 = reinterpret_cast<const float4*>(gs.rows + ws.Mp);
    float d0 = 0.f, d1 = 0.f;
#pragma unroll
    for (int t = 0; t < V; ++t) {
      const int s = t * (W * 32) + wig * 32 + lane;
      if (s < M4) {
        const float4 u0 = x0[s], u1 = x1[s];
        d0 += u0.x * r[t].x + u0.y * r[t].y + u0.z * r[t].z + u0.w * r[t].w;
        d1 += u1.x * r[t].x + u1.y * r[t].y + u1.z * r[t].z + u1.w * r[t].w;
      }
    }
    d0 = warp_sum_f(d0);
    d1 = warp_sum_f(d1);
    if (lane == 0) {
      gs.cpart[2 * wig] = d0;
      gs.cpart[2 * wig + 1] = d1;
    }
  }
  float qe2 = -1.f;  // squared norm of the next row's quantisation error (W == 1; -1: not known)
  if (W == 1 && !top1) {
    // The next step's quantised operand row, at this position: the compaction keeps it where
    // no signal before this one retired, and re-quantises from R32 otherwise. Same rounding as
    // the compaction's (BF16 round-to-nearest-even; E4M3 satfinite with the row's amax / 448).
    // E4M3: the squared norm of its rounding error feeds the next step's data-driven score bound
    // (BF16 keeps the worst case, already tight enough to prune, which costs nothing here).
    const int j = (k + 1) & 1;
    float e2 = 0.f;
    if (ws.prec == OMP_PREC_BF16) {
      __nv_bfloat162* dq = reinterpret_cast<__nv_bfloat162*>(
          static_cast<__nv_bfloat16*>(ws.Rq[j]) + static_cast<size_t>(p) * ws.Mp);
#pragma unroll
      for (int t = 0; t < V; ++t) {
        const int s = t * 32 + lane;
        if (s < M4) {
          const __nv_bfloat162 h0 = __floats2bfloat162_rn(r[t].x, r[t].y);
          const __nv_bfloat162 h1 = __floats2bfloat162_rn(r[t].z, r[t].w);
          dq[2 * s] = h0;
          dq[2 * s + 1] = h1;
        }
      }
    } else {
      float amax = 0.f;
#pragma unroll
      for (int t = 0; t < V; ++t) {
        const int s = t * 32 + lane;
        if (s < M4)
          amax = fmaxf(amax, fmaxf(fmaxf(fabsf(r[t].x), fabsf(r[t].y)), fmaxf(fabsf(r[t].z), fabsf(r[t].w))));
      }
      amax = warp_max(amax);
      const float inv = amax > 0.f ? 448.f / amax : 0.f;
      if (lane == 0) ws.sr[j][p] = amax > 0.f ? amax / 448.f : 0.f;
      const float sr = amax > 0.f ? amax / 448.f : 0.f;
      uint32_t* dq = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(ws.Rq[j]) + static_cast<size_t>(p) * ws.Mp);
#pragma unroll
      for (int t = 0; t < V; ++t) {
        const int s = t * 32 + lane;
        if (s < M4) {
          const __nv_fp8_storage_t b0 = __nv_cvt_float_to_fp8(r[t].x * inv, __NV_SATFINITE, __NV_E4M3);
          const __nv_fp8_storage_t b1 = __nv_cvt_float_to_fp8(r[t].y * inv, __NV_SATFINITE, __NV_E4M3);
          const __nv_fp8_storage_t b2 = __nv_cvt_float_to_fp8(r[t].z * inv, __NV_SATFINITE, __NV_E4M3);
          const __nv_fp8_storage_t b3 = __nv_cvt_float_to_fp8(r[t].w * inv, __NV_SATFINITE, __NV_E4M3);
          dq[s] = static_cast<uint32_t>(b0) | (static_cast<uint32_t>(b1) << 8) |
                  (static_cast<uint32_t>(b2) << 16) | (static_cast<uint32_t>(b3) << 24);
          if (ws.tau) {
            const float d0 = fmaf(e4m3_to_float(b0), sr, -r[t].x);
            const float d1 = fmaf(e4m3_to_float(b1), sr, -r[t].y);
            const float d2 = fmaf(e4m3_to_float(b2), sr, -r[t].z);
            const float d3 = fmaf(e4m3_to_float(b3), sr, -r[t].w);
            e2 += d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3;
          }
        }
      }
    }
    if (ws.prec == OMP_PREC_FP8_E4M3) qe2 = warp_sum_f(e2);
  }
  if (lane == 0) pf[8 + wig] = rr;
  group_sync(W, grp);
  float rk = 0.f;  // ||r_k||, first warp's lane 0
  if (wig == 0 && lane == 0) {
    float tot = 0.f;
    for (int w = 0; w < W; ++w) tot += pf[8 + w];
    rk = sqrtf(tot);
    const float rn = rk;
    ws.bv[static_cast<size_t>(id) * ws.Smax + kk] = static_cast<double>(bf);
    ws.sup[static_cast<size_t>(id) * ws.Smax + kk] = ns;
    ws.drop[static_cast<size_t>(id) * ws.Smax + kk] = rprev > 0.f ? (bf / rprev) * (bf / rprev) : 0.f;
    if (ws.margin) {
      float mg;
      if (top1) {  // the correlation's best and runner-up keys (FP32 scores)
        const unsigned long long k2 = ws.cand2[p];
        const float s1 = key_score(ws.cand1[p]), s2 = k2 ? key_score(k2) : 0.f;
        mg = s1 > 0.f ? (s1 - s2) / s1 : 0.f;
      } else {
        mg = gs.top2[1];
      }
      ws.margin[static_cast<size_t>(id) * ws.Smax + kk] = mg;
    }
    ws.niter[id] = kk + 1;
    ws.rnorm[id] = rn;
    const float thr = eps_rel ? eps * ynorm : eps;
    int cont = 1;
    if (rn <= thr) {
      cont = 0;
      ws.stop[id] = kStopEps;
    } else if (kk + 1 >= S) {
      cont = 0;
      ws.stop[id] = kStopIters;
    }
    ws.flag[p] = static_cast<uint8_t>(cont);
  }

  // ---------------------------------------------------------------- next step's threshold
  // BF16 path with the rescoring bound. The exact FP32 correlation of the new residual with a
  // runner-up candidate m of this step (one of the two best merged ones, not the pick), less
  // its rounding bound Mp 2^-23 ||r_k||, is a lower bound L on the next residual's best score.
  // A column whose quantised score is at most L - 3 rescore_eps ||r_k|| has an FP32 score more
  // than 2 rescore_eps ||r_k|| below the best, so it can be neither the pick nor a rescoring
  // candidate that changes it: the next correlation drops such columns before its top-8
  // insertion.
  if (ws.tau && wig == 0 && lane == 0) {
    float best = 0.f;
    for (int c = 0; c < 2 && c < ws.topk; ++c) {
      const int n = gs.cidx[c];
      if (n < 0 || n == ns) continue;
      float d = 0.f;
      for (int w = 0; w < W; ++w) d += gs.cpart[2 * w + c];
      best = fmaxf(best, fabsf(d) * gs.rinv[c]);
    }
    // the next step's bound: from the next row's actual quantisation error when this block
    // quantised it (one warp per signal), else the worst case
    float eps_n = ws.rescore_eps;
    if (qe2 >= 0.f && rk > 0.f) {
      const float er = sqrtf(qe2) / rk * (1.f + 0x1p-20f);
      eps_n = fminf(eps_n, data_bound(ws, *ws.ea, er));
    }
    const float lb = best * (1.f - 0x1p-20f) - static_cast<float>(ws.Mp) * 0x1p-23f * rk;
    const float tau = lb - 3.f * eps_n * rk;
    ws.tau[id] = TauRec{tau > 0.f ? tau : 0.f, eps_n, k + 1, 0};
  }
}

// The append/update kernel. Either one block per live position (P = false, grid = B), or
// persistent (P = true, ws.upd_persist): a grid of as many blocks as fit on the GPU, each taking
// the next position from the iteration's counter until none is left, so blocks stay resident
// across signals and a block whose signal finishes early (the rescoring skipped, a retirement)
// takes another. The two are separate kernels, so each holds one copy of the step's code.
// Resident warps asked of the compiler per SM, by the float4 slots V a lane holds: 16 warps
// (128 registers) for 8 slots, 24 (80 registers) for 4, 32 (64 registers) for 2 or 1; the
// one-warp form keeps 16 for 4 slots and 24 for fewer, where those limits spill nothing.
constexpr int update_min_warps(int W, int V) {
  return V >= 8 ? 16 : W == 1 ? (V == 4 ? 16 : 24) : V == 4 ? 24 : 32;
}

template <int W, int V, bool G24, bool P>
__global__ void __launch_bounds__(W * 32, update_min_warps(W, V) / W)
    append_update_kernel(Ws ws, int k, int S, float eps, int eps_rel) {
  k = iter_of(ws, k);
  const int L = ws.cnt[k + 1];
  extern __shared__ __align__(16) unsigned char smem[];
  if (!P) {
    if (static_cast<int>(blockIdx.x) < L)
      update_position<W, V, G24>(ws, k, L, blockIdx.x, S, eps, eps_rel, smem);
    return;
  }
  __shared__ int next_p;
  for (;;) {
    if (threadIdx.x == 0) next_p = atomicAdd(ws.upd_ctr + k, 1);
    __syncthreads();
    const int p = next_p;
    __syncthreads();  // every thread has read it before the next position is taken
    if (p >= L) break;
    update_position<W, V, G24>(ws, k, L, p, S, eps, eps_rel, smem);
  }
}

// resident blocks of one persistent append/update kernel variant on the device (0 if the query
// fails)
template <int W, int V, bool G24>
int resident_blocks(size_t smem) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 0;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &nb, append_update_kernel<W, V, G24, true>, W * 32, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb * sms;
}

// W warps per signal and V float4 slots per lane cover Mp <= 128 W V.
template <int W, int V, bool G24>
void launch_g(const Ws& ws, int k, int B, int S, float eps, int eps_rel, cudaStream_t s) {
  const size_t smem = group_bytes(ws);
  if (ws.upd_persist) {
    const int r = resident_blocks<W, V, G24>(smem);
    const int grid = r > 0 && r < B ? r : B;
    append_update_kernel<W, V, G24, true><<<grid, W * 32, smem, s>>>(ws, k, S, eps, eps_rel);
  } else {
    append_update_kernel<W, V, G24, false><<<B, W * 32, smem, s>>>(ws, k, S, eps, eps_rel);
  }
}

template <int W, int V>
void launch_t(const Ws& ws, int k, int B, int S, float eps, int eps_rel, cudaStream_t s) {
  if (ws.A24h)
    launch_g<W, V, true>(ws, k, B, S, eps, eps_rel, s);
  else
    launch_g<W, V, false>(ws, k, B, S, eps, eps_rel, s);
}

template <int W>
void launch_w(const Ws& ws, int V, int k, int B, int S, float eps, int eps_rel, cudaStream_t s) {
  if (V == 1) launch_t<W, 1>(ws, k, B, S, eps, eps_rel, s);
  else if (V == 2) launch_t<W, 2>(ws, k, B, S, eps, eps_rel, s);
  else if (V == 4) launch_t<W, 4>(ws, k, B, S, eps, eps_rel, s);
  else launch_t<W, 8>(ws, k, B, S, eps, eps_rel, s);
}

template <int W, int V>
cudaError_t set_attr_t(int bytes) {
  cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(append_update_kernel<W, V, false, false>), bytes);
  if (e == cudaSuccess)
    e = raise_smem_limit(reinterpret_cast<const void*>(append_update_kernel<W, V, true, false>), bytes);
  if (e == cudaSuccess)
    e = raise_smem_limit(reinterpret_cast<const void*>(append_update_kernel<W, V, false, true>), bytes);
  if (e == cudaSuccess)
    e = raise_smem_limit(reinterpret_cast<const void*>(append_update_kernel<W, V, true, true>), bytes);
  return e;
}

template <int W>
cudaError_t set_attr_w(const Ws& ws) {
  const int bytes = static_cast<int>(group_bytes(ws));
  cudaError_t e = set_attr_t<W, 1>(bytes);
  if (e == cudaSuccess) e = set_attr_t<W, 2>(bytes);
  if (e == cudaSuccess) e = set_attr_t<W, 4>(bytes);
  if (e == cudaSuccess) e = set_attr_t<W, 8>(bytes);
  return e;
}

}  // namespace

}  // namespace ompk
