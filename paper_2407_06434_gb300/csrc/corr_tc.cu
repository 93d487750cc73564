// Tensor-core correlation for the quantised paths (BF16 and FP8 E4M3), sm_103a tcgen05.
//
// C = Rq A_q^T over the live signals (Sec. 3.2 eq:bmm: one GEMM for all residuals) on the shared
// persistent mainloop of tcgemm.cuh. Signals are the MMA's M dimension (128 TMEM lanes), atoms
// its N dimension (256 TMEM columns), the padded signal length the K dimension. C is never
// written: each epilogue thread owns one signal (one TMEM lane) and keeps a running top-8 of the
// score |c_n| * escale[n] (escale = 1/||a_n||, times the atom's FP8 scale on the E4M3 path; the
// signal's own scale is omitted because it does not change the order within a signal), scanning
// atoms in ascending order with a strict '>' so that the lowest index keeps a tie. The update
// kernel merges the pieces' lists and rescores the best 8 in FP32.
//
// The EPI_PARTS epilogue warps of a lane quarter see different column parts of each unit, so each
// keeps its own list; a CTA flushes them for signal tile s into candidate slots
// EPI_PARTS (g - owner(s * Tn)) + part, so a tile's lists occupy consecutive slots; the
// mainloop's minimum units per CTA (`cmin`) bounds the pieces per tile by kPieces / EPI_PARTS.
//
// Each row may carry a pruning threshold from the previous step's update (a lower bound on its
// best score less three score error bounds, see append.cuh): columns at or below it are not
// inserted, which removes most of the insertion work once the solve is past its first step.
#include "tcgemm.cuh"

namespace ompk {

namespace tcg {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// rows x K operand (K contiguous), box = box_rows x 128 bytes, 128-byte swizzle, zero fill
// outside the tensor
bool make_kmajor_map(CUtensorMap* m, const void* ptr, int prec, uint64_t rows, uint64_t kelems,
                     uint32_t box_rows, uint64_t ld) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int esize = prec == OMP_PREC_BF16 ? 2 : 1;
  const cuuint64_t dims[2] = {kelems, rows};
  const cuuint64_t strides[1] = {(ld ? ld : kelems) * esize};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(KB / esize), box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(m, prec == OMP_PREC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8,
                        2, const_cast<void*>(ptr), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

cudaError_t set_smem_attr(const void* kernel, int bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace tcg

namespace {

using namespace tcg;

// Running top-8 per signal; flushed when the CTA moves to another signal tile and at the end.
// The column scales of the warp's EPI_COLS columns are staged in its shared scratch at each
// unit, and those of the next column tile are loaded meanwhile, so no chunk waits on a global
// load.
//
// The EPI_PARTS threads of a row (one per part of the columns) publish their 8th-best score,
// tagged with the signal tile, in shared slots. A score below another part's 8th best is beaten
// by 8 scores of the same row, so it cannot be in the row's top 8 and is not inserted; the lists
// are then no longer each part's own top 8, but their union still holds the row's top 8, which
// is all the merge downstream needs. A stale value (the slots are read without a barrier) is
// smaller and only prunes less; a value tagged with another tile is ignored.
template <int PREC>
struct EpiTop8 {
  // Rows may be pruned by a threshold; each list then also keeps its running best column
  // as a key (score bits with the low 5 mantissa bits replaced by 31 - the column's place in its
  // chunk, so that an integer max takes the higher score and, within 2^-18, the lower index) and
  // emits it if nothing passed the threshold, so the merged lists always offer a runner-up
  static constexpr bool kTrack = true;
  Ws ws;
  int L;
  int g, T, Geff, row, part, cur_s;
  float ts[8];
  int ti[8];
  float* scr;
  unsigned long long* peers;
  float4 pf;  // prefetched scales of column tile pf_t (this lane's 4 of the warp's 128)
  int pf_t;
  uint32_t lbk;  // running best key of the list (kTrack) and its column
  int lbi;
  float thr0;    // this row's pruning threshold in the current signal tile (-1: none)
  float pf_tau;  // the row's threshold in signal tile pf_tau_s, loaded ahead
  int pf_tau_s;
  float win0;    // this row's window below its running best (0: none)
  float pf_win;  // the row's window in signal tile pf_tau_s, loaded ahead

  __device__ void reset() {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      ts[q] = -1.f;
      ti[q] = -1;
    }
    lbk = 0;
    lbi = -1;
  }
  __device__ void flush(int s) {
    const int p = s * BM + row;
    if (p >= L) return;
    if (kTrack && ti[0] < 0 && lbi >= 0) {
      // nothing passed the threshold: the list's best column, its score rounded up (the
      // rescoring shortcut reads list scores as upper bounds of the second best)
      ts[0] = __uint_as_float(lbk | 31u);
      ti[0] = lbi;
    }
    const int piece = g - tc_owner(s / ws.tc_cl * ws.tc_tn, T, Geff);
    const size_t off =
        (static_cast<size_t>(p) * ws.pieces + EPI_PARTS * piece + part) * kMaxTopk;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      ws.cand_s[off + q] = ts[q];
      ws.cand_i[off + q] = ti[q];
    }
  }
  // The update kernel's lower bound on the row's best score, less three score error bounds
  // (written per live position by the compaction, in the units of the scores); a column at or
  // below it can be neither the pick nor a rescoring candidate that changes it.
  __device__ float load_tau(int s) const {
    const int p = s * BM + row;
    if (!ws.tau_pos || p >= L) return -1.f;
    const float v = __ldg(ws.tau_pos + p);
    return v > 0.f ? v : -1.f;
  }
  // Three score error bounds at the row's residual (written per live position by the
  // compaction, in the units of the scores): a column whose score is that far below the best
  // score the row has shown so far is more than two bounds below the row's final best score,
  // outside the window of the FP32 rescoring, and its FP32 score is at least one bound below the
  // best FP32 score, so it can be neither the pick nor a rescoring candidate that changes it.
  // This prunes where no previous step left a threshold (the first step) as well as past the
  // best column.
  __device__ float load_win(int s) const {
    const int p = s * BM + row;
    if (!ws.win_pos || p >= L) return 0.f;
    const float v = __ldg(ws.win_pos + p);
    return v > 0.f ? v : 0.f;
  }
  // this lane's EPI_COLS / 32 consecutive scales of the warp's columns of tile t
  __device__ float4 load_scales(int t) const {
    static_assert(EPI_COLS == 128, "one float4 per lane");
    return __ldg(reinterpret_cast<const float4*>(ws.escale + t * BN + part * EPI_COLS) + (row & 31));
  }
  __device__ void begin(int g_, int T_, int Geff_, int row_, int part_, float* scratch,
                        unsigned long long* peers_) {
    scr = scratch;
    peers = peers_;
    pf_t = -1;
    g = g_;
    T = T_;
    Geff = Geff_;
    row = row_;
    part = part_;
    cur_s = -1;
    thr0 = -1.f;
    pf_tau_s = -1;
    win0 = 0.f;
    reset();
  }
  __device__ void unit(int s, int t) {
    if (s != cur_s) {
      if (cur_s >= 0) flush(cur_s);
      cur_s = s;
      reset();
      thr0 = pf_tau_s == s ? pf_tau : load_tau(s);
      win0 = pf_tau_s == s ? pf_win : load_win(s);
      pf_tau_s = s + ws.tc_cl;  // the next signal tile of this CTA's range, if any
      pf_tau = load_tau(s + ws.tc_cl);
      pf_win = load_win(s + ws.tc_cl);
    }
    const float4 v = pf_t == t ? pf : load_scales(t);
    __syncwarp();  // every lane has finished with the previous unit's scales
    reinterpret_cast<float4*>(scr)[row & 31] = v;
    __syncwarp();
    pf_t = t + 1 < ws.tc_tn ? t + 1 : 0;  // the next unit's column tile (units run t-major)
    pf = load_scales(pf_t);
  }
  // A compare-only pass marks the columns whose score beats the threshold; only those are
  // inserted (few per chunk once the list is warm), each read back from the registers with a
  // select tree, so the warp neither diverges per column nor needs a staging buffer. A fresh list
  // is seeded, without a per-column loop, with the best column of each group of 4 (lowest index
  // on ties): those 8 are distinct columns of the chunk, so their smallest score is a safe
  // threshold for the rest (at least 8 scores reach it), and a high one, which keeps the first
  // chunk's insertions few. A row with a pruning threshold is not seeded: its threshold already
  // holds back all but the few columns near the best, so its list may stay short of 8.
  __device__ void chunk(int, int t, int c0, const uint32_t (&cur)[32]) {
    const int nb = t * BN + c0;
    const int lim = min(32, ws.N - nb);
    const float* scl = scr + (c0 - part * EPI_COLS);
    const float4* sc4 = reinterpret_cast<const float4*>(scl);
    uint32_t seeded = 0;
    if (ti[0] < 0 && thr0 < 0.f) {
#pragma unroll
      for (int g = 0; g < 8; ++g) {
        float bv = -1.f;
        int bj = -1;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = 4 * g + q;
          const float v = fabsf(__uint_as_float(cur[j])) * scl[j];
          if (j < lim && v > bv) {  // false for NaN
            bv = v;
            bj = j;
          }
        }
        if (bj >= 0) {
          top8_insert(ts, ti, bv, nb + bj);
          seeded |= 1u << bj;
        }
      }
    }
    // own 8th best, raised to just below each other part's when that one is positive and
    // belongs to the same signal tile (x >= other  <=>  x > its predecessor, for x >= 0)
    float thr = fmaxf(ts[7], thr0);
#pragma unroll
    for (int o = 1; o < EPI_PARTS; ++o) {
      const int q = (part + o) % EPI_PARTS;
      const unsigned long long v = *reinterpret_cast<volatile unsigned long long*>(peers + q * BM + row);
      const float othr = __uint_as_float(static_cast<uint32_t>(v));
      if (static_cast<int>(v >> 32) == cur_s && othr > 0.f)
        thr = fmaxf(thr, __uint_as_float(__float_as_uint(othr) - 1u));
    }
    // The chunk's scores, as bits, and their largest: scores are non-negative, so they order as
    // their bits do (a NaN's bits above every number's). One multiply and one integer max per
    // column; the per-column threshold test and the best-column search below run only for a lane
    // whose largest score beats its threshold or its list's best key (few, once lists are warm).
    uint32_t sv[32];
    uint32_t mbits = 0;
#pragma unroll
    for (int j4 = 0; j4 < 8; ++j4) {
      const float4 sc = sc4[j4];
      sv[4 * j4 + 0] = __float_as_uint(fabsf(__uint_as_float(cur[4 * j4 + 0])) * sc.x);
      sv[4 * j4 + 1] = __float_as_uint(fabsf(__uint_as_float(cur[4 * j4 + 1])) * sc.y);
      sv[4 * j4 + 2] = __float_as_uint(fabsf(__uint_as_float(cur[4 * j4 + 2])) * sc.z);
      sv[4 * j4 + 3] = __float_as_uint(fabsf(__uint_as_float(cur[4 * j4 + 3])) * sc.w);
#pragma unroll
      for (int q = 0; q < 4; ++q) mbits = max(mbits, sv[4 * j4 + q]);
    }
    // the list's best column as a key: score bits with the low 5 replaced by 31 - the column's
    // place, so that among scores equal above those bits the lowest column wins; columns past N
    // score 0 (zero escale), so they never beat a real column's key
    if (kTrack && (mbits & ~31u) > (lbk & ~31u)) {  // strictly higher: an earlier column keeps a tie
      int jb = 31;
#pragma unroll
      for (int j = 31; j >= 0; --j)
        if ((sv[j] & ~31u) == (mbits & ~31u)) jb = j;
      lbk = (mbits & ~31u) | static_cast<uint32_t>(31 - jb);
      lbi = nb + jb;
    }
    // the window below the running best (lower bounds of scores this thread has seen, this
    // chunk's largest included), rounded down
    if (win0 > 0.f) {
      const float best = fmaxf(ts[0], __uint_as_float(lbk & ~31u));
      thr = fmaxf(thr, best * (1.f - 0x1p-20f) - win0);
    }
    // x > thr for x, thr >= 0 exactly when bits(x) > bits(thr); a negative thr (an unfilled list
    // with no pruning threshold) passes every column
    uint32_t mask = 0;
    if (thr < 0.f || mbits > __float_as_uint(thr)) {
#pragma unroll
      for (int j = 0; j < 32; ++j) mask |= (__uint_as_float(sv[j]) > thr ? 1u : 0u) << j;
      if (lim < 32) mask &= lim > 0 ? (0xffffffffu >> (32 - lim)) : 0u;
      mask &= ~seeded;
    }
    while (mask) {
      const int j = __ffs(mask) - 1;
      mask &= mask - 1;
      const float score = __uint_as_float(pick32(sv, j));
      if (score > ts[7]) top8_insert(ts, ti, score, nb + j);
    }
    *reinterpret_cast<volatile unsigned long long*>(peers + part * BM + row) =
        (static_cast<unsigned long long>(static_cast<uint32_t>(cur_s)) << 32) | __float_as_uint(ts[7]);
  }
  __device__ void end(bool ok) {
    if (ok && cur_s >= 0) flush(cur_s);
  }
};

// CL CTAs per cluster (1, or a pair running the 2-SM MMA); tm_a's box is BN / CL atoms (each CTA
// of a pair loads half of the atom tile)
template <int PREC, int NST, int CL>
__global__ void __launch_bounds__(THREADS, 1)
    corr_tc_kernel(const __grid_constant__ CUtensorMap tm_r0, const __grid_constant__ CUtensorMap tm_r1,
                   const __grid_constant__ CUtensorMap tm_a, Ws ws, int k) {
  k = iter_of(ws, k);
  const int L = ws.cnt[k + 1];
  if (L <= 0) return;
  EpiTop8<PREC> epi;
  epi.ws = ws;
  epi.L = L;
  const int row_tiles = (L + BM - 1) / BM;
  const int ktiles = ws.Mp * (PREC == OMP_PREC_BF16 ? 2 : 1) / KB;
  gemm_body<PREC, EpiTop8<PREC>, NST, CL>((k & 1) ? &tm_r1 : &tm_r0, &tm_a, row_tiles, ws.tc_tn,
                                          ktiles, ws.tc_cmin, ws.err, epi);
}

}  // namespace

struct TcPlan {
  CUtensorMap r0, r1;
  CUtensorMap a[2];  // atoms in boxes of BN rows (one CTA) and BN / 2 rows (a pair)
  int grid;
};

int tc_pieces() { return kPieces; }

void tc_fill_sched(Ws& ws, int sm_count) {
  ws.tc_grid = sm_count;
  ws.tc_stages = STAGES;
  ws.tc_cl = 1;
  ws.tc_tn = (ws.N + BN - 1) / BN;
  // a tile of Tn units meets at most ceil(Tn / cmin) + 1 CTA ranges of >= cmin units
  constexpr int kMaxPieces = kPieces / EPI_PARTS;
  ws.tc_cmin = (ws.tc_tn + (kMaxPieces - 2) - 1) / (kMaxPieces - 2);
}

namespace {
template <int PREC, int NST, int CL>
const void* kern() {
  return reinterpret_cast<const void*>(corr_tc_kernel<PREC, NST, CL>);
}
// Pairs only where one CTA fills more than half an SM's shared memory (4 or 6 stages of 32 KB).
// Two CTAs on one SM would take turns at the whole of its TMEM (tcgen05.alloc waits), and two
// pairs, each with one CTA holding an SM's TMEM and one waiting for the other's SM, would wait
// for each other at the cluster barrier for ever.
static_assert(2 * smem_bytes(4, 2) > 232448, "a paired CTA must fill more than half an SM");
// every instantiation of one precision, by stages and cluster size: 2, 3, 4 stages of 48 KB for
// one CTA, 4 or 6 of 32 KB for a pair (the 2-SM MMA); nullptr for any other pair of values
template <int PREC>
const void* kern_of(int nst, int cl) {
  if (cl == 2) return nst == 4 ? kern<PREC, 4, 2>() : nst == 6 ? kern<PREC, 6, 2>() : nullptr;
  if (cl == 1)
    return nst == 2 ? kern<PREC, 2, 1>() : nst == 3 ? kern<PREC, 3, 1>() : nst == 4 ? kern<PREC, 4, 1>() : nullptr;
  return nullptr;
}
const void* kern_of(int prec, int nst, int cl) {
  return prec == OMP_PREC_BF16 ? kern_of<OMP_PREC_BF16>(nst, cl) : kern_of<OMP_PREC_FP8_E4M3>(nst, cl);
}
int cl_index(int cl) { return cl == 2 ? 1 : 0; }
}  // namespace

cudaError_t tc_setup(const Ws& ws, int sm_count, TcPlan** plan) {
  *plan = nullptr;
  TcPlan* p = new TcPlan();
  p->grid = sm_count;
  const void* a = ws.prec == OMP_PREC_BF16 ? static_cast<const void*>(ws.A16) : static_cast<const void*>(ws.A8);
  const bool ok = make_kmajor_map(&p->r0, ws.Rq[0], ws.prec, ws.Bpad, ws.Mp, BM) &&
                  make_kmajor_map(&p->r1, ws.Rq[1], ws.prec, ws.Bpad, ws.Mp, BM) &&
                  make_kmajor_map(&p->a[0], a, ws.prec, ws.N, ws.Mp, BN) &&
                  make_kmajor_map(&p->a[1], a, ws.prec, ws.N, ws.Mp, BN / 2);
  if (!ok) {
    delete p;
    return cudaErrorNotSupported;
  }
  cudaError_t e = cudaSuccess;
  for (int prec : {static_cast<int>(OMP_PREC_BF16), static_cast<int>(OMP_PREC_FP8_E4M3)})
    for (int nst : {2, 3, 4, 6})
      for (int cl = 1; cl <= 2; ++cl)
        if (e == cudaSuccess && kern_of(prec, nst, cl))
          e = set_smem_attr(kern_of(prec, nst, cl), smem_bytes(nst, cl));
  if (e != cudaSuccess) {
    delete p;
    return e;
  }
  *plan = p;
  return cudaSuccess;
}

void tc_destroy(TcPlan* plan) { delete plan; }

// The grid for clusters of `cl` CTAs: at most `grid` CTAs, a multiple of cl, no more clusters
// than fit on the device at once (0 if none fit, or if there is no such kernel).
int tc_fit_grid(int prec, int nst, int cl, int grid) {
  const int want = grid / cl;
  if (!kern_of(prec, nst, cl)) return 0;
  if (cl == 1 || want < 1) return want * cl;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(static_cast<unsigned>(want * cl));
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = smem_bytes(nst, cl);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern_of(prec, nst, cl), &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (n < want ? n : want) * cl;
}

void launch_corr_tc(const Ws& ws, const TcPlan* plan, int k, int B, cudaStream_t s) {
  (void)B;
  // the persistent grid is the workspace's (the candidate slots are laid out for it), a
  // multiple of the cluster size
  const int cl = ws.tc_cl;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(static_cast<unsigned>(ws.tc_grid));
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = smem_bytes(ws.tc_stages, cl);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = cl > 1 ? 1 : 0;
  const CUtensorMap* r0 = &plan->r0;
  const CUtensorMap* r1 = &plan->r1;
  const CUtensorMap* am = &plan->a[cl_index(cl)];
  void* args[] = {const_cast<CUtensorMap*>(r0), const_cast<CUtensorMap*>(r1), const_cast<CUtensorMap*>(am),
                  const_cast<Ws*>(&ws), &k};
  const void* kernel = kern_of(ws.prec, ws.tc_stages, cl);
  if (kernel && ws.tc_grid % cl == 0) cudaLaunchKernelExC(&cfg, kernel, args);  // else: no shape
}

}  // namespace ompk
