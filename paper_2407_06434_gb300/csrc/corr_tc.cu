// Tensor-core correlation for the quantised paths (BF16 and FP8 E4M3), sm_103a tcgen05.
//
// C = Rq A_q^T over the live signals (Sec. 3.2 eq:bmm: one GEMM for all residuals), never
// written to memory: signals are the MMA's M dimension (128 TMEM lanes), atoms its N dimension
// (256 TMEM columns), the padded signal length the K dimension. Each epilogue thread owns one
// signal (one TMEM lane) and keeps a running top-8 of the score |c_n| * escale[n]
// (escale = 1/||a_n||, times the atom's FP8 scale on the E4M3 path; the signal's own scale is
// omitted because it does not change the order within a signal), scanning atoms in ascending
// order with a strict '>' so that the lowest index keeps a tie. The K2 update kernel merges the
// pieces' lists and rescores the best 8 in FP32.
//
// Persistent schedule: work units are (signal tile s, atom tile t), ordered signal-major,
// u = s * Tn + t; CTA g of Geff owns the contiguous units [floor(g T / Geff), floor((g+1) T /
// Geff)). A CTA flushes its list for signal tile s into candidate slot g - owner(s * Tn), so a
// tile's lists occupy consecutive slots. Geff is limited so that every CTA owns at least
// `cmin` units, which bounds the pieces per tile by kPieces.
//
// Pipeline (one CTA per SM, 192 threads):
//   warp 0 lane 0  TMA producer: 128 x 128-byte residual box + 256 x 128-byte atom box per stage
//   warp 1         TMEM allocation; lane 0 issues tcgen05.mma (4 per stage) and commits
//   warps 2..5     epilogue: tcgen05.ld 32 columns at a time, score, top-8
// Barriers: full/empty per smem stage, tfull/tempty per TMEM accumulator (2 x 256 columns).
// Every wait is bounded; on timeout the CTA raises OMP_DEVERR_WAIT_TIMEOUT, drains its own
// asynchronous copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"

namespace ompk {

namespace {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int KB = 128;  // K bytes per stage: one 128-byte swizzle row
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * KB;
constexpr int B_BYTES = BN * KB;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int THREADS = 192;
constexpr int TMEM_COLS = 2 * BN;
constexpr int STAGE_ROW = 36;  // floats per staged score row (float4 stores without conflicts)
constexpr int EPI_STAGE_BYTES = 4 * 32 * STAGE_ROW * 4;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256 + EPI_STAGE_BYTES;
constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false on timeout (raises the error word and the CTA's abort flag) or when
// another role of the CTA has aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned int* err) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort_flag = 1;
      atomicOr(err, OMP_DEVERR_WAIT_TIMEOUT);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// K-major operand in 128-byte swizzled rows: 8-row atoms 1024 bytes apart (SBO), version 1,
// layout SWIZZLE_128B. The K offset inside a row is added to the start address.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (static_cast<uint64_t>(1) << 16) |
         (static_cast<uint64_t>(1024 >> 4) << 32) | (static_cast<uint64_t>(1) << 46) |
         (static_cast<uint64_t>(2) << 61);
}

// Instruction descriptor: FP32 accumulator, A/B K-major, N = 256, M = 128;
// A/B format BF16 (kind::f16) or E4M3 (kind::f8f6f4).
template <int PREC>
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4) | ((PREC == OMP_PREC_BF16 ? 1u : 0u) << 7) |
         ((PREC == OMP_PREC_BF16 ? 1u : 0u) << 10) | (static_cast<uint32_t>(BN >> 3) << 17) |
         (static_cast<uint32_t>(BM >> 4) << 24);
}

template <int PREC>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t accumulate) {
  if (PREC == OMP_PREC_BF16) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc<PREC>()), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc<PREC>()), "r"(accumulate)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld32_issue(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Insert (v, n) into a descending top-8; the caller has checked v > s[7]. Equal scores keep
// the earlier (lower-index) entry in front.
__device__ __forceinline__ void top8_insert(float (&s)[8], int (&ix)[8], float v, int n) {
  s[7] = v;
  ix[7] = n;
#pragma unroll
  for (int q = 7; q > 0; --q) {
    if (s[q] > s[q - 1]) {
      const float ts = s[q];
      s[q] = s[q - 1];
      s[q - 1] = ts;
      const int ti = ix[q];
      ix[q] = ix[q - 1];
      ix[q - 1] = ti;
    }
  }
}

template <int PREC>
__global__ void __launch_bounds__(THREADS, 1)
    corr_tc_kernel(const __grid_constant__ CUtensorMap tm_r0, const __grid_constant__ CUtensorMap tm_r1,
                   const __grid_constant__ CUtensorMap tm_a, Ws ws, int k) {
  extern __shared__ uint8_t smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int L = ws.cnt[k + 1];
  int T, Geff;
  tc_sched(L, gridDim.x, ws.tc_tn, ws.tc_cmin, T, Geff);
  const int g = blockIdx.x;
  if (L <= 0 || g >= Geff) return;  // uniform across the CTA
  const int Tn = ws.tc_tn;
  const int u0 = tc_start(g, T, Geff), u1 = tc_start(g + 1, T, Geff);

  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t bars = base + STAGES * STAGE_BYTES;
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (STAGES + s); };
  auto tfull = [&](int a) { return bars + 8u * (2 * STAGES + a); };
  auto tempty = [&](int a) { return bars + 8u * (2 * STAGES + 2 + a); };
  const uint32_t drain = bars + 8u * (2 * STAGES + 4);
  uint8_t* bars_gen = smem_raw + (bars - raw);
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(bars_gen + 8 * (2 * STAGES + 5));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars_gen + 8 * (2 * STAGES + 5) + 4);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull(a), 1);
      mbar_init(tempty(a), 4);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(const_cast<uint32_t*>(tmem_slot))),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int esize = PREC == OMP_PREC_BF16 ? 2 : 1;
  const int kelems = KB / esize;                  // K elements per stage
  const int nk = ws.Mp * esize / KB;              // stages per unit
  const CUtensorMap* tm_r = (k & 1) ? &tm_r1 : &tm_r0;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------------ TMA producer
    int stage = 0;
    uint32_t ph = 0;
    int last_ph[STAGES];
#pragma unroll
    for (int s = 0; s < STAGES; ++s) last_ph[s] = -1;
    bool ok = true;
    for (int u = u0; u < u1 && ok; ++u) {
      const int s = u / Tn, t = u - s * Tn;
      for (int kc = 0; kc < nk; ++kc) {
        if (!mbar_wait(empty(stage), ph ^ 1u, abort_flag, ws.err)) {
          ok = false;
          break;
        }
        const uint32_t dst = base + stage * STAGE_BYTES;
        mbar_expect_tx(full(stage), STAGE_BYTES);
        tma_load_2d(dst, tm_r, kc * kelems, s * BM, full(stage));
        tma_load_2d(dst + A_BYTES, &tm_a, kc * kelems, t * BN, full(stage));
        last_ph[stage] = static_cast<int>(ph);
        if (++stage == STAGES) {
          stage = 0;
          ph ^= 1u;
        }
      }
    }
    if (!ok) {
      // let every copy this thread issued land before the CTA exits
      volatile int no_abort = 0;
      for (int s = 0; s < STAGES; ++s)
        if (last_ph[s] >= 0) mbar_wait(full(s), static_cast<uint32_t>(last_ph[s]), &no_abort, ws.err);
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------------ MMA issuer
    int stage = 0;
    uint32_t ph = 0;
    int acc = 0;
    uint32_t aph = 0;
    bool ok = true;
    for (int u = u0; u < u1 && ok; ++u) {
      if (!mbar_wait(tempty(acc), aph ^ 1u, abort_flag, ws.err)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem + static_cast<uint32_t>(acc * BN);
      for (int kc = 0; kc < nk; ++kc) {
        if (!mbar_wait(full(stage), ph, abort_flag, ws.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_addr = base + stage * STAGE_BYTES;
        const uint32_t b_addr = a_addr + A_BYTES;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma<PREC>(d, sdesc(a_addr + kk * 32), sdesc(b_addr + kk * 32), (kc | kk) != 0);
        mma_commit(empty(stage));
        if (++stage == STAGES) {
          stage = 0;
          ph ^= 1u;
        }
      }
      if (!ok) break;
      mma_commit(tfull(acc));
      acc ^= 1;
      if (acc == 0) aph ^= 1u;
    }
    // wait until every MMA this thread issued has completed
    mma_commit(drain);
    volatile int no_abort = 0;
    mbar_wait(drain, 0, &no_abort, ws.err);
  } else if (warp >= 2) {
    // ------------------------------------------------------------------ epilogue
    const int lg = warp & 3;                 // TMEM lane quarter this warp may access
    const int row = lg * 32 + lane;          // signal row within the tile
    float* stage_row = reinterpret_cast<float*>(bars_gen + 256) + ((warp - 2) * 32 + lane) * STAGE_ROW;
    int acc = 0;
    uint32_t aph = 0;
    int cur_s = -1;
    float ts[8];
    int ti[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      ts[q] = -1.f;
      ti[q] = -1;
    }
    auto flush = [&](int s) {
      const int p = s * BM + row;
      if (p < L) {
        const int piece = g - tc_owner(s * Tn, T, Geff);
        const size_t off = (static_cast<size_t>(p) * ws.pieces + piece) * kMaxTopk;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          ws.cand_s[off + q] = ts[q];
          ws.cand_i[off + q] = ti[q];
        }
      }
    };
    bool ok = true;
    for (int u = u0; u < u1; ++u) {
      const int s = u / Tn, t = u - s * Tn;
      if (s != cur_s) {
        if (cur_s >= 0) flush(cur_s);
        cur_s = s;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          ts[q] = -1.f;
          ti[q] = -1;
        }
      }
      if (!mbar_wait(tfull(acc), aph, abort_flag, ws.err)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t taddr = tmem + (static_cast<uint32_t>(lg * 32) << 16) + static_cast<uint32_t>(acc * BN);
      const int n0 = t * BN;
      // Scores of a 32-column chunk go to this lane's row of the warp's staging buffer; a
      // compare-only pass marks the columns above the current 8th score, and only those are
      // inserted (few per chunk once the list is warm), so the warp does not diverge per column.
      // The next chunk's TMEM load is in flight while this one is scored.
      uint32_t va[32], vb[32];
      tmem_ld32_issue(taddr, va);
      tmem_ld_wait();
#pragma unroll
      for (int c = 0; c < BN / 32; ++c) {
        uint32_t (&cur)[32] = (c & 1) ? vb : va;
        uint32_t (&nxt)[32] = (c & 1) ? va : vb;
        if (c + 1 < BN / 32) tmem_ld32_issue(taddr + (c + 1) * 32, nxt);
        const int nb = n0 + c * 32;
        const int lim = min(32, ws.N - nb);
        const float4* sc4 = reinterpret_cast<const float4*>(ws.escale + nb);
        const float thr = ts[7];
        uint32_t mask = 0;
#pragma unroll
        for (int j4 = 0; j4 < 8; ++j4) {
          const float4 sc = __ldg(sc4 + j4);
          float4 o;
          o.x = fabsf(__uint_as_float(cur[4 * j4 + 0])) * sc.x;
          o.y = fabsf(__uint_as_float(cur[4 * j4 + 1])) * sc.y;
          o.z = fabsf(__uint_as_float(cur[4 * j4 + 2])) * sc.z;
          o.w = fabsf(__uint_as_float(cur[4 * j4 + 3])) * sc.w;
          mask |= (o.x > thr ? 1u : 0u) << (4 * j4 + 0);
          mask |= (o.y > thr ? 1u : 0u) << (4 * j4 + 1);
          mask |= (o.z > thr ? 1u : 0u) << (4 * j4 + 2);
          mask |= (o.w > thr ? 1u : 0u) << (4 * j4 + 3);
          *reinterpret_cast<float4*>(stage_row + 4 * j4) = o;
        }
        if (lim < 32) mask &= lim > 0 ? (0xffffffffu >> (32 - lim)) : 0u;
        while (mask) {
          const int j = __ffs(mask) - 1;
          mask &= mask - 1;
          const float score = stage_row[j];
          if (score > ts[7]) top8_insert(ts, ti, score, nb + j);
        }
        if (c + 1 < BN / 32) tmem_ld_wait();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty(acc));
      acc ^= 1;
      if (acc == 0) aph ^= 1u;
    }
    if (ok && cur_s >= 0) flush(cur_s);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                 : "memory");
  }
}

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

// rows x Kbytes operand (K contiguous), box = box_rows x 128 bytes, 128-byte swizzle
bool make_map(CUtensorMap* m, void* ptr, int prec, uint64_t rows, uint64_t kelems, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int esize = prec == OMP_PREC_BF16 ? 2 : 1;
  const cuuint64_t dims[2] = {kelems, rows};
  const cuuint64_t strides[1] = {kelems * esize};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(KB / esize), box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(m, prec == OMP_PREC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8,
                        2, ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

struct TcPlan {
  CUtensorMap r0, r1, a;
  int grid;
};

int tc_pieces() { return kPieces; }

void tc_fill_sched(Ws& ws, int sm_count) {
  ws.tc_grid = sm_count;
  ws.tc_tn = (ws.N + BN - 1) / BN;
  ws.tc_cmin = (ws.tc_tn + (kPieces - 2) - 1) / (kPieces - 2);
}

cudaError_t tc_setup(const Ws& ws, int sm_count, TcPlan** plan) {
  *plan = nullptr;
  TcPlan* p = new TcPlan();
  p->grid = sm_count;
  void* a = ws.prec == OMP_PREC_BF16 ? static_cast<void*>(ws.A16) : static_cast<void*>(ws.A8);
  const bool ok = make_map(&p->r0, ws.Rq[0], ws.prec, ws.Bpad, ws.Mp, BM) &&
                  make_map(&p->r1, ws.Rq[1], ws.prec, ws.Bpad, ws.Mp, BM) &&
                  make_map(&p->a, a, ws.prec, ws.N, ws.Mp, BN);
  if (!ok) {
    delete p;
    return cudaErrorNotSupported;
  }
  cudaError_t e = cudaFuncSetAttribute(corr_tc_kernel<OMP_PREC_BF16>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(corr_tc_kernel<OMP_PREC_FP8_E4M3>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) {
    delete p;
    return e;
  }
  *plan = p;
  return cudaSuccess;
}

void tc_destroy(TcPlan* plan) { delete plan; }

void launch_corr_tc(const Ws& ws, const TcPlan* plan, int k, int B, cudaStream_t s) {
  (void)B;
  if (ws.prec == OMP_PREC_BF16)
    corr_tc_kernel<OMP_PREC_BF16><<<plan->grid, THREADS, SMEM_BYTES, s>>>(plan->r0, plan->r1, plan->a, ws, k);
  else
    corr_tc_kernel<OMP_PREC_FP8_E4M3><<<plan->grid, THREADS, SMEM_BYTES, s>>>(plan->r0, plan->r1, plan->a, ws, k);
}

}  // namespace ompk
