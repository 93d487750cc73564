// Persistent tcgen05 GEMM mainloop shared by the correlation (corr_tc.cu) and the learned
// proposal network (mlp.cu): C = A_op B_op^T with both operands K-major in HBM, loaded by TMA
// with 128-byte swizzle, multiplied by tcgen05.mma into FP32 accumulators in TMEM, and handed to
// an epilogue functor 32 columns at a time. C is never written by the mainloop itself.
//
// Tiles: 128 rows of A_op (MMA M = the TMEM lanes) x 256 rows of B_op (MMA N = TMEM columns),
// K in 128-byte stages (64 BF16 or 128 E4M3 elements, 4 MMAs of 32 bytes each per stage).
// Schedule: units u = s * Tn + t over row tiles s and column tiles t; CTA g of Geff owns the
// contiguous range [floor(g T / Geff), floor((g + 1) T / Geff)), Geff = min(grid, T / cmin).
// CTA pairs (template CL = 2, the correlation's choice): the two CTAs of a cluster run the same
// column tiles in lockstep on two consecutive row tiles (units then run over row-tile pairs, g
// and Geff count pairs), as one 256-row MMA across the two SMs (see the mainloop).
//
// Roles (64 + 128 EPI_PARTS threads, one CTA per SM):
//   warp 0 lane 0  TMA producer, NST stages (4 by default; for the correlation 2, 3 or 4, the
//                  autotuner's choice) of 16 KB (A_op) + 32 KB (B_op), or for a CTA pair 4 or 6
//                  stages of 16 KB + 16 KB; with one CTA it issues the first NST stages as soon as
//                  it has initialised the barriers, before the tensor memory is allocated
//   warp 1         TMEM allocation (2 x 256 columns); lane 0 issues the MMAs and commits
//   warps 2..      epilogue, EPI_PARTS warps per TMEM lane quarter (a warp may only read the
//                  quarter warp % 4), each over EPI_COLS of the unit's 256 columns: tcgen05.ld
//                  of 32 columns, functor call
// Every mbarrier wait is bounded (about 2 s); a timeout raises OMP_DEVERR_WAIT_TIMEOUT, the
// roles drain their own copies and MMAs, TMEM is freed and the CTA returns.
//
// Epilogue functor interface (one object per epilogue thread, `row` = its TMEM lane 0..127,
// `part` = which EPI_COLS of the unit's 256 columns it sees, starting at part * EPI_COLS):
//   void begin(int g, int T, int Geff, int row, int part, float* scratch,
//              unsigned long long* peers);
//   void unit(int s, int t);                              // before the unit's chunks
// `scratch` is EPI_SCRATCH floats of shared memory private to the thread's warp; `peers` is
// EPI_PARTS x BM 8-byte shared slots, [part][row], through which the threads of a row may
// talk. The mainloop sets every slot to 0xffffffff00000000 before the first unit.
//   void chunk(int s, int t, int c0, const uint32_t (&v)[32]);   // columns c0..c0+31 of the tile
//   void end(bool ok);                                    // after the last unit
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"

namespace ompk {
namespace tcg {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int KB = 128;  // K bytes per stage: one 128-byte swizzle row
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * KB;
constexpr int B_BYTES = BN * KB;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int EPI_PARTS = kTcParts;           // epilogue warps per TMEM lane quarter
constexpr int EPI_WARPS = 4 * EPI_PARTS;
constexpr int EPI_COLS = BN / EPI_PARTS;      // columns of a unit each epilogue warp sees
constexpr int THREADS = 64 + 32 * EPI_WARPS;
static_assert(THREADS >= EPI_PARTS * BM, "the peer slots are initialised one per thread");
static_assert(EPI_COLS % 32 == 0, "epilogue chunks are 32 columns");
constexpr int TMEM_COLS = 2 * BN;
constexpr int EPI_SCRATCH = EPI_COLS;  // shared floats per epilogue warp
// Bytes of an operand stage: the A_op tile and the B_op tile, or for a CTA pair (cl = 2, the
// 2-SM MMA) the A_op tile and half the B_op tile.
__host__ __device__ constexpr int stage_bytes(int cl) { return BM * KB + (cl == 2 ? BN / 2 : BN) * KB; }
// dynamic shared memory of a mainloop with `nst` operand stages
__host__ __device__ constexpr int smem_bytes(int nst, int cl = 1) {
  return nst * stage_bytes(cl) + 1024 + 256 + EPI_WARPS * EPI_SCRATCH * 4 + EPI_PARTS * BM * 8;
}
static_assert(smem_bytes(6, 2) <= 232448, "6 pair stages fit in a CTA's shared memory");
constexpr int SMEM_BYTES = smem_bytes(STAGES);
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

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// every thread of every CTA of the cluster; orders the mbarrier initialisations before any
// peer's copy or arrival
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
// arrive on the mbarrier at shared offset `bar` of cluster CTA `rank`
__device__ __forceinline__ void mbar_arrive_remote(uint32_t bar, uint32_t rank) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(bar), "r"(rank));
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(ra) : "memory");
}
__device__ __forceinline__ bool mbar_try_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
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

// Instruction descriptor: FP32 accumulator, A/B K-major, N = 256, M = 128 (one CTA) or 256 (a CTA
// pair, PAIR); A/B format BF16 (kind::f16) or E4M3 (kind::f8f6f4).
template <int PREC, bool PAIR = false>
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4) | ((PREC == OMP_PREC_BF16 ? 1u : 0u) << 7) |
         ((PREC == OMP_PREC_BF16 ? 1u : 0u) << 10) | (static_cast<uint32_t>(BN >> 3) << 17) |
         (static_cast<uint32_t>((PAIR ? 2 * BM : BM) >> 4) << 24);
}

// One MMA. With PAIR (issued by the pair's even CTA only) it spans both CTAs: rows 0..127 of
// A_op and of D in this CTA, rows 128..255 in the peer, and half of B_op's rows in each, all at
// the same shared and tensor-memory offsets.
template <int PREC, bool PAIR = false>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t accumulate) {
  if (PREC == OMP_PREC_BF16 && !PAIR) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc<PREC, PAIR>()), "r"(accumulate)
        : "memory");
  } else if (!PAIR) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc<PREC, PAIR>()), "r"(accumulate)
        : "memory");
  } else if (PREC == OMP_PREC_BF16) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc<PREC, PAIR>()), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc<PREC, PAIR>()), "r"(accumulate)
        : "memory");
  }
}

// Arrive on the mbarrier at offset `bar` once this thread's MMAs have completed: of this CTA, or
// with `mask` of every cluster CTA in it. PAIR: the commit of pair MMAs (every tcgen05 operation
// of a pair kernel is cta_group::2).
template <bool PAIR = false>
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  if (PAIR)
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
  else
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
// The pair's commit: one arrival on the mbarrier at offset `bar` of each CTA of the pair (this
// one, and the peer through its shared::cluster address), once this thread's MMAs have completed
__device__ __forceinline__ void mma_commit_pair(uint32_t bar, uint32_t peer_bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(peer_bar)
               : "memory");
}

// A copy into this CTA's shared memory that completes on an mbarrier of either CTA of the pair
// (`bar_cl` a shared::cluster address)
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, int x, int y,
                                                 uint32_t bar_cl) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar_cl)
      : "memory");
}
// the shared::cluster address of offset `a` in cluster CTA `rank`
__device__ __forceinline__ uint32_t cluster_addr(uint32_t a, uint32_t rank) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  return ra;
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
// The same wait, with the loaded registers as its operands, so that no read of them is
// scheduled before it
__device__ __forceinline__ void tmem_ld_wait(uint32_t (&v)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]),
                 "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]),
                 "+r"(v[13]), "+r"(v[14]), "+r"(v[15]), "+r"(v[16]), "+r"(v[17]), "+r"(v[18]),
                 "+r"(v[19]), "+r"(v[20]), "+r"(v[21]), "+r"(v[22]), "+r"(v[23]), "+r"(v[24]),
                 "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]), "+r"(v[29]), "+r"(v[30]),
                 "+r"(v[31])
               :
               : "memory");
}

// v[j] for a run-time j without local memory: a 5-level select tree
__device__ __forceinline__ uint32_t pick32(const uint32_t (&v)[32], int j) {
  uint32_t a[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = (j & 16) ? v[i + 16] : v[i];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = (j & 8) ? a[i + 8] : a[i];
#pragma unroll
  for (int i = 0; i < 4; ++i) a[i] = (j & 4) ? a[i + 4] : a[i];
#pragma unroll
  for (int i = 0; i < 2; ++i) a[i] = (j & 2) ? a[i + 2] : a[i];
  return (j & 1) ? a[1] : a[0];
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


// ------------------------------------------------------------------------------- mainloop
// CL = 1: one CTA per unit. CL = 2: a CTA pair on two SMs runs one 256 x 256 MMA per K step
// (tcgen05 cta_group::2, issued by the even CTA): each CTA holds its own 128 A_op rows and half
// of the B_op tile, so an SM takes in 32 KB per stage instead of 48 KB; the peer's copies
// complete on the even CTA's full barriers, the even CTA's commits reach both CTAs' empty and
// accumulator barriers, and both CTAs' epilogues release the accumulator to the even CTA.
template <int PREC, class Epi, int NST = STAGES, int CL = 1>
__device__ __forceinline__ void gemm_body(const CUtensorMap* tm_a, const CUtensorMap* tm_b,
                                          int row_tiles, int col_tiles, int ktiles, int cmin,
                                          unsigned int* err, Epi& epi) {
  static_assert(CL == 1 || CL == 2, "one CTA or a CTA pair");
  constexpr bool PAIR = CL == 2;
  extern __shared__ uint8_t smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // with CL = 2 the launch is in clusters of two consecutive CTAs; rank r takes signal tile
  // 2 sg + r of each unit's tile pair sg and loads rows [r BN / 2, (r + 1) BN / 2) of the unit's
  // B_op tile
  const int rank = CL > 1 ? static_cast<int>(cluster_rank()) : 0;
  const bool lead = rank == 0;  // PAIR: the CTA that issues the MMAs
  const int T = (row_tiles + CL - 1) / CL * col_tiles;
  if (T <= 0) return;
  int Geff = T / (cmin > 0 ? cmin : 1);
  if (Geff < 1) Geff = 1;
  if (Geff > static_cast<int>(gridDim.x) / CL) Geff = gridDim.x / CL;
  const int g = blockIdx.x / CL;
  if (g >= Geff) return;  // uniform across the cluster
  const int Tn = col_tiles;
  constexpr int SA = A_BYTES;              // this CTA's A_op tile, then its B_op rows
  constexpr int SS = stage_bytes(CL);
  const int u0 = static_cast<int>(static_cast<long long>(g) * T / Geff);
  const int u1 = static_cast<int>(static_cast<long long>(g + 1) * T / Geff);

  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t bars = base + NST * SS;
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (NST + s); };
  auto tfull = [&](int a) { return bars + 8u * (2 * NST + a); };
  auto tempty = [&](int a) { return bars + 8u * (2 * NST + 2 + a); };
  const uint32_t drain = bars + 8u * (2 * NST + 4);
  const uint32_t done = bars + 8u * (2 * NST + 5);  // the cluster's CTAs have finished
  uint8_t* bars_gen = smem_raw + (bars - raw);
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(bars_gen + 8 * (2 * NST + 6));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars_gen + 8 * (2 * NST + 6) + 4);

  const int kelems = KB / (PREC == OMP_PREC_BF16 ? 2 : 1);  // K elements per stage
  int n_pre = 0;  // one CTA: stages the producer thread issued before the block barrier
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull(a), 1);
      mbar_init(tempty(a), PAIR ? 2 * EPI_WARPS : EPI_WARPS);  // PAIR: both CTAs' epilogues
    }
    mbar_init(drain, 1);
    mbar_init(done, CL);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (CL == 1) {
      // This thread is the producer: with one CTA it fetches both tensor maps and issues the
      // first NST stages now, in the producer loop's order, so that they are in flight while
      // warp 1 allocates the tensor memory and the block meets at the barrier below. (A pair
      // waits for the cluster barrier: its copies complete on the other CTA's barriers.)
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tm_a)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tm_b)) : "memory");
      for (int u = u0; u < u1 && n_pre < NST; ++u) {
        const int sg = u / Tn, t = u - sg * Tn;
        for (int kc = 0; kc < ktiles && n_pre < NST; ++kc) {
          const uint32_t dst = base + n_pre * SS;
          mbar_expect_tx(full(n_pre), SS);
          tma_load_2d(dst, tm_a, kc * kelems, sg * BM, full(n_pre));
          tma_load_2d(dst + SA, tm_b, kc * kelems, t * BN, full(n_pre));
          ++n_pre;
        }
      }
    }
  }
  unsigned long long* peers =
      reinterpret_cast<unsigned long long*>(bars_gen + 256 + EPI_WARPS * EPI_SCRATCH * 4);
  if (threadIdx.x < EPI_PARTS * BM) peers[threadIdx.x] = 0xffffffff00000000ull;  // tag -1
  if (warp == 1) {
    // PAIR: one warp of each CTA of the pair allocates, together
    if (PAIR) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(const_cast<uint32_t*>(tmem_slot))),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(const_cast<uint32_t*>(tmem_slot))),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  if (CL > 1) cluster_sync();  // no copy or arrival reaches a peer's barriers before their init
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------------ TMA producer
    int stage = 0;
    uint32_t ph = 0;
    int last_ph[NST];
#pragma unroll
    for (int s = 0; s < NST; ++s) last_ph[s] = -1;
    bool ok = true;
    for (int u = u0; u < u1 && ok; ++u) {
      const int sg = u / Tn, t = u - sg * Tn;
      const int s = sg * CL + rank;
      for (int kc = 0; kc < ktiles; ++kc) {
        if (n_pre > 0) {  // issued before the block barrier (stage n_pre counts up from 0)
          --n_pre;
        } else {
          if (!mbar_wait(empty(stage), ph ^ 1u, abort_flag, err)) {
            ok = false;
            break;
          }
          const uint32_t dst = base + stage * SS;
          if (PAIR) {
            // both CTAs' copies of the stage complete on the even CTA's full barrier, which
            // expects the bytes of both
            if (lead) mbar_expect_tx(full(stage), 2 * SS);
            const uint32_t fb = cluster_addr(full(stage), 0);
            tma_load_2d_pair(dst, tm_a, kc * kelems, s * BM, fb);
            tma_load_2d_pair(dst + SA, tm_b, kc * kelems, t * BN + rank * (BN / 2), fb);
          } else {
            mbar_expect_tx(full(stage), SS);
            tma_load_2d(dst, tm_a, kc * kelems, s * BM, full(stage));
            tma_load_2d(dst + SA, tm_b, kc * kelems, t * BN, full(stage));
          }
        }
#pragma unroll
        for (int q = 0; q < NST; ++q)  // static indices keep last_ph in registers
          if (q == stage) last_ph[q] = static_cast<int>(ph);
        if (++stage == NST) {
          stage = 0;
          ph ^= 1u;
        }
      }
    }
    if (!ok && (!PAIR || lead)) {
      // let every copy this thread issued land before the CTA exits (a pair's odd CTA cannot
      // see its copies complete: they signal the even CTA, which drains them with its own)
      volatile int no_abort = 0;
      for (int s = 0; s < NST; ++s)
        if (last_ph[s] >= 0) mbar_wait(full(s), static_cast<uint32_t>(last_ph[s]), &no_abort, err);
    }
  } else if (warp == 1 && lane == 0 && (!PAIR || lead)) {
    // ------------------------------------------------------------------ MMA issuer
    int stage = 0;
    uint32_t ph = 0;
    int acc = 0;
    uint32_t aph = 0;
    bool ok = true;
    for (int u = u0; u < u1 && ok; ++u) {
      if (!mbar_wait(tempty(acc), aph ^ 1u, abort_flag, err)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem + static_cast<uint32_t>(acc * BN);
      for (int kc = 0; kc < ktiles; ++kc) {
        if (!mbar_wait(full(stage), ph, abort_flag, err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_addr = base + stage * SS;
        const uint32_t b_addr = a_addr + SA;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma<PREC, PAIR>(d, sdesc(a_addr + kk * 32), sdesc(b_addr + kk * 32), (kc | kk) != 0);
        if (PAIR)
          mma_commit_pair(empty(stage), cluster_addr(empty(stage), 1));  // both may refill it
        else
          mma_commit<false>(empty(stage));
        if (++stage == NST) {
          stage = 0;
          ph ^= 1u;
        }
      }
      if (!ok) break;
      if (PAIR)
        mma_commit_pair(tfull(acc), cluster_addr(tfull(acc), 1));  // both accumulators are ready
      else
        mma_commit<false>(tfull(acc));
      acc ^= 1;
      if (acc == 0) aph ^= 1u;
    }
    // wait until every MMA this thread issued has completed
    mma_commit<PAIR>(drain);
    volatile int no_abort = 0;
    mbar_wait(drain, 0, &no_abort, err);
  } else if (warp >= 2) {
    // ------------------------------------------------------------------ epilogue
    const int lg = warp & 3;           // TMEM lane quarter this warp may access
    const int row = lg * 32 + lane;    // row within the tile
    const int part = (warp - 2) / 4;   // which EPI_COLS of the unit's columns
    constexpr int CH = EPI_COLS / 32;  // 32-column chunks per part
    float* scratch = reinterpret_cast<float*>(bars_gen + 256) + (warp - 2) * EPI_SCRATCH;
    epi.begin(g, T, Geff, row, part, scratch, peers);
    int acc = 0;
    uint32_t aph = 0;
    bool ok = true;
    for (int u = u0; u < u1; ++u) {
      const int sg = u / Tn, t = u - sg * Tn;
      const int s = sg * CL + rank;
      epi.unit(s, t);
      if (!mbar_wait(tfull(acc), aph, abort_flag, err)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t taddr = tmem + (static_cast<uint32_t>(lg * 32) << 16) +
                             static_cast<uint32_t>(acc * BN + part * EPI_COLS);
      // one 32-column load at a time (the wait takes the loaded registers as operands, so no
      // read of them moves above it); once the last load has landed the accumulator goes back
      // to the MMA (PAIR: to the even CTA's barrier) before that chunk is scanned
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        uint32_t cur[32];
        tmem_ld32_issue(taddr + c * 32, cur);
        tmem_ld_wait(cur);
        if (c + 1 == CH) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) {
            if (PAIR && !lead)
              mbar_arrive_remote(tempty(acc), 0);
            else
              mbar_arrive(tempty(acc));
          }
        }
        epi.chunk(s, t, part * EPI_COLS + c * 32, cur);
      }
      acc ^= 1;
      if (acc == 0) aph ^= 1u;
    }
    epi.end(ok);
  }
  tc_fence_before();
  __syncthreads();
  if (CL > 1) {
    // The even CTA's MMAs into the odd CTA's tensor memory and their arrivals on its barriers
    // must not outlive either CTA: each CTA, its MMAs drained, tells both, and goes on once both
    // have told it (bounded: a peer that timed out arrives within its own limits)
    if (threadIdx.x == 0) {
      for (int r = 0; r < CL; ++r) mbar_arrive_remote(done, static_cast<uint32_t>(r));
      const long long t0 = clock64();
      while (!mbar_try_cluster(done, 0)) {
        if (clock64() - t0 > 4 * kWaitCycles) {
          atomicOr(err, OMP_DEVERR_WAIT_TIMEOUT);
          break;
        }
      }
    }
    __syncthreads();
  }
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    if (PAIR)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                   : "memory");
  }
}

// --------------------------------------------------------------------------- host helpers
// ld: row stride in elements (0 = kelems)
bool make_kmajor_map(CUtensorMap* m, const void* ptr, int prec, uint64_t rows, uint64_t kelems,
                     uint32_t box_rows, uint64_t ld = 0);
cudaError_t set_smem_attr(const void* kernel, int bytes = SMEM_BYTES);

}  // namespace tcg
}  // namespace ompk
