// Internal definitions shared by the kernels and the host runtime of the batched OMP library.
//
// Data layout in HBM (one handle):
//   dictionary (prepared once per A):
//     A32   N x Mp  float   atom rows, zero padded to Mp (64; 128 for E4M3) -- update / rescoring
//     A24h  N x Mp  u16     optional 24-bit copy for the update's q gather: each element rounded
//     A24l  N x Mp  u8      to nearest at 24 bits, split into its high 16 and next 8 bits
//     A16   N x Mp  bf16    RN-even copy                                     -- BF16 correlation
//     A8    N x Mp  e4m3    per-atom scaled copy, sa[n] = amax_n / 448        -- FP8 correlation
//     inv_norm[N] float = 1/||a_n|| (from FP64), norm2[N] double = ||a_n||^2
//     gram  N x N   float   G = A^T A (Sec. 2.2 precompute)
//   per signal, indexed by the signal id b (its row in Y):
//     R32   Bmax x Mp float  residual r (the master copy)
//     F     Bmax x Smax(Smax+1)/2 double  packed upper-triangular inverse Cholesky factor,
//           column j holds F[0..j, j] at offset j(j+1)/2 (Sec. 2.3)
//     bv    Bmax x Smax double  b_j = q_j^T r_{j-1} (so x = F b)
//     sup   Bmax x Smax int     support in selection order
//     ynorm, rnorm (float), niter, stop (int)
//   per live position p (the compacted order of the signals still iterating):
//     live[2][Bmax]  position -> signal id, ping-pong by iteration parity
//     livek[2][Bmax] position -> the signal's own iteration count (its niter when the list was
//                    written), beside live, so the update reads both in one round trip
//     cnt[Smax+2]    cnt[j+1] = live count after compaction j (cnt[0] = B)
//     flag[Bmax]     1 if the signal at position p continues after this iteration
//     Rq[2]          Bpad x Mp quantised residual rows in position order (tensor-core operand)
//     sr[2][Bpad]    per-position FP8 scale of Rq
//     cand1[Bmax]    FP32 path: packed (score, ~index) key, merged with atomicMax
//     cand2[Bmax]    FP32 path, margins recorded: the runner-up's key (every key that loses a
//                    merge, and each tile's own second best, is merged into it)
//     cand_s/cand_i  quantised paths: per position, candidate pieces x 8 (score, index)
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "../../include/omp_gb300.h"

namespace ompk {

constexpr int kMpAlign = 64;          // M padding (x2 for E4M3): one 128-byte K stage
constexpr int kSigTile = 128;         // signals per correlation tile (TMEM lanes)
constexpr int kMaxTopk = 8;
constexpr int kTauSmax = 64;          // the BF16 pruning threshold is kept for max_iters <= 64
constexpr int kPieces = 32;           // candidate slots per position (quantised paths)
constexpr int kTcParts = 2;           // candidate lists per signal and correlation CTA
constexpr double kDepRtol = 1e-10;    // dependent-atom test: delta <= 1e-10 ||a||^2
constexpr int kStopIters = 0, kStopEps = 1, kStopDependent = 2, kStopZero = 3;

// Quantised paths: a signal's pruning threshold for the correlation of step `step` and the score
// error bound (per unit of ||r||) of that step's quantised residual (see append.cuh)
struct alignas(16) TauRec {
  float tau;
  float eps;
  int step;
  int pad;
};

struct Ws {
  int M, Mp, N, Smax, Bmax, Bpad;
  int prec;        // omp_precision
  int topk;        // candidates rescored per signal (1 for FP32)
  int pieces;      // candidate slots per position (quantised paths)
  int tc_grid;     // tensor-core correlation: persistent grid size
  int tc_tn;       // atom tiles of 256
  int tc_cmin;     // minimum work units per CTA (bounds the pieces per signal tile)
  int tc_stages;   // operand stages of the correlation's pipeline (2..4; a pair 4 or 6; autotuned)
  int tc_cl;       // CTAs per correlation tile: 1, or 2 for the 2-SM MMA pair (autotuned)
  int upd_w;       // append/update kernel: warps per signal (1, 2, 4, 8; autotuned)
  int upd_persist; // append/update kernel: persistent grid taking positions from upd_ctr (autotuned)
  int* upd_ctr;    // Smax + 1 per-iteration position counters of the persistent form (zeroed by init)
  int64_t Fstride; // Smax (Smax + 1) / 2 rounded up to a multiple of 4
  // dictionary
  float* A32;
  uint16_t* A24h;  // 24-bit gather copy (optional): the high 16 bits of each element rounded to
  uint8_t* A24l;   // 24 bits (sign, exponent, 15 mantissa bits), and the next 8 bits
  __nv_bfloat16* A16;
  uint8_t* A8;
  float* sa;
  float* inv_norm;
  float* escale;   // quantised paths: score scale per atom (1/||a|| or s_a/||a||), padded
  double* norm2;
  float* gram;
  float* c0;        // Bmax x N FP32 first correlation of the Gram-space solve (allocated on use)
  // signal state
  float* R32;
  void* Rq[2];
  float* sr[2];
  int* live[2];
  int* livek[2];   // per position: the signal's iteration count when the list was written
  int* cnt;
  int* kdev;       // iteration counter of the graph's device-side loop
  float rescore_eps;  // bound on |quantised score - FP32 score| per unit of ||r|| (0: none)
  float* ea;       // quantised paths: max over atoms of ||q(a_n) - a_n|| / ||a_n|| (device scalar)
  float gam_tc, gam_32;  // accumulation bounds over Mp terms: tensor core and FP32 rescoring
  TauRec* tau;     // quantised paths with the bound: per signal, next step's threshold and bound
  float* tau_pos;  // the same per live position of the current step (0: no pruning); or null
  float* win_pos;  // per live position: three score error bounds at the row's residual (the
                   // window below the row's running best outside which columns are pruned)
  uint8_t* flag;
  unsigned long long* cand1;
  float* cand_s;
  int* cand_i;
  double* F;
  float* F32;      // FP32 copy of F (same packing) for the per-iteration triangular products
  double* bv;
  int* sup;
  float* ynorm;
  float* rnorm;
  int* niter;
  int* stop;
  float* drop;     // Bmax x Smax: normalised residual drop b_k^2 / ||r_{k-1}||^2 of each step
  float* margin;   // Bmax x Smax: top-two score margin (s1 - s2) / s1 of each step; null unless
                   // the solve records it (then the quantised paths rescore every candidate)
  unsigned long long* cand2;  // FP32 path with margins: the runner-up's packed key per position
  int* fb;         // Bmax: learned solve, step at which the signal left the restricted phase
  unsigned int* err;
};

// Per-call user pointers, written to device memory by a one-thread kernel before each solve so
// that a captured graph stays valid for any caller buffers.
struct CallArgs {
  const float* Y;
  float* X;
  int* support;
  int* n_iter;
  float* resid;
  int* stop;
  int* topk_idx;     // omp_correlate_topk outputs
  float* topk_score;
  float* drop;       // optional B x S trace of normalised residual drops
  float* margin;     // optional B x S trace of top-two score margins
  int* fallback;     // optional B: learned solve fallback step (-1 = none)
};

__device__ __forceinline__ unsigned long long pack_key(float score, int idx) {
  // scores are >= 0, so their IEEE bits order like unsigned integers; the low word is
  // ~idx so that on equal scores the smaller index gives the larger key
  return (static_cast<unsigned long long>(__float_as_uint(score)) << 32) |
         static_cast<unsigned long long>(0xFFFFFFFFu - static_cast<unsigned>(idx));
}
__device__ __forceinline__ int key_index(unsigned long long key) {
  return static_cast<int>(0xFFFFFFFFu - static_cast<unsigned>(key & 0xFFFFFFFFull));
}
__device__ __forceinline__ float key_score(unsigned long long key) {
  return __uint_as_float(static_cast<unsigned>(key >> 32));
}
// (s, i) beats (t, j): higher score, or equal score and lower index
__device__ __forceinline__ bool better(float s, int i, float t, int j) {
  return s > t || (s == t && i < j);
}

// value of an E4M3 code (the conversion intrinsic through half precision, which holds it exactly)
__device__ __forceinline__ float e4m3_to_float(__nv_fp8_storage_t c) {
  return __half2float(__half(__nv_cvt_fp8_to_halfraw(c, __NV_E4M3)));
}

// The score error bound of one step, per unit of ||a|| ||r||, from the actual relative
// quantisation errors of the atoms (ea, at most) and of the residual row (er): by Cauchy-Schwarz
// |<q(a), q(r)> - <a, r>| <= (ea + er + ea er) ||a|| ||r||, plus the tensor-core and the FP32
// rescoring accumulations, and 1% for the rounding of the norms, scales and of this bound.
__device__ __forceinline__ float data_bound(const Ws& ws, float ea, float er) {
  return 1.01f * (ea + er + ea * er + (1.f + ea) * (1.f + er) * ws.gam_tc + ws.gam_32);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over a 256-thread block; `red` holds >= 9 doubles of shared memory. All threads return
// the total. Contains __syncthreads (every thread of the block must call it).
__device__ __forceinline__ double block_sum256(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < 8 ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[8] = t;
  }
  __syncthreads();
  const double out = red[8];
  __syncthreads();
  return out;
}

// (s, e) <- s + x with the rounding error of the sum added into e exactly (Knuth's two-sum):
// s + e carries a sum of FP32 numbers to about twice FP32 precision with FP32 arithmetic only
__device__ __forceinline__ void two_sum(float& s, float& e, float x) {
  const float t = __fadd_rn(s, x);
  const float xv = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, xv)), __fsub_rn(x, xv));
  s = t;
  e = __fadd_rn(e, err);
}

// Iteration index of a per-iteration kernel: the launch's own k, or, when the launch passes -1
// (the body of the graph's device-side while loop, identical for every iteration), the counter
// that the loop advances.
__device__ __forceinline__ int iter_of(const Ws& ws, int k) { return k >= 0 ? k : *ws.kdev; }


// Persistent schedule of the tensor-core correlation (shared by the correlation kernel, which
// writes candidate slots, and the kernels that merge them). The G CTAs form clusters of CL, and
// cluster rank r works on signal tile s = CL sg + r of each group sg of CL consecutive tiles.
// Units u = sg * Tn + t over tile groups sg and atom tiles t; Geff clusters each own a
// contiguous range of at least `cmin` units (with CL = 1 a cluster is one CTA).
__host__ __device__ __forceinline__ void tc_sched(int L, int G, int Tn, int cmin, int CL, int& T,
                                                  int& Geff) {
  const int St = (L + kSigTile - 1) / kSigTile;
  T = (St + CL - 1) / CL * Tn;
  int g = T / cmin;
  if (g < 1) g = 1;
  const int nc = G / CL;
  Geff = g < nc ? g : nc;
}
__host__ __device__ __forceinline__ int tc_start(int g, int T, int Geff) {
  return static_cast<int>(static_cast<long long>(g) * T / Geff);
}
// the cluster whose range contains unit u
__host__ __device__ __forceinline__ int tc_owner(int u, int T, int Geff) {
  return static_cast<int>((static_cast<long long>(u + 1) * Geff - 1) / T);
}
// candidate slots [0, count) of live position p hold its signal tile's lists: kTcParts per
// piece (one per part of the atom columns of each unit)
__device__ __forceinline__ int tc_piece_count(const Ws& ws, int L, int p) {
  int T, Geff;
  tc_sched(L, ws.tc_grid, ws.tc_tn, ws.tc_cmin, ws.tc_cl, T, Geff);
  const int sg = p / kSigTile / ws.tc_cl;
  return kTcParts * (tc_owner(sg * ws.tc_tn + ws.tc_tn - 1, T, Geff) - tc_owner(sg * ws.tc_tn, T, Geff) + 1);
}

// ---------------------------------------------------------------------------------------------
// A kernel's dynamic shared memory limit is one setting of the process, shared by every handle,
// so it is only ever raised: handles with smaller layouts leave a larger one's limit in place.
// Thread-safe (update.cu).
cudaError_t raise_smem_limit(const void* kernel, size_t bytes);

// Host-side launchers (defined in the .cu files).
void launch_prep(const Ws& ws, const float* A, cudaStream_t s);
void launch_gram_simt(const Ws& ws, cudaStream_t s);
void launch_corr_simt(const Ws& ws, int k, int B, cudaStream_t s);
void launch_c0_simt(const Ws& ws, int B, cudaStream_t s);
void launch_gram_solve(const Ws& ws, const CallArgs* args, int B, int S, float eps, int eps_rel,
                       cudaStream_t s);
cudaError_t configure_gram_solve(const Ws& ws);
void launch_init(const Ws& ws, const CallArgs* args, int B, cudaStream_t s);
void launch_load_rows(const Ws& ws, const float* R, int B, cudaStream_t s);
// reuse: the update kernel of step j-1 has just written step j's quantised rows at the old
// positions, so blocks whose positions do not move keep them
void launch_compact(const Ws& ws, int j, int B, int S, bool reuse, cudaStream_t s);
void launch_advance(const Ws& ws, int S, cudaGraphConditionalHandle cond, cudaStream_t s);
void launch_update(const Ws& ws, int k, int B, int S, float eps, int eps_rel, cudaStream_t s);
void launch_finalize(const Ws& ws, const CallArgs* args, int B, int S, cudaStream_t s);
void launch_topk_out(const Ws& ws, const CallArgs* args, int B, int topk, cudaStream_t s);
void launch_set_args(CallArgs* dst, const CallArgs& v, cudaStream_t s);
cudaError_t configure_update_kernels(const Ws& ws);
int update_slots(int Mp, int W);
int update_default_warps(int Mp);
// per warp count (append_w1.cu .. append_w8.cu)
cudaError_t configure_update_w1(const Ws& ws);
cudaError_t configure_update_w2(const Ws& ws);
cudaError_t configure_update_w4(const Ws& ws);
cudaError_t configure_update_w8(const Ws& ws);
void launch_update_w1(const Ws& ws, int V, int k, int B, int S, float eps, int eps_rel, cudaStream_t s);
void launch_update_w2(const Ws& ws, int V, int k, int B, int S, float eps, int eps_rel, cudaStream_t s);
void launch_update_w4(const Ws& ws, int V, int k, int B, int S, float eps, int eps_rel, cudaStream_t s);
void launch_update_w8(const Ws& ws, int V, int k, int B, int S, float eps, int eps_rel, cudaStream_t s);

// learned proposal (restricted.cu, mlp.cu)
size_t restricted_smem_per_signal(int S, int K, int Mp);
bool launch_restricted(const Ws& ws, const CallArgs* args, const int* cand, int K, const float* tau,
                       int B, int S, float eps, int eps_rel, int* fallback, cudaStream_t s);
const int* proposal_candidates(omp_proposal p);
int proposal_topk(omp_proposal p);
const float* proposal_tau(omp_proposal p);
int proposal_tau_len(omp_proposal p);
float* proposal_tau_mut(omp_proposal p);
bool proposal_run_inference(omp_proposal p, const float* A, const float* Y, int B, cudaStream_t s);

// tensor-core correlation (corr_tc.cu)
struct TcPlan;
int tc_pieces();
void tc_fill_sched(Ws& ws, int sm_count);
cudaError_t tc_setup(const Ws& ws, int sm_count, TcPlan** plan);
void tc_destroy(TcPlan* plan);
void launch_corr_tc(const Ws& ws, const TcPlan* plan, int k, int B, cudaStream_t s);
int tc_fit_grid(int prec, int nst, int cl, int grid);

}  // namespace ompk
