/*
 * omp_gb300.h -- batched Orthogonal Matching Pursuit on one NVIDIA GB300 (sm_103a).
 *
 * The method is Alg. 1 of "A Practical GPU-Accelerated Implementation of Orthogonal Matching
 * Pursuit" (arXiv 2407.06434): for k = 1..S pick n* = argmax_n |<r_{k-1}, a_n>| / ||a_n||, add
 * n* to the support, solve least squares on the support and set r_k = y - A_S x_k; stop when
 * ||r_k|| <= eps. The least squares step uses the inverse-Cholesky recurrence of Sec. 2.3
 * (F_k = V_k^{-T}, gamma = 1/sqrt(||a||^2 - ||z||^2)) with A^T a_{n*} read from the Gram matrix
 * (Sec. 2.2), and the projection y_hat = A_k F_k (A_k F_k)^T y, so each iteration updates the
 * residual by one orthonormal direction q_k = A_k F_k[:, k].
 *
 * Conventions shared by every entry point:
 *  - Layout. A is M x N column-major (lda = M): atom n is the M contiguous floats at A + n*M.
 *    Signals are rows: Y and R are B x M row-major. Per-signal outputs are B x S row-major.
 *  - Pointers. Every pointer is a DEVICE pointer on the handle's device unless the name ends in
 *    _host. Device pointers must be 16-byte aligned. The caller owns all of its buffers; the
 *    handle owns its workspaces and the prepared copies of the dictionary.
 *  - Streams. `stream` is a cudaStream_t (0 = the legacy default stream). Work is enqueued on it
 *    and the call returns without waiting, except the *_host entry point and omp_get_error.
 *  - Errors. Argument errors are returned synchronously and nothing is enqueued. A CUDA launch
 *    failure returns OMP_ERR_CUDA. Errors detected on the device (a bounded wait that ran out, a
 *    non-finite input) set a sticky error word that omp_get_error reads. No exception crosses
 *    this interface and there is no CPU fallback: a handle can only be created on an sm_103
 *    device.
 *  - Threads. One handle per host thread at a time; distinct handles are independent.
 *  - Ties. Wherever scores tie exactly, the smallest atom index wins.
 */
#ifndef OMP_GB300_H
#define OMP_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct omp_handle_s* omp_handle;

typedef enum {
  OMP_OK = 0,
  OMP_ERR_INVALID_ARGUMENT = 1,   /* bad pointer, size, alignment or option */
  OMP_ERR_UNSUPPORTED_DEVICE = 2, /* not a compute capability 10.3 device */
  OMP_ERR_OUT_OF_MEMORY = 3,      /* a workspace allocation failed */
  OMP_ERR_CUDA = 4,               /* a CUDA runtime call failed */
  OMP_ERR_DEVICE_TIMEOUT = 5,     /* a bounded device-side wait ran out (see omp_get_error) */
  OMP_ERR_NUMERICAL = 6           /* a signal had non-finite entries (it was returned empty) */
} omp_status;

typedef enum {
  OMP_PREC_FP32 = 0,     /* correlation A^T R in FP32 on the CUDA cores, fused top-1 */
  OMP_PREC_BF16 = 1,     /* BF16 tensor-core correlation, FP32 accumulate, top-8 rescored in FP32 */
  OMP_PREC_FP8_E4M3 = 2  /* E4M3 tensor-core correlation with per-atom and per-signal scales,
                            FP32 accumulate, top-8 rescored in FP32 */
} omp_precision;

/* Device error word bits (omp_get_error). */
#define OMP_DEVERR_WAIT_TIMEOUT 0x1  /* a bounded mbarrier / flag wait gave up */
#define OMP_DEVERR_NONFINITE 0x2     /* a signal contained NaN or Inf */
#define OMP_DEVERR_BAD_STATE 0x4     /* an internal index was out of range (skipped) */

typedef struct omp_desc {
  int64_t M;             /* signal length (rows of A), 1 <= M <= 8192 */
  int64_t N;             /* number of atoms (columns of A), 2 <= N <= 65536 */
  int64_t max_batch;     /* largest B any solve on this handle will pass, >= 1 */
  int32_t max_iters;     /* largest S any solve will pass, 1 <= max_iters <= min(M, N, 256) */
  int32_t precision;     /* omp_precision */
  int32_t rescore_topk;  /* quantised paths: candidates kept for the FP32 rescoring, 1..8 (0 means
                            8); of these only the ones within twice the score error bound
                            (omp_score_error_bound) of the quantised best are rescored, and none
                            when the best leads by more, which picks the same atom */
  int32_t eps_relative;  /* 1: stop when ||r_k|| <= eps * ||y||; 0: when ||r_k|| <= eps (Alg. 1) */
  int32_t use_graph;     /* capture each (B, S, eps) solve once as a CUDA graph and replay it:
                            1 with the S iterations unrolled (kernels of an iteration with no live
                            signal return at once), 2 with the iterations as a device-side while
                            loop that ends when no signal is live; 0: direct launches */
  int32_t device;        /* CUDA device ordinal the handle lives on */
  int32_t gather24;      /* 1: the update's gather of the support's atom rows (q = A_S F[:,k], the
                            residual update of Sec. 2.3) reads a 24-bit copy of A -- each element
                            rounded to nearest at a 15-bit mantissa (relative error <= 2^-16),
                            stored as 16 + 8 bit planes -- so 3 bytes per element move instead of
                            4 (N x Mp x 3 more bytes of HBM). The selection, the FP32 rescoring
                            and the factor are unchanged. 0 (default): FP32 rows. */
} omp_desc;

/* Fill `desc` with defaults for an M x N dictionary (precision BF16, rescore_topk 8,
 * eps_relative 1, use_graph 1, device 0, max_batch 4096, max_iters min(M, N, 64), gather24 0). */
void omp_desc_default(omp_desc* desc, int64_t M, int64_t N);

/* Create a handle: checks the device (sm_103 only), allocates every workspace for max_batch and
 * max_iters (including the N x N FP32 Gram matrix), and returns it in *out. No dictionary is
 * prepared yet. Returns OMP_ERR_UNSUPPORTED_DEVICE on any other device, OMP_ERR_OUT_OF_MEMORY if
 * an allocation fails (nothing is leaked). */
omp_status omp_create(const omp_desc* desc, omp_handle* out);

/* Release every resource of the handle (synchronises its device first). NULL is accepted. */
omp_status omp_destroy(omp_handle h);

/* Prepare the dictionary A (device, M x N column-major): column norms in FP64 (the 1/||a_n|| of
 * Alg. 1's score), a zero-padded FP32 copy, the BF16 or E4M3 copy with per-atom scales for the
 * tensor-core path, and the Gram matrix G = A^T A in FP32 (Sec. 2.2). Solves call this
 * implicitly when A differs from the last prepared pointer; the contents of A must not change
 * under the same pointer unless this function is called again. */
omp_status omp_prepare_dictionary(omp_handle h, const float* A, void* stream);

/* Solve B independent OMP problems with the shared dictionary A (Alg. 1).
 *   A            device, M x N column-major (prepared if it is not the cached pointer)
 *   Y            device, B x M row-major measurements
 *   B            1 <= B <= max_batch; S: 1 <= S <= max_iters; eps >= 0 (see eps_relative)
 *   X_out        device, B x S float: coefficients in selection order, in the scale of the
 *                caller's A (App. A), 0 past the signal's last iteration
 *   support_out  device, B x S int32: atom indices in selection order, -1 past the last one
 * A signal stops after S iterations, when ||r_k|| <= eps (relative or absolute), when the picked
 * atom is linearly dependent on its support (||a||^2 - ||z||^2 <= 1e-10 ||a||^2; the atom is not
 * added), or at once when y = 0 (empty support). */
omp_status omp_solve_batch(omp_handle h, const float* A, const float* Y, int64_t B, int32_t S,
                           float eps, float* X_out, int32_t* support_out, void* stream);

/* omp_solve_batch plus per-signal diagnostics (each pointer may be NULL):
 *   n_iter_out      device, B int32: iterations performed (= number of support entries)
 *   resid_norm_out  device, B float: final ||r|| as tracked by the update (FP32 residual)
 *   margin_out      device, B x S float: at each accepted step k the top-two score margin
 *                   (s1 - s2) / s1 of Alg. 1's selection (1 when every other score is 0), -1 past
 *                   the signal's last step. FP32 path: the correlation's best and runner-up over
 *                   all atoms. Quantised paths: the FP32 scores of the rescored candidates (the
 *                   rescore_topk best by quantised score); requesting margins makes such a solve
 *                   rescore every candidate, with no pruning -- the same picks, more time.
 *   stop_out        device, B int32: 0 = S reached, 1 = eps, 2 = dependent atom, 3 = y == 0 or
 *                   non-finite input
 * The margins are the selection statistic of Alg. 1 whose near-ties (margin <= 1e-3) are the
 * only places where two correct implementations may pick different atoms. */
omp_status omp_solve_batch_ex(omp_handle h, const float* A, const float* Y, int64_t B, int32_t S,
                              float eps, float* X_out, int32_t* support_out, int32_t* n_iter_out,
                              float* resid_norm_out, float* margin_out, int32_t* stop_out,
                              void* stream);

/* End-to-end variant with HOST buffers for the signals and results: copies Y_host (B x M) to
 * the device, solves, copies X_host (B x S) and support_host (B x S) back and waits for the
 * stream. Pinned host memory makes the copies asynchronous DMA; pageable memory works but is
 * slower. A stays a prepared device dictionary. */
omp_status omp_solve_batch_host(omp_handle h, const float* A, const float* Y_host, int64_t B,
                                int32_t S, float eps, float* X_host, int32_t* support_host,
                                void* stream);

/* One correlate-and-select step (Alg. 1's argmax) for B residuals R (device, B x M): the
 * handle's correlation path scores every atom, s_n = |<r, a_n>| / ||a_n|| (quantised paths:
 * |<q(r), q(a_n)>| times the atom's scale / ||a_n||, r's own scale omitted since it does not
 * change the order), and writes the `topk` best per signal in decreasing score, ties to the
 * lower index:  idx_out (device, B x topk int32) and score_out (device, B x topk float).
 * topk is 1 for OMP_PREC_FP32 and rescore_topk otherwise. No FP32 rescoring is applied here. */
omp_status omp_correlate_topk(omp_handle h, const float* A, const float* R, int64_t B,
                              int32_t topk, int32_t* idx_out, float* score_out, void* stream);

/* Per-launch timing. When enabled, the next solves record CUDA events around every correlation
 * and update launch (a separate captured graph with event-record nodes; results are the same
 * as without it). omp_profile_read synchronises `stream` and returns, for the most recent
 * solve, each iteration's correlation and update launch duration in milliseconds
 * (corr_ms, update_ms: S floats each, device-independent host arrays) and the live signal count
 * at the start of each iteration (live_out: S int32, may be NULL). S must equal that solve's S.
 * Returns OMP_ERR_INVALID_ARGUMENT if profiling was off for that solve. */
omp_status omp_profile_enable(omp_handle h, int32_t enable);
omp_status omp_profile_read(omp_handle h, int32_t S, float* corr_ms_host, float* update_ms_host,
                            int32_t* live_host, void* stream);

/* Largest B that omp_correlate_argmax_noalloc accepts. Its scratch is a fixed device array of
 * this many 8-byte keys (512 KiB), which every GPU that loads this library keeps until the
 * process exits. */
#define OMP_NOALLOC_MAX_SIGNALS 65536

/* Correlate-and-select that allocates nothing. The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- code running under a fixed memory
 * budget or inside a framework that owns every device allocation (cudaMalloc synchronises the
 * device and can fail at run time) -- and for callers that need one scoring pass without
 * creating a handle (omp_create allocates a whole solver's workspaces).
 *   A          device, M x N column-major dictionary (any column norms; they are computed here)
 *   R          device, B x M row-major residuals (or signals)
 *   idx_out    device, B int32: argmax_n |<r_b, a_n>| / ||a_n||, lowest index on exact ties;
 *              a zero-norm atom scores 0 (as on the handle path), so every signal gets a valid
 *              atom index (an all-zero dictionary gives atom 0 with score 0)
 *   score_out  device, B float: that score
 * The correlation runs in FP32 on the CUDA cores. Runs on the calling thread's current device;
 * every pointer must be on it and 4-byte aligned. B > OMP_NOALLOC_MAX_SIGNALS (or any other bad
 * argument) returns OMP_ERR_INVALID_ARGUMENT with nothing enqueued. The first call on a device
 * looks up the scratch array's device address (a one-time set-up), so make that first call
 * before any stream capture. All calls on a device share the one scratch array; each call
 * clears what it uses first, but calls that overlap on the GPU (unordered streams) race and
 * may return each other's results. */
omp_status omp_correlate_argmax_noalloc(const float* A, const float* R, int64_t M, int64_t N,
                                        int64_t B, int32_t* idx_out, float* score_out,
                                        void* stream);

/* omp_solve_batch plus a per-step trace: drop_out (device, B x S float) receives the normalised
 * residual drop b_k^2 / ||r_{k-1}||^2 of every accepted step k (b_k = q_k^T r_{k-1}, so the drop
 * is the fraction of the residual energy the step removed), 0 past the signal's last step. Used
 * to calibrate the learned proposal's residual-drop thresholds. */
omp_status omp_solve_batch_trace(omp_handle h, const float* A, const float* Y, int64_t B, int32_t S,
                                 float eps, float* X_out, int32_t* support_out, float* drop_out,
                                 void* stream);

/* Autotuner (the batching change's launch shapes, Sec. 3.5's batched solve): times solves of
 * (A, Y, B, S, eps) for each valid launch shape and keeps the fastest on the handle: first the
 * append/update kernel's warps per signal (1, 2, 4 or 8 for the padded signal length), then, on
 * the tensor-core paths, the correlation's CTAs per tile (1; or 2, a CTA pair running 256-row
 * MMAs across two SMs, each SM holding half of the atom tile), its pipeline depth (2, 3 or 4
 * operand stages of 48 KB; a pair 4 or 6 of 32 KB) and its persistent grid (every SM, or seven
 * eighths of them; a pair launch takes the largest even count whose pairs fit at once), then the update kernel's persistent form (a grid of the blocks that fit on
 * the GPU taking positions from a counter) against one block per signal. Each solve runs as a
 * solve does (a graph replay when the handle uses graphs); a challenger is timed alternately
 * with the incumbent, `repeats` solves each, and replaces it only when at least 3% faster, the
 * first valid shape of each choice being the incumbent. *choice_out (may be NULL) receives the
 * warps per signal; omp_tuning reads all five. If the environment variable OMP_AUTOTUNE_CACHE
 * names a file, a choice recorded there for the same GPU, M, N, precision, B and S is used
 * without timing ("key|warps,stages,ctas,persistent,cluster" lines; shorter lines keep the other
 * shapes), and new choices are appended to it. Synchronises `stream`. Captured graphs are
 * dropped when the choice changes. */
omp_status omp_autotune(omp_handle h, const float* A, const float* Y, int64_t B, int32_t S, float eps,
                        int32_t repeats, int32_t* choice_out, void* stream);

/* The handle's current launch shapes (each pointer may be NULL): update warps per signal, update
 * persistent form (0 or 1), correlation operand stages, persistent CTAs and CTAs per cluster (1,
 * or 2 for the 2-SM MMA pair; the last three 0 on the FP32 path). Host only. */
omp_status omp_tuning(omp_handle h, int32_t* update_warps, int32_t* update_persistent,
                      int32_t* corr_stages, int32_t* corr_ctas, int32_t* corr_cluster);

/* The descriptor the handle was created with (after defaults) and the device's SM count. */
omp_status omp_handle_info(omp_handle h, omp_desc* desc_out, int32_t* sm_count_out);

/* Passes of the device-side iteration loop in the last solve on `stream` (with use_graph = 2 the
 * captured graph runs the iterations as a conditional while node that stops after S passes or
 * as soon as no signal is live): the largest per-signal iteration count, at least 1; 0 when the
 * last solve ran its iterations unrolled (use_graph 0 or 1, or profiling on). Synchronises
 * `stream`. */
omp_status omp_loop_passes(omp_handle h, int32_t* passes_out, void* stream);

/* Gram-space solve (the v0 family of Sec. 2.3): the same problem as omp_solve_batch_ex, with
 * no correlation GEMM per step. One FP32 GEMM gives c = A^T y for the batch; then each signal's
 * block keeps c in shared memory and, per step, picks n* = argmax |c_n| / ||a_n|| (lowest index
 * on ties), appends the inverse-Cholesky column F_k from the Gram row of n* (gamma in FP64),
 * takes b_k = gamma c_{n*} and updates c <- c - b_k A^T q_k with A^T q_k = sum_j F[j,k] G[s_j,:].
 * ||r_k||^2 = ||r_{k-1}||^2 - b_k^2 drives the eps stop (only when eps > 0); at the end
 * x = F b and the residual y - A_S x is formed once for resid_norm_out. Any precision of the
 * handle; the handle's Gram matrix (N x N FP32) is used. Pays off when N is small next to M
 * (per step (k+1) N Gram reads instead of 2 M N FLOPs plus the update's atom-row gathers).
 * On first use it allocates an N x max_batch FP32 workspace (so the first call is not
 * graph-capturable). OMP_ERR_INVALID_ARGUMENT also when N floats + S (S + 1) / 2 floats of
 * per-signal shared memory exceed 227 KB. Outputs as omp_solve_batch_ex (optional ones may be
 * NULL); enqueued on `stream`. */
omp_status omp_solve_batch_gram(omp_handle h, const float* A, const float* Y, int64_t B, int32_t S,
                                float eps, float* X_out, int32_t* support_out, int32_t* n_iter_out,
                                float* resid_norm_out, int32_t* stop_out, void* stream);

/* Measurement helper (no part of the method): `blocks` blocks of 512 threads read the device
 * buffer `buf` (`bytes` a multiple of 16, 16-byte aligned) `reps` times with L2-only loads and
 * write one float per block to block_out[0..blocks). Timed around a buffer that fits in L2 it
 * gives the L2-to-SM read bandwidth the benchmark uses as the roofline of the update kernel when
 * the FP32 dictionary is L2-resident. Enqueued on `stream`; returns OMP_ERR_INVALID_ARGUMENT for
 * bad arguments, OMP_ERR_CUDA if the launch fails. */
omp_status omp_read_bandwidth_probe(const void* buf, int64_t bytes, int32_t reps, float* block_out,
                                    int32_t blocks, void* stream);

/* ------------------------------------------------------------------------------------------
 * Learned proposal. A small network maps the first correlation of a signal,
 *   x_n = <y, a_n> / (||a_n|| ||y||)                          (BF16 features)
 * to per-atom logits  o = W2 GELU(W1 x + b1) + b2 + beta |x|  (W1: hidden x N, W2: N x hidden,
 * BF16 GEMMs with FP32 accumulation, exact GELU, beta a learned scalar: the skip term carries each
 * atom's own correlation, which a hidden layer much narrower than N cannot pass through), and
 * proposes the `topk` atoms with the largest logits.
 * It is trained on the supports that plain OMP picks (omp_solve_batch on generated signals) by
 * mean binary cross-entropy with logits with a positive-class weight and AdamW on FP32 master
 * weights; forward and backward run in this library's own kernels. omp_solve_batch_learned then
 * runs the OMP iteration restricted to the proposed atoms (the projections of Sec. 2.3's D matrix
 * restricted to the candidates) and sends every signal whose step fails the residual-drop check
 * b_k^2 / ||r_{k-1}||^2 >= tau_k back to the full correlation from that step on.
 * The paper has no learned component; its results are checked against plain OMP's.
 * ------------------------------------------------------------------------------------------ */
typedef struct omp_proposal_s* omp_proposal;

typedef struct omp_proposal_desc {
  int32_t hidden;        /* hidden width, a multiple of 64 (1024) */
  int32_t topk;          /* candidates per signal, 1..256 (256) */
  int32_t max_batch;     /* largest inference batch, <= the handle's max_batch */
  int32_t train_batch;   /* largest training minibatch, a multiple of 64 (4096) */
  float lr, beta1, beta2, weight_decay, adam_eps;  /* AdamW (1e-3, 0.9, 0.999, 0, 1e-8) */
  float pos_weight;      /* BCE weight of the positive class, e.g. (N - S) / S */
} omp_proposal_desc;

void omp_proposal_desc_default(omp_proposal_desc* desc);

/* Create a proposal network for the handle's dictionary shape (N must be a multiple of 64).
 * Weights start at zero: set them with omp_proposal_set_weights. Thresholds start at 0 (every
 * restricted step accepted). */
omp_status omp_proposal_create(omp_handle h, const omp_proposal_desc* desc, omp_proposal* out);
omp_status omp_proposal_destroy(omp_proposal p);

/* FP32 parameters (device or host pointers): W1 hidden x N row-major, b1 hidden, W2 N x hidden
 * row-major, b2 N, beta 1. set_weights also resets the optimiser state; get_weights
 * synchronises. */
omp_status omp_proposal_set_weights(omp_proposal p, const float* W1, const float* b1, const float* W2,
                                    const float* b2, const float* beta, void* stream);
omp_status omp_proposal_get_weights(omp_proposal p, float* W1, float* b1, float* W2, float* b2,
                                    float* beta, void* stream);

/* One AdamW step on a minibatch: A (device, the handle's dictionary), Y (device, B x M signals),
 * labels (device, B x S int32 supports, -1 padded). B is a multiple of 64, <= train_batch.
 * loss_out (device float, may be NULL) receives the minibatch's mean weighted BCE. */
omp_status omp_proposal_train_step(omp_proposal p, const float* A, const float* Y, const int32_t* labels,
                                   int64_t B, int32_t S, float* loss_out, void* stream);

/* The same forward and backward pass without the update: gradients of the mean loss (device
 * pointers, shapes as the parameters; each may be NULL) and the loss. */
omp_status omp_proposal_gradients(omp_proposal p, const float* A, const float* Y, const int32_t* labels,
                                  int64_t B, int32_t S, float* dW1, float* db1, float* dW2, float* db2,
                                  float* dbeta, float* loss_out, void* stream);

/* Inference for B <= max_batch signals: cand_out (device, B x topk int32, ascending atom index)
 * and optionally the logits (device, B x N float). */
omp_status omp_proposal_infer(omp_proposal p, const float* A, const float* Y, int64_t B, int32_t* cand_out,
                              float* logits_out, void* stream);

/* Residual-drop thresholds tau[0..S) (host array). */
omp_status omp_proposal_set_thresholds(omp_proposal p, const float* tau_host, int32_t S);
omp_status omp_proposal_get_thresholds(omp_proposal p, float* tau_host, int32_t S);

/* Save the network (FP32 master weights W1, b1, W2, b2, beta) and its residual-drop thresholds
 * to a file, and load them back into a proposal of the same dictionary size N and hidden width.
 * The file holds a magic tag, the shape (N, hidden, topk, S), the parameters and thresholds as
 * little-endian FP32, and a 64-bit FNV-1a hash of all of it. Load refuses (with
 * OMP_ERR_INVALID_ARGUMENT, nothing changed) a file that is missing, truncated, altered or of
 * another shape; it resets the optimiser state as omp_proposal_set_weights does, and sets the
 * thresholds the file holds (any beyond them to 0). Both synchronise the device. The paper has no
 * learned component; these persist the proposal that restricts Alg. 1's selection. */
omp_status omp_proposal_save(omp_proposal p, const char* path);
omp_status omp_proposal_load(omp_proposal p, const char* path);

/* tau_k = the `quantile` (e.g. 0.001) of the positive entries of column k of drops (device,
 * B x S, from omp_solve_batch_trace on labelled training signals). */
omp_status omp_proposal_calibrate(omp_proposal p, const float* drops, int64_t B, int32_t S, float quantile,
                                  void* stream);

/* Per row of a rows x N matrix, the K largest entries' column indices (lowest index first among
 * equal values), in ascending index order (device pointers). */
omp_status omp_topk_rows(const float* logits, int64_t rows, int64_t N, int32_t K, int32_t* idx_out,
                         void* stream);

/* Candidates of the method without the network (for comparison): per signal the topk atoms of
 * |<y, a_n>| / ||a_n||, ascending atom index (device, B x topk int32). */
omp_status omp_proposal_baseline_candidates(omp_proposal p, const float* A, const float* Y, int64_t B,
                                            int32_t* cand_out, void* stream);

/* OMP restricted to given candidate atoms, with the residual-drop fallback to the full correlation:
 * cand (device, B x K int32, 1 <= K <= 256), tau (device, S float thresholds); other arguments
 * and results as omp_solve_batch_learned. */
omp_status omp_solve_batch_candidates(omp_handle h, const float* A, const float* Y, int64_t B, int32_t S,
                                      float eps, const int32_t* cand, int32_t K, const float* tau,
                                      float* X_out, int32_t* support_out, int32_t* n_iter_out,
                                      float* resid_norm_out, int32_t* fallback_out, void* stream);

/* Generated signals: Y_out (device, B x M) = sum_j coef[b, j] a_{sup[b, j]} + noise_b with A
 * (device, M x N column-major), sup (device, B x s int32, -1 skipped), coef (device, B x s),
 * noise (device, B x M, may be NULL). The input model of the problem statement. */
omp_status omp_synthesize_signals(const float* A, int64_t M, int64_t N, const int32_t* sup,
                                  const float* coef, const float* noise, int64_t B, int32_t s,
                                  float* Y_out, void* stream);

/* OMP with the learned proposal: same arguments and results as omp_solve_batch_ex, plus
 * fallback_out (device, B int32, may be NULL): the step at which the signal left the
 * candidate-restricted phase for the full correlation, or -1. */
omp_status omp_solve_batch_learned(omp_handle h, omp_proposal p, const float* A, const float* Y,
                                   int64_t B, int32_t S, float eps, float* X_out,
                                   int32_t* support_out, int32_t* n_iter_out,
                                   float* resid_norm_out, int32_t* fallback_out, void* stream);

/* Read and clear the device error word (OMP_DEVERR_* bits); synchronises the handle's work on
 * `stream` first. Returns OMP_ERR_DEVICE_TIMEOUT if the timeout bit was set, OMP_ERR_NUMERICAL
 * if only the non-finite bit was set, else OMP_OK. */
omp_status omp_get_error(omp_handle h, int32_t* flags, void* stream);

/* Human-readable name of a status code (static storage). */
const char* omp_status_string(omp_status s);

/* Host-only (no device work, callable without a GPU): the bound eps, per unit of ||a|| ||r||, on
 * |quantised score - FP32 score| that the quantised paths use to skip or trim the FP32 rescoring
 * and (BF16) to prune the correlation; Mp is the padded signal length. It covers rounding both
 * operands (BF16: unit roundoff 2^-8; E4M3 with a per-row scale amax/448: 2^-4 relative in the
 * normal range plus half the subnormal spacing of the scale), the tensor-core and FP32
 * accumulations over Mp terms, and 1% for the rounding of norms and scales. Returns 0 for
 * OMP_PREC_FP32, an unknown precision or Mp < 1 (no bound: the rescoring always runs).
 * The readings behind it: the rescoring of Sec. 3.7's reduced precision, our design. */
float omp_score_error_bound(int32_t precision, int64_t Mp);

#ifdef __cplusplus
}
#endif
#endif /* OMP_GB300_H */
