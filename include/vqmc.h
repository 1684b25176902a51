/*
 * vqmc.h -- C ABI of the GB300 (sm_103a) VQMC hot-path library.
 *
 * One variational iteration of "Overcoming barriers to scalability in
 * variational quantum Monte Carlo" (arXiv 2106.13308) on one GPU:
 *
 *   1. draw B exact samples s ~ pi_theta from a MADE autoregressive model
 *      (Sec. 2.3, Algorithm 1),
 *   2. evaluate log pi_theta(s)                               (Sec. 2.3),
 *   3. evaluate the diagonal Ising local energy
 *      E(s) = sum_{i<j} J_ij s_i s_j + sum_i h_i s_i          (Sec. 2.4),
 *   4. form the FP64 batch statistics and the score-function gradient
 *      g = sum_b (E_b - mean E)/B * grad log pi(s_b)          (Sec. 2.1),
 *   5. apply one Adam step (the paper's default optimiser, Sec. 5.1).
 *
 * Model.  n spins s_i in {-1,+1}, h hidden units, one masked hidden layer:
 *   a = (M1 . W1) s + b1,  g1 = act(a),  z = (M2 . W2) g1 + b2,
 *   pi_i(s_i = +1 | s_<i) = sigma(z_i),  log pi(s) = sum_i log sigma(s_i z_i).
 * Hidden unit k (0-based) has degree m(k) = 1 + floor(k (n-1) / h);
 * M1[k][j] = [m(k) >= j], M2[i][k] = [i > m(k)] with 1-based i, j.
 * act is the rectifier (the paper's choice) or the logistic sigmoid.
 *
 * Parameter layout (d = 2hn + h + n entries, Sec. 4), float32:
 *   theta = [ W1^T (n x h, row j = input j) | b1 (h) | W2 (n x h) | b2 (n) ].
 * Entries outside the masks are held at exactly zero by the library.
 *
 * Conventions for every call:
 *   - Pointers named d_* are device pointers owned by the caller; the library
 *     never frees them.  Pointers named h_* are host pointers.
 *   - Arrays are dense and row-major: spins int8 [B][n] with values +-1,
 *     uniforms float32 [B][n], energies int32 or float32 [B], log-probs
 *     float32 [B], gradients float32 [d] in the theta layout.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls only
 *     enqueue work and return; they never synchronise the device except
 *     where stated (vqmc_create, vqmc_set_params/get_params with host
 *     pointers, vqmc_check, vqmc_save/load).  Calls that share one context
 *     use its workspaces and must not run concurrently on different streams.
 *   - B must satisfy 0 <= B <= config.max_batch; B = 0 is a no-op.
 *   - Every call returns a vqmc_status; on failure vqmc_last_error() gives a
 *     thread-local message.  Device-side faults that a kernel can detect
 *     (a bounded wait that ran out, a non-finite energy) set bits in a sticky
 *     device error word that vqmc_check() reads and clears.
 */
#ifndef VQMC_H_
#define VQMC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vqmc_ctx vqmc_ctx;
typedef void* vqmc_stream; /* cudaStream_t */

typedef enum {
  VQMC_OK = 0,
  VQMC_ERR_INVALID_ARG = 1, /* bad pointer, size or enum value */
  VQMC_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  VQMC_ERR_OOM = 3,         /* device allocation failed */
  VQMC_ERR_NONFINITE = 4,   /* a NaN/Inf energy or statistic was produced */
  VQMC_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  VQMC_ERR_UNSUPPORTED = 6  /* size or option the library does not handle */
} vqmc_status;

enum { VQMC_ACT_RELU = 0, VQMC_ACT_SIGMOID = 1 };

/* Precision of the model inside the kernels.  FP32: FP32 weights and
 * activations, FP32 CUDA-core GEMMs.  BF16: the model has BF16 copies of W1,
 * W2 (rounded to nearest even from the FP32 master after every update) and
 * its hidden activations rounded to BF16 before the output layer, with FP32
 * accumulation everywhere; the log-prob/backward GEMMs run on the tcgen05
 * tensor cores with BF16 operands.  The master theta, Adam state and
 * gradients are FP32 in both modes; batch statistics are FP64. */
enum { VQMC_PREC_FP32 = 0, VQMC_PREC_BF16 = 1 };

/* Sampler implementation (vqmc_config.sampler).  All draw the same exact
 * samples of the model (Algorithm 1) from the same uniforms.
 *   AUTO: TENSOR_CORE where it applies, else CUDA_CORE.
 *   CUDA_CORE: one step at a time, FP32 FMAs on the CUDA cores; any model
 *     with h <= 5120 (BF16 weights) or h <= 2816 (FP32 weights).  Up to
 *     h = 2048 a CTA carries 16 samples; beyond, 4.
 *   CUDA_CORE_WIDE: the CUDA-core sampler with the layout it uses beyond
 *     h = 2048 (groups of four warps split the hidden units, 4 samples per
 *     CTA) at any h: four times the CTAs, fewer registers per sample; the
 *     batch autotuner chooses between the two per member.
 *   TENSOR_CORE: blocks of 64 or 128 steps whose bulk work (the logits from
 *     hidden units completed before the block, and the update of hidden
 *     units by the block's spins) runs as tcgen05 GEMMs, with a sequential
 *     solver for the units that complete inside the block.  BF16 precision
 *     only, h <= 2048, and at most 32 hidden units completing within 64
 *     consecutive steps (h up to about n/2); vqmc_create returns UNSUPPORTED
 *     when it is requested for any other model. */
enum { VQMC_SAMPLER_AUTO = 0, VQMC_SAMPLER_CUDA_CORE = 1, VQMC_SAMPLER_TENSOR_CORE = 2, VQMC_SAMPLER_CUDA_CORE_WIDE = 3 };

/* Hamiltonian storage. */
enum {
  VQMC_HAM_SPARSE_I32 = 0, /* CSR strict upper triangle, int32 weights; E is int32, exact */
  VQMC_HAM_SPARSE_F32 = 1, /* CSR strict upper triangle, float32 weights; E is float32 */
  VQMC_HAM_DENSE_F32 = 2   /* dense symmetric float32 J (zero diagonal); E is float32 */
};

/* Device error word bits (vqmc_check). */
enum {
  VQMC_DEVERR_TIMEOUT = 1u,   /* a bounded mbarrier/flag wait gave up */
  VQMC_DEVERR_NONFINITE = 2u  /* a non-finite energy or statistic */
};

typedef struct {
  int32_t n;          /* number of spins, >= 1 */
  int32_t h;          /* hidden units, >= 1 */
  int32_t max_batch;  /* largest B any call will pass, >= 1 */
  int32_t act;        /* VQMC_ACT_* */
  int32_t precision;  /* VQMC_PREC_* */
  float lr;           /* Adam learning rate (paper default 1e-2) */
  float beta1;        /* Adam beta1 (0.9) */
  float beta2;        /* Adam beta2 (0.999) */
  float eps;          /* Adam epsilon (1e-8) */
  uint32_t sampler;   /* VQMC_SAMPLER_* (0 = AUTO) */
  uint64_t seed;      /* Philox4x32-10 key for the internal uniforms */
} vqmc_config;

/* Problem instance, host memory, copied to the device by vqmc_create.
 * Sparse kinds: row_ptr int32 [n+1], col int32 [nnz] with col > row (the
 * strict upper triangle, each undirected edge once), w [nnz] int32 or float32
 * per kind.  Dense kind: J float32 [n][n] symmetric with zero diagonal.
 * field: h_i, [n] of the weight type (int32 for SPARSE_I32, float32
 * otherwise), or NULL for h = 0.
 * alpha: the transverse field of the transverse-field Ising model,
 * Eq. (hamiltonian): H = -sum_i (alpha_i X_i + beta_i Z_i)
 * - sum_{i<j} beta_ij Z_i Z_j, with the diagonal part given as above
 * (J_ij = -beta_ij, h_i = -beta_i); float32 [n], every alpha_i >= 0 and
 * finite (the paper's sign condition, Sec. 2.4), or NULL for none.  Only with
 * the float32 kinds (SPARSE_F32, DENSE_F32); INVALID_ARG otherwise. */
typedef struct {
  int32_t kind; /* VQMC_HAM_* */
  int32_t n;
  int32_t nnz;
  int32_t reserved;
  const int32_t* row_ptr;
  const int32_t* col;
  const void* w;
  const void* field;
  const float* J;
  const float* alpha;
} vqmc_instance;

/* Result of one vqmc_step, FP64 statistics of the batch's local energies
 * (Eq. (e:vmc) and Eq. (eq:stochastic_variance) estimated on the batch). */
typedef struct {
  double mean;          /* L = sum_b E_b / B */
  double var;           /* sum_b (E_b - L)^2 / B */
  double min;           /* lowest energy in the batch */
  double max;           /* highest energy in the batch */
  uint64_t iteration;   /* Philox iteration counter used for this step */
  uint32_t error_flags; /* snapshot of the device error word (VQMC_DEVERR_*) */
  uint32_t reserved;
} vqmc_step_stats;

/* Creates a context: validates cfg/inst, allocates the FP32 master theta
 * (zero), Adam state, BF16/FP32 weight copies and every workspace for up to
 * cfg->max_batch samples, and copies the instance to the device.  Synchronous.
 * Errors: INVALID_ARG (n, h, max_batch < 1, inst->n != cfg->n, bad kind or
 * NULL arrays), OOM, CUDA, UNSUPPORTED (sizes the library cannot tile). */
vqmc_status vqmc_create(const vqmc_config* cfg, const vqmc_instance* inst, vqmc_ctx** out);

/* Frees everything the context owns.  NULL is accepted. */
void vqmc_destroy(vqmc_ctx* ctx);

/* d = 2hn + h + n. */
int64_t vqmc_num_params(const vqmc_ctx* ctx);

/* Replaces theta (d floats, host or device per theta_on_device), zeroes the
 * entries outside the MADE masks, resets the Adam moments and step count and
 * refreshes the kernels' weight copies.  Synchronous when theta is on the
 * host.  Errors: INVALID_ARG, CUDA. */
vqmc_status vqmc_set_params(vqmc_ctx* ctx, const float* theta, int theta_on_device, vqmc_stream stream);

/* Copies the FP32 master theta out (d floats). */
vqmc_status vqmc_get_params(vqmc_ctx* ctx, float* theta, int theta_on_device, vqmc_stream stream);

/* Device pointer to the context's FP32 master theta (d floats, owned by the
 * context).  After writing to it, call vqmc_params_updated. */
float* vqmc_params_device(vqmc_ctx* ctx);

/* Re-applies the masks and refreshes the weight copies after theta was
 * written through vqmc_params_device (does not touch the Adam state). */
vqmc_status vqmc_params_updated(vqmc_ctx* ctx, vqmc_stream stream);

/* Writes the uniforms the sampler draws internally for Philox iteration
 * `iteration`: d_u[b][i] = word (i mod 4) of
 * Philox4x32-10(counter = (i/4, b, iteration_lo, iteration_hi), key = seed)
 * mapped to [0,1) as (x >> 8) * 2^-24.  d_u: float32 [B][n]. */
vqmc_status vqmc_uniforms(vqmc_ctx* ctx, int32_t B, uint64_t iteration, float* d_u, vqmc_stream stream);

/* Algorithm 1 (Sec. 2.3): draws B exact samples.  Spin i of sample b is +1
 * iff u_{b,i} < sigma(z_i(s_<i)), else -1, with u = d_u[b][i] when d_u is not
 * NULL, else the internal Philox uniforms of `iteration` (see vqmc_uniforms).
 * Writes d_s int8 [B][n] and, if d_logp is not NULL, log pi(s_b) float32 [B]
 * accumulated in FP32 while sampling.  The conditionals are computed in FP32
 * from the FP32 or BF16 weight copies (per precision). */
vqmc_status vqmc_sample(vqmc_ctx* ctx, int32_t B, const float* d_u, uint64_t iteration, int8_t* d_s,
                        float* d_logp, vqmc_stream stream);

/* Local energy l(s) = sum_y H_sy psi(y) / psi(s), psi = sqrt(pi) (Sec. 2.1),
 * of B configurations d_s int8 [B][n].  The diagonal part (Sec. 2.4):
 * E_b = sum_{i<j} J_ij s_i s_j + sum_i h_i s_i.  d_e is int32 [B] (exact)
 * for VQMC_HAM_SPARSE_I32 and float32 [B] otherwise.  The dense kind runs
 * S.J on the tensor cores in BF16 precision, with J split into a BF16 high
 * part and a BF16 remainder (16 significant bits of every coupling, FP32
 * accumulation: |E - E_exact| <= n^2 2^-16 max|J_ij|), and on the CUDA cores
 * in FP32 otherwise (|E - E_exact| <= n^2 2^-23 max|J_ij|).  With a transverse field
 * alpha, also -sum_i alpha_i sqrt(pi(s^(i)) / pi(s)) (s^(i): spin i flipped,
 * Eq. (e:tim)): the n flipped states of every sample and the sample itself
 * go through the model's log-prob GEMMs in chunks of rows, so this costs
 * about n + 1 log-prob evaluations per sample. */
vqmc_status vqmc_local_energy(vqmc_ctx* ctx, int32_t B, const int8_t* d_s, void* d_e, vqmc_stream stream);

/* log pi(s_b) (Sec. 2.3) of B configurations by the full masked forward
 * pass (two masked GEMMs).  d_logp float32 [B]. */
vqmc_status vqmc_logprob(vqmc_ctx* ctx, int32_t B, const int8_t* d_s, float* d_logp, vqmc_stream stream);

/* Adjoint of vqmc_logprob: d_grad[d] = sum_b d_gout[b] * grad_theta log pi(s_b)
 * (overwrites d_grad).  Hidden activations are recomputed, not taken from a
 * previous forward.  Entries outside the masks are written as 0. */
vqmc_status vqmc_logprob_backward(vqmc_ctx* ctx, int32_t B, const int8_t* d_s, const float* d_gout,
                                  float* d_grad, vqmc_stream stream);

/* FP64 batch statistics of energies d_e (int32 or float32 per instance kind):
 * d_stats double [4] = {mean, var, min, max} (var with 1/B), and, if d_coef
 * is not NULL, the score-function coefficients c_b = (E_b - mean)/B as
 * float32 [B].  For int32 energies the sums of E and E^2 are exact integers
 * (64 and 128 bits) and mean and var are each rounded once to FP64; c_b is
 * (B E_b - sum E) / B^2 rounded to float32 (exactly so when B is a power of
 * two).  Float energies accumulate in FP64 in a fixed order.  A non-finite
 * value sets VQMC_DEVERR_NONFINITE. */
vqmc_status vqmc_energy_stats(vqmc_ctx* ctx, int32_t B, const void* d_e, double* d_stats, float* d_coef,
                              vqmc_stream stream);

/* Score-function gradient of one batch (Sec. 2.1):
 * d_grad = sum_b (E_b - mean)/B * grad log pi(s_b); d_stats as above
 * (may be NULL). */
vqmc_status vqmc_grad(vqmc_ctx* ctx, int32_t B, const int8_t* d_s, const void* d_e, float* d_grad,
                      double* d_stats, vqmc_stream stream);

/* One Adam step on the master theta with gradient d_grad[d], then refreshes
 * the weight copies.  Increments the context's Adam step count. */
vqmc_status vqmc_adam(vqmc_ctx* ctx, const float* d_grad, vqmc_stream stream);

/* One full VQMC iteration: sample B configurations with the internal
 * uniforms of the context's iteration counter, local energies, FP64
 * statistics, score-function gradient and one Adam step; then increments the
 * iteration counter.  The result equals vqmc_sample + vqmc_local_energy +
 * vqmc_grad + vqmc_adam; for BF16 the weight-gradient GEMMs apply the Adam
 * step in their epilogue, so the weight gradient is never stored.  If h_out is not NULL it receives the step's statistics
 * by an asynchronous device-to-host copy on `stream` (synchronise before
 * reading; use pinned memory for a truly asynchronous copy). */
vqmc_status vqmc_step(vqmc_ctx* ctx, int32_t B, vqmc_stream stream, vqmc_step_stats* h_out);

/* Stochastic reconfiguration (natural gradient, Sec. 2.1; the paper's
 * "SGD+SR" optimiser of Sec. 5.1 with lambda = 1e-3 and lr = 0.1).  With
 * O_b = grad_theta log pi(s_b) the batch estimates of the paper's gradient
 * and Fisher forms are g = (1/B) sum_b (E_b - mean E) O_b and
 * I = (1/B) sum_b O_b O_b^T; the direction delta solves
 * (I + lambda 1) delta = g.  The d x d matrix is never formed: the library
 * builds the B x B Gram matrix O O^T from the MADE structure, factors
 * O O^T / B + lambda by Cholesky (FP32) and returns delta = O^T x.
 *
 * These calls need an FP32 context (VQMC_PREC_FP32): with BF16 the
 * per-sample operands are rounded to bfloat16, which would perturb the Gram
 * matrix by 2^-9 relative, amplified by its condition number.  They return
 * UNSUPPORTED for a BF16 context and for B > 16384.  The first SR call on a
 * context allocates its workspace of about 4 max_batch^2 bytes (padded to a
 * multiple of 64) with cudaMalloc and synchronises the device; later calls
 * allocate nothing.  A non-positive Cholesky pivot (only possible through
 * rounding or non-finite inputs) sets VQMC_DEVERR_NONFINITE. */

/* d_gram float32 [B][B] (row-major, both triangles) = O O^T of the B
 * configurations d_s int8 [B][n]. */
vqmc_status vqmc_sr_gram(vqmc_ctx* ctx, int32_t B, const int8_t* d_s, float* d_gram, vqmc_stream stream);

/* d_delta float32 [d] (theta layout) = the SR direction of the batch
 * (d_s int8 [B][n], energies d_e int32/float32 [B] per instance kind) with
 * regulariser lambda > 0 (INVALID_ARG otherwise); d_stats (NULL allowed):
 * the FP64 energy statistics as in vqmc_energy_stats.  B = 0 writes zeros. */
vqmc_status vqmc_sr_direction(vqmc_ctx* ctx, int32_t B, const int8_t* d_s, const void* d_e, float lambda,
                              float* d_delta, double* d_stats, vqmc_stream stream);

/* One SGD+SR iteration: B samples with the internal uniforms of the
 * iteration counter, local energies, FP64 statistics, the SR direction and
 * theta <- theta - lr delta (the Adam state is untouched); then increments
 * the iteration counter.  h_out as in vqmc_step.  While timing is enabled
 * (vqmc_timing_enable) it records the parts of vqmc_step, with GRAD = the SR
 * direction (per-sample operands, Gram matrix, Cholesky, solves, adjoint)
 * and ADAM = the SGD step with the weight-copy refresh. */
vqmc_status vqmc_sr_step(vqmc_ctx* ctx, int32_t B, float lr, float lambda, vqmc_stream stream,
                         vqmc_step_stats* h_out);

/* Captured iterations.  The kernels of an iteration read the Philox
 * iteration counter and the Adam step factors from device memory that the
 * iteration itself advances, so a CUDA graph of `steps` consecutive
 * iterations can be replayed for the iterations that follow, each replay
 * giving exactly what the same number of vqmc_step (optimizer
 * VQMC_OPT_ADAM) or vqmc_sr_step (VQMC_OPT_SR, with sr_lr and sr_lambda)
 * calls would.  Capturing runs nothing and leaves the counters unchanged; it
 * replaces any earlier graph of the context.  `stream` must not be the
 * legacy default stream (NULL).  SR graphs need an FP32 context; their
 * workspace is allocated before the capture.  Errors: those of the captured
 * call, INVALID_ARG, CUDA (capture or instantiation failed). */
enum { VQMC_OPT_ADAM = 0, VQMC_OPT_SR = 1 };
vqmc_status vqmc_graph_capture(vqmc_ctx* ctx, int32_t B, int32_t steps, int32_t optimizer, float sr_lr,
                               float sr_lambda, vqmc_stream stream);

/* Launches the captured iterations on `stream` (one graph launch) and
 * advances the context's counters by their number; h_out (NULL allowed)
 * receives the last iteration's statistics as in vqmc_step.  INVALID_ARG if
 * nothing was captured. */
vqmc_status vqmc_graph_launch(vqmc_ctx* ctx, vqmc_stream stream, vqmc_step_stats* h_out);

/* Sampling parallelism over GPUs (Sec. 4, "Sampling Parallelization"; the
 * multi-GPU runs of Sec. 5.4 and Tables 6-7).  The samples of an iteration
 * are independent draws from the same model, so L GPUs, each with its own
 * context holding the same parameters, draw disjoint shards of one batch of
 * B_tot samples and exchange one set of sums per iteration.  For any
 * constant c (the `shift`, the same on every rank) and g_b = grad log pi(s_b),
 *     sum_b (E_b - Ebar) g_b = sum_b (E_b - c) g_b - (Ebar - c) sum_b g_b,
 * so each rank writes S1 = sum_{b in shard} (E_b - c) g_b and
 * S0 = sum_{b in shard} g_b (float32, 2d values) and the FP64 scalars
 * {sum (E_b - c), sum (E_b - c)^2, B}; one element-wise sum of these over the
 * ranks (an all-reduce, done by the caller: NCCL, MPI or host code) lets
 * every rank form the exact global-baseline gradient
 * (1/B_tot) sum_b (E_b - Ebar) g_b of the whole batch (Sec. 2.1) and apply
 * the same Adam step, so the replicas stay identical.  A shift near Ebar
 * (for example the previous iteration's global mean) keeps the FP32 sums
 * well conditioned; 0 gives the plain sums. */

/* Index of this context's sample 0 in the Philox counter (default 0): the
 * internal uniforms of sample b are those of global sample b0 + b, so ranks
 * with offsets 0, B, 2B, ... draw disjoint streams whose union is the batch
 * one context with max_batch = B_tot would draw.  b0 + B must stay below
 * 2^32.  Affects vqmc_sample with d_u = NULL, vqmc_uniforms, vqmc_step and
 * vqmc_shard_sums; takes effect for calls enqueued after it. */
vqmc_status vqmc_set_sample_offset(vqmc_ctx* ctx, uint32_t b0);

/* This shard's sums.  d_s = NULL: draws B samples with the internal uniforms
 * of the context's iteration counter (and sample offset) and their local
 * energies into the context's batch buffers (vqmc_last_batch), as vqmc_step
 * does; otherwise uses d_s int8 [B][n] and d_e (int32/float32 [B] per
 * instance kind).  Writes d_sums float32 [2d] = [S1 | S0] (theta layout
 * each, zero outside the masks) and d_scalars double [3] =
 * {sum (E_b - shift), sum (E_b - shift)^2, B}.  Costs one hidden-activation
 * GEMM and two adjoint passes.  B = 0 writes zeros.  Errors: INVALID_ARG
 * (null outputs, d_s without d_e, non-finite shift), those of the kernels;
 * a non-finite energy sets VQMC_DEVERR_NONFINITE. */
vqmc_status vqmc_shard_sums(vqmc_ctx* ctx, int32_t B, const int8_t* d_s, const void* d_e, double shift, float* d_sums,
                            double* d_scalars, vqmc_stream stream);

/* The update from the sums of all ranks (d_sums [2d], d_scalars [3], summed
 * element-wise over the ranks; shift as given to vqmc_shard_sums): forms the
 * gradient (S1 - (Ebar - shift) S0) / B_tot with Ebar - shift =
 * sum (E_b - shift) / B_tot, writes it to d_grad [d] (NULL: the context's own
 * buffer), writes d_stats double [2] = {Ebar, variance with 1/B_tot} (NULL
 * allowed), applies one Adam step and advances the iteration counter.  Every
 * rank that passes the same sums applies the same update.  A total count
 * below 1 or non-finite scalars give a zero gradient and set
 * VQMC_DEVERR_NONFINITE. */
vqmc_status vqmc_shard_apply(vqmc_ctx* ctx, const float* d_sums, const double* d_scalars, double shift, float* d_grad,
                             double* d_stats, vqmc_stream stream);

/* A batch of independent problems (each member an ordinary context with its
 * own model, instance, optimiser and workspaces), stepped together: many
 * Max-Cut instances of different sizes trained at once, so that small
 * instances fill the GPU together.  The paper trains one instance at a time
 * (Sec. 5); this is the same iteration applied to each member. */
typedef struct vqmc_batch vqmc_batch;

/* Creates `count` >= 1 members, member i from cfgs[i] and insts[i] exactly as
 * vqmc_create would (same validation and errors; on any error nothing is
 * kept and *out is untouched), plus up to 8 internal streams.  Synchronous. */
vqmc_status vqmc_batch_create(const vqmc_config* cfgs, const vqmc_instance* insts, int32_t count,
                              vqmc_batch** out);

/* Frees the batch and every member.  NULL is accepted. */
void vqmc_batch_destroy(vqmc_batch* batch);

/* Number of members (0 for NULL). */
int32_t vqmc_batch_count(const vqmc_batch* batch);

/* Member i, borrowed: usable with every vqmc_* call, valid until
 * vqmc_batch_destroy, never to be passed to vqmc_destroy.  NULL if i is out
 * of range. */
vqmc_ctx* vqmc_batch_member(vqmc_batch* batch, int32_t i);

/* One vqmc_step of every member, member i with B[i] samples (B: `count`
 * host int32), spread over the internal streams after the work already
 * queued on `stream`; `stream` then waits for all of them (asynchronous, as
 * vqmc_step).  h_out: NULL, or `count` records receiving each member's
 * statistics.  Errors: those of vqmc_step, for the first member that fails
 * (the members before it have stepped), or INVALID_ARG for a NULL argument. */
vqmc_status vqmc_batch_step(vqmc_batch* batch, const int32_t* B, vqmc_stream stream, vqmc_step_stats* h_out);

/* Captures `steps` consecutive vqmc_batch_step calls (member i with B[i]
 * samples, the batch's current schedule) as one CUDA graph owned by the
 * batch, replacing any earlier one; as vqmc_graph_capture for one context
 * (runs nothing, counters unchanged, a non-default stream). */
vqmc_status vqmc_batch_graph_capture(vqmc_batch* batch, const int32_t* B, int32_t steps, vqmc_stream stream);

/* One graph launch of the captured batched iterations; every member's
 * counters advance by their number.  h_out: NULL or `count` records. */
vqmc_status vqmc_batch_graph_launch(vqmc_batch* batch, vqmc_stream stream, vqmc_step_stats* h_out);

/* Autotuner of the batch's schedule.  First it measures one iteration of
 * each member alone; a member on the CUDA-core sampler with at most 2048
 * hidden units is timed in both of its layouts (16 samples per CTA, and the
 * wide one of VQMC_SAMPLER_CUDA_CORE_WIDE) and keeps the faster.  Then it
 * times one captured batched iteration (graph replays) under each candidate
 * schedule -- 1, 2, 4, ... up to the batch's internal streams, with members
 * assigned round-robin in index order or longest first onto the
 * least-loaded stream -- and keeps the fastest schedule, with its captured
 * graph (one iteration, for vqmc_batch_graph_launch).  The iterations it
 * times are ordinary iterations of every member: each member advances by
 * 4 + 4 x (number of candidate schedules) iterations.  streams_out and ms_out (NULL allowed) receive the
 * chosen number of streams and its device time per batched iteration.
 * `stream`: not the legacy default stream. */
vqmc_status vqmc_batch_autotune(vqmc_batch* batch, const int32_t* B, vqmc_stream stream, int32_t* streams_out,
                                double* ms_out);

/* The batch's current schedule: the internal streams in use (streams_used),
 * and per member (arrays of `count`, each NULL allowed) its stream, its
 * sampler (VQMC_SAMPLER_TENSOR_CORE, _CUDA_CORE or _CUDA_CORE_WIDE) and the
 * device time of one of its iterations alone measured by the last
 * vqmc_batch_autotune (0 before any).  The longest of those times is a lower
 * bound on a batched iteration (each member's kernels run in order), and
 * their sum is the time of the members stepped one after another. */
vqmc_status vqmc_batch_schedule(const vqmc_batch* batch, int32_t* streams_used, int32_t* member_stream,
                                int32_t* member_sampler, double* member_ms);

/* Device pointers to the last vqmc_step's samples (int8 [B][n]) and energies
 * (int32/float32 [B]); owned by the context, overwritten by the next step. */
vqmc_status vqmc_last_batch(vqmc_ctx* ctx, const int8_t** d_s, const void** d_e);

/* Current Philox iteration counter and Adam step count. */
uint64_t vqmc_iteration(const vqmc_ctx* ctx);

/* Synchronises the device, reads and clears the sticky device error word.
 * Returns TIMEOUT or NONFINITE if the corresponding bit was set. */
vqmc_status vqmc_check(vqmc_ctx* ctx, uint32_t* flags_out);

/* Checkpoint: writes/reads theta, Adam moments, Adam step count, the Philox
 * seed and iteration counter and a hash of (n, h, act, instance) to/from a
 * binary file.  vqmc_load fails with INVALID_ARG on a shape/instance
 * mismatch.  Synchronous. */
vqmc_status vqmc_save(vqmc_ctx* ctx, const char* path);
vqmc_status vqmc_load(vqmc_ctx* ctx, const char* path);

/* Per-part timing of vqmc_step.  While enabled, every vqmc_step records CUDA
 * events on its stream between its parts (no synchronisation), for up to
 * 4096 steps.  vqmc_timing_read synchronises, and returns the summed device
 * time of each part over the recorded steps in ms_out[VQMC_NUM_PARTS], the
 * number of recorded steps and the number of kernels those steps launched.
 * Enabling resets the record. */
enum {
  VQMC_PART_SAMPLE = 0,   /* the sampler kernel (uniforms generated in-kernel) */
  VQMC_PART_ENERGY = 1,   /* local energies (and, after the CUDA-core sampler, the spins' GEMM layouts);
                             for a sparse instance without a transverse field the energies and the
                             statistics run beside the hidden-activation GEMM, and this part is that
                             GEMM's time */
  VQMC_PART_STATS = 2,    /* FP64 statistics and coefficients (in the overlapped case: the wait for
                             them after the hidden-activation GEMM) */
  VQMC_PART_GRAD = 3,     /* log-prob forward + adjoint GEMMs and reductions; for BF16 also the
                             Adam step on the weights, which the weight-gradient GEMMs apply */
  VQMC_PART_ADAM = 4,     /* Adam step (BF16: biases only) and weight-copy refresh */
  VQMC_NUM_PARTS = 5
};
vqmc_status vqmc_timing_enable(vqmc_ctx* ctx, int enable);
vqmc_status vqmc_timing_read(vqmc_ctx* ctx, double* ms_out, int64_t* steps_out, int64_t* launches_out);

/* Allocation-free variant of vqmc_logprob.  The paper has no counterpart to
 * this entry point: it exists for callers that cannot allocate device memory
 * at call time -- code whose device memory is owned by another framework's
 * pool, serving paths with a fixed memory budget, or code that must not let
 * a cudaMalloc/cudaFree synchronise the device.  It computes the same log pi
 * as vqmc_logprob (same kernels, same arithmetic) but takes its scratch (the
 * spin operand, the hidden activations and the row partial sums) from one
 * static device array of 64 MiB owned by the library instead of the context.
 * It calls no allocating routine.  Limits and caveats:
 *   - a call needs r(B np e) + r(B hp e) + r(ceil(n / 128) pad64(B) 4) bytes
 *     of scratch, with np = pad64(n), hp = pad64(h), e = 2 bytes per element
 *     in BF16 and 4 in FP32, and r() rounding up to a multiple of 256; a call
 *     that would need more than 64 MiB (67,108,864 bytes) returns
 *     VQMC_ERR_UNSUPPORTED with the byte count.  At n = 10,000, h = 2,000
 *     that allows B <= 2,738 in BF16 and B <= 1,377 in FP32;
 *   - every GPU that loads the library's module holds the 64 MiB until the
 *     process exits;
 *   - the first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture;
 *   - all calls share the array, so calls that overlap on the GPU (on other
 *     streams or from other threads) race and must be serialised by the
 *     caller.
 * Arguments and errors as vqmc_logprob. */
vqmc_status vqmc_logprob_noalloc(vqmc_ctx* ctx, int32_t B, const int8_t* d_s, float* d_logp, vqmc_stream stream);

/* Thread-local description of the last error. */
const char* vqmc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* VQMC_H_ */
