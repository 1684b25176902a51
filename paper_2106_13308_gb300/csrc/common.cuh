// Internal declarations shared by the CUDA translation units of libvqmc.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "vqmc.h"

namespace vqmc {

using bf16 = __nv_bfloat16;

// Leading dimensions of every kernel-side matrix are padded to this many
// elements, so rows start on 128-byte boundaries (bulk/TMA copies need 16).
constexpr int kPad = 64;
inline int pad_up(int x, int p = kPad) { return (x + p - 1) / p * p; }

// MADE degree of hidden unit k (0-based): m(k) = 1 + floor(k (n-1) / h).
// 32-bit arithmetic when k (n-1) fits (every size this library accepts).
__host__ __device__ inline int degree(int k, int n, int h) {
  const long long p = (long long)k * (long long)(n - 1);
  if (p < (1ll << 32)) return 1 + (int)((unsigned)p / (unsigned)h);
  return 1 + (int)(p / (long long)h);
}

// Number of hidden units whose degree is <= x, i.e. #{k : k (n-1) < x h}.
__host__ __device__ inline int count_deg_le(int x, int n, int h) {
  if (x < 1) return 0;
  if (n <= 1) return h;
  const long long p = (long long)x * h + (n - 2);
  const long long c = p < (1ll << 32) ? (long long)((unsigned)p / (unsigned)(n - 1)) : p / (n - 1);
  return c > h ? h : (int)c;
}

// The sampler streams SPS consecutive rows per copy; its weight copies have
// this many rows (wt_s row j = input j with row 0 zero, v_s row i = output i+1).
constexpr int kSamplerRowsPad = 8;
inline int sampler_rows(int n) { return (n + 1 + kSamplerRowsPad - 1) / kSamplerRowsPad * kSamplerRowsPad; }

// Device error word bits mirror VQMC_DEVERR_*.
constexpr uint32_t kErrTimeout = VQMC_DEVERR_TIMEOUT;
constexpr uint32_t kErrNonfinite = VQMC_DEVERR_NONFINITE;

// Bound on every device-side spin wait (try_wait iterations; each try_wait
// may itself suspend the thread for a hardware-chosen interval).
constexpr long long kSpinLimit = 1ll << 26;

// Counters of the iteration that the kernels read on the device, so that a
// captured CUDA graph replays consecutive iterations: the Philox iteration
// of the next step, the Adam step count and the bias corrections
// 1 / (1 - beta^t) of the current Adam step.  The context keeps host mirrors
// (iter, adam_t) that every enqueue advances in step.
struct DevState {
  unsigned long long iter;
  long long adam_t;
  float ibc1, ibc2;
};

// beta^t for integer t >= 0 by repeated squaring (a fixed function of t, so a
// run resumed from a checkpoint reproduces it exactly).
__device__ __forceinline__ double pow_int(double b, long long t) {
  double r = 1.0;
  while (t > 0) {
    if (t & 1) r *= b;
    b *= b;
    t >>= 1;
  }
  return r;
}

// The bias corrections 1 / (1 - beta^t) of Adam step t = s->adam_t (1 for t = 0).
__device__ __forceinline__ void adam_factors(DevState* s, float beta1, float beta2) {
  const long long t = s->adam_t;
  s->ibc1 = t < 1 ? 1.0f : (float)(1.0 / (1.0 - pow_int((double)beta1, t)));
  s->ibc2 = t < 1 ? 1.0f : (float)(1.0 / (1.0 - pow_int((double)beta2, t)));
}

}  // namespace vqmc

// The context behind the opaque handle of vqmc.h.
struct vqmc_ctx {
  vqmc_config cfg;
  int n, h, Bmax;
  int np, hp, Bp;  // padded n, h, batch
  int act, prec;   // VQMC_ACT_*, VQMC_PREC_*
  int ham;         // VQMC_HAM_*
  int sampler;     // VQMC_SAMPLER_CUDA_CORE or _TENSOR_CORE (resolved at create)
  int sampler_wide = 0;  // CUDA-core sampler in its four-warp-group layout
  int nnz;
  int64_t d;
  uint64_t inst_hash = 0;
  int device;
  int num_sms;
  // index of this context's sample 0 in the Philox counter: 0, or the first
  // global sample of the shard this context draws (vqmc_set_sample_offset)
  uint32_t sample_offset = 0;
  float* ones = nullptr;  // [Bmax] unit coefficients (the shard sums' sum of scores)

  // FP32 master parameters, optimiser state, gradient (d floats each)
  float* theta = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  float* grad = nullptr;
  int64_t adam_t = 0;
  uint64_t iter = 0;
  vqmc::DevState* dstate = nullptr;  // device copy of the counters
  // captured iterations (vqmc_graph_capture): the instantiated graph, its
  // number of iterations and whether they are Adam steps
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  bool graph_adam = false;
  // side stream of vqmc_step: the sparse energy and the statistics run on it
  // beside the hidden-activation GEMM (fork/join events)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  // Kernel-side weight copies, element type float (FP32) or bf16 (BF16):
  //   wt_s [sampler_rows(n)][hp]  row j = column j of W1 (input j, 1-based),
  //                               row 0 and rows > n zero; sampler
  //   v_s  [sampler_rows(n)][hp]  row i = row i of W2 (output i+1), rows >= n
  //                               zero; sampler and Z GEMM
  //   w_s  [h][np]  rows of W1 (unit k <- all inputs), hidden GEMM
  //   vt_s [h][np]  rows of W2^T (unit k -> all outputs), backward GEMM
  void* wt_s = nullptr;
  void* v_s = nullptr;
  void* w_s = nullptr;
  void* vt_s = nullptr;
  float* b1 = nullptr;  // aliases into theta
  float* b2 = nullptr;

  // instance
  int32_t* row_ptr = nullptr;
  int32_t* col = nullptr;
  void* w = nullptr;      // int32 or float [nnz]
  void* field = nullptr;  // int32 or float [n] or null
  float* J = nullptr;     // dense [n][np] float
  void* J_hi = nullptr;   // dense split, [n][np] bf16
  void* J_lo = nullptr;
  // transverse field alpha [n] (or null) and the workspaces of its
  // off-diagonal local energy: rows are (sample b, flipped spin i) pairs,
  // g = b (n + 1) + i, i = n standing for the sample itself; tim_rows rows
  // per chunk
  float* alpha = nullptr;
  int tim_rows = 0;
  float* tim_A = nullptr;         // [Bmax][hp] FP32 hidden pre-activations of the samples
  int8_t* tim_S8 = nullptr;       // [tim_rows][np] spins of the rows
  void* tim_H = nullptr;          // [tim_rows][hp] hidden activations of the rows
  float* tim_row_part = nullptr;  // [ceil(n/128)][tim_ld] partial log pi of every row per output tile
  long long tim_ld = 0;           // Bmax (n + 1), rounded up to 4

  // workspaces (element type per precision unless noted)
  int8_t* S = nullptr;     // int8 [Bmax][n] samples of vqmc_step
  uint32_t* Sbits = nullptr;  // sparse energy: [ceil(Bmax/32)][n] spins packed 32 samples per word
  void* eloc_part = nullptr;  // [eloc_slices][Bmax] partial energies (int32/float)
  int32_t* eloc_slice = nullptr;  // [eloc_slices + 1] first CSR row of each slice
  int32_t* erow = nullptr;        // [nnz] CSR row of each edge
  int eloc_slices = 1;
  int eloc_wbits = 32;            // bit length of the largest |J_ij| (int32 instances)
  void* E = nullptr;       // int32/float [Bmax]
  void* Sx = nullptr;      // [Bmax][np] spins as GEMM operand
  void* St = nullptr;      // [n][Bp] spins transposed
  void* H = nullptr;       // [Bmax][hp] hidden activations
  void* Ht = nullptr;      // [h][Bp]
  void* D = nullptr;       // [Bmax][np] output adjoint delta
  void* Dt = nullptr;      // [n][Bp]
  void* GAt = nullptr;     // [h][Bp] hidden pre-activation adjoint, transposed
  float* logp = nullptr;   // [Bmax]
  float* coef = nullptr;   // [Bmax]
  double* stats = nullptr; // [4]
  float* row_part = nullptr;  // [ceil(max(n,h)/128)][Bmax] partial row sums
  float* col_part = nullptr;  // [ceil(Bmax/128)][max(np,hp)] partial column sums
  int row_part_ld = 0, col_part_ld = 0, row_part_tiles = 0, col_part_tiles = 0;
  uint32_t* err = nullptr;   // sticky device error word
  // per-part step timing (vqmc_timing_*): events[step][part boundary]
  bool timing = false;
  int64_t timed_steps = 0;
  int64_t launches = 0;
  cudaEvent_t* events = nullptr;  // kMaxTimedSteps * (VQMC_NUM_PARTS + 1)
  vqmc_step_stats* step_stats = nullptr;  // device copy of the last step's stats
  // stochastic reconfiguration, allocated by the first SR call: the
  // Cholesky workspace [sr_ld][sr_ld] (lower triangle), its solution, a
  // vector of ones [sr_ld] (unit coefficients of the per-sample pass), the
  // inverse-transposed diagonal blocks of the factor [sr_ld / 64][64][64],
  // and the Gram kernel's event order [n + h]
  float* sr_A = nullptr;
  float* sr_x = nullptr;
  float* sr_ones = nullptr;
  float* sr_xinv = nullptr;
  int* sr_events = nullptr;
};

namespace vqmc {

// ---- sampler_bf16.cu / sampler_f32.cu: whether the CUDA-core sampler runs
// models with hp padded hidden units and weights of type WT (its register
// layout and shared-memory ring bound hp), in its default or wide layout
template <typename WT>
bool sampler_wt_supports(int hp, bool wide);
// ---- sampler.cu
// boff: index of sample 0 in the Philox counter
cudaError_t launch_uniforms(int B, int n, uint64_t seed, uint64_t iteration, float* d_u, cudaStream_t st,
                            uint32_t boff = 0);
// it_dev: when not null, the Philox iteration is read from it on the device
// (the context's DevState) instead of `iteration`
cudaError_t launch_sampler(const vqmc_ctx* c, int B, const float* d_u, uint64_t iteration, int8_t* d_s,
                           float* d_logp, cudaStream_t st, const unsigned long long* it_dev = nullptr);
// ---- adam.cu: the tensor-core sampler's weight copies (v_s, w_s) into L2
cudaError_t launch_prefetch_sampler_weights(const vqmc_ctx* c, cudaStream_t st);
// ---- sampler_tc.cu: block size of the tensor-core sampler for this model, 0
// if it does not apply; its launcher
int sampler_tc_block(const vqmc_ctx* c);
// sx, stt, sbits: optional copies of the spins for the rest of vqmc_step (the
// GEMM operands Sx, St and the packed layout of the sparse energy)
cudaError_t launch_sampler_tc(const vqmc_ctx* c, int B, const float* d_u, uint64_t iteration, int8_t* d_s,
                              float* d_logp, cudaStream_t st, void* sx = nullptr, void* stt = nullptr,
                              uint32_t* sbits = nullptr, const unsigned long long* it_dev = nullptr);

// ---- eloc.cu
// packed: c->Sbits already holds the spins (written by the sampler)
cudaError_t launch_eloc_sparse(const vqmc_ctx* c, int B, const int8_t* d_s, void* d_e, cudaStream_t st,
                               bool packed = false, bool beside = false);
cudaError_t launch_eloc_dense_finish(const vqmc_ctx* c, int B, const int8_t* d_s, void* d_e, cudaStream_t st);
// ---- tim.cu: adds the transverse field's off-diagonal local energy to d_e
// (float [B]); *launches (if not null) receives the number of kernels
cudaError_t launch_tim_offdiag(const vqmc_ctx* c, int B, const int8_t* d_s, float* d_e, cudaStream_t st,
                               int* launches = nullptr);
// rows per chunk of the flipped states for at most Bmax samples (padded
// sizes hp, np and the activation element size bound its workspace)
int tim_chunk_rows(int Bmax, int n, int hp, int np, int esize);
// advance: also start the next Adam step on the device (t += 1 and its
// factors), saving vqmc_step a launch; the caller advances the host mirror
cudaError_t launch_stats(const vqmc_ctx* c, int B, const void* d_e, double* d_stats, float* d_coef,
                         cudaStream_t st, bool advance = false);
cudaError_t launch_spins_to_operands(const vqmc_ctx* c, int B, const int8_t* d_s, void* Sx, void* St,
                                     cudaStream_t st);
cudaError_t launch_row_sum(const vqmc_ctx* c, int B, int ntiles, float* out, cudaStream_t st);
cudaError_t launch_col_sum(const vqmc_ctx* c, int N, int mtiles, float* out, cudaStream_t st);

// ---- gemm (gemm_simt.cu, gemm_tc.cu): the five masked GEMMs of the forward
// and adjoint passes plus the dense local-energy GEMM.  Operand and output
// layouts are fixed by the context (see vqmc_api.cu).
enum GemmOp {
  kOpHidden = 0,  // H = act(S W1^T + b1); writes H, Ht
  kOpOut = 1,     // Z = H W2^T + b2; logp row partials; if coef: delta, Dt, dc partials
  kOpDV = 2,      // dW2 = Dt . Ht^T  (masked) -> grad, or the Adam step on W2
  kOpGA = 3,      // G = D . W2 ; GA = G * act'(H) -> GAt ; db1 partials
  kOpDW = 4,      // dW1^T = St . GAt^T (masked) -> grad, or the Adam step on W1^T
  kOpEloc = 5     // T = S J (hi/lo) ; row partials 1/2 s.T
};
// Adam factors of one step for the weight-gradient GEMMs that apply the step
// in their epilogue: device pointer to {1 / (1 - beta1^t), 1 / (1 - beta2^t)}
// (the context's DevState).
struct AdamStep {
  const float* ibc;
};
cudaError_t launch_gemm(const vqmc_ctx* c, GemmOp op, int B, const int8_t* d_s, const float* coef,
                        float* grad, cudaStream_t st, const AdamStep* fuse = nullptr);

// ---- vqmc_api.cu: sets the thread-local message of vqmc_last_error
vqmc_status set_last_error(vqmc_status s, const std::string& msg);

// ---- noalloc.cu: scratch bytes vqmc_logprob_noalloc needs for B samples
size_t noalloc_scratch_bytes(const vqmc_ctx* c, int B);

// ---- sr.cu: stochastic reconfiguration (Gram matrix of the per-sample
// score vectors, Cholesky solve, SGD step)
constexpr int kSrMaxBatch = 16384;
int sr_blocks(int B);
int sr_ld(const vqmc_ctx* c);
// allocates the context's SR workspace on first use (synchronous)
cudaError_t sr_workspace(vqmc_ctx* c);
// out[b][c] = scale (O O^T)[b][c] + shift [b == c] from the per-sample
// operands St, Dt, Ht, GAt (unit coefficients); lower triangle, plus the
// upper if mirror; rows/columns [B, pad_to) of out set to the identity
cudaError_t launch_sr_gram(const vqmc_ctx* c, int B, float* out, int ldo, float scale, float shift, bool mirror,
                           int pad_to, cudaStream_t st);
// factors sr_A (B x B plus identity padding) in place and solves for x
cudaError_t launch_sr_solve(const vqmc_ctx* c, int B, const float* rhs, float* x, cudaStream_t st, int* launches);
// theta -= lr delta
cudaError_t launch_sgd(vqmc_ctx* c, const float* delta, float lr, cudaStream_t st);

// ---- adam.cu
cudaError_t launch_mask_params(vqmc_ctx* c, cudaStream_t st);
cudaError_t launch_refresh_weights(vqmc_ctx* c, cudaStream_t st);
// advance = false: the step count and factors were already advanced
cudaError_t launch_adam(vqmc_ctx* c, const float* d_grad, cudaStream_t st, bool advance = true);
// advances the step count t (host mirror and, on `st`, the device state,
// which computes the factors of step t); returns the factors' location
AdamStep adam_advance(vqmc_ctx* c, cudaStream_t st);
// writes the host mirrors of the counters into the device state
cudaError_t launch_set_state(vqmc_ctx* c, cudaStream_t st);
// Adam on the biases alone (their gradients in d_grad at theta's layout)
cudaError_t launch_adam_bias(vqmc_ctx* c, const float* d_grad, AdamStep a, cudaStream_t st);
cudaError_t launch_dense_split(vqmc_ctx* c, cudaStream_t st);

}  // namespace vqmc
