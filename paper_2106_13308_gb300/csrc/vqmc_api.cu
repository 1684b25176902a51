// C ABI of libvqmc (include/vqmc.h): context management and the VQMC
// iteration of the paper (Sec. 2.1, 2.3, 4, 5.1) as a sequence of kernels on
// one stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "gemm.cuh"

using namespace vqmc;

namespace {

thread_local std::string g_last_error;

vqmc_status fail(vqmc_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

#define VQ_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail(e_ == cudaErrorMemoryAllocation ? VQMC_ERR_OOM                               \
                  : e_ == cudaErrorNotSupported   ? VQMC_ERR_UNSUPPORTED                       \
                                                  : VQMC_ERR_CUDA,                             \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                         \
  } while (0)

template <typename P>
cudaError_t dalloc(P** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) return e;
  return cudaMemset(*p, 0, bytes);
}

uint64_t fnv1a(uint64_t h, const void* p, size_t bytes) {
  const unsigned char* c = (const unsigned char*)p;
  for (size_t i = 0; i < bytes; ++i) h = (h ^ c[i]) * 1099511628211ull;
  return h;
}

constexpr int64_t kMaxTimedSteps = 4096;

// the layouts the Python binding mirrors
static_assert(sizeof(vqmc_config) == 48 && sizeof(vqmc_instance) == 64 && sizeof(vqmc_step_stats) == 48,
              "C ABI structure layout");

size_t esize(const vqmc_ctx* c) { return c->prec == VQMC_PREC_BF16 ? 2 : 4; }

cudaStream_t S(vqmc_stream s) { return (cudaStream_t)s; }

vqmc_status check_B(const vqmc_ctx* c, int B) {
  if (!c) return fail(VQMC_ERR_INVALID_ARG, "null context");
  if (B < 0 || B > c->Bmax) return fail(VQMC_ERR_INVALID_ARG, "batch size outside [0, max_batch]");
  return VQMC_OK;
}

// ---- GEMM dispatch ---------------------------------------------------------

template <typename T>
GemmArgs<T> make_args(const vqmc_ctx* c, GemmOp op, int B, const int8_t* d_s, const float* coef, float* grad) {
  GemmArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  a.op = op;
  a.n = c->n;
  a.h = c->h;
  a.act = c->act;
  a.ldr = c->row_part_ld;
  a.ldc = c->col_part_ld;
  a.err = c->err;
  const int n = c->n, h = c->h;
  switch (op) {
    case kOpHidden:
      a.M = B, a.N = h, a.K = n;
      a.A = (const T*)c->Sx, a.lda = c->np;
      a.Bm = (const T*)c->w_s, a.ldb = c->np;
      a.bias = c->b1;
      a.out = (T*)c->H, a.ldo = c->hp;
      a.out_t = (T*)c->Ht, a.ldt = c->Bp;
      break;
    case kOpOut:
      a.M = B, a.N = n, a.K = h;
      a.A = (const T*)c->H, a.lda = c->hp;
      a.Bm = (const T*)c->v_s, a.ldb = c->hp;
      a.bias = c->b2;
      a.S8 = d_s, a.lds8 = n;
      a.coef = coef;
      a.out = (T*)c->D, a.ldo = c->np;
      a.out_t = (T*)c->Dt, a.ldt = c->Bp;
      a.row_part = c->row_part;
      a.col_part = coef ? c->col_part : nullptr;
      break;
    case kOpDV:
      a.M = n, a.N = h, a.K = B;
      a.A = (const T*)c->Dt, a.lda = c->Bp;
      a.Bm = (const T*)c->Ht, a.ldb = c->Bp;
      a.gout = grad + (size_t)n * h + h, a.ldg = h;
      break;
    case kOpGA:
      a.M = B, a.N = h, a.K = n;
      a.A = (const T*)c->D, a.lda = c->np;
      a.Bm = (const T*)c->vt_s, a.ldb = c->np;
      a.aux = (const T*)c->H, a.ldaux = c->hp;
      a.out_t = (T*)c->GAt, a.ldt = c->Bp;
      a.col_part = c->col_part;
      break;
    case kOpDW:
      a.M = n, a.N = h, a.K = B;
      a.A = (const T*)c->St, a.lda = c->Bp;
      a.Bm = (const T*)c->GAt, a.ldb = c->Bp;
      a.gout = grad, a.ldg = h;
      break;
    case kOpEloc:
      a.M = B, a.N = n, a.K = n;
      a.A = (const T*)c->Sx, a.lda = c->np;
      a.ldb = c->np;
      a.S8 = d_s, a.lds8 = n;
      a.row_part = c->row_part;
      break;
  }
  return a;
}

}  // namespace

namespace vqmc {

vqmc_status set_last_error(vqmc_status s, const std::string& msg) { return fail(s, msg); }

cudaError_t launch_gemm(const vqmc_ctx* c, GemmOp op, int B, const int8_t* d_s, const float* coef, float* grad,
                        cudaStream_t st, const AdamStep* fuse) {
  if (c->prec == VQMC_PREC_BF16) {
    GemmArgs<bf16> a = make_args<bf16>(c, op, B, d_s, coef, grad);
    if (op == kOpEloc) a.Bm = (const bf16*)c->J_hi, a.Bm2 = (const bf16*)c->J_lo;
    if (fuse && (op == kOpDV || op == kOpDW)) {
      // the Adam step in the epilogue: W2 (row copy v_s, transposed vt_s) or
      // W1^T (transposed w_s; the row copy wt_s, shifted by one row, only
      // for the CUDA-core sampler)
      const size_t off = op == kOpDV ? (size_t)c->n * c->h + c->h : 0;
      a.theta = c->theta + off, a.adam_m = c->adam_m + off, a.adam_v = c->adam_v + off;
      a.gout = nullptr;
      a.cp_t = (bf16*)(op == kOpDV ? c->vt_s : c->w_s), a.ld_cp_t = c->np;
      const bool row = op == kOpDV || c->sampler != VQMC_SAMPLER_TENSOR_CORE;
      a.cp_row = row ? (bf16*)(op == kOpDV ? c->v_s : c->wt_s) : nullptr;
      a.ld_cp_row = c->hp, a.cp_shift = op == kOpDV ? 0 : 1;
      a.lr = c->cfg.lr, a.beta1 = c->cfg.beta1, a.beta2 = c->cfg.beta2, a.eps = c->cfg.eps;
      a.ibc = fuse->ibc;
    }
    // BF16 GEMMs run on the tcgen05 tensor cores only (sm_103a); no fallback
    return launch_gemm_tc_bf16(a, st);
  }
  GemmArgs<float> a = make_args<float>(c, op, B, d_s, coef, grad);
  if (op == kOpEloc) a.Bm = c->J;
  return launch_gemm_simt_f32(a, st);
}

}  // namespace vqmc

namespace {

// Backward of log pi w.r.t. theta with per-sample weights gout (Sec. 2.1,
// chain rule through the MADE layer of Sec. 2.3).  Requires Sx/St to hold the
// spins.  Recomputes H instead of keeping it from any earlier forward pass.
// With fuse set (BF16), the two weight-gradient GEMMs apply that Adam step
// to W2 and W1^T in their epilogues instead of writing dW2 and dW1^T; both
// run after every GEMM that reads the old weights (hidden adjoint: W2).
// With hidden_done, H and Ht already hold this batch's hidden activations.
vqmc_status backward_from_operands(vqmc_ctx* c, int B, const int8_t* d_s, const float* gout, float* grad,
                                   cudaStream_t st, const AdamStep* fuse = nullptr, bool hidden_done = false) {
  const int n = c->n, h = c->h;
  const int mtiles = (B + 127) / 128;
  if (!hidden_done) VQ_CUDA(launch_gemm(c, kOpHidden, B, d_s, nullptr, nullptr, st));
  VQ_CUDA(launch_gemm(c, kOpOut, B, d_s, gout, nullptr, st));
  VQ_CUDA(launch_col_sum(c, n, mtiles, grad + (size_t)2 * n * h + h, st));  // db2
  VQ_CUDA(launch_gemm(c, kOpGA, B, d_s, nullptr, nullptr, st));
  VQ_CUDA(launch_col_sum(c, h, mtiles, grad + (size_t)n * h, st));          // db1
  VQ_CUDA(launch_gemm(c, kOpDV, B, d_s, nullptr, grad, st, fuse));          // dW2
  VQ_CUDA(launch_gemm(c, kOpDW, B, d_s, nullptr, grad, st, fuse));          // dW1^T
  return VQMC_OK;
}

}  // namespace

extern "C" {

const char* vqmc_last_error(void) { return g_last_error.c_str(); }

vqmc_status vqmc_create(const vqmc_config* cfg, const vqmc_instance* inst, vqmc_ctx** out) {
  if (!cfg || !inst || !out) return fail(VQMC_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  const int n = cfg->n, h = cfg->h, Bmax = cfg->max_batch;
  if (n < 1 || h < 1 || Bmax < 1) return fail(VQMC_ERR_INVALID_ARG, "n, h and max_batch must be >= 1");
  if (cfg->act != VQMC_ACT_RELU && cfg->act != VQMC_ACT_SIGMOID) return fail(VQMC_ERR_INVALID_ARG, "bad act");
  if (cfg->precision != VQMC_PREC_FP32 && cfg->precision != VQMC_PREC_BF16)
    return fail(VQMC_ERR_INVALID_ARG, "bad precision");
  if (inst->n != n) return fail(VQMC_ERR_INVALID_ARG, "instance n differs from config n");
  const int kind = inst->kind;
  if (kind == VQMC_HAM_SPARSE_I32 || kind == VQMC_HAM_SPARSE_F32) {
    if (!inst->row_ptr || inst->nnz < 0 || (inst->nnz > 0 && (!inst->col || !inst->w)))
      return fail(VQMC_ERR_INVALID_ARG, "sparse instance needs row_ptr, col, w");
    if (inst->row_ptr[0] != 0 || inst->row_ptr[n] != inst->nnz)
      return fail(VQMC_ERR_INVALID_ARG, "row_ptr must start at 0 and end at nnz");
    for (int i = 0; i < n; ++i) {
      if (inst->row_ptr[i + 1] < inst->row_ptr[i]) return fail(VQMC_ERR_INVALID_ARG, "row_ptr not monotone");
      for (int p = inst->row_ptr[i]; p < inst->row_ptr[i + 1]; ++p)
        if (inst->col[p] <= i || inst->col[p] >= n)
          return fail(VQMC_ERR_INVALID_ARG, "col must hold the strict upper triangle (i < j < n)");
    }
    if ((size_t)n * 4 > 200 * 1024) return fail(VQMC_ERR_UNSUPPORTED, "sparse energy supports n <= 51200");
  } else if (kind == VQMC_HAM_DENSE_F32) {
    if (!inst->J) return fail(VQMC_ERR_INVALID_ARG, "dense instance needs J");
  } else {
    return fail(VQMC_ERR_INVALID_ARG, "bad instance kind");
  }
  if (inst->alpha) {
    if (kind == VQMC_HAM_SPARSE_I32)
      return fail(VQMC_ERR_INVALID_ARG, "a transverse field needs a float32 instance kind");
    for (int i = 0; i < n; ++i)
      if (!(inst->alpha[i] >= 0.0f) || !std::isfinite(inst->alpha[i]))
        return fail(VQMC_ERR_INVALID_ARG, "alpha must be finite and >= 0");
  }
  if (cfg->sampler > VQMC_SAMPLER_CUDA_CORE_WIDE) return fail(VQMC_ERR_INVALID_ARG, "bad sampler");
  const bool wide = cfg->sampler == VQMC_SAMPLER_CUDA_CORE_WIDE;
  if (!(cfg->precision == VQMC_PREC_BF16 ? sampler_wt_supports<bf16>(pad_up(h), wide)
                                         : sampler_wt_supports<float>(pad_up(h), wide)))
    return fail(VQMC_ERR_UNSUPPORTED,
                "the CUDA-core sampler supports h <= 5120 with BF16 weights and h <= 2816 with FP32 weights");

  vqmc_ctx* c = new vqmc_ctx();
  c->cfg = *cfg;
  c->n = n, c->h = h, c->Bmax = Bmax;
  c->np = pad_up(n), c->hp = pad_up(h), c->Bp = pad_up(Bmax);
  c->act = cfg->act, c->prec = cfg->precision, c->ham = kind;
  c->nnz = (kind == VQMC_HAM_DENSE_F32) ? 0 : inst->nnz;
  c->d = 2ll * n * h + h + n;
  auto cleanup_fail = [&](vqmc_status s, const std::string& m) {
    vqmc_destroy(c);
    return fail(s, m);
  };
  {
    const bool tc_ok = sampler_tc_block(c) > 0 && gemm_tc_available();
    if (cfg->sampler == VQMC_SAMPLER_TENSOR_CORE && !tc_ok)
      return cleanup_fail(VQMC_ERR_UNSUPPORTED,
                          "tensor-core sampler needs BF16, a tcgen05 device and at most 32 hidden units "
                          "completing within 64 steps");
    const bool cc = cfg->sampler == VQMC_SAMPLER_CUDA_CORE || wide;
    c->sampler = (!cc && tc_ok) ? VQMC_SAMPLER_TENSOR_CORE : VQMC_SAMPLER_CUDA_CORE;
    c->sampler_wide = wide ? 1 : 0;
  }
#define VQ_ALLOC(ptr, bytes)                                                                         \
  do {                                                                                               \
    cudaError_t e_ = dalloc(&(ptr), (bytes));                                                        \
    if (e_ != cudaSuccess)                                                                           \
      return cleanup_fail(e_ == cudaErrorMemoryAllocation ? VQMC_ERR_OOM : VQMC_ERR_CUDA,             \
                          std::string("allocation of " #ptr ": ") + cudaGetErrorString(e_));        \
  } while (0)
  if (cudaGetDevice(&c->device) != cudaSuccess) return cleanup_fail(VQMC_ERR_CUDA, "no CUDA device");
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);

  const size_t es = esize(c);
  VQ_ALLOC(c->theta, c->d * 4);
  VQ_ALLOC(c->adam_m, c->d * 4);
  VQ_ALLOC(c->adam_v, c->d * 4);
  VQ_ALLOC(c->grad, c->d * 4);
  c->b1 = c->theta + (size_t)n * h;
  c->b2 = c->theta + (size_t)2 * n * h + h;
  VQ_ALLOC(c->wt_s, (size_t)sampler_rows(n) * c->hp * es);
  VQ_ALLOC(c->v_s, (size_t)sampler_rows(n) * c->hp * es);
  VQ_ALLOC(c->w_s, (size_t)h * c->np * es);
  VQ_ALLOC(c->vt_s, (size_t)h * c->np * es);

  VQ_ALLOC(c->S, (size_t)Bmax * n);
  VQ_ALLOC(c->E, (size_t)Bmax * 4);
  VQ_ALLOC(c->Sx, (size_t)Bmax * c->np * es);
  VQ_ALLOC(c->St, (size_t)n * c->Bp * es);
  VQ_ALLOC(c->H, (size_t)Bmax * c->hp * es);
  VQ_ALLOC(c->Ht, (size_t)h * c->Bp * es);
  VQ_ALLOC(c->D, (size_t)Bmax * c->np * es);
  VQ_ALLOC(c->Dt, (size_t)n * c->Bp * es);
  VQ_ALLOC(c->GAt, (size_t)h * c->Bp * es);
  VQ_ALLOC(c->logp, (size_t)Bmax * 4);
  VQ_ALLOC(c->coef, (size_t)Bmax * 4);
  VQ_ALLOC(c->ones, (size_t)Bmax * 4);
  {
    const std::vector<float> one((size_t)Bmax, 1.0f);
    if (cudaMemcpy(c->ones, one.data(), (size_t)Bmax * 4, cudaMemcpyHostToDevice) != cudaSuccess)
      return cleanup_fail(VQMC_ERR_CUDA, "copy of the unit coefficients failed");
  }
  VQ_ALLOC(c->stats, 8 * sizeof(double));
  c->row_part_tiles = (n + 127) / 128;
  c->row_part_ld = c->Bp;
  VQ_ALLOC(c->row_part, (size_t)c->row_part_tiles * c->row_part_ld * 4);
  c->col_part_tiles = (Bmax + 127) / 128;
  c->col_part_ld = c->np > c->hp ? c->np : c->hp;
  VQ_ALLOC(c->col_part, (size_t)c->col_part_tiles * c->col_part_ld * 4);
  VQ_ALLOC(c->err, 16);
  VQ_ALLOC(c->step_stats, sizeof(vqmc_step_stats));
  VQ_ALLOC(c->dstate, sizeof(DevState));
  // the side stream's short kernels (energy, statistics) are on the critical
  // path: give them the highest priority, the hidden GEMM fills in around them
  int prio_least = 0, prio_greatest = 0;
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  if (cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return cleanup_fail(VQMC_ERR_CUDA, "could not create the context's side stream");

  // instance
  uint64_t hsh = 1469598103934665603ull;
  hsh = fnv1a(hsh, &kind, sizeof(kind));
  if (kind == VQMC_HAM_DENSE_F32) {
    std::vector<float> Jp((size_t)n * c->np, 0.0f);
    for (int i = 0; i < n; ++i) std::memcpy(&Jp[(size_t)i * c->np], inst->J + (size_t)i * n, (size_t)n * 4);
    hsh = fnv1a(hsh, inst->J, (size_t)n * n * 4);
    VQ_ALLOC(c->J, Jp.size() * 4);
    if (cudaMemcpy(c->J, Jp.data(), Jp.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
      return cleanup_fail(VQMC_ERR_CUDA, "copy of J failed");
    if (c->prec == VQMC_PREC_BF16) {
      VQ_ALLOC(c->J_hi, Jp.size() * 2);
      VQ_ALLOC(c->J_lo, Jp.size() * 2);
      if (launch_dense_split(c, 0) != cudaSuccess) return cleanup_fail(VQMC_ERR_CUDA, "split of J failed");
    }
  } else {
    VQ_ALLOC(c->row_ptr, (size_t)(n + 1) * 4);
    VQ_ALLOC(c->col, (size_t)c->nnz * 4);
    VQ_ALLOC(c->w, (size_t)c->nnz * 4);
    bool ok = cudaMemcpy(c->row_ptr, inst->row_ptr, (size_t)(n + 1) * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    if (c->nnz > 0) {
      ok = ok && cudaMemcpy(c->col, inst->col, (size_t)c->nnz * 4, cudaMemcpyHostToDevice) == cudaSuccess;
      ok = ok && cudaMemcpy(c->w, inst->w, (size_t)c->nnz * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    }
    hsh = fnv1a(hsh, inst->row_ptr, (size_t)(n + 1) * 4);
    hsh = fnv1a(hsh, inst->col, (size_t)c->nnz * 4);
    hsh = fnv1a(hsh, inst->w, (size_t)c->nnz * 4);
    if (!ok) return cleanup_fail(VQMC_ERR_CUDA, "copy of the instance failed");
    // energy kernel: packed spins, and row slices of about equal edge counts so
    // that (Bmax/32 words) x slices CTAs cover the GPU about twice
    const int words = (Bmax + 31) / 32;
    int slices = (2 * c->num_sms + words - 1) / words;
    slices = slices < 1 ? 1 : (slices > 32 ? 32 : slices);
    if (slices > n) slices = n;
    std::vector<int32_t> rb(slices + 1, n);
    rb[0] = 0;
    for (int q = 1, i = 0; q < slices; ++q) {
      const long long target = (long long)c->nnz * q / slices;
      while (i < n && inst->row_ptr[i] < target) ++i;
      rb[q] = i;
    }
    c->eloc_slices = slices;
    if (c->ham == VQMC_HAM_SPARSE_I32) {
      long long wmax = 0;  // the bit-sliced energy kernel needs |J_ij| < 2^wbits
      for (long long p = 0; p < c->nnz; ++p) {
        const long long a = std::llabs((long long)((const int32_t*)inst->w)[p]);
        wmax = a > wmax ? a : wmax;
      }
      int wb = 0;
      while (wb < 32 && (1ll << wb) <= wmax) ++wb;
      c->eloc_wbits = wb;
    }
    std::vector<int32_t> er((size_t)c->nnz);
    for (int i = 0; i < n; ++i)
      for (int p = inst->row_ptr[i]; p < inst->row_ptr[i + 1]; ++p) er[(size_t)p] = i;
    VQ_ALLOC(c->erow, (size_t)(c->nnz > 0 ? c->nnz : 1) * 4);
    if (c->nnz > 0 && cudaMemcpy(c->erow, er.data(), (size_t)c->nnz * 4, cudaMemcpyHostToDevice) != cudaSuccess)
      return cleanup_fail(VQMC_ERR_CUDA, "copy of the edge rows failed");
    VQ_ALLOC(c->Sbits, (size_t)words * n * 4);
    VQ_ALLOC(c->eloc_part, (size_t)slices * Bmax * 4);
    VQ_ALLOC(c->eloc_slice, (size_t)(slices + 1) * 4);
    if (cudaMemcpy(c->eloc_slice, rb.data(), (size_t)(slices + 1) * 4, cudaMemcpyHostToDevice) != cudaSuccess)
      return cleanup_fail(VQMC_ERR_CUDA, "copy of the row slices failed");
  }
  if (inst->field) {
    VQ_ALLOC(c->field, (size_t)n * 4);
    if (cudaMemcpy(c->field, inst->field, (size_t)n * 4, cudaMemcpyHostToDevice) != cudaSuccess)
      return cleanup_fail(VQMC_ERR_CUDA, "copy of the field failed");
    hsh = fnv1a(hsh, inst->field, (size_t)n * 4);
  }
  if (inst->alpha) {
    VQ_ALLOC(c->alpha, (size_t)n * 4);
    if (cudaMemcpy(c->alpha, inst->alpha, (size_t)n * 4, cudaMemcpyHostToDevice) != cudaSuccess)
      return cleanup_fail(VQMC_ERR_CUDA, "copy of alpha failed");
    hsh = fnv1a(hsh, inst->alpha, (size_t)n * 4);
    c->tim_rows = tim_chunk_rows(Bmax, n, c->hp, c->np, (int)esize(c));
    const size_t rows = (size_t)c->tim_rows;
    VQ_ALLOC(c->tim_A, (size_t)Bmax * c->hp * 4);
    VQ_ALLOC(c->tim_S8, rows * c->np);
    VQ_ALLOC(c->tim_H, rows * c->hp * esize(c));
    c->tim_ld = ((long long)Bmax * (n + 1) + 3) / 4 * 4;
    VQ_ALLOC(c->tim_row_part, (size_t)((n + 127) / 128) * (size_t)c->tim_ld * 4);
  }
  c->inst_hash = hsh;
  if (launch_refresh_weights(c, 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
    return cleanup_fail(VQMC_ERR_CUDA, "initial weight refresh failed");
#undef VQ_ALLOC
  *out = c;
  return VQMC_OK;
}

void vqmc_destroy(vqmc_ctx* c) {
  if (!c) return;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->events) {
    for (int64_t q = 0; q < kMaxTimedSteps * (VQMC_NUM_PARTS + 1); ++q) cudaEventDestroy(c->events[q]);
    delete[] c->events;
  }
  void* ptrs[] = {c->theta, c->adam_m, c->adam_v, c->grad, c->wt_s, c->v_s, c->w_s, c->vt_s, c->row_ptr,
                  c->col, c->w, c->field, c->J, c->J_hi, c->J_lo, c->S, c->E, c->Sx, c->St, c->H, c->Ht,
                  c->D, c->Dt, c->GAt, c->logp, c->coef, c->stats, c->row_part, c->col_part, c->err,
                  c->step_stats, c->Sbits, c->eloc_part, c->eloc_slice, c->erow, c->alpha, c->tim_A,
                  c->tim_S8, c->tim_H, c->tim_row_part, c->sr_A, c->sr_x, c->sr_ones, c->sr_xinv,
                  c->sr_events, c->dstate, c->ones};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete c;
}

int64_t vqmc_num_params(const vqmc_ctx* c) { return c ? c->d : 0; }

float* vqmc_params_device(vqmc_ctx* c) { return c ? c->theta : nullptr; }

uint64_t vqmc_iteration(const vqmc_ctx* c) { return c ? c->iter : 0; }

vqmc_status vqmc_params_updated(vqmc_ctx* c, vqmc_stream stream) {
  if (!c) return fail(VQMC_ERR_INVALID_ARG, "null context");
  VQ_CUDA(launch_mask_params(c, S(stream)));
  VQ_CUDA(launch_refresh_weights(c, S(stream)));
  return VQMC_OK;
}

vqmc_status vqmc_set_params(vqmc_ctx* c, const float* theta, int on_device, vqmc_stream stream) {
  if (!c || !theta) return fail(VQMC_ERR_INVALID_ARG, "null argument");
  VQ_CUDA(cudaMemcpyAsync(c->theta, theta, c->d * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          S(stream)));
  VQ_CUDA(cudaMemsetAsync(c->adam_m, 0, c->d * 4, S(stream)));
  VQ_CUDA(cudaMemsetAsync(c->adam_v, 0, c->d * 4, S(stream)));
  c->adam_t = 0;
  VQ_CUDA(launch_set_state(c, S(stream)));
  vqmc_status s = vqmc_params_updated(c, stream);
  if (s != VQMC_OK) return s;
  if (!on_device) VQ_CUDA(cudaStreamSynchronize(S(stream)));
  return VQMC_OK;
}

vqmc_status vqmc_get_params(vqmc_ctx* c, float* theta, int on_device, vqmc_stream stream) {
  if (!c || !theta) return fail(VQMC_ERR_INVALID_ARG, "null argument");
  VQ_CUDA(cudaMemcpyAsync(theta, c->theta, c->d * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          S(stream)));
  if (!on_device) VQ_CUDA(cudaStreamSynchronize(S(stream)));
  return VQMC_OK;
}

vqmc_status vqmc_uniforms(vqmc_ctx* c, int32_t B, uint64_t iteration, float* d_u, vqmc_stream stream) {
  vqmc_status s = check_B(c, B);
  if (s != VQMC_OK) return s;
  if (B > 0 && !d_u) return fail(VQMC_ERR_INVALID_ARG, "null output");
  VQ_CUDA(launch_uniforms(B, c->n, c->cfg.seed, iteration, d_u, S(stream), c->sample_offset));
  return VQMC_OK;
}

vqmc_status vqmc_sample(vqmc_ctx* c, int32_t B, const float* d_u, uint64_t iteration, int8_t* d_s, float* d_logp,
                        vqmc_stream stream) {
  vqmc_status s = check_B(c, B);
  if (s != VQMC_OK) return s;
  if (B > 0 && !d_s) return fail(VQMC_ERR_INVALID_ARG, "null output");
  VQ_CUDA(launch_sampler(c, B, d_u, iteration, d_s, d_logp, S(stream)));
  return VQMC_OK;
}

vqmc_status vqmc_local_energy(vqmc_ctx* c, int32_t B, const int8_t* d_s, void* d_e, vqmc_stream stream) {
  vqmc_status s = check_B(c, B);
  if (s != VQMC_OK) return s;
  if (B == 0) return VQMC_OK;
  if (!d_s || !d_e) return fail(VQMC_ERR_INVALID_ARG, "null argument");
  if (c->ham == VQMC_HAM_DENSE_F32) {
    VQ_CUDA(launch_spins_to_operands(c, B, d_s, c->Sx, nullptr, S(stream)));
    VQ_CUDA(launch_gemm(c, kOpEloc, B, d_s, nullptr, nullptr, S(stream)));
    VQ_CUDA(launch_eloc_dense_finish(c, B, d_s, d_e, S(stream)));
  } else {
    VQ_CUDA(launch_eloc_sparse(c, B, d_s, d_e, S(stream)));
  }
  VQ_CUDA(launch_tim_offdiag(c, B, d_s, (float*)d_e, S(stream)));
  return VQMC_OK;
}

vqmc_status vqmc_logprob(vqmc_ctx* c, int32_t B, const int8_t* d_s, float* d_logp, vqmc_stream stream) {
  vqmc_status s = check_B(c, B);
  if (s != VQMC_OK) return s;
  if (B == 0) return VQMC_OK;
  if (!d_s || !d_logp) return fail(VQMC_ERR_INVALID_ARG, "null argument");
  VQ_CUDA(launch_spins_to_operands(c, B, d_s, c->Sx, nullptr, S(stream)));
  VQ_CUDA(launch_gemm(c, kOpHidden, B, d_s, nullptr, nullptr, S(stream)));
  VQ_CUDA(launch_gemm(c, kOpOut, B, d_s, nullptr, nullptr, S(stream)));
  VQ_CUDA(launch_row_sum(c, B, c->row_part_tiles, d_logp, S(stream)));
  return VQMC_OK;
}

vqmc_status vqmc_logprob_backward(vqmc_ctx* c, int32_t B, const int8_t* d_s, const float* d_gout, float* d_grad,
                                  vqmc_stream stream) {
  vqmc_status s = check_B(c, B);
  if (s != VQMC_OK) return s;
  if (!d_grad) return fail(VQMC_ERR_INVALID_ARG, "null gradient");
  if (B == 0) {
    VQ_CUDA(cudaMemsetAsync(d_grad, 0, c->d * 4, S(stream)));
    return VQMC_OK;
  }
  if (!d_s || !d_gout) return fail(VQMC_ERR_INVALID_ARG, "null argument");
  VQ_CUDA(launch_spins_to_operands(c, B, d_s, c->Sx, c->St, S(stream)));
  return backward_from_operands(c, B, d_s, d_gout, d_grad, S(stream));
}

vqmc_status vqmc_energy_stats(vqmc_ctx* c, int32_t B, const void* d_e, double* d_stats, float* d_coef,
                              vqmc_stream stream) {
  vqmc_status s = check_B(c, B);
  if (s != VQMC_OK) return s;
  if (B == 0) return VQMC_OK;
  if (!d_e || !d_stats) return fail(VQMC_ERR_INVALID_ARG, "null argument");
  VQ_CUDA(launch_stats(c, B, d_e, d_stats, d_coef, S(stream)));
  return VQMC_OK;
}

vqmc_status vqmc_grad(vqmc_ctx* c, int32_t B, const int8_t* d_s, const void* d_e, float* d_grad, double* d_stats,
                      vqmc_stream stream) {
  vqmc_status s = check_B(c, B);
  if (s != VQMC_OK) return s;
  if (!d_grad) return fail(VQMC_ERR_INVALID_ARG, "null gradient");
  if (B == 0) {
    VQ_CUDA(cudaMemsetAsync(d_grad, 0, c->d * 4, S(stream)));
    return VQMC_OK;
  }
  if (!d_s || !d_e) return fail(VQMC_ERR_INVALID_ARG, "null argument");
  VQ_CUDA(launch_stats(c, B, d_e, d_stats ? d_stats : c->stats, c->coef, S(stream)));
  VQ_CUDA(launch_spins_to_operands(c, B, d_s, c->Sx, c->St, S(stream)));
  return backward_from_operands(c, B, d_s, c->coef, d_grad, S(stream));
}

vqmc_status vqmc_adam(vqmc_ctx* c, const float* d_grad, vqmc_stream stream) {
  if (!c || !d_grad) return fail(VQMC_ERR_INVALID_ARG, "null argument");
  VQ_CUDA(launch_adam(c, d_grad, S(stream)));
  return VQMC_OK;
}

}  // extern "C"

namespace {
// The step's record, and the device iteration counter advanced for the next
// step (the sampler of this step read it).
__global__ void fill_step_stats(const double* st, DevState* ds, const uint32_t* err, vqmc_step_stats* out) {
  out->mean = st[0];
  out->var = st[1];
  out->min = st[2];
  out->max = st[3];
  out->iteration = ds->iter;
  out->error_flags = *err;
  out->reserved = 0;
  ds->iter += 1;
}
}  // namespace

extern "C" {

vqmc_status vqmc_step(vqmc_ctx* c, int32_t B, vqmc_stream stream, vqmc_step_stats* h_out) {
  vqmc_status s = check_B(c, B);
  if (s != VQMC_OK) return s;
  if (B == 0) return fail(VQMC_ERR_INVALID_ARG, "vqmc_step needs B >= 1");
  cudaStream_t st = S(stream);
  const bool timed = c->timing && c->timed_steps < kMaxTimedSteps;
  cudaEvent_t* ev = timed ? c->events + c->timed_steps * (VQMC_NUM_PARTS + 1) : nullptr;
  auto mark = [&](int part) {
    if (ev) cudaEventRecord(ev[part], st);
  };
  mark(0);
  // (a) exact samples; the tensor-core sampler also writes the spins' GEMM
  // operand layouts and the energy's packed layout, otherwise two kernels
  // produce them (timed with the energy part)
  const bool tc = c->sampler == VQMC_SAMPLER_TENSOR_CORE;
  const bool sparse = c->ham != VQMC_HAM_DENSE_F32;
  const unsigned long long* it_dev = &c->dstate->iter;
  if (tc)
    VQ_CUDA(launch_sampler_tc(c, B, nullptr, c->iter, c->S, nullptr, st, c->Sx, c->St, sparse ? c->Sbits : nullptr,
                              it_dev));
  else VQ_CUDA(launch_sampler(c, B, nullptr, c->iter, c->S, nullptr, st, it_dev));
  mark(1);
  if (!tc) VQ_CUDA(launch_spins_to_operands(c, B, c->S, c->Sx, c->St, st));
  // (c) local energies and (d) FP64 statistics with the score-function
  // coefficients; the statistics kernel also starts this iteration's Adam
  // step on the device (step count, factors).  For a sparse instance without
  // a transverse field both need only the samples, like the hidden-activation
  // GEMM of (b), and share no buffer with it: they run on the side stream
  // beside that GEMM.
  const bool overlap = sparse && !c->alpha;
  int tim_launches = 0;
  if (overlap) {
    VQ_CUDA(cudaEventRecord(c->ev_fork, st));
    VQ_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    VQ_CUDA(launch_eloc_sparse(c, B, c->S, c->E, c->side, /*packed=*/tc, /*beside=*/true));
    VQ_CUDA(launch_stats(c, B, c->E, c->stats, c->coef, c->side, /*advance=*/true));
    VQ_CUDA(cudaEventRecord(c->ev_join, c->side));
    VQ_CUDA(launch_gemm(c, kOpHidden, B, c->S, nullptr, nullptr, st));
    mark(2);
    VQ_CUDA(cudaStreamWaitEvent(st, c->ev_join, 0));
  } else {
    if (c->ham == VQMC_HAM_DENSE_F32) {
      VQ_CUDA(launch_gemm(c, kOpEloc, B, c->S, nullptr, nullptr, st));
      VQ_CUDA(launch_eloc_dense_finish(c, B, c->S, c->E, st));
    } else {
      VQ_CUDA(launch_eloc_sparse(c, B, c->S, c->E, st, /*packed=*/tc));
    }
    // transverse field: the off-diagonal part (n + 1 log-prob rows per sample)
    VQ_CUDA(launch_tim_offdiag(c, B, c->S, (float*)c->E, st, &tim_launches));
    mark(2);
    VQ_CUDA(launch_stats(c, B, c->E, c->stats, c->coef, st, /*advance=*/true));
  }
  c->adam_t += 1;
  mark(3);
  // (b) + adjoint: gradient with recomputed hidden activations; for BF16 the
  // weight-gradient GEMMs apply the Adam step to the weights themselves
  const bool fuse = c->prec == VQMC_PREC_BF16;
  const AdamStep astep{&c->dstate->ibc1};
  s = backward_from_operands(c, B, c->S, c->coef, c->grad, st, fuse ? &astep : nullptr, /*hidden_done=*/overlap);
  if (s != VQMC_OK) return s;
  mark(4);
  if (fuse) VQ_CUDA(launch_adam_bias(c, c->grad, astep, st));
  else VQ_CUDA(launch_adam(c, c->grad, st, /*advance=*/false));
  // the next step's sampler streams v_s and w_s: have them in L2 (the
  // optimiser's traffic evicted them)
  if (c->sampler == VQMC_SAMPLER_TENSOR_CORE) VQ_CUDA(launch_prefetch_sampler_weights(c, st));
  mark(5);
  fill_step_stats<<<1, 1, 0, st>>>(c->stats, c->dstate, c->err, c->step_stats);
  VQ_CUDA(cudaGetLastError());
  if (h_out) VQ_CUDA(cudaMemcpyAsync(h_out, c->step_stats, sizeof(vqmc_step_stats), cudaMemcpyDeviceToHost, st));
  if (timed) {
    c->timed_steps += 1;
    // sampler (+ operand layouts unless the tensor-core sampler writes them), energy (dense: GEMM +
    // finish; sparse: [pack,] slices [, slice sum]), stats (with the Adam step counter), 7 gradient
    // kernels, [Adam with the weight-copy refresh unless fused into the gradient GEMMs,] bias Adam,
    // [2 L2 prefetches,] step stats
    const int sampler = tc ? 1 : 2;
    const int energy = !sparse ? 2 : (tc ? 0 : 1) + 1 + (c->eloc_slices > 1 ? 1 : 0);
    c->launches += sampler + energy + tim_launches + 1 + 7 + (fuse ? 1 : 2) + (tc ? 2 : 0) + 1;
  }
  c->iter += 1;
  return VQMC_OK;
}

}  // extern "C"

// ------------------------------------------------- sampling parallelism
//
// Sec. 4: the samples of one iteration are independent, so L GPUs draw
// disjoint shards of the batch (each context's sample offset places its
// samples in the Philox counter) and combine their gradients.  With the
// global mean Ebar over all B_tot samples,
//     sum_b (E_b - Ebar) g_b = sum_b (E_b - c) g_b - (Ebar - c) sum_b g_b
// for any constant c, g_b = grad log pi(s_b): each shard writes the two
// d-vectors on the right and the FP64 sums of E_b - c and (E_b - c)^2; one
// all-reduce (sum) of those gives every replica the exact global-baseline
// gradient, and identical Adam steps keep the replicas identical.

namespace {

template <typename T>
__global__ void shard_coef_kernel(int B, const T* __restrict__ e, double shift, float* __restrict__ c1,
                                  double* __restrict__ scal, uint32_t* err) {
  __shared__ double s1[256], s2[256];
  const int tid = threadIdx.x;
  double a = 0.0, q = 0.0;
  bool bad = false;
  for (int b = tid; b < B; b += 256) {
    const double x = (double)e[b] - shift;
    bad |= !isfinite(x);
    c1[b] = (float)x;
    a += x;
    q += x * x;
  }
  s1[tid] = a, s2[tid] = q;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {  // fixed order: bit-reproducible sums
    if (tid < w) s1[tid] += s1[tid + w], s2[tid] += s2[tid + w];
    __syncthreads();
  }
  if (bad) atomicOr(err, kErrNonfinite);
  if (tid == 0) scal[0] = s1[0], scal[1] = s2[0], scal[2] = (double)B;
}

// grad = (S1 - (Ebar - c) S0) / B_tot from the reduced sums; block 0 writes
// the FP64 statistics {mean, var} and advances the Philox iteration
__global__ void shard_grad_kernel(long long d, const float* __restrict__ sums, const double* __restrict__ scal,
                                  double shift, float* __restrict__ grad, double* __restrict__ stats, DevState* ds,
                                  uint32_t* err) {
  const double Bt = scal[2];
  const bool ok = Bt >= 1.0 && isfinite(scal[0]) && isfinite(scal[1]);
  const double m = ok ? scal[0] / Bt : 0.0;  // Ebar - c
  const float a = (float)m, inv = ok ? (float)(1.0 / Bt) : 0.0f;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < d; j += (long long)gridDim.x * blockDim.x)
    grad[j] = fmaf(-a, sums[d + j], sums[j]) * inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (!ok) atomicOr(err, kErrNonfinite);
    if (stats) stats[0] = shift + m, stats[1] = ok ? scal[1] / Bt - m * m : 0.0;
    ds->iter += 1;
  }
}

}  // namespace

extern "C" {

vqmc_status vqmc_set_sample_offset(vqmc_ctx* c, uint32_t b0) {
  if (!c) return fail(VQMC_ERR_INVALID_ARG, "null context");
  c->sample_offset = b0;
  return VQMC_OK;
}

vqmc_status vqmc_shard_sums(vqmc_ctx* c, int32_t B, const int8_t* d_s, const void* d_e, double shift, float* d_sums,
                            double* d_scalars, vqmc_stream stream) {
  vqmc_status s = check_B(c, B);
  if (s != VQMC_OK) return s;
  if (!d_sums || !d_scalars) return fail(VQMC_ERR_INVALID_ARG, "null output");
  if (!std::isfinite(shift)) return fail(VQMC_ERR_INVALID_ARG, "shift must be finite");
  if (d_s && !d_e) return fail(VQMC_ERR_INVALID_ARG, "samples given without their energies");
  cudaStream_t st = S(stream);
  if (B == 0) {
    VQ_CUDA(cudaMemsetAsync(d_sums, 0, (size_t)c->d * 8, st));
    VQ_CUDA(cudaMemsetAsync(d_scalars, 0, 3 * sizeof(double), st));
    return VQMC_OK;
  }
  const bool sparse = c->ham != VQMC_HAM_DENSE_F32;
  if (!d_s) {
    // this shard's samples (internal Philox at the iteration counter, from
    // the sample offset) and their local energies, as in vqmc_step
    const bool tc = c->sampler == VQMC_SAMPLER_TENSOR_CORE;
    const unsigned long long* it_dev = &c->dstate->iter;
    if (tc)
      VQ_CUDA(launch_sampler_tc(c, B, nullptr, c->iter, c->S, nullptr, st, c->Sx, c->St, sparse ? c->Sbits : nullptr,
                                it_dev));
    else {
      VQ_CUDA(launch_sampler(c, B, nullptr, c->iter, c->S, nullptr, st, it_dev));
      VQ_CUDA(launch_spins_to_operands(c, B, c->S, c->Sx, c->St, st));
    }
    if (sparse) {
      VQ_CUDA(launch_eloc_sparse(c, B, c->S, c->E, st, /*packed=*/tc));
    } else {
      VQ_CUDA(launch_gemm(c, kOpEloc, B, c->S, nullptr, nullptr, st));
      VQ_CUDA(launch_eloc_dense_finish(c, B, c->S, c->E, st));
    }
    VQ_CUDA(launch_tim_offdiag(c, B, c->S, (float*)c->E, st));
    d_s = c->S, d_e = c->E;
  } else {
    VQ_CUDA(launch_spins_to_operands(c, B, d_s, c->Sx, c->St, st));
  }
  if (c->ham == VQMC_HAM_SPARSE_I32)
    shard_coef_kernel<int32_t><<<1, 256, 0, st>>>(B, (const int32_t*)d_e, shift, c->coef, d_scalars, c->err);
  else
    shard_coef_kernel<float><<<1, 256, 0, st>>>(B, (const float*)d_e, shift, c->coef, d_scalars, c->err);
  VQ_CUDA(cudaGetLastError());
  s = backward_from_operands(c, B, d_s, c->coef, d_sums, st);
  if (s != VQMC_OK) return s;
  return backward_from_operands(c, B, d_s, c->ones, d_sums + c->d, st, nullptr, /*hidden_done=*/true);
}

vqmc_status vqmc_shard_apply(vqmc_ctx* c, const float* d_sums, const double* d_scalars, double shift, float* d_grad,
                             double* d_stats, vqmc_stream stream) {
  if (!c) return fail(VQMC_ERR_INVALID_ARG, "null context");
  if (!d_sums || !d_scalars) return fail(VQMC_ERR_INVALID_ARG, "null argument");
  if (!std::isfinite(shift)) return fail(VQMC_ERR_INVALID_ARG, "shift must be finite");
  cudaStream_t st = S(stream);
  float* g = d_grad ? d_grad : c->grad;
  const long long work = (c->d + 255) / 256;
  const int grid = (int)std::min<long long>(work, 8LL * c->num_sms);
  shard_grad_kernel<<<grid, 256, 0, st>>>(c->d, d_sums, d_scalars, shift, g, d_stats, c->dstate, c->err);
  VQ_CUDA(cudaGetLastError());
  VQ_CUDA(launch_adam(c, g, st));
  c->iter += 1;
  return VQMC_OK;
}

}  // extern "C"

// ------------------------------------------- stochastic reconfiguration

namespace {

vqmc_status sr_check(vqmc_ctx* c, int B) {
  vqmc_status s = check_B(c, B);
  if (s != VQMC_OK) return s;
  if (c->prec != VQMC_PREC_FP32)
    return fail(VQMC_ERR_UNSUPPORTED, "stochastic reconfiguration needs an FP32 context");
  if (B > kSrMaxBatch) return fail(VQMC_ERR_UNSUPPORTED, "stochastic reconfiguration supports B <= 16384");
  VQ_CUDA(sr_workspace(c));
  return VQMC_OK;
}

// The adjoint pass's operands with unit coefficients: St, Dt, Ht, GAt hold
// each sample's s, delta, H and GA (Sec. 2.3 chain rule).
vqmc_status sr_operands(vqmc_ctx* c, int B, const int8_t* d_s, cudaStream_t st) {
  VQ_CUDA(launch_spins_to_operands(c, B, d_s, c->Sx, c->St, st));
  VQ_CUDA(launch_gemm(c, kOpHidden, B, d_s, nullptr, nullptr, st));
  VQ_CUDA(launch_gemm(c, kOpOut, B, d_s, c->sr_ones, nullptr, st));
  VQ_CUDA(launch_gemm(c, kOpGA, B, d_s, nullptr, nullptr, st));
  return VQMC_OK;
}

// delta = O^T x with (O O^T / B + lambda) x = (E - mean)/B (Sec. 2.1)
vqmc_status sr_direction(vqmc_ctx* c, int B, const int8_t* d_s, const void* d_e, float lambda, float* d_delta,
                         double* d_stats, cudaStream_t st, bool stats_done = false) {
  if (!stats_done) VQ_CUDA(launch_stats(c, B, d_e, d_stats, c->coef, st));
  vqmc_status s = sr_operands(c, B, d_s, st);
  if (s != VQMC_OK) return s;
  VQ_CUDA(launch_sr_gram(c, B, c->sr_A, sr_ld(c), 1.0f / (float)B, lambda, false, sr_blocks(B) * 64, st));
  VQ_CUDA(launch_sr_solve(c, B, c->coef, c->sr_x, st, nullptr));
  return backward_from_operands(c, B, d_s, c->sr_x, d_delta, st);
}

}  // namespace

extern "C" {

vqmc_status vqmc_sr_gram(vqmc_ctx* c, int32_t B, const int8_t* d_s, float* d_gram, vqmc_stream stream) {
  vqmc_status s = sr_check(c, B);
  if (s != VQMC_OK) return s;
  if (B == 0) return VQMC_OK;
  if (!d_s || !d_gram) return fail(VQMC_ERR_INVALID_ARG, "null argument");
  s = sr_operands(c, B, d_s, S(stream));
  if (s != VQMC_OK) return s;
  VQ_CUDA(launch_sr_gram(c, B, d_gram, B, 1.0f, 0.0f, true, 0, S(stream)));
  return VQMC_OK;
}

vqmc_status vqmc_sr_direction(vqmc_ctx* c, int32_t B, const int8_t* d_s, const void* d_e, float lambda,
                              float* d_delta, double* d_stats, vqmc_stream stream) {
  vqmc_status s = sr_check(c, B);
  if (s != VQMC_OK) return s;
  if (!(lambda > 0.0f) || !std::isfinite(lambda)) return fail(VQMC_ERR_INVALID_ARG, "lambda must be finite and > 0");
  if (!d_delta) return fail(VQMC_ERR_INVALID_ARG, "null direction");
  if (B == 0) {
    VQ_CUDA(cudaMemsetAsync(d_delta, 0, c->d * 4, S(stream)));
    return VQMC_OK;
  }
  if (!d_s || !d_e) return fail(VQMC_ERR_INVALID_ARG, "null argument");
  return sr_direction(c, B, d_s, d_e, lambda, d_delta, d_stats ? d_stats : c->stats, S(stream));
}

vqmc_status vqmc_sr_step(vqmc_ctx* c, int32_t B, float lr, float lambda, vqmc_stream stream, vqmc_step_stats* h_out) {
  vqmc_status s = sr_check(c, B);
  if (s != VQMC_OK) return s;
  if (B == 0) return fail(VQMC_ERR_INVALID_ARG, "vqmc_sr_step needs B >= 1");
  if (!(lambda > 0.0f) || !std::isfinite(lambda)) return fail(VQMC_ERR_INVALID_ARG, "lambda must be finite and > 0");
  if (!std::isfinite(lr)) return fail(VQMC_ERR_INVALID_ARG, "lr must be finite");
  cudaStream_t st = S(stream);
  const bool timed = c->timing && c->timed_steps < kMaxTimedSteps;
  cudaEvent_t* ev = timed ? c->events + c->timed_steps * (VQMC_NUM_PARTS + 1) : nullptr;
  auto mark = [&](int part) {
    if (ev) cudaEventRecord(ev[part], st);
  };
  mark(0);
  VQ_CUDA(launch_sampler(c, B, nullptr, c->iter, c->S, nullptr, st, &c->dstate->iter));
  mark(1);
  if (c->ham == VQMC_HAM_DENSE_F32) {
    VQ_CUDA(launch_spins_to_operands(c, B, c->S, c->Sx, nullptr, st));
    VQ_CUDA(launch_gemm(c, kOpEloc, B, c->S, nullptr, nullptr, st));
    VQ_CUDA(launch_eloc_dense_finish(c, B, c->S, c->E, st));
  } else {
    VQ_CUDA(launch_eloc_sparse(c, B, c->S, c->E, st));
  }
  int tim_launches = 0;
  VQ_CUDA(launch_tim_offdiag(c, B, c->S, (float*)c->E, st, &tim_launches));
  mark(2);
  VQ_CUDA(launch_stats(c, B, c->E, c->stats, c->coef, st));
  mark(3);
  s = sr_direction(c, B, c->S, c->E, lambda, c->grad, c->stats, st, /*stats_done=*/true);
  if (s != VQMC_OK) return s;
  mark(4);
  VQ_CUDA(launch_sgd(c, c->grad, lr, st));
  VQ_CUDA(launch_refresh_weights(c, st));
  mark(5);
  fill_step_stats<<<1, 1, 0, st>>>(c->stats, c->dstate, c->err, c->step_stats);
  VQ_CUDA(cudaGetLastError());
  if (h_out) VQ_CUDA(cudaMemcpyAsync(h_out, c->step_stats, sizeof(vqmc_step_stats), cudaMemcpyDeviceToHost, st));
  if (timed) {
    c->timed_steps += 1;
    // sampler, energy (dense: operands + GEMM + finish; sparse: pack + slices [+ sum]) [+ transverse
    // field], stats, SR direction (operands + 3 GEMMs, Gram, 2T - 1 Cholesky launches, solve, 7
    // adjoint kernels), SGD, refresh (3), step stats
    const int energy = c->ham == VQMC_HAM_DENSE_F32 ? 3 : 2 + (c->eloc_slices > 1 ? 1 : 0);
    c->launches += 1 + energy + tim_launches + 1 + (4 + 1 + 2 * sr_blocks(B) + 7) + 1 + 3 + 1;
  }
  c->iter += 1;
  return VQMC_OK;
}

}  // extern "C"

// ----------------------------------------------------- captured iterations

extern "C" {

vqmc_status vqmc_graph_capture(vqmc_ctx* c, int32_t B, int32_t steps, int32_t optimizer, float sr_lr,
                               float sr_lambda, vqmc_stream stream) {
  vqmc_status s = check_B(c, B);
  if (s != VQMC_OK) return s;
  if (B == 0 || steps < 1) return fail(VQMC_ERR_INVALID_ARG, "graph capture needs B >= 1 and steps >= 1");
  if (optimizer != VQMC_OPT_ADAM && optimizer != VQMC_OPT_SR) return fail(VQMC_ERR_INVALID_ARG, "bad optimizer");
  if (!stream) return fail(VQMC_ERR_INVALID_ARG, "graph capture needs a stream other than the legacy default stream");
  if (optimizer == VQMC_OPT_SR) {
    s = sr_check(c, B);  // allocates the SR workspace outside the capture
    if (s != VQMC_OK) return s;
  }
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    c->graph_steps = 0;
  }
  cudaStream_t st = S(stream);
  const bool timing = c->timing;
  const uint64_t iter0 = c->iter;
  const int64_t t0 = c->adam_t;
  VQ_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  c->timing = false;  // no timing events inside the graph
  for (int q = 0; q < steps && s == VQMC_OK; ++q)
    s = optimizer == VQMC_OPT_SR ? vqmc_sr_step(c, B, sr_lr, sr_lambda, stream, nullptr) : vqmc_step(c, B, stream, nullptr);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  // capturing enqueues nothing: the counters stay where they were
  c->timing = timing, c->iter = iter0, c->adam_t = t0;
  if (s != VQMC_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return s != VQMC_OK ? s : fail(VQMC_ERR_CUDA, std::string("stream capture: ") + cudaGetErrorString(e));
  }
  const cudaError_t ei = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    c->graph = nullptr;
    return fail(VQMC_ERR_CUDA, std::string("graph instantiation: ") + cudaGetErrorString(ei));
  }
  c->graph_steps = steps;
  c->graph_adam = optimizer == VQMC_OPT_ADAM;
  return VQMC_OK;
}

vqmc_status vqmc_graph_launch(vqmc_ctx* c, vqmc_stream stream, vqmc_step_stats* h_out) {
  if (!c) return fail(VQMC_ERR_INVALID_ARG, "null context");
  if (!c->graph) return fail(VQMC_ERR_INVALID_ARG, "no captured iterations (vqmc_graph_capture)");
  VQ_CUDA(cudaGraphLaunch(c->graph, S(stream)));
  c->iter += (uint64_t)c->graph_steps;
  if (c->graph_adam) c->adam_t += c->graph_steps;
  if (h_out) VQ_CUDA(cudaMemcpyAsync(h_out, c->step_stats, sizeof(vqmc_step_stats), cudaMemcpyDeviceToHost, S(stream)));
  return VQMC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches

struct vqmc_batch {
  std::vector<vqmc_ctx*> members;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;  // one per internal stream
  cudaEvent_t fork = nullptr;
  // schedule: internal streams in use (0 = all) and member -> stream (empty:
  // member i on stream i mod streams in use)
  int used = 0;
  std::vector<int> assign;
  // captured batched iterations (vqmc_batch_graph_capture)
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  // the last autotune's time of one iteration of each member alone (ms)
  std::vector<double> alone_ms;
};

namespace {

void batch_free(vqmc_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (vqmc_ctx* c : b->members) vqmc_destroy(c);
  for (cudaEvent_t e : b->done) cudaEventDestroy(e);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

}  // namespace

extern "C" {

vqmc_status vqmc_batch_create(const vqmc_config* cfgs, const vqmc_instance* insts, int32_t count,
                              vqmc_batch** out) {
  if (!cfgs || !insts || !out) return fail(VQMC_ERR_INVALID_ARG, "null argument");
  if (count < 1) return fail(VQMC_ERR_INVALID_ARG, "count must be >= 1");
  vqmc_batch* b = new vqmc_batch();
  for (int32_t i = 0; i < count; ++i) {
    vqmc_ctx* c = nullptr;
    const vqmc_status s = vqmc_create(&cfgs[i], &insts[i], &c);
    if (s != VQMC_OK) {
      const std::string msg = std::string("member ") + std::to_string(i) + ": " + vqmc_last_error();
      batch_free(b);
      return fail(s, msg);
    }
    b->members.push_back(c);
  }
  const int k = count < 8 ? count : 8;
  bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int q = 0; q < k && ok; ++q) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) b->streams.push_back(s);
    ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (ok) b->done.push_back(e);
  }
  if (!ok) {
    batch_free(b);
    return fail(VQMC_ERR_CUDA, "could not create the batch's streams");
  }
  *out = b;
  return VQMC_OK;
}

void vqmc_batch_destroy(vqmc_batch* b) {
  if (b) batch_free(b);
}

int32_t vqmc_batch_count(const vqmc_batch* b) { return b ? (int32_t)b->members.size() : 0; }

vqmc_ctx* vqmc_batch_member(vqmc_batch* b, int32_t i) {
  if (!b || i < 0 || i >= (int32_t)b->members.size()) return nullptr;
  return b->members[(size_t)i];
}

vqmc_status vqmc_batch_step(vqmc_batch* b, const int32_t* B, vqmc_stream stream, vqmc_step_stats* h_out) {
  if (!b || !B) return fail(VQMC_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = S(stream);
  VQ_CUDA(cudaEventRecord(b->fork, st));
  const size_t k = b->used > 0 ? (size_t)b->used : b->streams.size();
  for (size_t q = 0; q < k; ++q) VQ_CUDA(cudaStreamWaitEvent(b->streams[q], b->fork, 0));
  vqmc_status first = VQMC_OK;
  for (size_t i = 0; i < b->members.size() && first == VQMC_OK; ++i) {
    const size_t q = b->assign.empty() ? i % k : (size_t)b->assign[i];
    first = vqmc_step(b->members[i], B[i], (vqmc_stream)b->streams[q], h_out ? &h_out[i] : nullptr);
  }
  // join every internal stream back into the caller's, also after a failure
  for (size_t q = 0; q < k; ++q) {
    VQ_CUDA(cudaEventRecord(b->done[q], b->streams[q]));
    VQ_CUDA(cudaStreamWaitEvent(st, b->done[q], 0));
  }
  return first;
}

vqmc_status vqmc_batch_graph_capture(vqmc_batch* b, const int32_t* B, int32_t steps, vqmc_stream stream) {
  if (!b || !B) return fail(VQMC_ERR_INVALID_ARG, "null argument");
  if (steps < 1) return fail(VQMC_ERR_INVALID_ARG, "steps must be >= 1");
  if (!stream) return fail(VQMC_ERR_INVALID_ARG, "graph capture needs a stream other than the legacy default stream");
  for (size_t i = 0; i < b->members.size(); ++i) {
    vqmc_status s = check_B(b->members[i], B[i]);
    if (s != VQMC_OK) return s;
    if (B[i] == 0) return fail(VQMC_ERR_INVALID_ARG, "every member needs B >= 1");
  }
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_steps = 0;
  }
  const size_t m = b->members.size();
  std::vector<uint64_t> it0(m);
  std::vector<int64_t> t0(m);
  std::vector<char> timing(m);
  for (size_t i = 0; i < m; ++i)
    it0[i] = b->members[i]->iter, t0[i] = b->members[i]->adam_t, timing[i] = b->members[i]->timing;
  cudaStream_t st = S(stream);
  VQ_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  for (size_t i = 0; i < m; ++i) b->members[i]->timing = false;  // no timing events inside the graph
  vqmc_status s = VQMC_OK;
  for (int q = 0; q < steps && s == VQMC_OK; ++q) s = vqmc_batch_step(b, B, stream, nullptr);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  for (size_t i = 0; i < m; ++i)
    b->members[i]->iter = it0[i], b->members[i]->adam_t = t0[i], b->members[i]->timing = timing[i] != 0;
  if (s != VQMC_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return s != VQMC_OK ? s : fail(VQMC_ERR_CUDA, std::string("stream capture: ") + cudaGetErrorString(e));
  }
  const cudaError_t ei = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    b->graph = nullptr;
    return fail(VQMC_ERR_CUDA, std::string("graph instantiation: ") + cudaGetErrorString(ei));
  }
  b->graph_steps = steps;
  return VQMC_OK;
}

vqmc_status vqmc_batch_graph_launch(vqmc_batch* b, vqmc_stream stream, vqmc_step_stats* h_out) {
  if (!b) return fail(VQMC_ERR_INVALID_ARG, "null batch");
  if (!b->graph) return fail(VQMC_ERR_INVALID_ARG, "no captured iterations (vqmc_batch_graph_capture)");
  VQ_CUDA(cudaGraphLaunch(b->graph, S(stream)));
  for (size_t i = 0; i < b->members.size(); ++i) {
    vqmc_ctx* c = b->members[i];
    c->iter += (uint64_t)b->graph_steps;
    c->adam_t += b->graph_steps;
    if (h_out)
      VQ_CUDA(cudaMemcpyAsync(&h_out[i], c->step_stats, sizeof(vqmc_step_stats), cudaMemcpyDeviceToHost, S(stream)));
  }
  return VQMC_OK;
}

namespace {

// device milliseconds of `reps` launches of the batch's graph on st
vqmc_status time_batch_graph(vqmc_batch* b, cudaStream_t st, int reps, double* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  VQ_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(VQMC_ERR_CUDA, "event creation failed");
  }
  vqmc_status s = VQMC_OK;
  cudaError_t e = cudaEventRecord(e0, st);
  for (int r = 0; r < reps && s == VQMC_OK && e == cudaSuccess; ++r) s = vqmc_batch_graph_launch(b, st, nullptr);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float f = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&f, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != VQMC_OK) return s;
  if (e != cudaSuccess) return fail(VQMC_ERR_CUDA, std::string("timing: ") + cudaGetErrorString(e));
  *ms = (double)f / reps;
  return VQMC_OK;
}

}  // namespace

vqmc_status vqmc_batch_autotune(vqmc_batch* b, const int32_t* B, vqmc_stream stream, int32_t* streams_out,
                                double* ms_out) {
  if (!b || !B) return fail(VQMC_ERR_INVALID_ARG, "null argument");
  if (!stream) return fail(VQMC_ERR_INVALID_ARG, "autotuning captures graphs: pass a non-default stream");
  cudaStream_t st = S(stream);
  const size_t m = b->members.size();
  // 1. cost of one iteration of each member alone (after one warm-up step),
  // and for a member on the CUDA-core sampler up to 2048 hidden units the
  // faster of its two layouts (16 samples per CTA, or the wide one: groups of
  // four warps, 4 samples per CTA)
  std::vector<double> cost(m, 0.0);
  {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    VQ_CUDA(cudaEventCreate(&e0));
    VQ_CUDA(cudaEventCreate(&e1));
    vqmc_status s = VQMC_OK;
    auto time_alone = [&](size_t i, float* f) {
      s = vqmc_step(b->members[i], B[i], stream, nullptr);
      if (s == VQMC_OK && cudaEventRecord(e0, st) != cudaSuccess) s = fail(VQMC_ERR_CUDA, "event record failed");
      if (s == VQMC_OK) s = vqmc_step(b->members[i], B[i], stream, nullptr);
      if (s == VQMC_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
        s = fail(VQMC_ERR_CUDA, "event timing failed");
      *f = 0.0f;
      if (s == VQMC_OK) cudaEventElapsedTime(f, e0, e1);
    };
    for (size_t i = 0; i < m && s == VQMC_OK; ++i) {
      vqmc_ctx* c = b->members[i];
      float f = 0.0f;
      time_alone(i, &f);
      cost[i] = f;
      const bool other = c->sampler == VQMC_SAMPLER_CUDA_CORE && c->hp <= 2048 &&
                         (c->prec == VQMC_PREC_BF16 ? sampler_wt_supports<bf16>(c->hp, !c->sampler_wide)
                                                    : sampler_wt_supports<float>(c->hp, !c->sampler_wide));
      if (s == VQMC_OK && other) {
        c->sampler_wide ^= 1;
        time_alone(i, &f);
        if (s == VQMC_OK && f < cost[i]) cost[i] = f;
        else c->sampler_wide ^= 1;
      } else if (s == VQMC_OK) {
        time_alone(i, &f);  // every member advances by the same number of iterations
        if (s == VQMC_OK && f < cost[i]) cost[i] = f;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != VQMC_OK) return s;
  }
  b->alone_ms = cost;
  // 2. candidate schedules: 1, 2, 4, 8 streams (up to the batch's), members
  // round-robin in index order or longest-first onto the least-loaded stream
  std::vector<size_t> order(m);
  for (size_t i = 0; i < m; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
  double best = -1.0;
  int best_used = 1;
  std::vector<int> best_assign;
  const int smax = (int)b->streams.size();
  std::vector<int> counts;
  for (int S = 1; S < smax; S *= 2) counts.push_back(S);
  counts.push_back(smax);
  for (int S : counts) {
    for (int lpt = 0; lpt < (S > 1 ? 2 : 1); ++lpt) {
      std::vector<int> assign(m);
      if (lpt) {
        std::vector<double> load(S, 0.0);
        for (size_t i : order) {
          const int q = (int)(std::min_element(load.begin(), load.end()) - load.begin());
          assign[i] = q;
          load[q] += cost[i];
        }
      } else {
        for (size_t i = 0; i < m; ++i) assign[i] = (int)(i % S);
      }
      b->used = S, b->assign = assign;
      vqmc_status s = vqmc_batch_graph_capture(b, B, 1, stream);
      double ms = 0.0;
      if (s == VQMC_OK) s = time_batch_graph(b, st, 1, &ms);  // warm-up
      if (s == VQMC_OK) s = time_batch_graph(b, st, 3, &ms);
      if (s != VQMC_OK) return s;
      if (best < 0.0 || ms < best) best = ms, best_used = S, best_assign = assign;
    }
  }
  // 3. keep the fastest schedule and its graph
  b->used = best_used, b->assign = best_assign;
  vqmc_status s = vqmc_batch_graph_capture(b, B, 1, stream);
  if (s != VQMC_OK) return s;
  if (streams_out) *streams_out = best_used;
  if (ms_out) *ms_out = best;
  return VQMC_OK;
}

vqmc_status vqmc_batch_schedule(const vqmc_batch* b, int32_t* streams_used, int32_t* member_stream,
                                int32_t* member_sampler, double* member_ms) {
  if (!b) return fail(VQMC_ERR_INVALID_ARG, "null batch");
  const size_t m = b->members.size();
  const size_t k = b->used > 0 ? (size_t)b->used : b->streams.size();
  if (streams_used) *streams_used = (int32_t)k;
  for (size_t i = 0; i < m; ++i) {
    const vqmc_ctx* c = b->members[i];
    if (member_stream) member_stream[i] = (int32_t)(b->assign.empty() ? i % k : (size_t)b->assign[i]);
    if (member_sampler)
      member_sampler[i] = c->sampler == VQMC_SAMPLER_TENSOR_CORE ? VQMC_SAMPLER_TENSOR_CORE
                          : c->sampler_wide                      ? VQMC_SAMPLER_CUDA_CORE_WIDE
                                                                 : VQMC_SAMPLER_CUDA_CORE;
    if (member_ms) member_ms[i] = i < b->alone_ms.size() ? b->alone_ms[i] : 0.0;
  }
  return VQMC_OK;
}

vqmc_status vqmc_timing_enable(vqmc_ctx* c, int enable) {
  if (!c) return fail(VQMC_ERR_INVALID_ARG, "null context");
  if (enable && !c->events) {
    c->events = new cudaEvent_t[(size_t)kMaxTimedSteps * (VQMC_NUM_PARTS + 1)];
    for (int64_t q = 0; q < kMaxTimedSteps * (VQMC_NUM_PARTS + 1); ++q) VQ_CUDA(cudaEventCreate(&c->events[q]));
  }
  c->timing = enable != 0;
  c->timed_steps = 0;
  c->launches = 0;
  return VQMC_OK;
}

vqmc_status vqmc_timing_read(vqmc_ctx* c, double* ms_out, int64_t* steps_out, int64_t* launches_out) {
  if (!c) return fail(VQMC_ERR_INVALID_ARG, "null context");
  double acc[VQMC_NUM_PARTS] = {0};
  for (int64_t t = 0; t < c->timed_steps; ++t) {
    cudaEvent_t* ev = c->events + t * (VQMC_NUM_PARTS + 1);
    VQ_CUDA(cudaEventSynchronize(ev[VQMC_NUM_PARTS]));
    for (int p = 0; p < VQMC_NUM_PARTS; ++p) {
      float ms = 0.0f;
      VQ_CUDA(cudaEventElapsedTime(&ms, ev[p], ev[p + 1]));
      acc[p] += ms;
    }
  }
  if (ms_out)
    for (int p = 0; p < VQMC_NUM_PARTS; ++p) ms_out[p] = acc[p];
  if (steps_out) *steps_out = c->timed_steps;
  if (launches_out) *launches_out = c->launches;
  return VQMC_OK;
}

vqmc_status vqmc_last_batch(vqmc_ctx* c, const int8_t** d_s, const void** d_e) {
  if (!c) return fail(VQMC_ERR_INVALID_ARG, "null context");
  if (d_s) *d_s = c->S;
  if (d_e) *d_e = c->E;
  return VQMC_OK;
}

vqmc_status vqmc_check(vqmc_ctx* c, uint32_t* flags_out) {
  if (!c) return fail(VQMC_ERR_INVALID_ARG, "null context");
  VQ_CUDA(cudaDeviceSynchronize());
  uint32_t f = 0;
  VQ_CUDA(cudaMemcpy(&f, c->err, 4, cudaMemcpyDeviceToHost));
  VQ_CUDA(cudaMemset(c->err, 0, 4));
  if (flags_out) *flags_out = f;
  if (f & VQMC_DEVERR_TIMEOUT) return fail(VQMC_ERR_TIMEOUT, "a bounded device wait gave up");
  if (f & VQMC_DEVERR_NONFINITE) return fail(VQMC_ERR_NONFINITE, "non-finite energy statistics");
  return VQMC_OK;
}

// Checkpoint file: header, then theta, Adam m, Adam v (d floats each).
struct CkptHeader {
  char magic[8];
  uint32_t version;
  int32_t n, h, act;
  int64_t d;
  int64_t adam_t;
  uint64_t iter;
  uint64_t seed;
  uint64_t inst_hash;
};

vqmc_status vqmc_save(vqmc_ctx* c, const char* path) {
  if (!c || !path) return fail(VQMC_ERR_INVALID_ARG, "null argument");
  VQ_CUDA(cudaDeviceSynchronize());
  CkptHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, "VQMCCKP1", 8);
  hd.version = 1;
  hd.n = c->n, hd.h = c->h, hd.act = c->act, hd.d = c->d;
  hd.adam_t = c->adam_t, hd.iter = c->iter, hd.seed = c->cfg.seed, hd.inst_hash = c->inst_hash;
  std::vector<float> buf((size_t)c->d);
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(VQMC_ERR_INVALID_ARG, std::string("cannot open ") + path);
  bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1;
  float* arrs[3] = {c->theta, c->adam_m, c->adam_v};
  for (float* a : arrs) {
    if (!ok) break;
    if (cudaMemcpy(buf.data(), a, c->d * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
      std::fclose(f);
      return fail(VQMC_ERR_CUDA, "checkpoint copy failed");
    }
    ok = std::fwrite(buf.data(), 4, buf.size(), f) == buf.size();
  }
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(VQMC_ERR_INVALID_ARG, "checkpoint write failed");
  return VQMC_OK;
}

vqmc_status vqmc_load(vqmc_ctx* c, const char* path) {
  if (!c || !path) return fail(VQMC_ERR_INVALID_ARG, "null argument");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(VQMC_ERR_INVALID_ARG, std::string("cannot open ") + path);
  CkptHeader hd;
  if (std::fread(&hd, sizeof(hd), 1, f) != 1 || std::memcmp(hd.magic, "VQMCCKP1", 8) != 0 || hd.version != 1) {
    std::fclose(f);
    return fail(VQMC_ERR_INVALID_ARG, "not a vqmc checkpoint");
  }
  if (hd.n != c->n || hd.h != c->h || hd.act != c->act || hd.d != c->d || hd.inst_hash != c->inst_hash) {
    std::fclose(f);
    return fail(VQMC_ERR_INVALID_ARG, "checkpoint does not match this context (shape, activation or instance)");
  }
  std::vector<float> buf((size_t)c->d);
  float* arrs[3] = {c->theta, c->adam_m, c->adam_v};
  for (float* a : arrs) {
    if (std::fread(buf.data(), 4, buf.size(), f) != buf.size()) {
      std::fclose(f);
      return fail(VQMC_ERR_INVALID_ARG, "truncated checkpoint");
    }
    if (cudaMemcpy(a, buf.data(), c->d * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
      std::fclose(f);
      return fail(VQMC_ERR_CUDA, "checkpoint copy failed");
    }
  }
  std::fclose(f);
  c->adam_t = hd.adam_t;
  c->iter = hd.iter;
  c->cfg.seed = hd.seed;
  VQ_CUDA(launch_set_state(c, 0));
  VQ_CUDA(launch_refresh_weights(c, 0));
  VQ_CUDA(cudaDeviceSynchronize());
  return VQMC_OK;
}

}  // extern "C"
