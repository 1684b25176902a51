// Off-diagonal local energy of the transverse-field Ising model.
//
// The X_i terms of Eq. (hamiltonian) join x to the n states x^(i) that differ
// from x in spin i only (H_{x, x^(i)} = -alpha_i, Eq. (e:tim)), so with
// psi = sqrt(pi) (Sec. 2.1) they add
//     E_off(x) = -sum_i alpha_i exp((log pi(x^(i)) - log pi(x)) / 2)
// to the local energy.  Every sample expands into n + 1 rows (its n flipped
// states and itself, row g = b (n + 1) + i, i = n the sample itself); the
// rows run in chunks through the model's two log-prob GEMMs (hidden layer,
// then output layer with the log sigma(s z) row sums in the epilogue), and
// one warp per sample forms the sum.  Rows of one sample differ only from
// spin i on, so the terms of the outputs before i agree bit for bit and the
// difference of two row sums carries only FP32 rounding of the sums.
#include "gemm.cuh"

namespace vqmc {
namespace {

constexpr int kMaxChunkRows = 32768;  // multiple of 128

template <typename T>
__device__ __forceinline__ T from_spin(int v);
template <>
__device__ __forceinline__ float from_spin<float>(int v) { return (float)v; }
template <>
__device__ __forceinline__ bf16 from_spin<bf16>(int v) { return __float2bfloat16_rn((float)v); }

// Rows [g0, g0 + rows) of the expansion, one warp per row: the sample's
// spins with spin i negated, as the GEMM operand Sx (padding zero) and as
// int8 S8 for the output epilogue's signs.
template <typename T>
__global__ void tim_flip_kernel(int n, int np, long long g0, int rows, const int8_t* __restrict__ S,
                                T* __restrict__ Sx, int8_t* __restrict__ S8) {
  const int r = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (r >= rows) return;
  const long long g = g0 + r;
  const long long b = g / (n + 1);
  const int i = (int)(g - b * (n + 1));
  const int8_t* src = S + b * n;
  T* dx = Sx + (size_t)r * np;
  int8_t* d8 = S8 + (size_t)r * np;
  for (int k = lane; k < np; k += 32) {
    int v = k < n ? src[k] : 0;
    if (k == i) v = -v;
    d8[k] = (int8_t)v;
    dx[k] = from_spin<T>(v);
  }
}

// log pi of each row of the chunk: the sum of the output GEMM's tile
// partials in a fixed order.
__global__ void tim_rowsum_kernel(int rows, int ntiles, const float* __restrict__ part, int ld,
                                  float* __restrict__ lp) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  float s = 0.0f;
  for (int t = 0; t < ntiles; ++t) s += part[(size_t)t * ld + r];
  lp[r] = s;
}

// E[b] -= sum_i alpha_i exp((lp[b][i] - lp[b][n]) / 2), one warp per sample,
// FP64 terms and a fixed reduction order.
__global__ void tim_offdiag_kernel(int B, int n, const float* __restrict__ lp, const float* __restrict__ alpha,
                                   float* __restrict__ E) {
  const int b = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (b >= B) return;
  const float* l = lp + (size_t)b * (n + 1);
  const double l0 = (double)l[n];
  double acc = 0.0;
  for (int i = lane; i < n; i += 32) acc += (double)alpha[i] * exp(0.5 * ((double)l[i] - l0));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) E[b] = (float)((double)E[b] - acc);
}

// The two log-prob GEMMs of a chunk of `rows` rows.
template <typename T>
GemmArgs<T> chunk_args(const vqmc_ctx* c, GemmOp op, int rows) {
  GemmArgs<T> a{};
  a.op = op;
  a.n = c->n;
  a.h = c->h;
  a.act = c->act;
  a.err = c->err;
  a.M = rows;
  if (op == kOpHidden) {
    a.N = c->h, a.K = c->n;
    a.A = (const T*)c->tim_Sx, a.lda = c->np;
    a.Bm = (const T*)c->w_s, a.ldb = c->np;
    a.bias = c->b1;
    a.out = (T*)c->tim_H, a.ldo = c->hp;  // no transposed copy
  } else {
    a.N = c->n, a.K = c->h;
    a.A = (const T*)c->tim_H, a.lda = c->hp;
    a.Bm = (const T*)c->v_s, a.ldb = c->hp;
    a.bias = c->b2;
    a.S8 = c->tim_S8, a.lds8 = c->np;
    a.row_part = c->tim_row_part, a.ldr = c->tim_rows;
  }
  return a;
}

template <typename T>
cudaError_t chunk_gemm(const vqmc_ctx* c, GemmOp op, int rows, cudaStream_t st);
template <>
cudaError_t chunk_gemm<bf16>(const vqmc_ctx* c, GemmOp op, int rows, cudaStream_t st) {
  return launch_gemm_tc_bf16(chunk_args<bf16>(c, op, rows), st);
}
template <>
cudaError_t chunk_gemm<float>(const vqmc_ctx* c, GemmOp op, int rows, cudaStream_t st) {
  return launch_gemm_simt_f32(chunk_args<float>(c, op, rows), st);
}

template <typename T>
cudaError_t offdiag(const vqmc_ctx* c, int B, const int8_t* d_s, float* d_e, cudaStream_t st, int* launches) {
  const int n = c->n;
  const long long total = (long long)B * (n + 1);
  const int ntiles = (n + 127) / 128;
  int count = 0;
  for (long long g0 = 0; g0 < total; g0 += c->tim_rows) {
    const int rows = (int)(total - g0 < c->tim_rows ? total - g0 : c->tim_rows);
    tim_flip_kernel<T><<<(rows + 7) / 8, 256, 0, st>>>(n, c->np, g0, rows, d_s, (T*)c->tim_Sx, c->tim_S8);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = chunk_gemm<T>(c, kOpHidden, rows, st);
    if (e == cudaSuccess) e = chunk_gemm<T>(c, kOpOut, rows, st);
    if (e != cudaSuccess) return e;
    tim_rowsum_kernel<<<(rows + 255) / 256, 256, 0, st>>>(rows, ntiles, c->tim_row_part, c->tim_rows,
                                                         c->tim_lp + g0);
    count += 4;
  }
  tim_offdiag_kernel<<<(B + 7) / 8, 256, 0, st>>>(B, n, c->tim_lp, c->alpha, d_e);
  if (launches) *launches = count + 1;
  return cudaGetLastError();
}

}  // namespace

int tim_chunk_rows(int Bmax, int n) {
  const long long total = (long long)Bmax * (n + 1);
  const long long r = (total + 127) / 128 * 128;
  return (int)(r < kMaxChunkRows ? r : kMaxChunkRows);
}

cudaError_t launch_tim_offdiag(const vqmc_ctx* c, int B, const int8_t* d_s, float* d_e, cudaStream_t st,
                               int* launches) {
  if (launches) *launches = 0;
  if (B <= 0 || !c->alpha) return cudaSuccess;
  return c->prec == VQMC_PREC_BF16 ? offdiag<bf16>(c, B, d_s, d_e, st, launches)
                                   : offdiag<float>(c, B, d_s, d_e, st, launches);
}

}  // namespace vqmc
