// Off-diagonal local energy of the transverse-field Ising model.
//
// The X_i terms of Eq. (hamiltonian) join x to the n states x^(i) that differ
// from x in spin i only (H_{x, x^(i)} = -alpha_i, Eq. (e:tim)), so with
// psi = sqrt(pi) (Sec. 2.1) they add
//     E_off(x) = -sum_i alpha_i exp((log pi(x^(i)) - log pi(x)) / 2)
// to the local energy.  Every sample expands into n + 1 rows (its n flipped
// states and itself, row g = b (n + 1) + i, i = n the sample itself).
// Flipping spin i changes each hidden pre-activation by a rank-1 term,
//     a_k(x^(i)) = a_k(x) - 2 s_i W1_ki        (zero unless i < m(k)),
// so one hidden GEMM over the B samples gives a(x) in FP32, an elementwise
// kernel builds the hidden activations of every row from it and W1, and only
// the output layer runs as a GEMM over the rows (chunks of rows; log sigma(s z)
// partial sums per 128-column tile in its epilogue).  The outputs before spin
// i see the same units in both rows, so their terms cancel in
// log pi(x^(i)) - log pi(x): the GEMM skips the tiles that lie before the
// flipped spin of all its rows, and the log-ratio is summed from the partials
// of the remaining tiles (one warp per sample).
#include "gemm.cuh"

namespace vqmc {
namespace {

// Rows per chunk: as many as fit in about 256 MB of row workspace (the
// hidden activations and spins of a row), between 32,768 and 131,072, a
// multiple of 128; fewer chunks mean fewer dependent launches.
constexpr long long kChunkBytes = 256ll << 20;
constexpr int kMinChunkRows = 32768, kMaxChunkRows = 131072;

template <typename T>
__device__ __forceinline__ T to_t(float x);
template <>
__device__ __forceinline__ float to_t<float>(float x) { return x; }
template <>
__device__ __forceinline__ bf16 to_t<bf16>(float x) { return __float2bfloat16_rn(x); }

template <typename T>
__device__ __forceinline__ float weight(float w);  // the model's weight as the kernels use it
template <>
__device__ __forceinline__ float weight<float>(float w) { return w; }
template <>
__device__ __forceinline__ float weight<bf16>(float w) { return __bfloat162float(__float2bfloat16_rn(w)); }

// Rows [g0, g0 + rows) of the expansion, one warp per row: the hidden
// activations act(a(x) - 2 s_i W1_:,i) (the output GEMM's operand, padding
// zero; the BF16 model rounds them to BF16 like every hidden activation) and
// the row's spins as int8 for the output epilogue's signs, 8 activations and
// 16 spins per lane and 16-byte store.  A: a(x) [B][hp] FP32; W1t: the
// master W1^T [n][h] (FP32; rounded to BF16 for the BF16 model).  hp and np
// are multiples of 64.
template <typename T>
__device__ __forceinline__ void store8(T* p, const float (&x)[8]);
template <>
__device__ __forceinline__ void store8<float>(float* p, const float (&x)[8]) {
  reinterpret_cast<float4*>(p)[0] = make_float4(x[0], x[1], x[2], x[3]);
  reinterpret_cast<float4*>(p)[1] = make_float4(x[4], x[5], x[6], x[7]);
}
template <>
__device__ __forceinline__ void store8<bf16>(bf16* p, const float (&x)[8]) {
  uint32_t w[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
    w[q] = *reinterpret_cast<const uint32_t*>(&v);
  }
  *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}

template <typename T>
__global__ void tim_rows_kernel(int n, int h, int hp, int np, int act, long long g0, int rows,
                                const int8_t* __restrict__ S, const float* __restrict__ A,
                                const float* __restrict__ W1t, T* __restrict__ H, int8_t* __restrict__ S8) {
  const int r = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (r >= rows) return;
  const long long g = g0 + r;
  const long long b = g / (n + 1);
  const int i = (int)(g - b * (n + 1));
  const int8_t* src = S + b * n;
  const float* a0 = A + b * hp;
  const float two_s = i < n ? 2.0f * (float)src[i] : 0.0f;
  const float* wrow = W1t + (size_t)(i < n ? i : 0) * h;
  T* dh = H + (size_t)r * hp;
  for (int k0 = 8 * lane; k0 < hp; k0 += 256) {
    const float4 p0 = reinterpret_cast<const float4*>(a0 + k0)[0], p1 = reinterpret_cast<const float4*>(a0 + k0)[1];
    const float av[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
    float x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = k0 + e;
      x[e] = 0.0f;
      if (k < h) {
        const float a = i < n ? av[e] - two_s * weight<T>(wrow[k]) : av[e];
        x[e] = act == VQMC_ACT_RELU ? fmaxf(a, 0.0f) : 1.0f / (1.0f + expf(-a));
      }
    }
    store8<T>(dh + k0, x);
  }
  int8_t* d8 = S8 + (size_t)r * np;
  for (int k0 = 16 * lane; k0 < np; k0 += 512) {
    uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int k = k0 + e;
      int v = k < n ? src[k] : 0;
      if (k == i) v = -v;
      w[e >> 2] |= (uint32_t)(uint8_t)(int8_t)v << (8 * (e & 3));
    }
    *reinterpret_cast<uint4*>(d8 + k0) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// E[b] -= sum_i alpha_i exp(Delta_i / 2) with
//     Delta_i = log pi(x^(i)) - log pi(x) = sum_{t >= i / 128} (P[t][b, i] - P[t][b, n]),
// P[t][row] the output GEMM's partial log pi over columns [128 t, 128 t + 128):
// the terms of the columns before spin i are the same in both rows.  One warp
// per sample, FP64 terms, fixed reduction order.
__global__ void tim_offdiag_kernel(int B, int n, int ntiles, const float* __restrict__ P, long long ld,
                                   const float* __restrict__ alpha, float* __restrict__ E) {
  const int b = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (b >= B) return;
  const long long base = (long long)b * (n + 1), r0 = base + n;
  double acc = 0.0;
  for (int i = lane; i < n; i += 32) {
    double d = 0.0;
    for (int t = i / 128; t < ntiles; ++t) d += (double)P[t * ld + base + i] - (double)P[t * ld + r0];
    acc += (double)alpha[i] * exp(0.5 * d);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) E[b] = (float)((double)E[b] - acc);
}

// The hidden GEMM of the B samples (FP32 pre-activations into tim_A; the
// activations go to the step's H workspace, unused here), or the output GEMM
// of a chunk of `rows` rows.
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
    a.A = (const T*)c->Sx, a.lda = c->np;
    a.Bm = (const T*)c->w_s, a.ldb = c->np;
    a.bias = c->b1;
    a.out = (T*)c->H, a.ldo = c->hp;  // no transposed copy
    a.pre = c->tim_A, a.ldpre = c->hp;
  } else {
    a.N = c->n, a.K = c->h;
    a.A = (const T*)c->tim_H, a.lda = c->hp;
    a.Bm = (const T*)c->v_s, a.ldb = c->hp;
    a.bias = c->b2;
    a.S8 = c->tim_S8, a.lds8 = c->np;
    a.ldr = (int)c->tim_ld;  // row_part and row0 are set per chunk
    a.flip_rows = 1;
  }
  return a;
}

template <typename T>
cudaError_t chunk_gemm(const vqmc_ctx* c, GemmOp op, int rows, long long g0, cudaStream_t st);
template <>
cudaError_t chunk_gemm<bf16>(const vqmc_ctx* c, GemmOp op, int rows, long long g0, cudaStream_t st) {
  GemmArgs<bf16> a = chunk_args<bf16>(c, op, rows);
  a.row_part = c->tim_row_part + g0, a.row0 = g0;
  return launch_gemm_tc_bf16(a, st);
}
template <>
cudaError_t chunk_gemm<float>(const vqmc_ctx* c, GemmOp op, int rows, long long g0, cudaStream_t st) {
  GemmArgs<float> a = chunk_args<float>(c, op, rows);
  a.row_part = c->tim_row_part + g0, a.row0 = g0;
  return launch_gemm_simt_f32(a, st);
}

template <typename T>
cudaError_t offdiag(const vqmc_ctx* c, int B, const int8_t* d_s, float* d_e, cudaStream_t st, int* launches) {
  const int n = c->n;
  const long long total = (long long)B * (n + 1);
  const int ntiles = (n + 127) / 128;
  // a(x) of the B samples
  cudaError_t e = launch_spins_to_operands(c, B, d_s, c->Sx, nullptr, st);
  if (e == cudaSuccess) e = chunk_gemm<T>(c, kOpHidden, B, 0, st);
  if (e != cudaSuccess) return e;
  int count = 2;
  for (long long g0 = 0; g0 < total; g0 += c->tim_rows) {
    const int rows = (int)(total - g0 < c->tim_rows ? total - g0 : c->tim_rows);
    tim_rows_kernel<T><<<(rows + 7) / 8, 256, 0, st>>>(n, c->h, c->hp, c->np, c->act, g0, rows, d_s, c->tim_A,
                                                       c->theta, (T*)c->tim_H, c->tim_S8);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = chunk_gemm<T>(c, kOpOut, rows, g0, st);
    if (e != cudaSuccess) return e;
    count += 2;
  }
  tim_offdiag_kernel<<<(B + 7) / 8, 256, 0, st>>>(B, n, ntiles, c->tim_row_part, c->tim_ld, c->alpha, d_e);
  if (launches) *launches = count + 1;
  return cudaGetLastError();
}

}  // namespace

int tim_chunk_rows(int Bmax, int n, int hp, int np, int esize) {
  const long long total = (long long)Bmax * (n + 1);
  const long long r = (total + 127) / 128 * 128;
  long long cap = kChunkBytes / ((long long)hp * esize + np) / 128 * 128;
  cap = cap < kMinChunkRows ? kMinChunkRows : (cap > kMaxChunkRows ? kMaxChunkRows : cap);
  return (int)(r < cap ? r : cap);
}

cudaError_t launch_tim_offdiag(const vqmc_ctx* c, int B, const int8_t* d_s, float* d_e, cudaStream_t st,
                               int* launches) {
  if (launches) *launches = 0;
  if (B <= 0 || !c->alpha) return cudaSuccess;
  return c->prec == VQMC_PREC_BF16 ? offdiag<bf16>(c, B, d_s, d_e, st, launches)
                                   : offdiag<float>(c, B, d_s, d_e, st, launches);
}

}  // namespace vqmc
