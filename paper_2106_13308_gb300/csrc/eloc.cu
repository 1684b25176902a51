// Local energy (Sec. 2.1, Sec. 2.4), FP64 batch statistics (Eq. (e:vmc),
// Eq. (eq:stochastic_variance)) and spin-layout conversions.
//
// Sparse local energy.  For a diagonal Hamiltonian l(s) = H_ss =
// sum_{i<j} J_ij s_i s_j + sum_i h_i s_i.  One CTA handles 32 samples: it first
// packs their spins bit-transposed into shared memory (bits[i] bit l = [s_i of
// sample l is -1]), so one 32-bit xor of two words gives the sign of s_i s_j
// for all 32 samples; then the warps split the CSR rows and lane l
// accumulates sample l.  Integer weights accumulate in int32 (exact).
#include "common.cuh"

namespace vqmc {
namespace {

constexpr int kElocWarps = 8;

template <typename W, typename A>
__global__ void __launch_bounds__(kElocWarps * 32) eloc_sparse_kernel(int B, int n, const int8_t* __restrict__ S,
                                                                      const int32_t* __restrict__ row_ptr,
                                                                      const int32_t* __restrict__ col,
                                                                      const W* __restrict__ w,
                                                                      const W* __restrict__ field, A* __restrict__ E) {
  extern __shared__ uint32_t bits[];  // [n]
  __shared__ A red[kElocWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b0 = blockIdx.x * 32;
  const int b = b0 + lane;
  const int8_t* row = S + (size_t)(b < B ? b : b0) * n;
  for (int i = warp; i < n; i += kElocWarps) {
    const bool neg = b < B && __ldg(row + i) < 0;
    const uint32_t m = __ballot_sync(0xffffffffu, neg);
    if (lane == 0) bits[i] = m;
  }
  __syncthreads();
  A e = 0;
  for (int i = warp; i < n; i += kElocWarps) {
    const uint32_t bi = bits[i];
    if (field) {
      const A f = (A)__ldg(field + i);
      e += ((bi >> lane) & 1u) ? -f : f;
    }
    const int p1 = __ldg(row_ptr + i + 1);
    for (int p = __ldg(row_ptr + i); p < p1; ++p) {
      const uint32_t x = bi ^ bits[__ldg(col + p)];
      const A wt = (A)__ldg(w + p);
      e += ((x >> lane) & 1u) ? -wt : wt;
    }
  }
  red[warp][lane] = e;
  __syncthreads();
  if (warp == 0 && b < B) {
    A t = red[0][lane];
#pragma unroll
    for (int q = 1; q < kElocWarps; ++q) t += red[q][lane];
    E[b] = t;
  }
}

// E_b = sum over N-tiles of the GEMM's row partials (1/2 s^T J s) + h.s
__global__ void eloc_dense_finish_kernel(int B, int n, int ntiles, const float* __restrict__ part, int ld,
                                         const int8_t* __restrict__ S, const float* __restrict__ field,
                                         float* __restrict__ E) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float e = 0.0f;
  for (int t = 0; t < ntiles; ++t) e += part[(size_t)t * ld + b];
  if (field) {
    const int8_t* s = S + (size_t)b * n;
    for (int i = 0; i < n; ++i) e += s[i] > 0 ? field[i] : -field[i];
  }
  E[b] = e;
}

// FP64 statistics of B energies in one CTA with a fixed reduction order.
template <typename A>
__global__ void __launch_bounds__(1024) stats_kernel(int B, const A* __restrict__ E, double* __restrict__ out,
                                                     float* __restrict__ coef, uint32_t* __restrict__ err) {
  __shared__ double s_sum[1024], s_min[1024], s_max[1024];
  __shared__ double s_mean;
  const int t = threadIdx.x;
  double sum = 0.0, mn = 1.0 / 0.0, mx = -1.0 / 0.0;
  for (int b = t; b < B; b += 1024) {
    const double x = (double)E[b];
    sum += x;
    mn = fmin(mn, x);
    mx = fmax(mx, x);
  }
  s_sum[t] = sum;
  s_min[t] = mn;
  s_max[t] = mx;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (t < o) {
      s_sum[t] += s_sum[t + o];
      s_min[t] = fmin(s_min[t], s_min[t + o]);
      s_max[t] = fmax(s_max[t], s_max[t + o]);
    }
    __syncthreads();
  }
  if (t == 0) s_mean = s_sum[0] / (double)B;
  __syncthreads();
  const double mean = s_mean;
  double ss = 0.0;
  for (int b = t; b < B; b += 1024) {
    const double d = (double)E[b] - mean;
    ss += d * d;
  }
  __syncthreads();
  s_sum[t] = ss;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (t < o) s_sum[t] += s_sum[t + o];
    __syncthreads();
  }
  if (t == 0) {
    const double var = s_sum[0] / (double)B;
    out[0] = mean;
    out[1] = var;
    out[2] = s_min[0];
    out[3] = s_max[0];
    if (!isfinite(mean) || !isfinite(var)) atomicOr(err, kErrNonfinite);
  }
  if (coef)
    for (int b = t; b < B; b += 1024) coef[b] = (float)(((double)E[b] - mean) / (double)B);
}

template <typename T>
__device__ __forceinline__ T spin_val(int8_t s);
template <>
__device__ __forceinline__ float spin_val<float>(int8_t s) { return s > 0 ? 1.0f : -1.0f; }
template <>
__device__ __forceinline__ bf16 spin_val<bf16>(int8_t s) { return __float2bfloat16_rn(s > 0 ? 1.0f : -1.0f); }

// int8 [B][n] -> T [B][ldx] and T [n][ldt] (transposed through a 32x32 tile)
template <typename T>
__global__ void spins_convert_kernel(int B, int n, const int8_t* __restrict__ S, T* __restrict__ Sx, int ldx,
                                     T* __restrict__ St, int ldt) {
  __shared__ int8_t tile[32][33];
  const int i0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int b = b0 + r, i = i0 + tx;
    int8_t v = 1;
    if (b < B && i < n) {
      v = S[(size_t)b * n + i];
      if (Sx) Sx[(size_t)b * ldx + i] = spin_val<T>(v);
    }
    tile[r][tx] = v;
  }
  __syncthreads();
  if (!St) return;
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r, b = b0 + tx;
    if (i < n && b < B) St[(size_t)i * ldt + b] = spin_val<T>(tile[tx][r]);
  }
}

__global__ void tile_sum_kernel(int cnt, int ntiles, const float* __restrict__ part, int ld, float* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= cnt) return;
  float s = 0.0f;
  for (int t = 0; t < ntiles; ++t) s += part[(size_t)t * ld + q];
  out[q] = s;
}

}  // namespace

cudaError_t launch_eloc_sparse(const vqmc_ctx* c, int B, const int8_t* d_s, void* d_e, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  const size_t smem = (size_t)c->n * sizeof(uint32_t);
  const int grid = (B + 31) / 32;
  if (c->ham == VQMC_HAM_SPARSE_I32) {
    auto k = eloc_sparse_kernel<int32_t, int32_t>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kElocWarps * 32, smem, st>>>(B, c->n, d_s, c->row_ptr, c->col, (const int32_t*)c->w,
                                            (const int32_t*)c->field, (int32_t*)d_e);
  } else {
    auto k = eloc_sparse_kernel<float, float>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kElocWarps * 32, smem, st>>>(B, c->n, d_s, c->row_ptr, c->col, (const float*)c->w,
                                            (const float*)c->field, (float*)d_e);
  }
  return cudaGetLastError();
}

cudaError_t launch_eloc_dense_finish(const vqmc_ctx* c, int B, const int8_t* d_s, void* d_e, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  const int ntiles = (c->n + 127) / 128;
  eloc_dense_finish_kernel<<<(B + 255) / 256, 256, 0, st>>>(B, c->n, ntiles, c->row_part, c->row_part_ld, d_s,
                                                            (const float*)c->field, (float*)d_e);
  return cudaGetLastError();
}

cudaError_t launch_stats(const vqmc_ctx* c, int B, const void* d_e, double* d_stats, float* d_coef,
                         cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  if (c->ham == VQMC_HAM_SPARSE_I32)
    stats_kernel<int32_t><<<1, 1024, 0, st>>>(B, (const int32_t*)d_e, d_stats, d_coef, c->err);
  else
    stats_kernel<float><<<1, 1024, 0, st>>>(B, (const float*)d_e, d_stats, d_coef, c->err);
  return cudaGetLastError();
}

cudaError_t launch_spins_to_operands(const vqmc_ctx* c, int B, const int8_t* d_s, void* Sx, void* St,
                                     cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  dim3 grid((c->n + 31) / 32, (B + 31) / 32), block(32, 8);
  if (c->prec == VQMC_PREC_BF16)
    spins_convert_kernel<bf16><<<grid, block, 0, st>>>(B, c->n, d_s, (bf16*)Sx, c->np, (bf16*)St, c->Bp);
  else
    spins_convert_kernel<float><<<grid, block, 0, st>>>(B, c->n, d_s, (float*)Sx, c->np, (float*)St, c->Bp);
  return cudaGetLastError();
}

cudaError_t launch_row_sum(const vqmc_ctx* c, int B, int ntiles, float* out, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  tile_sum_kernel<<<(B + 255) / 256, 256, 0, st>>>(B, ntiles, c->row_part, c->row_part_ld, out);
  return cudaGetLastError();
}

cudaError_t launch_col_sum(const vqmc_ctx* c, int N, int mtiles, float* out, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  tile_sum_kernel<<<(N + 255) / 256, 256, 0, st>>>(N, mtiles, c->col_part, c->col_part_ld, out);
  return cudaGetLastError();
}

}  // namespace vqmc
