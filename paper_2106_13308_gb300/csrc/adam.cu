// Parameter maintenance: MADE masks on the master theta, the kernels' weight
// copies (BF16 rounded to nearest even, or FP32) and the Adam step (the
// paper's default optimiser, Sec. 5.1).
//
// theta = [W1^T (n x h) | b1 (h) | W2 (n x h) | b2 (n)].
#include "common.cuh"

namespace vqmc {
namespace {

template <typename T>
__device__ __forceinline__ T cvt(float x);
template <>
__device__ __forceinline__ float cvt<float>(float x) { return x; }
template <>
__device__ __forceinline__ bf16 cvt<bf16>(float x) { return __float2bfloat16_rn(x); }

// Zero W1^T[j'][k] unless j' < m(k), and W2[i'][k] unless m(k) <= i'.
__global__ void mask_kernel(int n, int h, float* __restrict__ theta) {
  const long long nh = (long long)n * h;
  float* W2 = theta + nh + h;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nh; q += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(q / h), k = (int)(q % h);
    const int m = degree(k, n, h);
    if (!(r < m)) theta[q] = 0.0f;
    if (!(m <= r)) W2[q] = 0.0f;
  }
}

// Row copies for the sampler: wt_s[j][k] = W1^T[j-1][k] (row 0 zero),
// v_s[i][k] = W2[i][k]; zero for k >= h and for rows past the matrix.
template <typename T>
__global__ void rows_kernel(int n, int h, int hp, int rows, const float* __restrict__ theta, T* __restrict__ wt_s,
                            T* __restrict__ v_s) {
  const float* W2 = theta + (long long)n * h + h;
  const long long tot = (long long)rows * hp;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot; q += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(q / hp), k = (int)(q % hp);
    const bool in = k < h;
    wt_s[q] = cvt<T>(in && r >= 1 && r <= n ? theta[(long long)(r - 1) * h + k] : 0.0f);
    v_s[q] = cvt<T>(in && r < n ? W2[(long long)r * h + k] : 0.0f);
  }
}

// Transposed copies through a 32x32 tile: dst[k][r] = src[r][k] for r < n,
// zero for n <= r < np.
template <typename T>
__global__ void transpose_kernel(int n, int h, int np, const float* __restrict__ src, T* __restrict__ dst) {
  __shared__ float tile[32][33];
  const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int q = ty; q < 32; q += 8) {
    const int r = r0 + q, k = k0 + tx;
    tile[q][tx] = (r < n && k < h) ? src[(long long)r * h + k] : 0.0f;
  }
  __syncthreads();
  for (int q = ty; q < 32; q += 8) {
    const int k = k0 + q, r = r0 + tx;
    if (k < h && r < np) dst[(long long)k * np + r] = cvt<T>(tile[tx][q]);
  }
}

__global__ void adam_kernel(long long d, float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, float lr, float b1, float b2, float inv_bc1,
                            float inv_bc2, float eps) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < d; q += (long long)gridDim.x * blockDim.x) {
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.0f - b1) * gq;
    const float vq = b2 * v[q] + (1.0f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    theta[q] -= lr * (mq * inv_bc1) / (sqrtf(vq * inv_bc2) + eps);
  }
}

__global__ void split_kernel(int n, int np, const float* __restrict__ J, bf16* __restrict__ hi, bf16* __restrict__ lo) {
  const long long tot = (long long)n * np;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot; q += (long long)gridDim.x * blockDim.x) {
    const float x = J[q];
    const bf16 xh = __float2bfloat16_rn(x);
    hi[q] = xh;
    lo[q] = __float2bfloat16_rn(x - __bfloat162float(xh));
  }
}

int grid_for(long long work, int block = 256) {
  long long g = (work + block - 1) / block;
  if (g > 152 * 32) g = 152 * 32;
  return (int)(g < 1 ? 1 : g);
}

template <typename T>
cudaError_t refresh(vqmc_ctx* c, cudaStream_t st) {
  const int rows = sampler_rows(c->n);
  rows_kernel<T><<<grid_for((long long)rows * c->hp), 256, 0, st>>>(c->n, c->h, c->hp, rows, c->theta, (T*)c->wt_s,
                                                                    (T*)c->v_s);
  dim3 grid((c->np + 31) / 32, (c->h + 31) / 32), block(32, 8);
  transpose_kernel<T><<<grid, block, 0, st>>>(c->n, c->h, c->np, c->theta, (T*)c->w_s);
  transpose_kernel<T><<<grid, block, 0, st>>>(c->n, c->h, c->np, c->theta + (long long)c->n * c->h + c->h,
                                               (T*)c->vt_s);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mask_params(vqmc_ctx* c, cudaStream_t st) {
  mask_kernel<<<grid_for((long long)c->n * c->h), 256, 0, st>>>(c->n, c->h, c->theta);
  return cudaGetLastError();
}

cudaError_t launch_refresh_weights(vqmc_ctx* c, cudaStream_t st) {
  return c->prec == VQMC_PREC_BF16 ? refresh<bf16>(c, st) : refresh<float>(c, st);
}

cudaError_t launch_adam(vqmc_ctx* c, const float* d_grad, cudaStream_t st) {
  c->adam_t += 1;
  const double t = (double)c->adam_t;
  const double bc1 = 1.0 - pow((double)c->cfg.beta1, t), bc2 = 1.0 - pow((double)c->cfg.beta2, t);
  adam_kernel<<<grid_for(c->d), 256, 0, st>>>(c->d, c->theta, c->adam_m, c->adam_v, d_grad, c->cfg.lr, c->cfg.beta1,
                                               c->cfg.beta2, (float)(1.0 / bc1), (float)(1.0 / bc2), c->cfg.eps);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_refresh_weights(c, st);
}

cudaError_t launch_dense_split(vqmc_ctx* c, cudaStream_t st) {
  split_kernel<<<grid_for((long long)c->n * c->np), 256, 0, st>>>(c->n, c->np, c->J, (bf16*)c->J_hi, (bf16*)c->J_lo);
  return cudaGetLastError();
}

}  // namespace vqmc
