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

// Kept columns [lo, hi) of row r of W1^T (z = 0: r < m(k)) or W2 (z = 1:
// m(k) <= r); the degrees are sorted, so each row keeps one range.
__device__ __forceinline__ void kept_range(int z, int r, int n, int h, int* lo, int* hi) {
  const int c = count_deg_le(r, n, h);  // units with m(k) <= r
  *lo = z == 0 ? c : 0;
  *hi = z == 0 ? h : c;
}
__device__ __forceinline__ bool kept(int z, int r, int k, int n, int h) {
  int lo, hi;
  kept_range(z, r, n, h, &lo, &hi);
  return k >= lo && k < hi;
}
// True if the rows [r0, r0 + nr) x columns [k0, k0 + nk) tile keeps nothing.
__device__ __forceinline__ bool tile_masked(int z, int r0, int nr, int k0, int nk, int n, int h) {
  const int r1 = min(r0 + nr, n) - 1, k1 = min(k0 + nk, h) - 1;
  if (z == 0) return k1 < count_deg_le(r0, n, h);  // the row with the most kept columns
  return k0 >= count_deg_le(r1, n, h);
}

// One Adam step on the weight matrices fused with the refresh of their
// kernel-side copies.  Grid (h/32, n/32, 2): z = 0 for W1^T, z = 1 for W2;
// each 32 x 32 tile is updated with coalesced accesses along k, written to
// the row copy (wt_s shifted by one row, v_s), and through shared memory to
// the transposed copy (w_s, vt_s).  Only entries inside the MADE masks are
// updated (fully masked tiles return at once), so the masked weights stay
// zero whatever the gradient holds there.  Padding of the copies is never
// written (zero since allocation).
template <typename T>
__global__ void __launch_bounds__(256) adam_refresh_kernel(int n, int h, int hp, int np, float* __restrict__ theta,
                                                           float* __restrict__ m, float* __restrict__ v,
                                                           const float* __restrict__ g, float lr, float b1, float b2,
                                                           const float* __restrict__ ibc, float eps, T* __restrict__ wt_s,
                                                           T* __restrict__ v_s, T* __restrict__ w_s,
                                                           T* __restrict__ vt_s) {
  __shared__ float tile[32][33];
  const int k0 = blockIdx.x * 32, r0 = blockIdx.y * 32, z = blockIdx.z;
  const int tx = threadIdx.x, ty = threadIdx.y;
  if (tile_masked(z, r0, 32, k0, 32, n, h)) return;
  const float inv_bc1 = __ldg(ibc), inv_bc2 = __ldg(ibc + 1);
  const long long off = z == 0 ? 0 : (long long)n * h + h;
  for (int rr = ty; rr < 32; rr += 8) {
    const int r = r0 + rr, k = k0 + tx;
    tile[rr][tx] = 0.0f;
    if (r < n && k < h && kept(z, r, k, n, h)) {
      // theta, the moments and the gradient stream through with the
      // evict-first policy, so that the weight copies written here (which the
      // next sampler and GEMMs read) stay in L2
      const long long q = off + (long long)r * h + k;
      const float gq = __ldcs(g + q);
      const float mq = b1 * __ldcs(m + q) + (1.0f - b1) * gq;
      const float vq = b2 * __ldcs(v + q) + (1.0f - b2) * gq * gq;
      __stcs(m + q, mq);
      __stcs(v + q, vq);
      const float th = __ldcs(theta + q) - lr * (mq * inv_bc1) / (sqrtf(vq * inv_bc2) + eps);
      __stcs(theta + q, th);
      if (z == 0) {
        if (wt_s) wt_s[(long long)(r + 1) * hp + k] = cvt<T>(th);
      } else {
        v_s[(long long)r * hp + k] = cvt<T>(th);
      }
      tile[rr][tx] = th;
    }
  }
  __syncthreads();
  T* dst = z == 0 ? w_s : vt_s;
  for (int kk = ty; kk < 32; kk += 8) {
    const int k = k0 + kk, r = r0 + tx;
    if (k < h && r < n && kept(z, r, k, n, h)) dst[(long long)k * np + r] = cvt<T>(tile[tx][kk]);
  }
}

// The same for h % 4 == 0 with 16-byte accesses: tiles of 32 rows x 128
// columns, each thread 4 rows x 4 consecutive columns, every load of a thread
// issued before its arithmetic.
template <typename T>
__device__ __forceinline__ void store4(T* p, float a, float b, float c, float d);
template <>
__device__ __forceinline__ void store4<float>(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
template <>
__device__ __forceinline__ void store4<bf16>(bf16* p, float a, float b, float c, float d) {
  const __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
  *reinterpret_cast<uint2*>(p) = make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
}

template <typename T>
__global__ void __launch_bounds__(256) adam_refresh4_kernel(int n, int h, int hp, int np, float* __restrict__ theta,
                                                            float* __restrict__ m, float* __restrict__ v,
                                                            const float* __restrict__ g, float lr, float b1, float b2,
                                                            const float* __restrict__ ibc, float eps,
                                                            T* __restrict__ wt_s, T* __restrict__ v_s,
                                                            T* __restrict__ w_s, T* __restrict__ vt_s) {
  __shared__ float tile[32][129];
  const int k0 = blockIdx.x * 128, r0 = blockIdx.y * 32, z = blockIdx.z;
  const int tx = threadIdx.x, ty = threadIdx.y;
  if (tile_masked(z, r0, 32, k0, 128, n, h)) return;
  const float inv_bc1 = __ldg(ibc), inv_bc2 = __ldg(ibc + 1);
  const long long off = z == 0 ? 0 : (long long)n * h + h;
  const int k = k0 + 4 * tx;
  float4 G[4], M[4], V[4], TH[4];
  bool in[4];
  int klo[4], khi[4];  // kept columns of row r: [klo, khi)
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = r0 + ty + 8 * j;
    kept_range(z, r, n, h, &klo[j], &khi[j]);
    in[j] = r < n && k < h && k + 3 >= klo[j] && k < khi[j];
    const long long q = off + (long long)r * h + k;
    if (in[j]) {
      G[j] = __ldcs(reinterpret_cast<const float4*>(g + q));
      M[j] = __ldcs(reinterpret_cast<const float4*>(m + q));
      V[j] = __ldcs(reinterpret_cast<const float4*>(v + q));
      TH[j] = __ldcs(reinterpret_cast<const float4*>(theta + q));
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = r0 + ty + 8 * j, rr = ty + 8 * j;
#pragma unroll
    for (int e = 0; e < 4; ++e) tile[rr][4 * tx + e] = 0.0f;
    if (!in[j]) continue;
    const long long q = off + (long long)r * h + k;
    float gq[4] = {G[j].x, G[j].y, G[j].z, G[j].w}, mq[4] = {M[j].x, M[j].y, M[j].z, M[j].w};
    float vq[4] = {V[j].x, V[j].y, V[j].z, V[j].w}, th[4] = {TH[j].x, TH[j].y, TH[j].z, TH[j].w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (k + e < klo[j] || k + e >= khi[j]) continue;  // masked: stays as it is (zero)
      mq[e] = b1 * mq[e] + (1.0f - b1) * gq[e];
      vq[e] = b2 * vq[e] + (1.0f - b2) * gq[e] * gq[e];
      th[e] -= lr * (mq[e] * inv_bc1) / (sqrtf(vq[e] * inv_bc2) + eps);
      tile[rr][4 * tx + e] = th[e];
    }
    __stcs(reinterpret_cast<float4*>(m + q), make_float4(mq[0], mq[1], mq[2], mq[3]));
    __stcs(reinterpret_cast<float4*>(v + q), make_float4(vq[0], vq[1], vq[2], vq[3]));
    __stcs(reinterpret_cast<float4*>(theta + q), make_float4(th[0], th[1], th[2], th[3]));
    if (z == 0) {
      if (wt_s) store4<T>(wt_s + (long long)(r + 1) * hp + k, th[0], th[1], th[2], th[3]);
    } else {
      store4<T>(v_s + (long long)r * hp + k, th[0], th[1], th[2], th[3]);
    }
  }
  __syncthreads();
  T* dst = z == 0 ? w_s : vt_s;
  for (int kk = ty; kk < 128; kk += 8) {
    const int kq = k0 + kk, r = r0 + tx;
    if (kq < h && r < n && kept(z, r, kq, n, h)) dst[(long long)kq * np + r] = cvt<T>(tile[tx][kk]);
  }
}

// Pulls [p, p + bytes) into L2 (evict-last), one prefetch per 128-byte line.
__global__ void l2_prefetch_kernel(const char* __restrict__ p, size_t bytes) {
  for (size_t o = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * 128; o < bytes;
       o += (size_t)gridDim.x * blockDim.x * 128)
    asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(p + o));
}

// Next Adam step: t += 1 and its bias corrections.
__global__ void adam_advance_kernel(DevState* s, float beta1, float beta2) {
  s->adam_t += 1;
  adam_factors(s, beta1, beta2);
}

__global__ void set_state_kernel(DevState* s, unsigned long long iter, long long adam_t, float beta1, float beta2) {
  s->iter = iter;
  s->adam_t = adam_t;
  adam_factors(s, beta1, beta2);
}

// Adam on the biases b1 (after W1^T) and b2 (after W2).
__global__ void adam_bias_kernel(int n, int h, float* __restrict__ theta, float* __restrict__ m,
                                 float* __restrict__ v, const float* __restrict__ g, float lr, float b1, float b2,
                                 const float* __restrict__ ibc, float eps) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= h + n) return;
  const float inv_bc1 = __ldg(ibc), inv_bc2 = __ldg(ibc + 1);
  const long long q = t < h ? (long long)n * h + t : 2ll * n * h + h + (t - h);
  const float gq = g[q];
  const float mq = b1 * m[q] + (1.0f - b1) * gq;
  const float vq = b2 * v[q] + (1.0f - b2) * gq * gq;
  m[q] = mq;
  v[q] = vq;
  theta[q] -= lr * (mq * inv_bc1) / (sqrtf(vq * inv_bc2) + eps);
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

// grid-stride launches: at most 32 CTAs of `block` threads per SM of the device
int grid_for(const vqmc_ctx* c, long long work, int block = 256) {
  long long g = (work + block - 1) / block;
  const long long cap = 32ll * (c->num_sms > 0 ? c->num_sms : 1);
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

template <typename T>
cudaError_t refresh(vqmc_ctx* c, cudaStream_t st) {
  const int rows = sampler_rows(c->n);
  rows_kernel<T><<<grid_for(c, (long long)rows * c->hp), 256, 0, st>>>(c->n, c->h, c->hp, rows, c->theta, (T*)c->wt_s,
                                                                    (T*)c->v_s);
  dim3 grid((c->np + 31) / 32, (c->h + 31) / 32), block(32, 8);
  transpose_kernel<T><<<grid, block, 0, st>>>(c->n, c->h, c->np, c->theta, (T*)c->w_s);
  transpose_kernel<T><<<grid, block, 0, st>>>(c->n, c->h, c->np, c->theta + (long long)c->n * c->h + c->h,
                                               (T*)c->vt_s);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mask_params(vqmc_ctx* c, cudaStream_t st) {
  mask_kernel<<<grid_for(c, (long long)c->n * c->h), 256, 0, st>>>(c->n, c->h, c->theta);
  return cudaGetLastError();
}

cudaError_t launch_refresh_weights(vqmc_ctx* c, cudaStream_t st) {
  return c->prec == VQMC_PREC_BF16 ? refresh<bf16>(c, st) : refresh<float>(c, st);
}

AdamStep adam_advance(vqmc_ctx* c, cudaStream_t st) {
  c->adam_t += 1;
  adam_advance_kernel<<<1, 1, 0, st>>>(c->dstate, c->cfg.beta1, c->cfg.beta2);
  return AdamStep{&c->dstate->ibc1};
}

cudaError_t launch_set_state(vqmc_ctx* c, cudaStream_t st) {
  set_state_kernel<<<1, 1, 0, st>>>(c->dstate, (unsigned long long)c->iter, (long long)c->adam_t, c->cfg.beta1,
                                    c->cfg.beta2);
  return cudaGetLastError();
}

cudaError_t launch_adam_bias(vqmc_ctx* c, const float* d_grad, AdamStep a, cudaStream_t st) {
  adam_bias_kernel<<<(c->h + c->n + 255) / 256, 256, 0, st>>>(c->n, c->h, c->theta, c->adam_m, c->adam_v, d_grad,
                                                              c->cfg.lr, c->cfg.beta1, c->cfg.beta2, a.ibc, c->cfg.eps);
  return cudaGetLastError();
}

cudaError_t launch_adam(vqmc_ctx* c, const float* d_grad, cudaStream_t st, bool advance) {
  const AdamStep a = advance ? adam_advance(c, st) : AdamStep{&c->dstate->ibc1};
  const float* ib = a.ibc;
  const bool vec = c->h % 4 == 0;  // rows of theta start on 16-byte boundaries
  const dim3 grid(vec ? (c->h + 127) / 128 : (c->h + 31) / 32, (c->n + 31) / 32, 2), block(32, 8);
  // the tensor-core sampler reads W1 through w_s; only the CUDA-core one needs wt_s
  const bool need_wt = c->sampler != VQMC_SAMPLER_TENSOR_CORE;
  if (vec && c->prec == VQMC_PREC_BF16)
    adam_refresh4_kernel<bf16><<<grid, block, 0, st>>>(
        c->n, c->h, c->hp, c->np, c->theta, c->adam_m, c->adam_v, d_grad, c->cfg.lr, c->cfg.beta1, c->cfg.beta2, ib,
        c->cfg.eps, need_wt ? (bf16*)c->wt_s : nullptr, (bf16*)c->v_s, (bf16*)c->w_s, (bf16*)c->vt_s);
  else if (vec)
    adam_refresh4_kernel<float><<<grid, block, 0, st>>>(
        c->n, c->h, c->hp, c->np, c->theta, c->adam_m, c->adam_v, d_grad, c->cfg.lr, c->cfg.beta1, c->cfg.beta2, ib,
        c->cfg.eps, need_wt ? (float*)c->wt_s : nullptr, (float*)c->v_s, (float*)c->w_s, (float*)c->vt_s);
  else if (c->prec == VQMC_PREC_BF16)
    adam_refresh_kernel<bf16><<<grid, block, 0, st>>>(
        c->n, c->h, c->hp, c->np, c->theta, c->adam_m, c->adam_v, d_grad, c->cfg.lr, c->cfg.beta1, c->cfg.beta2, ib,
        c->cfg.eps, need_wt ? (bf16*)c->wt_s : nullptr, (bf16*)c->v_s, (bf16*)c->w_s, (bf16*)c->vt_s);
  else
    adam_refresh_kernel<float><<<grid, block, 0, st>>>(
        c->n, c->h, c->hp, c->np, c->theta, c->adam_m, c->adam_v, d_grad, c->cfg.lr, c->cfg.beta1, c->cfg.beta2, ib,
        c->cfg.eps, need_wt ? (float*)c->wt_s : nullptr, (float*)c->v_s, (float*)c->w_s, (float*)c->vt_s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_adam_bias(c, d_grad, a, st);
}

cudaError_t launch_prefetch_sampler_weights(const vqmc_ctx* c, cudaStream_t st) {
  const size_t es = c->prec == VQMC_PREC_BF16 ? 2 : 4;
  l2_prefetch_kernel<<<c->num_sms * 4, 256, 0, st>>>((const char*)c->v_s, (size_t)sampler_rows(c->n) * c->hp * es);
  l2_prefetch_kernel<<<c->num_sms * 4, 256, 0, st>>>((const char*)c->w_s, (size_t)c->h * c->np * es);
  return cudaGetLastError();
}

cudaError_t launch_dense_split(vqmc_ctx* c, cudaStream_t st) {
  split_kernel<<<grid_for(c, (long long)c->n * c->np), 256, 0, st>>>(c->n, c->np, c->J, (bf16*)c->J_hi, (bf16*)c->J_lo);
  return cudaGetLastError();
}

}  // namespace vqmc
