// Stochastic reconfiguration (natural gradient, Sec. 2.1) on the GPU.
//
// With O_b = grad_theta log pi(s_b), the per-sample score vector (d entries),
// the batch estimates of the paper's population forms are
//   g = (1/B) sum_b (E_b - mean E) O_b,     I = (1/B) sum_b O_b O_b^T,
// and the natural-gradient direction solves (I + lambda 1) delta = g.  Here
// B << d, so the d x d matrix is never formed: by the push-through identity
//   delta = O^T x,   (O O^T / B + lambda) x = c,   c_b = (E_b - mean E) / B,
// one iteration needs the B x B Gram matrix G = O O^T, a Cholesky
// factorisation of G / B + lambda with two triangular solves, and one adjoint
// pass with the per-sample coefficients x (the kernels of the gradient).
//
// The Gram matrix comes from the MADE structure without forming O.  A
// sample's score vector has four blocks (theta layout, 1-based i, j):
//   dW1^T[j][k] = GA_k s_j [j <= m(k)],   db1[k] = GA_k,
//   dW2[i][k]   = delta_i H_k [i > m(k)], db2[i] = delta_i,
// with delta_i = s_i sigma(-s_i z_i), H = act(a) and
// GA_k = act'(a_k) sum_i delta_i W2_ik (the adjoint pass's operands Dt, Ht,
// GAt and St hold exactly these per sample when its coefficients are 1).
// With o the elementwise product of B x B matrices,
//   G = sum_i (delta_i delta_i^T) o P_i + sum_k (GA_k GA_k^T) o Q_{m(k)},
//   P_i = 1 + sum_{k: m(k) < i} H_k H_k^T,   Q_t = 1 + sum_{j <= t} s_j s_j^T,
// the ones standing for the two bias blocks.  Walking the spins in order and
// the hidden units in degree order (sorted degrees) updates P and Q by one
// outer product per event, so an entry of G costs 5 (n + h) flops (three
// FP32 instructions per event) instead of the 2 h n of a GEMM over explicit
// score vectors.
#include <climits>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace vqmc {

namespace {

constexpr int kGT = 64;  // Gram tile (samples x samples)
constexpr int kGE = 32;  // events (spins or hidden units) staged per chunk
constexpr int kNB = 64;  // Cholesky block

// (row, column) of the lower-triangular tile with linear index idx, row-major
__device__ __forceinline__ void tri_index(int idx, int* row, int* col) {
  int r = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
  while ((r + 1) * (r + 2) / 2 <= idx) ++r;
  while (r * (r + 1) / 2 > idx) --r;
  *row = r;
  *col = idx - r * (r + 1) / 2;
}

struct GramArgs {
  const float* St;    // [n][ld] spins
  const float* Dt;    // [n][ld] delta
  const float* Ht;    // [h][ld] hidden activations
  const float* GAt;   // [h][ld] hidden adjoint
  const int* events;  // [n + h]: spin t as t >= 0, hidden unit k as -1 - k, in walking order
  int ld;
  int n, h, B;
  float* out;
  int ldo;
  float scale, shift;  // out = scale G + shift 1
  int mirror;          // also write the upper triangle
  int pad_to;          // rows/columns [B, pad_to) of out get the identity
};

// Loads the two vectors of the events [e0, e0 + kGE) over the tile's 64 row
// samples (b0..) and 64 column samples (c0..): 2 x 32 x 128 floats, eight
// float4 per thread; zero past the batch or the last event.
__device__ __forceinline__ void gram_fetch(const GramArgs& a, int e0, int b0, int c0, int tid, float4 (&v)[8],
                                           int& ev) {
  const int total = a.n + a.h;
  ev = (tid < kGE && e0 + tid < total) ? __ldg(a.events + e0 + tid) : INT_MIN;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int L = tid + 256 * j;
    const int arr = L >> 10, rem = L & 1023, e = rem >> 5, q = rem & 31;
    const int col = q < 16 ? b0 + 4 * q : c0 + 4 * (q - 16);
    v[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (e0 + e < total) {
      const int code = __ldg(a.events + e0 + e);
      const float* base = code >= 0 ? (arr ? a.Dt : a.St) : (arr ? a.GAt : a.Ht);
      const float* p = base + (size_t)(code >= 0 ? code : -1 - code) * a.ld + col;
      if (col + 3 < a.B) {
        v[j] = __ldg(reinterpret_cast<const float4*>(p));
      } else {
        if (col < a.B) v[j].x = __ldg(p);
        if (col + 1 < a.B) v[j].y = __ldg(p + 1);
        if (col + 2 < a.B) v[j].z = __ldg(p + 2);
      }
    }
  }
}

// One CTA per 64 x 64 tile of the lower triangle; 256 threads, 4 x 4 entries
// each (rows b0 + 4 ty + r, columns c0 + 4 tx + q).  Events are staged 32 at a
// time in shared memory: the two vectors of a spin event (s_t, delta_t) or of
// a unit event (H_k, GA_k) over the tile's 64 row and 64 column samples; the
// next chunk is loaded into registers while the current one is consumed.
__global__ void __launch_bounds__(256) sr_gram_kernel(GramArgs a) {
  __shared__ __align__(16) float sx[kGE][2 * kGT];
  __shared__ __align__(16) float sy[kGE][2 * kGT];
  __shared__ int skind[kGE];  // 0 none, 1 spin, 2 hidden unit
  int bt, ct;
  tri_index(blockIdx.x, &bt, &ct);
  const int b0 = bt * kGT, c0 = ct * kGT;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float G[4][4], P[4][4], Q[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) G[r][q] = 0.0f, P[r][q] = 1.0f, Q[r][q] = 1.0f;
  const int total = a.n + a.h;
  float4 v[8];
  int ev;
  gram_fetch(a, 0, b0, c0, tid, v, ev);
  for (int e0 = 0; e0 < total; e0 += kGE) {
    // stage the fetched chunk
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int L = tid + 256 * j;
      const int arr = L >> 10, rem = L & 1023, e = rem >> 5, q = rem & 31;
      *reinterpret_cast<float4*>((arr ? &sy[e][0] : &sx[e][0]) + 4 * q) = v[j];
    }
    if (tid < kGE) skind[tid] = ev == INT_MIN ? 0 : (ev >= 0 ? 1 : 2);
    __syncthreads();
    if (e0 + kGE < total) gram_fetch(a, e0 + kGE, b0, c0, tid, v, ev);
    const int ne = total - e0 < kGE ? total - e0 : kGE;
    for (int e = 0; e < ne; ++e) {
      const float4 xr4 = *reinterpret_cast<const float4*>(&sx[e][4 * ty]);
      const float4 xc4 = *reinterpret_cast<const float4*>(&sx[e][kGT + 4 * tx]);
      const float4 yr4 = *reinterpret_cast<const float4*>(&sy[e][4 * ty]);
      const float4 yc4 = *reinterpret_cast<const float4*>(&sy[e][kGT + 4 * tx]);
      const float xr[4] = {xr4.x, xr4.y, xr4.z, xr4.w}, xc[4] = {xc4.x, xc4.y, xc4.z, xc4.w};
      const float yr[4] = {yr4.x, yr4.y, yr4.z, yr4.w}, yc[4] = {yc4.x, yc4.y, yc4.z, yc4.w};
      if (skind[e] == 1) {
        // spin t: Q += s_t s_t^T, G += (delta_t delta_t^T) o P
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            Q[r][q] = fmaf(xr[r], xc[q], Q[r][q]);
            G[r][q] = fmaf(yr[r] * yc[q], P[r][q], G[r][q]);
          }
      } else {
        // unit k: G += (GA_k GA_k^T) o Q, P += H_k H_k^T
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            G[r][q] = fmaf(yr[r] * yc[q], Q[r][q], G[r][q]);
            P[r][q] = fmaf(xr[r], xc[q], P[r][q]);
          }
      }
    }
    __syncthreads();  // the chunk is consumed before the next one is staged
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int b = b0 + 4 * ty + r, c = c0 + 4 * tx + q;
      if (b < a.B && c < a.B) {
        const float val = a.scale * G[r][q] + (b == c ? a.shift : 0.0f);
        a.out[(size_t)b * a.ldo + c] = val;
        if (a.mirror && b != c) a.out[(size_t)c * a.ldo + b] = val;
      } else if (b < a.pad_to && c < a.pad_to) {
        a.out[(size_t)b * a.ldo + c] = b == c ? 1.0f : 0.0f;
      }
    }
}

// Blocked right-looking Cholesky, step k.  Every CTA factors the diagonal
// block A_kk = L_kk L_kk^T in registers (thread (r, q) holds row r, columns
// 4 m + q; the current column is passed through shared memory, one barrier
// per column).  CTA 0 stores X_k = L_kk^-T (the panel solve below applied to
// the identity) for the triangular solves, which need nothing else of the
// diagonal blocks; A_kk itself is left as it is, so that no CTA of this
// launch can read a partly overwritten block.  CTA i > 0 solves the panel
// block X L_kk^T = A_(k+i),k in place.  Only the lower triangle of A is
// read.  A non-positive pivot (rounding or non-finite input) sets the device
// error word (VQMC_DEVERR_NONFINITE) and propagates a NaN.
__global__ void __launch_bounds__(256) chol_panel_kernel(float* __restrict__ A, int ld, int k, float* __restrict__ Xinv,
                                                         uint32_t* err) {
  __shared__ float L[kNB][kNB + 1];
  __shared__ float colbuf[2][kNB];
  __shared__ float inv_d[kNB];
  const int tid = threadIdx.x, r = tid >> 2, q = tid & 3, grp = (tid & 31) & ~3;
  const size_t kk = (size_t)k * kNB;
  float v[16];
  {
    const float* row = A + (kk + r) * ld + kk;
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = 4 * m + q <= r ? row[4 * m + q] : 0.0f;
  }
  if (q == 0) colbuf[0][r] = v[0];
  __syncthreads();
  bool bad = false;
#pragma unroll
  for (int j = 0; j < kNB; ++j) {
    const float* cb = colbuf[j & 1];
    const float d = cb[j];
    const float rs = rsqrtf(d);  // NaN for d < 0, inf for d = 0
    bad |= !(d > 0.0f);
    const float cr = cb[r];
    if (q == (j & 3)) {
      if (r == j) v[j >> 2] = d * rs;
      else if (r > j) v[j >> 2] = cr * rs;
    }
    // trailing columns c in (j, r]: A_rc -= A_rj A_cj / A_jj
    const float ar = cr * (rs * rs);
#pragma unroll
    for (int m = (j + 1) >> 2; m < 16; ++m) {
      const int c = 4 * m + q;
      if (c > j && c <= r) v[m] -= ar * cb[c];
    }
    if (j + 1 < kNB && q == ((j + 1) & 3) && r >= j + 1) colbuf[(j + 1) & 1][r] = v[(j + 1) >> 2];
    __syncthreads();
  }
  if (bad && tid == 0 && blockIdx.x == 0) atomicOr(err, kErrNonfinite);
#pragma unroll
  for (int m = 0; m < 16; ++m) L[r][4 * m + q] = v[m];
  __syncthreads();
  if (tid < kNB) inv_d[tid] = 1.0f / L[tid][tid];
  __syncthreads();
  // panel rows (CTA i > 0) or the identity (CTA 0): X L_kk^T = P, row by
  // row, 4 threads per row; thread q holds columns 4 m + q
  float* prow = blockIdx.x == 0 ? Xinv + ((size_t)k * kNB + r) * kNB : A + (kk + (size_t)blockIdx.x * kNB + r) * ld + kk;
#pragma unroll
  for (int m = 0; m < 16; ++m) v[m] = blockIdx.x == 0 ? (4 * m + q == r ? 1.0f : 0.0f) : prow[4 * m + q];
#pragma unroll
  for (int j = 0; j < kNB; ++j) {
    float x = v[j >> 2] * inv_d[j];  // meaningful in the owner lane only
    x = __shfl_sync(0xffffffffu, x, grp | (j & 3));
    if (q == (j & 3)) v[j >> 2] = x;
#pragma unroll
    for (int m = j >> 2; m < 16; ++m)
      if (4 * m + q > j) v[m] -= x * L[4 * m + q][j];
  }
#pragma unroll
  for (int m = 0; m < 16; ++m) prow[4 * m + q] = v[m];
}

// Trailing update of step k: A_ij -= L_ik L_jk^T for k < j <= i < T, one CTA
// per tile, 4 x 4 entries per thread.
__global__ void __launch_bounds__(256) chol_update_kernel(float* __restrict__ A, int ld, int k) {
  __shared__ __align__(16) float si[kNB][kNB + 4];  // si[l][r] = L_ik[r][l]
  __shared__ __align__(16) float sj[kNB][kNB + 4];
  int ii, jj;
  tri_index(blockIdx.x, &ii, &jj);
  const size_t i0 = (size_t)(k + 1 + ii) * kNB, j0 = (size_t)(k + 1 + jj) * kNB, k0 = (size_t)k * kNB;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int idx = tid; idx < kNB * kNB; idx += 256) {
    const int r = idx >> 6, l = idx & 63;
    si[l][r] = A[(i0 + r) * ld + k0 + l];
    sj[l][r] = A[(j0 + r) * ld + k0 + l];
  }
  __syncthreads();
  float acc[4][4] = {};
#pragma unroll 8
  for (int l = 0; l < kNB; ++l) {
    const float4 a4 = *reinterpret_cast<const float4*>(&si[l][4 * ty]);
    const float4 b4 = *reinterpret_cast<const float4*>(&sj[l][4 * tx]);
    const float av[4] = {a4.x, a4.y, a4.z, a4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(av[r], bv[q], acc[r][q]);
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) A[(i0 + 4 * ty + r) * ld + j0 + 4 * tx + q] -= acc[r][q];
}

// L L^T x = rhs with the factor from the kernels above (T blocks of 64; rows
// >= B are the identity) and X_k = L_kk^-T.  One CTA of 1024 threads; per
// block a reduction over the solved part, then a 64 x 64 product with the
// inverse diagonal block: y_k = X_k^T (rhs_k - sum_{j<k} L_kj y_j), then
// x_k = X_k (y_k - sum_{j>k} L_jk^T x_j).  x may alias rhs.
__global__ void __launch_bounds__(1024) chol_solve_kernel(const float* __restrict__ A, int ld, int T,
                                                          const float* __restrict__ Xinv, const float* rhs, int B,
                                                          float* x) {
  extern __shared__ float sm[];
  float* y = sm;                      // [T * 64]
  float* part = y + (size_t)T * kNB;  // [16][64]
  float* rv = part + 16 * kNB;        // [64]
  const int tid = threadIdx.x;
  const int N = T * kNB;
  for (int i = tid; i < N; i += 1024) y[i] = i < B ? rhs[i] : 0.0f;
  __syncthreads();
  // forward
  for (int kb = 0; kb < T; ++kb) {
    const size_t r0 = (size_t)kb * kNB;
    {
      const int r = tid >> 4, p = tid & 15;
      const float* row = A + (r0 + r) * ld;
      float s = 0.0f;
      for (int l = p; l < (int)r0; l += 16) s = fmaf(row[l], y[l], s);
#pragma unroll
      for (int off = 8; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (p == 0) rv[r] = y[r0 + r] - s;
    }
    __syncthreads();
    {
      const int i = tid & 63, p = tid >> 6;
      const float* X = Xinv + r0 * kNB;
      float s = 0.0f;
#pragma unroll
      for (int l = p; l < kNB; l += 16) s = fmaf(X[(size_t)l * kNB + i], rv[l], s);
      part[p * kNB + i] = s;
    }
    __syncthreads();
    if (tid < kNB) {
      float s = 0.0f;
#pragma unroll
      for (int p = 0; p < 16; ++p) s += part[p * kNB + tid];
      y[r0 + tid] = s;
    }
    __syncthreads();
  }
  // backward
  for (int kb = T - 1; kb >= 0; --kb) {
    const size_t r0 = (size_t)kb * kNB;
    {
      const int r = tid & 63, p = tid >> 6;
      float s = 0.0f;
      for (int l = (int)r0 + kNB + p; l < N; l += 16) s = fmaf(A[(size_t)l * ld + r0 + r], y[l], s);
      part[p * kNB + r] = s;
    }
    __syncthreads();
    if (tid < kNB) {
      float s = 0.0f;
#pragma unroll
      for (int p = 0; p < 16; ++p) s += part[p * kNB + tid];
      rv[tid] = y[r0 + tid] - s;
    }
    __syncthreads();
    {
      const int i = tid >> 4, p = tid & 15;
      const float* X = Xinv + (r0 + i) * kNB;
      float s = 0.0f;
#pragma unroll
      for (int l = p; l < kNB; l += 16) s = fmaf(X[l], rv[l], s);
#pragma unroll
      for (int off = 8; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (p == 0) y[r0 + i] = s;
    }
    __syncthreads();
  }
  for (int i = tid; i < B; i += 1024) x[i] = y[i];
}

__global__ void sgd_kernel(long long d, float lr, const float* __restrict__ delta, float* __restrict__ theta) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < d; i += (long long)gridDim.x * blockDim.x)
    theta[i] -= lr * delta[i];
}

__global__ void fill_kernel(int n, float v, float* __restrict__ p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

size_t solve_smem(int T) { return ((size_t)T * kNB + 17 * kNB) * sizeof(float); }

}  // namespace

int sr_blocks(int B) { return (B + kNB - 1) / kNB; }

int sr_ld(const vqmc_ctx* c) { return sr_blocks(c->Bmax) * kNB; }

cudaError_t sr_workspace(vqmc_ctx* c) {
  if (c->sr_A) return cudaSuccess;
  const size_t N = (size_t)sr_blocks(c->Bmax) * kNB;
  // the Gram kernel's walking order: unit k right after spin m(k) (1-based)
  std::vector<int> ev;
  ev.reserve((size_t)c->n + c->h);
  for (int t = 0, k = 0; t < c->n || k < c->h;) {
    if (k < c->h && degree(k, c->n, c->h) <= t) ev.push_back(-1 - k++);
    else ev.push_back(t++);
  }
  cudaError_t e = cudaMalloc((void**)&c->sr_A, N * N * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->sr_x, N * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->sr_ones, N * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->sr_xinv, N * kNB * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->sr_events, ev.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(c->sr_events, ev.data(), ev.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    fill_kernel<<<(unsigned)((N + 255) / 256), 256>>>((int)N, 1.0f, c->sr_ones);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(chol_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)solve_smem(sr_blocks(kSrMaxBatch)));
  if (e != cudaSuccess) {
    cudaFree(c->sr_A), cudaFree(c->sr_x), cudaFree(c->sr_ones), cudaFree(c->sr_xinv), cudaFree(c->sr_events);
    c->sr_A = c->sr_x = c->sr_ones = c->sr_xinv = nullptr;
    c->sr_events = nullptr;
  }
  return e;
}

cudaError_t launch_sr_gram(const vqmc_ctx* c, int B, float* out, int ldo, float scale, float shift, bool mirror,
                           int pad_to, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  GramArgs a;
  a.St = (const float*)c->St, a.Dt = (const float*)c->Dt, a.Ht = (const float*)c->Ht, a.GAt = (const float*)c->GAt;
  a.events = c->sr_events;
  a.ld = c->Bp, a.n = c->n, a.h = c->h, a.B = B;
  a.out = out, a.ldo = ldo, a.scale = scale, a.shift = shift, a.mirror = mirror ? 1 : 0, a.pad_to = pad_to;
  const int T = (B + kGT - 1) / kGT;
  sr_gram_kernel<<<T * (T + 1) / 2, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sr_solve(const vqmc_ctx* c, int B, const float* rhs, float* x, cudaStream_t st, int* launches) {
  const int T = sr_blocks(B);
  const int ld = sr_ld(c);
  for (int k = 0; k < T; ++k) {
    chol_panel_kernel<<<T - k, 256, 0, st>>>(c->sr_A, ld, k, c->sr_xinv, c->err);
    const int R = T - k - 1;
    if (R > 0) chol_update_kernel<<<R * (R + 1) / 2, 256, 0, st>>>(c->sr_A, ld, k);
  }
  chol_solve_kernel<<<1, 1024, solve_smem(T), st>>>(c->sr_A, ld, T, c->sr_xinv, rhs, B, x);
  if (launches) *launches = 2 * T;
  return cudaGetLastError();
}

cudaError_t launch_sgd(vqmc_ctx* c, const float* delta, float lr, cudaStream_t st) {
  long long g = (c->d + 255) / 256;
  if (g > 4 * c->num_sms * 8) g = 4 * c->num_sms * 8;
  sgd_kernel<<<(unsigned)g, 256, 0, st>>>(c->d, lr, delta, c->theta);
  return cudaGetLastError();
}

}  // namespace vqmc
