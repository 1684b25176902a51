// Local energy (Sec. 2.1, Sec. 2.4), FP64 batch statistics (Eq. (e:vmc),
// Eq. (eq:stochastic_variance)) and spin-layout conversions.
//
// Sparse local energy.  For a diagonal Hamiltonian l(s) = H_ss =
// sum_{i<j} J_ij s_i s_j + sum_i h_i s_i.  The spins are first packed
// bit-transposed, 32 samples per word: Sbits[w][i] bit l = [s_i of sample
// 32w + l is -1] (one warp per 32 x 32 tile, coalesced reads).  Then one CTA
// per (word, slice of rows) loads its n words into shared memory, so one
// 32-bit xor of two words gives the sign of s_i s_j for all 32 samples, the
// warps take the slice's CSR rows in turn and lane l accumulates sample l.
// Slices hold about equal numbers of edges; their partial energies are summed
// in slice order.  Integer weights accumulate in int32 (exact).
#include "common.cuh"

namespace vqmc {
namespace {

constexpr int kElocWarps = 8;

// Sbits[w][i] for a 32-site x 32-sample tile per warp.
__global__ void __launch_bounds__(256) pack_bits_kernel(int B, int n, const int8_t* __restrict__ S,
                                                        uint32_t* __restrict__ bits) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = (blockIdx.x * 8 + warp) * 32, w = blockIdx.y;
  if (i0 >= n) return;
  const int b = 32 * w + lane;
  // lane l: bit i = [s_{i0+i} of sample b is -1]
  uint32_t m = 0;
  if (b < B) {
    const int8_t* row = S + (size_t)b * n + i0;
    const int cnt = min(32, n - i0);
    if (cnt == 32 && (reinterpret_cast<uintptr_t>(row) & 15) == 0) {
      const uint4 q0 = __ldg(reinterpret_cast<const uint4*>(row)), q1 = __ldg(reinterpret_cast<const uint4*>(row) + 1);
      const uint32_t wv[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        // sign bits of the 4 bytes of word k (spins are +-1: bit 7 set iff -1)
        const uint32_t sg = (wv[k] >> 7) & 0x01010101u;
        m |= ((sg * 0x01020408u) >> 24 & 0xFu) << (4 * k);
      }
    } else {
      for (int i = 0; i < cnt; ++i) m |= (__ldg(row + i) < 0 ? 1u : 0u) << i;
    }
  }
  uint32_t out = 0;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const uint32_t t = __ballot_sync(0xffffffffu, (m >> i) & 1u);
    if (lane == i) out = t;
  }
  if (i0 + lane < n) bits[(size_t)w * n + i0 + lane] = out;
}

// Edges of slice q are split evenly among the warps; each warp reads 32
// edges at a time (row, column, weight) with coalesced loads and broadcasts
// them with shuffles, so no load waits on another.
template <typename W, typename A>
__global__ void __launch_bounds__(kElocWarps * 32) eloc_sparse_kernel(int B, int n, const uint32_t* __restrict__ Sbits,
                                                                      const int32_t* __restrict__ row_ptr,
                                                                      const int32_t* __restrict__ erow,
                                                                      const int32_t* __restrict__ col,
                                                                      const W* __restrict__ w,
                                                                      const W* __restrict__ field,
                                                                      const int32_t* __restrict__ slice,
                                                                      A* __restrict__ part, int ldp) {
  extern __shared__ uint32_t bits[];  // [n]
  __shared__ A red[kElocWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wd = blockIdx.x, q = blockIdx.y;
  const uint32_t* src = Sbits + (size_t)wd * n;
  for (int i = threadIdx.x; i < n; i += kElocWarps * 32) bits[i] = __ldg(src + i);
  __syncthreads();
  A e = 0;
  const int r0 = __ldg(slice + q), r1 = __ldg(slice + q + 1);
  if (field)
    for (int i = r0 + warp; i < r1; i += kElocWarps) {
      const A f = (A)__ldg(field + i);
      e += ((bits[i] >> lane) & 1u) ? -f : f;
    }
  const int pa = __ldg(row_ptr + r0), pb = __ldg(row_ptr + r1);
  const int per = (pb - pa + kElocWarps - 1) / kElocWarps;
  const int p0 = pa + warp * per, p1 = min(pb, p0 + per);
  for (int pc = p0; pc < p1; pc += 32) {
    const int p = pc + lane;
    const bool in = p < p1;
    const int ei = in ? __ldg(erow + p) : 0, ej = in ? __ldg(col + p) : 0;
    const A ew = in ? (A)__ldg(w + p) : (A)0;
    const int cnt = min(32, p1 - pc);
#pragma unroll 4
    for (int k = 0; k < cnt; ++k) {
      const int i = __shfl_sync(0xffffffffu, ei, k), j = __shfl_sync(0xffffffffu, ej, k);
      const A wt = __shfl_sync(0xffffffffu, ew, k);
      const uint32_t x = bits[i] ^ bits[j];
      e += ((x >> lane) & 1u) ? -wt : wt;
    }
  }
  red[warp][lane] = e;
  __syncthreads();
  const int b = 32 * wd + lane;
  if (warp == 0 && b < B) {
    A t = red[0][lane];
#pragma unroll
    for (int k = 1; k < kElocWarps; ++k) t += red[k][lane];
    part[(size_t)q * ldp + b] = t;
  }
}

// Bit-sliced variant for small integer weights (|J_ij| < 2^(PL - 5)): the
// lanes take different edges and each handles all 32 samples of the word at
// once.  With x = bit_i xor bit_j (bit set: s_i s_j = -1), the slice's part
// of E_b is W - 2 sum_e J_e x_{e,b}, W the slice's weight sum.  A lane adds
// J_e x_e into a two's-complement counter kept as bit planes (bit b of plane
// t: bit t of sample b's partial sum; each addition a ripple of full adders
// over the planes): PL planes for runs of 15 edges (15 (2^(PL-5) - 1) <
// 2^(PL-1)), each run then sign-extended into 32 planes.  The lanes' and then
// the warps' counters are added plane-wise in a fixed order, and lane b
// finally reads sample b's integer off the planes.  The result equals the
// plain kernel's bit for bit (both are W - 2 sum J x in int32).
__device__ __forceinline__ void add_planes32(uint32_t (&C)[32], const uint32_t (&a)[32]) {
  uint32_t c = 0;
#pragma unroll
  for (int t = 0; t < 32; ++t) {
    const uint32_t s = C[t] ^ a[t] ^ c;
    c = (C[t] & a[t]) | (c & (C[t] ^ a[t]));
    C[t] = s;
  }
}

template <int PL, bool STAGE>
__global__ void __launch_bounds__(kElocWarps * 32) eloc_sliced_kernel(int B, int n, const uint32_t* __restrict__ Sbits,
                                                                     const int32_t* __restrict__ row_ptr,
                                                                     const int32_t* __restrict__ erow,
                                                                     const int32_t* __restrict__ col,
                                                                     const int32_t* __restrict__ w,
                                                                     const int32_t* __restrict__ field,
                                                                     const int32_t* __restrict__ slice,
                                                                     int32_t* __restrict__ part, int ldp) {
  // STAGE: the word's n spin words in shared memory; otherwise read through
  // L1 (no shared memory, so that the CTAs fit beside a GEMM's)
  extern __shared__ uint32_t staged[];  // [n] if STAGE
  __shared__ uint32_t planes[kElocWarps][32];
  __shared__ int32_t fpart[kElocWarps][32];
  __shared__ int32_t wpart[kElocWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wd = blockIdx.x, q = blockIdx.y;
  const uint32_t* src = Sbits + (size_t)wd * n;
  if constexpr (STAGE) {
    for (int i = threadIdx.x; i < n; i += kElocWarps * 32) staged[i] = __ldg(src + i);
    __syncthreads();
  }
  auto bit_word = [&](int i) -> uint32_t {
    if constexpr (STAGE) return staged[i];
    else return __ldg(src + i);
  };
  const int r0 = __ldg(slice + q), r1 = __ldg(slice + q + 1);
  // the field: lane = sample, as in the plain kernel
  int32_t fe = 0;
  if (field)
    for (int i = r0 + warp; i < r1; i += kElocWarps) {
      const int32_t f = __ldg(field + i);
      fe += ((bit_word(i) >> lane) & 1u) ? -f : f;
    }
  const int pa = __ldg(row_ptr + r0), pb = __ldg(row_ptr + r1);
  uint32_t C[32];
#pragma unroll
  for (int t = 0; t < 32; ++t) C[t] = 0u;
  int32_t ws = 0;
  for (int p = pa + (int)threadIdx.x; p < pb;) {
    uint32_t L[PL];
#pragma unroll
    for (int t = 0; t < PL; ++t) L[t] = 0u;
    for (int k = 0; k < 15 && p < pb; ++k, p += kElocWarps * 32) {
      const int32_t wt = __ldg(w + p);
      const uint32_t x = bit_word(__ldg(erow + p)) ^ bit_word(__ldg(col + p));
      ws += wt;
      uint32_t c = 0;
#pragma unroll
      for (int t = 0; t < PL; ++t) {
        const uint32_t a = ((uint32_t)wt >> t) & 1u ? x : 0u;  // plane t of wt x (two's complement)
        const uint32_t sum = L[t] ^ a ^ c;
        c = (L[t] & a) | (c & (L[t] ^ a));
        L[t] = sum;
      }
    }
    uint32_t a[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) a[t] = L[t < PL ? t : PL - 1];  // sign extension
    add_planes32(C, a);
  }
  // the warp's lanes, then the CTA's warps (fixed order)
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t o[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) o[t] = __shfl_xor_sync(0xffffffffu, C[t], d);
    add_planes32(C, o);
    ws += __shfl_xor_sync(0xffffffffu, ws, d);
  }
  planes[warp][lane] = C[lane];
  fpart[warp][lane] = fe;
  if (lane == 0) wpart[warp] = ws;
  __syncthreads();
  if (warp == 0) {
    uint32_t T[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) T[t] = planes[0][t];
    int32_t wsum = wpart[0], f = fpart[0][lane];
    for (int k = 1; k < kElocWarps; ++k) {
      uint32_t o[32];
#pragma unroll
      for (int t = 0; t < 32; ++t) o[t] = planes[k][t];
      add_planes32(T, o);
      wsum += wpart[k];
      f += fpart[k][lane];
    }
    uint32_t v = 0;  // sample lane's sum of J x (two's complement)
#pragma unroll
    for (int t = 0; t < 32; ++t) v |= ((T[t] >> lane) & 1u) << t;
    const int b = 32 * wd + lane;
    if (b < B) part[(size_t)q * ldp + b] = (int32_t)((uint32_t)wsum - 2u * v) + f;
  }
}

// E_b = sum of the slices' partial energies, in slice order
template <typename A>
__global__ void eloc_sum_kernel(int B, int nslices, const A* __restrict__ part, int ldp, A* __restrict__ E) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  A t = part[b];
  for (int q = 1; q < nslices; ++q) t += part[(size_t)q * ldp + b];
  E[b] = t;
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
// With ds set, thread 0 also starts the next Adam step (t += 1 and its bias
// corrections), which the gradient kernels after it read.  Float energies
// (this kernel); the coefficients (E_b - mean) / B multiply by 1 / B (exact
// for B a power of two; otherwise within one rounding of the quotient before
// the conversion to FP32).  Integer energies: stats_int_kernel below.
template <typename A>
struct StatAcc;
template <>
struct StatAcc<float> {
  using S = double;
  using M = double;
  static __device__ __forceinline__ M lo() { return 1.0 / 0.0; }
  static __device__ __forceinline__ M hi() { return -1.0 / 0.0; }
};

template <typename V>
__device__ __forceinline__ V shfl_down_v(V v, int d) {
  return __shfl_down_sync(0xffffffffu, v, d);
}

// Sum, min and max over the CTA (warp shuffles, then one warp over the 32
// warps' values): the result in every thread.  Fixed order.
template <typename S, typename M>
__device__ __forceinline__ void cta_reduce(S& sum, M& mn, M& mx, S* ws, M* wmn, M* wmx) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    sum += shfl_down_v(sum, d);
    const M a = shfl_down_v(mn, d), b = shfl_down_v(mx, d);
    mn = a < mn ? a : mn;
    mx = b > mx ? b : mx;
  }
  if (lane == 0) ws[warp] = sum, wmn[warp] = mn, wmx[warp] = mx;
  __syncthreads();
  if (warp == 0) {
    sum = ws[lane], mn = wmn[lane], mx = wmx[lane];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      sum += shfl_down_v(sum, d);
      const M a = shfl_down_v(mn, d), b = shfl_down_v(mx, d);
      mn = a < mn ? a : mn;
      mx = b > mx ? b : mx;
    }
    if (lane == 0) ws[0] = sum, wmn[0] = mn, wmx[0] = mx;
  }
  __syncthreads();
  sum = ws[0], mn = wmn[0], mx = wmx[0];
}

template <typename A>
__global__ void __launch_bounds__(1024) stats_kernel(int B, const A* __restrict__ E, double* __restrict__ out,
                                                     float* __restrict__ coef, uint32_t* __restrict__ err,
                                                     DevState* ds, float beta1, float beta2) {
  using S = typename StatAcc<A>::S;
  using M = typename StatAcc<A>::M;
  __shared__ S ws[32];
  __shared__ M wmn[32], wmx[32];
  __shared__ double wv[32];
  __shared__ M dummy_mn[32], dummy_mx[32];
  const int t = threadIdx.x;
  if (ds && t == 0) {
    ds->adam_t += 1;
    adam_factors(ds, beta1, beta2);
  }
  S sum = 0;
  M mn = StatAcc<A>::lo(), mx = StatAcc<A>::hi();
  for (int b = t; b < B; b += blockDim.x) {
    const A x = E[b];
    sum += (S)x;
    mn = (M)x < mn ? (M)x : mn;
    mx = (M)x > mx ? (M)x : mx;
  }
  cta_reduce(sum, mn, mx, ws, wmn, wmx);
  const double mean = (double)sum / (double)B;
  double ss = 0.0;
  for (int b = t; b < B; b += blockDim.x) {
    const double d = (double)E[b] - mean;
    ss += d * d;
  }
  M u0 = 0, u1 = 0;
  cta_reduce(ss, u0, u1, wv, dummy_mn, dummy_mx);
  if (t == 0) {
    const double var = ss / (double)B;
    out[0] = mean;
    out[1] = var;
    out[2] = (double)mn;
    out[3] = (double)mx;
    if (!isfinite(mean) || !isfinite(var)) atomicOr(err, kErrNonfinite);
  }
  if (coef) {
    const double inv = 1.0 / (double)B;
    for (int b = t; b < B; b += blockDim.x) coef[b] = (float)(((double)E[b] - mean) * inv);
  }
}

// Integer energies: the same statistics with integer arithmetic only
// (FP64 is slow on this part).  mean = S / B from S = sum E (int64); the
// variance (B Q - S^2) / B^2 from Q = sum E^2 (128-bit integers: exact before
// its one rounding); the coefficients (B E_b - S) / B^2 as an FP32 product,
// equal to the FP64 path's (E_b - mean) / B rounded to FP32 when B is a power
// of two (otherwise within about one rounding of it).
__global__ void __launch_bounds__(1024) stats_int_kernel(int B, const int32_t* __restrict__ E, double* __restrict__ out,
                                                         float* __restrict__ coef, uint32_t* __restrict__ err,
                                                         DevState* ds, float beta1, float beta2) {
  __shared__ long long ws[32];
  __shared__ unsigned long long wql[32];
  __shared__ long long wqh[32];
  __shared__ int32_t wmn[32], wmx[32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = (int)(blockDim.x >> 5);
  if (ds && t == 0) {
    ds->adam_t += 1;
    adam_factors(ds, beta1, beta2);
  }
  long long sum = 0;
  __int128 sq = 0;
  int32_t mn = 0x7fffffff, mx = -0x7fffffff - 1;
  for (int b = t; b < B; b += blockDim.x) {
    const long long x = E[b];
    sum += x;
    sq += (__int128)(x * x);
    mn = (int32_t)x < mn ? (int32_t)x : mn;
    mx = (int32_t)x > mx ? (int32_t)x : mx;
  }
  auto reduce_warp = [&]() {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      sum += __shfl_down_sync(0xffffffffu, sum, d);
      const unsigned long long lo = (unsigned long long)sq, olo = __shfl_down_sync(0xffffffffu, lo, d);
      const long long hi = (long long)(sq >> 64), ohi = __shfl_down_sync(0xffffffffu, hi, d);
      sq += (__int128)(((unsigned __int128)(unsigned long long)ohi << 64) | olo);
      const int32_t a = __shfl_down_sync(0xffffffffu, mn, d), c = __shfl_down_sync(0xffffffffu, mx, d);
      mn = a < mn ? a : mn;
      mx = c > mx ? c : mx;
    }
  };
  reduce_warp();
  if (lane == 0) ws[warp] = sum, wql[warp] = (unsigned long long)sq, wqh[warp] = (long long)(sq >> 64),
                 wmn[warp] = mn, wmx[warp] = mx;
  __syncthreads();
  if (warp == 0) {
    sum = lane < nw ? ws[lane] : 0;
    sq = lane < nw ? (__int128)(((unsigned __int128)(unsigned long long)wqh[lane] << 64) | wql[lane]) : 0;
    mn = lane < nw ? wmn[lane] : 0x7fffffff;
    mx = lane < nw ? wmx[lane] : -0x7fffffff - 1;
    reduce_warp();
    if (lane == 0) ws[0] = sum, wql[0] = (unsigned long long)sq, wqh[0] = (long long)(sq >> 64), wmn[0] = mn, wmx[0] = mx;
  }
  __syncthreads();
  const long long S = ws[0];
  const double mean = (double)S / (double)B;
  if (t == 0) {
    const __int128 Q = (__int128)(((unsigned __int128)(unsigned long long)wqh[0] << 64) | wql[0]);
    const __int128 num = (__int128)B * Q - (__int128)S * (__int128)S;  // B^2 var >= 0
    const double var = (double)num / ((double)B * (double)B);
    out[0] = mean;
    out[1] = var;
    out[2] = (double)wmn[0];
    out[3] = (double)wmx[0];
    if (!isfinite(mean) || !isfinite(var)) atomicOr(err, kErrNonfinite);
  }
  if (coef) {
    const float inv2 = (float)(1.0 / ((double)B * (double)B));
    for (int b = t; b < B; b += blockDim.x) coef[b] = (float)((long long)B * E[b] - S) * inv2;
  }
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

template <int PL>
cudaError_t eloc_sliced(const vqmc_ctx* c, int B, void* d_e, cudaStream_t st, bool stage) {
  const size_t smem = stage ? (size_t)c->n * sizeof(uint32_t) : 0;
  auto k = stage ? eloc_sliced_kernel<PL, true> : eloc_sliced_kernel<PL, false>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int ns = c->eloc_slices;
  int32_t* part = ns > 1 ? (int32_t*)c->eloc_part : (int32_t*)d_e;
  k<<<dim3((B + 31) / 32, ns), kElocWarps * 32, smem, st>>>(B, c->n, c->Sbits, c->row_ptr, c->erow, c->col,
                                                           (const int32_t*)c->w, (const int32_t*)c->field,
                                                           c->eloc_slice, part, c->Bmax);
  if (ns > 1) eloc_sum_kernel<int32_t><<<(B + 255) / 256, 256, 0, st>>>(B, ns, part, c->Bmax, (int32_t*)d_e);
  return cudaGetLastError();
}

template <typename W, typename A>
cudaError_t eloc_sparse(const vqmc_ctx* c, int B, void* d_e, cudaStream_t st) {
  const size_t smem = (size_t)c->n * sizeof(uint32_t);
  auto k = eloc_sparse_kernel<W, A>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int ns = c->eloc_slices;
  A* part = ns > 1 ? (A*)c->eloc_part : (A*)d_e;
  k<<<dim3((B + 31) / 32, ns), kElocWarps * 32, smem, st>>>(B, c->n, c->Sbits, c->row_ptr, c->erow, c->col,
                                                           (const W*)c->w, (const W*)c->field, c->eloc_slice, part,
                                                           c->Bmax);
  if (ns > 1) eloc_sum_kernel<A><<<(B + 255) / 256, 256, 0, st>>>(B, ns, part, c->Bmax, (A*)d_e);
  return cudaGetLastError();
}

cudaError_t launch_eloc_sparse(const vqmc_ctx* c, int B, const int8_t* d_s, void* d_e, cudaStream_t st,
                               bool packed, bool beside) {
  if (B <= 0) return cudaSuccess;
  if (!packed) pack_bits_kernel<<<dim3((c->n + 255) / 256, (B + 31) / 32), 256, 0, st>>>(B, c->n, d_s, c->Sbits);
  if (c->ham == VQMC_HAM_SPARSE_I32) {
    // weights of at most 8 bits (magnitude): the bit-sliced kernel
    // beside: the launch shares the GPU with a GEMM, so the spin words are
    // read through L1 instead of taking shared memory
    if (c->eloc_wbits <= 1) return eloc_sliced<6>(c, B, d_e, st, !beside);
    if (c->eloc_wbits <= 4) return eloc_sliced<9>(c, B, d_e, st, !beside);
    if (c->eloc_wbits <= 8) return eloc_sliced<13>(c, B, d_e, st, !beside);
    return eloc_sparse<int32_t, int32_t>(c, B, d_e, st);
  }
  return eloc_sparse<float, float>(c, B, d_e, st);
}

cudaError_t launch_eloc_dense_finish(const vqmc_ctx* c, int B, const int8_t* d_s, void* d_e, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  const int ntiles = (c->n + 127) / 128;
  eloc_dense_finish_kernel<<<(B + 255) / 256, 256, 0, st>>>(B, c->n, ntiles, c->row_part, c->row_part_ld, d_s,
                                                            (const float*)c->field, (float*)d_e);
  return cudaGetLastError();
}

cudaError_t launch_stats(const vqmc_ctx* c, int B, const void* d_e, double* d_stats, float* d_coef,
                         cudaStream_t st, bool advance) {
  if (B <= 0) return cudaSuccess;
  DevState* ds = advance ? c->dstate : nullptr;
  const float b1 = c->cfg.beta1, b2 = c->cfg.beta2;
  if (c->ham == VQMC_HAM_SPARSE_I32)
    stats_int_kernel<<<1, 1024, 0, st>>>(B, (const int32_t*)d_e, d_stats, d_coef, c->err, ds, b1, b2);
  else
    stats_kernel<float><<<1, 1024, 0, st>>>(B, (const float*)d_e, d_stats, d_coef, c->err, ds, b1, b2);
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
