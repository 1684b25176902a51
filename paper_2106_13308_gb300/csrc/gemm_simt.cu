// CUDA-core (FFMA) implementation of the masked GEMMs with fused epilogues:
// the plain FP32 precision (FP32 operands, FP32 accumulation).  The BF16
// precision runs the same GEMMs on the tcgen05 tensor cores (gemm_tc.cu).
//
// Tile 128 x 128 x 16, 256 threads, 8 x 8 outputs per thread (rows
// m0 + 8*ty + i, columns n0 + 8*tx + j), register-staged double buffering.
#include "gemm.cuh"

namespace vqmc {
namespace {

constexpr int BM = 128, BN = 128, BK = 16;

template <typename T>
struct Vec8;
template <>
struct Vec8<float> {
  static __device__ __forceinline__ void load(const float* p, float* v) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    const float4 b = *reinterpret_cast<const float4*>(p + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  }
};
template <>
struct Vec8<bf16> {
  static __device__ __forceinline__ void load(const bf16* p, float* v) {
    const uint4 q = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      v[2 * e] = __uint_as_float(w[e] << 16);
      v[2 * e + 1] = __uint_as_float(w[e] & 0xffff0000u);
    }
  }
};

template <typename T>
__device__ __forceinline__ float to_f(T x);
template <>
__device__ __forceinline__ float to_f<float>(float x) { return x; }
template <>
__device__ __forceinline__ float to_f<bf16>(bf16 x) { return __bfloat162float(x); }
template <typename T>
__device__ __forceinline__ T of_f(float x);
template <>
__device__ __forceinline__ float of_f<float>(float x) { return x; }
template <>
__device__ __forceinline__ bf16 of_f<bf16>(float x) { return __float2bfloat16_rn(x); }

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }
// log sigma(x) and sigma(-x) of an output element from one exponential,
// e = exp(-|x|): log sigma(x) = min(x, 0) - log(1 + e), sigma(-x) =
// (x >= 0 ? e : 1) / (1 + e), on the hardware exp2/log2 approximations and
// the approximate division (absolute error of the log term below 4e-7 for
// 1 + e in (1, 2], relative error of sigma a few 2^-23: far inside the FP32
// model's tolerances on log pi and the gradient)
__device__ __forceinline__ void log_sigmoid_pair(float x, float& ls, float& sm) {
  const float e = __expf(-fabsf(x));
  ls = fminf(x, 0.0f) - __logf(1.0f + e);
  sm = __fdividef(x >= 0.0f ? e : 1.0f, 1.0f + e);
}

// 8 consecutive K-elements of row r starting at k (zeros outside [.., khi) or r >= R)
template <typename T>
__device__ __forceinline__ void load8(const T* base, int ld, int r, int R, int k, int khi, float* v) {
  if (r < R && k + 8 <= khi) {
    Vec8<T>::load(base + (size_t)r * ld + k, v);
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = (r < R && k + e < khi) ? to_f(base[(size_t)r * ld + k + e]) : 0.0f;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) gemm_simt_kernel(const GemmArgs<T> g) {
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN + 4];
  __shared__ float colbuf[16][BN];

  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int m1 = min(m0 + BM, g.M), n1 = min(n0 + BN, g.N);
  const int op = g.op;

  if (op == kOpDV || op == kOpDW) {
    if (gemm_tile_masked(op, m0, m1, n0, n1, g.n, g.h)) {
      for (int q = tid; q < BM * BN; q += 256) {
        const int m = m0 + q / BN, nn = n0 + q % BN;
        if (m < g.M && nn < g.N) g.gout[(size_t)m * g.ldg + nn] = 0.0f;
      }
      return;
    }
  }
  if (op == kOpOut && g.flip_rows) {
    // single-flip rows of the transverse field: a tile whose columns all
    // precede the flipped spin of each of its rows (one sample, no unflipped
    // row) contributes nothing the log-ratios read, so it is skipped
    const long long ga = g.row0 + m0;
    const int ia = (int)(ga % (g.n + 1));
    const int last = m1 - 1 - m0;
    if (ia + last < g.n && n0 + BN <= ia) return;
  }
  int klo, khi;
  gemm_k_range(op, n0, n1, g.K, g.n, g.h, &klo, &khi);
  klo = klo / BK * BK;

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

  const int lr = tid >> 1, lk = (tid & 1) * 8;
  const int passes = g.Bm2 ? 2 : 1;
  for (int pass = 0; pass < passes; ++pass) {
    const T* Bmat = pass == 0 ? g.Bm : g.Bm2;
    float ra[8], rb[8];
    int k0 = klo;
    if (k0 < khi) {
      load8(g.A, g.lda, m0 + lr, g.M, k0 + lk, khi, ra);
      load8(Bmat, g.ldb, n0 + lr, g.N, k0 + lk, khi, rb);
    }
    int buf = 0;
    for (; k0 < khi; k0 += BK) {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        As[buf][lk + e][lr] = ra[e];
        Bs[buf][lk + e][lr] = rb[e];
      }
      __syncthreads();
      if (k0 + BK < khi) {
        load8(g.A, g.lda, m0 + lr, g.M, k0 + BK + lk, khi, ra);
        load8(Bmat, g.ldb, n0 + lr, g.N, k0 + BK + lk, khi, rb);
      }
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8 + 4]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 8]);
        const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 8 + 4]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
      buf ^= 1;
    }
    __syncthreads();
  }

  // ---------------------------------------------------------------- epilogue
  const int mb = m0 + ty * 8, nb = n0 + tx * 8;
  float rowsum[8], colsum[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) rowsum[i] = 0.0f, colsum[i] = 0.0f;

  if (op == kOpHidden) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int m = mb + i;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int nn = nb + j;
        if (m < g.M && nn < g.N) {
          float v = acc[i][j] + g.bias[nn];
          if (g.pre) g.pre[(size_t)m * g.ldpre + nn] = v;
          v = g.act == VQMC_ACT_RELU ? fmaxf(v, 0.0f) : sigmoidf_(v);
          const T tv = of_f<T>(v);
          g.out[(size_t)m * g.ldo + nn] = tv;
          if (g.out_t) g.out_t[(size_t)nn * g.ldt + m] = tv;
        }
      }
    }
  } else if (op == kOpOut) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int m = mb + i;
      const float cm = (g.coef && m < g.M) ? g.coef[m] : 0.0f;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int nn = nb + j;
        if (m < g.M && nn < g.N) {
          const float z = acc[i][j] + g.bias[nn];
          const float s = g.S8[(size_t)m * g.lds8 + nn] > 0 ? 1.0f : -1.0f;
          float ls, sm;
          log_sigmoid_pair(s * z, ls, sm);
          rowsum[i] += ls;
          if (g.coef) {
            const float d = cm * s * sm;
            const T tv = of_f<T>(d);
            g.out[(size_t)m * g.ldo + nn] = tv;
            g.out_t[(size_t)nn * g.ldt + m] = tv;
            colsum[j] += d;
          }
        }
      }
    }
  } else if (op == kOpGA) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int m = mb + i;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int nn = nb + j;
        if (m < g.M && nn < g.N) {
          const float hv = to_f(g.aux[(size_t)m * g.ldaux + nn]);
          const float dact = g.act == VQMC_ACT_RELU ? (hv > 0.0f ? 1.0f : 0.0f) : hv * (1.0f - hv);
          const float v = acc[i][j] * dact;
          g.out_t[(size_t)nn * g.ldt + m] = of_f<T>(v);
          colsum[j] += v;
        }
      }
    }
  } else if (op == kOpDV || op == kOpDW) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int m = mb + i;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int nn = nb + j;
        if (m < g.M && nn < g.N)
          g.gout[(size_t)m * g.ldg + nn] = gemm_out_kept(op, m, nn, g.n, g.h) ? acc[i][j] : 0.0f;
      }
    }
  } else if (op == kOpEloc) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int m = mb + i;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int nn = nb + j;
        if (m < g.M && nn < g.N) {
          const float s = g.S8[(size_t)m * g.lds8 + nn] > 0 ? 0.5f : -0.5f;
          rowsum[i] = fmaf(s, acc[i][j], rowsum[i]);
        }
      }
    }
  }

  // row partials: reduce over the 16 tx lanes of each half-warp
  if (g.row_part && (op == kOpOut || op == kOpEloc)) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float v = rowsum[i];
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      v += __shfl_xor_sync(0xffffffffu, v, 4);
      v += __shfl_xor_sync(0xffffffffu, v, 8);
      if (tx == 0 && mb + i < g.M) g.row_part[(size_t)blockIdx.x * g.ldr + mb + i] = v;
    }
  }
  // column partials: reduce over the 16 ty rows in a fixed order
  if (g.col_part && ((op == kOpOut && g.coef) || op == kOpGA)) {
#pragma unroll
    for (int j = 0; j < 8; ++j) colbuf[ty][tx * 8 + j] = colsum[j];
    __syncthreads();
    if (tid < BN) {
      float v = 0.0f;
#pragma unroll
      for (int q = 0; q < 16; ++q) v += colbuf[q][tid];
      if (n0 + tid < g.N) g.col_part[(size_t)blockIdx.y * g.ldc + n0 + tid] = v;
    }
  }
}

template <typename T>
cudaError_t launch_simt(const GemmArgs<T>& a, cudaStream_t st) {
  if (a.M <= 0 || a.N <= 0) return cudaSuccess;
  dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM);
  gemm_simt_kernel<T><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_simt_f32(const GemmArgs<float>& a, cudaStream_t st) { return launch_simt(a, st); }

}  // namespace vqmc
