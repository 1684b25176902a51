// Shared description of the masked GEMMs of the MADE forward and adjoint
// passes (Sec. 2.3; gradient of Sec. 2.1), used by the CUDA-core and the
// tcgen05 implementations.
//
// All GEMMs are C[m][n] = sum_k A[m][k] * Bm[n][k] with both operands stored
// K-contiguous ("TN").  With sorted MADE degrees the weight matrices are block
// staircases, so each N-tile only visits the K-range where its weights can be
// non-zero, and fully masked output tiles of the weight gradients are written
// as zeros without a main loop.
#pragma once

#include "common.cuh"

namespace vqmc {

template <typename T>
struct GemmArgs {
  int op;       // GemmOp
  int M, N, K;
  const T* A;
  int lda;
  const T* Bm;
  const T* Bm2;  // second K pass (dense local energy, lo part), or null
  int ldb;
  int n, h;     // model sizes (masks, K ranges)
  int act;
  // epilogue operands
  const float* bias;   // [N]
  const int8_t* S8;    // int8 spins [M][lds8]
  int lds8;
  const float* coef;   // [M] or null
  T* out;              // row-major [M][ldo]
  int ldo;
  T* out_t;            // transposed [N][ldt] (kOpHidden: optional)
  int ldt;
  float* pre;          // kOpHidden, optional: FP32 pre-activations a = S W1^T + b1, [M][ldpre]
  int ldpre;
  // kOpOut over the single-flip expansion of the transverse field (rows
  // g = row0 + m = b (n + 1) + i, i = n the unflipped sample): when set,
  // an output tile whose columns all precede the flipped spin of every row
  // of the tile is skipped (those terms equal the unflipped row's), and its
  // row partials are not written
  int flip_rows;
  long long row0;
  const T* aux;        // [M][ldaux] (H for kOpGA)
  int ldaux;
  float* gout;         // FP32 gradient block [M][ldg]
  int ldg;
  float* row_part;     // [N-tile][ldr]
  int ldr;
  float* col_part;     // [M-tile][ldc]
  int ldc;
  uint32_t* err;       // device error word (bounded waits)
  // Adam step fused into the weight-gradient epilogue (tensor-core path,
  // kOpDV / kOpDW with theta set; gout unused): theta, adam_m and adam_v
  // point at the weight block, [M][ldg]; the refreshed weights also go to
  // the transposed copy cp_t[k][m] (row ld_cp_t) and, if set, to the row
  // copy cp_row[m + cp_shift][k] (row ld_cp_row)
  float* theta;
  float* adam_m;
  float* adam_v;
  T* cp_t;
  int ld_cp_t;
  T* cp_row;
  int ld_cp_row, cp_shift;
  float lr, beta1, beta2, eps;
  const float* ibc;  // device {1 / (1 - beta1^t), 1 / (1 - beta2^t)}
};

// K-range [lo, hi) of the N-tile [n0, n1) (clamped to N) for op.
__host__ __device__ inline void gemm_k_range(int op, int n0, int n1, int K, int n, int h, int* lo, int* hi) {
  *lo = 0;
  *hi = K;
  if (op == kOpHidden) {
    // unit k reads inputs j' < m(k): the tile's last unit has the largest degree
    *hi = degree(n1 - 1, n, h);
  } else if (op == kOpOut) {
    // output i' reads units with m(k) <= i'
    *hi = count_deg_le(n1 - 1, n, h);
  } else if (op == kOpGA) {
    // unit k feeds outputs i' >= m(k)
    *lo = degree(n0, n, h);
  }
  if (*hi > K) *hi = K;
  if (*lo > *hi) *lo = *hi;
}

// True if every output of tile [m0,m1) x [n0,n1) is outside the mask (weight
// gradient ops only).
__host__ __device__ inline bool gemm_tile_masked(int op, int m0, int m1, int n0, int n1, int n, int h) {
  if (op == kOpDV) return degree(n0, n, h) > m1 - 1;        // need m(k) <= i'
  if (op == kOpDW) return m0 >= degree(n1 - 1, n, h);       // need j' < m(k)
  return false;
}

__host__ __device__ inline bool gemm_out_kept(int op, int m, int k, int n, int h) {
  if (op == kOpDV) return degree(k, n, h) <= m;
  if (op == kOpDW) return m < degree(k, n, h);
  return true;
}

cudaError_t launch_gemm_simt_f32(const GemmArgs<float>& a, cudaStream_t st);
// tcgen05 path (BF16 operands, FP32 accumulation in tensor memory).
cudaError_t launch_gemm_tc_bf16(const GemmArgs<bf16>& a, cudaStream_t st);
bool gemm_tc_available();

}  // namespace vqmc
