// tcgen05 tensor-core implementation of the masked GEMMs (BF16 operands, FP32
// accumulation in tensor memory) with the same fused epilogues as the
// CUDA-core path (gemm_simt.cu).  Used for every GEMM of the BF16 precision:
// the log-prob forward (Sec. 2.3), its adjoint (gradient of Sec. 2.1) and the
// dense local energy.
//
// One CTA computes one 128 x 128 output tile with 8 warps:
//   warp 0 allocates 128 TMEM columns; its lane 0 streams K-tiles of A
//          (128 x 64) and B (128 x 64) into a 3-stage shared-memory ring with
//          TMA (cp.async.bulk.tensor, 128-byte swizzle, zero fill beyond the
//          tensor), mbarrier transaction counts marking each stage full;
//   warp 1 lane 0 issues tcgen05.mma (M = 128, N = 128, K = 16, four per
//          K-tile) into the TMEM accumulator and tcgen05.commit-s each stage
//          back to the producer and, after the last K-tile, to the epilogue;
//   all 8 warps run the op's epilogue: warp w reads TMEM lanes
//          32 (w % 4) .. + 31 (its tile rows), columns 64 (w / 4) .. + 63,
//          with tcgen05.ld.  The epilogue operands that do not depend on the
//          accumulator (spins, stored activations, bias; the optimiser state
//          of the fused Adam step) are requested while the main loop runs.
// With ~100 KB of shared memory two CTAs share an SM, so one CTA's epilogue
// overlaps the other's main loop.
//
// The weight-gradient ops can apply the Adam step (Sec. 5.1) in their
// epilogue: a CTA holds the complete gradient of its tile (K = all samples),
// so it updates theta and the moments of the tile's unmasked entries and
// writes the refreshed BF16 weight copies; the gradient itself is not
// stored.  Fully masked tiles then do nothing at all: their weights, moments
// and copies are zero and stay zero.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "gemm.cuh"
#include "tc_ptx.cuh"

namespace vqmc {
namespace {

constexpr int BM = 128, BN = 128, BK = 64, NSTAGE = 3;
constexpr int kThreads = 256;
constexpr int kHalf = BN / 2;  // columns per epilogue thread
constexpr int TILE_A_BYTES = BM * BK * 2;  // 16 KB
constexpr int TILE_B_BYTES = BN * BK * 2;  // 16 KB
constexpr int TMEM_COLS = BN;  // FP32 accumulator: 128 lanes x BN columns
// A stage holds KC consecutive 64-wide K chunks of A and of B: [A chunk
// 0 .. KC-1][B chunk 0 .. KC-1].  With KC = 1 two CTAs share an SM (one's
// epilogue runs beside the other's main loop); with KC = 2 each operand's
// chunks arrive in one 32 KB copy (a 3D view of the operand), which the copy
// engine streams about twice as fast as two 16 KB copies, and one CTA holds
// the SM.  Shared memory: tiles | barriers (256) | column partials [4][BN] |
// bias [BN] | row partials [BM].
constexpr int kNumOps = 6;
// K chunks per stage for each GemmOp, chosen by timing both settings at
// n = 10000, h = 2000, B = 2048: the hidden GEMM and the hidden adjoint gain
// 2-3% from the larger copies; the ops with heavy epilogues (log pi and the
// output adjoint, the fused Adam steps) lose 20-30% without a second CTA
// beside them (dW2 119 -> 144 us, dW1 113 -> 140 us, kOpOut 92 -> 122 us).
constexpr int kStageChunks[kNumOps] = {2, 1, 1, 2, 1, 1};
template <int KC>
struct Stages {
  static constexpr int kStage = KC * (TILE_A_BYTES + TILE_B_BYTES);
  static constexpr int kOffBars = NSTAGE * kStage;
  static constexpr int kOffCol = kOffBars + 256;
  static constexpr int kOffBias = kOffCol + 4 * BN * 4;
  static constexpr int kOffRow = kOffBias + BN * 4;
  static constexpr int kSmem = 1024 /*alignment slack*/ + kOffRow + BM * 4;
  static constexpr int kMinBlocks = KC == 1 ? 2 : 1;
  static_assert(kMinBlocks * kSmem <= 232448, "shared memory per SM");
};

using namespace tc;

// Instruction descriptor of the 128 x 128 tile.
constexpr uint32_t kIdesc = idesc_bf16(BM, BN);

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }

// Sum of v over the 32 lanes for 16 columns by recursive halving: afterwards
// lane l holds the warp's sum of column colsum16_col(l) (lanes 2c and 2c+1
// hold the same value).
__device__ __forceinline__ float colsum16(float (&v)[16], int lane) {
  float x[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const bool up = lane & 16;
    const float keep = up ? v[e + 8] : v[e], send = up ? v[e] : v[e + 8];
    x[e] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float y[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const bool up = lane & 8;
    const float keep = up ? x[e + 4] : x[e], send = up ? x[e] : x[e + 4];
    y[e] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float z[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const bool up = lane & 4;
    const float keep = up ? y[e + 2] : y[e], send = up ? y[e] : y[e + 2];
    z[e] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  const bool up = lane & 2;
  float w = (up ? z[1] : z[0]) + __shfl_xor_sync(0xffffffffu, up ? z[0] : z[1], 2);
  w += __shfl_xor_sync(0xffffffffu, w, 1);
  return w;  // column index within the chunk: 8*b4 + 4*b3 + 2*b2 + b1 of the lane
}
__device__ __forceinline__ int colsum16_col(int lane) {
  return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

// log sigma(x) and sigma(-x) from one exponential: with e = exp(-|x|),
// log sigma(x) = min(x, 0) - log(1 + e) and sigma(-x) = (x >= 0 ? e : 1) / (1 + e).
// The epilogue runs this for every output element, so it uses the hardware
// approximations of exp2/log2 and of the division (relative errors of a few
// 2^-23 for 1 + e in [1, 2], far below the BF16 model's tolerances); where
// e < 2^-24 the log term rounds to 0, an absolute error below 6e-8.
__device__ __forceinline__ float log_one_plus(float e) { return __logf(1.0f + e); }
__device__ __forceinline__ void logsig_pair(float x, float& ls, float& sm) {
  const float e = __expf(-fabsf(x));
  ls = fminf(x, 0.0f) - log_one_plus(e);
  sm = __fdividef(x >= 0.0f ? e : 1.0f, 1.0f + e);
}

// 16 consecutive BF16 values as two 16-byte stores
__device__ __forceinline__ void store16_bf16(bf16* dst, const float (&x)[16]) {
  uint32_t w[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
    w[q] = *reinterpret_cast<const uint32_t*>(&p);
  }
  reinterpret_cast<uint4*>(dst)[0] = make_uint4(w[0], w[1], w[2], w[3]);
  reinterpret_cast<uint4*>(dst)[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// Bits of the 16 spins src[0..15] (bit q set: spin q is -1); columns at or
// past `valid` read as +1.  One 16-byte load when all 16 are inside and the
// address is aligned.
__device__ __forceinline__ uint32_t neg_bits16(const int8_t* src, int valid) {
  uint32_t neg = 0;
  if (valid >= 16 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    const uint4 w = __ldg(reinterpret_cast<const uint4*>(src));
    const uint32_t wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t sg = (wv[k] >> 7) & 0x01010101u;  // sign bit of each byte
      neg |= ((sg * 0x01020408u) >> 24 & 0xFu) << (4 * k);
    }
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q)
      if (q < valid && src[q] < 0) neg |= 1u << q;
  }
  return neg;
}

// Row stride (floats) of a warp's staging block in shared memory: 32 rows x
// 64 columns, padded so that both row- and column-wise accesses are free of
// bank conflicts.
constexpr int kStageLd = kHalf + 1;

// The weight-gradient epilogue of one warp after its 32 x 64 block of the
// gradient (rows m0w.., columns c0..) was staged in G: row r of the block
// keeps columns [kl, kh) of lane r's (kl_me, kh_me).  Lanes run along the
// columns for the row-major arrays (theta, moments, gradient, row copy: one
// 128-byte line per warp access) and along the rows for the transposed copy.
// With the fused Adam step, every kept entry gets one Adam update (Sec. 5.1)
// and the refreshed weight goes to the BF16 copies; otherwise the gradient
// is stored, zero outside the mask.
__device__ __forceinline__ void wgrad_block(const GemmArgs<bf16>& g, bool fused, float* G, int m0w, int c0,
                                            int lane, int kl_me, int kh_me) {
  const float ibc1 = fused ? __ldg(g.ibc) : 0.0f, ibc2 = fused ? __ldg(g.ibc + 1) : 0.0f;
  for (int r0 = 0; r0 < 32; r0 += 4) {
    float gq[8], mq[8], vq[8], tq[8];
    bool keep[8], in[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int r = r0 + (j >> 1), col = lane + 32 * (j & 1);
      const int kl = __shfl_sync(0xffffffffu, kl_me, r), kh = __shfl_sync(0xffffffffu, kh_me, r);
      const int m = m0w + r, k = c0 + col;
      in[j] = m < g.M && k < g.N;
      keep[j] = in[j] && k >= kl && k < kh;
      gq[j] = G[r * kStageLd + col];
      if (fused && keep[j]) {
        const size_t q = (size_t)m * g.ldg + k;
        mq[j] = __ldcs(g.adam_m + q);
        vq[j] = __ldcs(g.adam_v + q);
        tq[j] = __ldcs(g.theta + q);
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int r = r0 + (j >> 1), col = lane + 32 * (j & 1);
      const int m = m0w + r, k = c0 + col;
      const size_t q = (size_t)m * g.ldg + k;
      if (!fused) {
        if (in[j]) g.gout[q] = keep[j] ? gq[j] : 0.0f;
        continue;
      }
      float t = 0.0f;
      if (keep[j]) {
        const float mn = g.beta1 * mq[j] + (1.0f - g.beta1) * gq[j];
        const float vn = g.beta2 * vq[j] + (1.0f - g.beta2) * gq[j] * gq[j];
        t = tq[j] - g.lr * (mn * ibc1) / (sqrtf(vn * ibc2) + g.eps);
        __stcs(g.adam_m + q, mn);
        __stcs(g.adam_v + q, vn);
        __stcs(g.theta + q, t);
        if (g.cp_row) g.cp_row[(size_t)(m + g.cp_shift) * g.ld_cp_row + k] = __float2bfloat16_rn(t);
      }
      G[r * kStageLd + col] = t;
    }
  }
  if (!fused) return;
  __syncwarp();
  const int m = m0w + lane;
  if (m < g.M)
    for (int col = 0; col < kHalf; ++col) {
      const int k = c0 + col;
      if (k >= kl_me && k < kh_me && k < g.N) g.cp_t[(size_t)k * g.ld_cp_t + m] = __float2bfloat16_rn(G[lane * kStageLd + col]);
    }
}

template <int OP, int KC>
__global__ void __launch_bounds__(kThreads, Stages<KC>::kMinBlocks)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   const __grid_constant__ CUtensorMap mapB2, const __grid_constant__ CUtensorMap mapAc,
                   const __grid_constant__ CUtensorMap mapBc, const __grid_constant__ CUtensorMap mapB2c,
                   const GemmArgs<bf16> g, int two_pass, int kfull) {
  using St = Stages<KC>;
  constexpr int STAGE_BYTES = St::kStage, kOffBars = St::kOffBars, kOffCol = St::kOffCol,
                kOffBias = St::kOffBias, kOffRow = St::kOffRow;
  uint32_t* err = g.err;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // 1024-byte aligned tiles (128B swizzle atoms)
  unsigned char* smem = smem_raw + (base - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kOffBars);
  uint64_t* empty = full + NSTAGE;
  uint64_t* done = empty + NSTAGE;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  float* colbuf = reinterpret_cast<float*>(smem + kOffCol);    // [4][BN]
  float* bias_s = reinterpret_cast<float*>(smem + kOffBias);   // [BN]
  float* rowbuf = reinterpret_cast<float*>(smem + kOffRow);    // [BM]

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = warp & 3, half = warp >> 2;
  constexpr int op = OP;
  constexpr bool kWgrad = op == kOpDV || op == kOpDW;
  const bool fused = kWgrad && g.theta != nullptr;
  // Tiles in launch order, heaviest K range first where the masks make the
  // ranges uneven (the hidden GEMM and the output GEMM: K grows with the
  // N-tile; the hidden adjoint: K shrinks with it), so that the last wave
  // holds the light tiles.
  int tm = blockIdx.y, tn = blockIdx.x;
  if constexpr (OP == kOpHidden || OP == kOpGA || OP == kOpOut) {
    const int L = blockIdx.y * gridDim.x + blockIdx.x;  // launch order
    tm = L % gridDim.y;
    tn = OP == kOpGA ? L / (int)gridDim.y : (int)gridDim.x - 1 - L / (int)gridDim.y;
  }
  const int m0 = tm * BM, n0 = tn * BN;
  const int m1 = min(m0 + BM, g.M), n1 = min(n0 + BN, g.N);

  // fully masked weight-gradient tiles: zeros (or, with the fused Adam step, nothing)
  if (kWgrad && gemm_tile_masked(op, m0, m1, n0, n1, g.n, g.h)) {
    if (!fused)
      for (int q = tid; q < BM * BN; q += kThreads) {
        const int m = m0 + q / BN, nn = n0 + q % BN;
        if (m < g.M && nn < g.N) g.gout[(size_t)m * g.ldg + nn] = 0.0f;
      }
    return;
  }
  if (op == kOpOut && g.flip_rows) {
    // flipped spin of the tile's first row; any unflipped row (i = n) or a
    // new sample inside the tile needs every column
    const long long ga = g.row0 + m0;
    const int ia = (int)(ga % (g.n + 1));
    const int last = m1 - 1 - m0;  // rows of the tile after the first
    if (ia + last < g.n && n0 + BN <= ia) return;
  }
  int klo, khi;
  gemm_k_range(op, n0, n1, g.K, g.n, g.h, &klo, &khi);
  const int kt0 = klo / BK;
  const int kt1 = (khi + BK - 1) / BK;
  const int per_pass = kt1 > kt0 ? (kt1 - kt0 + KC - 1) / KC : 0;  // stages per pass
  const int nkt = per_pass * (two_pass ? 2 : 1);

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------- producer
    for (int it = 0; it < nkt && ok; ++it) {
      const int s = it % NSTAGE;
      if (it >= NSTAGE) ok = mbar_wait(smem_u32(&empty[s]), (uint32_t)((it / NSTAGE - 1) & 1), err);
      if (!ok) break;
      const int pass = it / per_pass, kt = kt0 + KC * (it - pass * per_pass);
      const int nch = min(KC, kt1 - kt);  // K chunks of this stage
      const uint32_t sa = base + s * STAGE_BYTES, sb = sa + KC * TILE_A_BYTES;
      const uint32_t bar = smem_u32(&full[s]);
      mbar_expect_tx(bar, (uint32_t)(nch * (TILE_A_BYTES + TILE_B_BYTES)));
      if (KC > 1 && nch == KC && kt + KC <= kfull) {
        // KC whole chunks inside the chunked view (kfull = floor(K / 64))
        tma_load_3d(sa, &mapAc, 0, m0, kt, bar);
        tma_load_3d(sb, pass == 0 ? &mapBc : &mapB2c, 0, n0, kt, bar);
      } else {
        for (int c = 0; c < nch; ++c) {
          tma_load_2d(sa + c * TILE_A_BYTES, &mapA, (kt + c) * BK, m0, bar);
          tma_load_2d(sb + c * TILE_B_BYTES, pass == 0 ? &mapB : &mapB2, (kt + c) * BK, n0, bar);
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // --------------------------------------------------------- MMA issuer
    for (int it = 0; it < nkt && ok; ++it) {
      const int s = it % NSTAGE;
      ok = mbar_poll(smem_u32(&full[s]), (uint32_t)((it / NSTAGE) & 1), err);
      if (!ok) break;
      fence_after();
      const int pass = it / per_pass, kt = kt0 + KC * (it - pass * per_pass);
      const int nch = min(KC, kt1 - kt);
      const uint32_t sa = base + s * STAGE_BYTES, sb = sa + KC * TILE_A_BYTES;
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        if (c >= nch) break;
        const uint64_t da = smem_desc_sw128(sa + c * TILE_A_BYTES), db = smem_desc_sw128(sb + c * TILE_B_BYTES);
#pragma unroll
        for (int k = 0; k < BK / 16; ++k)  // advance 16 BF16 = 32 bytes along K inside the swizzle atom
          mma_bf16(tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), kIdesc,
                   (it > 0 || c > 0 || k > 0) ? 1u : 0u);
      }
      mma_commit(smem_u32(&empty[s]));
    }
    if (nkt > 0 && ok) mma_commit(smem_u32(done));
    else mbar_arrive(smem_u32(done));
  }
  __syncwarp();

  // ------------------------------------ epilogue operands, during the main loop
  const int m = m0 + quad * 32 + lane;  // this thread's tile row
  const bool mvalid = m < g.M;
  const int c0 = n0 + kHalf * half;     // this thread's first column
  if (tid < BN) bias_s[tid] = ((op == kOpHidden || op == kOpOut) && n0 + tid < g.N) ? g.bias[n0 + tid] : 0.0f;
  uint32_t neg[kHalf / 16];  // kOpOut / kOpEloc: bit q of neg[c]: spin of column c0 + 16c + q is -1
  uint4 hpre[kHalf / 8];     // kOpGA: stored activations H[m][c0 .. c0 + 63]
  if constexpr (op == kOpOut || op == kOpEloc) {
#pragma unroll
    for (int c = 0; c < kHalf / 16; ++c)
      neg[c] = mvalid ? neg_bits16(g.S8 + (size_t)m * g.lds8 + c0 + 16 * c, g.N - (c0 + 16 * c)) : 0u;
  }
  if constexpr (op == kOpGA) {
    const bf16* hrow = g.aux + (size_t)m * g.ldaux + c0;
    const bool vec = mvalid && c0 + kHalf <= g.N && (reinterpret_cast<uintptr_t>(hrow) & 15) == 0;
#pragma unroll
    for (int c = 0; c < kHalf / 8; ++c) {
      if (vec) {
        hpre[c] = __ldg(reinterpret_cast<const uint4*>(hrow) + c);
      } else {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int k0 = c0 + 8 * c + 2 * q;
          const uint32_t lo = (mvalid && k0 < g.N) ? (uint32_t)__bfloat16_as_ushort(hrow[8 * c + 2 * q]) : 0u;
          const uint32_t hi = (mvalid && k0 + 1 < g.N) ? (uint32_t)__bfloat16_as_ushort(hrow[8 * c + 2 * q + 1]) : 0u;
          w[q] = lo | (hi << 16);
        }
        hpre[c] = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
  }
  // kept columns of row m in a weight-gradient block: [kl, kh)
  int kl = 0, kh = g.N;
  if constexpr (kWgrad) {
    const int cd = count_deg_le(m, g.n, g.h);  // units with m(k) <= m
    if (op == kOpDV) kh = min(cd, g.N);         // W2[m][k] needs m(k) <= m
    else kl = cd;                               // W1^T[m][k] needs m < m(k)
  }

  // ----------------------------------------------------------- epilogue
  const bool done_ok = mbar_wait(smem_u32(done), 0u, err);
  __syncwarp();
  fence_after();
  __syncthreads();  // bias_s
  const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(kHalf * half);
  // warp-uniform: tcgen05.ld is executed by all lanes of a warp or none
  const bool acc_valid = __all_sync(0xffffffffu, nkt > 0 && done_ok);
  float rowsum = 0.0f;
  const bool want_col = g.col_part && ((op == kOpOut && g.coef) || op == kOpGA);
  const float cm = (op == kOpOut && g.coef && mvalid) ? g.coef[m] : 0.0f;

#pragma unroll
  for (int c = 0; c < kHalf / 16; ++c) {
    float v[16];
    if (acc_valid) {
      tmem_ld16(trow + (uint32_t)(16 * c), v);
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = 0.0f;
    }
    const int nb = c0 + 16 * c;                  // first column of the chunk
    const int lb = nb - n0;                      // its column inside the tile
    const bool full = mvalid && nb + 16 <= g.N;  // all 16 columns inside
    float cs[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) cs[q] = 0.0f;
    if constexpr (op == kOpHidden) {
      float x[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float a = v[q] + bias_s[lb + q];
        if (g.pre && mvalid && nb + q < g.N) g.pre[(size_t)m * g.ldpre + nb + q] = a;
        x[q] = g.act == VQMC_ACT_RELU ? fmaxf(a, 0.0f) : sigmoidf_(a);
      }
      if (full) {
        store16_bf16(g.out + (size_t)m * g.ldo + nb, x);
      } else if (mvalid) {
#pragma unroll
        for (int q = 0; q < 16; ++q)
          if (nb + q < g.N) g.out[(size_t)m * g.ldo + nb + q] = __float2bfloat16_rn(x[q]);
      }
      if (g.out_t)
#pragma unroll
        for (int q = 0; q < 16; ++q)
          if (mvalid && nb + q < g.N) g.out_t[(size_t)(nb + q) * g.ldt + m] = __float2bfloat16_rn(x[q]);
    } else if constexpr (op == kOpOut) {
      float d[16];
      if (g.coef) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const bool in = mvalid && nb + q < g.N;
          const float z = v[q] + bias_s[lb + q];
          const float sgn = (neg[c] >> q) & 1u ? -1.0f : 1.0f;
          float ls, sm;
          logsig_pair(sgn * z, ls, sm);
          if (in) rowsum += ls;
          d[q] = in ? cm * sgn * sm : 0.0f;
          cs[q] = d[q];
        }
      } else {  // log pi only
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const float x = ((neg[c] >> q) & 1u ? -1.0f : 1.0f) * (v[q] + bias_s[lb + q]);
          if (mvalid && nb + q < g.N) rowsum += fminf(x, 0.0f) - log_one_plus(__expf(-fabsf(x)));
        }
      }
      if (g.coef) {
        if (full) {
          store16_bf16(g.out + (size_t)m * g.ldo + nb, d);
        } else if (mvalid) {
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (nb + q < g.N) g.out[(size_t)m * g.ldo + nb + q] = __float2bfloat16_rn(d[q]);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q)
          if (mvalid && nb + q < g.N) g.out_t[(size_t)(nb + q) * g.ldt + m] = __float2bfloat16_rn(d[q]);
      }
    } else if constexpr (op == kOpGA) {
      // the adjoint of the pre-activation: (D V)[m][k] * act'(a), act' from H
      const uint32_t w[8] = {hpre[2 * c].x, hpre[2 * c].y, hpre[2 * c].z, hpre[2 * c].w,
                             hpre[2 * c + 1].x, hpre[2 * c + 1].y, hpre[2 * c + 1].z, hpre[2 * c + 1].w};
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float hv = (q & 1) ? __uint_as_float(w[q >> 1] & 0xffff0000u) : __uint_as_float(w[q >> 1] << 16);
        const bool in = mvalid && nb + q < g.N;
        const float da = g.act == VQMC_ACT_RELU ? (hv > 0.0f ? 1.0f : 0.0f) : hv * (1.0f - hv);
        const float x = in ? v[q] * da : 0.0f;
        if (in) g.out_t[(size_t)(nb + q) * g.ldt + m] = __float2bfloat16_rn(x);
        cs[q] = x;
      }
    } else if constexpr (kWgrad) {
      // staged for the warp's row-wise pass (the ring is free: every MMA has completed)
      float* G = reinterpret_cast<float*>(smem) + warp * 32 * kStageLd;
#pragma unroll
      for (int q = 0; q < 16; ++q) G[lane * kStageLd + 16 * c + q] = v[q];
    } else if constexpr (op == kOpEloc) {
#pragma unroll
      for (int q = 0; q < 16; ++q)
        if (mvalid && nb + q < g.N) rowsum = fmaf((neg[c] >> q) & 1u ? -0.5f : 0.5f, v[q], rowsum);
    }
    if (want_col) {
      const float w = colsum16(cs, lane);
      if ((lane & 1) == 0) colbuf[quad * BN + lb + colsum16_col(lane)] = w;
    }
  }
  if constexpr (kWgrad) {
    __syncwarp();
    wgrad_block(g, fused, reinterpret_cast<float*>(smem) + warp * 32 * kStageLd, m0 + quad * 32, c0, lane, kl, kh);
  }
  constexpr bool kRows = op == kOpOut || op == kOpEloc;
  if (kRows && half == 1) rowbuf[quad * 32 + lane] = rowsum;
  fence_before();
  __syncthreads();
  if (kRows && half == 0 && g.row_part && mvalid)
    g.row_part[(size_t)tn * g.ldr + m] = rowsum + rowbuf[quad * 32 + lane];
  if (want_col && tid < BN && n0 + tid < g.N) {
    const float v = colbuf[tid] + colbuf[BN + tid] + colbuf[2 * BN + tid] + colbuf[3 * BN + tid];
    g.col_part[(size_t)tm * g.ldc + n0 + tid] = v;
  }
  if (warp == 0) {
    fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ------------------------------------------------------------ host side

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_once;
bool g_have_tc = false;

void init_once() {
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess && fn) {
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  g_have_tc = g_encode != nullptr && major == 10 && minor == 3;
  const void* k1[] = {(const void*)gemm_tc_kernel<kOpHidden, 1>, (const void*)gemm_tc_kernel<kOpOut, 1>,
                      (const void*)gemm_tc_kernel<kOpDV, 1>,     (const void*)gemm_tc_kernel<kOpGA, 1>,
                      (const void*)gemm_tc_kernel<kOpDW, 1>,     (const void*)gemm_tc_kernel<kOpEloc, 1>};
  const void* k2[] = {(const void*)gemm_tc_kernel<kOpHidden, 2>, (const void*)gemm_tc_kernel<kOpOut, 2>,
                      (const void*)gemm_tc_kernel<kOpDV, 2>,     (const void*)gemm_tc_kernel<kOpGA, 2>,
                      (const void*)gemm_tc_kernel<kOpDW, 2>,     (const void*)gemm_tc_kernel<kOpEloc, 2>};
  for (const void* k : k1)
    if (g_have_tc && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Stages<1>::kSmem) != cudaSuccess)
      g_have_tc = false;
  for (const void* k : k2)
    if (g_have_tc && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Stages<2>::kSmem) != cudaSuccess)
      g_have_tc = false;
}

bool encode(CUtensorMap* map, const void* ptr, int rows, int cols, int ld) {
  return tc_encode_bf16(map, ptr, rows, cols, ld, BM);
}

}  // namespace

bool tc_encode_bf16(CUtensorMap* map, const void* ptr, int rows, int cols, int ld, int box_rows) {
  if (!gemm_tc_available()) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool tc_encode_bf16_chunks(CUtensorMap* map, const void* ptr, int rows, int cols, int ld, int box_rows,
                           int box_chunks) {
  if (!gemm_tc_available() || cols % BK || box_chunks < 1 || box_chunks > 8) return false;
  // chunk c of row r starts at element r * ld + 64 c: the view covers
  // exactly the rows x cols elements of the 2D matrix
  cuuint64_t dims[3] = {(cuuint64_t)BK, (cuuint64_t)rows, (cuuint64_t)(cols / BK)};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)BK * 2};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, (cuuint32_t)box_chunks};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(ptr), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool gemm_tc_available() {
  std::call_once(g_once, init_once);
  return g_have_tc;
}

cudaError_t launch_gemm_tc_bf16(const GemmArgs<bf16>& a, cudaStream_t st) {
  if (!gemm_tc_available()) return cudaErrorNotSupported;
  if (a.M <= 0 || a.N <= 0) return cudaSuccess;
  // operand row strides must be multiples of 16 bytes, K at least one element
  if ((a.lda * 2) % 16 || (a.ldb * 2) % 16 || a.K <= 0) return cudaErrorInvalidValue;
  CUtensorMap ma, mb, mb2;
  if (!encode(&ma, a.A, a.M, a.K, a.lda) || !encode(&mb, a.Bm, a.N, a.K, a.ldb)) return cudaErrorInvalidValue;
  if (a.Bm2) {
    if (!encode(&mb2, a.Bm2, a.N, a.K, a.ldb)) return cudaErrorInvalidValue;
  } else {
    mb2 = mb;
  }
  dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM);
  const int two = a.Bm2 ? 1 : 0;
  if (a.op < 0 || a.op >= kNumOps) return cudaErrorInvalidValue;
  // K chunks per stage: the chunked views cover the floor(K / 64) whole
  // chunks (the partial last chunk goes through the 2D maps' zero fill)
  const int kfull = a.K / BK;
  const int kc = kfull >= 2 ? kStageChunks[a.op] : 1;
  CUtensorMap mac = ma, mbc = mb, mb2c = mb2;
  if (kc == 2 && (!tc_encode_bf16_chunks(&mac, a.A, a.M, kfull * BK, a.lda, BM, 2) ||
                  !tc_encode_bf16_chunks(&mbc, a.Bm, a.N, kfull * BK, a.ldb, BN, 2) ||
                  (a.Bm2 && !tc_encode_bf16_chunks(&mb2c, a.Bm2, a.N, kfull * BK, a.ldb, BN, 2))))
    return cudaErrorInvalidValue;
  if (kc == 2 && !a.Bm2) mb2c = mbc;
#define VQMC_GEMM_LAUNCH(OP)                                                                                   \
  case OP:                                                                                                     \
    if (kc == 2)                                                                                               \
      gemm_tc_kernel<OP, 2><<<grid, kThreads, Stages<2>::kSmem, st>>>(ma, mb, mb2, mac, mbc, mb2c, a, two, kfull); \
    else                                                                                                       \
      gemm_tc_kernel<OP, 1><<<grid, kThreads, Stages<1>::kSmem, st>>>(ma, mb, mb2, mac, mbc, mb2c, a, two, kfull); \
    break;
  switch (a.op) {
    VQMC_GEMM_LAUNCH(kOpHidden)
    VQMC_GEMM_LAUNCH(kOpOut)
    VQMC_GEMM_LAUNCH(kOpDV)
    VQMC_GEMM_LAUNCH(kOpGA)
    VQMC_GEMM_LAUNCH(kOpDW)
    VQMC_GEMM_LAUNCH(kOpEloc)
    default: return cudaErrorInvalidValue;
  }
#undef VQMC_GEMM_LAUNCH
  return cudaGetLastError();
}

}  // namespace vqmc
