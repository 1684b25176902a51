// vqmc_logprob_noalloc: the log-prob forward of vqmc_logprob for callers that
// cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not an option -- inside a
// host framework whose memory is entirely owned by its own pool allocator, on
// a serving path with a fixed memory budget that must never grow, or where a
// cudaMalloc/cudaFree (which can synchronise the device) would stall other
// work.  vqmc_logprob itself allocates nothing per call either, but its
// scratch lives in the context, sized for max_batch when the context is
// created; this entry point instead takes its scratch from one static device
// array of fixed size, so the call's memory footprint is known up front and
// independent of the context's max_batch.
//
// The scratch is a file-scope __device__ array of kNoAllocScratchBytes
// (64 MiB).  Every GPU that loads this library's module holds it until the
// process exits.  In host code the array's name is not a device address, so
// the entry point looks the address up once per device with
// cudaGetSymbolAddress (the first call on a device does that set-up; make the
// first call before any stream capture) and passes that address to the
// kernels.  All calls share the array: calls that overlap on the GPU (other
// streams, other threads) race on it.  Every scratch value a call reads is
// written by the same call first, so nothing needs clearing between calls.
#include <mutex>
#include <string>
#include <unordered_map>

#include "common.cuh"
#include "gemm.cuh"

namespace vqmc {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
std::unordered_map<int, unsigned char*> g_scratch_addr;  // device -> device address of g_noalloc_scratch

// Device address of the scratch array on the current device (set up once).
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_scratch_addr.find(dev);
  if (it != g_scratch_addr.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  *out = static_cast<unsigned char*>(p);
  return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

__global__ void row_total_kernel(int B, int ntiles, const float* __restrict__ part, int ld, float* __restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float s = 0.0f;
  for (int t = 0; t < ntiles; ++t) s += part[(size_t)t * ld + b];
  out[b] = s;
}

template <typename T>
cudaError_t forward(const vqmc_ctx* c, int B, const int8_t* d_s, float* d_logp, unsigned char* scratch, int ldb,
                    cudaStream_t st) {
  const size_t es = sizeof(T);
  // scratch layout: spin operand Sx [B][np], hidden activations H [B][hp],
  // log-pi partial sums [ceil(n/128)][ldb]; each part 256-byte aligned
  T* Sx = reinterpret_cast<T*>(scratch);
  T* H = reinterpret_cast<T*>(scratch + align256((size_t)B * c->np * es));
  float* part = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(H) + align256((size_t)B * c->hp * es));
  const int ntiles = (c->n + 127) / 128;

  cudaError_t e = launch_spins_to_operands(c, B, d_s, Sx, nullptr, st);
  if (e != cudaSuccess) return e;

  GemmArgs<T> a{};
  a.n = c->n, a.h = c->h, a.act = c->act, a.err = c->err;
  a.op = kOpHidden;
  a.M = B, a.N = c->h, a.K = c->n;
  a.A = Sx, a.lda = c->np;
  a.Bm = reinterpret_cast<const T*>(c->w_s), a.ldb = c->np;
  a.bias = c->b1;
  a.out = H, a.ldo = c->hp;
  a.out_t = nullptr;  // the transposed activations feed only the adjoint, which this call does not run
  GemmArgs<T> z{};
  z.n = c->n, z.h = c->h, z.act = c->act, z.err = c->err;
  z.op = kOpOut;
  z.M = B, z.N = c->n, z.K = c->h;
  z.A = H, z.lda = c->hp;
  z.Bm = reinterpret_cast<const T*>(c->v_s), z.ldb = c->hp;
  z.bias = c->b2;
  z.S8 = d_s, z.lds8 = c->n;
  z.row_part = part, z.ldr = ldb;
  if constexpr (sizeof(T) == 2) {
    e = launch_gemm_tc_bf16(a, st);
    if (e == cudaSuccess) e = launch_gemm_tc_bf16(z, st);
  } else {
    e = launch_gemm_simt_f32(a, st);
    if (e == cudaSuccess) e = launch_gemm_simt_f32(z, st);
  }
  if (e != cudaSuccess) return e;
  row_total_kernel<<<(B + 255) / 256, 256, 0, st>>>(B, ntiles, part, ldb, d_logp);
  return cudaGetLastError();
}

}  // namespace

size_t noalloc_scratch_bytes(const vqmc_ctx* c, int B) {
  const size_t es = c->prec == VQMC_PREC_BF16 ? 2 : 4;
  const size_t ldb = (size_t)pad_up(B);
  return align256((size_t)B * c->np * es) + align256((size_t)B * c->hp * es) +
         align256((size_t)((c->n + 127) / 128) * ldb * 4);
}

}  // namespace vqmc

extern "C" vqmc_status vqmc_logprob_noalloc(vqmc_ctx* c, int32_t B, const int8_t* d_s, float* d_logp,
                                            vqmc_stream stream) {
  using namespace vqmc;
  if (!c) return set_last_error(VQMC_ERR_INVALID_ARG, "null context");
  if (B < 0 || B > c->Bmax) return set_last_error(VQMC_ERR_INVALID_ARG, "batch size outside [0, max_batch]");
  if (B == 0) return VQMC_OK;
  if (!d_s || !d_logp) return set_last_error(VQMC_ERR_INVALID_ARG, "null argument");
  const size_t need = noalloc_scratch_bytes(c, B);
  if (need > kNoAllocScratchBytes)
    return set_last_error(VQMC_ERR_UNSUPPORTED,
                          "vqmc_logprob_noalloc: this batch needs " + std::to_string(need) +
                              " bytes of scratch, above the fixed limit of " +
                              std::to_string(kNoAllocScratchBytes) + " bytes; use a smaller B or vqmc_logprob");
  unsigned char* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess)
    return set_last_error(VQMC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  cudaStream_t st = (cudaStream_t)stream;
  const int ldb = pad_up(B);
  e = c->prec == VQMC_PREC_BF16 ? forward<bf16>(c, B, d_s, d_logp, scratch, ldb, st)
                                : forward<float>(c, B, d_s, d_logp, scratch, ldb, st);
  if (e != cudaSuccess) return set_last_error(VQMC_ERR_CUDA, std::string("noalloc forward: ") + cudaGetErrorString(e));
  return VQMC_OK;
}
