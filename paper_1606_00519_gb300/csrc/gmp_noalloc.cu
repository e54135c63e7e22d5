// gmp_noalloc.cu - decompression of one stream without any device
// allocation.
//
// Some callers cannot call cudaMalloc: host callbacks and other code where
// re-entering the CUDA allocator is not allowed, and applications whose
// memory manager owns the whole device and forbids allocations by
// libraries.  gmp_decompress needs a context, and creating one allocates its
// scratch.  This entry point instead uses a scratch area that lives in a
// file-scope __device__ array of fixed size, so the library loads it with the
// module and the call itself allocates nothing.  The caller still provides
// the stream, the block index, the output buffer and the status word.
//
// Limits: blocks of at most kMaxBlockOut (256 KiB) of output, decoded by
// kSlots (32) warps at a time.  The array holds one scratch slot per warp plus
// a header with the work counter; every GPU that loads this library keeps
// about 53 MB of it until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "gmp.h"
#include "gmp_internal.h"

namespace {

constexpr uint32_t kMaxBlockOut = 256u << 10;
constexpr uint32_t kSlots = 32;
constexpr uint32_t kWarpsPerCta = 4;
constexpr uint32_t kMaxSeq = kMaxBlockOut / 3 + 2;
constexpr uint64_t kRecBytes = ((uint64_t)kMaxSeq * 16 + 255) & ~uint64_t(255);
constexpr uint64_t kShadowBytes = (uint64_t)kMaxBlockOut + 16ull * gmp::kMaxSub + 64;
constexpr uint64_t kSlotBytes = (kRecBytes + kShadowBytes + 255) & ~uint64_t(255);
constexpr uint64_t kHeaderBytes = 256;  // work counter and statistics words
constexpr uint64_t kScratchBytes = kHeaderBytes + kSlotBytes * kSlots;
// device addresses of the scratch, one per CUDA context that has called
// (a context's id is never reused within the process, unlike its handle)
constexpr int kMaxContexts = 64;
struct CtxAddr {
  unsigned long long ctx_id;
  uint8_t* addr;
};
std::mutex g_mu;
CtxAddr g_addr[kMaxContexts] = {};
int g_n_addr = 0;

}  // namespace

// The scratch of gmp_decompress_noalloc.  In host code this name is only a
// stand-in for the device object; kernels receive the device address that
// cudaGetSymbolAddress returns in the current context.
static __device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

namespace {

// Id of the calling thread's current CUDA context; false if there is none.
// The two driver calls are fetched through the runtime, so the library does
// not link the driver library itself.  Called with g_mu held.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return false;
    get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext c = nullptr;
  return get_current(&c) == CUDA_SUCCESS && c && get_id(c, id) == CUDA_SUCCESS;
}

// Device address of the scratch in the current context.  The address is the
// array's instance in one context: a context made after cudaDeviceReset, or
// another context current on the same device, has its own.  So the set-up
// (cudaGetSymbolAddress, which also loads this file's module and makes the
// device's primary context current if no context is) runs once per context,
// keyed by the context's id, and later calls look the address up.
int scratch_address(uint8_t** out) {
  unsigned long long id = 0;
  std::lock_guard<std::mutex> g(g_mu);
  if (current_context_id(&id)) {
    for (int i = 0; i < g_n_addr; i++)
      if (g_addr[i].ctx_id == id) {
        *out = g_addr[i].addr;
        return GMP_OK;
      }
  }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) return gmp::cuda_error(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                                                     "cudaGetSymbolAddress");
  if (!current_context_id(&id)) return GMP_ERR_CUDA;
  // a full table starts over (only a process that cycles through more than
  // kMaxContexts contexts gets here)
  if (g_n_addr == kMaxContexts) g_n_addr = 0;
  g_addr[g_n_addr++] = CtxAddr{id, static_cast<uint8_t*>(p)};
  *out = static_cast<uint8_t*>(p);
  return GMP_OK;
}

}  // namespace

extern "C" {

void gmp_noalloc_limits(uint32_t* max_block_out, uint32_t* warps, uint64_t* scratch_bytes) {
  if (max_block_out) *max_block_out = kMaxBlockOut;
  if (warps) *warps = kSlots;
  if (scratch_bytes) *scratch_bytes = kScratchBytes;
}

int gmp_decompress_noalloc(const uint8_t* d_comp, size_t comp_bytes, const gmp_block_ref* d_index,
                           size_t n_blocks, uint32_t max_block_out, uint8_t* d_out, size_t out_cap,
                           int32_t* d_status, void* stream) {
  if (!d_status || (n_blocks && (!d_comp || !d_index || !d_out))) return GMP_ERR_INVALID_ARG;
  if (((uintptr_t)d_comp & 15) || (n_blocks && comp_bytes < gmp::kHeaderBytes)) return GMP_ERR_INVALID_ARG;
  if (max_block_out > kMaxBlockOut) return GMP_ERR_CAPACITY;
  uint8_t* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess) return GMP_ERR_CUDA;
  if (n_blocks == 0) return GMP_OK;
  // the work counter (and the statistics words after it) must start at zero
  if (cudaMemsetAsync(scratch, 0, kHeaderBytes, s) != cudaSuccess) return GMP_ERR_CUDA;
  gmp::LaunchShape shape;
  shape.warps_per_cta = (int)kWarpsPerCta;
  shape.smem_bytes = kWarpsPerCta * gmp::warp_smem_bytes(false);
  shape.deep = false;
  shape.grid = (int)(kSlots / kWarpsPerCta);
  const uint64_t ctas_needed = (n_blocks + kWarpsPerCta - 1) / kWarpsPerCta;
  if ((uint64_t)shape.grid > ctas_needed) shape.grid = (int)ctas_needed;
  gmp_file_desc F{d_comp, comp_bytes, d_index, n_blocks, d_out, out_cap};
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(scratch);
  cudaError_t e = gmp::launch_decode(shape, nullptr, nullptr, 0, &F, d_status, counter, scratch + kHeaderBytes,
                                     kSlotBytes, kRecBytes, kMaxSeq, kMaxBlockOut, counter + 8, 0, 0, s);
  return e == cudaSuccess ? GMP_OK : GMP_ERR_CUDA;
}

}  // extern "C"
