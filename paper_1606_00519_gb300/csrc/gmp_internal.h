// gmp_internal.h - declarations shared by the host runtime and the kernels of
// libgmp.  Not part of the C ABI.
#ifndef GMP_INTERNAL_H_
#define GMP_INTERNAL_H_

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "gmp.h"

namespace gmp {

struct LaunchShape {
  int grid;           // CTAs of the persistent launch
  int warps_per_cta;  // one block of a stream per warp at a time
  size_t smem_bytes;  // dynamic shared memory per CTA
  bool deep;          // the 96-register kernel (more than 16 warps per SM; warps_per_cta <= 4)
};

// warps per SM that the 128-register kernel holds
constexpr int kWideWarpsPerSm = 16;

// shared memory per warp of the 128-register (deep = false) and the
// 96-register (deep = true) kernel
size_t warp_smem_bytes(bool deep);
cudaError_t configure_kernel(bool deep, size_t smem_bytes);
cudaError_t occupancy(int warps_per_cta, size_t smem_bytes, bool deep, int* ctas_per_sm);
cudaError_t launch_decode(const LaunchShape& shape, const gmp_file_desc* files, const uint64_t* item_start,
                          uint32_t n_files, const gmp_file_desc* single, int32_t* status,
                          unsigned long long* counter, uint8_t* scratch, uint64_t slot_bytes, uint64_t shadow_off,
                          uint32_t max_seq, uint32_t max_out, unsigned long long* stats, int collect_stats,
                          int resolve, cudaStream_t stream, int spread = 1);
// compiled architecture of decode_kernel (cudaFuncGetAttributes)
cudaError_t kernel_arch(int* binary_version, int* ptx_version);
cudaError_t launch_batch_prefix(const gmp_file_desc* files, uint32_t n_files, uint64_t* item_start,
                                cudaStream_t stream);

// Stream-format constants (format version 1).
constexpr uint32_t kHeaderBytes = 64;
constexpr uint32_t kBlockFixed = 192;
constexpr uint32_t kMaxSub = 64;
constexpr uint32_t kLitLenSyms = 319;
constexpr uint32_t kOffsetSyms = 30;
// scratch partitions of the pipelined host-to-host calls (work counters
// 48..63 of a context)
constexpr uint32_t kPipeParts = 8;

// GPU compressor (gmp_gpucompress.cu) and its host half (gmp_compress.cpp):
// a block's parse as {literal length, (distance << 8) | match length}.
struct ParseToken {
  uint32_t lit_len, match;
};
int encode_token_blocks(const uint8_t* in, size_t n, const gmp_compress_opts& o, const ParseToken* tok,
                        const uint32_t* count, const uint64_t* first, void* host_out, size_t cap, size_t* out_bytes);
bool compress_opts_ok(const gmp_compress_opts& o);
// records a CUDA failure for gmp_last_cuda_error; returns GMP_ERR_CUDA
int cuda_error(cudaError_t e, const char* what);

}  // namespace gmp

#endif  // GMP_INTERNAL_H_
