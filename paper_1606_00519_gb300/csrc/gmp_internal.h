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
// Flags of a host-to-host launch (device arrays, one word per file of the
// launch; see gmp_host.cpp): in_ready[f] reaches gen when file f's input has
// been copied in (*abort_wait, zeroed before the launch, is set once a wait
// runs out); the kernel sets out_ready[f] to gen when file f is decoded,
// counting its blocks in done[f] and its exiting warps in *exited (both
// zeroed before the launch).  in_ready and abort_wait alone may be given.
// A wait for in_ready gives up after wait_ns of the GPU's global timer.
struct PipeFlags {
  const uint32_t* in_ready;
  uint32_t* abort_wait;
  unsigned long long wait_ns;
  uint32_t* out_ready;
  uint32_t* done;
  uint32_t* exited;
  uint32_t gen;
};
cudaError_t launch_decode(const LaunchShape& shape, const gmp_file_desc* files, const uint64_t* item_start,
                          uint32_t n_files, const gmp_file_desc* single, int32_t* status,
                          unsigned long long* counter, uint8_t* scratch, uint64_t slot_bytes, uint64_t shadow_off,
                          uint32_t max_seq, uint32_t max_out, unsigned long long* stats, int collect_stats,
                          int resolve, cudaStream_t stream, int spread = 1, const PipeFlags* pipe = nullptr);
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
// copy-back streams of the host-to-host calls (their launch uses work
// counter 48 of a context)
constexpr uint32_t kPipeParts = 8;

// GPU compressor (gmp_gpucompress.cu) and its host half (gmp_compress.cpp):
// a block's parse as {literal length, (distance << 8) | match length}.
struct ParseToken {
  uint32_t lit_len, match;
};
// GPU entropy coding of GPU parses (gmp_gpuencode.cu): per block, a plan
// (token checks, code lengths, sub-block split and sizes), then the block's
// bytes at an offset computed from the planned sizes.
struct EncBlockPlan {
  uint64_t bytes, bits;  // encoded size (a multiple of 16), bitstream bits
  uint32_t n_seq, out_bytes, n_lit, err;
  uint32_t sub_first[kMaxSub + 1];  // first token of each sub-block; [K] = n_seq
  uint32_t sub_out[kMaxSub];        // output bytes of each sub-block
  uint64_t sub_bits[kMaxSub];       // bits of each sub-block
  uint8_t lens[kLitLenSyms + kOffsetSyms];
};
struct EncLaunch {
  const uint8_t* in;  // device input
  uint64_t n;
  uint32_t block_size, n_sub, cwl, window, max_match;
  int byte_mode;
  uint64_t n_blocks;
  const ParseToken* tok;  // block b's tokens at tok + b * stride
  const uint32_t* tpos;   // block-relative position of each token's literals
  uint64_t stride;
  const uint32_t* count;  // tokens per block
  EncBlockPlan* plan;
  uint64_t* block_bytes;  // encoded size per block
  int* error;             // set to 1 if a token fails its checks
  unsigned grid;
  cudaStream_t stream;
};
cudaError_t launch_encode_plan(const EncLaunch& L);
cudaError_t launch_encode_write(const EncLaunch& L, const uint64_t* offsets, uint8_t* out);
// Stream layout (gmp_compress.cpp): block offsets (absolute, 16-byte
// aligned) after the header and offset table, and the total size with the
// tail padding; returns the first block's offset.
uint64_t stream_layout(const uint64_t* block_bytes, size_t nb, uint64_t* offsets, uint64_t* total);
// The file header and block offset table at out[0 ..), and the 16 zero bytes
// of tail padding at out[total - 16 ..).
void write_stream_header(const gmp_compress_opts& o, size_t n, size_t nb, const uint64_t* offsets, uint64_t total,
                         uint8_t* out);
bool compress_opts_ok(const gmp_compress_opts& o);
// records a CUDA failure for gmp_last_cuda_error; returns GMP_ERR_CUDA
int cuda_error(cudaError_t e, const char* what);

}  // namespace gmp

#endif  // GMP_INTERNAL_H_
