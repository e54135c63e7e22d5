// gmp_host.cpp - host runtime of libgmp: stream header and block index,
// decoder contexts (scratch sizing, launch shape), launches, CUDA graphs of
// batched launches, statistics, and the host-to-host convenience call.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "gmp.h"
#include "gmp_internal.h"

namespace {

thread_local std::string g_cuda_err;

int cuda_fail(cudaError_t e, const char* what) {
  g_cuda_err = std::string(what) + ": " + cudaGetErrorString(e);
  return GMP_ERR_CUDA;
}
#define GMP_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

uint32_t rd16(const uint8_t* p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 8); }
uint32_t rd32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
uint64_t rd64(const uint8_t* p) { return (uint64_t)rd32(p) | ((uint64_t)rd32(p + 4) << 32); }

// Restores the caller's current device when a call returns.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Stream memory operations of the host-to-host pipeline: a copy stream
// writes a word once the copies before it have completed (with a memory
// barrier first), or waits until a word reaches a value (cyclic >=).  The
// driver functions are fetched through the runtime, so the library does not
// link the driver library itself.
using StreamValueFn = CUresult (*)(CUstream, CUdeviceptr, cuuint32_t, unsigned int);
struct StreamValueOps {
  StreamValueFn write = nullptr, wait = nullptr;
};
const StreamValueOps* stream_value_ops() {
  static StreamValueOps ops;
  static std::once_flag once;
  std::call_once(once, [] {
    void* w = nullptr;
    void* t = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuStreamWriteValue32", &w, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuStreamWaitValue32", &t, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess && w && t) {
      ops.write = reinterpret_cast<StreamValueFn>(w);
      ops.wait = reinterpret_cast<StreamValueFn>(t);
    }
  });
  return ops.write ? &ops : nullptr;
}
int cu_fail(CUresult r, const char* what) {
  g_cuda_err = std::string(what) + ": CUresult " + std::to_string((int)r);
  return GMP_ERR_CUDA;
}

}  // namespace

namespace gmp {
int cuda_error(cudaError_t e, const char* what) { return cuda_fail(e, what); }
}  // namespace gmp

struct gmp_context {
  int device = 0;
  int sm_count = 0;
  gmp_context_opts opts{};
  gmp::LaunchShape shape{};
  int occ_wide = 0, occ_deep = 0;  // CTAs per SM of the two kernels at this shape's warps per CTA
  uint32_t max_seq = 0, max_out = 0;
  uint64_t slot_bytes = 0, shadow_off = 0;
  uint8_t* scratch = nullptr;
  size_t scratch_bytes = 0;
  unsigned long long* counter = nullptr;  // 64 words: [0] work counter, [48, 56) pipeline partitions' counters
  unsigned long long* stats = nullptr;    // counter + 16: 32 statistics words (gmp_stats_read)
  uint64_t* item_start = nullptr;         // batch prefix, max_files + 1
  // staging of gmp_decompress_host
  uint8_t* h_comp = nullptr;
  size_t h_comp_cap = 0;
  uint8_t* h_out = nullptr;
  size_t h_out_cap = 0;
  uint8_t* h_meta = nullptr;  // block indexes, piece descriptors, item prefix
  size_t h_meta_cap = 0;
  int32_t* h_status = nullptr;
  size_t h_status_cap = 0;
  // flags of the host-to-host launch: in_ready, out_ready and done, h_flags_n
  // words each, then the exited-warps word; in_ready and out_ready keep the
  // generation numbers of earlier calls (pipe_gen)
  uint32_t* h_flags = nullptr;
  size_t h_flags_n = 0;
  uint32_t pipe_gen = 0;
  unsigned long long input_wait_ns = 10000000000ull;  // the kernel's limit per wait for a piece
  int64_t drop_flag = -1;  // test hook: the next host call does not flag this piece's input
  // streams of the host-to-host calls: the launch, the copies in, the copies
  // back (several, so that a piece whose copy waits does not hold up the
  // others), and events between them
  cudaStream_t pipe = nullptr;
  cudaStream_t h2d = nullptr;
  cudaStream_t d2h[gmp::kPipeParts] = {};
  cudaEvent_t ev[2] = {};
};

struct gmp_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" {

const char* gmp_last_cuda_error(void) { return g_cuda_err.c_str(); }

int gmp_kernel_arch(int* binary_version, int* ptx_version) {
  const cudaError_t e = gmp::kernel_arch(binary_version, ptx_version);
  return e == cudaSuccess ? GMP_OK : gmp::cuda_error(e, "cudaFuncGetAttributes");
}

int gmp_stream_info_parse(const void* host_stream, size_t bytes, gmp_stream_info* info) {
  if (!host_stream || !info) return GMP_ERR_INVALID_ARG;
  const uint8_t* s = static_cast<const uint8_t*>(host_stream);
  if (bytes < gmp::kHeaderBytes || memcmp(s, "GMP1", 4) != 0) return GMP_ERR_FORMAT;
  gmp_stream_info I{};
  I.version = rd16(s + 4);
  I.flags = rd16(s + 6);
  I.block_size = rd32(s + 8);
  I.n_sub = rd16(s + 12);
  I.cwl = s[14];
  I.window = rd32(s + 16);
  I.min_match = s[20];
  I.max_match = s[21];
  I.orig_size = rd64(s + 24);
  I.n_blocks = rd64(s + 32);
  I.stream_bytes = rd64(s + 40);
  if (I.version != GMP_VERSION) return GMP_ERR_UNSUPPORTED;
  if (I.flags & ~3u) return GMP_ERR_UNSUPPORTED;
  const bool huffman = (I.flags & 2u) != 0;  // else byte-level blocks: no trees, no sub-blocks
  if (huffman ? (I.n_sub == 0 || I.n_sub > gmp::kMaxSub || I.cwl == 0 || I.cwl > 12) : (I.n_sub != 0 || I.cwl != 0))
    return GMP_ERR_FORMAT;
  if (I.block_size == 0 || I.window == 0 || I.window > 32768 || I.min_match != 3 || I.max_match < 3 ||
      I.max_match > 64)
    return GMP_ERR_FORMAT;
  if (I.n_blocks != (I.orig_size + I.block_size - 1) / I.block_size) return GMP_ERR_FORMAT;
  if (I.stream_bytes > bytes || I.stream_bytes < gmp::kHeaderBytes + 8 * I.n_blocks) return GMP_ERR_FORMAT;
  *info = I;
  return GMP_OK;
}

int gmp_index_build(const void* host_stream, size_t bytes, gmp_block_ref* out, size_t cap, size_t* n_blocks,
                    gmp_stream_info* info) {
  if (!host_stream || !n_blocks) return GMP_ERR_INVALID_ARG;
  gmp_stream_info I;
  int rc = gmp_stream_info_parse(host_stream, bytes, &I);
  if (rc) return rc;
  *n_blocks = (size_t)I.n_blocks;
  if (cap < I.n_blocks) {
    if (info) *info = I;
    return out || cap ? GMP_ERR_CAPACITY : GMP_OK;
  }
  const uint8_t* s = static_cast<const uint8_t*>(host_stream);
  const uint64_t table_end = gmp::kHeaderBytes + 8 * I.n_blocks;
  const uint64_t blk_hdr = (I.flags & 2u) ? (gmp::kBlockFixed + 12ull * I.n_sub + 15) & ~15ull : 16ull;
  uint32_t max_out = 0, max_seq = 0;
  for (uint64_t b = 0; b < I.n_blocks; b++) {
    uint64_t off = rd64(s + gmp::kHeaderBytes + 8 * b);
    uint64_t next = b + 1 < I.n_blocks ? rd64(s + gmp::kHeaderBytes + 8 * (b + 1)) : I.stream_bytes - 16;
    if ((off & 15) || off < table_end || next < off + blk_hdr || next > I.stream_bytes) return GMP_ERR_FORMAT;
    uint32_t n_seq = rd32(s + off), ob = rd32(s + off + 4);
    uint64_t expect = b + 1 < I.n_blocks ? I.block_size : I.orig_size - b * (uint64_t)I.block_size;
    if (ob != expect) return GMP_ERR_FORMAT;
    out[b].comp_offset = off;
    out[b].comp_bytes = next - off;
    out[b].out_offset = b * (uint64_t)I.block_size;
    out[b].out_bytes = ob;
    max_out = std::max(max_out, ob);
    max_seq = std::max(max_seq, n_seq);
  }
  I.max_block_out = max_out;
  I.max_block_seq = max_seq;
  if (info) *info = I;
  return GMP_OK;
}

void gmp_context_opts_default(gmp_context_opts* o) {
  o->max_block_out = 256u << 10;
  o->warps_per_cta = 0;
  o->ctas_per_sm = 0;
  o->collect_stats = 0;
  o->max_files = 65536;
  o->resolve = GMP_RESOLVE_AUTO;
  o->concurrent = 0;
}

static int context_alloc_scratch(gmp_context* c) {
  // launch shape: persistent grid, as many CTAs per SM as fit
  int wpc = c->opts.warps_per_cta ? (int)c->opts.warps_per_cta : 4;
  if (wpc < 1 || wpc > 16) return GMP_ERR_INVALID_ARG;
  // CTAs per SM of the 128-register kernel and, for CTAs of at most 4 warps,
  // of the 96-register one (each with its own shared memory per warp);
  // shapes beyond the first need the second
  const size_t smem_wide = (size_t)wpc * gmp::warp_smem_bytes(false);
  const size_t smem_deep = (size_t)wpc * gmp::warp_smem_bytes(true);
  int occ_wide = 0, occ_deep = 0;
  GMP_CUDA(gmp::configure_kernel(false, smem_wide));
  GMP_CUDA(gmp::occupancy(wpc, smem_wide, false, &occ_wide));
  if (wpc <= 4) {
    GMP_CUDA(gmp::configure_kernel(true, smem_deep));
    GMP_CUDA(gmp::occupancy(wpc, smem_deep, true, &occ_deep));
  }
  const int occ = std::max(occ_wide, occ_deep);
  if (occ < 1) return GMP_ERR_INVALID_ARG;
  int per_sm = c->opts.ctas_per_sm ? std::min<int>((int)c->opts.ctas_per_sm, occ) : occ;
  c->occ_wide = occ_wide;
  c->occ_deep = occ_deep;
  c->shape.grid = per_sm * c->sm_count;
  c->shape.warps_per_cta = wpc;
  c->shape.deep = per_sm > occ_wide;
  c->shape.smem_bytes = c->shape.deep ? smem_deep : smem_wide;
  // one scratch slot per resident warp: records (16 B per sequence; a block
  // holds at most out/3 + 1 sequences) and the literal shadow (output layout
  // plus 16 bytes of separation per sub-block)
  c->max_out = c->opts.max_block_out;
  c->max_seq = c->max_out / 3 + 2;
  uint64_t rec = ((uint64_t)c->max_seq * 16 + 255) & ~255ull;
  uint64_t shadow = (uint64_t)c->max_out + 16ull * gmp::kMaxSub + 64;
  c->shadow_off = rec;
  c->slot_bytes = (rec + shadow + 255) & ~255ull;
  size_t need = (size_t)c->slot_bytes * (size_t)c->shape.grid * (size_t)wpc;
  if (c->scratch && c->scratch_bytes >= need) return GMP_OK;
  if (c->scratch) cudaFree(c->scratch);
  c->scratch = nullptr;
  c->scratch_bytes = 0;
  GMP_CUDA(cudaMalloc(&c->scratch, need));
  c->scratch_bytes = need;
  return GMP_OK;
}

int gmp_context_create(gmp_context** ctx, int device, const gmp_context_opts* opts) {
  if (!ctx) return GMP_ERR_INVALID_ARG;
  *ctx = nullptr;
  gmp_context* c = new (std::nothrow) gmp_context();
  if (!c) return GMP_ERR_NOMEM;
  if (opts) c->opts = *opts;
  else gmp_context_opts_default(&c->opts);
  if (c->opts.max_block_out == 0 || c->opts.max_block_out > (64u << 20) || c->opts.max_files == 0 ||
      c->opts.resolve > GMP_RESOLVE_SC) {
    delete c;
    return GMP_ERR_INVALID_ARG;
  }
  c->device = device;
  DeviceGuard guard(device);
  cudaError_t e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaDeviceGetAttribute");
  }
  int rc = context_alloc_scratch(c);
  if (rc == GMP_OK) {
    e = cudaMalloc(&c->counter, 64 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&c->item_start, (c->opts.max_files + 1) * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMemset(c->counter, 0, 64 * sizeof(unsigned long long));
    if (e != cudaSuccess) rc = cuda_fail(e, "context alloc");
    c->stats = c->counter + 16;
  }
  if (rc != GMP_OK) {
    gmp_context_destroy(c);
    return rc;
  }
  *ctx = c;
  return GMP_OK;
}

void gmp_context_destroy(gmp_context* c) {
  if (!c) return;
  DeviceGuard guard(c->device);
  if (c->scratch) cudaFree(c->scratch);
  if (c->counter) cudaFree(c->counter);
  if (c->item_start) cudaFree(c->item_start);
  if (c->h_comp) cudaFree(c->h_comp);
  if (c->h_out) cudaFree(c->h_out);
  if (c->h_meta) cudaFree(c->h_meta);
  if (c->h_status) cudaFree(c->h_status);
  if (c->h_flags) cudaFree(c->h_flags);
  if (c->pipe) cudaStreamDestroy(c->pipe);
  if (c->h2d) cudaStreamDestroy(c->h2d);
  for (cudaStream_t t : c->d2h)
    if (t) cudaStreamDestroy(t);
  for (cudaEvent_t e : c->ev)
    if (e) cudaEventDestroy(e);
  delete c;
}

int gmp_context_set_input_wait(gmp_context* c, uint32_t ms) {
  if (!c) return GMP_ERR_INVALID_ARG;
  c->input_wait_ns = (ms ? (unsigned long long)ms : 10000ull) * 1000000ull;
  return GMP_OK;
}

int gmp_context_debug_drop_input_flag(gmp_context* c, int64_t piece) {
  if (!c || piece < -1) return GMP_ERR_INVALID_ARG;
  c->drop_flag = piece;
  return GMP_OK;
}

int gmp_context_set_launch(gmp_context* c, uint32_t warps_per_cta, uint32_t ctas_per_sm) {
  if (!c || warps_per_cta > 16) return GMP_ERR_INVALID_ARG;
  DeviceGuard guard(c->device);
  c->opts.warps_per_cta = warps_per_cta;
  c->opts.ctas_per_sm = ctas_per_sm;
  return context_alloc_scratch(c);
}

size_t gmp_context_scratch_bytes(const gmp_context* c) { return c ? c->scratch_bytes : 0; }

int gmp_decompress(gmp_context* c, const uint8_t* d_comp, size_t comp_bytes, const gmp_block_ref* d_index,
                   size_t n_blocks, uint8_t* d_out, size_t out_cap, int32_t* d_status, void* stream) {
  if (!c || !d_status || (n_blocks && (!d_comp || !d_index || !d_out))) return GMP_ERR_INVALID_ARG;
  if ((uintptr_t)d_comp & 15) return GMP_ERR_INVALID_ARG;
  if (n_blocks && comp_bytes < gmp::kHeaderBytes) return GMP_ERR_INVALID_ARG;
  DeviceGuard guard(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  GMP_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int32_t), s));
  if (n_blocks == 0) return GMP_OK;
  GMP_CUDA(cudaMemsetAsync(c->counter, 0, sizeof(unsigned long long), s));
  gmp_file_desc F{d_comp, comp_bytes, d_index, n_blocks, d_out, out_cap};
  gmp::LaunchShape shape = c->shape;
  // when the 128-register kernel holds a warp for every block, it decodes
  // each block faster; at most one CTA per block, and the kernel spreads the
  // blocks over the CTAs (a CTA's first warp, then its second, ...), so that
  // a small input does not crowd a few SMs
  const uint64_t ctas_needed = (n_blocks + shape.warps_per_cta - 1) / shape.warps_per_cta;
  const uint64_t wide_ctas = (uint64_t)c->occ_wide * (uint64_t)c->sm_count;
  if (shape.deep && ctas_needed <= wide_ctas) {
    shape.deep = false;
    shape.smem_bytes = (size_t)shape.warps_per_cta * gmp::warp_smem_bytes(false);
    if ((uint64_t)shape.grid > wide_ctas) shape.grid = (int)wide_ctas;
  }
  if ((uint64_t)shape.grid > n_blocks) shape.grid = (int)n_blocks;
  GMP_CUDA(gmp::launch_decode(shape, nullptr, nullptr, 0, &F, d_status, c->counter, c->scratch, c->slot_bytes,
                              c->shadow_off, c->max_seq, c->max_out, c->stats, (int)c->opts.collect_stats,
                              (int)c->opts.resolve, s, c->opts.concurrent ? 0 : 1));
  return GMP_OK;
}

int gmp_decompress_batch(gmp_context* c, const gmp_file_desc* d_files, size_t n_files, int32_t* d_status,
                         void* stream) {
  if (!c || (n_files && (!d_files || !d_status))) return GMP_ERR_INVALID_ARG;
  if (n_files > c->opts.max_files) return GMP_ERR_CAPACITY;
  if (n_files == 0) return GMP_OK;
  DeviceGuard guard(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  GMP_CUDA(cudaMemsetAsync(d_status, 0, n_files * sizeof(int32_t), s));
  GMP_CUDA(cudaMemsetAsync(c->counter, 0, sizeof(unsigned long long), s));
  GMP_CUDA(gmp::launch_batch_prefix(d_files, (uint32_t)n_files, c->item_start, s));
  GMP_CUDA(gmp::launch_decode(c->shape, d_files, c->item_start, (uint32_t)n_files, nullptr, d_status, c->counter,
                              c->scratch, c->slot_bytes, c->shadow_off, c->max_seq, c->max_out, c->stats,
                              (int)c->opts.collect_stats, (int)c->opts.resolve, s, c->opts.concurrent ? 0 : 1));
  return GMP_OK;
}

int gmp_batch_graph_create(gmp_context* c, const gmp_file_desc* d_files, size_t n_files, int32_t* d_status,
                           void* stream, gmp_graph** g) {
  if (!c || !g) return GMP_ERR_INVALID_ARG;
  *g = nullptr;
  DeviceGuard guard(c->device);
  cudaStream_t cap;
  GMP_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  gmp_graph* gr = new (std::nothrow) gmp_graph();
  if (!gr) {
    cudaStreamDestroy(cap);
    return GMP_ERR_NOMEM;
  }
  int rc = GMP_OK;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rc = gmp_decompress_batch(c, d_files, n_files, d_status, cap);
    cudaError_t e2 = cudaStreamEndCapture(cap, &gr->graph);
    if (rc == GMP_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "cudaStreamEndCapture");
  } else {
    rc = cuda_fail(e, "cudaStreamBeginCapture");
  }
  if (rc == GMP_OK) {
    e = cudaGraphInstantiate(&gr->exec, gr->graph, 0);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaGraphInstantiate");
  }
  cudaStreamDestroy(cap);
  (void)stream;
  if (rc != GMP_OK) {
    gmp_graph_destroy(gr);
    return rc;
  }
  *g = gr;
  return GMP_OK;
}

int gmp_graph_launch(gmp_graph* g, void* stream) {
  if (!g || !g->exec) return GMP_ERR_INVALID_ARG;
  GMP_CUDA(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)));
  return GMP_OK;
}

void gmp_graph_destroy(gmp_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

int gmp_autotune(gmp_context* c, const gmp_file_desc* d_files, size_t n_files, int32_t* d_status, void* stream,
                 gmp_tuning* out) {
  if (!c || !out || !d_files || !d_status || n_files == 0) return GMP_ERR_INVALID_ARG;
  DeviceGuard guard(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  GMP_CUDA(cudaEventCreate(&e0));
  GMP_CUDA(cudaEventCreate(&e1));
  const gmp_context_opts saved = c->opts;
  double best = 1e300;
  uint32_t best_w = 0, best_c = 0, tried = 0;
  int rc = GMP_OK;
  for (uint32_t w : {1u, 2u, 4u, 8u, 16u}) {
    int occ_wide = 0, occ_deep = 0;
    const size_t smem_wide = (size_t)w * gmp::warp_smem_bytes(false);
    const size_t smem_deep = (size_t)w * gmp::warp_smem_bytes(true);
    if (gmp::configure_kernel(false, smem_wide) != cudaSuccess ||
        gmp::occupancy((int)w, smem_wide, false, &occ_wide) != cudaSuccess)
      continue;
    if (w <= 4 && (gmp::configure_kernel(true, smem_deep) != cudaSuccess ||
                   gmp::occupancy((int)w, smem_deep, true, &occ_deep) != cudaSuccess))
      occ_deep = 0;
    // every SM full with the 96-register kernel, full and half full with the
    // 128-register one
    const int cands[3] = {occ_deep > occ_wide ? occ_deep : 0, occ_wide, occ_wide / 2};
    for (int cps : cands) {
      if (cps < 1 || (cps == occ_wide / 2 && occ_wide / 2 == occ_wide)) continue;
      c->opts.warps_per_cta = w;
      c->opts.ctas_per_sm = (uint32_t)cps;
      if ((rc = context_alloc_scratch(c)) != GMP_OK) break;
      if ((rc = gmp_decompress_batch(c, d_files, n_files, d_status, s)) != GMP_OK) break;
      cudaEventRecord(e0, s);
      for (int r = 0; r < 3 && rc == GMP_OK; r++) rc = gmp_decompress_batch(c, d_files, n_files, d_status, s);
      cudaEventRecord(e1, s);
      if (rc) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "gmp_autotune");
        break;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      tried++;
      if (ms / 3.0 < best) {
        best = ms / 3.0;
        best_w = w;
        best_c = (uint32_t)cps;
      }
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == GMP_OK && tried) {
    c->opts.warps_per_cta = best_w;
    c->opts.ctas_per_sm = best_c;
    rc = context_alloc_scratch(c);
    out->warps_per_cta = best_w;
    out->ctas_per_sm = best_c;
    out->best_ms = best;
    out->shapes_tried = tried;
  } else {
    c->opts = saved;
    int rc2 = context_alloc_scratch(c);
    if (rc == GMP_OK) rc = tried ? rc2 : GMP_ERR_CUDA;
  }
  return rc;
}

int gmp_stats_reset(gmp_context* c, void* stream) {
  if (!c) return GMP_ERR_INVALID_ARG;
  DeviceGuard guard(c->device);
  GMP_CUDA(cudaMemsetAsync(c->stats, 0, 32 * sizeof(unsigned long long), static_cast<cudaStream_t>(stream)));
  return GMP_OK;
}

int gmp_stats_read(gmp_context* c, gmp_stats* out) {
  if (!c || !out) return GMP_ERR_INVALID_ARG;
  DeviceGuard guard(c->device);
  unsigned long long v[32];
  GMP_CUDA(cudaDeviceSynchronize());
  GMP_CUDA(cudaMemcpy(v, c->stats, sizeof(v), cudaMemcpyDeviceToHost));
  out->groups = v[0];
  out->rounds = v[1];
  out->de_fallback_groups = v[2];
  out->blocks = v[3];
  out->max_rounds = v[4];
  out->cycles_tables = v[5];
  out->cycles_huffman = v[6];
  out->cycles_lz77 = v[7];
  for (int i = 0; i < 8; i++) {
    out->detail[i] = v[8 + i];
    out->round_bytes[i] = v[16 + i];
    out->round_groups[i] = v[24 + i];
  }
  return GMP_OK;
}

// Host streams in; outputs in host memory (to_device false: decoded into the
// context's device staging and copied back piece by piece) or in device
// memory (to_device true: decoded straight into the caller's buffers).
//
// One persistent launch decodes every block of every stream.  The blocks are
// cut into pieces (runs of consecutive blocks of one stream), which are the
// files of that launch.  The pieces' compressed bytes are copied in, in
// piece order, on one copy stream; after each copy the stream sets the
// piece's in_ready word, and a warp waits (bounded) for that word before it
// reads any byte of the piece, so the decoding starts with the first piece.
// The kernel sets a piece's out_ready word once all its blocks are decoded,
// and the piece's copy back waits for that word on one of the copy-back
// streams, so outputs go back while later pieces still decode.
//
// A piece's copy in runs on to the next 128-byte boundary of the staging
// (into the next piece's bytes, which that piece's copy writes again with the
// same values), and each stream's staging starts on a 128-byte boundary: the
// cache lines a piece's blocks share with a later piece are then complete
// when the piece is flagged, so no SM caches a line before all of its bytes
// have arrived.
static int decompress_from_host(gmp_context* c, size_t n_files, const void* const* host_streams, const size_t* bytes,
                                void* const* outs, const size_t* out_caps, int32_t* statuses, void* stream,
                                bool to_device) {
  void* const* host_outs = outs;
  if (!c || (n_files && (!host_streams || !bytes || !host_outs || !out_caps || !statuses))) return GMP_ERR_INVALID_ARG;
  DeviceGuard guard(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t drop_flag = c->drop_flag;  // the test hook applies to this call only
  c->drop_flag = -1;
  const StreamValueOps* ops = stream_value_ops();
  if (!ops) return cuda_fail(cudaErrorNotSupported, "cuStreamWriteValue32 / cuStreamWaitValue32 entry points");
  // ---- parse every stream; lay out the device staging
  struct File {
    std::vector<gmp_block_ref> idx;
    gmp_stream_info info;
    uint64_t comp_off, out_off, idx_off;
  };
  std::vector<File> files;
  uint64_t comp_total = 0, out_total = 0, n_total = 0;
  try {
    files.resize(n_files);
    for (size_t f = 0; f < n_files; f++) {
      if (!host_streams[f] || (!host_outs[f] && out_caps[f])) return GMP_ERR_INVALID_ARG;
      size_t nb = 0;
      int rc = gmp_index_build(host_streams[f], bytes[f], nullptr, 0, &nb, &files[f].info);
      if (rc) return rc;
      files[f].idx.resize(nb);
      rc = gmp_index_build(host_streams[f], bytes[f], files[f].idx.data(), nb, &nb, &files[f].info);
      if (rc) return rc;
      if (files[f].info.orig_size > out_caps[f] || files[f].info.max_block_out > c->max_out) return GMP_ERR_CAPACITY;
      files[f].comp_off = comp_total;
      files[f].out_off = out_total;
      files[f].idx_off = n_total;
      comp_total += (bytes[f] + 127) & ~uint64_t(127);
      out_total += (files[f].info.orig_size + 15) & ~uint64_t(15);
      n_total += nb;
    }
  } catch (...) {
    return GMP_ERR_NOMEM;
  }
  // ---- pieces: about kPieces of them, of kPieceMin to kPieceMax blocks.
  // Each piece's copy in ends with a flag write, whose memory barrier keeps
  // the next copy from starting at once: with 128 pieces the copies in of a
  // 0.66 GB input took 4.3-5.9 ms, with 32 about 3.7 ms.
  constexpr uint64_t kPieces = 32, kPieceMin = 8, kPieceMax = 256;
  const uint64_t piece_blocks = std::min(kPieceMax, std::max(kPieceMin, (n_total + kPieces - 1) / kPieces));
  struct Piece {
    size_t file;
    uint64_t b0, b1;
  };
  std::vector<Piece> pieces;
  try {
    for (size_t f = 0; f < n_files; f++)
      for (uint64_t b = 0; b < files[f].idx.size(); b += piece_blocks)
        pieces.push_back(Piece{f, b, std::min<uint64_t>(files[f].idx.size(), b + piece_blocks)});
  } catch (...) {
    return GMP_ERR_NOMEM;
  }
  const size_t n_pieces = pieces.size();
  for (size_t f = 0; f < n_files; f++) statuses[f] = 0;
  if (n_pieces == 0) return GMP_OK;  // only empty streams
  if (n_pieces > (size_t)INT32_MAX) return GMP_ERR_CAPACITY;
  // ---- device buffers (kept in the context): staging, metadata (block
  // indexes, one descriptor per piece, the work-item prefix over the pieces),
  // statuses and flags
  const size_t desc_off = (n_total * sizeof(gmp_block_ref) + 63) & ~size_t(63);
  const size_t pre_off = desc_off + ((n_pieces * sizeof(gmp_file_desc) + 63) & ~size_t(63));
  const size_t meta_bytes = pre_off + (n_pieces + 1) * sizeof(uint64_t);
  auto grow = [&](auto** p, size_t* cap, size_t need) -> int {
    if (*cap >= need) return GMP_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    GMP_CUDA(cudaMalloc((void**)p, need));
    *cap = need;
    return GMP_OK;
  };
  int rc;
  if ((rc = grow(&c->h_comp, &c->h_comp_cap, comp_total))) return rc;
  if (!to_device && (rc = grow(&c->h_out, &c->h_out_cap, std::max<uint64_t>(out_total, 16)))) return rc;
  if ((rc = grow(&c->h_meta, &c->h_meta_cap, meta_bytes))) return rc;
  if ((rc = grow(&c->h_status, &c->h_status_cap, n_pieces * sizeof(int32_t)))) return rc;
  if (c->h_flags_n < n_pieces) {
    if (c->h_flags) cudaFree(c->h_flags);
    c->h_flags = nullptr;
    c->h_flags_n = 0;
    const size_t n = std::max<size_t>(n_pieces, 1024);
    GMP_CUDA(cudaMalloc((void**)&c->h_flags, (3 * n + 2) * sizeof(uint32_t)));
    GMP_CUDA(cudaMemset(c->h_flags, 0, (3 * n + 2) * sizeof(uint32_t)));
    c->h_flags_n = n;
  }
  if (!c->pipe) GMP_CUDA(cudaStreamCreateWithFlags(&c->pipe, cudaStreamNonBlocking));
  if (!c->h2d) GMP_CUDA(cudaStreamCreateWithFlags(&c->h2d, cudaStreamNonBlocking));
  for (uint32_t k = 0; k < gmp::kPipeParts; k++)
    if (!c->d2h[k]) GMP_CUDA(cudaStreamCreateWithFlags(&c->d2h[k], cudaStreamNonBlocking));
  for (cudaEvent_t& e : c->ev)
    if (!e) GMP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  const size_t fn = c->h_flags_n;
  uint32_t* in_ready = c->h_flags;
  uint32_t* out_ready = c->h_flags + fn;
  uint32_t* done = c->h_flags + 2 * fn;  // then the exited-warps word and the abort word
  // Generation of this call: the flags of earlier calls hold smaller ones
  // (compared cyclically); restarted from 1, with the flags cleared, long
  // before the comparison could wrap.
  if (c->pipe_gen >= (1u << 30)) {
    GMP_CUDA(cudaMemsetAsync(c->h_flags, 0, 2 * fn * sizeof(uint32_t), s));
    c->pipe_gen = 0;
  }
  const uint32_t gen = ++c->pipe_gen;
  // ---- metadata, assembled on the host and copied in once
  std::vector<uint8_t> meta;
  try {
    meta.assign(meta_bytes, 0);
  } catch (...) {
    return GMP_ERR_NOMEM;
  }
  gmp_block_ref* m_idx = reinterpret_cast<gmp_block_ref*>(meta.data());
  gmp_file_desc* m_desc = reinterpret_cast<gmp_file_desc*>(meta.data() + desc_off);
  uint64_t* m_pre = reinterpret_cast<uint64_t*>(meta.data() + pre_off);
  const gmp_block_ref* d_idx = reinterpret_cast<const gmp_block_ref*>(c->h_meta);
  for (size_t f = 0; f < n_files; f++)
    if (!files[f].idx.empty())
      memcpy(m_idx + files[f].idx_off, files[f].idx.data(), files[f].idx.size() * sizeof(gmp_block_ref));
  uint64_t items = 0;
  for (size_t j = 0; j < n_pieces; j++) {
    const Piece& q = pieces[j];
    const File& F = files[q.file];
    uint8_t* dec_out = to_device ? static_cast<uint8_t*>(outs[q.file]) : c->h_out + F.out_off;
    m_desc[j] = gmp_file_desc{c->h_comp + F.comp_off, bytes[q.file], d_idx + F.idx_off + q.b0, q.b1 - q.b0, dec_out,
                              F.info.orig_size};
    m_pre[j] = items;
    items += q.b1 - q.b0;
  }
  m_pre[n_pieces] = items;
  // ---- on the caller's stream: metadata, stream headers (with the block
  // offset tables), zeroed statuses, block counts, exit word and work counter
  unsigned long long* counter = c->counter + 48;
  GMP_CUDA(cudaMemcpyAsync(c->h_meta, meta.data(), meta_bytes, cudaMemcpyHostToDevice, s));
  for (size_t f = 0; f < n_files; f++) {
    if (files[f].idx.empty()) continue;
    GMP_CUDA(cudaMemcpyAsync(c->h_comp + files[f].comp_off, host_streams[f], files[f].idx[0].comp_offset,
                             cudaMemcpyHostToDevice, s));
  }
  GMP_CUDA(cudaMemsetAsync(c->h_status, 0, n_pieces * sizeof(int32_t), s));
  GMP_CUDA(cudaMemsetAsync(done, 0, (fn + 2) * sizeof(uint32_t), s));
  GMP_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
  GMP_CUDA(cudaEventRecord(c->ev[0], s));
  // ---- the copies in, in piece order, each followed by its piece's flag.
  // They are queued before the launch: they wait on nothing, and a launch
  // that blocks the host (CUDA_LAUNCH_BLOCKING, or a profiler replaying the
  // kernel alone) then still finds its input arriving.
  rc = GMP_OK;
  cudaError_t ce = cudaStreamWaitEvent(c->h2d, c->ev[0], 0);
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamWaitEvent");
  for (size_t j = 0; j < n_pieces && rc == GMP_OK; j++) {
    const Piece& q = pieces[j];
    const File& F = files[q.file];
    const uint8_t* src = static_cast<const uint8_t*>(host_streams[q.file]);
    const uint64_t c0 = F.idx[q.b0].comp_offset;
    const uint64_t c1 = q.b1 == F.idx.size() ? bytes[q.file] : F.idx[q.b1].comp_offset;
    const uint64_t c1x = std::min<uint64_t>(bytes[q.file], (c1 + 127) & ~uint64_t(127));
    ce = cudaMemcpyAsync(c->h_comp + F.comp_off + c0, src + c0, c1x - c0, cudaMemcpyHostToDevice, c->h2d);
    if (ce != cudaSuccess) {
      rc = cuda_fail(ce, "cudaMemcpyAsync (piece in)");
      break;
    }
    if ((int64_t)j == drop_flag) continue;  // the test hook's dropped flag
    const CUresult r = ops->write(c->h2d, (CUdeviceptr)(in_ready + j), gen, CU_STREAM_WRITE_VALUE_DEFAULT);
    if (r != CUDA_SUCCESS) rc = cu_fail(r, "cuStreamWriteValue32");
  }
  // ---- the launch, before any copy-back wait is queued, so that it never
  // waits behind one (streams may share a hardware queue)
  if (rc == GMP_OK) {
    ce = cudaStreamWaitEvent(c->pipe, c->ev[0], 0);
    if (ce == cudaSuccess) {
      const gmp::PipeFlags pf{in_ready,
                              done + fn + 1,
                              c->input_wait_ns,
                              to_device ? nullptr : out_ready,
                              to_device ? nullptr : done,
                              to_device ? nullptr : done + fn,
                              gen};
      ce = gmp::launch_decode(c->shape, reinterpret_cast<const gmp_file_desc*>(c->h_meta + desc_off),
                              reinterpret_cast<const uint64_t*>(c->h_meta + pre_off), (uint32_t)n_pieces, nullptr,
                              c->h_status, counter, c->scratch, c->slot_bytes, c->shadow_off, c->max_seq, c->max_out,
                              c->stats, (int)c->opts.collect_stats, (int)c->opts.resolve, c->pipe, 1, &pf);
    }
    if (ce != cudaSuccess) rc = cuda_fail(ce, "decode launch (host pipeline)");
  }
  if (rc) {
    // no launch, or no complete input: wait for the copies queued so far
    // (and a launch whose waits for missing pieces end by themselves)
    cudaStreamSynchronize(c->h2d);
    cudaStreamSynchronize(c->pipe);
    return rc;
  }
  // ---- the copies back, each after its piece's flag (queued last, so no
  // copy in and not the launch waits behind them)
  for (size_t j = 0; j < n_pieces && rc == GMP_OK && !to_device; j++) {
    const Piece& q = pieces[j];
    const File& F = files[q.file];
    const uint64_t o0 = F.idx[q.b0].out_offset;
    const uint64_t o1 = F.idx[q.b1 - 1].out_offset + F.idx[q.b1 - 1].out_bytes;
    cudaStream_t u = c->d2h[j % gmp::kPipeParts];
    const CUresult r = ops->wait(u, (CUdeviceptr)(out_ready + j), gen, CU_STREAM_WAIT_VALUE_GEQ);
    if (r != CUDA_SUCCESS) {
      rc = cu_fail(r, "cuStreamWaitValue32");
      break;
    }
    if (o1 > o0) {
      ce = cudaMemcpyAsync(static_cast<uint8_t*>(host_outs[q.file]) + o0, c->h_out + F.out_off + o0, o1 - o0,
                           cudaMemcpyDeviceToHost, u);
      if (ce != cudaSuccess) rc = cuda_fail(ce, "cudaMemcpyAsync (piece back)");
    }
  }
  // ---- join: the launch, the copies in and every copy back end before the
  // statuses are read
  auto join = [&](cudaStream_t from) {
    cudaError_t e = cudaEventRecord(c->ev[1], from);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->d2h[0], c->ev[1], 0);
    return e;
  };
  ce = join(c->pipe);
  if (ce == cudaSuccess) ce = join(c->h2d);
  for (uint32_t k = 1; k < gmp::kPipeParts && ce == cudaSuccess; k++) ce = join(c->d2h[k]);
  std::vector<int32_t> st(n_pieces, 0);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(st.data(), c->h_status, n_pieces * sizeof(int32_t), cudaMemcpyDeviceToHost, c->d2h[0]);
  const cudaError_t ce2 = cudaStreamSynchronize(c->d2h[0]);
  if (ce == cudaSuccess) ce = ce2;
  if (ce != cudaSuccess) {
    // the joins could not be queued: wait for everything of this call
    cudaStreamSynchronize(c->pipe);
    cudaStreamSynchronize(c->h2d);
    for (cudaStream_t t : c->d2h) cudaStreamSynchronize(t);
    return rc ? rc : cuda_fail(ce, "host pipeline join");
  }
  if (rc) return rc;
  // the caller's stream: ordered after this call's work
  GMP_CUDA(cudaEventRecord(c->ev[1], c->d2h[0]));
  GMP_CUDA(cudaStreamWaitEvent(s, c->ev[1], 0));
  for (size_t j = 0; j < n_pieces; j++)
    if (st[j] && !statuses[pieces[j].file]) statuses[pieces[j].file] = st[j];
  return GMP_OK;
}

int gmp_decompress_host_batch(gmp_context* c, size_t n_files, const void* const* host_streams, const size_t* bytes,
                              void* const* host_outs, const size_t* out_caps, int32_t* statuses, void* stream) {
  return decompress_from_host(c, n_files, host_streams, bytes, host_outs, out_caps, statuses, stream, false);
}

int gmp_decompress_from_host_batch(gmp_context* c, size_t n_files, const void* const* host_streams,
                                   const size_t* bytes, void* const* d_outs, const size_t* out_caps, int32_t* statuses,
                                   void* stream) {
  return decompress_from_host(c, n_files, host_streams, bytes, d_outs, out_caps, statuses, stream, true);
}

int gmp_decompress_host(gmp_context* c, const void* host_stream, size_t bytes, void* host_out, size_t out_cap,
                        int32_t* status, void* stream) {
  if (!c || !host_stream || !status || (!host_out && out_cap)) return GMP_ERR_INVALID_ARG;
  return gmp_decompress_host_batch(c, 1, &host_stream, &bytes, &host_out, &out_cap, status, stream);
}

}  // extern "C"
