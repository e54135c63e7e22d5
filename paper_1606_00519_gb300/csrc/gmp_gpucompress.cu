// gmp_gpucompress.cu - compression with the LZ77 parse on the GPU.
//
// Sec. 3.1: the input is cut into blocks that are compressed independently,
// hence in parallel; Sec. 4.2 adds the dependency rule of DE streams.  Here
// every step runs on the GPU: the match search and the parse of every block
// (this file), then the entropy coding (Huffman trees and sub-blocks, or Byte
// records; gmp_gpuencode.cu), writing the same stream format as
// gmp_compress.  The host only lays out the blocks from their sizes and
// writes the 64-byte file header and the block offset table.
//
//  match_kernel: one CTA per block.  The CTA walks the block 512 positions
//  at a time, one per thread, with the block's bytes streaming through a ring
//  in shared memory.  Hash-chain heads of 3-byte prefixes and the chain
//  links are in shared memory too; each thread follows its bucket's chain
//  for up to chain_depth candidates within the window, keeps the longest
//  match (at most max_match bytes) and stores its length and distance; then
//  every position of the step is linked in.  Lookups of a step see only
//  positions of earlier steps, so a candidate always lies before its
//  position, in the same block.
//  parse_kernel: one warp per block stages the per-position matches in
//  shared memory and lane 0 walks them from the block start: a match of at
//  least 3 bytes is taken unless the next position has a longer one
//  (one-step lazy evaluation), otherwise the byte becomes a literal.  For DE
//  streams a candidate is cut at the first source byte that an earlier
//  back-reference of the same 32-sequence group writes, as in gmp_compress;
//  for Byte streams literal strings are cut into runs of at most 1023
//  bytes, which count as sequences of their group.
//  Every token's position in its block is written beside it for the
//  entropy coder.
//
// Positions of the same step do not see each other, and one hash bucket per
// prefix is shared by several prefixes, so the parse can differ from
// gmp_compress's; any parse the checks accept is a valid stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "gmp.h"
#include "gmp_internal.h"

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr uint32_t kByteMaxLit = 1023;
constexpr int kMatchThreads = 512;       // positions per step of the match search
constexpr int kHeadBits = 12;            // hash buckets of 3-byte prefixes
constexpr uint32_t kLinkRing = 32768;    // chain links kept (>= the window)
constexpr uint32_t kInRing = 65536;      // input bytes kept (the window, a step and a match past it)
constexpr uint32_t kLook = 64;           // longest match

struct MatchSmem {
  uint32_t head[1 << kHeadBits];  // per bucket: latest position + 1 of an earlier step, 0 = none
  uint16_t link[kLinkRing];       // per position: distance to the bucket's previous position, 0 = none
  uint8_t ring[kInRing];          // the block's bytes [loaded - kInRing, loaded)
};

// Bytes x .. x + 3 of the ring (positions taken modulo its size), the first
// in the low byte: two aligned words and a funnel shift.
__device__ __forceinline__ uint32_t ring_word(const uint8_t* ring, uint32_t x) {
  constexpr uint32_t WM = kInRing / 4 - 1;
  const uint32_t* r = reinterpret_cast<const uint32_t*>(ring);
  const uint32_t wa = x >> 2;
  return __funnelshift_r(r[wa & WM], r[(wa + 1) & WM], (x & 3u) * 8u);
}

__device__ __forceinline__ uint32_t prefix_hash(uint32_t b0, uint32_t b1, uint32_t b2) {
  return ((b0 | (b1 << 8) | (b2 << 16)) * 0x9E3779B1u) >> (32 - kHeadBits);
}

// One CTA per block; positions in steps of kMatchThreads, one per thread.
// The block's bytes stream through a ring in shared memory that always holds
// the window below the step and the step plus a longest match above it; the
// hash-chain heads and links live in shared memory as well.
__global__ void __launch_bounds__(kMatchThreads) match_kernel(const uint8_t* in, uint64_t n, uint32_t block_size,
                                                              uint32_t window, uint32_t max_match,
                                                              uint32_t chain_depth, uint64_t n_blocks,
                                                              uint8_t* best_len, uint16_t* best_dist,
                                                              unsigned long long* counter) {
  extern __shared__ __align__(16) unsigned char match_smem[];
  MatchSmem& M = *reinterpret_cast<MatchSmem*>(match_smem);
  __shared__ unsigned long long next_block;
  const uint32_t tid = threadIdx.x;
  constexpr uint32_t RM = kInRing - 1, LM = kLinkRing - 1;
  for (;;) {
    if (tid == 0) next_block = atomicAdd(counter, 1ull);
    __syncthreads();
    const uint64_t b = next_block;
    __syncthreads();  // every thread has read next_block before thread 0 writes it again
    if (b >= n_blocks) break;
    const uint64_t base = b * (uint64_t)block_size;
    const uint32_t len = (uint32_t)min((uint64_t)block_size, n - base);
    const uint8_t* blk = in + base;
    for (uint32_t i = tid; i < (1u << kHeadBits); i += kMatchThreads) M.head[i] = 0;
    uint32_t loaded = 0;  // the same in every thread
    auto load_to = [&](uint32_t upto) {
      for (uint32_t x = loaded + tid; x < upto; x += kMatchThreads) M.ring[x & RM] = __ldg(blk + x);
      loaded = upto;
    };
    load_to(min(len, (uint32_t)kMatchThreads + kLook));
    __syncthreads();
    for (uint32_t s = 0; s < len; s += kMatchThreads) {
      const uint32_t p = s + tid;
      uint32_t h = 0, ml = 0, dist = 0, c0 = 0;
      const bool has_prefix = p + 3 <= len;
      if (has_prefix) {
        h = prefix_hash(M.ring[p & RM], M.ring[(p + 1) & RM], M.ring[(p + 2) & RM]);
        const uint32_t lim = min(max_match, len - p);
        c0 = M.head[h];
        uint32_t c = c0;  // position + 1
        for (uint32_t depth = 0; c && depth < chain_depth; depth++) {
          const uint32_t cand = c - 1, d = p - cand;
          if (d > window) break;  // links run back in position
          // a candidate that differs at the current best length cannot beat it
          if (ml >= lim || M.ring[(cand + ml) & RM] == M.ring[(p + ml) & RM]) {
            // match length: four bytes per step (the first differing byte
            // of a word from the XOR's lowest set bit), the last 0..3 bytes
            // one at a time
            uint32_t k = 0;
            for (;;) {
              if (k + 4 > lim) {
                while (k < lim && M.ring[(cand + k) & RM] == M.ring[(p + k) & RM]) k++;
                break;
              }
              const uint32_t x = ring_word(M.ring, cand + k) ^ ring_word(M.ring, p + k);
              if (x) {
                k += (uint32_t)(__ffs((int)x) - 1) >> 3;
                break;
              }
              k += 4;
            }
            if (k >= 3 && k > ml) {
              ml = k;
              dist = d;
              if (k == lim) break;
            }
          }
          const uint32_t delta = M.link[cand & LM];
          c = delta ? c - delta : 0u;
        }
      }
      if (p < len) {
        best_len[base + p] = (uint8_t)ml;
        best_dist[base + p] = (uint16_t)dist;
      }
      __syncthreads();  // the step's lookups are done
      if (has_prefix) {
        // each position links to the bucket's latest position before the
        // step (positions of one step do not see each other)
        M.link[p & LM] = (c0 && p + 1 - c0 <= 0xffffu) ? (uint16_t)(p + 1 - c0) : (uint16_t)0;
        atomicMax(M.head + h, p + 1);
      }
      load_to(min(len, s + 2 * kMatchThreads + kLook));
      __syncthreads();
    }
  }
}

struct ParseState {
  uint32_t glo[32], ghi[32];  // DE: output ranges of the current group's back-references
  uint32_t in_grp;
  uint32_t lo_min;            // start of the group's first back-reference (~0u: none yet)
};

// DE rule (Sec. 4.2, as read in gmp_compress): the source bytes before the
// current position must avoid the group's earlier back-references; the
// candidate is cut at the first such byte (0 if fewer than 3 bytes remain).
// The group's ranges rise with their index (empty ranges stand for
// literal-only sequences): a source that ends below the first of them is
// free (the common case: most sources lie before the group); otherwise the
// scan runs backwards and stops at the first range that ends at or below
// the source.
__device__ __forceinline__ uint32_t de_cut(const ParseState& st, uint32_t q, uint32_t L, uint32_t D) {
  if (L == 0) return 0;
  const uint32_t src = q - D, src_end = min(src + L, q);
  if (src_end <= st.lo_min) return L >= 3 ? L : 0u;
  for (int g = (int)st.in_grp - 1; g >= 0; g--) {
    if (st.glo[g] == st.ghi[g]) continue;
    if (st.ghi[g] <= src) break;
    if (st.glo[g] < src_end) L = min(L, st.glo[g] > src ? st.glo[g] - src : 0u);
  }
  return L >= 3 ? L : 0u;
}

constexpr int kParseWarps = 4;
constexpr uint32_t kChunk = 2048;  // positions staged in shared memory per warp

// One warp per block: the warp stages the per-position matches of the next
// kChunk positions in shared memory, lane 0 parses them.
__global__ void __launch_bounds__(32 * kParseWarps) parse_kernel(const uint8_t* best_len, const uint16_t* best_dist,
                                                                 uint64_t n, uint32_t block_size, uint64_t n_blocks,
                                                                 uint32_t max_match, int de, int byte_mode, int lazy,
                                                                 gmp::ParseToken* tok, uint32_t* tpos,
                                                                 uint64_t stride, uint32_t* count) {
  __shared__ uint8_t chunk_len[kParseWarps][kChunk];
  __shared__ uint16_t chunk_dist[kParseWarps][kChunk];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint64_t b = (uint64_t)blockIdx.x * kParseWarps + warp;
  if (b >= n_blocks) return;
  uint8_t* cl = chunk_len[warp];
  uint16_t* cd = chunk_dist[warp];
  const uint64_t base = b * (uint64_t)block_size;
  const uint32_t len = (uint32_t)min((uint64_t)block_size, n - base);
  gmp::ParseToken* t = tok + b * stride;
  uint32_t* tp = tpos + b * stride;
  uint32_t nt = 0, p = 0, lit_start = 0;
  ParseState st;
  st.in_grp = 0;
  st.lo_min = ~0u;
  auto emit = [&](uint32_t ll, uint32_t ml, uint32_t d) {
    if (nt < stride) {
      t[nt] = gmp::ParseToken{ll, (d << 8) | ml};
      tp[nt] = lit_start;
    }
    nt++;
  };
  auto add_to_group = [&](uint32_t lo, uint32_t hi) {
    if (de) {
      if (lo != hi && st.lo_min == ~0u) st.lo_min = lo;
      st.glo[st.in_grp] = lo;
      st.ghi[st.in_grp] = hi;
      if (++st.in_grp == 32) {
        st.in_grp = 0;
        st.lo_min = ~0u;
      }
    }
  };
  while (p < len) {
    const uint32_t c0 = p, cn = min(kChunk, len - c0);
    for (uint32_t i = lane; i < cn; i += 32) {
      cl[i] = best_len[base + c0 + i];
      cd[i] = best_dist[base + c0 + i];
    }
    __syncwarp();
    if (lane == 0) {
      auto match_at = [&](uint32_t q, uint32_t& D) -> uint32_t {
        const uint32_t L = cl[q - c0];
        D = cd[q - c0];
        if (L < 3) return 0;
        return de ? de_cut(st, q, L, D) : L;
      };
      // parse while the lazy look at p + 1 stays in the chunk (or the chunk
      // ends the block)
      const uint32_t end = c0 + cn, stop = end == len ? len : end - 1;
      while (p < stop) {
        uint32_t D = 0;
        uint32_t L = match_at(p, D);
        if (L && lazy) {
          while (p + 1 < end && L < max_match) {
            uint32_t D2 = 0;
            const uint32_t L2 = match_at(p + 1, D2);
            if (L2 <= L) break;
            p++;  // the byte at p stays a literal
            L = L2;
            D = D2;
          }
        }
        if (L) {
          while (byte_mode && p - lit_start > kByteMaxLit) {
            emit(kByteMaxLit, 0, 0);
            lit_start += kByteMaxLit;
            add_to_group(0, 0);
          }
          emit(p - lit_start, L, D);
          add_to_group(p, p + L);
          p += L;
          lit_start = p;
        } else {
          p++;
        }
      }
    }
    p = __shfl_sync(kFull, p, 0);
    __syncwarp();
  }
  if (lane == 0) {
    for (; byte_mode && len - lit_start > kByteMaxLit; lit_start += kByteMaxLit) emit(kByteMaxLit, 0, 0);
    if (lit_start < len) emit(len - lit_start, 0, 0);
    count[b] = nt;
  }
}

// Device times of the calling thread's last gmp_compress_gpu.
thread_local gmp_gpu_compress_times g_times = {0, 0, 0, 0};

struct DeviceBuffers {
  void* p[12] = {};
  ~DeviceBuffers() {
    for (void* q : p)
      if (q) cudaFree(q);
  }
};

}  // namespace

extern "C" {

int gmp_compress_gpu(int device, const void* host_in, size_t n, const gmp_compress_opts* opts, void* host_out,
                     size_t cap, size_t* out_bytes) {
  if ((!host_in && n) || !opts || !host_out || !out_bytes) return GMP_ERR_INVALID_ARG;
  const gmp_compress_opts o = *opts;
  if (!gmp::compress_opts_ok(o)) return GMP_ERR_INVALID_ARG;
  const uint8_t* in = static_cast<const uint8_t*>(host_in);
  const uint64_t nb = (n + o.block_size - 1) / o.block_size;
  g_times = gmp_gpu_compress_times{0, 0, 0, 0};
  if (nb == 0) {
    uint64_t total = 0;
    gmp::stream_layout(nullptr, 0, nullptr, &total);
    if (total > cap) return GMP_ERR_CAPACITY;
    gmp::write_stream_header(o, 0, 0, nullptr, total, static_cast<uint8_t*>(host_out));
    *out_bytes = total;
    return GMP_OK;
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return gmp::cuda_error(e, "cudaSetDevice");
  int rc = GMP_OK;
  {
    // tokens per block: at most one per 3 bytes plus the literal-only runs
    const uint64_t stride = o.block_size / 3 + o.block_size / kByteMaxLit + 4;
    DeviceBuffers D;
    cudaEvent_t ev[5] = {};
    auto check = [&](cudaError_t err, const char* what) {
      if (err != cudaSuccess && rc == GMP_OK) rc = gmp::cuda_error(err, what);
      return rc == GMP_OK;
    };
    for (auto& x : ev) check(cudaEventCreate(&x), "cudaEventCreate");
    int sms = 0;
    check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device), "cudaDeviceGetAttribute");
    uint8_t* d_in = nullptr;
    uint8_t* d_len = nullptr;
    uint16_t* d_dist = nullptr;
    gmp::ParseToken* d_tok = nullptr;
    uint32_t* d_tpos = nullptr;
    uint32_t* d_count = nullptr;
    unsigned long long* d_counter = nullptr;
    gmp::EncBlockPlan* d_plan = nullptr;
    uint64_t* d_bytes = nullptr;
    if (check(cudaMalloc(&D.p[0], n), "cudaMalloc") && check(cudaMalloc(&D.p[1], n), "cudaMalloc") &&
        check(cudaMalloc(&D.p[2], 2 * n), "cudaMalloc") &&
        check(cudaMalloc(&D.p[3], nb * stride * sizeof(gmp::ParseToken)), "cudaMalloc") &&
        check(cudaMalloc(&D.p[4], nb * stride * sizeof(uint32_t)), "cudaMalloc") &&
        check(cudaMalloc(&D.p[5], nb * sizeof(uint32_t)), "cudaMalloc") &&
        check(cudaMalloc(&D.p[6], 2 * sizeof(unsigned long long)), "cudaMalloc") &&
        check(cudaMalloc(&D.p[7], nb * sizeof(gmp::EncBlockPlan)), "cudaMalloc") &&
        check(cudaMalloc(&D.p[8], nb * sizeof(uint64_t)), "cudaMalloc")) {
      d_in = static_cast<uint8_t*>(D.p[0]);
      d_len = static_cast<uint8_t*>(D.p[1]);
      d_dist = static_cast<uint16_t*>(D.p[2]);
      d_tok = static_cast<gmp::ParseToken*>(D.p[3]);
      d_tpos = static_cast<uint32_t*>(D.p[4]);
      d_count = static_cast<uint32_t*>(D.p[5]);
      d_counter = static_cast<unsigned long long*>(D.p[6]);
      d_plan = static_cast<gmp::EncBlockPlan*>(D.p[7]);
      d_bytes = static_cast<uint64_t*>(D.p[8]);
    }
    int* d_error = reinterpret_cast<int*>(d_counter + 1);
    if (rc == GMP_OK) {
      check(cudaMemcpy(d_in, in, n, cudaMemcpyHostToDevice), "cudaMemcpy");
      check(cudaMemset(d_counter, 0, 2 * sizeof(unsigned long long)), "cudaMemset");
    }
    if (rc == GMP_OK) {
      check(cudaEventRecord(ev[0]), "cudaEventRecord");
      const int smem = (int)sizeof(MatchSmem);
      int occ = 0;
      check(cudaFuncSetAttribute(match_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
            "cudaFuncSetAttribute");
      check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, match_kernel, kMatchThreads, smem),
            "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
      const uint64_t grid = std::min<uint64_t>((uint64_t)std::max(occ, 1) * (uint64_t)std::max(sms, 1), nb);
      if (rc == GMP_OK) {
        match_kernel<<<(unsigned)grid, kMatchThreads, smem>>>(d_in, n, o.block_size, o.window, o.max_match,
                                                              std::min(o.chain_depth, 64u), nb, d_len, d_dist,
                                                              d_counter);
        check(cudaGetLastError(), "match_kernel");
      }
    }
    if (rc == GMP_OK) {
      check(cudaEventRecord(ev[1]), "cudaEventRecord");
      parse_kernel<<<(unsigned)((nb + kParseWarps - 1) / kParseWarps), 32 * kParseWarps>>>(
          d_len, d_dist, n, o.block_size, nb, o.max_match, o.de ? 1 : 0, o.byte_mode ? 1 : 0, o.lazy ? 1 : 0, d_tok,
          d_tpos, stride, d_count);
      check(cudaGetLastError(), "parse_kernel");
    }
    // entropy coding on the GPU: plan every block (sizes), lay the blocks out
    // on the host, write them
    gmp::EncLaunch L{d_in, n, o.block_size, o.byte_mode ? 0u : o.n_sub, o.cwl, o.window, o.max_match,
                     o.byte_mode ? 1 : 0, nb, d_tok, d_tpos, stride, d_count, d_plan, d_bytes, d_error,
                     (unsigned)std::min<uint64_t>(nb, (uint64_t)std::max(sms, 1) * 8), nullptr};
    if (rc == GMP_OK) {
      check(cudaEventRecord(ev[2]), "cudaEventRecord");
      check(gmp::launch_encode_plan(L), "plan_kernel");
    }
    std::vector<uint64_t> sizes(nb), offsets(nb);
    int h_error = 0;
    if (rc == GMP_OK) check(cudaMemcpy(sizes.data(), d_bytes, nb * sizeof(uint64_t), cudaMemcpyDeviceToHost),
                            "cudaMemcpy");
    if (rc == GMP_OK) check(cudaMemcpy(&h_error, d_error, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy");
    if (rc == GMP_OK && h_error) rc = GMP_ERR_INVALID_ARG;  // a parse that fails its checks (not expected)
    uint64_t total = 0, first = 0;
    if (rc == GMP_OK) {
      first = gmp::stream_layout(sizes.data(), nb, offsets.data(), &total);
      if (total > cap) rc = GMP_ERR_CAPACITY;
    }
    const uint64_t body = total - first - 16;  // the blocks, back to back
    if (rc == GMP_OK && check(cudaMalloc(&D.p[9], std::max<uint64_t>(body, 16)), "cudaMalloc") &&
        check(cudaMalloc(&D.p[10], nb * sizeof(uint64_t)), "cudaMalloc")) {
      uint64_t* d_off = static_cast<uint64_t*>(D.p[10]);
      for (uint64_t b = 0; b < nb; b++) offsets[b] -= first;
      check(cudaMemcpy(d_off, offsets.data(), nb * sizeof(uint64_t), cudaMemcpyHostToDevice), "cudaMemcpy");
      if (rc == GMP_OK) check(gmp::launch_encode_write(L, d_off, static_cast<uint8_t*>(D.p[9])), "write_kernel");
      if (rc == GMP_OK) check(cudaEventRecord(ev[3]), "cudaEventRecord");
      uint8_t* out = static_cast<uint8_t*>(host_out);
      if (rc == GMP_OK) check(cudaMemcpy(out + first, D.p[9], body, cudaMemcpyDeviceToHost), "cudaMemcpy");
      if (rc == GMP_OK) {
        for (uint64_t b = 0; b < nb; b++) offsets[b] += first;
        gmp::write_stream_header(o, n, nb, offsets.data(), total, out);
        *out_bytes = total;
        float t = 0;
        if (cudaEventElapsedTime(&t, ev[0], ev[1]) == cudaSuccess) g_times.match_ms = t;
        if (cudaEventElapsedTime(&t, ev[1], ev[2]) == cudaSuccess) g_times.parse_ms = t;
        if (cudaEventElapsedTime(&t, ev[2], ev[3]) == cudaSuccess) g_times.encode_ms = t;
        g_times.compressed_bytes = total;
      }
    }
    for (auto& x : ev)
      if (x) cudaEventDestroy(x);
  }
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}

void gmp_compress_gpu_last_times(gmp_gpu_compress_times* t) {
  if (t) *t = g_times;
}

}  // extern "C"
