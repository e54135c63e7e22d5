// gmp_gpuencode.cu - entropy coding of GPU parses on the GPU.
//
// Sec. 3.1: each block is compressed independently; Huffman-coded blocks
// (Gompresso/Bit) carry two trees, one for literals and match lengths and
// one for offsets, and are cut into sub-blocks whose sizes in bits are
// stored so that the decoder can start every sub-block at once (Sec. 3.2.1).
// Given the LZ77 parse of every block in device memory (tokens {literal
// length, (distance << 8) | match length} and each token's position), two
// kernels write the stream's blocks in the format gmp_compress writes:
//
//  plan_kernel, one CTA per block:
//   - checks every token against its block;
//   - frequencies of both alphabets: the literal/length histogram is the
//     histogram of all the block's bytes, minus the bytes that
//     back-references cover, plus one match-length or end symbol per token,
//     so that long literal runs spread over the CTA;
//   - code lengths limited to cwl bits per tree (one warp each): Huffman
//     code lengths by the two-queue method (van Leeuwen, 1976) on the
//     symbols sorted by frequency, then limited to cwl bits by the
//     bit-length adjustment of ITU-T T.81 (JPEG), Annex K.3, which moves
//     leaves up from depths over the limit while keeping the code complete
//     (Kraft sum 1); lengths go to the symbols in order of frequency;
//   - the sub-block split, equal in decoding work as gmp_compress makes it
//     (a token costs its literals + 1 lookups): a scan of per-thread token
//     costs and, per sub-block, a search for the token where the running
//     cost reaches (j + 1) / K of the total;
//   - the bits of every sub-block (the same decomposition: code bits of all
//     bytes of its output range, minus those of the bytes back-references
//     cover, plus each token's length, offset and extra bits), hence the
//     block's encoded size.
//  write_kernel, one CTA per block at the offset the host computed from the
//   sizes: the block header (code lengths, sub-block table), canonical codes
//   (Sec. 3.1) from the lengths, then thread j packs sub-block j's codes
//   LSB-first at its bit offset (the words it shares with its neighbours by
//   atomicOr, the others by plain stores).
//  Byte blocks (Gompresso/Byte) get their 4-byte records and literal bytes
//  written the same way, without trees.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gmp.h"
#include "gmp_internal.h"

namespace gmp {
namespace {

constexpr int kEncThreads = 256;
constexpr int kMaxDepth = 64;
constexpr uint32_t kNLL = kLitLenSyms, kNOff = kOffsetSyms;
constexpr uint32_t kSymEnd = 256;

// Per-tree workspace of the code-length construction (one warp).
struct TreeWS {
  uint16_t sorted[kNLL + 1];           // used symbols by (frequency, symbol)
  uint16_t par_leaf[kNLL + 1];         // parent (internal index) of leaf i of `sorted`
  uint16_t par_int[kNLL + 1];          // parent of internal node k
  uint8_t depth_int[kNLL + 1];
  unsigned long long w_int[kNLL + 1];  // weight of internal node k
  uint32_t bits[kMaxDepth];            // leaves per depth
  uint32_t m;                          // used symbols
};

struct PlanSmem {
  uint32_t h1[kNLL + 1], h2[kNOff + 2];
  unsigned long long csum[kEncThreads];  // token cost per thread chunk, then its exclusive prefix
  uint32_t lsum[kEncThreads];            // literal bytes per thread chunk, then prefix
  uint32_t g[kMaxSub], qs[kMaxSub + 1], so[kMaxSub + 1];
  unsigned long long sbits[kMaxSub];
  uint8_t lens[kNLL + kNOff + 1];
  TreeWS ws[2];
  unsigned long long total_cost;
  uint32_t n_lit, err;
};

// Distance code of the stream format: symbol, extra bit count and extra bits
// of a distance 1..32768.
__device__ __forceinline__ void dist_symbol(uint32_t d, uint32_t& sym, uint32_t& ne, uint32_t& ex) {
  const uint32_t v = d - 1;
  if (v < 4) {
    sym = v;
    ne = 0;
    ex = 0;
    return;
  }
  const uint32_t k = 31u - (uint32_t)__clz(v);
  sym = 2 * k + ((v >> (k - 1)) & 1u);
  ne = k - 1;
  ex = v & ((1u << ne) - 1u);
}

// Code lengths (<= limit) of the symbols with non-zero frequency in
// freq[0..n); one warp.  A single used symbol gets length 1 together with a
// dummy second symbol, so that the code is complete.
__device__ void build_lengths(const uint32_t* freq, uint32_t n, uint32_t limit, uint8_t* len, TreeWS& W) {
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t used = 0;
  for (uint32_t s = lane; s < n; s += 32) {
    len[s] = 0;
    const uint32_t f = freq[s];
    if (!f) continue;
    used++;
    uint32_t r = 0;
    for (uint32_t t = 0; t < n; t++) {
      const uint32_t ft = freq[t];
      r += (ft != 0 && (ft < f || (ft == f && t < s))) ? 1u : 0u;
    }
    W.sorted[r] = (uint16_t)s;
  }
  for (int d = 16; d >= 1; d >>= 1) used += __shfl_xor_sync(0xffffffffu, used, d);
  __syncwarp();
  if (lane == 0) {
    const uint32_t m = used;
    if (m == 1) {
      const uint32_t s = W.sorted[0];
      len[s] = 1;
      len[s == 0 ? 1 : 0] = 1;
    } else if (m > 1) {
      // two queues: the leaves in order of weight, and the internal nodes,
      // which are made in order of weight
      uint32_t li = 0, ii = 0, ni = 0;
      for (uint32_t step = 0; step + 1 < m; step++) {
        unsigned long long w2 = 0;
        for (int pick = 0; pick < 2; pick++) {
          if (li < m && (ii >= ni || (unsigned long long)freq[W.sorted[li]] <= W.w_int[ii])) {
            w2 += freq[W.sorted[li]];
            W.par_leaf[li++] = (uint16_t)ni;
          } else {
            w2 += W.w_int[ii];
            W.par_int[ii++] = (uint16_t)ni;
          }
        }
        W.w_int[ni++] = w2;
      }
      // depths: the root is the last internal node; parents come later
      W.depth_int[ni - 1] = 0;
      for (int k = (int)ni - 2; k >= 0; k--) W.depth_int[k] = (uint8_t)(W.depth_int[W.par_int[k]] + 1);
      for (int d = 0; d < kMaxDepth; d++) W.bits[d] = 0;
      for (uint32_t i = 0; i < m; i++) {
        const uint32_t d = W.depth_int[W.par_leaf[i]] + 1u;
        W.bits[d < (uint32_t)kMaxDepth ? d : kMaxDepth - 1]++;
      }
      // T.81 Annex K.3: while a depth over the limit has leaves, take two
      // sibling leaves there (their parent becomes a leaf one level up) and
      // split the deepest leaf at least two levels above into two children
      for (uint32_t i = kMaxDepth - 1; i > limit; i--) {
        while (W.bits[i] > 0) {
          uint32_t j = i - 2;
          while (W.bits[j] == 0) j--;
          W.bits[i] -= 2;
          W.bits[i - 1] += 1;
          W.bits[j + 1] += 2;
          W.bits[j] -= 1;
        }
      }
      // the most frequent symbols take the shortest lengths
      uint32_t d = 1, left = W.bits[1];
      for (uint32_t r = 0; r < m; r++) {
        while (left == 0) left = W.bits[++d];
        len[W.sorted[m - 1 - r]] = (uint8_t)d;
        left--;
      }
    }
  }
  __syncwarp();
}

// Index of the last entry of the ascending array a[0..n) that is <= x
// (a[0] <= x is assumed).
template <class T>
__device__ __forceinline__ uint32_t last_le(const T* a, uint32_t n, T x) {
  uint32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (a[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

struct EncParams {
  const uint8_t* in;
  uint64_t n;
  uint32_t block_size, n_sub, cwl, window, max_match;
  int byte_mode;
  uint64_t n_blocks;
  const ParseToken* tok;
  const uint32_t* tpos;
  uint64_t stride;
  const uint32_t* count;
  EncBlockPlan* plan;
  uint64_t* block_bytes;
  int* error;
};

__global__ void __launch_bounds__(kEncThreads) plan_kernel(const EncParams E) {
  __shared__ PlanSmem S;
  const uint32_t tid = threadIdx.x, warp = tid >> 5;
  for (uint64_t b = blockIdx.x; b < E.n_blocks; b += gridDim.x) {
    const uint64_t base = b * (uint64_t)E.block_size;
    const uint32_t len = (uint32_t)min((uint64_t)E.block_size, E.n - base);
    const uint8_t* blk = E.in + base;
    const uint32_t n = E.count[b];
    const ParseToken* t = E.tok + b * E.stride;
    const uint32_t* tp = E.tpos + b * E.stride;
    const uint32_t K = E.byte_mode ? 0u : E.n_sub;
    for (uint32_t i = tid; i < kNLL + 1; i += kEncThreads) S.h1[i] = 0;
    if (tid < kNOff + 2) S.h2[tid] = 0;
    if (tid == 0) S.err = (n == 0 || n > E.stride) ? 1u : 0u;
    __syncthreads();
    const uint32_t nn = min(n, (uint32_t)E.stride);
    const uint32_t C = (nn + kEncThreads - 1) / kEncThreads;
    const uint32_t k0 = min(tid * C, nn), k1 = min(k0 + C, nn);
    // pass 1 over the thread's tokens: checks, work and literal counts, the
    // symbol frequencies, and the bytes under back-references out of the
    // byte histogram
    unsigned long long cost = 0;
    uint32_t lits = 0;
    bool bad = false;
    for (uint32_t k = k0; k < k1; k++) {
      const uint32_t ll = t[k].lit_len, ml = t[k].match & 0xffu, d = t[k].match >> 8, p = tp[k];
      const uint64_t end = (uint64_t)p + ll + ml;
      const uint64_t next = k + 1 < nn ? tp[k + 1] : len;
      bool ok = end == next && (k != 0 || p == 0) && end <= len;
      if (ml) ok = ok && ml >= 3 && ml <= E.max_match && d >= 1 && d <= E.window && d <= p + ll;
      else ok = ok && (E.byte_mode || k + 1 == nn);
      if (E.byte_mode) ok = ok && ll <= 1023;
      if (!ok) {
        bad = true;
        break;
      }
      cost += ll + 1ull;
      lits += ll;
      if (!E.byte_mode) {
        if (ml) {
          uint32_t sym, ne, ex;
          dist_symbol(d, sym, ne, ex);
          atomicAdd(&S.h1[254 + ml], 1u);
          atomicAdd(&S.h2[sym], 1u);
          const uint8_t* src = blk + p + ll;
          for (uint32_t i = 0; i < ml; i++) atomicSub(&S.h1[src[i]], 1u);
        } else {
          atomicAdd(&S.h1[kSymEnd], 1u);
        }
      }
    }
    S.csum[tid] = cost;
    S.lsum[tid] = lits;
    if (bad) atomicOr(&S.err, 1u);
    if (!E.byte_mode)
      for (uint32_t x = tid; x < len; x += kEncThreads) atomicAdd(&S.h1[blk[x]], 1u);
    __syncthreads();
    if (tid == 0) {
      unsigned long long rc = 0;
      uint32_t rl = 0;
      for (int c = 0; c < kEncThreads; c++) {
        const unsigned long long v = S.csum[c];
        const uint32_t l = S.lsum[c];
        S.csum[c] = rc;
        S.lsum[c] = rl;
        rc += v;
        rl += l;
      }
      S.total_cost = rc;
      S.n_lit = rl;
      if (rc != (unsigned long long)nn + S.n_lit) S.err = 1;
    }
    __syncthreads();
    EncBlockPlan& P = E.plan[b];
    if (S.err) {
      if (tid == 0) {
        P.err = 1;
        E.block_bytes[b] = 0;
        atomicExch(E.error, 1);
      }
      __syncthreads();
      continue;
    }
    if (E.byte_mode) {
      if (tid == 0) {
        P.err = 0;
        P.n_seq = nn;
        P.out_bytes = len;
        P.n_lit = S.n_lit;
        P.bits = 0;
        const uint64_t bytes = ((16ull + 4ull * nn + 15) & ~15ull) + ((S.n_lit + 15ull) & ~15ull);
        P.bytes = bytes;
        E.block_bytes[b] = bytes;
      }
      __syncthreads();
      continue;
    }
    // code lengths of both trees, one warp each
    if (warp == 0) build_lengths(S.h1, kNLL, E.cwl, S.lens, S.ws[0]);
    else if (warp == 1) build_lengths(S.h2, kNOff, E.cwl, S.lens + kNLL, S.ws[1]);
    // sub-block ends: thread j finds the first token whose running cost
    // reaches (j + 1) / K of the total
    if (tid < K) {
      const unsigned long long T = S.total_cost * (tid + 1) / K;
      uint32_t g = 0;
      if (T > 0) {
        const uint32_t c = last_le<unsigned long long>(S.csum, kEncThreads, T - 1);  // last chunk starting below T
        unsigned long long run = S.csum[c];
        const uint32_t c0 = min(c * C, nn), c1 = min(c0 + C, nn);
        g = c1;
        for (uint32_t k = c0; k < c1; k++) {
          run += t[k].lit_len + 1ull;
          if (run >= T) {
            g = k;
            break;
          }
        }
      }
      S.g[tid] = T > 0 ? g : 0xffffffffu;  // T = 0: the sub-block is empty
    }
    __syncthreads();
    if (tid == 0) {
      uint32_t qi = 0;
      for (uint32_t j = 0; j < K; j++) {
        // the host's rule: the sub-block takes tokens while the running cost
        // is below the target (the last one takes the rest)
        const uint32_t g = S.g[j];
        const uint32_t qe = (j + 1 == K) ? nn : (g == 0xffffffffu || qi > g) ? qi : min(g + 1, nn);
        S.qs[j] = qi;
        qi = qe;
      }
      S.qs[K] = nn;
    }
    __syncthreads();
    if (tid <= K) S.so[tid] = S.qs[tid] < nn ? tp[S.qs[tid]] : len;
    if (tid < K) S.sbits[tid] = 0;
    __syncthreads();
    // bits per sub-block: literal codes of every byte of its output range
    // (a contiguous range of bytes per thread) ...
    {
      const uint32_t L = (len + kEncThreads - 1) / kEncThreads;
      const uint32_t x0 = min(tid * L, len), x1 = min(x0 + L, len);
      if (x0 < x1) {
        uint32_t j = last_le<uint32_t>(S.so, K, x0);
        long long acc = 0;
        for (uint32_t x = x0; x < x1; x++) {
          while (j + 1 < K && x >= S.so[j + 1]) {
            atomicAdd(&S.sbits[j], (unsigned long long)acc);
            acc = 0;
            j++;
          }
          acc += S.lens[blk[x]];
        }
        atomicAdd(&S.sbits[j], (unsigned long long)acc);
      }
    }
    // ... minus the bytes under back-references, plus each token's length
    // or end code and its offset code and extra bits
    if (k0 < k1) {
      uint32_t j = last_le<uint32_t>(S.qs, K, k0);
      while (j + 1 < K && S.qs[j + 1] <= k0) j++;  // empty sub-blocks share a start
      long long acc = 0;
      for (uint32_t k = k0; k < k1; k++) {
        while (j + 1 < K && k >= S.qs[j + 1]) {
          atomicAdd(&S.sbits[j], (unsigned long long)acc);
          acc = 0;
          j++;
        }
        const uint32_t ll = t[k].lit_len, ml = t[k].match & 0xffu, d = t[k].match >> 8;
        if (ml) {
          uint32_t sym, ne, ex;
          dist_symbol(d, sym, ne, ex);
          acc += (long long)S.lens[254 + ml] + S.lens[kNLL + sym] + ne;
          const uint8_t* src = blk + tp[k] + ll;
          for (uint32_t i = 0; i < ml; i++) acc -= S.lens[src[i]];
        } else {
          acc += S.lens[kSymEnd];
        }
      }
      atomicAdd(&S.sbits[j], (unsigned long long)acc);
    }
    __syncthreads();
    if (tid < K) {
      P.sub_first[tid] = S.qs[tid];
      P.sub_out[tid] = S.so[tid + 1] - S.so[tid];
      P.sub_bits[tid] = S.sbits[tid];
    }
    for (uint32_t i = tid; i < kNLL + kNOff; i += kEncThreads) P.lens[i] = S.lens[i];
    if (tid == 0) {
      unsigned long long bits = 0;
      for (uint32_t j = 0; j < K; j++) bits += S.sbits[j];
      P.sub_first[K] = nn;
      P.err = 0;
      P.n_seq = nn;
      P.out_bytes = len;
      P.n_lit = S.n_lit;
      P.bits = bits;
      const uint64_t hdr = (kBlockFixed + 12ull * K + 15) & ~15ull;
      const uint64_t bytes = hdr + (((bits + 7) / 8 + 15) & ~15ull);
      P.bytes = bytes;
      E.block_bytes[b] = bytes;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void put_le32(uint8_t* p, uint32_t v) { *reinterpret_cast<uint32_t*>(p) = v; }

__global__ void __launch_bounds__(kEncThreads) write_kernel(const EncParams E, const uint64_t* offsets, uint8_t* out) {
  __shared__ uint16_t rc[kNLL + kNOff];  // canonical codes, bit-reversed for LSB-first output
  __shared__ uint8_t lens[kNLL + kNOff];
  __shared__ uint32_t lsum[kEncThreads];
  const uint32_t tid = threadIdx.x;
  for (uint64_t b = blockIdx.x; b < E.n_blocks; b += gridDim.x) {
    const EncBlockPlan& P = E.plan[b];
    uint8_t* dst = out + offsets[b];
    const uint64_t base = b * (uint64_t)E.block_size;
    const uint8_t* blk = E.in + base;
    const uint32_t n = P.n_seq;
    const ParseToken* t = E.tok + b * E.stride;
    const uint32_t* tp = E.tpos + b * E.stride;
    // zero the block (P.bytes is a multiple of 16, dst 16-byte aligned)
    for (uint64_t i = 16ull * tid; i < P.bytes; i += 16ull * kEncThreads)
      *reinterpret_cast<uint4*>(dst + i) = make_uint4(0, 0, 0, 0);
    if (!E.byte_mode) {
      for (uint32_t i = tid; i < kNLL + kNOff; i += kEncThreads) lens[i] = P.lens[i];
    }
    __syncthreads();
    if (E.byte_mode) {
      // {n_seq, out_bytes, n_lit, 0}, one record per sequence, the literals
      const uint32_t C = (n + kEncThreads - 1) / kEncThreads;
      const uint32_t k0 = min(tid * C, n), k1 = min(k0 + C, n);
      uint32_t l = 0;
      for (uint32_t k = k0; k < k1; k++) l += t[k].lit_len;
      lsum[tid] = l;
      __syncthreads();
      if (tid == 0) {
        uint32_t r = 0;
        for (int c = 0; c < kEncThreads; c++) {
          const uint32_t v = lsum[c];
          lsum[c] = r;
          r += v;
        }
        put_le32(dst, n);
        put_le32(dst + 4, P.out_bytes);
        put_le32(dst + 8, P.n_lit);
      }
      __syncthreads();
      const uint64_t lit_sec = (16ull + 4ull * n + 15) & ~15ull;
      uint32_t lo = lsum[tid];
      for (uint32_t k = k0; k < k1; k++) {
        const uint32_t ll = t[k].lit_len, ml = t[k].match & 0xffu, d = t[k].match >> 8;
        put_le32(dst + 16 + 4ull * k, ll | (ml ? ((ml - 2) << 10) | ((d - 1) << 16) : 0u));
        const uint8_t* src = blk + tp[k];
        for (uint32_t i = 0; i < ll; i++) dst[lit_sec + lo + i] = src[i];
        lo += ll;
      }
      __syncthreads();
      continue;
    }
    const uint32_t K = E.n_sub;
    const uint64_t hdr = (kBlockFixed + 12ull * K + 15) & ~15ull;
    // header: sizes, code lengths (4 bits each, low nibble first), sub-block table
    if (tid == 0) {
      put_le32(dst, n);
      put_le32(dst + 4, P.out_bytes);
    }
    if (tid < (kNLL + 1) / 2) {
      const uint32_t s = 2 * tid;
      dst[8 + tid] = (uint8_t)(lens[s] | ((s + 1 < kNLL ? lens[s + 1] : 0u) << 4));
    }
    if (tid < kNOff / 2) dst[168 + tid] = (uint8_t)(lens[kNLL + 2 * tid] | (lens[kNLL + 2 * tid + 1] << 4));
    if (tid < K) {
      put_le32(dst + kBlockFixed + 12 * tid, (uint32_t)P.sub_bits[tid]);
      put_le32(dst + kBlockFixed + 12 * tid + 4, P.sub_out[tid]);
      put_le32(dst + kBlockFixed + 12 * tid + 8, P.sub_first[tid + 1] - P.sub_first[tid]);
    }
    // canonical codes: per length, consecutive codes in symbol order
    if (tid < 2) {
      const uint32_t s0 = tid ? kNLL : 0, ns = tid ? kNOff : kNLL;
      uint32_t cnt[16] = {0}, next[16];
      for (uint32_t s = 0; s < ns; s++) cnt[lens[s0 + s]]++;
      uint32_t c = 0;
      cnt[0] = 0;
      for (int l = 1; l < 16; l++) {
        next[l] = c;
        c = (c + cnt[l]) << 1;
      }
      for (uint32_t s = 0; s < ns; s++) {
        const uint32_t l = lens[s0 + s];
        rc[s0 + s] = l ? (uint16_t)(__brev(next[l]++) >> (32 - l)) : (uint16_t)0;
      }
    }
    __syncthreads();
    if (tid < K) {
      // sub-block tid's bits, from its bit offset in the block's bitstream
      uint64_t start = 0;
      for (uint32_t j = 0; j < tid; j++) start += P.sub_bits[j];
      uint32_t* W = reinterpret_cast<uint32_t*>(dst + hdr);
      uint64_t w = start >> 5;
      unsigned long long acc = 0;
      uint32_t na = (uint32_t)(start & 31u);
      bool first = true;
      auto put = [&](uint32_t bits, uint32_t nb) {
        acc |= (unsigned long long)bits << na;
        na += nb;
        if (na >= 32) {
          if (first) atomicOr(W + w, (uint32_t)acc);
          else W[w] = (uint32_t)acc;
          first = false;
          w++;
          acc >>= 32;
          na -= 32;
        }
      };
      for (uint32_t k = P.sub_first[tid]; k < P.sub_first[tid + 1]; k++) {
        const uint32_t ll = t[k].lit_len, ml = t[k].match & 0xffu, d = t[k].match >> 8;
        const uint8_t* src = blk + tp[k];
        for (uint32_t i = 0; i < ll; i++) {
          const uint32_t c = src[i];
          put(rc[c], lens[c]);
        }
        if (ml) {
          uint32_t sym, ne, ex;
          dist_symbol(d, sym, ne, ex);
          put(rc[254 + ml], lens[254 + ml]);
          put(rc[kNLL + sym], lens[kNLL + sym]);
          if (ne) put(ex, ne);
        } else {
          put(rc[kSymEnd], lens[kSymEnd]);
        }
      }
      if (na) atomicOr(W + w, (uint32_t)acc);
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_encode_plan(const EncLaunch& L) {
  EncParams E{L.in, L.n, L.block_size, L.n_sub, L.cwl, L.window, L.max_match, L.byte_mode, L.n_blocks, L.tok,
              L.tpos, L.stride, L.count, L.plan, L.block_bytes, L.error};
  plan_kernel<<<L.grid, kEncThreads, 0, L.stream>>>(E);
  return cudaGetLastError();
}

cudaError_t launch_encode_write(const EncLaunch& L, const uint64_t* offsets, uint8_t* out) {
  EncParams E{L.in, L.n, L.block_size, L.n_sub, L.cwl, L.window, L.max_match, L.byte_mode, L.n_blocks, L.tok,
              L.tpos, L.stride, L.count, L.plan, L.block_bytes, L.error};
  write_kernel<<<L.grid, kEncThreads, 0, L.stream>>>(E, offsets, out);
  return cudaGetLastError();
}

}  // namespace gmp
