// gmp_compress.cpp - host compressor of libgmp (multi-threaded over blocks).
//
// Writes stream format version 1 (see gmp.h).  Steps per block (Sec. 3.1):
// LZ77 with a sliding window, greedy parse over hash chains of 3-byte
// prefixes; sequences = literal string + back-reference; in DE mode the
// dependency rule of Sec. 4.2 (Fig. 7); two Huffman trees per block (literals
// and lengths; offsets) limited to cwl bits; canonical codes; K sub-blocks.
// Code lengths come from an ordinary Huffman merge followed by a Kraft repair
// that lengthens rarely used codes until the code fits in cwl bits and then
// shortens frequent ones until the Kraft sum is exactly one (the decoder needs
// a complete code).  With byte_mode the same parse is written as fixed
// 4-byte records and raw literals (Gompresso/Byte, Sec. 3.1) instead of
// Huffman bitstreams.  Any valid stream decodes to the same bytes, so this
// compressor's choices need not match any other encoder's.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <queue>
#include <thread>
#include <vector>

#include "gmp.h"
#include "gmp_internal.h"

namespace {

constexpr int kHashBits = 16;
constexpr uint32_t kNil = 0xffffffffu;
constexpr uint32_t kByteMaxLit = 1023;  // literal length field of a Byte record (10 bits)

struct Seq {
  uint32_t lit_start, lit_len, mlen, dist;
};

// Distance code (gmp.h): symbol and extra bits for d in 1..32768.
inline void dist_code(uint32_t d, uint32_t& sym, uint32_t& nbits, uint32_t& bits) {
  uint32_t v = d - 1;
  if (v < 4) {
    sym = v;
    nbits = 0;
    bits = 0;
    return;
  }
  uint32_t k = 31u - (uint32_t)__builtin_clz(v);
  sym = 2 * k + ((v >> (k - 1)) & 1u);
  nbits = k - 1;
  bits = v & ((1u << nbits) - 1u);
}

inline uint32_t hash_at(const uint8_t* p) {
  uint32_t x = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16);
  return (x * 0x9E3779B1u) >> (32 - kHashBits);
}

// LZ77 over one block: at each position the longest match among the hash
// chain's candidates (nearest first on ties); with o.lazy, while the next
// position has a longer match, the current byte becomes a literal and the
// search moves on (one-step lazy evaluation).  Fewer, longer sequences make
// the stream smaller and faster to decode.
void parse_block(const uint8_t* in, uint32_t n, const gmp_compress_opts& o, std::vector<Seq>& seqs,
                 std::vector<uint32_t>& head, std::vector<uint32_t>& chain) {
  seqs.clear();
  std::fill(head.begin(), head.end(), kNil);
  if (chain.size() < n) chain.resize(n);
  uint32_t lit_start = 0, i = 0, ins = 0;
  // DE: output intervals of the back-references of the current group
  uint32_t grp_lo[32], grp_hi[32];
  uint32_t in_grp = 0;
  auto insert_upto = [&](uint32_t p) {  // every position below p is in the chains
    for (; ins < p; ins++) {
      if (ins + 3 <= n) {
        const uint32_t h = hash_at(in + ins);
        chain[ins] = head[h];
        head[h] = ins;
      }
    }
  };
  auto find = [&](uint32_t p, uint32_t& best_len, uint32_t& best_dist) {
    best_len = best_dist = 0;
    if (p + 3 > n) return;
    const uint32_t lim = std::min<uint32_t>(o.max_match, n - p);
    uint32_t cand = head[hash_at(in + p)];
    for (uint32_t tries = 0; cand != kNil && tries < o.chain_depth; tries++, cand = chain[cand]) {
      const uint32_t dist = p - cand;
      if (dist > o.window) break;
      if (best_len < lim && in[cand + best_len] != in[p + best_len]) continue;  // cannot beat best
      uint32_t len = 0;
      while (len < lim && in[cand + len] == in[p + len]) len++;
      if (o.de) {
        // the source bytes before p must avoid this group's earlier copies
        const uint32_t src_end = std::min(cand + len, p);
        for (uint32_t g = 0; g < in_grp; g++) {
          if (grp_hi[g] > cand && grp_lo[g] < src_end) len = std::min(len, grp_lo[g] > cand ? grp_lo[g] - cand : 0u);
        }
      }
      if (len >= 3 && len > best_len) {
        best_len = len;
        best_dist = dist;
        if (len == lim) break;
      }
    }
  };
  while (i < n) {
    insert_upto(i);
    uint32_t len = 0, dist = 0;
    find(i, len, dist);
    if (len && o.lazy) {
      while (i + 1 < n && len < o.max_match) {
        insert_upto(i + 1);
        uint32_t l2 = 0, d2 = 0;
        find(i + 1, l2, d2);
        if (l2 <= len) break;
        i++;  // the byte at i stays a literal
        len = l2;
        dist = d2;
      }
    }
    if (len) {
      if (o.byte_mode) {
        // a Byte record holds at most 1023 literals: longer literal strings
        // are cut into literal-only sequences, members of their DE group like
        // any other sequence.  (The match was searched before the cut was
        // known; the cut can only move it into a later group, whose earlier
        // back-references are a subset of the ones it avoided.)
        while (i - lit_start > kByteMaxLit) {
          seqs.push_back(Seq{lit_start, kByteMaxLit, 0, 0});
          lit_start += kByteMaxLit;
          if (o.de) {
            grp_lo[in_grp] = grp_hi[in_grp] = 0;  // no back-reference
            if (++in_grp == 32) in_grp = 0;
          }
        }
      }
      seqs.push_back(Seq{lit_start, i - lit_start, len, dist});
      if (o.de) {
        grp_lo[in_grp] = i;
        grp_hi[in_grp] = i + len;
        if (++in_grp == 32) in_grp = 0;
      }
      i += len;
      lit_start = i;
    } else {
      i++;
    }
  }
  if (o.byte_mode)
    for (; n - lit_start > kByteMaxLit; lit_start += kByteMaxLit) seqs.push_back(Seq{lit_start, kByteMaxLit, 0, 0});
  if (lit_start < n) seqs.push_back(Seq{lit_start, n - lit_start, 0, 0});
}

// Huffman code lengths limited to `limit` bits, complete (Kraft sum = 1).
void code_lengths(const std::vector<uint64_t>& freq, uint32_t limit, std::vector<uint8_t>& len) {
  const size_t n = freq.size();
  len.assign(n, 0);
  std::vector<uint32_t> used;
  for (size_t s = 0; s < n; s++)
    if (freq[s]) used.push_back((uint32_t)s);
  if (used.empty()) return;
  if (used.size() == 1) {
    len[used[0]] = 1;
    len[used[0] == 0 ? 1 : 0] = 1;
    return;
  }
  // ordinary Huffman merge: parent links, then depth of each leaf
  struct Node {
    uint64_t w;
    int32_t parent;
  };
  std::vector<Node> nodes;
  nodes.reserve(2 * used.size());
  using Item = std::pair<uint64_t, int32_t>;
  std::priority_queue<Item, std::vector<Item>, std::greater<Item>> pq;
  for (uint32_t s : used) {
    nodes.push_back(Node{freq[s], -1});
    pq.push(Item(freq[s], (int32_t)nodes.size() - 1));
  }
  while (pq.size() > 1) {
    Item a = pq.top();
    pq.pop();
    Item b = pq.top();
    pq.pop();
    nodes.push_back(Node{a.first + b.first, -1});
    int32_t p = (int32_t)nodes.size() - 1;
    nodes[a.second].parent = p;
    nodes[b.second].parent = p;
    pq.push(Item(a.first + b.first, p));
  }
  std::vector<uint32_t> depth(nodes.size(), 0);
  for (int32_t k = (int32_t)nodes.size() - 2; k >= 0; k--) depth[k] = depth[nodes[k].parent] + 1;
  const uint64_t full = 1ull << limit;
  uint64_t kraft = 0;
  for (size_t k = 0; k < used.size(); k++) {
    uint32_t d = std::min<uint32_t>(depth[k], limit);
    len[used[k]] = (uint8_t)d;
    kraft += 1ull << (limit - d);
  }
  // Kraft repair: rare symbols first when lengthening, frequent first when shortening
  std::vector<uint32_t> order(used);
  std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return freq[a] < freq[b]; });
  while (kraft > full) {
    for (uint32_t s : order) {
      if (len[s] < limit) {
        kraft -= 1ull << (limit - len[s] - 1);
        len[s]++;
        if (kraft <= full) break;
      }
    }
  }
  while (kraft < full) {
    for (auto it = order.rbegin(); it != order.rend(); ++it) {
      uint32_t s = *it;
      if (len[s] > 1 && kraft + (1ull << (limit - len[s])) <= full) {
        kraft += 1ull << (limit - len[s]);
        len[s]--;
        if (kraft == full) break;
      }
    }
  }
}

// Canonical codes (Sec. 3.1), most significant bit first, returned
// bit-reversed so that they can be sent LSB-first.
void canonical_reversed(const std::vector<uint8_t>& len, std::vector<uint32_t>& rcode) {
  uint32_t count[16] = {0}, next[16] = {0};
  for (uint8_t l : len)
    if (l) count[l]++;
  uint32_t c = 0;
  for (int b = 1; b < 16; b++) {
    next[b] = c;
    c = (c + count[b]) << 1;
  }
  rcode.assign(len.size(), 0);
  for (size_t s = 0; s < len.size(); s++) {
    uint32_t l = len[s];
    if (!l) continue;
    uint32_t code = next[l]++, r = 0;
    for (uint32_t k = 0; k < l; k++) r |= ((code >> k) & 1u) << (l - 1 - k);
    rcode[s] = r;
  }
}

class BitSink {
 public:
  explicit BitSink(std::vector<uint8_t>& v) : v_(v) {}
  void put(uint32_t bits, uint32_t n) {  // n <= 32
    acc_ |= (uint64_t)bits << fill_;
    fill_ += n;
    total_ += n;
    while (fill_ >= 8) {
      v_.push_back((uint8_t)acc_);
      acc_ >>= 8;
      fill_ -= 8;
    }
  }
  uint64_t bits() const { return total_; }
  void finish() {
    if (fill_) v_.push_back((uint8_t)acc_);
    acc_ = 0;
    fill_ = 0;
    while (v_.size() & 15) v_.push_back(0);
  }

 private:
  std::vector<uint8_t>& v_;
  uint64_t acc_ = 0;
  uint32_t fill_ = 0;
  uint64_t total_ = 0;
};

void put_le(uint8_t* p, uint64_t v, int n) {
  for (int i = 0; i < n; i++) p[i] = (uint8_t)(v >> (8 * i));
}

// Encode one block's sequences into `blk` (header + bitstream).
void encode_block(const uint8_t* in, uint32_t n, const std::vector<Seq>& seqs, const gmp_compress_opts& o,
                  std::vector<uint8_t>& blk) {
  std::vector<uint64_t> f1(gmp::kLitLenSyms, 0), f2(gmp::kOffsetSyms, 0);
  for (const Seq& q : seqs) {
    for (uint32_t k = 0; k < q.lit_len; k++) f1[in[q.lit_start + k]]++;
    if (q.mlen) {
      uint32_t sym, nb, bits;
      dist_code(q.dist, sym, nb, bits);
      f1[254 + q.mlen]++;
      f2[sym]++;
    } else {
      f1[256]++;
    }
  }
  std::vector<uint8_t> l1, l2;
  code_lengths(f1, o.cwl, l1);
  code_lengths(f2, o.cwl, l2);
  std::vector<uint32_t> c1, c2;
  canonical_reversed(l1, c1);
  canonical_reversed(l2, c2);
  const uint32_t K = o.n_sub;
  const size_t hdr = (gmp::kBlockFixed + 12 * K + 15) & ~size_t(15);
  blk.assign(hdr, 0);
  put_le(&blk[0], seqs.size(), 4);
  put_le(&blk[4], n, 4);
  for (uint32_t s = 0; s < gmp::kLitLenSyms; s++) blk[8 + s / 2] |= (uint8_t)(l1[s] << (4 * (s & 1)));
  for (uint32_t s = 0; s < gmp::kOffsetSyms; s++) blk[168 + s / 2] |= (uint8_t)(l2[s] << (4 * (s & 1)));
  BitSink bs(blk);
  // Sub-blocks of equal decoding work: a lane decodes one literal/length
  // symbol per step, so sequence q costs lit_len + 1 steps; sub-block j ends
  // where the running cost first reaches (j + 1) / K of the block's total.
  // (A block's first sequences carry most of its literals, since its window
  // starts empty, so an even split by sequence count is uneven in work.)
  uint64_t total_cost = 0;
  for (const Seq& q : seqs) total_cost += q.lit_len + 1ull;
  uint64_t run_cost = 0;
  size_t qi = 0;
  for (uint32_t j = 0; j < K; j++) {
    const uint64_t target = total_cost * (j + 1) / K;
    size_t qe = qi;
    while (qe < seqs.size() && (run_cost < target || j + 1 == K)) run_cost += seqs[qe++].lit_len + 1ull;
    const uint64_t b0 = bs.bits();
    uint32_t outn = 0;
    const uint32_t nseq = (uint32_t)(qe - qi);
    for (; qi < qe; qi++) {
      const Seq& q = seqs[qi];
      for (uint32_t k = 0; k < q.lit_len; k++) {
        uint8_t b = in[q.lit_start + k];
        bs.put(c1[b], l1[b]);
      }
      if (q.mlen) {
        uint32_t ls = 254 + q.mlen, sym, nb, bits;
        bs.put(c1[ls], l1[ls]);
        dist_code(q.dist, sym, nb, bits);
        bs.put(c2[sym], l2[sym]);
        if (nb) bs.put(bits, nb);
      } else {
        bs.put(c1[256], l1[256]);
      }
      outn += q.lit_len + q.mlen;
    }
    uint8_t* e = &blk[gmp::kBlockFixed + 12 * j];
    put_le(e, bs.bits() - b0, 4);
    put_le(e + 4, outn, 4);
    put_le(e + 8, nseq, 4);
  }
  bs.finish();
}

// Encode one block in the byte-level format (Gompresso/Byte, Sec. 3.1):
// header {n_seq, out_bytes, n_lit, 0}, one 4-byte record per sequence
// (literal length | (match length - 2) << 10 | (distance - 1) << 16; match
// code 0 when the sequence has no back-reference), zero padding to 16 bytes,
// the block's literal bytes in order, zero padding to 16 bytes.
void encode_block_byte(const uint8_t* in, uint32_t n, const std::vector<Seq>& seqs, std::vector<uint8_t>& blk) {
  uint64_t n_lit = 0;
  for (const Seq& q : seqs) n_lit += q.lit_len;
  const size_t rec_end = (16 + 4 * seqs.size() + 15) & ~size_t(15);
  blk.assign(rec_end + ((n_lit + 15) & ~uint64_t(15)), 0);
  put_le(&blk[0], seqs.size(), 4);
  put_le(&blk[4], n, 4);
  put_le(&blk[8], n_lit, 4);
  size_t lp = rec_end;
  for (size_t k = 0; k < seqs.size(); k++) {
    const Seq& q = seqs[k];
    const uint32_t rec = q.lit_len | (q.mlen ? ((q.mlen - 2) << 10) | ((q.dist - 1) << 16) : 0u);
    put_le(&blk[16 + 4 * k], rec, 4);
    memcpy(&blk[lp], in + q.lit_start, q.lit_len);
    lp += q.lit_len;
  }
}

// File header, block offset table, blocks and tail padding (gmp.h).
int assemble(const gmp_compress_opts& o, size_t n, const std::vector<std::vector<uint8_t>>& blocks, void* host_out,
             size_t cap, size_t* out_bytes) {
  const size_t nb = blocks.size();
  std::vector<uint64_t> sizes(nb), offsets(nb);
  for (size_t b = 0; b < nb; b++) sizes[b] = blocks[b].size();
  uint64_t total = 0;
  gmp::stream_layout(sizes.data(), nb, offsets.data(), &total);
  if (total > cap) return GMP_ERR_CAPACITY;
  uint8_t* out = static_cast<uint8_t*>(host_out);
  gmp::write_stream_header(o, n, nb, offsets.data(), total, out);
  for (size_t b = 0; b < nb; b++) memcpy(out + offsets[b], blocks[b].data(), blocks[b].size());
  *out_bytes = total;
  return GMP_OK;
}

bool opts_ok(const gmp_compress_opts& o) {
  if (o.block_size == 0 || o.window == 0 || o.window > 32768 || o.max_match < 3 || o.max_match > 64 ||
      o.chain_depth == 0 || o.byte_mode > 1)
    return false;
  return o.byte_mode || (o.n_sub >= 1 && o.n_sub <= gmp::kMaxSub && o.cwl >= 9 && o.cwl <= 12);
}

}  // namespace

namespace gmp {

bool compress_opts_ok(const gmp_compress_opts& o) { return opts_ok(o); }

uint64_t stream_layout(const uint64_t* block_bytes, size_t nb, uint64_t* offsets, uint64_t* total) {
  const uint64_t first = (kHeaderBytes + 8 * (uint64_t)nb + 15) & ~uint64_t(15);
  uint64_t pos = first;
  for (size_t b = 0; b < nb; b++) {
    offsets[b] = pos;
    pos += block_bytes[b];
  }
  *total = pos + 16;
  return first;
}

void write_stream_header(const gmp_compress_opts& o, size_t n, size_t nb, const uint64_t* offsets, uint64_t total,
                         uint8_t* out) {
  const uint64_t first = (kHeaderBytes + 8 * (uint64_t)nb + 15) & ~uint64_t(15);
  memset(out, 0, first);
  memcpy(out, "GMP1", 4);
  put_le(out + 4, GMP_VERSION, 2);
  put_le(out + 6, (o.de ? 1u : 0u) | (o.byte_mode ? 0u : 2u), 2);
  put_le(out + 8, o.block_size, 4);
  put_le(out + 12, o.byte_mode ? 0u : o.n_sub, 2);
  out[14] = (uint8_t)(o.byte_mode ? 0u : o.cwl);
  put_le(out + 16, o.window, 4);
  out[20] = 3;
  out[21] = (uint8_t)o.max_match;
  put_le(out + 24, n, 8);
  put_le(out + 32, nb, 8);
  put_le(out + 40, total, 8);
  for (size_t b = 0; b < nb; b++) put_le(out + kHeaderBytes + 8 * b, offsets[b], 8);
  memset(out + total - 16, 0, 16);
}

}  // namespace gmp

extern "C" {

void gmp_compress_opts_default(gmp_compress_opts* o) {
  o->block_size = 256u << 10;
  o->n_sub = 32;
  o->window = 32768;
  o->cwl = 12;
  o->max_match = 64;
  o->chain_depth = 64;
  o->de = 0;
  o->n_threads = 0;
  o->lazy = 1;
  o->byte_mode = 0;
}

size_t gmp_compress_bound(size_t n, const gmp_compress_opts* o) {
  if (!o || o->block_size == 0) return 0;
  size_t nb = (n + o->block_size - 1) / o->block_size;
  // Byte blocks: at most one 4-byte record per byte plus the literals
  if (o->byte_mode) return gmp::kHeaderBytes + 8 * nb + 16 + nb * 48 + 5 * n + 32;
  size_t per_block = ((gmp::kBlockFixed + 12 * (size_t)o->n_sub + 15) & ~size_t(15)) + 32;
  return gmp::kHeaderBytes + 8 * nb + 16 + nb * per_block + (n * 12 + 7) / 8 + 2 * nb + 32;
}

int gmp_compress(const void* host_in, size_t n, const gmp_compress_opts* opts, void* host_out, size_t cap,
                 size_t* out_bytes) {
  if ((!host_in && n) || !opts || !host_out || !out_bytes) return GMP_ERR_INVALID_ARG;
  gmp_compress_opts o = *opts;
  if (!opts_ok(o)) return GMP_ERR_INVALID_ARG;
  const uint8_t* in = static_cast<const uint8_t*>(host_in);
  const size_t nb = (n + o.block_size - 1) / o.block_size;
  std::vector<std::vector<uint8_t>> blocks;
  try {
    blocks.resize(nb);
  } catch (...) {
    return GMP_ERR_NOMEM;
  }
  unsigned nt = o.n_threads ? o.n_threads : std::max(1u, std::thread::hardware_concurrency());
  nt = (unsigned)std::min<size_t>(nt, std::max<size_t>(nb, 1));
  std::atomic<size_t> next{0};
  std::atomic<bool> failed{false};
  auto worker = [&]() {
    try {
      std::vector<Seq> seqs;
      std::vector<uint32_t> head(size_t(1) << kHashBits), chain;
      for (;;) {
        size_t b = next.fetch_add(1);
        if (b >= nb) break;
        size_t s = b * (size_t)o.block_size;
        uint32_t len = (uint32_t)std::min<size_t>(o.block_size, n - s);
        parse_block(in + s, len, o, seqs, head, chain);
        if (o.byte_mode) encode_block_byte(in + s, len, seqs, blocks[b]);
        else encode_block(in + s, len, seqs, o, blocks[b]);
      }
    } catch (...) {
      failed = true;
    }
  };
  std::vector<std::thread> th;
  for (unsigned t = 1; t < nt; t++) th.emplace_back(worker);
  worker();
  for (auto& t : th) t.join();
  if (failed) return GMP_ERR_NOMEM;
  return assemble(o, n, blocks, host_out, cap, out_bytes);
}

int gmp_encode_tokens(const uint32_t* lit_len, const uint32_t* match_len, const uint32_t* dist, size_t n_seq,
                      const uint8_t* lits, size_t n_lits, const gmp_compress_opts* opts, void* host_out, size_t cap,
                      size_t* out_bytes) {
  if (!opts || !host_out || !out_bytes || (n_seq && (!lit_len || !match_len || !dist)) || (n_lits && !lits))
    return GMP_ERR_INVALID_ARG;
  const gmp_compress_opts& o = *opts;
  if (!opts_ok(o)) return GMP_ERR_INVALID_ARG;
  std::vector<Seq> seqs;
  std::vector<std::vector<uint8_t>> blocks(1);
  uint64_t pos = 0, lp = 0;
  try {
    seqs.reserve(n_seq);
    for (size_t i = 0; i < n_seq; i++) {
      const uint32_t ll = lit_len[i], ml = match_len[i], d = dist[i];
      if (lp + ll > n_lits) return GMP_ERR_INVALID_ARG;
      if (ml && (ml < 3 || ml > o.max_match || d == 0 || d > o.window || d > pos + ll)) return GMP_ERR_INVALID_ARG;
      // Huffman blocks end a sequence without a back-reference only at the end of the block
      if (!ml && !o.byte_mode && i + 1 != n_seq) return GMP_ERR_INVALID_ARG;
      uint32_t start = (uint32_t)lp, rest = ll;
      for (; o.byte_mode && rest > kByteMaxLit; rest -= kByteMaxLit, start += kByteMaxLit)
        seqs.push_back(Seq{start, kByteMaxLit, 0, 0});
      seqs.push_back(Seq{start, rest, ml, ml ? d : 0});
      lp += ll;
      pos += (uint64_t)ll + ml;
      if (pos > o.block_size) return GMP_ERR_INVALID_ARG;
    }
    if (lp != n_lits) return GMP_ERR_INVALID_ARG;
    if (o.byte_mode) encode_block_byte(lits, (uint32_t)pos, seqs, blocks[0]);
    else encode_block(lits, (uint32_t)pos, seqs, o, blocks[0]);
  } catch (...) {
    return GMP_ERR_NOMEM;
  }
  if (pos == 0) blocks.clear();  // an empty stream has no blocks
  return assemble(o, pos, blocks, host_out, cap, out_bytes);
}

}  // extern "C"
