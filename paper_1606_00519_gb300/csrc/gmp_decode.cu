// gmp_decode.cu - sm_103a decompression kernels of libgmp (Gompresso-style,
// arXiv:1606.00519).
//
// One persistent launch; each warp repeatedly takes a work item (one block of
// one stream) from a device counter and decodes it in two phases:
//
//  Phase A, Huffman decoding (Sec. 3.2.1): the warp builds the 4096-entry
//  lookup tables of the block's two canonical trees in shared memory, then
//  lane j decodes sub-block j (lanes take j, j+32 for K > 32), starting at
//  the bit offset given by the prefix sum of the stored sub-block sizes.
//  One table lookup per symbol, no tree walk.  Each lane writes its
//  sequences as 8-byte records {lit_len, (distance << 8) | match_len} and its
//  literal bytes to the warp's scratch slot (device memory, as in the paper,
//  where the decoder's token stream goes to device memory).
//
//  Phase B, LZ77 decompression (Sec. 3.2.2, Sec. 4): the warp walks the
//  block's sequences 32 at a time, one per lane: an exclusive prefix sum of
//  (literal length + match length) by shuffle gives each lane's output
//  position, a second one of the literal lengths its literal source; the
//  lanes copy their literal strings, then resolve their back-references by
//  Multi-Round Resolution (Fig. 5) or, for a DE stream (Fig. 6), all in one
//  pass.  Output bytes go to a 16 KiB ring in shared memory that also serves
//  recent back-reference sources; completed 16-byte chunks are flushed to the
//  caller's buffer with coalesced 16-byte stores, so every output byte is
//  written to device memory once.
//
// MRR reading (the printed algorithm is ambiguous, see the comment at
// resolve_mrr): HWM = write position of the lowest pending lane; a lane may
// copy once min(read_pos + length, write_pos) <= HWM.
//
// Every read of the compressed stream is bounds-checked; every loop over
// input data is bounded by sizes checked against the block header; corrupt
// input sets the caller's status word and abandons the block.  No waits on
// other warps or blocks exist.

#include <cuda_runtime.h>
#include <stdint.h>

#include "gmp.h"
#include "gmp_internal.h"

namespace gmp {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int LUT_BITS = 12;
constexpr int LUT_SIZE = 1 << LUT_BITS;
constexpr int N_LL = 319;
constexpr int N_OFF = 30;
constexpr int MAX_SUB = 64;
constexpr int RING = 16384;  // shared-memory output ring per warp (bytes)
constexpr uint32_t RING_MASK = RING - 1;
constexpr uint32_t GROUP_FAST_MAX = RING / 2;

struct __align__(16) WarpSmem {
  union {
    struct {
      uint16_t ll[LUT_SIZE];
      uint16_t off[LUT_SIZE];
    } lut;
    uint8_t ring[RING];
  } u;
  uint32_t sb_bit[MAX_SUB];      // sub-block start bit (from the bitstream start)
  uint32_t sb_bits[MAX_SUB];     // sub-block size in bits
  uint32_t sb_out[MAX_SUB];      // sub-block output start (block-relative)
  uint32_t sb_outn[MAX_SUB];     // sub-block output bytes
  uint32_t sb_seq[MAX_SUB + 1];  // sub-block first sequence; sb_seq[K] = n_seq
  uint32_t sb_seqn[MAX_SUB];
  uint32_t sb_lit[MAX_SUB];      // literal count, then literal-source delta
  uint32_t cnt[16];              // LUT build: code count per length
  uint32_t idx[16];              // LUT build: first sorted index per length
  uint32_t first[16];            // LUT build: first canonical code per length
  uint32_t run[16];              // LUT build: running rank per length
  uint16_t sorted[N_LL + 1];
  uint8_t lens[N_LL + N_OFF + 3];
};

struct KParams {
  const gmp_file_desc* files;  // batch mode; nullptr in single-stream mode
  const uint64_t* item_start;  // batch mode: n_files + 1 prefix sums
  uint32_t n_files;
  gmp_file_desc single;  // single-stream mode
  int32_t* status;       // one per file
  unsigned long long* counter;
  uint8_t* scratch;
  uint64_t slot_bytes;
  uint32_t max_seq, max_out;
  unsigned long long* stats;  // [groups, rounds, de_fallback, blocks, max_rounds]
  int collect_stats;
};

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ void set_status(int32_t* st, int code) { atomicCAS(st, 0, code); }

__device__ __forceinline__ uint32_t ld_u32_nc(const uint8_t* p) { return __ldg(reinterpret_cast<const uint32_t*>(p)); }
__device__ __forceinline__ uint64_t ld_u64_nc(const uint8_t* p) {
  return __ldg(reinterpret_cast<const unsigned long long*>(p));
}

// inclusive warp scan of a 32-bit value
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const uint32_t lane = lane_id();
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t y = __shfl_up_sync(FULL, v, d);
    if (lane >= (uint32_t)d) v += y;
  }
  return v;
}

// ---------------------------------------------------------------------------
// Lookup table of one canonical tree (Sec. 3.1, 3.2.1).  Entry for the 12-bit
// LSB-first peek e: the code whose bit-reversed value prefixes e; stored as
// (length << 9) | symbol, 0 = no code.  Returns false when the code lengths
// do not form a complete prefix code (Kraft sum != 1) and are not all zero.
__device__ bool build_lut(WarpSmem& S, const uint8_t* lens, int n, uint16_t* lut) {
  const uint32_t lane = lane_id();
  if (lane < 16) { S.cnt[lane] = 0; S.run[lane] = 0; }
  __syncwarp();
  for (int base = 0; base < n; base += 32) {
    int s = base + (int)lane;
    uint32_t L = s < n ? lens[s] : 0u;
    uint32_t m = __match_any_sync(FULL, L);
    if ((__ffs(m) - 1) == (int)lane) S.cnt[L] += __popc(m);
    __syncwarp();
  }
  // Kraft sum and first codes
  bool ok = true;
  uint32_t used = 0;
  if (lane == 0) {
    uint32_t k = 0, code = 0, id = 0;
    for (int L = 1; L <= LUT_BITS; L++) {
      k += S.cnt[L] << (LUT_BITS - L);
      S.first[L] = code;
      S.idx[L] = id;
      id += S.cnt[L];
      code = (code + S.cnt[L]) << 1;
    }
    used = id;
    // lengths above 12 have no table slot: such a header is invalid
    const bool too_long = (S.cnt[13] | S.cnt[14] | S.cnt[15]) != 0;
    S.idx[0] = (!too_long && (used == 0 || k == (uint32_t)LUT_SIZE)) ? 1u : 0u;  // validity flag
    S.first[0] = used;
  }
  __syncwarp();
  ok = S.idx[0] != 0;
  used = S.first[0];
  if (!ok) return false;
  if (used == 0) {
    for (int e = (int)lane; e < LUT_SIZE; e += 32) lut[e] = 0;
    __syncwarp();
    return true;
  }
  // symbols sorted by (length, symbol)
  for (int base = 0; base < n; base += 32) {
    int s = base + (int)lane;
    uint32_t L = s < n ? lens[s] : 0u;
    uint32_t m = __match_any_sync(FULL, L);
    uint32_t r = __popc(m & ((1u << lane) - 1u));
    if (L) S.sorted[S.idx[L] + S.run[L] + r] = (uint16_t)s;
    __syncwarp();
    if (r == 0) S.run[L] += __popc(m);
    __syncwarp();
  }
  // limits of each length's code range, left-justified to 12 bits
  uint32_t lim[LUT_BITS + 1];
#pragma unroll
  for (int L = 1; L <= LUT_BITS; L++) lim[L] = (S.first[L] + S.cnt[L]) << (LUT_BITS - L);
  for (int e = (int)lane; e < LUT_SIZE; e += 32) {
    uint32_t v = __brev((uint32_t)e) >> (32 - LUT_BITS);  // peek bits, most significant first
    uint32_t L = 1;
#pragma unroll
    for (int i = 1; i < LUT_BITS; i++) L += (v >= lim[i]) ? 1u : 0u;
    uint32_t sh = LUT_BITS - L;
    uint32_t sym = S.sorted[S.idx[L] + (v >> sh) - S.first[L]];
    lut[e] = (uint16_t)((L << 9) | sym);
  }
  __syncwarp();
  return true;
}

// ---------------------------------------------------------------------------
// Back-reference copy of one lane into the ring: ml bytes from rpos to wpos
// (block-relative), byte by byte in order, so an overlapping copy (distance <
// length) repeats its pattern.  Sources below ring_lo come from the output in
// device memory, which is complete below ring_lo.
__device__ __forceinline__ void copy_match_ring(uint8_t* ring, const uint8_t* out_blk, uint32_t rpos, uint32_t wpos,
                                                uint32_t ml, uint32_t ring_lo) {
  for (uint32_t i = 0; i < ml; i++) {
    uint32_t s = rpos + i;
    uint8_t v = (s >= ring_lo) ? ring[s & RING_MASK] : out_blk[s];
    ring[(wpos + i) & RING_MASK] = v;
  }
}

__device__ __forceinline__ void copy_match_global(uint8_t* out_blk, uint32_t rpos, uint32_t wpos, uint32_t ml) {
  for (uint32_t i = 0; i < ml; i++) out_blk[wpos + i] = out_blk[rpos + i];
}

// Multi-Round Resolution (Fig. 5, Sec. 4.1).  The figure names the last
// writer with count_leading_zero_bits(ballot) and waits for read_pos + length
// <= HWM; the first picks the highest pending lane rather than the last
// completed one, and the second never admits an overlapping copy (offset <
// length), whose source extends into its own output.  Reading used here: the
// lowest pending lane f = ffs(ballot(pending)) - 1 has every earlier lane
// complete and its own literals written, so HWM = write_pos(f); a pending lane
// copies once min(read_pos + length, write_pos) <= HWM.  Lane f always
// qualifies, so every round resolves at least one lane and a group needs at
// most 32 rounds; a group whose back-references do not depend on each other
// resolves in one round.  Returns the number of rounds, or -1 on no progress.
template <bool RING_PATH>
__device__ int resolve_mrr(uint8_t* ring, uint8_t* out_blk, uint32_t rpos, uint32_t wpos, uint32_t ml, bool pending,
                           uint32_t ring_lo) {
  int rounds = 0;
  for (;;) {
    uint32_t votes = __ballot_sync(FULL, pending);
    if (votes == 0) break;
    if (rounds == 32) return -1;
    int f = __ffs(votes) - 1;
    uint32_t hwm = __shfl_sync(FULL, wpos, f);
    uint32_t lim = min(rpos + ml, wpos);
    if (pending && lim <= hwm) {
      if (RING_PATH) copy_match_ring(ring, out_blk, rpos, wpos, ml, ring_lo);
      else copy_match_global(out_blk, rpos, wpos, ml);
      pending = false;
    }
    __syncwarp();
    rounds++;
  }
  return rounds;
}

// DE property check of one group (Sec. 4.2): each back-reference's source
// bytes before its own write position must avoid every other back-reference
// of the group.  Write positions rise with the lane, so the only candidate to
// test is the last lane whose write position lies below the source's end.
__device__ __forceinline__ bool de_group_ok(uint32_t rpos, uint32_t wpos, uint32_t ml) {
  const uint32_t lane = lane_id();
  uint32_t b = min(rpos + ml, wpos);
  int lo = -1;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    int cand = lo + step;
    uint32_t w = __shfl_sync(FULL, wpos, min(cand, 31));
    if (cand <= 31 && w < b) lo = cand;
  }
  uint32_t end_lo = __shfl_sync(FULL, wpos + ml, max(lo, 0));
  bool bad = ml > 0 && lo >= 0 && lo != (int)lane && rpos < end_lo;
  return __ballot_sync(FULL, bad) == 0;
}

// ---------------------------------------------------------------------------
// Decode one block.  Returns false if an error was recorded.
__device__ void decode_block(WarpSmem& S, const KParams& P, const gmp_file_desc& F, uint64_t b, int32_t* status,
                             uint8_t* slot, unsigned long long* st_acc) {
  const uint32_t lane = lane_id();
  const uint8_t* comp = F.comp;
  // ---- stream header (64 bytes), block reference
  int err = 0;
  uint32_t flags = 0, K = 0, window = 0, max_match = 0;
  if (F.comp_bytes < 64 || (((uintptr_t)comp) & 15u)) {
    if (lane == 0) set_status(status, GMP_STATUS_BAD_HEADER);
    return;
  }
  {
    uint32_t magic = ld_u32_nc(comp);
    uint32_t w1 = ld_u32_nc(comp + 4);
    uint32_t w3 = ld_u32_nc(comp + 12);
    window = ld_u32_nc(comp + 16);
    uint32_t w5 = ld_u32_nc(comp + 20);
    flags = w1 >> 16;
    K = w3 & 0xffffu;
    uint32_t cwl = (w3 >> 16) & 0xffu;
    max_match = (w5 >> 8) & 0xffu;
    if (magic != 0x31504d47u || (w1 & 0xffffu) != 1u || !(flags & 2u) || K == 0 || K > MAX_SUB || cwl == 0 ||
        cwl > 12 || window == 0 || window > 32768 || (w5 & 0xffu) != 3u || max_match < 3 || max_match > 64)
      err = GMP_STATUS_BAD_HEADER;
  }
  const gmp_block_ref br = F.index[b];
  if (!err) {
    if ((br.comp_offset & 15) || br.comp_offset > F.comp_bytes || br.comp_bytes > F.comp_bytes - br.comp_offset ||
        br.out_offset > F.out_cap || br.out_bytes > F.out_cap - br.out_offset)
      err = GMP_STATUS_OUTPUT_OVERRUN;
    else if (br.comp_bytes < 192 + 12ull * K)
      err = GMP_STATUS_BAD_HEADER;
  }
  if (err) {
    if (lane == 0) set_status(status, err);
    return;
  }
  const uint8_t* B = comp + br.comp_offset;
  const uint32_t n_seq = ld_u32_nc(B);
  const uint32_t out_bytes = ld_u32_nc(B + 4);
  if (out_bytes != br.out_bytes) err = GMP_STATUS_BAD_HEADER;
  else if (out_bytes > P.max_out || n_seq > P.max_seq) err = GMP_STATUS_CAPACITY;
  if (err) {
    if (lane == 0) set_status(status, err);
    return;
  }
  const uint32_t bs_off = (192u + 12u * K + 15u) & ~15u;  // bitstream start within the block
  const uint64_t bits_avail = (br.comp_bytes - bs_off) * 8ull;

  // ---- sub-block table: prefix sums of bit sizes, output sizes, sequences
  {
    uint32_t carry_bit = 0, carry_out = 0, carry_seq = 0;
    for (uint32_t base = 0; base < K; base += 32) {
      uint32_t j = base + lane;
      uint32_t nb = 0, no = 0, ns = 0;
      if (j < K) {
        const uint8_t* e = B + 192 + 12 * j;
        nb = ld_u32_nc(e);
        no = ld_u32_nc(e + 4);
        ns = ld_u32_nc(e + 8);
      }
      uint32_t ib = warp_incl_scan(nb), io = warp_incl_scan(no), is = warp_incl_scan(ns);
      if (j < K) {
        S.sb_bit[j] = carry_bit + ib - nb;
        S.sb_bits[j] = nb;
        S.sb_out[j] = carry_out + io - no;
        S.sb_outn[j] = no;
        S.sb_seq[j] = carry_seq + is - ns;
        S.sb_seqn[j] = ns;
      }
      // sizes are checked below against 64-bit totals, so a wrapped 32-bit
      // sum cannot pass: the totals are bounded by out_bytes / n_seq.
      carry_bit += __shfl_sync(FULL, ib, 31);
      carry_out += __shfl_sync(FULL, io, 31);
      carry_seq += __shfl_sync(FULL, is, 31);
    }
    if (lane == 0) S.sb_seq[K] = carry_seq;
    // overflow-safe totals
    uint64_t tb = 0, to = 0, ts = 0;
    for (uint32_t j = lane; j < K; j += 32) {
      const uint8_t* e = B + 192 + 12 * j;
      tb += ld_u32_nc(e);
      to += ld_u32_nc(e + 4);
      ts += ld_u32_nc(e + 8);
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
      tb += __shfl_xor_sync(FULL, tb, d);
      to += __shfl_xor_sync(FULL, to, d);
      ts += __shfl_xor_sync(FULL, ts, d);
    }
    if (ts != n_seq || to != out_bytes) err = GMP_STATUS_BAD_HEADER;
    else if (tb > bits_avail) err = GMP_STATUS_BITSTREAM;
  }
  if (err) {
    if (lane == 0) set_status(status, err);
    return;
  }

  // ---- code lengths and lookup tables (Sec. 3.2.1)
  for (uint32_t i = lane; i < (uint32_t)(N_LL + N_OFF); i += 32) {
    uint32_t sym = i < (uint32_t)N_LL ? i : i - N_LL;
    uint32_t byte = i < (uint32_t)N_LL ? 8 + (sym >> 1) : 168 + (sym >> 1);
    uint8_t v = __ldg(B + byte);
    S.lens[i] = (sym & 1) ? (v >> 4) : (v & 15);
  }
  __syncwarp();
  bool ok1 = build_lut(S, S.lens, N_LL, S.u.lut.ll);
  bool ok2 = build_lut(S, S.lens + N_LL, N_OFF, S.u.lut.off);
  if (!ok1 || !ok2) {
    if (lane == 0) set_status(status, GMP_STATUS_BAD_HEADER);
    return;
  }

  // ---- Phase A: lane per sub-block Huffman decode
  uint2* rec = reinterpret_cast<uint2*>(slot);
  uint8_t* shadow = slot + (uint64_t)P.max_seq * 8;
  const uint8_t* bs = B + bs_off;
  const uint64_t bs_words = (br.comp_bytes - bs_off) / 4;  // whole 32-bit words inside the block
  for (uint32_t j = lane; j < K; j += 32) {
    uint32_t pos = S.sb_bit[j];
    const uint32_t end = pos + S.sb_bits[j];
    uint32_t wi = pos >> 5;
    auto ldw = [&](uint32_t w) -> uint32_t { return (uint64_t)w < bs_words ? ld_u32_nc(bs + 4ull * w) : 0u; };
    uint64_t buf = ((uint64_t)ldw(wi) | ((uint64_t)ldw(wi + 1) << 32)) >> (pos & 31);
    int nb = 64 - (int)(pos & 31);
    wi += 2;
    uint32_t outp = S.sb_out[j];
    const uint32_t out_end = outp + S.sb_outn[j];
    uint32_t lit_dst = ((S.sb_out[j] + 15u) & ~15u) + 16u * j;
    uint32_t nlit = 0;
    uint32_t q = S.sb_seq[j];
    const uint32_t q_end = q + S.sb_seqn[j];
    for (; q < q_end && !err; q++) {
      uint32_t lit_run = 0, ml = 0, dist = 0;
      for (;;) {
        if (nb < 32) {
          buf |= (uint64_t)ldw(wi++) << nb;
          nb += 32;
        }
        uint32_t e = S.u.lut.ll[buf & (LUT_SIZE - 1)];
        uint32_t L = e >> 9, sym = e & 511u;
        buf >>= L;
        nb -= (int)L;
        pos += L;
        if (L == 0) { err = GMP_STATUS_CORRUPT_SYMBOL; break; }
        if (pos > end) { err = GMP_STATUS_BITSTREAM; break; }
        if (sym < 256) {
          if (outp >= out_end) { err = GMP_STATUS_OUTPUT_OVERRUN; break; }
          shadow[lit_dst + nlit] = (uint8_t)sym;
          nlit++;
          lit_run++;
          outp++;
          continue;
        }
        if (sym == 256) {
          if (q + 1 != n_seq) err = GMP_STATUS_CORRUPT_SYMBOL;  // only the block's last sequence
          break;
        }
        ml = sym - 254u;
        if (nb < 32) {
          buf |= (uint64_t)ldw(wi++) << nb;
          nb += 32;
        }
        uint32_t e2 = S.u.lut.off[buf & (LUT_SIZE - 1)];
        uint32_t L2 = e2 >> 9, os = e2 & 31u;
        if (L2 == 0 || os >= (uint32_t)N_OFF) { err = GMP_STATUS_CORRUPT_SYMBOL; break; }
        buf >>= L2;
        uint32_t ne = os < 4 ? 0u : (os >> 1) - 1u;
        uint32_t extra = (uint32_t)buf & ((1u << ne) - 1u);
        buf >>= ne;
        nb -= (int)(L2 + ne);
        pos += L2 + ne;
        if (pos > end) { err = GMP_STATUS_BITSTREAM; break; }
        dist = os < 4 ? os + 1u : ((2u | (os & 1u)) << ne) + extra + 1u;
        if (ml > max_match) { err = GMP_STATUS_CORRUPT_SYMBOL; break; }
        if (dist > window || dist > outp) { err = GMP_STATUS_BAD_OFFSET; break; }
        if (ml > out_end - outp) { err = GMP_STATUS_OUTPUT_OVERRUN; break; }
        outp += ml;
        break;
      }
      if (err) break;
      rec[q] = make_uint2(lit_run, (dist << 8) | ml);
    }
    if (!err && (pos != end)) err = GMP_STATUS_BITSTREAM;
    if (!err && outp != out_end) err = GMP_STATUS_OUTPUT_OVERRUN;
    S.sb_lit[j] = nlit;
  }
  if (err) set_status(status, err);
  if (__ballot_sync(FULL, err != 0)) return;
  __syncwarp();  // phase A's records and literals are visible to the whole warp

  // literal-source delta per sub-block: shadow start minus literals before it
  {
    uint32_t carry = 0;
    for (uint32_t base = 0; base < K; base += 32) {
      uint32_t j = base + lane;
      uint32_t n = j < K ? S.sb_lit[j] : 0u;
      uint32_t inc = warp_incl_scan(n);
      if (j < K) S.sb_lit[j] = (((S.sb_out[j] + 15u) & ~15u) + 16u * j) - (carry + inc - n);
      carry += __shfl_sync(FULL, inc, 31);
    }
  }
  __syncwarp();

  // ---- Phase B: 32 sequences per step (Sec. 3.2.2)
  uint8_t* out_blk = F.out + br.out_offset;
  const bool vec_ok = (((uintptr_t)out_blk) & 15u) == 0;
  const bool de = (flags & 1u) != 0;
  uint8_t* ring = S.u.ring;
  uint32_t G0 = 0, litpos = 0, flushed = 0, ring_valid_lo = 0;
  uint32_t jc = 0;
  unsigned long long n_groups = 0, n_rounds = 0, n_fallback = 0, max_rounds = 0;
  const uint32_t n_groups_total = (n_seq + 31) / 32;
  for (uint32_t g = 0; g < n_groups_total; g++) {
    const uint32_t t = g * 32 + lane;
    const bool valid = t < n_seq;
    uint2 r = valid ? rec[t] : make_uint2(0, 0);
    const uint32_t ll = r.x, ml = r.y & 0xffu, dist = r.y >> 8;
    const uint32_t tot = ll + ml;
    const uint32_t inc_tot = warp_incl_scan(tot);
    const uint32_t inc_ll = warp_incl_scan(ll);
    const uint32_t g_total = __shfl_sync(FULL, inc_tot, 31);
    const uint32_t g_lits = __shfl_sync(FULL, inc_ll, 31);
    const uint32_t dst = G0 + inc_tot - tot;
    uint32_t j = jc;
    if (valid)
      while (j + 1 < K && t >= S.sb_seq[j + 1]) j++;
    const uint32_t lsrc = S.sb_lit[j] + litpos + inc_ll - ll;
    jc = __shfl_sync(FULL, j, 31);
    const uint32_t wpos = dst + ll;
    const uint32_t rpos = wpos - dist;
    const bool pending = valid && ml > 0;
    int rounds;
    if (g_total <= GROUP_FAST_MAX) {
      const uint32_t ring_lo = max(ring_valid_lo, G0 > RING / 2 ? G0 - RING / 2 : 0u);
      for (uint32_t i = 0; i < ll; i++) ring[(dst + i) & RING_MASK] = shadow[lsrc + i];
      __syncwarp();
      if (de && de_group_ok(rpos, wpos, ml)) {
        if (pending) copy_match_ring(ring, out_blk, rpos, wpos, ml, ring_lo);
        __syncwarp();
        rounds = __ballot_sync(FULL, pending) ? 1 : 0;
      } else {
        if (de) n_fallback++;
        rounds = resolve_mrr<true>(ring, out_blk, rpos, wpos, ml, pending, ring_lo);
      }
      // flush completed 16-byte chunks; after a large group `flushed` may be
      // unaligned, so its first partial chunk goes out byte by byte
      const uint32_t fend = (G0 + g_total) & ~15u;
      if (fend > flushed) {
        const uint32_t head_end = min((flushed + 15u) & ~15u, fend);
        if (lane < head_end - flushed) out_blk[flushed + lane] = ring[(flushed + lane) & RING_MASK];
        if (vec_ok) {
          for (uint32_t c = head_end + 16u * lane; c < fend; c += 512u)
            *reinterpret_cast<uint4*>(out_blk + c) = *reinterpret_cast<const uint4*>(ring + (c & RING_MASK));
        } else {
          for (uint32_t c = head_end + lane; c < fend; c += 32u) out_blk[c] = ring[c & RING_MASK];
        }
        flushed = fend;
      }
    } else {
      // a group too large for the ring: write it straight to device memory
      for (uint32_t c = flushed + lane; c < G0; c += 32u) out_blk[c] = ring[c & RING_MASK];
      __syncwarp();
      for (uint32_t i = 0; i < ll; i++) out_blk[dst + i] = shadow[lsrc + i];
      __syncwarp();
      if (de && de_group_ok(rpos, wpos, ml)) {
        if (pending) copy_match_global(out_blk, rpos, wpos, ml);
        __syncwarp();
        rounds = __ballot_sync(FULL, pending) ? 1 : 0;
      } else {
        if (de) n_fallback++;
        rounds = resolve_mrr<false>(ring, out_blk, rpos, wpos, ml, pending, 0);
      }
      flushed = G0 + g_total;
      ring_valid_lo = flushed;
    }
    if (rounds < 0) {
      if (lane == 0) set_status(status, GMP_STATUS_MRR_NO_PROGRESS);
      return;
    }
    __syncwarp();
    if (rounds > 0) n_groups++;
    n_rounds += (unsigned)rounds;
    if ((unsigned long long)rounds > max_rounds) max_rounds = (unsigned)rounds;
    G0 += g_total;
    litpos += g_lits;
  }
  // tail bytes not yet flushed
  for (uint32_t c = flushed + lane; c < out_bytes; c += 32u) out_blk[c] = ring[c & RING_MASK];
  if (G0 != out_bytes && lane == 0) set_status(status, GMP_STATUS_OUTPUT_OVERRUN);
  __syncwarp();
  st_acc[0] += n_groups;
  st_acc[1] += n_rounds;
  st_acc[2] += n_fallback;
  st_acc[3] += 1;
  if (max_rounds > st_acc[4]) st_acc[4] = max_rounds;
}

// Persistent kernel: warps take work items until none are left.
__global__ void __launch_bounds__(32 * 16) decode_kernel(const KParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t lane = lane_id();
  WarpSmem& S = reinterpret_cast<WarpSmem*>(smem_raw)[warp];
  const uint64_t gw = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  uint8_t* slot = P.scratch + gw * P.slot_bytes;
  uint64_t total;
  if (P.files) total = P.item_start[P.n_files];
  else total = P.single.n_blocks;
  unsigned long long st_acc[5] = {0, 0, 0, 0, 0};
  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(P.counter, 1ull);
    item = __shfl_sync(FULL, item, 0);
    if (item >= total) break;
    uint32_t file = 0;
    uint64_t b = item;
    gmp_file_desc F;
    if (P.files) {
      // last file whose first item <= item
      uint32_t lo = 0, hi = P.n_files - 1;
      while (lo < hi) {
        uint32_t mid = (lo + hi + 1) >> 1;
        if (P.item_start[mid] <= item) lo = mid;
        else hi = mid - 1;
      }
      file = lo;
      b = item - P.item_start[file];
      F = P.files[file];
    } else {
      F = P.single;
    }
    decode_block(S, P, F, b, P.status + file, slot, st_acc);
    __syncwarp();
  }
  if (P.collect_stats && lane == 0 && st_acc[3]) {
    atomicAdd(&P.stats[0], st_acc[0]);
    atomicAdd(&P.stats[1], st_acc[1]);
    atomicAdd(&P.stats[2], st_acc[2]);
    atomicAdd(&P.stats[3], st_acc[3]);
    atomicMax(&P.stats[4], st_acc[4]);
  }
}

// Work-item prefix over the files of a batch: item_start[i] = sum of the
// block counts of files before i.  One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) batch_prefix_kernel(const gmp_file_desc* files, uint32_t n_files,
                                                            uint64_t* item_start) {
  __shared__ unsigned long long warp_sums[32];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  for (uint32_t base = 0; base < n_files; base += 1024) {
    uint32_t i = base + threadIdx.x;
    unsigned long long v = i < n_files ? files[i].n_blocks : 0ull;
    unsigned long long x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      unsigned long long y = __shfl_up_sync(FULL, x, d);
      if (lane >= (uint32_t)d) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      unsigned long long w = warp_sums[lane];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        unsigned long long y = __shfl_up_sync(FULL, w, d);
        if (lane >= (uint32_t)d) w += y;
      }
      warp_sums[lane] = w;
    }
    __syncthreads();
    unsigned long long excl = carry + (warp ? warp_sums[warp - 1] : 0ull) + x - v;
    if (i < n_files) item_start[i] = excl;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sums[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) item_start[n_files] = carry;
}

}  // namespace gmp

// ---------------------------------------------------------------------------
// Launch helpers used by the host side (gmp_host.cpp).

namespace gmp {

size_t warp_smem_bytes() { return sizeof(WarpSmem); }

cudaError_t configure_kernel(size_t smem_bytes) {
  return cudaFuncSetAttribute(decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

cudaError_t occupancy(int warps_per_cta, size_t smem_bytes, int* ctas_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, decode_kernel, warps_per_cta * 32, smem_bytes);
}

cudaError_t launch_decode(const LaunchShape& shape, const gmp_file_desc* files, const uint64_t* item_start,
                          uint32_t n_files, const gmp_file_desc* single, int32_t* status,
                          unsigned long long* counter, uint8_t* scratch, uint64_t slot_bytes, uint32_t max_seq,
                          uint32_t max_out, unsigned long long* stats, int collect_stats, cudaStream_t stream) {
  KParams P;
  P.files = files;
  P.item_start = item_start;
  P.n_files = n_files;
  if (single) P.single = *single;
  else memset(&P.single, 0, sizeof(P.single));
  P.status = status;
  P.counter = counter;
  P.scratch = scratch;
  P.slot_bytes = slot_bytes;
  P.max_seq = max_seq;
  P.max_out = max_out;
  P.stats = stats;
  P.collect_stats = collect_stats;
  // the attribute is per kernel, so set it for this launch's shape (contexts
  // with different shapes may share the process)
  cudaError_t e = configure_kernel(shape.smem_bytes);
  if (e != cudaSuccess) return e;
  decode_kernel<<<shape.grid, shape.warps_per_cta * 32, shape.smem_bytes, stream>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_batch_prefix(const gmp_file_desc* files, uint32_t n_files, uint64_t* item_start,
                                cudaStream_t stream) {
  batch_prefix_kernel<<<1, 1024, 0, stream>>>(files, n_files, item_start);
  return cudaGetLastError();
}

}  // namespace gmp
