// gmp_decode.cu - sm_103a decompression kernels of libgmp (Gompresso-style,
// arXiv:1606.00519).
//
// One persistent launch; each warp repeatedly takes a work item (one block of
// one stream; the first one fixed per warp, the rest from a device counter)
// and decodes it in two phases:
//
//  Phase A, Huffman decoding (Sec. 3.2.1): the warp builds the lookup
//  tables of the block's two canonical trees in shared memory (4096 or 2048
//  literal/length entries, by kernel instance, and 1024 offset entries; the
//  rare longer codes are decoded from the canonical arrays),
//  then lane j decodes sub-block j (lanes take j, j+32 for K > 32), starting
//  at the bit offset given by the prefix sum of the stored sub-block sizes.
//  One table lookup per symbol, no tree walk.  Each lane writes its
//  sequences as 16-byte records {output position, literal source, literal
//  length, (distance << 8) | match length} and its literal bytes to the
//  warp's scratch slot (device memory, as in the paper, where the decoder's
//  token stream goes to device memory): literals eight at a time, records
//  (in the 96-register instance) two at a time, since every store of the 32
//  lanes to 32 places costs a memory request per lane.  The lane knows each sequence's
//  output position and literal source as it decodes it, so the records carry
//  the results of the two prefix sums of Sec. 3.2.2.
//
//  Phase B, LZ77 decompression (Sec. 3.2.2, Sec. 4): the warp walks the
//  block's sequences 32 at a time, one per lane: the lanes copy their
//  literal strings, then resolve their back-references by Multi-Round
//  Resolution (Fig. 5) or, for a DE stream (Fig. 7), all in one pass.
//  Output bytes go to a 4 KiB ring in shared memory that also serves recent
//  back-reference sources (older ones are staged by cp.async one group
//  ahead); completed 16-byte chunks are flushed to the caller's buffer with
//  coalesced 16-byte stores, so every output byte is written to device
//  memory once.
//
//  Byte blocks (Gompresso/Byte, Sec. 3.1) have no phase A: their sequence
//  records and literal bytes are read by phase B straight from the stream,
//  positions by one shuffle scan per group, with each group's records
//  checked before it is staged or copied.
//
// MRR reading (the printed algorithm is ambiguous, see the comment at
// resolve_group): HWM = write position of the lowest pending lane; a lane may
// copy once min(read_pos + length, write_pos) <= HWM.  For ablation a context
// can force MRR on DE streams or resolve by Sequential Copying (Sec. 5.1).
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

// Optional stage timers of the LZ77 phase (profiling builds only: compile
// with -DGMP_PHASE_TIMERS); they add SM-clock deltas per stage into the
// statistics' detail counters.
#ifdef GMP_PHASE_TIMERS
#define GMP_TSTAMP(v) const long long v = clock64()
#define GMP_TADD(slot, a, b) tdet[slot] += (unsigned long long)((b) - (a))
#else
#define GMP_TSTAMP(v)
#define GMP_TADD(slot, a, b)
#endif
constexpr int LUT_BITS = 12;  // the longest code (cwl <= 12)
constexpr int LUT_SIZE = 1 << LUT_BITS;
// The lookup tables cover codes of up to LLB (literal/length tree: 12 bits in
// the 128-register kernel, 11 in the 96-register one, whose 20 warps per SM
// need a smaller table) and OFF_BITS (offset tree) bits; the rare longer
// codes are decoded from the tree's canonical arrays (decode_long).
constexpr int OFF_BITS = 10;
constexpr int OFF_SIZE = 1 << OFF_BITS;
constexpr uint16_t LONG_CODE = 0xffff;
constexpr int N_LL = 319;
constexpr int N_OFF = 30;
constexpr int MAX_SUB = 64;
constexpr int RING = 4096;  // shared-memory output ring per warp (bytes)
constexpr uint32_t RING_MASK = RING - 1;
// back-reference sources at most NEAR bytes below the group start are read
// from the ring; older ("far") ones are staged from device memory by cp.async
// one group ahead
constexpr uint32_t NEAR = RING / 2;
constexpr uint32_t GROUP_FAST_MAX = NEAR - 16;
// per lane: a 64-byte source spans at most 5 aligned 16-byte chunks
constexpr int FAR_STAGE = 80;
// per group: the group's literal bytes when they are one contiguous run of
// the shadow (all in one sub-block) and fit, with alignment, in 32 chunks
constexpr int LIT_STAGE = 512;
constexpr uint32_t RING_WMASK = RING / 4 - 1;

// Canonical arrays of one tree (Sec. 3.1): per code length its code count,
// its first index in the symbol list sorted by (length, symbol), and its
// first code.
struct Canon {
  uint32_t cnt[16], idx[16], first[16];
};

// Phase A: the lookup tables, the trees' canonical arrays and the sub-block
// table of the block being decoded.
template <int LLB>
struct PhaseASmem {
  uint16_t ll[1 << LLB];
  uint16_t off[OFF_SIZE];
  Canon cll, coff;
  uint32_t run[16];            // LUT build: running rank per length
  uint32_t sb_bit[MAX_SUB];    // sub-block start bit (from the bitstream start)
  uint32_t sb_bits[MAX_SUB];   // sub-block size in bits
  uint32_t sb_out[MAX_SUB];    // sub-block output start (block-relative)
  uint32_t sb_outn[MAX_SUB];   // sub-block output bytes
  uint32_t sb_seq[MAX_SUB + 1];  // sub-block first sequence; sb_seq[K] = n_seq
  uint32_t sb_seqn[MAX_SUB];   // sub-block sequence count
  uint16_t sorted_ll[N_LL + 1];
  uint16_t sorted_off[N_OFF + 2];
  uint8_t lens[N_LL + N_OFF + 3];
};

// Phase B: the output ring and the staging of the next group.
struct PhaseBSmem {
  uint8_t ring[RING];
  uint8_t far[2][32][FAR_STAGE];
  uint8_t lit[2][LIT_STAGE];
};

template <int LLB>
struct __align__(16) WarpSmem {
  union {
    PhaseASmem<LLB> a;
    PhaseBSmem b;
  } u;
  unsigned long long rstat[16];  // statistics: bytes copied in round r (0..7, 7 = later), groups reaching round r
};
static_assert(sizeof(PhaseASmem<11>) <= sizeof(PhaseBSmem), "the 11-bit phase A fits in the phase B space");

struct KParams {
  const gmp_file_desc* files;  // batch mode; nullptr in single-stream mode
  const uint64_t* item_start;  // batch mode: n_files + 1 prefix sums
  uint32_t n_files;
  gmp_file_desc single;  // single-stream mode
  int32_t* status;       // one per file
  unsigned long long* counter;
  uint8_t* scratch;
  uint64_t slot_bytes;
  uint64_t shadow_off;  // offset of the literal shadow inside a slot (256-byte aligned)
  uint32_t max_seq, max_out;
  unsigned long long* stats;  // [groups, rounds, de_fallback, blocks, max_rounds, cycles x3]
  int collect_stats;
  int resolve;  // 0: by the stream's DE flag, 1: MRR always, 2: sequential copying (SC)
  int spread;   // 1: first items fixed and interleaved over the CTAs; 0: all from the counter
  // Host-to-host pipeline (all null otherwise): a file's input is complete
  // once in_ready[file] reaches gen (written by the copy stream after the
  // copy); out_ready[file] is set to gen once all its blocks are decoded
  // (done[file] counts them), and by the last warp to exit (exited counts
  // the warps) for every file.
  const uint32_t* in_ready;
  uint32_t* abort_wait;  // set once a wait has run out: later waits give up at once
  unsigned long long wait_ns;
  uint32_t* out_ready;
  uint32_t* done;
  uint32_t* exited;
  uint32_t gen;
};

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Two 16-byte records as one 32-byte store (p 32-byte aligned).
__device__ __forceinline__ void st_global_32B(void* p, const uint4& a, const uint4& b) {
  asm volatile("st.global.v8.u32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"l"(p), "r"(a.x), "r"(a.y), "r"(a.z),
               "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w)
               : "memory");
}

__device__ __forceinline__ void set_status(int32_t* st, int code) { atomicCAS(st, 0, code); }

// ---- host-to-host pipeline flags
// The wait for a file's input is bounded: the host's limit (10 s unless the
// context sets another) of the global timer, and at most 2^24 polls; past
// that the file gets GMP_STATUS_INPUT_TIMEOUT, its blocks are skipped and
// every later wait of the launch gives up at once, so the launch always ends.
constexpr uint32_t kInputWaitPolls = 1u << 24;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t ld_acquire_sys(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(uint32_t* p, uint32_t v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Whole warp: true once *flag has reached gen (cyclic comparison, as the
// copy stream's flag values wrap), false if the wait ran out.  The warp polls
// and sleeps as one: with lane 0 polling and sleeping alone while the other
// lanes waited at a shuffle, the warps decoded their next blocks 2 to 2.7
// times slower (measured on text256m, (In) mode).
__device__ __noinline__ bool wait_input(const uint32_t* flag, uint32_t* abort_wait, uint32_t gen,
                                        unsigned long long wait_ns) {
  const unsigned long long t0 = global_ns();
  bool ok = false;
  for (uint32_t i = 0; i < kInputWaitPolls; i++) {
    // lane 0 reads the flag, the abort word and the clock; every decision
    // below is taken on its values, so the lanes leave the loop together
    uint32_t v = 0, stop = 0;
    if ((threadIdx.x & 31u) == 0) {
      v = ld_acquire_sys(flag);
      stop = *reinterpret_cast<volatile uint32_t*>(abort_wait) != 0u || global_ns() - t0 > wait_ns;
    }
    v = __shfl_sync(0xffffffffu, v, 0);
    stop = __shfl_sync(0xffffffffu, stop, 0);
    if ((int32_t)(v - gen) >= 0) {
      ok = true;
      break;
    }
    if (stop) break;
    __nanosleep(i < 64 ? 64 : 1024);
  }
  if (!ok && (threadIdx.x & 31u) == 0) atomicExch(abort_wait, 1u);
  __syncwarp();
  return ok;
}

// Whole warp, after a block of `file` (n_blocks blocks) is decoded: every
// lane's output stores are made visible before the block is counted, and
// the count that completes the file publishes its out_ready flag.
__device__ __noinline__ void block_done(uint32_t* done, uint32_t* out_ready, uint32_t gen, uint64_t n_blocks) {
  __threadfence();
  __syncwarp();
  if ((threadIdx.x & 31u) == 0) {
    const uint32_t d = atomicAdd(done, 1u) + 1u;
    if (d == (uint32_t)n_blocks) {
      __threadfence_system();
      st_release_sys(out_ready, gen);
    }
  }
  __syncwarp();
}

// Whole warp, on leaving the persistent loop: the last warp of the launch
// sets every file's out_ready flag, so that no copy stream waits on a flag
// that is never written.
__device__ __noinline__ void pipeline_exit(uint32_t* exited, uint32_t* out_ready, uint32_t gen, uint32_t n_files,
                                           uint32_t n_warps) {
  __threadfence();
  uint32_t last = 0;
  if ((threadIdx.x & 31u) == 0) last = atomicAdd(exited, 1u) + 1u == n_warps;
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last) {
    __threadfence_system();
    for (uint32_t f = threadIdx.x & 31u; f < n_files; f += 32) st_release_sys(out_ready + f, gen);
  }
}

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
// Lookup table of one canonical tree (Sec. 3.1, 3.2.1).  Entry for the
// TB-bit LSB-first peek e: the code whose bit-reversed value prefixes e,
// stored as (length << 9) | symbol; 0 = no code (an empty tree); LONG_CODE =
// the code is longer than TB bits (then decode_long below applies).  Leaves
// the tree's canonical arrays in C and its sorted symbols in `sorted` (run:
// scratch of 16 words).  Returns false
// when the code lengths do not form a complete prefix code (Kraft sum != 1)
// and are not all zero.
template <int TB>
__device__ bool build_lut(Canon& C, uint32_t* run, uint16_t* sorted, const uint8_t* lens, int n, uint16_t* lut) {
  const uint32_t lane = lane_id();
  if (lane < 16) { C.cnt[lane] = 0; run[lane] = 0; }
  __syncwarp();
  for (int base = 0; base < n; base += 32) {
    int s = base + (int)lane;
    uint32_t L = s < n ? lens[s] : 0u;
    uint32_t m = __match_any_sync(FULL, L);
    if ((__ffs(m) - 1) == (int)lane) C.cnt[L] += __popc(m);
    __syncwarp();
  }
  // Kraft sum and first codes
  bool ok = true;
  uint32_t used = 0;
  if (lane == 0) {
    uint32_t k = 0, code = 0, id = 0;
    for (int L = 1; L <= LUT_BITS; L++) {
      k += C.cnt[L] << (LUT_BITS - L);
      C.first[L] = code;
      C.idx[L] = id;
      id += C.cnt[L];
      code = (code + C.cnt[L]) << 1;
    }
    used = id;
    // lengths above 12 have no table slot: such a header is invalid
    const bool too_long = (C.cnt[13] | C.cnt[14] | C.cnt[15]) != 0;
    C.idx[0] = (!too_long && (used == 0 || k == (uint32_t)LUT_SIZE)) ? 1u : 0u;  // validity flag
    C.first[0] = used;
  }
  __syncwarp();
  ok = C.idx[0] != 0;
  used = C.first[0];
  if (!ok) return false;
  if (used == 0) {
    for (int e = (int)lane; e < (1 << TB); e += 32) lut[e] = 0;
    __syncwarp();
    return true;
  }
  // symbols sorted by (length, symbol)
  for (int base = 0; base < n; base += 32) {
    int s = base + (int)lane;
    uint32_t L = s < n ? lens[s] : 0u;
    uint32_t m = __match_any_sync(FULL, L);
    uint32_t r = __popc(m & ((1u << lane) - 1u));
    if (L) sorted[C.idx[L] + run[L] + r] = (uint16_t)s;
    __syncwarp();
    if (r == 0) run[L] += __popc(m);
    __syncwarp();
  }
  // limits of each length's code range, left-justified to TB bits
  uint32_t lim[TB + 1];
#pragma unroll
  for (int L = 1; L <= TB; L++) lim[L] = (C.first[L] + C.cnt[L]) << (TB - L);
  for (int e = (int)lane; e < (1 << TB); e += 32) {
    uint32_t v = __brev((uint32_t)e) >> (32 - TB);  // peek bits, most significant first
    uint32_t L = 1;
#pragma unroll
    for (int i = 1; i <= TB; i++) L += (v >= lim[i]) ? 1u : 0u;
    if (L > (uint32_t)TB) {
      lut[e] = LONG_CODE;
    } else {
      uint32_t sym = sorted[C.idx[L] + (v >> (TB - L)) - C.first[L]];
      lut[e] = (uint16_t)((L << 9) | sym);
    }
  }
  __syncwarp();
  return true;
}

// A code longer than the table's bits, by the canonical ranges: the 12-bit
// peek, most significant bit first, lies in length L's range [first_L,
// first_L + cnt_L) shifted left by 12 - L.  Returns (L << 9) | symbol.
template <int TB>
__device__ __forceinline__ uint32_t decode_long(const Canon& C, const uint16_t* sorted, uint32_t peek12) {
  const uint32_t v = __brev(peek12) >> (32 - LUT_BITS);
  for (int L = TB + 1; L <= LUT_BITS; L++) {
    const uint32_t code = v >> (LUT_BITS - L);
    if (code - C.first[L] < C.cnt[L]) return ((uint32_t)L << 9) | sorted[C.idx[L] + code - C.first[L]];
  }
  return 0;
}

// ---------------------------------------------------------------------------
// cp.async (16-byte, L2-only) global -> shared copies and their groups.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ void copy_match_global(uint8_t* out_blk, uint32_t rpos, uint32_t wpos, uint32_t ml) {
  for (uint32_t i = 0; i < ml; i++) out_blk[wpos + i] = out_blk[rpos + i];
}

// Resolution of one group's back-references (Sec. 3.2.2 step (c)); `copy`
// performs the calling lane's copy.  Strategies:
//  RES_ONE_PASS: every back-reference at once (Dependency Elimination, Fig. 7,
//    Sec. 4.2), for a group whose sources avoid the group's other copies;
//  RES_MRR: Multi-Round Resolution (Fig. 5, Sec. 4.1).  The figure names the
//    last writer with count_leading_zero_bits(ballot) and waits for read_pos +
//    length <= HWM; the first picks the highest pending lane rather than the
//    last completed one, and the second never admits an overlapping copy
//    (offset < length), whose source extends into its own output.  Reading
//    used here: the lowest pending lane f = ffs(ballot(pending)) - 1 has every
//    earlier lane complete and its own literals written, so HWM =
//    write_pos(f); a pending lane copies once min(read_pos + length,
//    write_pos) <= HWM.  Lane f always qualifies, so every round resolves at
//    least one lane and a group needs at most 32 rounds; a group whose
//    back-references do not depend on each other resolves in one round;
//  RES_SC: Sequential Copying, the baseline of Sec. 5.1: one back-reference
//    per round, in sequence order.
// Returns the number of rounds, or -1 if a round made no progress.  rstat
// (statistics only, else null): bytes copied in round r and groups reaching
// round r, rounds past 7 counted in bin 7.
enum { RES_ONE_PASS = 0, RES_MRR = 1, RES_SC = 2 };

// Statistics of one round: the warp's copied bytes (bytes_lane per lane).
__device__ __forceinline__ void note_round(unsigned long long* rstat, int round, uint32_t bytes_lane) {
  const uint32_t b = __reduce_add_sync(FULL, bytes_lane);
  if (lane_id() == 0 && b) {
    rstat[min(round, 7)] += b;
    rstat[8 + min(round, 7)] += 1;
  }
}

template <class Copy>
__device__ __forceinline__ int resolve_group(int how, bool pending, uint32_t rpos, uint32_t wpos, uint32_t ml,
                                             Copy&& copy, unsigned long long* rstat) {
  const uint32_t lane = lane_id();
  int rounds = 0;
  for (;;) {
    const uint32_t votes = __ballot_sync(FULL, pending);
    if (votes == 0) break;
    if (rounds == 32) return -1;
    const int f = __ffs(votes) - 1;
    bool go = pending;
    if (how == RES_SC) {
      go = (int)lane == f;
    } else if (how == RES_MRR) {
      const uint32_t hwm = __shfl_sync(FULL, wpos, f);
      go = pending && min(rpos + ml, wpos) <= hwm;
    }
    if (go) {
      copy();
      pending = false;
    }
    if (rstat) note_round(rstat, rounds, go ? ml : 0u);
    __syncwarp();
    rounds++;
  }
  return rounds;
}

// One lane's back-reference copy into the ring (Sec. 3.2.2, step (c)):
// ml bytes from rpos to wpos.  Bytes up to the next 4-byte boundary of the
// destination go one by one; then whole aligned destination words, each built
// from an unaligned source word (two aligned loads and a funnel shift); then
// the tail bytes.  The aligned words lie inside this lane's own output range,
// so no other lane writes them.  A source word is complete before it is read
// when the distance is at least 4 (earlier bytes of this copy included); a
// copy with distance 1..3 repeats its pattern byte by byte.
struct SrcView {
  const uint8_t* ring;
  const uint8_t* far;  // the lane's far staging (16-byte aligned)
  const uint8_t* out;  // block output in device memory
  uint32_t ring_lo, far_lo, far_hi;
  __device__ __forceinline__ uint8_t byte(uint32_t x) const {
    if (x >= ring_lo) return ring[x & RING_MASK];
    if (x >= far_lo && x < far_hi) return far[x - far_lo];
    return out[x];
  }
  __device__ __forceinline__ uint32_t word(uint32_t x) const {
    if (x >= ring_lo) {
      const uint32_t* r32 = reinterpret_cast<const uint32_t*>(ring);
      const uint32_t wa = x >> 2;
      return __funnelshift_r(r32[wa & RING_WMASK], r32[(wa + 1) & RING_WMASK], (x & 3u) * 8u);
    }
    if (x >= far_lo && x + 4 <= far_hi && x - far_lo + 8 <= (uint32_t)FAR_STAGE) {
      const uint32_t r = x - far_lo;
      const uint32_t* f32 = reinterpret_cast<const uint32_t*>(far);
      return __funnelshift_r(f32[r >> 2], f32[(r >> 2) + 1], (r & 3u) * 8u);
    }
    return (uint32_t)byte(x) | ((uint32_t)byte(x + 1) << 8) | ((uint32_t)byte(x + 2) << 16) |
           ((uint32_t)byte(x + 3) << 24);
  }
};

// The copy with every access wrapped by the ring mask (a source wholly in
// the ring, in_ring, or wholly in the lane's far staging).
__device__ __forceinline__ void copy_match_masked(uint8_t* ring, const SrcView& v, uint32_t rpos, uint32_t wpos,
                                                  uint32_t ml, bool in_ring) {
  // one linear view of the source: byte x at base[(x - off) & mask], word a
  // (bytes 4a .. 4a + 3 of the view) at base32[a & wmask]; the staging is
  // 16-byte aligned, so a source's offset within its word is x & 3 either way
  const uint8_t* base = in_ring ? v.ring : v.far;
  const uint32_t* base32 = reinterpret_cast<const uint32_t*>(base);
  const uint32_t off = in_ring ? 0u : v.far_lo;
  const uint32_t mask = in_ring ? RING_MASK : 0xffffffffu;
  const uint32_t wmask = in_ring ? RING_WMASK : 0xffffffffu;
  const uint32_t dist = wpos - rpos;
  if (dist < 4) {  // distance 1..3 (a ring source): the pattern repeats byte by byte
    for (uint32_t i = 0; i < ml; i++) ring[(wpos + i) & RING_MASK] = base[(rpos + i - off) & mask];
    return;
  }
  // head: the bytes up to the destination's next 4-byte boundary (at most 3),
  // loaded together, then stored; their sources precede them (distance >= 4).
  // Loads past a short source read bytes that are not used (the ring wraps,
  // the staging has room).
  const uint32_t h = min(ml, (4u - (wpos & 3u)) & 3u);
  {
    const uint8_t b0 = base[(rpos - off) & mask], b1 = base[(rpos + 1u - off) & mask];
    const uint8_t b2 = base[(rpos + 2u - off) & mask];
    if (h > 0) ring[wpos & RING_MASK] = b0;
    if (h > 1) ring[(wpos + 1u) & RING_MASK] = b1;
    if (h > 2) ring[(wpos + 2u) & RING_MASK] = b2;
  }
  uint32_t* r32 = reinterpret_cast<uint32_t*>(ring);
  const uint32_t nw = (ml - h) >> 2;  // whole aligned destination words
  const uint32_t x0 = rpos + h - off, d0 = (wpos + h) >> 2, sh = ((rpos + h) & 3u) * 8u;
  if (dist >= 16 || !in_ring) {
    // four words per step: a step's 16 source bytes lie before its
    // destination (or in the staging), so its five loads issue together and
    // a copy of up to 16 bytes takes one shared-memory latency
    for (uint32_t k = 0; k < nw; k += 4) {
      const uint32_t a = (x0 >> 2) + k, d = d0 + k;
      const uint32_t w0 = base32[a & wmask], w1 = base32[(a + 1u) & wmask], w2 = base32[(a + 2u) & wmask];
      const uint32_t w3 = base32[(a + 3u) & wmask], w4 = base32[(a + 4u) & wmask];
      r32[d & RING_WMASK] = __funnelshift_r(w0, w1, sh);
      if (k + 1u < nw) r32[(d + 1u) & RING_WMASK] = __funnelshift_r(w1, w2, sh);
      if (k + 2u < nw) r32[(d + 2u) & RING_WMASK] = __funnelshift_r(w2, w3, sh);
      if (k + 3u < nw) r32[(d + 3u) & RING_WMASK] = __funnelshift_r(w3, w4, sh);
    }
  } else {
    // distance 4..15 in the ring: a source word may hold bytes this copy has
    // just written, so one word at a time
    for (uint32_t k = 0; k < nw; k++) {
      const uint32_t a = (x0 >> 2) + k;
      r32[(d0 + k) & RING_WMASK] = __funnelshift_r(base32[a & wmask], base32[(a + 1u) & wmask], sh);
    }
  }
  // tail: fewer than 4 bytes, loaded together (their sources precede them)
  const uint32_t i = h + 4u * nw, t = ml - i;
  {
    const uint8_t b0 = base[(rpos + i - off) & mask], b1 = base[(rpos + i + 1u - off) & mask];
    const uint8_t b2 = base[(rpos + i + 2u - off) & mask];
    if (t > 0) ring[(wpos + i) & RING_MASK] = b0;
    if (t > 1) ring[(wpos + i + 1u) & RING_MASK] = b1;
    if (t > 2) ring[(wpos + i + 2u) & RING_MASK] = b2;
  }
}

__device__ __forceinline__ void copy_match_words(uint8_t* ring, const SrcView& v, uint32_t rpos, uint32_t wpos,
                                                 uint32_t ml) {
  const bool in_ring = rpos >= v.ring_lo;                                      // whole source in the ring
  const bool in_far = !in_ring && rpos >= v.far_lo && rpos + ml <= v.far_hi;   // whole source staged
  if (!(in_ring || in_far)) {
    for (uint32_t i = 0; i < ml; i++) ring[(wpos + i) & RING_MASK] = v.byte(rpos + i);
    return;
  }
  copy_match_masked(ring, v, rpos, wpos, ml, in_ring);
}

// Out of line, for copy_match_linear's rare cases (a source or destination
// that crosses the ring's end, or a ring source closer than 16 bytes).
__device__ __noinline__ void copy_match_general(uint8_t* ring, const SrcView v, uint32_t rpos, uint32_t wpos,
                                                uint32_t ml, bool in_ring) {
  copy_match_masked(ring, v, rpos, wpos, ml, in_ring);
}

// copy_match_words with the common case in linear addressing (used by the
// 128-register kernel instance, whose registers hold it without spilling).
__device__ __forceinline__ void copy_match_linear(uint8_t* ring, const SrcView& v, uint32_t rpos, uint32_t wpos,
                                                 uint32_t ml) {
  const bool in_ring = rpos >= v.ring_lo;                                      // whole source in the ring
  const bool in_far = !in_ring && rpos >= v.far_lo && rpos + ml <= v.far_hi;   // whole source staged
  if (!(in_ring || in_far)) {
    for (uint32_t i = 0; i < ml; i++) ring[(wpos + i) & RING_MASK] = v.byte(rpos + i);
    return;
  }
  // Linear case: the destination and (for a ring source) the source plus
  // the 16 bytes its word loads may read past it do not cross the ring's end,
  // and the distance is at least 16 (a far source is more than NEAR bytes
  // back), so that no source word holds bytes this copy writes in the same
  // step.  Every access is then one base register plus an immediate offset.
  {
    const uint32_t rs = rpos & RING_MASK, ws = wpos & RING_MASK;
    if ((in_far || (wpos - rpos >= 16u && rs + ml + 16u <= (uint32_t)RING)) && ws + ml <= (uint32_t)RING) {
      const uint8_t* src = in_ring ? ring + rs : v.far + (rpos - v.far_lo);
      uint8_t* dst = ring + ws;
      // head: up to the destination's next 4-byte boundary
      const uint32_t h = min(ml, (4u - (wpos & 3u)) & 3u);
      {
        const uint8_t b0 = src[0], b1 = src[1], b2 = src[2];
        if (h > 0) dst[0] = b0;
        if (h > 1) dst[1] = b1;
        if (h > 2) dst[2] = b2;
      }
      // whole destination words, four per step, from unaligned source words
      const uint32_t nw = (ml - h) >> 2;
      const uintptr_t sp = reinterpret_cast<uintptr_t>(src + h);
      const uint32_t* s32 = reinterpret_cast<const uint32_t*>(sp & ~static_cast<uintptr_t>(3));
      const uint32_t sh = static_cast<uint32_t>(sp & 3u) * 8u;
      uint32_t* d32 = reinterpret_cast<uint32_t*>(dst + h);
      for (uint32_t k = 0; k < nw; k += 4) {
        const uint32_t w0 = s32[k], w1 = s32[k + 1], w2 = s32[k + 2], w3 = s32[k + 3], w4 = s32[k + 4];
        d32[k] = __funnelshift_r(w0, w1, sh);
        if (k + 1 < nw) d32[k + 1] = __funnelshift_r(w1, w2, sh);
        if (k + 2 < nw) d32[k + 2] = __funnelshift_r(w2, w3, sh);
        if (k + 3 < nw) d32[k + 3] = __funnelshift_r(w3, w4, sh);
      }
      // tail: fewer than 4 bytes
      const uint32_t i = h + 4u * nw, t = ml - i;
      const uint8_t b0 = src[i], b1 = src[i + 1], b2 = src[i + 2];
      if (t > 0) dst[i] = b0;
      if (t > 1) dst[i + 1] = b1;
      if (t > 2) dst[i + 2] = b2;
      return;
    }
  }
  copy_match_general(ring, v, rpos, wpos, ml, in_ring);
}

// Out-of-line resolutions, kept out of the decode loop's code: Sequential
// Copying of a ring-resident group (ablation only), and every strategy for a
// group written straight to device memory (groups too large for the ring).
__device__ __noinline__ int resolve_sc_ring(uint8_t* ring, SrcView sv, uint32_t rpos, uint32_t wpos, uint32_t ml,
                                            bool pending, unsigned long long* rstat) {
  return resolve_group(RES_SC, pending, rpos, wpos, ml, [&] { copy_match_words(ring, sv, rpos, wpos, ml); }, rstat);
}
__device__ __noinline__ int resolve_global(int how, uint8_t* out_blk, uint32_t rpos, uint32_t wpos, uint32_t ml,
                                           bool pending, unsigned long long* rstat) {
  return resolve_group(how, pending, rpos, wpos, ml, [&] { copy_match_global(out_blk, rpos, wpos, ml); }, rstat);
}

// DE property check of one group (Sec. 4.2): each back-reference's source
// bytes before its own write position must avoid every other back-reference
// of the group.  Write positions rise with the lane, so the only candidate to
// test is the last lane whose write position lies below the source's end.
__device__ __forceinline__ bool de_group_ok(uint32_t rpos, uint32_t wpos, uint32_t ml) {
  const uint32_t lane = lane_id();
  uint32_t b = min(rpos + ml, wpos);
  int lo = -1;  // largest lane with wpos < b; the steps from -1 reach lane 31
#pragma unroll
  for (int step = 32; step >= 1; step >>= 1) {
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
template <bool STATS, int LLB>
__device__ void decode_block(WarpSmem<LLB>& S, const KParams& P, const gmp_file_desc& F, uint64_t b, int32_t* status,
                             uint8_t* slot, unsigned long long* st_acc) {
  const uint32_t lane = lane_id();
  const uint8_t* comp = F.comp;
  const long long t_begin = STATS ? clock64() : 0;
#ifdef GMP_PHASE_TIMERS
  unsigned long long tdet[6] = {0, 0, 0, 0, 0, 0};
#endif
  // ---- stream header (64 bytes), block reference
  int err = 0;
  uint32_t flags = 0, K = 0, window = 0, max_match = 0;
  bool byte_fmt = false;  // Gompresso/Byte block: records and raw literals, no Huffman phase
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
    byte_fmt = !(flags & 2u);
    if (magic != 0x31504d47u || (w1 & 0xffffu) != 1u || flags > 3u || window == 0 || window > 32768 ||
        (w5 & 0xffu) != 3u || max_match < 3 || max_match > 64)
      err = GMP_STATUS_BAD_HEADER;
    else if (byte_fmt ? (K != 0 || cwl != 0) : (K == 0 || K > MAX_SUB || cwl == 0 || cwl > 12))
      err = GMP_STATUS_BAD_HEADER;
  }
  const gmp_block_ref br = F.index[b];
  if (!err) {
    if ((br.comp_offset & 15) || br.comp_offset > F.comp_bytes || br.comp_bytes > F.comp_bytes - br.comp_offset ||
        br.out_offset > F.out_cap || br.out_bytes > F.out_cap - br.out_offset)
      err = GMP_STATUS_OUTPUT_OVERRUN;
    else if (br.comp_bytes < (byte_fmt ? 16ull : (192 + 12ull * K + 15) & ~15ull))  // through the bitstream start
      err = GMP_STATUS_BAD_HEADER;
  }
  if (err) {
    if (lane == 0) set_status(status, err);
    return;
  }
  const uint8_t* B = comp + br.comp_offset;
  const uint32_t n_seq = ld_u32_nc(B);
  const uint32_t out_bytes = ld_u32_nc(B + 4);
  // Byte blocks: literal count and the literal section's offset in the block
  uint32_t n_lit = 0;
  uint64_t lit_off = 0;
  if (out_bytes != br.out_bytes) {
    err = GMP_STATUS_BAD_HEADER;
  } else if (byte_fmt) {
    // the records and the padded literal section lie inside the block (whole
    // 16-byte chunks, which the literal staging reads)
    n_lit = ld_u32_nc(B + 8);
    lit_off = (16ull + 4ull * n_seq + 15ull) & ~15ull;
    if (lit_off + ((n_lit + 15ull) & ~15ull) > br.comp_bytes) err = GMP_STATUS_BAD_HEADER;
  } else if (out_bytes > P.max_out || n_seq > P.max_seq) {
    err = GMP_STATUS_CAPACITY;
  }
  if (err) {
    if (lane == 0) set_status(status, err);
    return;
  }
  // phase A output (Huffman blocks): records and the literal shadow in the
  // warp's scratch slot
  uint4* rec = reinterpret_cast<uint4*>(slot);
  uint8_t* shadow = slot + P.shadow_off;
  const uint8_t* lits = shadow;  // phase B's literal source
  long long t_tables, t_phase_a;
  if (byte_fmt) {
    // phase B reads the records from the stream and the literals from the
    // block's literal section
    lits = B + lit_off;
    t_tables = t_phase_a = STATS ? clock64() : 0;
    __syncwarp();
  } else {
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
          S.u.a.sb_bit[j] = carry_bit + ib - nb;
          S.u.a.sb_bits[j] = nb;
          S.u.a.sb_out[j] = carry_out + io - no;
          S.u.a.sb_outn[j] = no;
          S.u.a.sb_seq[j] = carry_seq + is - ns;
          S.u.a.sb_seqn[j] = ns;
        }
        // sizes are checked below against 64-bit totals, so a wrapped 32-bit
        // sum cannot pass: the totals are bounded by out_bytes / n_seq.
        carry_bit += __shfl_sync(FULL, ib, 31);
        carry_out += __shfl_sync(FULL, io, 31);
        carry_seq += __shfl_sync(FULL, is, 31);
      }
      if (lane == 0) S.u.a.sb_seq[K] = carry_seq;
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
      S.u.a.lens[i] = (sym & 1) ? (v >> 4) : (v & 15);
    }
    __syncwarp();
    PhaseASmem<LLB>& SA = S.u.a;
    const bool ok1 = build_lut<LLB>(SA.cll, SA.run, SA.sorted_ll, SA.lens, N_LL, SA.ll);
    const bool ok2 = build_lut<OFF_BITS>(SA.coff, SA.run, SA.sorted_off, SA.lens + N_LL, N_OFF, SA.off);
    if (!ok1 || !ok2) {
      if (lane == 0) set_status(status, GMP_STATUS_BAD_HEADER);
      return;
    }

    t_tables = STATS ? clock64() : 0;
    // ---- Phase A: lane per sub-block Huffman decode (Sec. 3.2.1)
    // Every lane of the warp takes one symbol per step (a literal, or a length
    // followed by its offset), with the literal / back-reference work done under
    // predicates and the lanes reconverged after each step, so the warp issues
    // one instruction stream for all 32 sub-blocks.
    const uint8_t* bs = B + bs_off;
    // 16-byte chunks of the block's bitstream; chunks past the block read as 0
    const uint64_t bs_chunks = (br.comp_bytes - bs_off) / 16;
    auto ld4 = [&](uint32_t c) -> uint4 {
      return (uint64_t)c < bs_chunks ? __ldg(reinterpret_cast<const uint4*>(bs) + c) : make_uint4(0, 0, 0, 0);
    };
    for (uint32_t jb = 0; jb < K; jb += 32) {
      const uint32_t j = jb + lane;
      bool act = j < K;
      uint32_t pos = 0, end = 0, outp = 0, out_end = 0, lit_dst = 0, nlit = 0, q = 0, q_end = 0;
      uint32_t lit_run = 0;
      // literal bytes of the lane, gathered eight at a time and stored as one
      // aligned 8-byte word (lit_dst is 16-byte aligned): 32 lanes storing
      // single bytes to 32 places cost a memory request each
      unsigned long long lacc = 0;
      uint32_t lit_end8 = 0;
      // records likewise go out two at a time (32 bytes, one sector) in the
      // 96-register instance: a record with an even index waits in `held` for
      // the next one (in the 128-register instance, whose launches hold fewer
      // warps, the pairing's extra instructions cost more than it saves)
      constexpr bool PAIR_RECORDS = LLB != LUT_BITS;
      uint4 held = make_uint4(0, 0, 0, 0);
      bool holding = false;
      // bit buffer (nb valid bits), a stash of up to 4 words (lo, hi) and the
      // next 16-byte chunk, loaded one chunk ahead of use
      uint64_t buf = 0, lo = 0, hi = 0;
      int nb = 0;
      uint32_t scnt = 0, ci = 0;
      uint4 pre = make_uint4(0, 0, 0, 0);
      // refill before a literal/length code, the common part without a
      // branch: the stash is reloaded first if it is empty (every fourth word)
      auto refill_ll = [&]() {
        if (scnt == 0) {
          lo = (uint64_t)pre.x | ((uint64_t)pre.y << 32);
          hi = (uint64_t)pre.z | ((uint64_t)pre.w << 32);
          scnt = 4;
          pre = ld4(ci++);
        }
        const bool need = nb <= 32;
        buf |= (uint64_t)(need ? (uint32_t)lo : 0u) << (nb & 63);
        nb += need ? 32 : 0;
        const uint64_t lo2 = (lo >> 32) | (hi << 32), hi2 = hi >> 32;
        lo = need ? lo2 : lo;
        hi = need ? hi2 : hi;
        scnt -= need ? 1u : 0u;
      };
      auto next_word = [&]() -> uint32_t {
        if (scnt == 0) {
          lo = (uint64_t)pre.x | ((uint64_t)pre.y << 32);
          hi = (uint64_t)pre.z | ((uint64_t)pre.w << 32);
          scnt = 4;
          pre = ld4(ci++);
        }
        const uint32_t w = (uint32_t)lo;
        lo = (lo >> 32) | (hi << 32);
        hi >>= 32;
        scnt--;
        return w;
      };
      if (act) {
        pos = S.u.a.sb_bit[j];
        end = pos + S.u.a.sb_bits[j];
        // the stash starts with chunk c0 minus the words before the start word
        const uint32_t w0 = pos >> 5, c0 = w0 >> 2;
        const uint4 c = ld4(c0);
        lo = (uint64_t)c.x | ((uint64_t)c.y << 32);
        hi = (uint64_t)c.z | ((uint64_t)c.w << 32);
        for (uint32_t k = 0; k < (w0 & 3u); k++) {
          lo = (lo >> 32) | (hi << 32);
          hi >>= 32;
        }
        scnt = 4u - (w0 & 3u);
        pre = ld4(c0 + 1);
        ci = c0 + 2;
        buf = (uint64_t)(next_word() >> (pos & 31u));
        nb = 32 - (int)(pos & 31u);
        buf |= (uint64_t)next_word() << nb;
        nb += 32;
        outp = S.u.a.sb_out[j];
        out_end = outp + S.u.a.sb_outn[j];
        lit_dst = ((S.u.a.sb_out[j] + 15u) & ~15u) + 16u * j;
        // end of the lane's literal region, rounded up to the 8-byte words it
        // is stored in (the next lane's region starts at or after it)
        lit_end8 = lit_dst + ((S.u.a.sb_outn[j] + 7u) & ~7u);
        q = S.u.a.sb_seq[j];
        q_end = q + S.u.a.sb_seqn[j];
        act = q < q_end;
      }
      // The bit buffer is refilled to more than 32 bits before each
      // literal/length code, so that a code (<= 12 bits) and, after it, an
      // offset code with its extra bits (<= 12 + 13) rarely need a second
      // refill: fewer divergent branches per step.
      while (__any_sync(FULL, act)) {
  #ifdef GMP_PHASE_TIMERS
        tdet[5]++;
  #endif
        // two symbols per lane per warp step (the second only if the lane is
        // still active), halving the votes and reconvergence points
        if (act) {
          refill_ll();
          uint32_t e = S.u.a.ll[buf & ((1u << LLB) - 1u)];
          if (LLB < LUT_BITS && e == LONG_CODE)
            e = decode_long<LLB>(S.u.a.cll, S.u.a.sorted_ll, (uint32_t)buf & (LUT_SIZE - 1));
          const uint32_t L = e >> 9, sym = e & 511u;
          buf >>= L;
          nb -= (int)L;
          pos += L;
          if (sym < 256) {
            lacc |= (unsigned long long)sym << (8u * (nlit & 7u));
            if ((nlit & 7u) == 7u) {
              const uint32_t c = lit_dst + (nlit & ~7u);
              // past the region only on a corrupt stream (caught below)
              if (c + 8u <= lit_end8) *reinterpret_cast<unsigned long long*>(shadow + c) = lacc;
              lacc = 0;
            }
            nlit++;
            lit_run++;
            outp++;
          } else {
            uint32_t ml = 0, dist = 0;
            if (sym > 256) {
              ml = sym - 254u;
              if (nb < 25) {
                buf |= (uint64_t)next_word() << nb;
                nb += 32;
              }
              uint32_t e2 = S.u.a.off[buf & (OFF_SIZE - 1)];
              if (e2 == LONG_CODE)
                e2 = decode_long<OFF_BITS>(S.u.a.coff, S.u.a.sorted_off, (uint32_t)buf & (LUT_SIZE - 1));
              const uint32_t L2 = e2 >> 9, os = e2 & 31u;
              const uint32_t ne = os < 4 ? 0u : (os >> 1) - 1u;
              const uint32_t extra = (uint32_t)(buf >> L2) & ((1u << ne) - 1u);
              buf >>= L2 + ne;
              nb -= (int)(L2 + ne);
              pos += L2 + ne;
              dist = os < 4 ? os + 1u : ((2u | (os & 1u)) << ne) + extra + 1u;
              if (L2 == 0 || os >= (uint32_t)N_OFF || ml > max_match) err = GMP_STATUS_CORRUPT_SYMBOL;
              else if (dist > window || dist > outp) err = GMP_STATUS_BAD_OFFSET;
              else if (ml > out_end - min(outp, out_end)) err = GMP_STATUS_OUTPUT_OVERRUN;
            } else if (q + 1 != n_seq) {
              err = GMP_STATUS_CORRUPT_SYMBOL;  // the end symbol only closes the block's last sequence
            }
            // the record carries the sequence's output position and literal
            // source, so that the LZ77 phase needs no prefix sums for it
            {
              const uint4 r = make_uint4(outp - lit_run, lit_dst + nlit - lit_run, lit_run, (dist << 8) | ml);
              if (!PAIR_RECORDS) {
                rec[q] = r;
              } else if (q & 1u) {
                if (holding) st_global_32B(rec + (q - 1), held, r);
                else rec[q] = r;
                holding = false;
              } else {
                held = r;
                holding = true;
              }
            }
            q++;
            lit_run = 0;
            outp += ml;
          }
          // a lane that runs past its sub-block stops here (this bounds the
          // loop on corrupt input); sizes are checked when the sub-block ends
          if (L == 0) err = GMP_STATUS_CORRUPT_SYMBOL;
          else if (pos > end) err = GMP_STATUS_BITSTREAM;
          act = !err && q < q_end;
        }
        if (act) {  // second symbol of the step
          refill_ll();
          uint32_t e = S.u.a.ll[buf & ((1u << LLB) - 1u)];
          if (LLB < LUT_BITS && e == LONG_CODE)
            e = decode_long<LLB>(S.u.a.cll, S.u.a.sorted_ll, (uint32_t)buf & (LUT_SIZE - 1));
          const uint32_t L = e >> 9, sym = e & 511u;
          buf >>= L;
          nb -= (int)L;
          pos += L;
          if (sym < 256) {
            lacc |= (unsigned long long)sym << (8u * (nlit & 7u));
            if ((nlit & 7u) == 7u) {
              const uint32_t c = lit_dst + (nlit & ~7u);
              // past the region only on a corrupt stream (caught below)
              if (c + 8u <= lit_end8) *reinterpret_cast<unsigned long long*>(shadow + c) = lacc;
              lacc = 0;
            }
            nlit++;
            lit_run++;
            outp++;
          } else {
            uint32_t ml = 0, dist = 0;
            if (sym > 256) {
              ml = sym - 254u;
              if (nb < 25) {
                buf |= (uint64_t)next_word() << nb;
                nb += 32;
              }
              uint32_t e2 = S.u.a.off[buf & (OFF_SIZE - 1)];
              if (e2 == LONG_CODE)
                e2 = decode_long<OFF_BITS>(S.u.a.coff, S.u.a.sorted_off, (uint32_t)buf & (LUT_SIZE - 1));
              const uint32_t L2 = e2 >> 9, os = e2 & 31u;
              const uint32_t ne = os < 4 ? 0u : (os >> 1) - 1u;
              const uint32_t extra = (uint32_t)(buf >> L2) & ((1u << ne) - 1u);
              buf >>= L2 + ne;
              nb -= (int)(L2 + ne);
              pos += L2 + ne;
              dist = os < 4 ? os + 1u : ((2u | (os & 1u)) << ne) + extra + 1u;
              if (L2 == 0 || os >= (uint32_t)N_OFF || ml > max_match) err = GMP_STATUS_CORRUPT_SYMBOL;
              else if (dist > window || dist > outp) err = GMP_STATUS_BAD_OFFSET;
              else if (ml > out_end - min(outp, out_end)) err = GMP_STATUS_OUTPUT_OVERRUN;
            } else if (q + 1 != n_seq) {
              err = GMP_STATUS_CORRUPT_SYMBOL;  // the end symbol only closes the block's last sequence
            }
            // the record carries the sequence's output position and literal
            // source, so that the LZ77 phase needs no prefix sums for it
            {
              const uint4 r = make_uint4(outp - lit_run, lit_dst + nlit - lit_run, lit_run, (dist << 8) | ml);
              if (!PAIR_RECORDS) {
                rec[q] = r;
              } else if (q & 1u) {
                if (holding) st_global_32B(rec + (q - 1), held, r);
                else rec[q] = r;
                holding = false;
              } else {
                held = r;
                holding = true;
              }
            }
            q++;
            lit_run = 0;
            outp += ml;
          }
          // a lane that runs past its sub-block stops here (this bounds the
          // loop on corrupt input); sizes are checked when the sub-block ends
          if (L == 0) err = GMP_STATUS_CORRUPT_SYMBOL;
          else if (pos > end) err = GMP_STATUS_BITSTREAM;
          act = !err && q < q_end;
        }
        __syncwarp();
      }
      if (j < K) {
        if (holding) rec[q - 1] = held;  // the lane's last record, alone
        // the last, partial word of literals
        if (nlit & 7u) {
          const uint32_t c = lit_dst + (nlit & ~7u);
          if (c + 8u <= lit_end8) *reinterpret_cast<unsigned long long*>(shadow + c) = lacc;
        }
        if (!err && pos != end) err = GMP_STATUS_BITSTREAM;
        if (!err && outp != out_end) err = GMP_STATUS_OUTPUT_OVERRUN;
      }
    }
    if (err) set_status(status, err);
    if (__ballot_sync(FULL, err != 0)) return;
    __syncwarp();  // phase A's records and literals are visible to the whole warp
    t_phase_a = STATS ? clock64() : 0;
  }  // Huffman blocks

  // ---- Phase B: 32 sequences per step (Sec. 3.2.2)
  // Group g+1 is prepared while group g runs: its two prefix sums are taken
  // and its literal runs and far back-reference sources are copied into the
  // stage (g+1)&1 by cp.async, so that group g's work reads shared memory only.
  uint8_t* out_blk = F.out + br.out_offset;
  const bool vec_ok = (((uintptr_t)out_blk) & 15u) == 0;
  const bool de = (flags & 1u) != 0;
  PhaseBSmem& SB = S.u.b;
  uint8_t* ring = SB.ring;
  uint32_t G0 = 0, litpos = 0, flushed = 0, ring_valid_lo = 0;
  unsigned long long n_groups = 0, n_rounds = 0, n_fallback = 0, max_rounds = 0;
  unsigned long long* rstat = STATS ? S.rstat : nullptr;
  const uint32_t n_groups_total = (n_seq + 31) / 32;

  // A group's per-lane values, packed to keep the two live copies (the group
  // being resolved and the one being staged) small: w = (distance << 8) |
  // match length as in the records; far = staged window start (16-byte
  // aligned) | its 16-byte chunk count; lit = literal staging start (16-byte
  // aligned) | staged flag (bit 0) | (Byte blocks) a failed check's status
  // << 1.  Write position = dst + ll, source = write position - distance.
  struct Prep {
    uint32_t ll, w, dst, lsrc, gtot, glits, far, lit;
  };
  // sequence t: Huffman blocks {output position, literal source, literal
  // length, (distance << 8) | match length} from phase A; Byte blocks
  // {0, 0, literal length, (distance << 8) | match length} from the stream;
  // zero past the end
  auto load_rec = [&](uint32_t t) -> uint4 {
    if (t >= n_seq) return make_uint4(0, 0, 0, 0);
    if (!byte_fmt) return rec[t];
    // match code 63 has no length; it decodes as 65 > max_match and is caught in prep
    const uint32_t r = ld_u32_nc(B + 16 + 4ull * t), m = (r >> 10) & 63u;
    return make_uint4(0, 0, r & 1023u, m ? ((((r >> 16) + 1u) << 8) | (m + 2u)) : 0u);
  };
  // positions and staging of group h; G0h / litposh: where its output and
  // (Byte blocks) its literals start
  auto prep = [&](uint32_t h, uint4 r, uint32_t G0h, uint32_t litposh, bool allow, int stage) {
    Prep q;
    const uint32_t t = h * 32 + lane;
    const bool valid = t < n_seq;
    q.ll = r.z;
    q.w = r.w;
    const uint32_t ml = r.w & 0xffu;
    const uint32_t dist = r.w >> 8;
    // the group's literal run in the literal source, [lit_a, lit_b), and
    // whether the group's literals lie in it back to back
    uint32_t lit_a, lit_b;
    bool lit_run;
    if (!byte_fmt) {
      q.gtot = __reduce_max_sync(FULL, valid ? r.x + q.ll + ml : G0h) - G0h;
      // lanes past the block's last sequence sit at the group's end, so that
      // write positions never fall with the lane
      q.dst = valid ? r.x : G0h + q.gtot;
      q.lsrc = r.y;
      q.glits = __reduce_add_sync(FULL, q.ll);
      lit_a = __reduce_min_sync(FULL, q.ll ? q.lsrc : 0xffffffffu);
      lit_b = __reduce_max_sync(FULL, q.ll ? q.lsrc + q.ll : 0u);
      lit_run = lit_b - lit_a == q.glits;  // one sub-block's literals
    } else {
      // one reduction and one scan of (literal length << 16 | total length):
      // a record's lengths are below 2^11, a group's sums below 2^16
      const uint32_t packed = (q.ll << 16) | (q.ll + ml);
      const uint32_t sum = __reduce_add_sync(FULL, packed);
      const uint32_t inc = warp_incl_scan(packed) - packed;
      q.gtot = sum & 0xffffu;
      q.glits = sum >> 16;
      q.dst = G0h + (inc & 0xffffu);
      q.lsrc = litposh + (inc >> 16);
      lit_a = litposh;
      lit_b = litposh + q.glits;
      lit_run = true;
    }
    const uint32_t wpos = q.dst + q.ll, rpos = wpos - dist;
    q.far = 0;
    q.lit = 0;
    int err = 0;
    if (byte_fmt) {
      // phase A checks Huffman records as it decodes them; Byte records are
      // checked here, before anything is staged or copied for the group
      if (__any_sync(FULL, ml > max_match)) err = GMP_STATUS_CORRUPT_SYMBOL;
      else if (__any_sync(FULL, ml > 0 && (dist > window || dist > wpos))) err = GMP_STATUS_BAD_OFFSET;
      else if ((uint64_t)G0h + q.gtot > out_bytes || (uint64_t)litposh + q.glits > n_lit)
        err = GMP_STATUS_OUTPUT_OVERRUN;
      if (err) allow = false;
    }
    if (allow && vec_ok && q.gtot <= GROUP_FAST_MAX) {
      // far part of the source: below the ring's reach, already in device memory
      const uint32_t rlo = max(ring_valid_lo, G0h > NEAR ? G0h - NEAR : 0u);
      if (ml > 0 && rpos < rlo) {
        const uint32_t fe = min(rpos + ml, rlo);
        const uint32_t a0 = rpos & ~15u;
        const uint32_t a1 = min((fe + 15u) & ~15u, flushed & ~15u);
        uint8_t* dstage = SB.far[stage][lane];
#pragma unroll
        for (uint32_t c = 0; c < (uint32_t)FAR_STAGE / 16u; c++)
          if (a0 + 16u * c < a1) cp_async16(dstage + 16u * c, out_blk + a0 + 16u * c);
        q.far = a0 | (a1 > a0 ? (a1 - a0) >> 4 : 0u);
      }
    }
    // the group's literals, one contiguous run of the literal source when
    // they all belong to one sub-block: lane i stages the run's i-th 16-byte
    // chunk
    if (allow && q.glits > 0 && q.gtot <= GROUP_FAST_MAX) {
      const uint32_t l0 = lit_a & ~15u, l1 = (lit_b + 15u) & ~15u;
      if (lit_run && l1 - l0 <= (uint32_t)LIT_STAGE) {
        const uint32_t c = l0 + 16u * lane;
        if (c < l1) cp_async16(SB.lit[stage] + (c - l0), lits + c);
        q.lit = l0 | 1u;
      }
    }
    q.lit |= (uint32_t)err << 1;
    cp_async_commit();
    return q;
  };

  uint4 r_next = load_rec(lane);
  Prep cur = prep(0, r_next, 0, 0, true, 0);
  r_next = load_rec(32 + lane);
  for (uint32_t g = 0; g < n_groups_total; g++) {
    if (cur.lit & 14u) {
      cp_async_wait_all();
      if (lane == 0) set_status(status, (int)((cur.lit >> 1) & 7u));
      return;
    }
    const int stage = (int)(g & 1u);
    const bool fast = cur.gtot <= GROUP_FAST_MAX;
    // prepare group g+1 (staging only if this group leaves the ring's reach unchanged)
    GMP_TSTAMP(tg0);
    Prep nxt = prep(g + 1, r_next, G0 + cur.gtot, litpos + cur.glits, fast, stage ^ 1);
    GMP_TSTAMP(tg1);
    GMP_TADD(0, tg0, tg1);
    r_next = load_rec((g + 2) * 32 + lane);
    cp_async_wait_1();  // this group's staging has landed
    __syncwarp();
    GMP_TSTAMP(tg2);
    GMP_TADD(1, tg1, tg2);
    const uint32_t ll = cur.ll, ml = cur.w & 0xffu, dst = cur.dst, lsrc = cur.lsrc, wpos = dst + ll,
                   rpos = wpos - (cur.w >> 8);
    const bool pending = ml > 0;  // lanes past the block's end have no match
    const bool lit_staged = cur.lit & 1u;
    const uint32_t lit_lo = cur.lit & ~15u, far_lo = cur.far & ~15u, far_hi = far_lo + 16u * (cur.far & 15u);
    const uint32_t G1 = G0 + cur.gtot;
    int rounds;
    if (fast) {
      const uint32_t ring_lo = max(ring_valid_lo, G0 > NEAR ? G0 - NEAR : 0u);
      // literal strings, four bytes per step loaded together (the staging
      // has room for the reads past a string's end; other sources are read
      // only up to it)
      if (cur.glits) {
        if (lit_staged && (dst & RING_MASK) + ll <= (uint32_t)RING) {
          // the literal string does not cross the ring's end: base + offset
          const uint8_t* ls = SB.lit[stage] + (lsrc - lit_lo);
          uint8_t* rd = ring + (dst & RING_MASK);
          for (uint32_t i = 0; i < ll; i += 4) {
            const uint8_t b0 = ls[i], b1 = ls[i + 1], b2 = ls[i + 2], b3 = ls[i + 3];
            rd[i] = b0;
            if (i + 1 < ll) rd[i + 1] = b1;
            if (i + 2 < ll) rd[i + 2] = b2;
            if (i + 3 < ll) rd[i + 3] = b3;
          }
        } else if (lit_staged) {
          const uint8_t* ls = SB.lit[stage] + (lsrc - lit_lo);
          for (uint32_t i = 0; i < ll; i += 4) {
            const uint8_t b0 = ls[i], b1 = ls[i + 1], b2 = ls[i + 2], b3 = ls[i + 3];
            ring[(dst + i) & RING_MASK] = b0;
            if (i + 1 < ll) ring[(dst + i + 1) & RING_MASK] = b1;
            if (i + 2 < ll) ring[(dst + i + 2) & RING_MASK] = b2;
            if (i + 3 < ll) ring[(dst + i + 3) & RING_MASK] = b3;
          }
        } else {
          for (uint32_t i = 0; i < ll; i++) ring[(dst + i) & RING_MASK] = lits[lsrc + i];
        }
      }
      __syncwarp();
      GMP_TSTAMP(tg3);
      GMP_TADD(2, tg2, tg3);
      const SrcView sv{ring, SB.far[stage][lane], out_blk, ring_lo, far_lo, far_hi};
      // DE: every source below the group start passes at once; otherwise the
      // exact per-group check decides (de_group_ok); a group that fails it is
      // resolved by MRR
      const bool de_ok = de && P.resolve == 0 &&
                         (__all_sync(FULL, !pending || rpos + ml <= G0) || de_group_ok(rpos, wpos, ml));
      if (de_ok) {
        if (pending) {
          if (LLB == LUT_BITS) copy_match_linear(ring, sv, rpos, wpos, ml);
          else copy_match_words(ring, sv, rpos, wpos, ml);
        }
        __syncwarp();
        rounds = __ballot_sync(FULL, pending) ? 1 : 0;
        if (rstat) note_round(rstat, 0, pending ? ml : 0u);
      } else if (P.resolve != 2) {
        if (de && P.resolve == 0) n_fallback++;
        // Multi-Round Resolution (reading at resolve_group): HWM = write
        // position of the lowest pending lane
        bool pend = pending;
        rounds = 0;
        for (;;) {
          const uint32_t votes = __ballot_sync(FULL, pend);
          if (votes == 0) break;
          if (rounds == 32) {
            rounds = -1;
            break;
          }
          const uint32_t hwm = __shfl_sync(FULL, wpos, __ffs(votes) - 1);
          const bool go = pend && min(rpos + ml, wpos) <= hwm;
          if (go) {
            if (LLB == LUT_BITS) copy_match_linear(ring, sv, rpos, wpos, ml);
            else copy_match_words(ring, sv, rpos, wpos, ml);
            pend = false;
          }
          if (rstat) note_round(rstat, rounds, go ? ml : 0u);
          __syncwarp();
          rounds++;
        }
      } else {
        rounds = resolve_sc_ring(ring, sv, rpos, wpos, ml, pending, rstat);
      }
      GMP_TSTAMP(tg4);
      GMP_TADD(3, tg3, tg4);
      // flush completed 16-byte chunks; after a large group `flushed` may be
      // unaligned, so its first partial chunk goes out byte by byte
      const uint32_t fend = G1 & ~15u;
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
      GMP_TSTAMP(tg5);
      GMP_TADD(4, tg4, tg5);
    } else {
      // a group too large for the ring: write it straight to device memory
      for (uint32_t c = flushed + lane; c < G0; c += 32u) out_blk[c] = ring[c & RING_MASK];
      __syncwarp();
      for (uint32_t i = 0; i < ll; i++) out_blk[dst + i] = lits[lsrc + i];
      __syncwarp();
      int how = P.resolve == 2 ? RES_SC : RES_MRR;
      if (de && P.resolve == 0) {
        if (de_group_ok(rpos, wpos, ml)) how = RES_ONE_PASS;
        else n_fallback++;
      }
      rounds = resolve_global(how, out_blk, rpos, wpos, ml, pending, rstat);
      flushed = G1;
      ring_valid_lo = G1;
    }
    if (rounds < 0) {
      cp_async_wait_all();
      if (lane == 0) set_status(status, GMP_STATUS_MRR_NO_PROGRESS);
      return;
    }
    __syncwarp();
    if (rounds > 0) n_groups++;
    n_rounds += (unsigned)rounds;
    if ((unsigned long long)rounds > max_rounds) max_rounds = (unsigned)rounds;
    G0 = G1;
    litpos += cur.glits;
    cur = nxt;
  }
  cp_async_wait_all();
  __syncwarp();
  // tail bytes not yet flushed
  for (uint32_t c = flushed + lane; c < out_bytes; c += 32u) out_blk[c] = ring[c & RING_MASK];
  if ((G0 != out_bytes || (byte_fmt && litpos != n_lit)) && lane == 0) set_status(status, GMP_STATUS_OUTPUT_OVERRUN);
  __syncwarp();
  const long long t_end = STATS ? clock64() : 0;
  st_acc[0] += n_groups;
  st_acc[1] += n_rounds;
  st_acc[2] += n_fallback;
  st_acc[3] += 1;
  if (max_rounds > st_acc[4]) st_acc[4] = max_rounds;
  st_acc[5] += (unsigned long long)(t_tables - t_begin);
  st_acc[6] += (unsigned long long)(t_phase_a - t_tables);
  st_acc[7] += (unsigned long long)(t_end - t_phase_a);
#ifdef GMP_PHASE_TIMERS
  for (int i = 0; i < 6; i++) st_acc[8 + i] += tdet[i];
#endif
}

// Persistent kernel: warps take work items until none are left.
// STATS: the statistics build (per-block counters, clocks and round
// histograms); the other instance carries none of that code.
// DEEP: at most 4 warps per CTA and 96 registers per thread, so that 20
// warps fit per SM (more blocks in flight for inputs of many waves); the
// other instance keeps 128 registers (16 warps per SM), which makes a single
// block's decode faster when every block is in flight at once.
// PIPE: the host-to-host pipeline's flag waits and counts (the statistics
// instances always carry them); the instances without it are the ones the
// device-resident calls launch, whose code the flags would otherwise change
// (0.8 % slower on csv1g in the 96-register instance).
template <bool STATS, bool DEEP, bool PIPE>
__global__ void __launch_bounds__(DEEP ? 128 : 512, DEEP ? 5 : 1) decode_kernel(const KParams P) {
  constexpr bool kPipe = PIPE || STATS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t lane = lane_id();
  constexpr int LLB = DEEP ? 11 : 12;
  WarpSmem<LLB>& S = reinterpret_cast<WarpSmem<LLB>*>(smem_raw)[warp];
  const uint64_t gw = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  uint8_t* slot = P.scratch + gw * P.slot_bytes;
  uint64_t total;
  if (P.files) total = P.item_start[P.n_files];
  else total = P.single.n_blocks;
  unsigned long long st_acc[14] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (lane < 16) S.rstat[lane] = 0;
  __syncwarp();
  // With `spread`, a warp's first item is fixed and interleaved over the
  // CTAs (warp w of CTA c takes w * CTAs + c), so that a launch with fewer
  // items than warps spreads them evenly over the SMs; later items come from
  // the work counter, numbered after the fixed ones.  Without it (launches
  // that share the GPU, whose CTAs may not all be resident at once) every
  // item comes from the counter, in the order the warps arrive.
  const unsigned long long fixed = P.spread ? (unsigned long long)gridDim.x * (blockDim.x >> 5) : 0ull;
  unsigned long long item = 0;
  if (P.spread) {
    item = (unsigned long long)warp * gridDim.x + blockIdx.x;
  } else {
    if (lane == 0) item = atomicAdd(P.counter, 1ull);
    item = __shfl_sync(FULL, item, 0);
  }
  while (item < total) {
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
    if (!kPipe || !P.in_ready || wait_input(P.in_ready + file, P.abort_wait, P.gen, P.wait_ns)) {
      decode_block<STATS, LLB>(S, P, F, b, P.status + file, slot, st_acc);
    } else if (lane == 0) {
      set_status(P.status + file, GMP_STATUS_INPUT_TIMEOUT);
    }
    __syncwarp();
    if (kPipe && P.out_ready) block_done(P.done + file, P.out_ready + file, P.gen, F.n_blocks);
    unsigned long long next = 0;
    if (lane == 0) next = fixed + atomicAdd(P.counter, 1ull);
    item = __shfl_sync(FULL, next, 0);
  }
  if (kPipe && P.out_ready) pipeline_exit(P.exited, P.out_ready, P.gen, P.files ? P.n_files : 1u, gridDim.x * (blockDim.x >> 5));
  if (STATS && lane == 0 && st_acc[3]) {
    atomicAdd(&P.stats[0], st_acc[0]);
    atomicAdd(&P.stats[1], st_acc[1]);
    atomicAdd(&P.stats[2], st_acc[2]);
    atomicAdd(&P.stats[3], st_acc[3]);
    atomicMax(&P.stats[4], st_acc[4]);
    atomicAdd(&P.stats[5], st_acc[5]);
    atomicAdd(&P.stats[6], st_acc[6]);
    atomicAdd(&P.stats[7], st_acc[7]);
#ifdef GMP_PHASE_TIMERS
    for (int i = 8; i < 14; i++) atomicAdd(&P.stats[i], st_acc[i]);
#endif
  }
  if (STATS && st_acc[3]) {
    __syncwarp();
    if (lane < 16 && S.rstat[lane]) atomicAdd(&P.stats[16 + lane], S.rstat[lane]);
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

size_t warp_smem_bytes(bool deep) { return deep ? sizeof(WarpSmem<11>) : sizeof(WarpSmem<12>); }

// The dynamic shared memory limit of each kernel instance is set to the
// largest size any launch shape of that instance uses (16 warps per CTA of
// the 128-register kernel, 4 of the 96-register one), not to the size of the
// launch at hand: the attribute is per kernel and process-wide, so a smaller
// value set by one host thread could otherwise fail another thread's wider
// launch.  smem_bytes is only checked against that limit.
cudaError_t configure_kernel(bool deep, size_t smem_bytes) {
  const size_t lim = deep ? 4 * sizeof(WarpSmem<11>) : (size_t)kWideWarpsPerSm * sizeof(WarpSmem<12>);
  if (smem_bytes > lim) return cudaErrorInvalidValue;
  const int b = (int)lim;
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e;
  if (deep) {
    e = cudaFuncSetAttribute(decode_kernel<false, true, false>, a, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(decode_kernel<false, true, true>, a, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(decode_kernel<true, true, true>, a, b);
  } else {
    e = cudaFuncSetAttribute(decode_kernel<false, false, false>, a, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(decode_kernel<false, false, true>, a, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(decode_kernel<true, false, true>, a, b);
  }
  return e;
}

cudaError_t occupancy(int warps_per_cta, size_t smem_bytes, bool deep, int* ctas_per_sm) {
  if (deep)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, decode_kernel<false, true, false>, warps_per_cta * 32,
                                                         smem_bytes);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, decode_kernel<false, false, false>, warps_per_cta * 32,
                                                       smem_bytes);
}

cudaError_t launch_decode(const LaunchShape& shape, const gmp_file_desc* files, const uint64_t* item_start,
                          uint32_t n_files, const gmp_file_desc* single, int32_t* status,
                          unsigned long long* counter, uint8_t* scratch, uint64_t slot_bytes, uint64_t shadow_off,
                          uint32_t max_seq, uint32_t max_out, unsigned long long* stats, int collect_stats,
                          int resolve, cudaStream_t stream, int spread, const PipeFlags* pipe) {
  KParams P;
  P.spread = spread;
  P.in_ready = pipe ? pipe->in_ready : nullptr;
  P.abort_wait = pipe ? pipe->abort_wait : nullptr;
  P.wait_ns = pipe ? pipe->wait_ns : 0ull;
  P.out_ready = pipe ? pipe->out_ready : nullptr;
  P.done = pipe ? pipe->done : nullptr;
  P.exited = pipe ? pipe->exited : nullptr;
  P.gen = pipe ? pipe->gen : 0u;
  // in_ready needs the abort word, out_ready its counters
  if ((P.in_ready && !P.abort_wait) || (P.out_ready && (!P.done || !P.exited))) return cudaErrorInvalidValue;
  P.files = files;
  P.item_start = item_start;
  P.n_files = n_files;
  if (single) P.single = *single;
  else memset(&P.single, 0, sizeof(P.single));
  P.status = status;
  P.counter = counter;
  P.scratch = scratch;
  P.slot_bytes = slot_bytes;
  P.shadow_off = shadow_off;
  P.max_seq = max_seq;
  P.max_out = max_out;
  P.stats = stats;
  P.collect_stats = collect_stats;
  P.resolve = resolve;
  const bool deep = shape.deep && shape.warps_per_cta <= 4;
  cudaError_t e = configure_kernel(deep, shape.smem_bytes);
  if (e != cudaSuccess) return e;
  const dim3 grid(shape.grid), block(shape.warps_per_cta * 32);
  if (collect_stats) {
    if (deep) decode_kernel<true, true, true><<<grid, block, shape.smem_bytes, stream>>>(P);
    else decode_kernel<true, false, true><<<grid, block, shape.smem_bytes, stream>>>(P);
  } else if (pipe) {
    if (deep) decode_kernel<false, true, true><<<grid, block, shape.smem_bytes, stream>>>(P);
    else decode_kernel<false, false, true><<<grid, block, shape.smem_bytes, stream>>>(P);
  } else {
    if (deep) decode_kernel<false, true, false><<<grid, block, shape.smem_bytes, stream>>>(P);
    else decode_kernel<false, false, false><<<grid, block, shape.smem_bytes, stream>>>(P);
  }
  return cudaGetLastError();
}

cudaError_t kernel_arch(int* binary_version, int* ptx_version) {
  cudaFuncAttributes fa;
  const cudaError_t e = cudaFuncGetAttributes(&fa, decode_kernel<false, false, false>);
  if (e != cudaSuccess) return e;
  if (binary_version) *binary_version = fa.binaryVersion;
  if (ptx_version) *ptx_version = fa.ptxVersion;
  return cudaSuccess;
}

cudaError_t launch_batch_prefix(const gmp_file_desc* files, uint32_t n_files, uint64_t* item_start,
                                cudaStream_t stream) {
  batch_prefix_kernel<<<1, 1024, 0, stream>>>(files, n_files, item_start);
  return cudaGetLastError();
}

}  // namespace gmp
