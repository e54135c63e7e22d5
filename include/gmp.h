/*
 * gmp.h - C ABI of the GB300 Gompresso-style decompressor (libgmp.so).
 *
 * Method: "Massively-Parallel Lossless Data Decompression" (Sitaridi, Mueller,
 * Kaldewey, Lohman, Ross; arXiv:1606.00519).  A stream is cut into blocks that
 * are compressed independently (Sec. 3.1).  Decompression of a block
 * Huffman-decodes its sub-blocks in parallel, one lane per sub-block, with
 * lookup tables of both trees in on-chip memory (Sec. 3.2.1), then resolves
 * the block's LZ77 sequences 32 at a time in one warp: two exclusive prefix
 * sums by shuffle, literal copy, then back-reference copy (Sec. 3.2.2), either
 * by Multi-Round Resolution (Fig. 5, Sec. 4.1) or, for streams written with
 * Dependency Elimination, in a single pass (Fig. 7, Sec. 4.2).  Streams in
 * the byte-level format (Gompresso/Byte, Sec. 3.1) skip the Huffman phase:
 * the warp reads the block's fixed-size sequence records and literal bytes
 * directly and resolves them the same way.
 *
 * Conventions for every function:
 *   - Return value: GMP_OK (0) or a negative gmp_error.  No exception crosses
 *     the ABI.  Argument and launch errors are returned synchronously.
 *   - Data errors found while decoding (a corrupt stream) are asynchronous:
 *     the kernel writes a positive gmp_status into the caller's int32 status
 *     word (first error wins) and abandons the damaged block; read it after
 *     the stream has synchronised.  The output of a damaged block is
 *     undefined; other blocks are still decoded.
 *   - "device" pointers are CUDA device (or managed) memory of the context's
 *     device; "host" pointers are ordinary host memory.  The caller owns every
 *     buffer it passes; the library never frees caller memory.
 *   - A context owns its scratch memory and is used by one stream at a time:
 *     calls on one context must be ordered on one CUDA stream.  Use one
 *     context per concurrent stream.
 *
 * Stream format (version 1; integers little-endian).  Written by
 * gmp_compress, read by the decoders.  The paper gives the structure (a file
 * header, then blocks, each with two canonical Huffman trees, sub-blocks with
 * their size in bits, and the bitstream; Sec. 3.1); the field layout is this
 * project's.
 *   File header, 64 bytes:
 *     0  "GMP1"            4  u16 version = 1      6  u16 flags (bit0 DE, bit1 Huffman)
 *     8  u32 block_size   12  u16 n_sub (K, 1..64; Byte 0) 14 u8 cwl (1..12; Byte 0)  15 u8 0
 *    16  u32 window (1..32768)  20 u8 min_match = 3  21 u8 max_match (3..64)  22 u16 0
 *    24  u64 orig_size    32  u64 n_blocks         40 u64 stream_bytes   48 16 bytes 0
 *   Block offset table at 64: u64 per block, byte offset of the block from the
 *   start of the stream (a multiple of 16).  The stream ends with >= 16 zero
 *   bytes of padding.
 *   Huffman block (Gompresso/Bit), at a 16-byte aligned offset:
 *     0  u32 n_seq   4 u32 out_bytes (block_size, except the last block)
 *     8  160 bytes: 4-bit code lengths of the 319 literal/length symbols
 *        (symbol s in byte s/2, low nibble for even s; 0 = unused)
 *   168  15 bytes: 4-bit code lengths of the 30 offset symbols   183 9 bytes 0
 *   192  n_sub entries {u32 bit_len, u32 out_bytes, u32 n_seq}: per sub-block
 *        its size in bits (Sec. 3.1), and two extensions of this format, its
 *        decompressed size and sequence count
 *   then, at the next 16-byte boundary, the bitstream: the sub-blocks' bits
 *   back to back (sub-block j starts at the sum of the earlier bit_len),
 *   LSB-first within bytes, Huffman codes sent most significant bit first,
 *   zero-padded to a 16-byte boundary.
 *   Literal/length symbols: 0..255 literal byte; 256 end of a block whose last
 *   sequence has no back-reference; 257..318 match length 3..64, followed by
 *   an offset symbol.  Offset symbol for distance d, v = d - 1: v < 4 gives
 *   symbol v; otherwise, with k = floor(log2 v), symbol 2k + bit (k-1) of v,
 *   followed by k-1 extra bits holding v mod 2^(k-1), LSB-first.
 *   Sub-blocks: a block's n_seq sequences are cut into K consecutive runs of
 *   whole sequences (runs may be empty); the decoder accepts any such split.
 *   gmp_compress makes the runs equal in decoding steps (literals + sequences).
 *   A sequence is a literal string followed by one back-reference (Sec. 3.2.2).
 *   Canonical codes (Sec. 3.1): codes of each length are consecutive in
 *   symbol order; the first code of length L is (first(L-1) + count(L-1)) << 1.
 *   Byte blocks (Gompresso/Byte, Sec. 3.1: the sequences coded at byte
 *   level, without Huffman trees, so that decoding is a plain read of the
 *   records; file header flags bit1 = 0, n_sub = 0, cwl = 0):
 *     0  u32 n_seq   4 u32 out_bytes   8 u32 n_lit (literal bytes)   12 u32 0
 *    16  n_seq records, u32 each: bits 0-9 literal length (0..1023), bits
 *        10-15 match code m (0 = no back-reference, 1..62 = match length
 *        m + 2), bits 16-31 distance - 1
 *   then, at the next 16-byte boundary, the n_lit literal bytes of the block
 *   in sequence order, zero-padded to a 16-byte boundary.  Any sequence may
 *   lack a back-reference (a literal string longer than 1023 bytes is written
 *   as several sequences).
 *   DE flag: every back-reference of a 32-sequence group (numbered from the
 *   block start) reads only bytes produced before the group's copies start:
 *   bytes before the group, the group's literal strings, or earlier bytes of
 *   its own copy.  The decoder checks this per group and falls back to MRR for
 *   a group that breaks it, so a wrong flag costs speed, never correctness.
 */
#ifndef GMP_H_
#define GMP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GMP_VERSION 1

typedef enum {
  GMP_OK = 0,
  GMP_ERR_INVALID_ARG = -1, /* null pointer, bad size or alignment, bad option */
  GMP_ERR_CAPACITY = -2,    /* a caller buffer or the context's scratch is too small */
  GMP_ERR_CUDA = -3,        /* a CUDA runtime call failed (see gmp_last_cuda_error) */
  GMP_ERR_UNSUPPORTED = -4, /* valid stream feature this build does not decode */
  GMP_ERR_FORMAT = -5,      /* host-side parse found a malformed stream header */
  GMP_ERR_NOMEM = -6        /* host allocation failed */
} gmp_error;

/* Values written to the caller's int32 status word by the decoder. */
typedef enum {
  GMP_STATUS_OK = 0,
  GMP_STATUS_BAD_HEADER = 1,        /* block header inconsistent (sizes, code lengths, Kraft) */
  GMP_STATUS_CORRUPT_SYMBOL = 2,    /* bit pattern with no code, or end symbol before the end */
  GMP_STATUS_BITSTREAM = 3,         /* a sub-block read past its stored size or did not use it all */
  GMP_STATUS_BAD_OFFSET = 4,        /* distance 0, beyond the window, or before the block start */
  GMP_STATUS_OUTPUT_OVERRUN = 5,    /* decoded sizes disagree with the header or exceed out_cap */
  GMP_STATUS_MRR_NO_PROGRESS = 6,   /* a resolution round made no progress (cannot happen on valid input) */
  GMP_STATUS_CAPACITY = 7,          /* a block needs more scratch than the context reserved */
  GMP_STATUS_INPUT_TIMEOUT = 8      /* host-to-host calls: a piece's input copy did not complete within the
                                       kernel's wait limit (about 10 s); its blocks were not decoded */
} gmp_status;

/* ------------------------------------------------------------------------ */
/* Stream header and block index (host, no CUDA).                           */

typedef struct {
  uint32_t version, flags, block_size, n_sub, cwl, window, min_match, max_match;
  uint64_t orig_size, n_blocks, stream_bytes;
  /* filled by gmp_index_build from the block headers: */
  uint32_t max_block_out, max_block_seq;
} gmp_stream_info;

/* One block of a stream: where its compressed bytes are (relative to the
   stream start) and where its output goes (relative to the output start). */
typedef struct {
  uint64_t comp_offset, comp_bytes, out_offset, out_bytes;
} gmp_block_ref;

/* Parse the 64-byte file header.  host_stream: host pointer to at least
   `bytes` bytes of the stream.  Returns GMP_ERR_FORMAT on a bad header. */
int gmp_stream_info_parse(const void* host_stream, size_t bytes, gmp_stream_info* info);

/* Build the block index (Sec. 3.2.2: each warp finds its block from the block
   offsets; all blocks but the last have block_size bytes of output).
   host_stream: the whole stream in host memory.  out: host array of `cap`
   entries (may be NULL with cap 0 to query *n_blocks).  Also checks every
   block header's sizes against the file header and fills info (may be NULL).
   Returns GMP_ERR_CAPACITY if cap < n_blocks (with *n_blocks set). */
int gmp_index_build(const void* host_stream, size_t bytes, gmp_block_ref* out, size_t cap, size_t* n_blocks,
                    gmp_stream_info* info);

/* ------------------------------------------------------------------------ */
/* Compressor (host, multi-threaded over blocks).  Not on the decode path; it
   writes the format above (Sec. 3.1: block split, LZ77, two length-limited
   canonical Huffman trees per block, sub-blocks; Sec. 4.2 for DE).         */

typedef struct {
  uint32_t block_size;  /* bytes per block (default 256 KiB) */
  uint32_t n_sub;       /* K sub-blocks per block, 1..64 (default 32) */
  uint32_t window;      /* LZ77 window, 1..32768 (default 32 KiB) */
  uint32_t cwl;         /* Huffman code length limit, 9..12 (default 12; 319 symbols need 9) */
  uint32_t max_match;   /* 3..64 (default 64) */
  uint32_t chain_depth; /* match candidates tried per position (default 64) */
  uint32_t de;          /* 1: Dependency Elimination (Sec. 4.2), 0: plain (MRR) */
  uint32_t n_threads;   /* host threads, 0 = all cores */
  uint32_t lazy;        /* 1: one-step lazy match evaluation (default), 0: greedy */
  uint32_t byte_mode;   /* 1: byte-level blocks (Gompresso/Byte, no Huffman; n_sub and cwl
                           are ignored), 0: Huffman blocks (Gompresso/Bit, default) */
} gmp_compress_opts;

void gmp_compress_opts_default(gmp_compress_opts* o);
/* Upper bound of the compressed size of n input bytes. */
size_t gmp_compress_bound(size_t n, const gmp_compress_opts* o);
/* host_in: n bytes; host_out: cap bytes.  *out_bytes receives the stream size.
   GMP_ERR_CAPACITY if cap < the stream size (use gmp_compress_bound). */
int gmp_compress(const void* host_in, size_t n, const gmp_compress_opts* o, void* host_out, size_t cap,
                 size_t* out_bytes);

/* Compression on the GPU `device`, every step of it (Sec. 3.1: blocks are
   compressed independently, so all of them at once; Sec. 4.2 for DE).
   Match search: a CTA per block finds, for 512 positions at a time, the
   longest match among up to min(o->chain_depth, 64) earlier positions with
   the same 3-byte prefix hash (input window, chain heads and links in shared
   memory).  Parse: a warp per block (lazy evaluation, the DE rule when
   o->de, 1023-byte literal runs for Byte blocks).  Entropy coding: a CTA
   per block counts both alphabets, builds code lengths limited to o->cwl
   bits (two-queue Huffman, then the bit-length adjustment of ITU-T T.81
   Annex K.3), canonical codes, the sub-block split (equal decoding work) and
   sizes, then packs each sub-block's codes at its bit offset; Byte blocks
   get their records and literals.  The host lays the blocks out from their
   sizes and writes the file header and block offset table; the stream
   format is gmp_compress's.  Positions of one step do not see each other
   and the code lengths are built differently, so ratios differ slightly
   from gmp_compress's.  Host buffers; uses about 10 bytes of device memory
   per input byte, freed before it returns.  Synchronous.  GMP_ERR_CUDA on a
   CUDA failure (gmp_last_cuda_error), GMP_ERR_CAPACITY if cap is too small
   (gmp_compress_bound). */
int gmp_compress_gpu(int device, const void* host_in, size_t n, const gmp_compress_opts* o, void* host_out,
                     size_t cap, size_t* out_bytes);

/* Device times (CUDA events) of the calling thread's last successful
   gmp_compress_gpu: match search, parse, and entropy coding (planning and
   writing every block), in milliseconds; all zero before the first call. */
typedef struct {
  double match_ms, parse_ms, encode_ms;
  uint64_t compressed_bytes;
} gmp_gpu_compress_times;
void gmp_compress_gpu_last_times(gmp_gpu_compress_times* t);

/* One-block stream holding a given LZ77 parse (the entropy-coding half of
   the compressor, for callers with their own match finder, and for streams
   with a chosen dependency structure such as the nesting-depth data sets of
   Sec. 5.1).  Sequence i is lit_len[i] literal bytes, taken in order from
   lits (n_lits bytes in all), then a back-reference of match_len[i] bytes
   (0 = none) at distance dist[i].  Host arrays.  Checks: match lengths 3 ..
   o->max_match, distances 1 .. min(o->window, bytes before the copy), total
   output <= o->block_size, the literals used exactly; for Huffman blocks only
   the last sequence may lack a back-reference (Byte blocks cut literal
   strings over 1023 bytes).  The DE flag (o->de) is written as given and not
   verified; the decoder checks it per group.  GMP_ERR_INVALID_ARG on a bad
   parse, GMP_ERR_CAPACITY if cap is too small (2 * n_lits + 5 * n_seq +
   1280 bytes always suffice). */
int gmp_encode_tokens(const uint32_t* lit_len, const uint32_t* match_len, const uint32_t* dist, size_t n_seq,
                      const uint8_t* lits, size_t n_lits, const gmp_compress_opts* o, void* host_out, size_t cap,
                      size_t* out_bytes);

/* ------------------------------------------------------------------------ */
/* Decoder context. */

typedef struct gmp_context gmp_context;

typedef struct {
  uint32_t max_block_out;   /* largest block output the scratch must hold (default 256 KiB) */
  uint32_t warps_per_cta;   /* 0 = tuned default */
  uint32_t ctas_per_sm;     /* 0 = as many as fit */
  uint32_t collect_stats;   /* 1: count groups and MRR rounds (small cost) */
  uint32_t max_files;       /* largest n_files of gmp_decompress_batch (default 65536) */
  uint32_t resolve;         /* back-reference resolution, a gmp_resolve (default GMP_RESOLVE_AUTO) */
  uint32_t concurrent;      /* 1: launches run beside other kernels (a serving loop's overlapping
                               batches): every warp takes its blocks from the work counter as it
                               arrives; 0 (default): a warp's first block is fixed, interleaved
                               over the CTAs, which spreads a launch's blocks evenly over the SMs
                               when all its CTAs are resident at once */
} gmp_context_opts;

/* How a context resolves each 32-sequence group's back-references.  AUTO:
   streams with the DE flag in one pass (groups that break the DE property by
   MRR), others by Multi-Round Resolution (Fig. 5, Sec. 4.1).  MRR: MRR even
   for DE streams.  SC: Sequential Copying, one back-reference at a time in
   sequence order, the paper's baseline (Sec. 5.1).  All give the same bytes;
   MRR and SC exist to measure the strategies against each other. */
typedef enum { GMP_RESOLVE_AUTO = 0, GMP_RESOLVE_MRR = 1, GMP_RESOLVE_SC = 2 } gmp_resolve;

void gmp_context_opts_default(gmp_context_opts* o);
/* Creates a context on `device`: allocates the scratch of one persistent
   launch (one slot per resident warp) and a small device work counter.
   opts may be NULL.  A context is not thread-safe, and its launches share
   the scratch: calls on one context must not run at the same time, from
   several host threads or on streams whose work overlaps (use a context per
   stream, as the serving loop's lanes do). */
int gmp_context_create(gmp_context** ctx, int device, const gmp_context_opts* opts);
void gmp_context_destroy(gmp_context* ctx);
/* Change launch shape (an autotuner result); reallocates scratch if needed. */
int gmp_context_set_launch(gmp_context* ctx, uint32_t warps_per_cta, uint32_t ctas_per_sm);
/* Bytes of device scratch the context holds. */
size_t gmp_context_scratch_bytes(const gmp_context* ctx);
/* Host-to-host calls: how long a warp waits for a piece's input copy before
   the piece's file gets GMP_STATUS_INPUT_TIMEOUT (ms; 0 = the default,
   10 000).  A longer limit suits slow pageable copies. */
int gmp_context_set_input_wait(gmp_context* ctx, uint32_t ms);
/* Test hook (fault injection on the host): the context's next host-to-host
   call copies piece `piece` (0-based, in the call's piece order) in but does
   not write its flag, so the warps waiting for it run out their wait and the
   files of the call report GMP_STATUS_INPUT_TIMEOUT; -1 clears it.  The
   kernel ends by itself, and the context stays usable. */
int gmp_context_debug_drop_input_flag(gmp_context* ctx, int64_t piece);

/* ------------------------------------------------------------------------ */
/* Decompression of one stream (Sec. 3.2): one persistent launch, a warp per
   block taken from a work counter.
   d_comp: device, the whole stream (16-byte aligned); comp_bytes its size.
   d_index: device array of n_blocks gmp_block_ref (from gmp_index_build).
   d_out: device output buffer of out_cap bytes (16-byte aligned for the
   vectorised store path; other alignments use byte stores).
   d_status: device int32, set to 0 by this call (stream-ordered) and then to
   the first gmp_status error if any.  stream: a cudaStream_t (NULL = legacy
   default stream).  Asynchronous; no allocation. */
int gmp_decompress(gmp_context* ctx, const uint8_t* d_comp, size_t comp_bytes, const gmp_block_ref* d_index,
                   size_t n_blocks, uint8_t* d_out, size_t out_cap, int32_t* d_status, void* stream);

/* ------------------------------------------------------------------------ */
/* Batched decompression: many independent streams in ONE persistent launch.
   Every (file, block) pair is a work item; warps take items from a device
   counter, so files of uneven sizes share the GPU.                         */
typedef struct {
  const uint8_t* comp;          /* device, 16-byte aligned stream */
  uint64_t comp_bytes;
  const gmp_block_ref* index;   /* device, n_blocks entries */
  uint64_t n_blocks;
  uint8_t* out;                 /* device output buffer */
  uint64_t out_cap;
} gmp_file_desc;

/* d_files: device array of n_files descriptors.  d_status: device array of
   n_files int32, each zeroed by this call and then set to the file's first
   error.  A small single-CTA kernel first forms the work-item prefix over the
   files' block counts in context scratch (n_files <= max_files of the
   context, else GMP_ERR_CAPACITY); the persistent kernel then maps each item
   to its (file, block) by binary search.  Asynchronous; no allocation;
   capturable in a CUDA graph (gmp_batch_graph_create does that). */
int gmp_decompress_batch(gmp_context* ctx, const gmp_file_desc* d_files, size_t n_files, int32_t* d_status,
                         void* stream);

/* A CUDA graph holding one batched launch (counter reset + status reset +
   the persistent kernel), replayed with gmp_graph_launch. */
typedef struct gmp_graph gmp_graph;
int gmp_batch_graph_create(gmp_context* ctx, const gmp_file_desc* d_files, size_t n_files, int32_t* d_status,
                           void* stream, gmp_graph** g);
int gmp_graph_launch(gmp_graph* g, void* stream);
void gmp_graph_destroy(gmp_graph* g);

/* ------------------------------------------------------------------------ */
/* Launch-shape autotuner: times the batched decode of a sample (device file
   descriptors, as for gmp_decompress_batch) under several shapes (warps per
   CTA 1, 2, 4, 8, 16; CTAs per SM as many as fit and half of that), keeps
   the fastest in the context and reports it.  Each shape is run once to
   warm up and three times timed with CUDA events on `stream`; the context's
   scratch is reallocated when a shape needs more.  Synchronous. */
typedef struct {
  uint32_t warps_per_cta, ctas_per_sm; /* the chosen shape */
  double best_ms;                      /* its mean time per batched launch */
  uint32_t shapes_tried;
} gmp_tuning;
int gmp_autotune(gmp_context* ctx, const gmp_file_desc* d_files, size_t n_files, int32_t* d_status, void* stream,
                 gmp_tuning* out);

/* ------------------------------------------------------------------------ */
/* Statistics of the launches since gmp_stats_reset (collect_stats=1):
   32-sequence groups resolved, resolution rounds, groups of a DE stream that
   broke the DE property and were resolved by MRR, blocks decoded, the largest
   round count of a group, and SM clock cycles summed over warps spent on
   block setup (headers and lookup tables), Huffman decoding and LZ77
   resolution.  Per round r (rounds after the 8th in bin 7): back-reference
   bytes copied in round r and groups that ran a round r, so that
   round_bytes[r] / round_groups[r] is the mean bytes resolved per group in
   round r (the quantity of the paper's bytes-per-round measurement, Sec. 5.1). */
typedef struct {
  uint64_t groups, rounds, de_fallback_groups, blocks, max_rounds;
  uint64_t cycles_tables, cycles_huffman, cycles_lz77;
  uint64_t detail[8]; /* stage timers of profiling builds (GMP_PHASE_TIMERS), else 0 */
  uint64_t round_bytes[8], round_groups[8];
} gmp_stats;
int gmp_stats_reset(gmp_context* ctx, void* stream);
int gmp_stats_read(gmp_context* ctx, gmp_stats* out); /* synchronises the device */

/* ------------------------------------------------------------------------ */
/* Host-to-host decompression (the paper's "(In/Out)" mode, Sec. 5.4: input
   and output in host memory, transfers included).  One persistent launch
   decodes all the streams' blocks, which are cut into pieces of consecutive
   blocks (about 32 pieces, 8 to 256 blocks each).  The pieces are copied in,
   in order, on one copy stream, which sets a device flag after each piece;
   a warp waits for its piece's flag before reading it, so decoding starts
   with the first piece.  The kernel sets a second flag once a piece is
   decoded, and the piece's copy back waits for that flag (a stream memory
   operation, cuStreamWaitValue32) on one of 8 copy-back streams, so outputs
   go back while later pieces decode.  A warp's wait for its input is bounded
   (about 10 s; then the file's status is GMP_STATUS_INPUT_TIMEOUT), so the
   call always ends.  Host buffers should be pinned (cudaHostAlloc /
   cudaHostRegister) for the copies to overlap; pageable buffers work but
   serialise the copies.  Uses (and grows) device staging buffers owned by
   the context.  GMP_ERR_CUDA if the driver lacks stream memory operations.
   gmp_decompress_host_batch: n_files streams (host_streams[f], bytes[f]) into
   host_outs[f] (out_caps[f] bytes each); statuses[f] (host) receives file
   f's decoder status.  GMP_ERR_CAPACITY if an output buffer is too small or
   a block exceeds the context's max_block_out.  Synchronous: returns when
   every output is in host memory; work is ordered after earlier work on
   `stream` (the block indexes and stream headers are copied on it first)
   and later work on `stream` is ordered after this call's. */
int gmp_decompress_host_batch(gmp_context* ctx, size_t n_files, const void* const* host_streams, const size_t* bytes,
                              void* const* host_outs, const size_t* out_caps, int32_t* statuses, void* stream);
/* One stream: host_out holds out_cap bytes; *status receives the status. */
int gmp_decompress_host(gmp_context* ctx, const void* host_stream, size_t bytes, void* host_out, size_t out_cap,
                        int32_t* status, void* stream);
/* The paper's "(In)" mode (Sec. 5.4: compressed input in host memory, the
   decompressed output left on the GPU): as gmp_decompress_host_batch, but
   d_outs[f] are device buffers of the context's device (out_caps[f] bytes
   each), which the launch decodes into directly; there are no copies back.
   The input copies overlap the decoding of earlier pieces.  Synchronous in
   the same way (returns with every output in device memory and statuses[f]
   filled in on the host). */
int gmp_decompress_from_host_batch(gmp_context* ctx, size_t n_files, const void* const* host_streams,
                                   const size_t* bytes, void* const* d_outs, const size_t* out_caps, int32_t* statuses,
                                   void* stream);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of decompression requests under a device
   memory budget (host runtime, one scheduler thread).  A request is a
   compressed stream in host memory; its block index is built at submit.  The
   scheduler admits requests in arrival order whenever the device arena has
   room for the request's compressed bytes, index and output, and launches
   the admitted ones as a batch (gmp_decompress_batch) on the first idle lane
   (a context with its own CUDA stream).  Requests that arrive while batches
   run join the next batch, and batches on different lanes overlap on the
   GPU.  Outputs stay in device memory until released.  Timestamps are
   seconds on the server's monotonic clock (gmp_server_now). */
typedef struct gmp_server gmp_server;
typedef struct {
  uint64_t budget_bytes;  /* device arena for request buffers (default 32 GiB) */
  uint32_t n_lanes;       /* batches in flight at once (default 8); each lane is a context with
                             its own scratch (about 1.7 MB per resident warp for 256 KiB blocks) */
  uint32_t max_batch;     /* requests per launch (default 64; 1 = one launch per request) */
  uint32_t max_block_out; /* largest block output of any request (default 256 KiB) */
  uint32_t warps_per_cta; /* launch shape of the lanes' contexts (0 = default) */
} gmp_server_opts;
typedef struct {
  uint64_t id;
  int32_t status;        /* gmp_status of the decode */
  uint8_t* d_out;        /* device output, valid until gmp_server_release(id) */
  uint64_t out_bytes;
  double t_submit, t_start, t_done;  /* host clock (s): submitted, its batch launched, batch done */
  /* device clock (s, CUDA events on the lane's stream, from the server's
     creation): its batch's inputs copied in and the decode next on the
     stream, and the decode ended.  Batches whose intervals overlap ran on
     the GPU at the same time. */
  double t_gpu_ready, t_gpu_done;
} gmp_completion;

void gmp_server_opts_default(gmp_server_opts* o);
/* Allocates the arena (budget_bytes of device memory) and the lanes. */
int gmp_server_create(gmp_server** s, int device, const gmp_server_opts* opts);
/* host_stream must stay valid and unchanged until the request completes.
   GMP_ERR_CAPACITY if the request alone exceeds the budget or its blocks
   exceed max_block_out.  Thread-safe. */
int gmp_server_submit(gmp_server* s, const void* host_stream, size_t bytes, uint64_t* id);
/* Moves up to cap completions into out (*n set), waiting up to wait_ms for
   the first one.  Returns a sticky gmp_error if the scheduler failed. */
int gmp_server_poll(gmp_server* s, gmp_completion* out, size_t cap, size_t* n, int wait_ms);
/* Frees a completed request's device memory (its output included). */
int gmp_server_release(gmp_server* s, uint64_t id);
/* Waits until every submitted request has completed. */
int gmp_server_drain(gmp_server* s);
/* Copies a completed request's output (out_bytes of it, at most cap) to dst,
   a host pointer (dst_is_device 0) or a device pointer of the server's device
   (dst_is_device 1).  Synchronous. */
int gmp_server_copy_out(gmp_server* s, uint64_t id, void* dst, size_t cap, int dst_is_device);
double gmp_server_now(gmp_server* s);
uint64_t gmp_server_bytes_in_use(gmp_server* s);
void gmp_server_destroy(gmp_server* s);

/* ------------------------------------------------------------------------ */
/* Decompression without any device allocation.  The paper has no
   counterpart; this is an interface for callers that cannot call cudaMalloc:
   host callbacks and other code where the CUDA allocator must not be
   re-entered, and applications whose memory manager owns the whole device
   and forbids allocations by libraries.  gmp_decompress needs a context,
   whose creation allocates scratch; this call instead uses a scratch area
   held in a fixed-size __device__ array of the library (about 53 MB on every
   GPU that loads the library, kept until the process exits).
   Same arguments as gmp_decompress, without a context, plus max_block_out:
   the largest block output of the stream (gmp_stream_info.max_block_out or
   block_size).  Limits: blocks of at most 256 KiB of output (larger:
   GMP_ERR_CAPACITY, and a block found larger on the device sets
   GMP_STATUS_CAPACITY), decoded by 32 warps at a time.
   Set-up: the array's device address belongs to one CUDA context.  The
   first call in each context (on each device, and again after a
   cudaDeviceReset) looks it up with cudaGetSymbolAddress, which loads the
   module on that device; later calls in that context reuse it.
   Every call shares the one array and clears its work counter: calls whose
   work overlaps on the GPU (different streams, or several host threads)
   race and must be serialised by the caller.
   Allocates nothing, neither with cudaMalloc nor through any library. */
int gmp_decompress_noalloc(const uint8_t* d_comp, size_t comp_bytes, const gmp_block_ref* d_index,
                           size_t n_blocks, uint32_t max_block_out, uint8_t* d_out, size_t out_cap,
                           int32_t* d_status, void* stream);
/* The fixed limits of gmp_decompress_noalloc (any pointer may be NULL). */
void gmp_noalloc_limits(uint32_t* max_block_out, uint32_t* warps, uint64_t* scratch_bytes);

/* Last CUDA error string of this thread (for GMP_ERR_CUDA). */
const char* gmp_last_cuda_error(void);

/* The architecture the library's decode kernel was compiled for, as the CUDA
   runtime reports it on the current device (cudaFuncGetAttributes):
   binary_version = 10 * major + minor of the kernel's machine code (103 for
   sm_103a), ptx_version likewise for the virtual architecture it was
   compiled from.  Either pointer may be NULL.  Needs a GPU: GMP_ERR_CUDA
   when the runtime has no usable device or no code for it. */
int gmp_kernel_arch(int* binary_version, int* ptx_version);

#ifdef __cplusplus
}
#endif
#endif /* GMP_H_ */
