/*
 * CPU ORACLE for the Gompresso-style decompression path.  TEST INFRASTRUCTURE
 * ONLY: the tests, the smoke check and the benchmark's CPU-baseline leg use
 * it; the product library never links, loads or calls it, and it shares no
 * code with the CUDA path (only the documented stream format is common).
 *
 * Plain, slow and serial on purpose.  What it computes, with the paper's
 * passages ("Massively-Parallel Lossless Data Decompression", Sitaridi et
 * al., arXiv:1606.00519):
 *
 *   - block split, LZ77 with a sliding window and literal/back-reference
 *     tokens grouped into sequences (Sec. 2.1, Fig. 1; Sec. 3.1; Sec. 3.2.2
 *     "sequence"), greedy parse with trigram hash chains;
 *   - Dependency Elimination, the modified LZ77 of Fig. 7 (Sec. 4.2): per
 *     group of 32 sequences, matches are looked for below warpHWM = the
 *     position where the group started;
 *   - two Huffman trees per block (literals + match lengths, and offsets;
 *     Sec. 3.1), length-limited to CWL bits (Sec. 5.3) by package-merge
 *     (Larmore and Hirschberg, 1990), written in canonical form (Sec. 3.1);
 *   - sub-blocks, each stored with its size in bits (Sec. 3.1, 3.2.1);
 *   - the serial decoder: canonical decoding one bit at a time, then the
 *     sequential LZ77 copy (Sec. 4: resolving back-references sequentially
 *     gives the correct output);
 *   - validators (Kraft equality, code lengths <= CWL, window and block
 *     bounds, the DE invariant of Sec. 4.2) and a simulator of Multi-Round
 *     Resolution (Fig. 5, Sec. 4.1) that counts rounds per 32-sequence group.
 *
 * Readings where the paper is silent or garbled:
 *   - MRR's HWM is the write position of the lowest-numbered pending lane
 *     (all lanes before it are complete and its literals are written), and a
 *     lane can copy once min(read_pos + length, write_pos) <= HWM, which also
 *     admits overlapping copies (offset < length).  The printed
 *     count_leading_zero_bits / read_pos + length rule is not used as is.
 *   - DE (Fig. 7, Sec. 4.2): read literally, a block's first group never
 *     gets a match (warpHWM = 0 until 32 matches close the group).  The DE
 *     compressor here lets a match read every byte the one-pass decoder has
 *     finished before a group's copies run: the bytes below warpHWM and the
 *     group's literal strings, but no byte an earlier back-reference of the
 *     same group writes (the candidate is cut at the first such byte).
 *   - A back-reference stores its distance (current position - source).
 *   - Sub-blocks: the block's n_seq sequences are cut into K runs of
 *     ceil(n_seq / K) sequences; trailing runs may be shorter or empty.
 *
 * Stream format (little-endian), shared by contract with the product:
 *   file header (64 B): "GMP1", u16 version=1, u16 flags (bit0 DE, bit1
 *   Huffman), u32 block_size, u16 n_sub, u8 cwl, u8 0, u32 window, u8
 *   min_match, u8 max_match, u16 0, u64 orig_size, u64 n_blocks, u64
 *   stream_bytes, 16 B zero; then u64 block offsets; blocks at 16-B aligned
 *   offsets; >= 16 zero bytes of tail padding.
 *   block: u32 n_seq, u32 out_bytes, 160 B lit/len code lengths (319 x 4 bit,
 *   low nibble first), 15 B offset code lengths (30 x 4 bit), 9 B zero; at
 *   192: n_sub x {u32 bit_len, u32 out_bytes, u32 n_seq}; bitstream at the
 *   next 16-B boundary, sub-blocks bit-contiguous, LSB-first, codes written
 *   most significant bit first; zero padding to 16 B.
 *   lit/len symbols: 0..255 literal, 256 end of block with no match (only in
 *   the block's last sequence), 257..318 match length 3..64.
 *   offset symbols: distance d, v = d - 1: v < 4 -> symbol v; else with
 *   k = floor(log2 v): symbol 2k + bit (k-1) of v, then k-1 extra bits
 *   v mod 2^(k-1), written LSB-first after the symbol.
 *   Byte streams (Gompresso/Byte, Sec. 3.1 and 3.2: byte-level encoding, no
 *   Huffman trees; flags bit1 = 0, n_sub = cwl = 0): block = u32 n_seq, u32
 *   out_bytes, u32 n_lit, u32 0, then n_seq 4-byte records (bits 0-9 literal
 *   length 0..1023, bits 10-15 match code m: 0 = no back-reference, 1..62 =
 *   length m + 2, bits 16-31 distance - 1), zero padding to 16 bytes, the
 *   n_lit literal bytes of the block in order, zero padding to 16 bytes.  A
 *   literal string longer than 1023 bytes is cut into literal-only
 *   sequences, which the parse counts like any other sequence.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

/* status values (documented in the stream format; the same numbers appear in
   the product's header, written separately there) */
enum {
  ORC_OK = 0,
  ORC_BAD_HEADER = 1,
  ORC_CORRUPT_SYMBOL = 2,
  ORC_BITSTREAM = 3,
  ORC_BAD_OFFSET = 4,
  ORC_OUTPUT_OVERRUN = 5,
  ORC_MRR_NO_PROGRESS = 6,
  ORC_ERR_ARG = -1,
  ORC_ERR_CAP = -2,
  ORC_ERR_NOMEM = -3,
};

#define N_LL 319
#define N_OFF 30
#define SYM_EOB 256
#define HDR_BYTES 64
#define BLK_FIXED 192
#define MAX_CWL 12

typedef struct {
  uint32_t block_size;
  uint32_t n_sub;
  uint32_t window;
  uint32_t cwl;
  uint32_t min_match;
  uint32_t max_match;
  uint32_t chain_depth;
  uint32_t de;
  uint32_t byte_mode; /* 1: Gompresso/Byte records instead of Huffman bitstreams */
} orc_params;

static void put16(uint8_t* p, uint32_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
static void put32(uint8_t* p, uint32_t v) { for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static void put64(uint8_t* p, uint64_t v) { for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static uint32_t get16(const uint8_t* p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 8); }
static uint32_t get32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static uint64_t get64(const uint8_t* p) {
  uint64_t v = 0;
  for (int i = 7; i >= 0; i--) v = (v << 8) | p[i];
  return v;
}
static uint64_t up16(uint64_t x) { return (x + 15) & ~(uint64_t)15; }

/* ------------------------------------------------------------------------ */
/* Offset symbols (format definition above; the distance code of Sec. 3.1's
   second tree).                                                             */
int orc_offset_encode(uint32_t d, uint32_t* sym, uint32_t* nextra, uint32_t* extra) {
  if (d < 1 || d > 32768) return ORC_ERR_ARG;
  uint32_t v = d - 1;
  if (v < 4) { *sym = v; *nextra = 0; *extra = 0; return 0; }
  uint32_t k = 0;
  while ((v >> (k + 1)) != 0) k++; /* k = floor(log2 v) */
  *sym = 2 * k + ((v >> (k - 1)) & 1u);
  *nextra = k - 1;
  *extra = v & ((1u << (k - 1)) - 1u);
  return 0;
}
uint32_t orc_offset_nextra(uint32_t sym) { return sym < 4 ? 0 : (sym >> 1) - 1; }
uint32_t orc_offset_decode(uint32_t sym, uint32_t extra) {
  if (sym < 4) return sym + 1;
  uint32_t k = sym >> 1;
  return (((2u + (sym & 1u)) << (k - 1)) + extra) + 1;
}

/* ------------------------------------------------------------------------ */
/* Length-limited Huffman code lengths by package-merge (Larmore and
   Hirschberg, "A fast algorithm for optimal length-limited Huffman codes",
   JACM 1990).  The L list: leaves sorted by weight; each further list merges
   the leaves with packages made of adjacent pairs of the previous list; the
   first 2m-2 items of the last list are selected, and a symbol's code length
   is the number of selected items that contain it.  An alphabet with one
   used symbol gets that symbol and one dummy symbol, both of length 1.      */
typedef struct { uint64_t w; int32_t left, right, sym; } pm_node;

static int pm_cmp_leaf(const void* a, const void* b) {
  const pm_node* x = (const pm_node*)a;
  const pm_node* y = (const pm_node*)b;
  if (x->w != y->w) return x->w < y->w ? -1 : 1;
  return x->sym - y->sym;
}

int orc_package_merge(const uint64_t* freq, int n, int limit, uint8_t* len_out) {
  if (n <= 0 || limit < 1 || limit > 30) return ORC_ERR_ARG;
  memset(len_out, 0, (size_t)n);
  int m = 0;
  for (int i = 0; i < n; i++) m += freq[i] > 0;
  if (m == 0) return 0;
  if (m == 1) {
    int s = 0;
    while (freq[s] == 0) s++;
    len_out[s] = 1;
    if (n > 1) len_out[s == 0 ? 1 : 0] = 1;
    return 0;
  }
  if (limit < 30 && (uint64_t)m > ((uint64_t)1 << limit)) return ORC_ERR_ARG;
  size_t cap = (size_t)m * (size_t)(limit + 1) + 8;
  pm_node* pool = (pm_node*)malloc(cap * sizeof(pm_node));
  int32_t* leaves = (int32_t*)malloc((size_t)m * sizeof(int32_t));
  int32_t* list = (int32_t*)malloc((size_t)2 * m * sizeof(int32_t));
  int32_t* next = (int32_t*)malloc((size_t)2 * m * sizeof(int32_t));
  int32_t* stack = (int32_t*)malloc(cap * sizeof(int32_t));
  if (!pool || !leaves || !list || !next || !stack) {
    free(pool); free(leaves); free(list); free(next); free(stack);
    return ORC_ERR_NOMEM;
  }
  int np = 0;
  for (int i = 0; i < n; i++)
    if (freq[i] > 0) { pool[np].w = freq[i]; pool[np].left = pool[np].right = -1; pool[np].sym = i; np++; }
  qsort(pool, (size_t)m, sizeof(pm_node), pm_cmp_leaf);
  for (int i = 0; i < m; i++) leaves[i] = i;
  int nl = m;
  for (int i = 0; i < m; i++) list[i] = leaves[i];
  for (int level = 1; level < limit; level++) {
    /* packages of adjacent pairs of the current list */
    int npk = nl / 2;
    int first_pkg = np;
    for (int i = 0; i < npk; i++) {
      pool[np].w = pool[list[2 * i]].w + pool[list[2 * i + 1]].w;
      pool[np].left = list[2 * i];
      pool[np].right = list[2 * i + 1];
      pool[np].sym = -1;
      np++;
    }
    /* merge leaves and packages by weight (a leaf goes first on ties) */
    int a = 0, b = 0, k = 0;
    while (a < m || b < npk) {
      if (b >= npk || (a < m && pool[leaves[a]].w <= pool[first_pkg + b].w)) next[k++] = leaves[a++];
      else next[k++] = first_pkg + b++;
    }
    nl = k;
    int32_t* t = list; list = next; next = t;
  }
  int take = 2 * m - 2;
  for (int i = 0; i < take; i++) {
    int sp = 0;
    stack[sp++] = list[i];
    while (sp) {
      int32_t x = stack[--sp];
      if (pool[x].sym >= 0) len_out[pool[x].sym]++;
      else { stack[sp++] = pool[x].left; stack[sp++] = pool[x].right; }
    }
  }
  free(pool); free(leaves); free(list); free(next); free(stack);
  return 0;
}

/* Canonical codes (Sec. 3.1): symbols sorted by (length, symbol value) get
   consecutive codes; when the length grows the next code is shifted left.
   Codes are returned most-significant-bit first.                            */
int orc_canonical_codes(const uint8_t* len, int n, uint32_t* code) {
  uint32_t count[MAX_CWL + 2] = {0}, nextc[MAX_CWL + 2] = {0};
  for (int s = 0; s < n; s++) {
    if (len[s] > MAX_CWL) return ORC_ERR_ARG;
    if (len[s]) count[len[s]]++;
  }
  uint32_t c = 0;
  for (int b = 1; b <= MAX_CWL; b++) {
    c = (c + count[b - 1]) << 1;
    if (b == 1) c = 0;
    nextc[b] = c;
  }
  for (int s = 0; s < n; s++) code[s] = len[s] ? nextc[len[s]]++ : 0;
  return 0;
}

/* Kraft sum over used symbols, scaled by 2^limit (an integer). */
uint64_t orc_kraft_scaled(const uint8_t* len, int n, int limit) {
  uint64_t s = 0;
  for (int i = 0; i < n; i++)
    if (len[i]) s += (uint64_t)1 << (limit - len[i]);
  return s;
}

/* ------------------------------------------------------------------------ */
/* Sequences: lit_len[i] literal bytes, then mlen[i] bytes copied from
   distance off[i] (mlen 0: the block's final literal-only sequence).      */
typedef struct {
  uint32_t *lit_len, *mlen, *off;
  size_t n, cap;
  uint8_t* lits;
  size_t nlits, lits_cap;
} seqbuf;

static int seq_push(seqbuf* s, const uint8_t* lit, uint32_t ll, uint32_t ml, uint32_t off) {
  if (s->n == s->cap) {
    size_t nc = s->cap ? 2 * s->cap : 1024;
    uint32_t* a = (uint32_t*)realloc(s->lit_len, nc * 4);
    if (!a) return ORC_ERR_NOMEM;
    s->lit_len = a;
    a = (uint32_t*)realloc(s->mlen, nc * 4);
    if (!a) return ORC_ERR_NOMEM;
    s->mlen = a;
    a = (uint32_t*)realloc(s->off, nc * 4);
    if (!a) return ORC_ERR_NOMEM;
    s->off = a;
    s->cap = nc;
  }
  if (s->nlits + ll > s->lits_cap) {
    size_t nc = s->lits_cap ? 2 * s->lits_cap : 4096;
    while (nc < s->nlits + ll) nc *= 2;
    uint8_t* a = (uint8_t*)realloc(s->lits, nc);
    if (!a) return ORC_ERR_NOMEM;
    s->lits = a;
    s->lits_cap = nc;
  }
  memcpy(s->lits + s->nlits, lit, ll);
  s->nlits += ll;
  s->lit_len[s->n] = ll;
  s->mlen[s->n] = ml;
  s->off[s->n] = off;
  s->n++;
  return 0;
}
static int lit_push(seqbuf* s, uint8_t b) {
  if (s->nlits == s->lits_cap) {
    size_t nc = s->lits_cap ? 2 * s->lits_cap : 4096;
    uint8_t* a = (uint8_t*)realloc(s->lits, nc);
    if (!a) return ORC_ERR_NOMEM;
    s->lits = a;
    s->lits_cap = nc;
  }
  s->lits[s->nlits++] = b;
  return 0;
}
static void seq_free(seqbuf* s) { free(s->lit_len); free(s->mlen); free(s->off); free(s->lits); memset(s, 0, sizeof(*s)); }

/* ------------------------------------------------------------------------ */
/* Greedy LZ77 of one block with trigram hash chains (the trigram key as in
   Sec. 4.2), at most chain_depth candidates per position, longest match in
   [min_match, max_match], distance <= window and <= position in the block;
   the nearest candidate wins ties.
   DE mode (Fig. 7, Sec. 4.2): per group of 32 sequences, warpHWM is the
   position where the group started.  Read literally, Fig. 7 never finds a
   match in a block's first group (warpHWM = 0 and a group only closes after
   32 matches), so this oracle takes the reading that matches what the DE
   decoder has finished before the group's copies run: every byte below
   warpHWM, and the literal strings of the group (the decoder writes all of a
   group's literals first).  A candidate's source bytes before the current
   position must avoid the bytes written by the group's earlier
   back-references; the candidate is cut at the first such byte.  Bytes at or
   after the current position belong to the copy itself (an overlapping
   copy), which one lane produces in order.                                  */
#define HBITS 15
static uint32_t hash3(const uint8_t* p) {
  uint32_t x = ((uint32_t)p[0] << 16) | ((uint32_t)p[1] << 8) | p[2];
  return (x * 2654435761u) >> (32 - HBITS);
}

static int lz77_block(const uint8_t* in, uint32_t n, const orc_params* P, seqbuf* out) {
  int32_t* head = (int32_t*)malloc(sizeof(int32_t) << HBITS);
  int32_t* prev = (int32_t*)malloc(sizeof(int32_t) * (n ? n : 1));
  if (!head || !prev) { free(head); free(prev); return ORC_ERR_NOMEM; }
  for (uint32_t i = 0; i < (1u << HBITS); i++) head[i] = -1;
  uint32_t pos = 0, lit_start = 0, in_group = 0;
  /* DE: destination intervals of this group's back-references so far */
  uint32_t gm_lo[32], gm_hi[32];
  int rc = 0;
#define INSERT(p_) do { uint32_t q_ = (p_); if (q_ + 3 <= n) { uint32_t h_ = hash3(in + q_); prev[q_] = head[h_]; head[h_] = (int32_t)q_; } } while (0)
  while (pos < n) {
    uint32_t best = 0, best_off = 0;
    if (pos + P->min_match <= n && pos + 3 <= n) {
      int32_t cand = head[hash3(in + pos)];
      uint32_t depth = 0;
      uint32_t maxl = n - pos < P->max_match ? n - pos : P->max_match;
      while (cand >= 0 && depth < P->chain_depth) {
        uint32_t c = (uint32_t)cand;
        if (pos - c > P->window) break;
        uint32_t l = 0;
        while (l < maxl && in[c + l] == in[pos + l]) l++;
        if (P->de) {
          /* cut at the first source byte (before pos) that an earlier copy of
             this group writes */
          for (uint32_t g = 0; g < in_group; g++) {
            uint32_t a = c, b = c + l < pos ? c + l : pos;
            if (gm_hi[g] <= a || gm_lo[g] >= b) continue;
            uint32_t lim = gm_lo[g] > c ? gm_lo[g] - c : 0;
            if (l > lim) l = lim;
          }
        }
        if (l >= P->min_match && l > best) { best = l; best_off = pos - c; }
        cand = prev[c];
        depth++;
      }
    }
    if (best) {
      rc = seq_push(out, in + lit_start, pos - lit_start, best, best_off);
      if (rc) break;
      for (uint32_t i = 0; i < best; i++) INSERT(pos + i);
      gm_lo[in_group] = pos;
      gm_hi[in_group] = pos + best;
      pos += best;
      lit_start = pos;
      if (++in_group == 32) in_group = 0; /* next group: warpHWM = pos */
    } else {
      INSERT(pos);
      pos++;
      if (P->byte_mode && pos - lit_start == 1023 && pos < n) {
        /* a Byte record holds at most 1023 literals: close a literal-only
           sequence (it counts towards the DE group like any other) */
        rc = seq_push(out, in + lit_start, 1023, 0, 0);
        if (rc) break;
        lit_start = pos;
        if (++in_group == 32) in_group = 0;
      }
    }
  }
  if (!rc && lit_start < n) rc = seq_push(out, in + lit_start, n - lit_start, 0, 0);
#undef INSERT
  free(head);
  free(prev);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Bit writer: LSB-first into a zeroed buffer. */
typedef struct { uint8_t* buf; uint64_t cap_bits, nbits; int overflow; } bitw;
static void bw_bit(bitw* w, uint32_t b) {
  if (w->nbits >= w->cap_bits) { w->overflow = 1; return; }
  if (b) w->buf[w->nbits >> 3] |= (uint8_t)(1u << (w->nbits & 7));
  w->nbits++;
}
static void bw_int(bitw* w, uint32_t v, uint32_t n) { for (uint32_t i = 0; i < n; i++) bw_bit(w, (v >> i) & 1u); }
static void bw_code(bitw* w, uint32_t code, uint32_t len) {
  for (int i = (int)len - 1; i >= 0; i--) bw_bit(w, (code >> i) & 1u);
}

/* Encode one block from its sequences (Sec. 3.1): per-block frequencies,
   two length-limited canonical trees, K sub-blocks each with its size in
   bits.  Returns the number of bytes written at dst or a negative error.   */
static int64_t encode_block(const seqbuf* S, uint32_t out_bytes, const orc_params* P, uint8_t* dst,
                            uint64_t cap) {
  uint64_t fl[N_LL] = {0}, fo[N_OFF] = {0};
  size_t li = 0;
  for (size_t i = 0; i < S->n; i++) {
    for (uint32_t k = 0; k < S->lit_len[i]; k++) fl[S->lits[li + k]]++;
    li += S->lit_len[i];
    if (S->mlen[i]) {
      if (S->mlen[i] < P->min_match || S->mlen[i] > P->max_match) return ORC_ERR_ARG;
      uint32_t sym, ne, ex;
      if (orc_offset_encode(S->off[i], &sym, &ne, &ex)) return ORC_ERR_ARG;
      fl[257 + S->mlen[i] - 3]++;
      fo[sym]++;
    } else {
      if (i + 1 != S->n) return ORC_ERR_ARG; /* only the last sequence may lack a match */
      fl[SYM_EOB]++;
    }
  }
  uint8_t ll[N_LL], lo[N_OFF];
  uint32_t cl[N_LL], co[N_OFF];
  if (orc_package_merge(fl, N_LL, (int)P->cwl, ll)) return ORC_ERR_ARG;
  if (orc_package_merge(fo, N_OFF, (int)P->cwl, lo)) return ORC_ERR_ARG;
  orc_canonical_codes(ll, N_LL, cl);
  orc_canonical_codes(lo, N_OFF, co);
  uint32_t K = P->n_sub;
  uint64_t bs_off = up16(BLK_FIXED + 12ull * K);
  if (cap < bs_off) return ORC_ERR_CAP;
  memset(dst, 0, bs_off);
  put32(dst, (uint32_t)S->n);
  put32(dst + 4, out_bytes);
  for (int s = 0; s < N_LL; s++) dst[8 + (s >> 1)] |= (uint8_t)(ll[s] << (4 * (s & 1)));
  for (int s = 0; s < N_OFF; s++) dst[168 + (s >> 1)] |= (uint8_t)(lo[s] << (4 * (s & 1)));
  bitw w = {dst + bs_off, (cap - bs_off) * 8, 0, 0};
  memset(dst + bs_off, 0, cap - bs_off);
  size_t per = (S->n + K - 1) / K;
  size_t seq = 0;
  li = 0;
  for (uint32_t j = 0; j < K; j++) {
    size_t end = seq + per < S->n ? seq + per : S->n;
    uint64_t b0 = w.nbits;
    uint32_t ob = 0, ns = 0;
    for (; seq < end; seq++) {
      for (uint32_t k = 0; k < S->lit_len[seq]; k++) {
        uint8_t b = S->lits[li + k];
        bw_code(&w, cl[b], ll[b]);
      }
      li += S->lit_len[seq];
      ob += S->lit_len[seq] + S->mlen[seq];
      if (S->mlen[seq]) {
        uint32_t s = 257 + S->mlen[seq] - 3;
        bw_code(&w, cl[s], ll[s]);
        uint32_t sym, ne, ex;
        orc_offset_encode(S->off[seq], &sym, &ne, &ex);
        bw_code(&w, co[sym], lo[sym]);
        bw_int(&w, ex, ne);
      } else {
        bw_code(&w, cl[SYM_EOB], ll[SYM_EOB]);
      }
      ns++;
    }
    uint8_t* e = dst + BLK_FIXED + 12 * j;
    put32(e, (uint32_t)(w.nbits - b0));
    put32(e + 4, ob);
    put32(e + 8, ns);
  }
  if (w.overflow) return ORC_ERR_CAP;
  return (int64_t)(bs_off + up16((w.nbits + 7) / 8));
}

/* Byte-level block (Gompresso/Byte): fixed 4-byte records, then the
   literal bytes.  Returns the bytes written or a negative error. */
static int64_t encode_block_byte(const seqbuf* S, uint32_t out_bytes, const orc_params* P, uint8_t* dst,
                                 uint64_t cap) {
  uint64_t rec_end = up16(16 + 4ull * S->n);
  uint64_t total = rec_end + up16(S->nlits);
  if (total > cap) return ORC_ERR_CAP;
  memset(dst, 0, total);
  put32(dst, (uint32_t)S->n);
  put32(dst + 4, out_bytes);
  put32(dst + 8, (uint32_t)S->nlits);
  for (size_t i = 0; i < S->n; i++) {
    uint32_t ll = S->lit_len[i], ml = S->mlen[i], d = S->off[i];
    if (ll > 1023) return ORC_ERR_ARG;
    if (ml && (ml < P->min_match || ml > P->max_match || d < 1 || d > 65536)) return ORC_ERR_ARG;
    uint32_t rec = ll | ((ml ? ml - 2 : 0u) << 10) | ((ml ? d - 1 : 0u) << 16);
    put32(dst + 16 + 4 * i, rec);
  }
  memcpy(dst + rec_end, S->lits, S->nlits);
  return (int64_t)total;
}

static int params_ok(const orc_params* P) {
  if (P->byte_mode)
    return P->block_size >= 1 && P->window >= 1 && P->window <= 32768 && P->min_match == 3 &&
           P->max_match >= 3 && P->max_match <= 64 && P->chain_depth >= 1;
  return P->block_size >= 1 && P->n_sub >= 1 && P->n_sub <= 64 && P->window >= 1 && P->window <= 32768 &&
         P->cwl >= 1 && P->cwl <= MAX_CWL && P->min_match == 3 && P->max_match >= 3 && P->max_match <= 64 &&
         P->chain_depth >= 1;
}

uint64_t orc_compress_bound(uint64_t n, const orc_params* P) {
  uint64_t nb = (n + P->block_size - 1) / P->block_size;
  /* every byte a literal of at most 12 bits plus one end symbol per block */
  /* Byte streams: at most one 4-byte record per byte plus the literals */
  if (P->byte_mode) return HDR_BYTES + up16(8 * nb) + nb * 48 + 5 * n + 64;
  return HDR_BYTES + up16(8 * nb) + nb * (up16(BLK_FIXED + 12ull * P->n_sub) + 32) + (n * 12 + 7) / 8 +
         nb * 2 + 64;
}

static void write_header(uint8_t* out, const orc_params* P, uint64_t n, uint64_t nb, uint64_t total) {
  memset(out, 0, HDR_BYTES);
  memcpy(out, "GMP1", 4);
  put16(out + 4, 1);
  put16(out + 6, (P->de ? 1u : 0u) | (P->byte_mode ? 0u : 2u));
  put32(out + 8, P->block_size);
  put16(out + 12, P->byte_mode ? 0u : P->n_sub);
  out[14] = (uint8_t)(P->byte_mode ? 0u : P->cwl);
  put32(out + 16, P->window);
  out[20] = (uint8_t)P->min_match;
  out[21] = (uint8_t)P->max_match;
  put64(out + 24, n);
  put64(out + 32, nb);
  put64(out + 40, total);
}

/* Whole-stream compressor (Sec. 3.1): blocks are compressed independently.
   Returns the stream size in bytes or a negative error. */
int64_t orc_compress(const uint8_t* in, uint64_t n, const orc_params* P, uint8_t* out, uint64_t cap) {
  if (!params_ok(P)) return ORC_ERR_ARG;
  uint64_t nb = (n + P->block_size - 1) / P->block_size;
  uint64_t pos = up16(HDR_BYTES + 8 * nb);
  if (cap < pos + 16) return ORC_ERR_CAP;
  memset(out, 0, pos);
  for (uint64_t b = 0; b < nb; b++) {
    uint64_t s = b * P->block_size;
    uint32_t len = (uint32_t)(n - s < P->block_size ? n - s : P->block_size);
    seqbuf S = {0};
    int rc = lz77_block(in + s, len, P, &S);
    if (rc) { seq_free(&S); return rc; }
    put64(out + HDR_BYTES + 8 * b, pos);
    int64_t w = P->byte_mode ? encode_block_byte(&S, len, P, out + pos, cap - pos)
                             : encode_block(&S, len, P, out + pos, cap - pos);
    seq_free(&S);
    if (w < 0) return w;
    pos += (uint64_t)w;
  }
  if (cap < pos + 16) return ORC_ERR_CAP;
  memset(out + pos, 0, 16);
  pos += 16;
  write_header(out, P, n, nb, pos);
  return (int64_t)pos;
}

/* A one-block stream from given sequences (for token streams built by
   construction, such as the Fig. 1 example or the nesting-depth sets).  The
   block holds out_bytes = sum(lit_len + mlen) <= block_size bytes.         */
int64_t orc_encode_tokens(const uint32_t* lit_len, const uint32_t* mlen, const uint32_t* off, uint64_t n_seq,
                          const uint8_t* lits, const orc_params* P, uint8_t* out, uint64_t cap) {
  if (!params_ok(P)) return ORC_ERR_ARG;
  uint64_t tot = 0, nl = 0;
  for (uint64_t i = 0; i < n_seq; i++) {
    /* every copy must stay inside the window and the block */
    uint64_t wpos = tot + lit_len[i];
    if (mlen[i] && (off[i] < 1 || off[i] > P->window || off[i] > wpos)) return ORC_ERR_ARG;
    tot = wpos + mlen[i];
    nl += lit_len[i];
  }
  if (tot > P->block_size || tot == 0) return ORC_ERR_ARG;
  seqbuf S;
  S.lit_len = (uint32_t*)lit_len;
  S.mlen = (uint32_t*)mlen;
  S.off = (uint32_t*)off;
  S.n = n_seq;
  S.cap = n_seq;
  S.lits = (uint8_t*)lits;
  S.nlits = nl;
  S.lits_cap = nl;
  uint64_t pos = up16(HDR_BYTES + 8);
  if (cap < pos + 16) return ORC_ERR_CAP;
  memset(out, 0, pos);
  put64(out + HDR_BYTES, pos);
  int64_t w = P->byte_mode ? encode_block_byte(&S, (uint32_t)tot, P, out + pos, cap - pos)
                           : encode_block(&S, (uint32_t)tot, P, out + pos, cap - pos);
  if (w < 0) return w;
  pos += (uint64_t)w;
  if (cap < pos + 16) return ORC_ERR_CAP;
  memset(out + pos, 0, 16);
  pos += 16;
  write_header(out, P, tot, 1, pos);
  return (int64_t)pos;
}

/* ------------------------------------------------------------------------ */
/* Decoding. */
typedef struct {
  uint32_t flags, block_size, n_sub, cwl, window, min_match, max_match;
  uint64_t orig_size, n_blocks, stream_bytes;
} orc_info;

int orc_stream_info(const uint8_t* s, uint64_t len, orc_info* I) {
  if (len < HDR_BYTES || memcmp(s, "GMP1", 4) != 0 || get16(s + 4) != 1) return ORC_BAD_HEADER;
  I->flags = get16(s + 6);
  I->block_size = get32(s + 8);
  I->n_sub = get16(s + 12);
  I->cwl = s[14];
  I->window = get32(s + 16);
  I->min_match = s[20];
  I->max_match = s[21];
  I->orig_size = get64(s + 24);
  I->n_blocks = get64(s + 32);
  I->stream_bytes = get64(s + 40);
  if (!(I->flags & 2u)) {
    /* Byte stream: no trees, no sub-blocks */
    if (I->n_sub != 0 || I->cwl != 0 || I->block_size == 0 || I->window == 0 || I->window > 32768 ||
        I->min_match != 3 || I->max_match < 3 || I->max_match > 64)
      return ORC_BAD_HEADER;
  } else if (I->block_size == 0 || I->n_sub == 0 || I->n_sub > 64 || I->cwl == 0 ||
      I->cwl > MAX_CWL || I->window == 0 || I->window > 32768 || I->min_match != 3 || I->max_match < 3 ||
      I->max_match > 64)
    return ORC_BAD_HEADER;
  if (I->stream_bytes > len) return ORC_BAD_HEADER;
  if (I->n_blocks != (I->orig_size + I->block_size - 1) / I->block_size) return ORC_BAD_HEADER;
  if (HDR_BYTES + 8 * I->n_blocks > len) return ORC_BAD_HEADER;
  return 0;
}

/* canonical decoding table of one tree */
typedef struct {
  uint32_t count[MAX_CWL + 1], first[MAX_CWL + 1], index[MAX_CWL + 1];
  uint16_t sorted[N_LL];
  int used;
} canon;

static int canon_build(const uint8_t* len, int n, int cwl, canon* c) {
  memset(c, 0, sizeof(*c));
  for (int s = 0; s < n; s++) {
    if (len[s] > cwl) return ORC_BAD_HEADER;
    if (len[s]) { c->count[len[s]]++; c->used++; }
  }
  if (c->used == 0) return 0;
  /* Kraft equality: a complete prefix code */
  uint64_t k = 0;
  for (int b = 1; b <= cwl; b++) k += (uint64_t)c->count[b] << (cwl - b);
  if (k != ((uint64_t)1 << cwl)) return ORC_BAD_HEADER;
  uint32_t code = 0, idx = 0;
  for (int b = 1; b <= cwl; b++) {
    c->first[b] = code;
    c->index[b] = idx;
    for (int s = 0; s < n; s++)
      if (len[s] == b) c->sorted[idx++] = (uint16_t)s;
    code = (code + c->count[b]) << 1;
  }
  return 0;
}

typedef struct { const uint8_t* p; uint64_t pos, end; int overrun; } bitr;
static uint32_t br_bit(bitr* r) {
  if (r->pos >= r->end) { r->overrun = 1; return 0; }
  uint32_t b = (r->p[r->pos >> 3] >> (r->pos & 7)) & 1u;
  r->pos++;
  return b;
}
/* one symbol: read bits one at a time, most significant code bit first */
static int canon_decode(const canon* c, int cwl, bitr* r) {
  if (c->used == 0) return -1;
  uint32_t code = 0;
  for (int b = 1; b <= cwl; b++) {
    code = (code << 1) | br_bit(r);
    if (r->overrun) return -2;
    if (code - c->first[b] < c->count[b]) return c->sorted[c->index[b] + code - c->first[b]];
  }
  return -1;
}

/* Decode the sequences of block b, checking every sub-block against its
   stored bit size, output size and sequence count.  Caller frees S.        */
/* Sequences of a Byte block: the records in order, literals from the
   block's literal section (format in the header comment). */
static int block_tokens_byte(const uint8_t* s, uint64_t len, const orc_info* I, uint64_t b, seqbuf* S,
                             uint32_t* out_bytes_p) {
  uint64_t bo = get64(s + HDR_BYTES + 8 * b);
  if (bo & 15 || bo + 16 > len) return ORC_BAD_HEADER;
  const uint8_t* B = s + bo;
  uint32_t n_seq = get32(B), out_bytes = get32(B + 4), n_lit = get32(B + 8);
  uint64_t expect = b + 1 < I->n_blocks ? I->block_size : I->orig_size - b * (uint64_t)I->block_size;
  if (out_bytes != expect) return ORC_BAD_HEADER;
  uint64_t lit_off = up16(16 + 4ull * n_seq);
  if (bo + lit_off + n_lit > len) return ORC_BAD_HEADER;
  uint64_t lp = 0, produced = 0;
  for (uint32_t i = 0; i < n_seq; i++) {
    uint32_t rec = get32(B + 16 + 4ull * i);
    uint32_t ll = rec & 1023u, m = (rec >> 10) & 63u;
    if (m > 62) return ORC_CORRUPT_SYMBOL;
    uint32_t ml = m ? m + 2 : 0, d = m ? (rec >> 16) + 1 : 0;
    if (ml > I->max_match) return ORC_CORRUPT_SYMBOL;
    if (lp + ll > n_lit) return ORC_OUTPUT_OVERRUN;
    if (seq_push(S, B + lit_off + lp, ll, ml, d)) return ORC_ERR_NOMEM;
    lp += ll;
    produced += ll + ml;
    if (produced > out_bytes) return ORC_OUTPUT_OVERRUN;
  }
  if (lp != n_lit || produced != out_bytes) return ORC_OUTPUT_OVERRUN;
  *out_bytes_p = out_bytes;
  return 0;
}

static int block_tokens(const uint8_t* s, uint64_t len, const orc_info* I, uint64_t b, seqbuf* S,
                        uint32_t* out_bytes_p) {
  if (!(I->flags & 2u)) return block_tokens_byte(s, len, I, b, S, out_bytes_p);
  uint64_t bo = get64(s + HDR_BYTES + 8 * b);
  uint64_t bs_off = up16(BLK_FIXED + 12ull * I->n_sub);
  if (bo & 15 || bo + bs_off > len) return ORC_BAD_HEADER;
  const uint8_t* B = s + bo;
  uint32_t n_seq = get32(B), out_bytes = get32(B + 4);
  uint64_t expect = b + 1 < I->n_blocks ? I->block_size : I->orig_size - b * (uint64_t)I->block_size;
  if (out_bytes != expect) return ORC_BAD_HEADER;
  uint8_t ll[N_LL], lo[N_OFF];
  for (int i = 0; i < N_LL; i++) ll[i] = (B[8 + (i >> 1)] >> (4 * (i & 1))) & 15;
  for (int i = 0; i < N_OFF; i++) lo[i] = (B[168 + (i >> 1)] >> (4 * (i & 1))) & 15;
  canon c1, c2;
  if (canon_build(ll, N_LL, (int)I->cwl, &c1) || canon_build(lo, N_OFF, (int)I->cwl, &c2)) return ORC_BAD_HEADER;
  uint64_t bit0 = (bo + bs_off) * 8, tot_seq = 0, tot_out = 0, bitpos = bit0;
  for (uint32_t j = 0; j < I->n_sub; j++) {
    const uint8_t* e = B + BLK_FIXED + 12 * j;
    uint64_t nbits = get32(e);
    uint32_t sb_out = get32(e + 4), sb_seq = get32(e + 8);
    bitr r = {s, bitpos, bitpos + nbits, 0};
    if ((bitpos + nbits + 7) / 8 > len) return ORC_BITSTREAM;
    uint32_t produced = 0;
    for (uint32_t q = 0; q < sb_seq; q++) {
      uint32_t ll_n = 0, ml = 0, off = 0;
      size_t lit0 = S->nlits;
      for (;;) {
        int sym = canon_decode(&c1, (int)I->cwl, &r);
        if (sym == -2) return ORC_BITSTREAM;
        if (sym < 0) return ORC_CORRUPT_SYMBOL;
        if (sym < 256) {
          if (lit_push(S, (uint8_t)sym)) return ORC_ERR_NOMEM;
          ll_n++;
          continue;
        }
        if (sym == SYM_EOB) break;
        ml = (uint32_t)sym - 254;
        int os = canon_decode(&c2, (int)I->cwl, &r);
        if (os == -2) return ORC_BITSTREAM;
        if (os < 0) return ORC_CORRUPT_SYMBOL;
        uint32_t ne = orc_offset_nextra((uint32_t)os), ex = 0;
        for (uint32_t i = 0; i < ne; i++) ex |= br_bit(&r) << i;
        if (r.overrun) return ORC_BITSTREAM;
        off = orc_offset_decode((uint32_t)os, ex);
        break;
      }
      if (ml == 0 && tot_seq + 1 != n_seq) return ORC_CORRUPT_SYMBOL; /* end symbol only at the end */
      if (ml > I->max_match) return ORC_CORRUPT_SYMBOL;
      /* the literal bytes are already in place at lits[lit0 ..) */
      S->nlits = lit0;
      if (seq_push(S, S->lits + lit0, ll_n, ml, off)) return ORC_ERR_NOMEM;
      produced += ll_n + ml;
      tot_seq++;
      if (produced > sb_out) return ORC_OUTPUT_OVERRUN;
    }
    if (r.pos != r.end) return ORC_BITSTREAM;
    if (produced != sb_out) return ORC_OUTPUT_OVERRUN;
    bitpos += nbits;
    tot_out += sb_out;
  }
  if (tot_seq != n_seq || tot_out != out_bytes) return ORC_BAD_HEADER;
  *out_bytes_p = out_bytes;
  return 0;
}

/* Sequential LZ77 decode of one block's sequences (byte by byte, so an
   overlapping copy repeats its pattern).  Every copy must lie inside the
   window and at or after the block's start.                               */
static int lz77_decode(const seqbuf* S, uint32_t window, uint8_t* out, uint64_t cap, uint64_t* n_out) {
  uint64_t p = 0;
  size_t li = 0;
  for (size_t i = 0; i < S->n; i++) {
    if (p + S->lit_len[i] > cap) return ORC_OUTPUT_OVERRUN;
    memcpy(out + p, S->lits + li, S->lit_len[i]);
    li += S->lit_len[i];
    p += S->lit_len[i];
    uint32_t d = S->off[i], m = S->mlen[i];
    if (m) {
      if (d < 1 || d > window || d > p) return ORC_BAD_OFFSET;
      if (p + m > cap) return ORC_OUTPUT_OVERRUN;
      for (uint32_t k = 0; k < m; k++) out[p + k] = out[p - d + k];
      p += m;
    }
  }
  *n_out = p;
  return 0;
}

/* Serial LZ77 decode of a plain token list (lits back to back). */
int orc_lz77_decode(const uint32_t* lit_len, const uint32_t* mlen, const uint32_t* off, uint64_t n_seq,
                    const uint8_t* lits, uint32_t window, uint8_t* out, uint64_t cap, uint64_t* n_out) {
  seqbuf S;
  uint64_t nl = 0;
  for (uint64_t i = 0; i < n_seq; i++) nl += lit_len[i];
  S.lit_len = (uint32_t*)lit_len;
  S.mlen = (uint32_t*)mlen;
  S.off = (uint32_t*)off;
  S.n = n_seq;
  S.cap = n_seq;
  S.lits = (uint8_t*)lits;
  S.nlits = nl;
  S.lits_cap = nl;
  return lz77_decode(&S, window, out, cap, n_out);
}

int orc_decompress_block(const uint8_t* s, uint64_t len, uint64_t b, uint8_t* out, uint64_t cap) {
  orc_info I;
  int rc = orc_stream_info(s, len, &I);
  if (rc) return rc;
  if (b >= I.n_blocks) return ORC_ERR_ARG;
  seqbuf S = {0};
  uint32_t ob;
  rc = block_tokens(s, len, &I, b, &S, &ob);
  uint64_t n = 0;
  if (!rc) rc = lz77_decode(&S, I.window, out, cap, &n);
  if (!rc && n != ob) rc = ORC_OUTPUT_OVERRUN;
  seq_free(&S);
  return rc;
}

int orc_decompress(const uint8_t* s, uint64_t len, uint8_t* out, uint64_t cap, uint64_t* out_len) {
  orc_info I;
  int rc = orc_stream_info(s, len, &I);
  if (rc) return rc;
  if (I.orig_size > cap) return ORC_OUTPUT_OVERRUN;
  for (uint64_t b = 0; b < I.n_blocks; b++) {
    uint64_t o = b * (uint64_t)I.block_size;
    rc = orc_decompress_block(s, len, b, out + o, cap - o);
    if (rc) return rc;
  }
  *out_len = I.orig_size;
  return 0;
}

/* Token dump of block b (arrays sized by the caller; returns counts). */
int orc_block_tokens(const uint8_t* s, uint64_t len, uint64_t b, uint32_t* lit_len, uint32_t* mlen,
                     uint32_t* off, uint64_t seq_cap, uint8_t* lits, uint64_t lits_cap, uint64_t* n_seq,
                     uint64_t* n_lits) {
  orc_info I;
  int rc = orc_stream_info(s, len, &I);
  if (rc) return rc;
  if (b >= I.n_blocks) return ORC_ERR_ARG;
  seqbuf S = {0};
  uint32_t ob;
  rc = block_tokens(s, len, &I, b, &S, &ob);
  if (!rc) {
    if (S.n > seq_cap || S.nlits > lits_cap) rc = ORC_ERR_CAP;
    else {
      memcpy(lit_len, S.lit_len, S.n * 4);
      memcpy(mlen, S.mlen, S.n * 4);
      memcpy(off, S.off, S.n * 4);
      memcpy(lits, S.lits, S.nlits);
      *n_seq = S.n;
      *n_lits = S.nlits;
    }
  }
  seq_free(&S);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* MRR simulator (Fig. 5, Sec. 4.1) for one block's sequences, one group of
   32 consecutive sequences at a time.  All literals of the group are written
   first.  Each round: HWM = write position of the lowest pending lane; every
   pending lane with min(read_pos + length, write_pos) <= HWM copies its
   back-reference.  Copies of one round run "in parallel": a byte written in
   this round is not readable by another lane until the next round (only the
   lane's own earlier bytes are).  The simulator fails if any copy reads a
   byte that is not yet available, or if a round makes no progress.
   With de_single_pass, each group instead runs every copy in one pass after
   its literals (the DE decoder), which fails if the stream breaks the
   no-same-group-dependency property.                                       */
typedef struct {
  uint64_t groups, rounds, max_rounds, copies, hist[34];
} mrr_stats;

static int mrr_block(const seqbuf* S, uint32_t out_bytes, int de_single_pass, const uint8_t* expect, mrr_stats* st,
                     uint32_t* per_group) {
  uint8_t* out = (uint8_t*)calloc(out_bytes ? out_bytes : 1, 1);
  uint32_t* avail = (uint32_t*)calloc(out_bytes ? out_bytes : 1, 4); /* round stamp at which the byte appeared; 0 = not yet */
  if (!out || !avail) { free(out); free(avail); return ORC_ERR_NOMEM; }
  int rc = 0;
  uint64_t G0 = 0, li = 0;
  uint32_t stamp = 1; /* increases every round across the whole block */
  for (size_t g = 0; g * 32 < S->n && !rc; g++) {
    size_t n = S->n - g * 32 < 32 ? S->n - g * 32 : 32;
    uint64_t wpos[32], rpos[32];
    uint32_t ml[32];
    int pending[32];
    uint64_t p = G0;
    /* literals of the whole group first */
    for (size_t l = 0; l < n; l++) {
      size_t i = g * 32 + l;
      for (uint32_t k = 0; k < S->lit_len[i]; k++) { out[p + k] = S->lits[li + k]; avail[p + k] = stamp; }
      li += S->lit_len[i];
      p += S->lit_len[i];
      wpos[l] = p;
      ml[l] = S->mlen[i];
      rpos[l] = p - S->off[i];
      pending[l] = ml[l] > 0;
      p += ml[l];
    }
    stamp++;
    uint32_t rounds = 0;
    for (;;) {
      int f = -1;
      for (size_t l = 0; l < n; l++)
        if (pending[l]) { f = (int)l; break; }
      if (f < 0) break;
      uint64_t hwm = wpos[f];
      int progressed = 0;
      for (size_t l = 0; l < n; l++) {
        if (!pending[l]) continue;
        uint64_t lim = rpos[l] + ml[l] < wpos[l] ? rpos[l] + ml[l] : wpos[l];
        int go = de_single_pass ? 1 : (lim <= hwm);
        if (!go) continue;
        for (uint32_t k = 0; k < ml[l]; k++) {
          uint64_t src = rpos[l] + k, dst = wpos[l] + k;
          /* readable: written before this round, or by this lane itself */
          int own = src >= wpos[l] && src < dst;
          if (!own && (avail[src] == 0 || avail[src] >= stamp)) { rc = ORC_MRR_NO_PROGRESS; break; }
          out[dst] = out[src];
          avail[dst] = stamp;
        }
        if (rc) break;
        pending[l] = 0;
        progressed = 1;
        st->copies++;
      }
      if (rc) break;
      stamp++;
      rounds++;
      if (!progressed || rounds > 32) { rc = ORC_MRR_NO_PROGRESS; break; }
      if (de_single_pass) {
        for (size_t l = 0; l < n; l++)
          if (pending[l]) rc = ORC_MRR_NO_PROGRESS;
        break;
      }
    }
    if (rc) break;
    if (per_group) per_group[g] = rounds;
    if (rounds) {
      st->groups++;
      st->rounds += rounds;
      if (rounds > st->max_rounds) st->max_rounds = rounds;
      st->hist[rounds]++;
    } else {
      st->hist[0]++;
    }
    G0 = p;
  }
  if (!rc && G0 != out_bytes) rc = ORC_OUTPUT_OVERRUN;
  if (!rc && expect && memcmp(out, expect, out_bytes) != 0) rc = ORC_MRR_NO_PROGRESS;
  free(out);
  free(avail);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Validation report over a whole stream. */
typedef struct {
  uint64_t n_blocks, n_seq, n_matches, lit_bytes, match_bytes;
  int32_t kraft_ok, lengths_ok, offsets_ok, blocks_ok, subblocks_ok, de_weak_ok, mrr_ok;
  uint64_t groups, rounds, max_rounds, copies;
  uint64_t round_hist[34];
  int32_t first_error;
  int32_t subblocks_even;
} orc_report;

int orc_validate(const uint8_t* s, uint64_t len, orc_report* R) {
  memset(R, 0, sizeof(*R));
  R->kraft_ok = R->lengths_ok = R->offsets_ok = R->blocks_ok = R->subblocks_ok = 1;
  R->de_weak_ok = R->mrr_ok = 1;
  R->subblocks_even = 1;
  orc_info I;
  int rc = orc_stream_info(s, len, &I);
  if (rc) { R->first_error = rc; return rc; }
  R->n_blocks = I.n_blocks;
  mrr_stats st;
  memset(&st, 0, sizeof(st));
  for (uint64_t b = 0; b < I.n_blocks; b++) {
    uint64_t bo = get64(s + HDR_BYTES + 8 * b);
    if (bo + ((I.flags & 2u) ? BLK_FIXED : 16u) > len) {
      R->blocks_ok = 0;
      R->first_error = ORC_BAD_HEADER;
      return ORC_BAD_HEADER;
    }
    const uint8_t* B = s + bo;
    const int is_byte = !(I.flags & 2u);
    if (!is_byte) {
      uint8_t ll[N_LL], lo[N_OFF];
      for (int i = 0; i < N_LL; i++) ll[i] = (B[8 + (i >> 1)] >> (4 * (i & 1))) & 15;
      for (int i = 0; i < N_OFF; i++) lo[i] = (B[168 + (i >> 1)] >> (4 * (i & 1))) & 15;
      for (int i = 0; i < N_LL; i++) if (ll[i] > I.cwl) R->lengths_ok = 0;
      for (int i = 0; i < N_OFF; i++) if (lo[i] > I.cwl) R->lengths_ok = 0;
      uint64_t k1 = orc_kraft_scaled(ll, N_LL, (int)I.cwl), k2 = orc_kraft_scaled(lo, N_OFF, (int)I.cwl);
      if (k1 != ((uint64_t)1 << I.cwl) || (k2 != 0 && k2 != ((uint64_t)1 << I.cwl))) R->kraft_ok = 0;
    }
    seqbuf S = {0};
    uint32_t ob;
    rc = block_tokens(s, len, &I, b, &S, &ob);
    if (rc) {
      seq_free(&S);
      R->subblocks_ok = 0;
      R->first_error = rc;
      return rc;
    }
    /* The format only fixes that the K sub-blocks are consecutive runs of
       whole sequences whose stored sizes match their bits (block_tokens
       checked that).  Whether the runs are the even split of c5, ceil(n_seq
       / K) sequences each (this oracle's own choice), is reported apart. */
    if (!is_byte) {
      uint64_t per = (S.n + I.n_sub - 1) / I.n_sub, left = S.n;
      for (uint32_t j = 0; j < I.n_sub; j++) {
        uint32_t ns = get32(B + BLK_FIXED + 12 * j + 8);
        uint64_t want = left < per ? left : per;
        if (ns != want) R->subblocks_even = 0;
        left -= want;
      }
    }
    uint64_t expect = b + 1 < I.n_blocks ? I.block_size : I.orig_size - b * (uint64_t)I.block_size;
    if (ob != expect) R->blocks_ok = 0;
    /* window and block bounds of every back-reference */
    uint64_t p = 0;
    for (size_t i = 0; i < S.n; i++) {
      p += S.lit_len[i];
      R->lit_bytes += S.lit_len[i];
      if (S.mlen[i]) {
        R->n_matches++;
        R->match_bytes += S.mlen[i];
        uint32_t d = S.off[i];
        if (d < 1 || d > I.window || d > p) R->offsets_ok = 0;
      }
      p += S.mlen[i];
    }
    /* weak DE property: no copy reads bytes that another copy of the same
       group writes (checked by running each group in one pass) */
    uint8_t* ref = (uint8_t*)malloc(ob ? ob : 1);
    uint64_t nn = 0;
    rc = ref ? lz77_decode(&S, I.window, ref, ob, &nn) : ORC_ERR_NOMEM;
    if (rc) { free(ref); seq_free(&S); R->first_error = rc; return rc; }
    mrr_stats dummy;
    memset(&dummy, 0, sizeof(dummy));
    if (mrr_block(&S, ob, 1, ref, &dummy, NULL) != 0) R->de_weak_ok = 0;
    if (mrr_block(&S, ob, 0, ref, &st, NULL) != 0) R->mrr_ok = 0;
    free(ref);
    R->n_seq += S.n;
    seq_free(&S);
  }
  R->groups = st.groups;
  R->rounds = st.rounds;
  R->max_rounds = st.max_rounds;
  R->copies = st.copies;
  memcpy(R->round_hist, st.hist, sizeof(st.hist));
  return 0;
}

/* MRR round counts of a plain token list treated as one block: rounds_out[g]
   receives the number of rounds of 32-sequence group g (0 for a group with
   no back-reference).  Fails if MRR (or, with de_single_pass, the one-pass
   DE schedule) would read a byte before it is available or would stall. */
int orc_mrr_rounds(const uint32_t* lit_len, const uint32_t* mlen, const uint32_t* off, uint64_t n_seq,
                   const uint8_t* lits, int de_single_pass, uint32_t* rounds_out, uint64_t* n_groups) {
  seqbuf S;
  uint64_t nl = 0, tot = 0;
  for (uint64_t i = 0; i < n_seq; i++) { nl += lit_len[i]; tot += lit_len[i] + mlen[i]; }
  if (tot > 0xFFFFFFFFull) return ORC_ERR_ARG;
  S.lit_len = (uint32_t*)lit_len;
  S.mlen = (uint32_t*)mlen;
  S.off = (uint32_t*)off;
  S.n = n_seq;
  S.cap = n_seq;
  S.lits = (uint8_t*)lits;
  S.nlits = nl;
  S.lits_cap = nl;
  uint8_t* ref = (uint8_t*)malloc(tot ? tot : 1);
  if (!ref) return ORC_ERR_NOMEM;
  uint64_t nn;
  int rc = lz77_decode(&S, 32768, ref, tot, &nn);
  mrr_stats st;
  memset(&st, 0, sizeof(st));
  if (!rc) rc = mrr_block(&S, (uint32_t)tot, de_single_pass, ref, &st, rounds_out);
  *n_groups = (n_seq + 31) / 32;
  free(ref);
  return rc;
}
