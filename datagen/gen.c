/*
 * Seeded synthetic inputs for the Gompresso-style decompression path.
 *
 * This file makes test and benchmark INPUTS only.  It holds none of the
 * codec's arithmetic (no LZ77 parsing, no Huffman coding, no decoding); both
 * the CPU oracle and the CUDA path are fed from here.
 *
 * Every random draw is a counter-based splitmix64 value: value(seed, i) =
 * mix64(seed + (i + 1) * 0x9E3779B97F4A7C15), where mix64 is the splitmix64
 * finaliser (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014).  Large inputs are produced in independent
 * 1 MiB chunks, each seeded by (seed, chunk index), so the bytes do not depend
 * on the number of threads used to make them.
 *
 * The paper measures on an English Wikipedia XML dump and a Matrix-Market CSV
 * file (Section 5).  Neither is available here; these generators stand in for
 * them with the same kind of structure: order-k byte Markov text with
 * English-like letter statistics, and CSV-like numeric records.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <stdlib.h>
#include <math.h>
#include <pthread.h>

#define GEN_CHUNK ((size_t)1 << 20)

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static inline uint64_t draw(uint64_t seed, uint64_t i) {
  return mix64(seed + (i + 1) * 0x9E3779B97F4A7C15ull);
}
/* uniform in [0, 1) with 53 bits */
static inline double unif(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* ------------------------------------------------------------------------ */
/* English-like unigram: a generic public letter-frequency table (percent of
 * letters), space at about 18 % of all characters, a little punctuation and a
 * newline, and a floor of noise spread over all 256 byte values (the 4096-
 * entry inverse CDF below keeps the values whose mass reaches its steps).    */
static const char  kLetters[] = "etaoinshrdlcumwfgypbvkjxqz";
static const double kLetterPct[26] = {12.7, 9.1, 8.2, 7.5, 7.0, 6.7, 6.3, 6.1, 6.0, 4.3, 4.0, 2.8, 2.8,
                                      2.4, 2.4, 2.2, 2.0, 2.0, 1.9, 1.5, 1.0, 0.8, 0.15, 0.15, 0.1, 0.07};
#define UNI_Q 4096 /* quantised inverse CDF */
static uint8_t g_uni[UNI_Q];
static pthread_once_t g_uni_once = PTHREAD_ONCE_INIT;

static void build_unigram(void) {
  double w[256];
  double letters = 0;
  for (int i = 0; i < 26; i++) letters += kLetterPct[i];
  for (int i = 0; i < 256; i++) w[i] = 0.015 / 256.0; /* noise floor: 1.5 % */
  w[' '] += 0.18;
  w['.'] += 0.010;
  w[','] += 0.010;
  w['\n'] += 0.005;
  double rest = 1.0 - 0.015 - 0.18 - 0.025;
  for (int i = 0; i < 26; i++) {
    double p = rest * kLetterPct[i] / letters;
    w[(uint8_t)kLetters[i]] += p * 0.96;          /* lower case */
    w[(uint8_t)(kLetters[i] - 'a' + 'A')] += p * 0.04; /* capitals */
  }
  double tot = 0;
  for (int i = 0; i < 256; i++) tot += w[i];
  double acc = 0;
  int b = 0;
  for (int q = 0; q < UNI_Q; q++) {
    double target = (q + 0.5) / UNI_Q * tot;
    while (b < 255 && acc + w[b] < target) { acc += w[b]; b++; }
    g_uni[q] = (uint8_t)b;
  }
}
static inline uint8_t unigram(uint64_t r) { return g_uni[r >> 52]; }

/* ------------------------------------------------------------------------ */
/* Order-k byte Markov text.  For context c (the previous k bytes), the next
 * byte is drawn from a mixture: with probability lambda from a peaked
 * distribution over 4..8 successors fixed by hash(seed, c) (successor i has
 * weight rho^i), otherwise from the unigram above.  lambda and rho are the
 * concentration knobs that set how repetitive (compressible) the text is.  */
typedef struct {
  uint8_t* out;
  size_t n;
  uint64_t seed;
  int order;
  double lambda, rho;
  size_t c0, c1;
} markov_job;

static void markov_chunk(uint8_t* out, size_t len, uint64_t seed, int order, double lambda, double rho,
                         uint64_t chunk) {
  uint64_t cs = mix64(seed ^ (0xC2B2AE3D27D4EB4Full * (chunk + 1)));
  uint32_t ctx = 0x20202020u; /* spaces */
  uint32_t mask = order >= 4 ? 0xFFFFFFFFu : ((1u << (8 * order)) - 1u);
  uint64_t ctr = 0;
  for (size_t i = 0; i < len; i++) {
    uint32_t c = ctx & mask;
    uint64_t r = draw(cs, ctr++);
    uint8_t b;
    if (unif(r) < lambda) {
      uint64_t h = mix64(seed * 0x9E3779B97F4A7C15ull + c + 0x632BE59BD9B4E019ull);
      int nsucc = 4 + (int)(h % 5);
      /* pick successor i with weight rho^i (renormalised over nsucc) */
      uint64_t r2 = draw(cs, ctr++);
      double tot = (1.0 - pow(rho, nsucc)) / (1.0 - rho);
      double u = unif(r2) * tot;
      int k = 0;
      double w = 1.0, acc = 1.0;
      while (k < nsucc - 1 && u >= acc) { k++; w *= rho; acc += w; }
      b = unigram(mix64(h + 0x1000193ull * (uint64_t)(k + 1)));
    } else {
      b = unigram(draw(cs, ctr++));
    }
    out[i] = b;
    ctx = (ctx << 8) | b;
  }
}

static void* markov_worker(void* arg) {
  markov_job* j = (markov_job*)arg;
  for (size_t c = j->c0; c < j->c1; c++) {
    size_t off = c * GEN_CHUNK;
    size_t len = j->n - off < GEN_CHUNK ? j->n - off : GEN_CHUNK;
    markov_chunk(j->out + off, len, j->seed, j->order, j->lambda, j->rho, c);
  }
  return NULL;
}

typedef void* (*worker_fn)(void*);

static void run_chunks(void* jobs, size_t job_size, size_t nchunks, int nthreads, worker_fn fn,
                       size_t off_c0, size_t off_c1) {
  if (nthreads < 1) nthreads = 1;
  if ((size_t)nthreads > nchunks) nthreads = (int)(nchunks ? nchunks : 1);
  pthread_t th[256];
  if (nthreads > 256) nthreads = 256;
  for (int t = 0; t < nthreads; t++) {
    char* j = (char*)jobs + (size_t)t * job_size;
    *(size_t*)(j + off_c0) = nchunks * t / nthreads;
    *(size_t*)(j + off_c1) = nchunks * (t + 1) / nthreads;
  }
  for (int t = 1; t < nthreads; t++) pthread_create(&th[t], NULL, fn, (char*)jobs + (size_t)t * job_size);
  fn(jobs);
  for (int t = 1; t < nthreads; t++) pthread_join(th[t], NULL);
}

int gen_markov_text(uint8_t* out, size_t n, uint64_t seed, int order, double lambda, double rho, int nthreads) {
  if (order < 1 || order > 4 || lambda < 0 || lambda > 1 || rho <= 0 || rho >= 1) return -1;
  pthread_once(&g_uni_once, build_unigram);
  size_t nchunks = (n + GEN_CHUNK - 1) / GEN_CHUNK;
  if (nchunks == 0) return 0;
  markov_job jobs[256];
  for (int t = 0; t < 256; t++) {
    jobs[t].out = out; jobs[t].n = n; jobs[t].seed = seed; jobs[t].order = order; jobs[t].lambda = lambda; jobs[t].rho = rho;
  }
  run_chunks(jobs, sizeof(markov_job), nchunks, nthreads, markov_worker, offsetof(markov_job, c0),
             offsetof(markov_job, c1));
  return 0;
}

/* ------------------------------------------------------------------------ */
/* CSV-like numeric records: 8 fields per row,
 *   id1,id2         Zipf(s) over ranks 1..999999 (the id is the rank)
 *   price1,price2   uniform cents in [1, 999999], printed %d.%02d
 *   date1,date2     uniform day in 2015-01-01 .. 2019-12-31, YYYY-MM-DD
 *   cat1,cat2       one of 20 seeded tokens (4..12 lower-case letters), Zipf(s)
 * ',' between fields and '\n' after each row.  With probability p_repeat a
 * row repeats one of the last 64 rows with one field resampled, which gives
 * long and chained back-references.                                          */
#define ZIPF_N 999999
static double* g_zipf_cdf = NULL;
static double g_zipf_s = -1;
static pthread_mutex_t g_zipf_mu = PTHREAD_MUTEX_INITIALIZER;

static const double* zipf_table(double s) {
  pthread_mutex_lock(&g_zipf_mu);
  if (!g_zipf_cdf || g_zipf_s != s) {
    if (!g_zipf_cdf) g_zipf_cdf = (double*)malloc(sizeof(double) * ZIPF_N);
    double acc = 0;
    for (int k = 1; k <= ZIPF_N; k++) { acc += pow((double)k, -s); g_zipf_cdf[k - 1] = acc; }
    for (int k = 0; k < ZIPF_N; k++) g_zipf_cdf[k] /= acc;
    g_zipf_s = s;
  }
  pthread_mutex_unlock(&g_zipf_mu);
  return g_zipf_cdf;
}
static int zipf_pick(const double* cdf, int n, double u) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (cdf[mid] > u) hi = mid; else lo = mid + 1;
  }
  return lo + 1;
}

typedef struct {
  char tok[20][13];
  double tok_cdf[20];
  const double* id_cdf;
} csv_tables;

static void days_to_ymd(int z, int* y, int* m, int* d) {
  /* civil date from days since 1970-01-01 (proleptic Gregorian) */
  z += 719468;
  int era = (z >= 0 ? z : z - 146096) / 146097;
  unsigned doe = (unsigned)(z - era * 146097);
  unsigned yoe = (doe - doe / 1460 + doe / 36524 - doe / 146096) / 365;
  int yy = (int)yoe + era * 400;
  unsigned doy = doe - (365 * yoe + yoe / 4 - yoe / 100);
  unsigned mp = (5 * doy + 2) / 153;
  unsigned dd = doy - (153 * mp + 2) / 5 + 1;
  unsigned mm = mp < 10 ? mp + 3 : mp - 9;
  *y = yy + (mm <= 2);
  *m = (int)mm;
  *d = (int)dd;
}

static int put_uint(char* p, unsigned v) {
  char tmp[12];
  int n = 0;
  do { tmp[n++] = (char)('0' + v % 10); v /= 10; } while (v);
  for (int i = 0; i < n; i++) p[i] = tmp[n - 1 - i];
  return n;
}

typedef struct { unsigned v[8]; } csv_row;

static unsigned csv_field(const csv_tables* T, int f, uint64_t r) {
  double u = unif(r);
  switch (f >> 1) {
    case 0: return (unsigned)zipf_pick(T->id_cdf, ZIPF_N, u);
    case 1: return 1u + (unsigned)(u * 999999.0);
    case 2: return 16436u + (unsigned)(u * 1826.0); /* 2015-01-01 is day 16436 */
    default: return (unsigned)(zipf_pick(T->tok_cdf, 20, u) - 1);
  }
}

static int csv_print(const csv_tables* T, const csv_row* row, char* p) {
  int n = 0;
  for (int f = 0; f < 8; f++) {
    unsigned v = row->v[f];
    switch (f >> 1) {
      case 0: n += put_uint(p + n, v); break;
      case 1: {
        n += put_uint(p + n, v / 100);
        p[n++] = '.';
        p[n++] = (char)('0' + (v % 100) / 10);
        p[n++] = (char)('0' + v % 10);
        break;
      }
      case 2: {
        int y, m, d;
        days_to_ymd((int)v, &y, &m, &d);
        n += put_uint(p + n, (unsigned)y);
        p[n++] = '-';
        p[n++] = (char)('0' + m / 10); p[n++] = (char)('0' + m % 10);
        p[n++] = '-';
        p[n++] = (char)('0' + d / 10); p[n++] = (char)('0' + d % 10);
        break;
      }
      default: {
        const char* t = T->tok[v];
        size_t l = strlen(t);
        memcpy(p + n, t, l);
        n += (int)l;
      }
    }
    p[n++] = (f == 7) ? '\n' : ',';
  }
  return n;
}

typedef struct {
  uint8_t* out;
  size_t n;
  uint64_t seed;
  double p_repeat;
  const csv_tables* T;
  size_t c0, c1;
} csv_job;

static void csv_chunk(uint8_t* out, size_t len, uint64_t seed, double p_repeat, const csv_tables* T,
                      uint64_t chunk) {
  uint64_t cs = mix64(seed ^ (0x165667B19E3779F9ull * (chunk + 1)));
  uint64_t ctr = 0;
  csv_row hist[64];
  int nh = 0, hpos = 0;
  size_t pos = 0;
  char line[256];
  while (pos < len) {
    csv_row row;
    if (nh > 0 && unif(draw(cs, ctr++)) < p_repeat) {
      int back = (int)(draw(cs, ctr++) % (uint64_t)nh);
      row = hist[(hpos - 1 - back + 64) & 63];
      int f = (int)(draw(cs, ctr++) % 8u);
      row.v[f] = csv_field(T, f, draw(cs, ctr++));
    } else {
      for (int f = 0; f < 8; f++) row.v[f] = csv_field(T, f, draw(cs, ctr++));
    }
    hist[hpos] = row;
    hpos = (hpos + 1) & 63;
    if (nh < 64) nh++;
    int l = csv_print(T, &row, line);
    size_t take = (size_t)l < len - pos ? (size_t)l : len - pos;
    memcpy(out + pos, line, take);
    pos += take;
  }
}

static void* csv_worker(void* arg) {
  csv_job* j = (csv_job*)arg;
  for (size_t c = j->c0; c < j->c1; c++) {
    size_t off = c * GEN_CHUNK;
    size_t len = j->n - off < GEN_CHUNK ? j->n - off : GEN_CHUNK;
    csv_chunk(j->out + off, len, j->seed, j->p_repeat, j->T, c);
  }
  return NULL;
}

int gen_csv_records(uint8_t* out, size_t n, uint64_t seed, double zipf_s, double p_repeat, int nthreads) {
  if (zipf_s <= 0 || p_repeat < 0 || p_repeat > 1) return -1;
  csv_tables T;
  T.id_cdf = zipf_table(zipf_s);
  /* 20 categorical tokens of 4..12 lower-case letters, fixed by the seed */
  uint64_t ts = mix64(seed ^ 0xA0761D6478BD642Full);
  double acc = 0;
  for (int t = 0; t < 20; t++) {
    int l = 4 + (int)(draw(ts, 100 + t) % 9u);
    for (int i = 0; i < l; i++) T.tok[t][i] = (char)('a' + draw(ts, 1000 + 16 * t + i) % 26u);
    T.tok[t][l] = 0;
    acc += pow((double)(t + 1), -zipf_s);
    T.tok_cdf[t] = acc;
  }
  for (int t = 0; t < 20; t++) T.tok_cdf[t] /= acc;
  size_t nchunks = (n + GEN_CHUNK - 1) / GEN_CHUNK;
  if (nchunks == 0) return 0;
  csv_job jobs[256];
  for (int t = 0; t < 256; t++) {
    jobs[t].out = out; jobs[t].n = n; jobs[t].seed = seed; jobs[t].p_repeat = p_repeat; jobs[t].T = &T;
  }
  run_chunks(jobs, sizeof(csv_job), nchunks, nthreads, csv_worker, offsetof(csv_job, c0),
             offsetof(csv_job, c1));
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Nesting-depth token streams (Section 5.1, the artificial data sets of the
 * MRR experiment).  A 16-byte string is repeated; each repetition changes one
 * byte, alternately the first and the last one, and is preceded by a
 * separator byte drawn from a set disjoint from the string's bytes ('0'..'9'
 * against 'a'..'z').  With m interleaved strings (m = 1, 2, 4, ...) every
 * back-reference copies 15 bytes from the previous instance of its own
 * string, m sequences earlier, so a group of 32 sequences holds chains of
 * 32/m back-references that each depend on the one before.
 *
 * The token stream is emitted directly, so its nesting depth does not depend
 * on any compressor's parse.  Instance k occupies 17 bytes (separator, then
 * the string).  Instances 0..m-1 form a prelude written as literals of the
 * first sequence; instances m .. m+n_inst-1 each end one sequence with a
 * 15-byte back-reference at distance 17m.  When the last byte changed, the new
 * byte follows the copy and becomes the first literal of the next sequence;
 * a trailing literal-only sequence (match length 0) holds it at the end.
 * The decoded size is 17 * (m + n_inst) bytes.                               */
int gen_nesting_tokens(uint64_t seed, int m, size_t n_inst, uint32_t* lit_len, uint32_t* mlen,
                       uint32_t* off, size_t seq_cap, uint8_t* lits, size_t lits_cap,
                       size_t* n_seq, size_t* n_lits) {
  if (m < 1 || m > 32) return -1;
  uint8_t cur[32][16];
  uint64_t ctr = 0;
  for (int s = 0; s < m; s++)
    for (int i = 0; i < 16; i++) cur[s][i] = (uint8_t)('a' + draw(seed, ctr++) % 26u);
  size_t nl = 0, q = 0;
  uint32_t ll = 0;
#define PUT(b) do { if (nl >= lits_cap) return -2; lits[nl++] = (uint8_t)(b); ll++; } while (0)
  for (int s = 0; s < m; s++) {
    PUT('0' + draw(seed, ctr++) % 10u);
    for (int i = 0; i < 16; i++) PUT(cur[s][i]);
  }
  for (size_t k = (size_t)m; k < (size_t)m + n_inst; k++) {
    int s = (int)(k % (size_t)m);
    int first = (int)((k / (size_t)m) & 1u);
    int pos = first ? 0 : 15;
    uint8_t nb;
    do { nb = (uint8_t)('a' + draw(seed, ctr++) % 26u); } while (nb == cur[s][pos]);
    cur[s][pos] = nb;
    PUT('0' + draw(seed, ctr++) % 10u);
    if (first) PUT(cur[s][0]);
    if (q >= seq_cap) return -3;
    lit_len[q] = ll; mlen[q] = 15; off[q] = (uint32_t)(17 * m); q++;
    ll = 0;
    if (!first) PUT(cur[s][15]);
  }
  if (ll > 0) {
    if (q >= seq_cap) return -3;
    lit_len[q] = ll; mlen[q] = 0; off[q] = 0; q++;
  }
#undef PUT
  *n_seq = q;
  *n_lits = nl;
  return 0;
}
