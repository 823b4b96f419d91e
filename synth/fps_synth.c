/*
 * Seeded synthetic MACCS-166-like fingerprints.
 *
 * This module makes inputs only: it holds none of the search method's
 * arithmetic (no distance, no ranking).  It stands in for the PubChem MACCS
 * library of the paper (Sec. 4.1-4.2: ~95.4 M molecules, 166 keys each),
 * which is not available here.
 *
 * Recipe (all draws are counter-based, so the output does not depend on the
 * thread count or on the order records are produced in):
 *   - a "chemistry" vector p_j, j = 1..165, p_j ~ Beta(0.5, 2), drawn once
 *     from the chemistry seed; key 0 is always 0 (p_0 = 0).
 *     Beta(a, b) = X / (X + Y) with X ~ Gamma(0.5) = Z^2/2 (Z standard normal
 *     from Box-Muller) and Y ~ Gamma(2) = -ln(U1 U2).  p_j is rounded to a
 *     multiple of 2^-20 so that libm differences between hosts cannot change
 *     a single record bit;
 *   - record i of a library with record seed s: bit j = [u(s, i, j) < p_j];
 *   - 1 % planted near-duplicates: a record whose hash says so copies a
 *     uniformly chosen earlier record and flips m ~ U{1..5} distinct bits
 *     among positions 1..165.
 * The random source is SplitMix64: state = mix(seed) + counter * gamma,
 * output = the SplitMix64 finaliser of the state.
 *
 * Bit order of the packed form: character j of the text line is word j/64,
 * bit j%64 (LSB first); bits 166..191 are zero.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SYN_BITS 166
#define SYN_WORDS 3

static inline uint64_t sm_final(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* One 64-bit draw for (seed, record, slot); slot < 4096. */
static inline uint64_t draw(uint64_t seed, uint64_t rec, uint64_t slot) {
  uint64_t key = sm_final(seed + 0x6A09E667F3BCC909ULL);
  uint64_t ctr = (rec << 12) | (slot & 0xFFFULL);
  return sm_final(key + (ctr + 1) * 0x9E3779B97F4A7C15ULL);
}

static inline double unit_open(uint64_t h) { /* (0, 1] */
  return ((double)(h >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}

/* Thresholds T_j: bit j is set iff the high 32 bits of its draw are < T_j. */
void synth_thresholds(uint64_t chem_seed, uint32_t* T /* 166 */, double* p /* 166, nullable */) {
  const double two_pi = 6.283185307179586476925286766559;
  T[0] = 0;
  if (p) p[0] = 0.0;
  for (int j = 1; j < SYN_BITS; ++j) {
    double u1 = unit_open(draw(chem_seed, 0xFFFFFFull, 4 * j + 0));
    double u2 = unit_open(draw(chem_seed, 0xFFFFFFull, 4 * j + 1));
    double u3 = unit_open(draw(chem_seed, 0xFFFFFFull, 4 * j + 2));
    double u4 = unit_open(draw(chem_seed, 0xFFFFFFull, 4 * j + 3));
    double z = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
    double x = 0.5 * z * z;
    double y = -log(u3 * u4);
    double pj = (x + y) > 0.0 ? x / (x + y) : 0.0;
    double q = floor(pj * 1048576.0 + 0.5);         /* multiple of 2^-20 */
    if (q >= 1048576.0) q = 1048575.0;
    if (q < 0.0) q = 0.0;
    T[j] = (uint32_t)q << 12;
    if (p) p[j] = q / 1048576.0;
  }
}

/* Planting decision and its parameters for record i. */
int synth_planted(uint64_t seed, uint64_t i, uint64_t* src, int* m, int* pos /* >= 5 */) {
  if (i == 0) return 0;
  if (draw(seed, i, 1000) % 100ULL != 0ULL) return 0;
  if (src) *src = draw(seed, i, 1001) % i;
  int mm = 1 + (int)(draw(seed, i, 1002) % 5ULL);
  if (m) *m = mm;
  if (pos) {
    int got = 0;
    for (uint64_t t = 0; got < mm; ++t) {
      int cand = 1 + (int)(draw(seed, i, 1003 + t) % 165ULL);
      int dup = 0;
      for (int a = 0; a < got; ++a) dup |= (pos[a] == cand);
      if (!dup) pos[got++] = cand;
    }
  }
  return 1;
}

static void gen_record(const uint32_t* T, uint64_t seed, uint64_t i, uint64_t w[SYN_WORDS]) {
  uint64_t src;
  int m, pos[5];
  if (synth_planted(seed, i, &src, &m, pos)) {
    gen_record(T, seed, src, w);
    for (int a = 0; a < m; ++a) w[pos[a] >> 6] ^= 1ULL << (pos[a] & 63);
    return;
  }
  w[0] = w[1] = w[2] = 0;
  for (int s = 0; s < 83; ++s) {          /* two keys per draw: j = 2s+1, 2s+2 */
    uint64_t h = draw(seed, i, (uint64_t)s);
    int j0 = 2 * s + 1, j1 = 2 * s + 2;
    if ((uint32_t)(h & 0xFFFFFFFFu) < T[j0]) w[j0 >> 6] |= 1ULL << (j0 & 63);
    if (j1 < SYN_BITS && (uint32_t)(h >> 32) < T[j1]) w[j1 >> 6] |= 1ULL << (j1 & 63);
  }
}

typedef struct {
  const uint32_t* T;
  uint64_t seed, start, begin, end;
  uint64_t* packed;
  char* text;
} job_t;

static void* run_job(void* arg) {
  job_t* jb = (job_t*)arg;
  for (uint64_t r = jb->begin; r < jb->end; ++r) {
    uint64_t w[SYN_WORDS];
    gen_record(jb->T, jb->seed, jb->start + r, w);
    if (jb->packed) memcpy(jb->packed + 3 * r, w, sizeof w);
    if (jb->text) {
      char* line = jb->text + (size_t)r * (SYN_BITS + 1);
      for (int j = 0; j < SYN_BITS; ++j) line[j] = (char)('0' + ((w[j >> 6] >> (j & 63)) & 1ULL));
      line[SYN_BITS] = '\n';
    }
  }
  return NULL;
}

static void run_parallel(const uint32_t* T, uint64_t seed, uint64_t start, uint64_t n, int nthreads,
                         uint64_t* packed, char* text) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((uint64_t)nthreads > n) nthreads = n ? (int)n : 1;
  pthread_t th[256];
  int started[256];
  job_t jobs[256];
  uint64_t chunk = (n + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    uint64_t b = chunk * t, e = b + chunk;
    if (b > n) b = n;
    if (e > n) e = n;
    jobs[t] = (job_t){T, seed, start, b, e, packed, text};
    started[t] = nthreads > 1 && pthread_create(&th[t], NULL, run_job, &jobs[t]) == 0;
    if (!started[t]) run_job(&jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t)
    if (started[t]) pthread_join(th[t], NULL);
}

/* Records [start, start+n) of library `seed` under chemistry `chem_seed`, packed 3 words each. */
void synth_packed(uint64_t chem_seed, uint64_t seed, uint64_t start, uint64_t n, int nthreads, uint64_t* out) {
  uint32_t T[SYN_BITS];
  synth_thresholds(chem_seed, T, NULL);
  run_parallel(T, seed, start, n, nthreads, out, NULL);
}

/* Same records as text: n lines of 166 '0'/'1' characters plus '\n' (167 bytes each). */
void synth_text(uint64_t chem_seed, uint64_t seed, uint64_t start, uint64_t n, int nthreads, char* out) {
  uint32_t T[SYN_BITS];
  synth_thresholds(chem_seed, T, NULL);
  run_parallel(T, seed, start, n, nthreads, NULL, out);
}

/* Records chosen by index (e.g. queries sampled from library entries). */
void synth_packed_at(uint64_t chem_seed, uint64_t seed, const uint64_t* idx, uint64_t n, uint64_t* out) {
  uint32_t T[SYN_BITS];
  synth_thresholds(chem_seed, T, NULL);
  for (uint64_t r = 0; r < n; ++r) gen_record(T, seed, idx[r], out + 3 * r);
}

/* A raw uniform 64-bit draw, for seeded choices made by callers (query picks, k mixes, arrivals). */
uint64_t synth_draw(uint64_t seed, uint64_t rec, uint64_t slot) { return draw(seed, rec, slot); }

/* ------------------------------------------------------------------ wide
 * Longer fingerprints (n_bits up to 4096, W = ceil(n_bits / 64) words, bits
 * past n_bits zero), for the n-bit / Tanimoto search.  Same SplitMix64 draws;
 * the density is that of hashed circular fingerprints rather than MACCS keys:
 *   - p_j ~ Beta(0.5, 8) for every bit j (mean ~ 0.059), rounded to 2^-20:
 *     X = Z^2/2 (Z from Box-Muller), Y = -ln(U1 ... U8), p = X / (X + Y), the
 *     ten uniforms of bit j drawn from the chemistry seed at record
 *     0xFFFFF0 - (j >> 8), slots 16 (j & 255) .. +9;
 *   - record i: bit j = [32-bit half (j & 1) of draw(seed, i, j >> 1) < T_j];
 *   - 1 % planted near-duplicates (decision slot 3000, source 3001, count
 *     3002, positions 3003...): a copy of an earlier record with m ~ U{1..5}
 *     distinct bits flipped anywhere in [0, n_bits). */
#define WIDE_MAX_BITS 4096

void synth_wide_thresholds(uint64_t chem_seed, int n_bits, uint32_t* T) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int j = 0; j < n_bits; ++j) {
    const uint64_t rec = 0xFFFFF0ull - (uint64_t)(j >> 8), sl = 16 * (uint64_t)(j & 255);
    double u1 = unit_open(draw(chem_seed, rec, sl + 0));
    double u2 = unit_open(draw(chem_seed, rec, sl + 1));
    double y = 0.0;
    for (int t = 0; t < 8; ++t) y -= log(unit_open(draw(chem_seed, rec, sl + 2 + (uint64_t)t)));
    double z = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
    double x = 0.5 * z * z;
    double pj = (x + y) > 0.0 ? x / (x + y) : 0.0;
    double q = floor(pj * 1048576.0 + 0.5);
    if (q >= 1048576.0) q = 1048575.0;
    if (q < 0.0) q = 0.0;
    T[j] = (uint32_t)q << 12;
  }
}

static void gen_wide(const uint32_t* T, int n_bits, uint64_t seed, uint64_t i, uint64_t* w) {
  const int W = (n_bits + 63) / 64;
  if (i > 0 && draw(seed, i, 3000) % 100ULL == 0ULL) {
    gen_wide(T, n_bits, seed, draw(seed, i, 3001) % i, w);
    const int m = 1 + (int)(draw(seed, i, 3002) % 5ULL);
    int pos[5], got = 0;
    for (uint64_t t = 0; got < m; ++t) {
      int cand = (int)(draw(seed, i, 3003 + t) % (uint64_t)n_bits);
      int dup = 0;
      for (int a = 0; a < got; ++a) dup |= (pos[a] == cand);
      if (!dup) pos[got++] = cand;
    }
    for (int a = 0; a < m; ++a) w[pos[a] >> 6] ^= 1ULL << (pos[a] & 63);
    return;
  }
  for (int a = 0; a < W; ++a) w[a] = 0;
  for (int s = 0; 2 * s < n_bits; ++s) {
    uint64_t h = draw(seed, i, (uint64_t)s);
    int j0 = 2 * s, j1 = 2 * s + 1;
    if ((uint32_t)(h & 0xFFFFFFFFu) < T[j0]) w[j0 >> 6] |= 1ULL << (j0 & 63);
    if (j1 < n_bits && (uint32_t)(h >> 32) < T[j1]) w[j1 >> 6] |= 1ULL << (j1 & 63);
  }
}

typedef struct {
  const uint32_t* T;
  int n_bits;
  uint64_t seed, start, begin, end;
  uint64_t* packed;
  char* text;
} wjob_t;

static void* run_wjob(void* arg) {
  wjob_t* jb = (wjob_t*)arg;
  const int W = (jb->n_bits + 63) / 64;
  uint64_t w[WIDE_MAX_BITS / 64];
  for (uint64_t r = jb->begin; r < jb->end; ++r) {
    gen_wide(jb->T, jb->n_bits, jb->seed, jb->start + r, w);
    if (jb->packed) memcpy(jb->packed + (size_t)W * r, w, sizeof(uint64_t) * W);
    if (jb->text) {
      char* line = jb->text + (size_t)r * (jb->n_bits + 1);
      for (int j = 0; j < jb->n_bits; ++j) line[j] = (char)('0' + ((w[j >> 6] >> (j & 63)) & 1ULL));
      line[jb->n_bits] = '\n';
    }
  }
  return NULL;
}

/* Records [start, start+n) of wide library `seed`: packed (W words each) and/or text (n_bits + 1 bytes each).
   Returns 0, or -1 if n_bits is outside 1..4096. */
int synth_wide(uint64_t chem_seed, uint64_t seed, uint64_t start, uint64_t n, int n_bits, int nthreads,
               uint64_t* packed, char* text) {
  if (n_bits < 1 || n_bits > WIDE_MAX_BITS) return -1;
  uint32_t* T = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n_bits);
  if (!T) return -1;
  synth_wide_thresholds(chem_seed, n_bits, T);
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((uint64_t)nthreads > n) nthreads = n ? (int)n : 1;
  pthread_t th[256];
  int started[256];
  wjob_t jobs[256];
  uint64_t chunk = (n + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    uint64_t b = chunk * t, e = b + chunk;
    if (b > n) b = n;
    if (e > n) e = n;
    jobs[t] = (wjob_t){T, n_bits, seed, start, b, e, packed, text};
    started[t] = nthreads > 1 && pthread_create(&th[t], NULL, run_wjob, &jobs[t]) == 0;
    if (!started[t]) run_wjob(&jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t)
    if (started[t]) pthread_join(th[t], NULL);
  free(T);
  return 0;
}

/* Wide records chosen by index. */
int synth_wide_at(uint64_t chem_seed, uint64_t seed, const uint64_t* idx, uint64_t n, int n_bits, uint64_t* out) {
  if (n_bits < 1 || n_bits > WIDE_MAX_BITS) return -1;
  uint32_t* T = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n_bits);
  if (!T) return -1;
  synth_wide_thresholds(chem_seed, n_bits, T);
  const int W = (n_bits + 63) / 64;
  for (uint64_t r = 0; r < n; ++r) gen_wide(T, n_bits, seed, idx[r], out + (size_t)W * r);
  free(T);
  return 0;
}
