/*
 * CPU oracle for FPScreen's similarity search -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline /
 * reference legs may call this code.  The CUDA search path never links,
 * imports or runs it, and it shares no code with that path.
 *
 * What it computes is the plain definition of the paper's search
 * (Sec. 4.3, the Manhattan formula and the six steps of Fig. 3):
 *   1. read every molecule of library text F and its CID (Fig. 3 step 1);
 *   2. take the target fingerprint b (step 2);
 *   3-4. for each library row i, K_i = sum_j |A_ij - b_j| over the n = 166
 *      keys (Sec. 4.3 formula; steps 3-4).  The oracle evaluates |a - b| on
 *      the '0'/'1' characters themselves: one term is 1 iff the characters
 *      differ;
 *   5. pair each K_i with its row (step 5);
 *   6. sort all pairs ascending and take the first k (step 6; Fig. 2 lists
 *      results "in ascending order of distance").
 * Several libraries searched separately are combined by concatenating their
 * result lists and sorting again (the text after Fig. 3).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - ties in distance are ordered by ascending 0-based line index, which makes
 *     the result unique;
 *   - the query itself, if present in the library, is returned at distance 0
 *     (Fig. 2 and Sec. 3.3 return the query CID at 0.0);
 *   - k > N returns all N rows; k = 0 returns nothing;
 *   - a line is either 166 '0'/'1' characters, or "<cid><sep><166 bits>" with
 *     sep one of space, tab or comma; a trailing '\r' is dropped; with
 *     ORACLE_ACCEPT_167 a 167-character line whose first character is '0' loses
 *     that character.  Any other line is a parse error (1-based line number
 *     reported).  Without a CID column the CID is the 0-based line index.
 *
 * The distance step may run on several threads over contiguous row ranges;
 * the sort is a single full qsort of all (distance, index) pairs.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_BITS 166
#define ORACLE_OK 0
#define ORACLE_ERR_ARG 1
#define ORACLE_ERR_PARSE 3
#define ORACLE_ERR_NOMEM 9
#define ORACLE_ACCEPT_167 1u

typedef struct {
  const char** bits;  /* pointer to the 166 key characters of each row */
  int64_t* cid;
  int64_t n;
} rows_t;

static void rows_free(rows_t* r) {
  free(r->bits);
  free(r->cid);
  r->bits = NULL;
  r->cid = NULL;
  r->n = 0;
}

static int all01(const char* s, int64_t len) {
  for (int64_t j = 0; j < len; ++j)
    if (s[j] != '0' && s[j] != '1') return 0;
  return 1;
}

/* Fig. 3 step 1: every line of F becomes one row (key characters + CID). */
static int parse_rows(const char* text, size_t len, unsigned flags, rows_t* out, int64_t* err_line) {
  int64_t lines = 0;
  for (size_t p = 0; p < len; ++p) lines += text[p] == '\n';
  if (len && text[len - 1] != '\n') lines += 1;
  out->n = 0;
  out->bits = (const char**)malloc(sizeof(char*) * (size_t)(lines ? lines : 1));
  out->cid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(lines ? lines : 1));
  if (!out->bits || !out->cid) {
    rows_free(out);
    return ORACLE_ERR_NOMEM;
  }
  size_t p = 0;
  int64_t line_no = 0;
  while (p < len) {
    size_t e = p;
    while (e < len && text[e] != '\n') ++e;
    ++line_no;
    const char* s = text + p;
    int64_t L = (int64_t)(e - p);
    if (L > 0 && s[L - 1] == '\r') --L;
    const char* bits = NULL;
    int64_t cid = out->n;
    if (L == OR_BITS && all01(s, L)) {
      bits = s;
    } else if (L == OR_BITS + 1 && (flags & ORACLE_ACCEPT_167) && s[0] == '0' && all01(s, L)) {
      bits = s + 1;
    } else {
      int64_t sep = -1;
      for (int64_t j = 0; j < L; ++j)
        if (s[j] == ' ' || s[j] == '\t' || s[j] == ',') { sep = j; break; }
      if (sep > 0 && L - sep - 1 == OR_BITS && all01(s + sep + 1, OR_BITS)) {
        int ok = 1;
        int64_t v = 0;
        for (int64_t j = 0; j < sep; ++j) {
          if (s[j] < '0' || s[j] > '9' || v > (INT64_MAX - 9) / 10) { ok = 0; break; }
          v = v * 10 + (s[j] - '0');
        }
        if (ok) {
          bits = s + sep + 1;
          cid = v;
        }
      }
    }
    if (!bits) {
      if (err_line) *err_line = line_no;
      rows_free(out);
      return ORACLE_ERR_PARSE;
    }
    out->bits[out->n] = bits;
    out->cid[out->n] = cid;
    out->n += 1;
    p = e + 1;
  }
  return ORACLE_OK;
}

/* Sec. 4.3: dist_man = sum over the 166 keys of |a_j - b_j|, with a_j, b_j in {0, 1}. */
static int32_t manhattan(const char* a, const char* b) {
  int32_t s = 0;
  for (int j = 0; j < OR_BITS; ++j) {
    int aj = a[j] - '0', bj = b[j] - '0';
    s += aj > bj ? aj - bj : bj - aj;
  }
  return s;
}

typedef struct {
  const rows_t* rows;
  const char* q;
  int32_t* d;
  int64_t lo, hi;
} dist_job_t;

static void* dist_job(void* arg) {
  dist_job_t* jb = (dist_job_t*)arg;
  for (int64_t i = jb->lo; i < jb->hi; ++i) jb->d[i] = manhattan(jb->rows->bits[i], jb->q);
  return NULL;
}

static void all_distances(const rows_t* rows, const char* q, int nthreads, int32_t* d) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (rows->n < 4096) nthreads = 1;
  pthread_t th[256];
  int started[256];
  dist_job_t jobs[256];
  int64_t chunk = (rows->n + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    int64_t lo = chunk * t, hi = lo + chunk;
    if (lo > rows->n) lo = rows->n;
    if (hi > rows->n) hi = rows->n;
    jobs[t] = (dist_job_t){rows, q, d, lo, hi};
    started[t] = nthreads > 1 && pthread_create(&th[t], NULL, dist_job, &jobs[t]) == 0;
    if (!started[t]) dist_job(&jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t)
    if (started[t]) pthread_join(th[t], NULL);
}

/* Fig. 3 step 5: the (distance, row) pair; step 6 orders pairs by distance, then row. */
typedef struct {
  int32_t d;
  int32_t i;
} pair_t;

static int pair_cmp(const void* a, const void* b) {
  const pair_t* x = (const pair_t*)a;
  const pair_t* y = (const pair_t*)b;
  if (x->d != y->d) return x->d < y->d ? -1 : 1;
  if (x->i != y->i) return x->i < y->i ? -1 : 1;
  return 0;
}

static int query_ok(const char* q) {
  if (!q) return 0;
  for (int j = 0; j < OR_BITS; ++j)
    if (q[j] != '0' && q[j] != '1') return 0;
  return 1;
}

static int topk_rows(const rows_t* rows, const char* q, int64_t k, int nthreads, int32_t* out_idx,
                     int32_t* out_dist, int64_t* out_cid, int64_t* out_n) {
  if (!query_ok(q) || k < 0) return ORACLE_ERR_ARG;
  int64_t n = rows->n;
  int32_t* d = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
  pair_t* pr = (pair_t*)malloc(sizeof(pair_t) * (size_t)(n ? n : 1));
  if (!d || !pr) {
    free(d);
    free(pr);
    return ORACLE_ERR_NOMEM;
  }
  all_distances(rows, q, nthreads, d);
  for (int64_t i = 0; i < n; ++i) pr[i] = (pair_t){d[i], (int32_t)i};
  qsort(pr, (size_t)n, sizeof(pair_t), pair_cmp);
  int64_t m = k < n ? k : n;
  for (int64_t r = 0; r < m; ++r) {
    out_idx[r] = pr[r].i;
    out_dist[r] = pr[r].d;
    if (out_cid) out_cid[r] = rows->cid[pr[r].i];
  }
  *out_n = m;
  free(d);
  free(pr);
  return ORACLE_OK;
}

/* Number of rows of a library text, or a parse error with its 1-based line. */
int oracle_count(const char* text, size_t len, unsigned flags, int64_t* out_n, int64_t* err_line) {
  rows_t rows = {0};
  int st = parse_rows(text, len, flags, &rows, err_line);
  if (st == ORACLE_OK) *out_n = rows.n;
  rows_free(&rows);
  return st;
}

/* K_i for every row i (Fig. 3 steps 3-4). out_d holds N entries. */
int oracle_distances(const char* text, size_t len, unsigned flags, const char* query, int nthreads,
                     int32_t* out_d, int64_t cap, int64_t* out_n, int64_t* err_line) {
  if (!query_ok(query)) return ORACLE_ERR_ARG;
  rows_t rows = {0};
  int st = parse_rows(text, len, flags, &rows, err_line);
  if (st != ORACLE_OK) return st;
  if (rows.n > cap) {
    rows_free(&rows);
    return ORACLE_ERR_ARG;
  }
  all_distances(&rows, query, nthreads, out_d);
  *out_n = rows.n;
  rows_free(&rows);
  return ORACLE_OK;
}

/* CIDs of every row (step 1 "construct CID"). */
int oracle_cids(const char* text, size_t len, unsigned flags, int64_t* out_cid, int64_t cap, int64_t* out_n,
                int64_t* err_line) {
  rows_t rows = {0};
  int st = parse_rows(text, len, flags, &rows, err_line);
  if (st != ORACLE_OK) return st;
  if (rows.n > cap) {
    rows_free(&rows);
    return ORACLE_ERR_ARG;
  }
  memcpy(out_cid, rows.cid, sizeof(int64_t) * (size_t)rows.n);
  *out_n = rows.n;
  rows_free(&rows);
  return ORACLE_OK;
}

/* The first min(k, N) rows in ascending (distance, index) order: Fig. 3 steps 1-6. */
int oracle_topk(const char* text, size_t len, unsigned flags, const char* query, int64_t k, int nthreads,
                int32_t* out_idx, int32_t* out_dist, int64_t* out_cid, int64_t* out_n, int64_t* err_line) {
  rows_t rows = {0};
  int st = parse_rows(text, len, flags, &rows, err_line);
  if (st != ORACLE_OK) return st;
  st = topk_rows(&rows, query, k, nthreads, out_idx, out_dist, out_cid, out_n);
  rows_free(&rows);
  return st;
}

/*
 * Many queries against one library (the library is parsed once).  queries
 * holds Q x 166 characters back to back; query q writes its min(k[q], N)
 * results at offset off[q] of the output arrays and its count to out_n[q].
 */
int oracle_topk_many(const char* text, size_t len, unsigned flags, const char* queries, int64_t Q,
                     const int64_t* k, const int64_t* off, int nthreads, int32_t* out_idx, int32_t* out_dist,
                     int64_t* out_n, int64_t* err_line) {
  rows_t rows = {0};
  int st = parse_rows(text, len, flags, &rows, err_line);
  if (st != ORACLE_OK) return st;
  for (int64_t q = 0; q < Q && st == ORACLE_OK; ++q)
    st = topk_rows(&rows, queries + q * OR_BITS, k[q], nthreads, out_idx + off[q], out_dist + off[q], NULL,
                   &out_n[q]);
  rows_free(&rows);
  return st;
}

/*
 * "Combined and sorted" (text after Fig. 3): concatenated per-library result
 * lists (distance, global index) are sorted again and the first k kept.
 */
int oracle_combine(const int32_t* idx, const int32_t* dist, int64_t n, int64_t k, int32_t* out_idx,
                   int32_t* out_dist, int64_t* out_n) {
  if (k < 0 || n < 0) return ORACLE_ERR_ARG;
  pair_t* pr = (pair_t*)malloc(sizeof(pair_t) * (size_t)(n ? n : 1));
  if (!pr) return ORACLE_ERR_NOMEM;
  for (int64_t r = 0; r < n; ++r) pr[r] = (pair_t){dist[r], idx[r]};
  qsort(pr, (size_t)n, sizeof(pair_t), pair_cmp);
  int64_t m = k < n ? k : n;
  for (int64_t r = 0; r < m; ++r) {
    out_idx[r] = pr[r].i;
    out_dist[r] = pr[r].d;
  }
  *out_n = m;
  free(pr);
  return ORACLE_OK;
}

/* ====================================================================== wide
 * Longer fingerprints and the Tanimoto measure (an extension beyond the
 * paper's 166 MACCS keys: its conclusion names more features as future work).
 * A wide library is text of lines of exactly n_bits '0'/'1' characters (a
 * trailing '\r' is dropped; no CID column).  Per row, on the characters:
 *   ORACLE_MANHATTAN: d = #{j : q_j != x_j}, ranked ascending;
 *   ORACLE_TANIMOTO:  c = #{j : q_j = x_j = '1'}, u = #{j : q_j = '1' or
 *                     x_j = '1'}, similarity c / u (1 when u = 0: two empty
 *                     sets are equal), ranked descending; two similarities are
 *                     compared exactly as c1 u2 vs c2 u1.
 * Ties are ranked by ascending 0-based row.  Outputs per result: row, and the
 * measure as num / den (Manhattan: d / 1; Tanimoto: c / u, with 0 / 0 for u = 0).
 * All rows are scored (several threads over contiguous ranges), then one full
 * qsort orders them. */
#define ORACLE_MANHATTAN 0
#define ORACLE_TANIMOTO 1

typedef struct {
  int32_t num, den, i;
} wpair_t;

typedef struct {
  const char* text;
  const int64_t* line_start;
  const char* q;
  int n_bits, metric;
  wpair_t* out;
  int64_t lo, hi;
} wjob_t;

static void* wide_job(void* arg) {
  wjob_t* jb = (wjob_t*)arg;
  for (int64_t i = jb->lo; i < jb->hi; ++i) {
    const char* x = jb->text + jb->line_start[i];
    int32_t a = 0, b = 0;
    if (jb->metric == ORACLE_MANHATTAN) {
      for (int j = 0; j < jb->n_bits; ++j) a += (x[j] != jb->q[j]);
      b = 1;
    } else {
      for (int j = 0; j < jb->n_bits; ++j) {
        const int qj = jb->q[j] == '1', xj = x[j] == '1';
        a += qj & xj;
        b += qj | xj;
      }
    }
    jb->out[i] = (wpair_t){a, b, (int32_t)i};
  }
  return NULL;
}

/* Tanimoto order: larger c/u first (u = 0 counts as 1), then smaller row. */
static int tanimoto_cmp(const void* pa, const void* pb) {
  const wpair_t* x = (const wpair_t*)pa;
  const wpair_t* y = (const wpair_t*)pb;
  const int64_t xn = x->den ? x->num : 1, xd = x->den ? x->den : 1;
  const int64_t yn = y->den ? y->num : 1, yd = y->den ? y->den : 1;
  const int64_t l = xn * yd, r = yn * xd;
  if (l != r) return l > r ? -1 : 1;
  if (x->i != y->i) return x->i < y->i ? -1 : 1;
  return 0;
}

static int manhattan_cmp(const void* pa, const void* pb) {
  const wpair_t* x = (const wpair_t*)pa;
  const wpair_t* y = (const wpair_t*)pb;
  if (x->num != y->num) return x->num < y->num ? -1 : 1;
  if (x->i != y->i) return x->i < y->i ? -1 : 1;
  return 0;
}

int oracle_wide_topk(const char* text, size_t len, int n_bits, const char* query, int64_t k, int metric,
                     int nthreads, int32_t* out_idx, int32_t* out_num, int32_t* out_den, int64_t* out_n,
                     int64_t* err_line) {
  if (!text && len) return ORACLE_ERR_ARG;
  if (!query || n_bits < 1 || k < 0 || (metric != ORACLE_MANHATTAN && metric != ORACLE_TANIMOTO))
    return ORACLE_ERR_ARG;
  if (!all01(query, n_bits)) return ORACLE_ERR_ARG;
  /* rows: every line must be n_bits '0'/'1' characters (optionally followed by '\r') */
  int64_t cap = 1024, n = 0;
  int64_t* ls = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
  if (!ls) return ORACLE_ERR_NOMEM;
  size_t p = 0;
  while (p < len) {
    size_t e = p;
    while (e < len && text[e] != '\n') ++e;
    size_t l = e - p;
    if (l > 0 && text[p + l - 1] == '\r') --l;
    if ((int64_t)l != n_bits || !all01(text + p, (int64_t)l)) {
      if (err_line) *err_line = n + 1;
      free(ls);
      return ORACLE_ERR_PARSE;
    }
    if (n == cap) {
      cap *= 2;
      int64_t* g = (int64_t*)realloc(ls, sizeof(int64_t) * (size_t)cap);
      if (!g) {
        free(ls);
        return ORACLE_ERR_NOMEM;
      }
      ls = g;
    }
    ls[n++] = (int64_t)p;
    p = e + 1;
  }
  wpair_t* pr = (wpair_t*)malloc(sizeof(wpair_t) * (size_t)(n ? n : 1));
  if (!pr) {
    free(ls);
    return ORACLE_ERR_NOMEM;
  }
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (n < 4096) nthreads = 1;
  pthread_t th[256];
  int started[256];
  wjob_t jobs[256];
  int64_t chunk = (n + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    int64_t lo = chunk * t, hi = lo + chunk;
    if (lo > n) lo = n;
    if (hi > n) hi = n;
    jobs[t] = (wjob_t){text, ls, query, n_bits, metric, pr, lo, hi};
    started[t] = nthreads > 1 && pthread_create(&th[t], NULL, wide_job, &jobs[t]) == 0;
    if (!started[t]) wide_job(&jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t)
    if (started[t]) pthread_join(th[t], NULL);
  qsort(pr, (size_t)n, sizeof(wpair_t), metric == ORACLE_MANHATTAN ? manhattan_cmp : tanimoto_cmp);
  int64_t m = k < n ? k : n;
  for (int64_t r = 0; r < m; ++r) {
    out_idx[r] = pr[r].i;
    out_num[r] = pr[r].num;
    out_den[r] = pr[r].den;
  }
  *out_n = m;
  free(pr);
  free(ls);
  return ORACLE_OK;
}
