/*
 * fps.h -- C ABI of the GB300 exact fingerprint search (FPScreen hot path).
 *
 * The paper (Sec. 4.3, Fig. 3) searches a library of MACCS-166 fingerprints
 * for the molecules closest to a target: Manhattan distance over the 166
 * 0/1 keys, every library row paired with its distance, all pairs sorted
 * ascending, first k returned with their PubChem CIDs (Fig. 3: the inputs are
 * the target's MACCS-166 keys and the library file, the output each hit's CID
 * with its distance).  Here the
 * library is parsed once, packed to 24-byte records and kept in GPU memory;
 * each search is an exhaustive scan plus an exact top-k on the GPU.
 *
 * Result order (every path, every size): ascending distance, ties broken by
 * ascending 0-based library index.  This is a total order, so the answer is
 * unique and every path returns exactly the same bytes.
 *
 * Conventions shared by every entry point:
 *   - every function returns an fps_status; nothing throws or aborts across
 *     the ABI;
 *   - the library handle owns all of its device memory (packed records,
 *     index permutation, per-stream workspaces) until fps_release;
 *   - the caller owns every query and result buffer it passes in;
 *   - a handle is read-only after loading, so searches may run concurrently
 *     on different CUDA streams; searches on one stream run in stream order.
 *     fps_release must not race searches still in flight (the caller's duty);
 *   - bit order of a packed record or query: key j (character j of the text
 *     line, 0-based) is bit j % 64 of 64-bit word j / 64; bits 166..191 are 0;
 *   - k = 0 is valid and returns no results; out_count = min(k, N); the
 *     result slots from out_count up to k (k > N) hold -1 in every output
 *     array (index, distance, CID); slots past k, where the offsets of a
 *     batched call leave room, are left untouched;
 *   - k may not exceed FPS_K_MAX (FPS_ERR_UNSUPPORTED otherwise).
 */
#ifndef FPS_H
#define FPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FPS_BITS 166          /* MACCS keys per fingerprint (Sec. 4.2) */
#define FPS_WORDS 3           /* uint64 words per packed record */
#define FPS_K_MAX 1920        /* largest k any search accepts */

typedef enum {
  FPS_OK = 0,
  FPS_ERR_INVALID_ARG = 1,       /* null required pointer, k < 0, Q < 0, bad query characters ... */
  FPS_ERR_IO = 2,                /* the library file cannot be read */
  FPS_ERR_PARSE = 3,             /* a library line is malformed (see fps_load_desc.err_line) */
  FPS_ERR_BUDGET = 4,            /* the library would exceed hbm_budget_bytes; nothing was allocated */
  FPS_ERR_CUDA = 5,              /* a CUDA runtime call failed (no device, out of memory, launch error) */
  FPS_ERR_TIMEOUT = 6,           /* a bounded device-side wait ran out; results of that search are invalid */
  FPS_ERR_OVERFLOW_INTERNAL = 7, /* an internal candidate buffer overflowed and could not be recovered */
  FPS_ERR_UNSUPPORTED = 8,       /* a valid request this build does not serve (k > FPS_K_MAX, missing operand) */
  FPS_ERR_NOMEM = 9              /* host allocation failed */
} fps_status;

typedef struct fps_library_s* fps_library;

/* ---------------------------------------------------------------- loading */

#define FPS_LOAD_ACCEPT_167 0x1u  /* a 167-character line starting with '0' loses that character */
#define FPS_LOAD_NO_BUCKETS 0x2u  /* keep library order: no popcount buckets, so no pruning */
#define FPS_LOAD_TC_OPERAND 0x4u  /* also build the 0/1 FP8 operand the tensor-core batch path needs
                                     (192 bytes per record, bucketed layout only) */
#define FPS_LOAD_TC_INT8 0x8u     /* INT8 operand: always FPS_ERR_UNSUPPORTED (sm_103a has no tcgen05 kind::i8) */
#define FPS_LOAD_TC_FP4 0x10u     /* also build the packed 0/1 FP4 operand of FPS_PATH_TC_FP4 (96 bytes per
                                     record: two E2M1 keys per byte; bucketed layout only) */

/*
 * Exactly one library source must be given: a file path, an in-memory text
 * buffer, or already-packed records.
 *
 * Text format (Fig. 3 step 1: every molecule of the library file is read and
 * gives one row of the 0/1 matrix and one CID): one molecule per line,
 * either 166 '0'/'1' characters or "<cid><sep><166 characters>" with sep a
 * space, tab or comma and cid a
 * non-negative decimal integer.  A trailing '\r' is dropped; the final line
 * may lack its '\n'.  Any other line -- including an empty line before the
 * end -- fails the load with FPS_ERR_PARSE and its 1-based number in
 * *err_line.  Without a CID column the CID of a row is its 0-based index.
 *
 * Packed source: n_packed records of FPS_WORDS uint64 each (host memory, bit
 * order above; pad bits must be zero, else FPS_ERR_INVALID_ARG), with an
 * optional host array of n_packed CIDs.
 *
 * hbm_budget_bytes: 0 = unlimited; otherwise the load fails with
 * FPS_ERR_BUDGET, before allocating any device memory, if the device bytes
 * the library needs exceed it.
 */
typedef struct {
  const char* path;              /* library text file, or NULL */
  const char* text;              /* in-memory library text, or NULL */
  size_t text_len;
  const uint64_t* packed;        /* packed records (host), or NULL */
  size_t n_packed;
  const int64_t* cids;           /* optional CIDs of the packed records (host), or NULL */
  int device;                    /* CUDA device ordinal */
  size_t hbm_budget_bytes;
  uint32_t flags;                /* FPS_LOAD_* */
  size_t* err_line;              /* out (optional): line of the first parse error */
} fps_load_desc;

/* Parse (or take) the library, pack it, lay it out by popcount bucket and copy it to the device. */
fps_status fps_library_load(const fps_load_desc* desc, fps_library* out);

/* Release a library and all device memory it owns.  NULL is accepted (no-op).
 * The paper keeps no resident state (it re-reads the library file for every
 * search, Sec. 2.2); this is the end of the resident library's lifetime that
 * loading once begins. */
fps_status fps_release(fps_library lib);

typedef struct {
  int64_t n_records;             /* N */
  int64_t n_tiles;               /* 128-record scan tiles, including bucket padding */
  size_t device_bytes;           /* device memory held by the library (workspaces excluded) */
  int device;
  int bucketed;                  /* 1 = popcount-bucketed layout (pruning on) */
  int has_tc_operand;            /* 1 = the FP8 tensor-core operand is resident */
  int64_t bucket_count[FPS_BITS + 1]; /* records per popcount 0..166 */
  int has_tc_fp4;                /* 1 = the FP4 tensor-core operand is resident */
} fps_library_info;

fps_status fps_library_info_get(fps_library lib, fps_library_info* info);

/* CID of library row `index` (host lookup). */
fps_status fps_library_cid(fps_library lib, int64_t index, int64_t* cid);

/* --------------------------------------------------------------- searching */

typedef enum {
  FPS_PATH_AUTO = 0,     /* batch calls: an autotuner picks the kernel and its tile shape per size class
                            (see "Autotuning" below) */
  FPS_PATH_POPC = 1,     /* popcount scan: one launch per query (single-query kernel) */
  FPS_PATH_POPC_BATCH = 2, /* popcount scan, many queries per launch */
  FPS_PATH_TC_FP8 = 3,   /* tensor-core contraction on 0/1 FP8 operands */
  FPS_PATH_TC_I8 = 4,    /* INT8 tensor-core contraction: FPS_ERR_UNSUPPORTED on sm_103a (no kind::i8) */
  FPS_PATH_LEARNED = 5,  /* predicted per-query threshold, exact fallback */
  FPS_PATH_TC_FP4 = 6    /* tensor-core contraction on packed 0/1 FP4 operands (unit block scales) */
} fps_path;

#define FPS_SEARCH_DEVICE_IO 0x1u /* queries, k, offsets and outputs are device pointers; the call only
                                     enqueues work on the stream and returns (results valid after the
                                     stream is synchronised; errors reported by fps_sync) */

typedef struct {
  int64_t queries;               /* queries served by the call */
  int64_t fallbacks;             /* queries that needed the exact fallback scan */
  int64_t candidates;            /* records accepted under the running bounds (batched paths) */
  int64_t path_used;             /* fps_path of the kernel that ran (with FPS_PATH_LEARNED: the batched
                                    kernel that started from the predicted bounds) */
  int64_t device_fallbacks;      /* of the fallbacks, those re-run inside a batch plan's graph */
  int64_t tile_param;            /* the tile shape used: library tiles per work item (tensor-core paths)
                                    or queries per work item (FPS_PATH_POPC_BATCH); 0 otherwise */
} fps_search_stats;

/*
 * Autotuning (FPS_PATH_AUTO; the paper has no counterpart).  Batched calls fall
 * into size classes: ceil(log2 Q), ceil(log2 (max k + 1)), and whether learned
 * bounds are given.  The first call of a class on a library times, on the
 * call's own queries, every batched kernel the library holds an operand for
 * (popcount batch; FP8 and FP4 tensor cores) at its default tile shape, then
 * the fastest kernel at its other tile shapes (tensor cores: 1/2 and 2 x the
 * default library tiles per work item; popcount batch: 32, 64 or 128 queries
 * per work item), and keeps the fastest (kernel, shape) for the class.  Every
 * candidate returns the same exact results, so the call's results do not
 * depend on the choice.  When the environment variable FPS_TUNE_CACHE names a
 * file, choices are read from it (entries keyed by device name, library size
 * N and class) before tuning, and each new choice is merged into it.
 */
#define FPS_TUNE_CLASS_LEN 32
/* Class name of a batch ("q<ceil log2 Q>-k<ceil log2 (kmax + 1)>-l<0|1>") into out (FPS_TUNE_CLASS_LEN). */
fps_status fps_tune_class(int Q, int k_max, int learned, char* out);
/* Host-only access to a cache file: look up / merge one entry.  fps_tune_cache_get returns
   FPS_ERR_IO when the file or the entry does not exist. */
fps_status fps_tune_cache_get(const char* path, const char* device, int64_t n, const char* cls, int* fps_path_out,
                              int* tile_param, double* ms);
fps_status fps_tune_cache_put(const char* path, const char* device, int64_t n, const char* cls, int fps_path_in,
                              int tile_param, double ms);

typedef struct {
  int path;                      /* fps_path */
  uint32_t flags;                /* FPS_SEARCH_* */
  double timeout_s;              /* bound on any device-side wait; <= 0 = 2 s */
  fps_search_stats* stats;       /* optional out (host memory; filled by fps_search_batch in both forms) */
  const float* tau;              /* FPS_PATH_LEARNED: per-query predicted k-th distances (host or device like
                                    the queries); the scan starts from bound ceil(tau), clamped to 0..166 */
} fps_search_opts;

/*
 * The paper's single-molecule search (Fig. 3): query166 is 166 '0'/'1'
 * characters (FPS_ERR_INVALID_ARG otherwise).  Host outputs, synchronous.
 * out_index / out_dist receive min(k, N) entries; out_cid (nullable) the
 * CIDs; *out_count their number.  cuda_stream may be NULL (default stream).
 */
fps_status fps_search(fps_library lib, const char* query166, int k, int32_t* out_index, int32_t* out_dist,
                      int64_t* out_cid, int* out_count, void* cuda_stream);

/*
 * Single query in packed form (FPS_WORDS words).  Without FPS_SEARCH_DEVICE_IO
 * every pointer is host memory and the call returns when results are written.
 * With it, query, out_index, out_dist and out_count are device pointers, the
 * call is asynchronous on cuda_stream and *out_count is an int32 on the
 * device.  opts may be NULL (defaults).
 */
fps_status fps_search_packed(fps_library lib, const uint64_t* query, int k, int32_t* out_index, int32_t* out_dist,
                             int32_t* out_count, const fps_search_opts* opts, void* cuda_stream);

/*
 * Batched search.  The paper searches one target at a time (Fig. 3) and lists
 * batch processing of query molecules only for its clustering search
 * (Sec. 4.4); this entry point runs Q independent Fig. 3 searches in one
 * call, each with the result of its own single search.
 * Q queries (Q x FPS_WORDS packed words) with per-query k[q].  Results of
 * query q go to out_index/out_dist[out_offsets[q] .. out_offsets[q] + k[q]),
 * out_offsets holding Q + 1 entries (out_offsets[q+1] - out_offsets[q] >= k[q]);
 * out_count[q] = min(k[q], N).  k and out_offsets are always host arrays (the
 * launch plan is made on the host); queries, out_index, out_dist and
 * out_count are host or device memory per opts->flags, as in
 * fps_search_packed.  opts->path selects the kernel (FPS_PATH_AUTO lets the
 * library choose).  Slots min(k[q], N) .. k[q] of each query hold -1; slots
 * past k[q] are not written.  With a library of no records every path gives
 * count 0 without launching a scan (stats->path_used = FPS_PATH_POPC).
 */
fps_status fps_search_batch(fps_library lib, const uint64_t* queries, int Q, const int32_t* k,
                            const int64_t* out_offsets, int32_t* out_index, int32_t* out_dist, int32_t* out_count,
                            const fps_search_opts* opts, void* cuda_stream);

/*
 * Single-query search that allocates no device memory (the paper has no
 * counterpart: it exists for callers that cannot allocate when they search --
 * code whose device memory is all owned by another allocator, code with a
 * hard latency budget that cannot take a cudaMalloc and its implicit
 * synchronisation, code that searches on many short-lived streams where
 * fps_search_packed would create a workspace per stream).
 *
 * query (FPS_WORDS words), out_index and out_dist (k entries each) and
 * out_count (one int32) are device pointers owned by the caller; the call
 * enqueues work on cuda_stream and returns.  Results equal fps_search_packed's.
 * The scan's scratch is one fixed array inside this library, about 2.6 MB,
 * that every GPU which loads the library holds until the process exits.
 * Limits: k <= FPS_NOALLOC_K_MAX and at most 160 SMs (FPS_ERR_UNSUPPORTED
 * otherwise).  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) -- make that first call before any stream capture.
 * All calls on a device share the array: calls that may overlap on the GPU
 * (different streams without ordering between them) race and give wrong
 * results; order them on one stream.  Each call clears the scratch it needs.
 * With no records (or k = 0) *out_count = 0 and, as on every path, the k
 * result slots hold -1.  Each device-side wait is bounded by 2 s (the
 * environment variable FPS_NOALLOC_TIMEOUT_NS, read on every call, replaces
 * that bound; tests use it to make a wait run out).  A device-side failure (a
 * bounded wait that ran out) leaves *out_count = -1.
 */
#define FPS_NOALLOC_K_MAX 128
fps_status fps_search_noalloc(fps_library lib, const uint64_t* query, int k, int32_t* out_index, int32_t* out_dist,
                              int32_t* out_count, void* cuda_stream);

/*
 * A batch whose shape is fixed -- Q queries with per-query k[q] (host array),
 * path FPS_PATH_POPC_BATCH, FPS_PATH_TC_FP8 or FPS_PATH_AUTO, optionally
 * learned bounds -- captured once as a CUDA graph with its own buffers: copy
 * of the plan in, bounds, scan, per-query select, results out.  Each run takes
 * host queries (Q x FPS_WORDS) and, when learned, host predictions tau[Q];
 * results go to host arrays laid out by the prefix sums of k (as in
 * fps_search_batch); the call returns when they are written.  Queries that
 * need the exact fallback (candidate overflow, or a predicted bound below the
 * k-th distance) are re-run inside the graph: a conditional WHILE node runs the
 * single-query scan once per such query, reading the query, k and output
 * places from a device-side descriptor, so no host round trip is needed.  A
 * plan must not be run concurrently with itself; it must be released before
 * its library.  A plan on a library of no records holds no device state; its
 * runs write count 0 and -1 in each query's k slots on the host.
 */
typedef struct fps_batch_plan_s* fps_batch_plan;
fps_status fps_batch_plan_create(fps_library lib, int Q, const int32_t* k, int path, int learned, fps_batch_plan* out);
fps_status fps_batch_plan_run(fps_batch_plan plan, const uint64_t* queries, const float* tau, int32_t* out_index,
                              int32_t* out_dist, int32_t* out_count, fps_search_stats* stats, void* cuda_stream);
fps_status fps_batch_plan_release(fps_batch_plan plan);

/* Wait for cuda_stream and report (then clear) any device-side error of searches enqueued on it. */
fps_status fps_sync(fps_library lib, void* cuda_stream);

/* ---------------------------------------------------- learned threshold (MLP)
 *
 * The paper has no counterpart: this small network predicts a query's k-th
 * nearest distance so the batched scan (FPS_PATH_LEARNED) can start from a
 * tight per-query bound instead of the sampled one.  Results stay exact: a
 * query whose prediction was too low (fewer than k records at or under it) is
 * re-run by the exact scan.
 *   x  = [166 query bits, popc(q)/166];  h1 = relu(W1 x + b1)  (256);
 *   h2 = relu(W2 h1 + b2) (256);  y = w3 . h2 + b3.
 * BF16 weights in every product (FP32 masters for Adam), FP32 accumulation,
 * mean pinball loss at a chosen quantile.  Parameters are one flat FP32 array
 * in the order W1 (256 x 167, row-major), b1, W2 (256 x 256), b2, w3, b3.
 */
typedef struct fps_mlp_s* fps_mlp;

/* Number of FP32 parameters (109057). */
size_t fps_mlp_param_count(void);
/* A model on `device` with all parameters zero (set them with fps_mlp_set_params). */
fps_status fps_mlp_create(int device, fps_mlp* out);
fps_status fps_mlp_release(fps_mlp mlp);
/* Copy parameters in (resets the Adam moments and step) / out; host arrays of fps_mlp_param_count() floats. */
fps_status fps_mlp_set_params(fps_mlp mlp, const float* host, size_t n);
fps_status fps_mlp_get_params(fps_mlp mlp, float* host, size_t n);
/* Predicted thresholds for Q packed queries; queries and out are device pointers; asynchronous on the stream. */
fps_status fps_mlp_predict(fps_mlp mlp, const uint64_t* queries, int Q, float* out, void* cuda_stream);
/* Forward + backward on B examples (device queries and targets); gradients stay on the device and are copied
   to grad_host (fps_mlp_param_count() floats) and the mean loss to loss_host when those are non-NULL. */
fps_status fps_mlp_grad(fps_mlp mlp, const uint64_t* queries, const float* targets, int B, float quantile,
                        float* grad_host, float* loss_host, void* cuda_stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on B examples; loss_host (nullable) gets the mean loss. */
fps_status fps_mlp_train_step(fps_mlp mlp, const uint64_t* queries, const float* targets, int B, float quantile,
                              float lr, float* loss_host, void* cuda_stream);

/*
 * "Combined and sorted" (the text after Fig. 3: several library files are
 * searched separately and their results merged): k-way merge of `parts`
 * result lists, each already in ascending (distance, index) order with
 * indices global to the combined library.  List p holds the entries
 * [part_off[p], part_off[p+1]) of idx/dist (host arrays).  Writes the first
 * min(k, total) entries of the combined order; *out_n their number.  Host only.
 */
fps_status fps_merge_topk(const int32_t* idx, const int32_t* dist, const int64_t* part_off, int parts, int k,
                          int32_t* out_index, int32_t* out_dist, int* out_n);

/*
 * Several resident libraries searched as one (the paper's parallel strides:
 * separate datasets searched at the same time, results "combined and
 * sorted", with each stride's progress shown; Sec. 2.1, Sec. 4.4).  libs[s]
 * holds the records whose global indices start at index_base[s] (nullable:
 * the prefix sums of the libraries' sizes, in order); the index ranges must
 * not overlap.  All libraries live on one device; at most FPS_SHARDS_MAX.
 * Queries, k, out_offsets and outputs are as in fps_search_batch (host or
 * device per opts->flags, opts->path per shard); out_index holds global
 * indices and out_count[q] = min(k[q], total records).  Every shard runs the
 * batched search into device staging, then one kernel merges the per-shard
 * lists of each query on the device (k-way merge of ascending (distance,
 * global index) keys).  progress (nullable) is host memory of n_libs int64
 * that the device can write: pinned, mapped memory (cudaMallocHost,
 * cudaHostAlloc), or any host memory on systems whose GPU addresses pageable
 * memory; FPS_ERR_INVALID_ARG if cudaHostGetDevicePointer refuses it.
 * progress[s] is set to Q by the device, in stream order, once shard s's
 * results are complete, so another thread can watch the strides finish.
 */
#define FPS_SHARDS_MAX 32
fps_status fps_search_shards(const fps_library* libs, int n_libs, const int64_t* index_base, const uint64_t* queries,
                             int Q, const int32_t* k, const int64_t* out_offsets, int32_t* out_index,
                             int32_t* out_dist, int32_t* out_count, const fps_search_opts* opts, int64_t* progress,
                             void* cuda_stream);

/*
 * Longer fingerprints (an extension beyond the paper's 166 MACCS keys; its
 * conclusion names more features as future work): records of n_bits bits
 * (1..FPS_WIDE_MAX_BITS), W = ceil(n_bits / 64) words each, bit j of a record
 * = word j/64, bit j%64 (bits past n_bits zero).  Two measures:
 *   FPS_METRIC_MANHATTAN  d = popc(q XOR x), ascending;
 *   FPS_METRIC_TANIMOTO   c / u with c = popc(q AND x), u = popc(q OR x)
 *                         (1 when u = 0), descending, compared exactly;
 * ties by ascending record index.  The library is resident in device memory
 * (word-major tiles of 128 records; no popcount buckets) until released.
 * fps_wide_load takes text (lines of n_bits '0'/'1' characters; a trailing
 * '\r' is dropped; FPS_ERR_PARSE with *err_line otherwise) or packed words
 * (n_packed x W, host), not both; FPS_ERR_BUDGET if the device copy would
 * exceed hbm_budget_bytes (0 = no limit).
 * fps_wide_search: query holds W words; writes min(k, N) results: out_index,
 * and the measure as out_num / out_den (Manhattan: d / 1; Tanimoto: c / u,
 * 0 / 0 for two empty sets).  Host memory and synchronous, or with
 * FPS_SEARCH_DEVICE_IO device memory and asynchronous on cuda_stream.
 */
#define FPS_WIDE_MAX_BITS 2048
#define FPS_METRIC_MANHATTAN 0
#define FPS_METRIC_TANIMOTO 1
typedef struct fps_wide_library_s* fps_wide_library;
fps_status fps_wide_load(const char* text, size_t text_len, const uint64_t* packed, size_t n_packed, int n_bits,
                         int device, size_t hbm_budget_bytes, fps_wide_library* out, size_t* err_line);
fps_status fps_wide_info(fps_wide_library lib, int64_t* n_records, int* n_bits, size_t* device_bytes);
fps_status fps_wide_search(fps_wide_library lib, const uint64_t* query, int k, int metric, int32_t* out_index,
                           int32_t* out_num, int32_t* out_den, int32_t* out_count, uint32_t flags,
                           void* cuda_stream);
fps_status fps_wide_release(fps_wide_library lib);

/*
 * Batch clustering search (the paper's second search function, Sec. 4.4 and
 * the results after Fig. 1: a batch of query molecules is clustered, the
 * number of clusters chosen by the silhouette ("contour") coefficient, and
 * the top molecules are listed per cluster).  The paper names no algorithm;
 * this one (all integer, every tie to the smaller query index) is:
 * k-medoids over the Manhattan distances between the Q queries, seeded with
 * the most central query then farthest-first, alternating nearest-medoid
 * assignment and medoid update (the member with the smallest sum of
 * distances to its cluster) for at most 30 rounds; for every count c in
 * [c_min, min(c_max, Q - 1)] the score is sum_i floor(s_i * 2^32) with s_i
 * the silhouette of query i; the largest score (smaller c on ties) wins, and
 * each of its clusters is searched with its medoid: the k nearest library
 * records by (distance, index).  With Q - 1 < c_min there is one cluster
 * around the most central query.
 * Host memory, synchronous.  1 <= Q <= FPS_CLUSTER_MAX_Q; 2 <= c_min <= c_max
 * <= FPS_CLUSTER_MAX_C; 0 <= k <= FPS_K_MAX.  Outputs: *out_c; out_labels[Q]
 * (cluster of every query, 0 .. c-1); out_medoids[c] (query index of each
 * cluster's medoid); out_scores[c_max - c_min + 1] (nullable; INT64_MIN for
 * counts not tried); out_index / out_dist [c * k] and out_count[c]: cluster t's
 * results at t * k.
 */
#define FPS_CLUSTER_MAX_Q 4096
#define FPS_CLUSTER_MAX_C 16
fps_status fps_cluster_search(fps_library lib, const uint64_t* queries, int Q, int c_min, int c_max, int k,
                              int* out_c, int32_t* out_labels, int32_t* out_medoids, int64_t* out_scores,
                              int32_t* out_index, int32_t* out_dist, int32_t* out_count, void* cuda_stream);

/* ----------------------------------------------------------------- helpers */

const char* fps_status_string(fps_status st);

/* Pack 166 '0'/'1' characters into FPS_WORDS words (host). */
fps_status fps_pack_query(const char* query166, uint64_t out[FPS_WORDS]);

/*
 * Host-only parse of library text into packed records (the load's first
 * step, exposed for tools and tests).  Call with out_packed = NULL to get the
 * record count in *out_n; otherwise cap records are available at out_packed
 * (cap x FPS_WORDS words) and out_cids (nullable).
 */
fps_status fps_pack_text(const char* text, size_t text_len, uint32_t flags, uint64_t* out_packed,
                         int64_t* out_cids, size_t cap, size_t* out_n, size_t* err_line);

#ifdef __cplusplus
}
#endif

#endif /* FPS_H */
