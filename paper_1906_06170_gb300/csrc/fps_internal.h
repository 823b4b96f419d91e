// Internal declarations shared by the host library code and the CUDA kernels.
// Nothing here crosses the C ABI (include/fps.h is the public boundary).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fps.h"

namespace fps {

constexpr int kBits = FPS_BITS;        // 166 MACCS keys (Sec. 4.2)
constexpr int kWords = FPS_WORDS;      // 3 x uint64 per record
constexpr int kTile = 128;             // records per scan tile: [3][128] uint64 = 3 KB contiguous
constexpr int kTileBytes = kTile * kWords * 8;
constexpr int kBucketAlign = 256;      // every popcount bucket starts on a 256-record boundary
constexpr int kNumBuckets = kBits + 1; // popcounts 0..166
constexpr int kKMax = FPS_K_MAX;

// A kernel's dynamic shared memory limit is an attribute of the function in each
// device's context, so it is set once per device: bit d of *done records device d.
// Threads racing on a device's first launch both set it, which is harmless.
template <typename F>
cudaError_t smem_attr_once(F* kernel, size_t bytes, std::atomic<uint64_t>* done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
  if (bit != 0 && (done->load(std::memory_order_acquire) & bit) != 0) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
  if (e == cudaSuccess && bit != 0) done->fetch_or(bit, std::memory_order_release);
  return e;
}

// Device view of a resident library, passed to kernels by value.
//   words:    [n_tiles][3][kTile] uint64, word-major inside a tile, so a warp's
//             loads of one word of 32 consecutive records are one 256-byte line;
//   perm:     [n_tiles * kTile] original 0-based index of each position (-1 = pad);
//   tile_off: [kNumBuckets + 1] first tile of each popcount bucket (bucket b holds
//             the records with popc == b in ascending index, tiles tile_off[b]..);
//   bcount:   [kNumBuckets] records per bucket.
// Without buckets, bucket 0 holds every record in index order and pruning is off.
struct DevLib {
  const uint64_t* words;
  const int32_t* perm;
  const int32_t* tile_off;
  const int32_t* bcount;
  int64_t n;
  int64_t n_tiles;
  int bucketed;
};

// Running state of one single-query scan.  Lives at the start of a per-stream
// workspace (256-byte aligned); the last block of every scan restores it to
// the initial values, so consecutive scans on one stream need no memset.
// The first 16 bytes (the two thresholds) are fetched by the bulk copy of every
// scan tile, so warps see tightened thresholds without a dependent load.
constexpr int kScanSmallMaxBlocks = 256;   // largest grid of the small-library scan

struct ScanState {
  unsigned long long thr_key;    // upper bound on the k-th key (d << 32 | index)
  uint32_t thr_d;                // upper bound on the k-th distance
  uint32_t pad0;
  uint32_t done;                 // blocks finished
  uint32_t ncand;                // keys written to the candidate array
  uint32_t pad1[2];
  uint32_t hist[168];            // accepted records per distance (distinct records)
  uint32_t queue[16 * 32];       // tail work queues: counter c at queue[32 c] (one 128-byte line each)
  uint32_t bcnt[kScanSmallMaxBlocks];   // small-library scan: each block's candidate counts and bound
};
static_assert(sizeof(ScanState) % 16 == 0, "ScanState keeps 16-byte alignment");

// Per-stream staging for host-IO searches; device copy and pinned host copy
// share the layout so one copy moves each direction.
struct HostIO {
  uint64_t query[4];             // packed query (3 words used)
  uint32_t err;                  // device error bits (FPS_DEVERR_*)
  int32_t count;                 // results written
  int32_t res[2 * kKMax];        // [index k][distance k]
};

enum : uint32_t { DEVERR_TIMEOUT = 1u, DEVERR_INTERNAL = 2u, DEVERR_OVERFLOW = 4u };

struct Workspace {
  ScanState* st = nullptr;       // device
  HostIO* io = nullptr;          // device
  HostIO* io_host = nullptr;     // pinned host
  unsigned long long* cand = nullptr;
  // second scan state and candidate array: consecutive searches of one sequence alternate
  ScanState* st2 = nullptr;
  unsigned long long* cand2 = nullptr;
  size_t cand_cap = 0;
  void* block = nullptr;         // the one device allocation holding st, io and cand
  // batched-path scratch (grown on demand)
  void* batch_block = nullptr;
  size_t batch_bytes = 0;
  void* batch_host = nullptr;
  size_t batch_host_bytes = 0;
  // shard-search staging (grown on demand)
  void* shard_block = nullptr;
  size_t shard_bytes = 0;
  void* shard_host = nullptr;
  size_t shard_host_bytes = 0;
  void* cluster_block = nullptr;    // batch clustering scratch (device), grown on demand
  size_t cluster_bytes = 0;
  void* cluster_host = nullptr;     // its pinned round-state words
  size_t cluster_host_bytes = 0;
};

struct Library {
  int device = 0;
  DevLib dev{};
  std::vector<void*> allocations;
  size_t device_bytes = 0;
  int64_t n = 0;
  int64_t n_tiles = 0;
  int bucketed = 1;
  std::vector<int64_t> cids;     // empty = CID is the index
  int64_t bucket_count[kNumBuckets] = {};
  int num_sms = 0;
  std::mutex mu;
  std::map<cudaStream_t, Workspace*> ws;
  uint8_t* tc_fp8 = nullptr;     // 0/1 FP8 operand (tensor-core path), or null
  uint8_t* tc_fp4 = nullptr;     // packed 0/1 FP4 operand (tensor-core path), or null
  // autotuner: size class -> fastest (batched path, tile parameter); the cache file's
  // entries for this library are read once, on the first tuned call
  struct Choice {
    int path = 0;
    int param = 0;
  };
  std::map<std::string, Choice> tuned;
  bool tune_cache_read = false;
};

// Per-query state of a batched search (device pointers; fps_batch.cu).
//   thr[q]   upper bound on the k-th distance of query q (starts from the pilot
//            or from a predicted threshold, only ever tightened);
//   hist[q]  accepted records of q per distance (168 bins, each record once);
//   cnt[q]   candidate keys appended for q (may exceed its capacity: overflow);
//   cand     keys d << 32 | layout position (the select kernel maps positions
//            to library indices), query q owns [cand_off[q], cand_off[q+1]).
struct BatchDev {
  int Q;
  const uint64_t* queries;       // Q x 3 words
  const int32_t* k;              // Q
  const int64_t* cand_off;       // Q + 1
  const int64_t* out_off;        // Q + 1
  uint32_t* thr;
  uint32_t* hist;
  uint32_t* cnt;
  unsigned long long* cand;
  int32_t* out_idx;
  int32_t* out_dist;
  int32_t* out_count;            // -2 = candidate overflow (host falls back), else min(k, N)
  uint32_t* err;
};

// ---- batched kernels (fps_batch.cu)
cudaError_t batch_prepare(const DevLib& lib, const BatchDev& b, int use_pilot, cudaStream_t s);
// Starting bounds from predicted distances: thr[q] = clamp(ceil(tau[q]), 0, 166).
cudaError_t batch_thr_from_tau(const BatchDev& b, const float* tau, cudaStream_t s);
// qb: queries per work item, 32, 64 or 128 (<= 0: the default, 64)
cudaError_t batch_scan_popc(const DevLib& lib, const BatchDev& b, int num_sms, uint32_t* work_counter, int qb,
                            cudaStream_t s);
constexpr int kPopcBatchDefaultQB = 64;
cudaError_t batch_select(const DevLib& lib, const BatchDev& b, cudaStream_t s);

// ---- shard merge (fps_batch.cu): per-shard result lists of one batch (device memory, laid out
// by the batch's output offsets) and the global index of each shard's first record
constexpr int kShardsMax = 32;
struct ShardLists {
  int n;
  const int32_t* idx[kShardsMax];
  const int32_t* dist[kShardsMax];
  const int32_t* count[kShardsMax];
  int64_t base[kShardsMax];
};
// out_count[q] = entries written for query q (<= off[q+1] - off[q])
cudaError_t launch_shard_merge(const ShardLists& sl, int Q, const int64_t* off, const int32_t* k, int32_t* out_idx,
                               int32_t* out_dist, int32_t* out_count, cudaStream_t s);
// *slot_dev = value, in stream order (slot_dev: device view of pinned host memory)
cudaError_t launch_progress(int64_t* slot_dev, int64_t value, cudaStream_t s);

// ---- batch clustering (fps_cluster.cu); every tie goes to the smaller query index
// A kernel whose bounded wait ran out still waits, this long at least, for its own bulk
// copies and MMAs in flight before it leaves (they complete in microseconds; a caller's
// short timeout must not let a CTA exit or free TMEM under them).
constexpr uint64_t kDrainNs = 1000000000ull;

constexpr int kClusterMaxC = 16;    // largest cluster count
constexpr int kClusterIters = 30;   // k-medoids rounds at most
cudaError_t cluster_qdist(const uint64_t* q, int Q, int32_t* D, cudaStream_t s);            // Q x Q distances
// out[i] = sum_j D[i][j] (lab == nullptr) or the sum over i's own cluster
cudaError_t cluster_rowsum(const int32_t* D, int Q, const int32_t* lab, int32_t* out, cudaStream_t s);
cudaError_t cluster_near(const int32_t* D, int Q, const int32_t* m, bool first, int32_t* near, cudaStream_t s);
// *out = argmin (or argmax) of val over the queries not in ex[0..n_ex) (lab == nullptr) or with lab == want
cudaError_t cluster_select(const int32_t* val, int Q, bool largest, const int32_t* ex, int n_ex, const int32_t* lab,
                           int want, int32_t* out, cudaStream_t s);
// k-medoids rounds for every cluster count at once (slot s: c_min + s clusters).
// state[4 s] = {active, rounds done, needs a final assignment, unused}; any_active has
// kClusterIters words, word r set when some slot goes on after round r.
struct ClusterRounds {
  const int32_t* D;
  int Q;
  int c_min;
  int n_slots;
  int32_t* med;          // [n_slots][kClusterMaxC], starts as the seeds
  int32_t* lab;          // [n_slots][Q]
  int32_t* cost;         // [n_slots][Q]
  int32_t* state;        // [n_slots][4]
  int32_t* any_active;   // [kClusterIters]
};
cudaError_t cluster_round(const ClusterRounds& r, int round, cudaStream_t s);
cudaError_t cluster_final_assign(const ClusterRounds& r, cudaStream_t s);
// *score += sum_i floor(s_i 2^32) (two's complement in 64 bits)
cudaError_t cluster_silhouette(const int32_t* D, int Q, const int32_t* lab, int c, int32_t* sizes,
                               unsigned long long* score, cudaStream_t s);

// ---- autotuner: size classes and the JSON cache of chosen kernels and tile shapes (fps_tune.cpp)
std::string tune_class_name(int Q, int k_max, bool learned);
bool tune_cache_get(const char* path, const char* device, int64_t n, const std::string& cls, int* path_out,
                    int* param, double* ms);
bool tune_cache_put(const char* path, const char* device, int64_t n, const std::string& cls, int path_in, int param,
                    double ms);

// ---- tensor-core batched scan (fps_tc.cu)
// Operand formats: 0/1 FP8 E4M3 bytes (kind::f8f6f4, 256-record tiles) or packed
// FP4 E2M1 nibbles with unit block scales (kind::mxf4, 128-record tiles).
constexpr int kTcFp8 = 0;
constexpr int kTcFp4 = 1;
int64_t tc_tiles(int fmt, int64_t n_tiles128);         // library tiles of the format
int tc_tile_rows(int fmt);                              // records per library tile
size_t tc_operand_bytes(int fmt, int64_t n_tiles128);
size_t tc_query_operand_bytes(int fmt, int Q);
cudaError_t tc_pack_library(int fmt, const DevLib& lib, uint8_t* op, cudaStream_t s);
cudaError_t tc_pack_queries(int fmt, const uint64_t* q, int Q, uint8_t* op, cudaStream_t s);
// chunk: library tiles per work item (<= 0: the format's default)
cudaError_t tc_scan(int fmt, const DevLib& lib, const BatchDev& b, const uint8_t* lib_op, const uint8_t* q_op,
                    int num_sms, int chunk, double timeout_s, cudaStream_t s);
int tc_default_chunk(int fmt);

// Description of one search for the indirect scan launch (device memory).  The device-side
// fallback of a captured batch fills it for each query it re-runs; cursor and nfallback are
// that loop's position and count.
struct ScanSlot {
  const uint64_t* query;
  int32_t* out_idx;
  int32_t* out_dist;
  int32_t* out_count;
  int32_t k;
  int32_t cursor;
  uint32_t nfallback;
  uint32_t pad;
};

// ---- kernels (fps_scan.cu)
// Scan configuration chosen for a given k.
struct ScanConfig {
  int warps;
  int cap;
  int kmax;
  size_t smem;
};
ScanConfig scan_config_for(int k);
size_t scan_cand_capacity(int num_sms);  // keys needed by the largest configuration
cudaError_t scan_state_init(ScanState* st, cudaStream_t s);
// programmatic: launch as a programmatic dependent of the previous kernel on s, which must be
// a scan of the same sequence using the other scan state (and the other candidate array); the
// grid then streams while that scan merges (see batch_sequential).
cudaError_t launch_scan_single(const DevLib& lib, const uint64_t* d_query, int k, ScanState* st,
                               unsigned long long* cand, int32_t* out_idx, int32_t* out_dist, int32_t* out_count,
                               uint32_t* err, int num_sms, double timeout_s, cudaStream_t s,
                               bool programmatic = false);
// The search a ScanSlot describes (k <= FPS_K_MAX); call scan_indirect_prepare once before
// capturing such a launch into a graph.
cudaError_t scan_indirect_prepare();
cudaError_t launch_scan_indirect(const DevLib& lib, const ScanSlot* slot, ScanState* st, unsigned long long* cand,
                                 uint32_t* err, int num_sms, double timeout_s, cudaStream_t s);
// Captured into a graph only: picks the next query with count -2 into the slot and sets the
// WHILE node's condition h (first = start from query 0 and reset the count).
cudaError_t launch_fallback_pick(const uint64_t* queries, const int32_t* k, const int64_t* out_off, int32_t* oi,
                                 int32_t* od, int32_t* oc, int Q, ScanSlot* slot, bool first,
                                 cudaGraphConditionalHandle h, cudaStream_t s);

}  // namespace fps
