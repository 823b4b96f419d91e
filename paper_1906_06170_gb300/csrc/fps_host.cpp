// Host side of the C ABI: library parsing/packing, popcount-bucketed layout,
// device residency, per-stream workspaces and the search entry points.
//
// Paper: Fig. 3 step 1 (read every molecule of the library file, build the
// CID column and the 0/1 matrix) becomes a one-time parse of the library text
// into packed 24-byte records that stay in GPU memory; step 2 (the target's vector B)
// becomes fps_pack_query; steps 3-6 run on the GPU (fps_scan.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "fps_internal.h"

using namespace fps;

namespace {

// ------------------------------------------------------------------ utilities
int hw_threads() {
  unsigned n = std::thread::hardware_concurrency();
  return n ? static_cast<int>(std::min(n, 64u)) : 4;
}

template <class F>
void parallel_for(int64_t n, int threads, F&& fn) {  // fn(t, lo, hi)
  if (threads < 1) threads = 1;
  if (n < 65536) threads = 1;
  int64_t chunk = (n + threads - 1) / threads;
  std::vector<std::thread> pool;
  for (int t = 1; t < threads; ++t) {
    int64_t lo = std::min<int64_t>(n, chunk * t), hi = std::min<int64_t>(n, lo + chunk);
    pool.emplace_back([&fn, t, lo, hi] { fn(t, lo, hi); });
  }
  fn(0, 0, std::min<int64_t>(n, chunk));
  for (auto& th : pool) th.join();
}

inline int popc3(const uint64_t* w) {
  return __builtin_popcountll(w[0]) + __builtin_popcountll(w[1]) + __builtin_popcountll(w[2]);
}

struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// ---------------------------------------------------------------- text parse
// One line (without '\n') -> packed record + CID.  Returns false on a format error.
bool parse_line(const char* s, int64_t len, uint32_t flags, uint64_t w[3], int64_t* cid, bool* has_cid) {
  if (len > 0 && s[len - 1] == '\r') --len;
  const char* bits = nullptr;
  *has_cid = false;
  auto all01 = [](const char* p, int64_t n) {
    for (int64_t j = 0; j < n; ++j)
      if (p[j] != '0' && p[j] != '1') return false;
    return true;
  };
  if (len == kBits && all01(s, len)) {
    bits = s;
  } else if (len == kBits + 1 && (flags & FPS_LOAD_ACCEPT_167) && s[0] == '0' && all01(s, len)) {
    bits = s + 1;
  } else {
    int64_t sep = -1;
    for (int64_t j = 0; j < len; ++j) {
      char c = s[j];
      if (c == ' ' || c == '\t' || c == ',') {
        sep = j;
        break;
      }
    }
    if (sep <= 0 || len - sep - 1 != kBits || !all01(s + sep + 1, kBits)) return false;
    int64_t v = 0;
    for (int64_t j = 0; j < sep; ++j) {
      char c = s[j];
      if (c < '0' || c > '9' || v > (INT64_MAX - 9) / 10) return false;
      v = v * 10 + (c - '0');
    }
    bits = s + sep + 1;
    *cid = v;
    *has_cid = true;
  }
  w[0] = w[1] = w[2] = 0;
  for (int j = 0; j < kBits; ++j) w[j >> 6] |= static_cast<uint64_t>(bits[j] - '0') << (j & 63);
  return true;
}

struct Parsed {
  std::vector<uint64_t> packed;
  std::vector<int64_t> cids;
  bool any_cid = false;
  int64_t n = 0;
};

// Multi-threaded parse: chunks split at line boundaries, counted, then filled in place.
fps_status parse_text(const char* text, size_t len, uint32_t flags, Parsed* out, size_t* err_line) {
  const int T = len < (1u << 20) ? 1 : hw_threads();
  std::vector<size_t> cut(T + 1, len);
  cut[0] = 0;
  for (int t = 1; t < T; ++t) {
    size_t p = len * static_cast<size_t>(t) / T;
    while (p < len && text[p - 1] != '\n') ++p;
    cut[t] = std::max(p, cut[t - 1]);
  }
  std::vector<int64_t> lines(T, 0);
  auto count_lines = [&](int t) {
    int64_t c = 0;
    for (size_t p = cut[t]; p < cut[t + 1]; ++p) c += text[p] == '\n';
    if (cut[t + 1] == len && len > cut[t] && text[len - 1] != '\n') c += 1;
    lines[t] = c;
  };
  {
    std::vector<std::thread> pool;
    for (int t = 1; t < T; ++t) pool.emplace_back(count_lines, t);
    count_lines(0);
    for (auto& th : pool) th.join();
  }
  std::vector<int64_t> first(T + 1, 0);
  for (int t = 0; t < T; ++t) first[t + 1] = first[t] + lines[t];
  const int64_t n = first[T];
  if (n >= (static_cast<int64_t>(1) << 31) - 1) return FPS_ERR_UNSUPPORTED;
  try {
    out->packed.assign(static_cast<size_t>(n) * 3, 0);
    out->cids.assign(static_cast<size_t>(n), 0);
  } catch (const std::bad_alloc&) {
    return FPS_ERR_NOMEM;
  }
  std::vector<int64_t> bad(T, -1);
  std::vector<char> saw_cid(T, 0);
  auto fill = [&](int t) {
    int64_t row = first[t];
    size_t p = cut[t];
    while (p < cut[t + 1]) {
      size_t e = p;
      while (e < len && text[e] != '\n') ++e;
      int64_t cid = row;
      bool hc = false;
      if (!parse_line(text + p, static_cast<int64_t>(e - p), flags, &out->packed[3 * row], &cid, &hc)) {
        bad[t] = row;
        return;
      }
      out->cids[row] = cid;
      saw_cid[t] |= hc;
      ++row;
      p = e + 1;
    }
  };
  {
    std::vector<std::thread> pool;
    for (int t = 1; t < T; ++t) pool.emplace_back(fill, t);
    fill(0);
    for (auto& th : pool) th.join();
  }
  for (int t = 0; t < T; ++t) {
    if (bad[t] >= 0) {
      if (err_line) *err_line = static_cast<size_t>(bad[t] + 1);
      return FPS_ERR_PARSE;
    }
    out->any_cid |= saw_cid[t] != 0;
  }
  out->n = n;
  return FPS_OK;
}

// --------------------------------------------------------------- device alloc
fps_status dev_alloc(Library* L, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  L->allocations.push_back(*p);
  L->device_bytes += bytes;
  return FPS_OK;
}

void free_library(Library* L) {
  if (!L) return;
  DeviceGuard g(L->device);
  for (auto& kv : L->ws) {
    Workspace* w = kv.second;
    if (w->block) cudaFree(w->block);
    if (w->io_host) cudaFreeHost(w->io_host);
    if (w->batch_block) cudaFree(w->batch_block);
    if (w->batch_host) cudaFreeHost(w->batch_host);
    if (w->shard_block) cudaFree(w->shard_block);
    if (w->shard_host) cudaFreeHost(w->shard_host);
    if (w->cluster_block) cudaFree(w->cluster_block);
    if (w->cluster_host) cudaFreeHost(w->cluster_host);
    delete w;
  }
  L->ws.clear();
  for (void* p : L->allocations) cudaFree(p);
  L->allocations.clear();
  delete L;
}

// Bytes the resident layout needs on the device.
struct Layout {
  int64_t n_tiles = 0;
  int64_t pos_base[kNumBuckets + 1] = {};
  int64_t count[kNumBuckets] = {};
  size_t bytes = 0;
};

Layout plan_layout(const uint64_t* packed, int64_t n, bool bucketed, std::vector<uint8_t>* popc) {
  Layout lay;
  if (bucketed) {
    popc->resize(static_cast<size_t>(n));
    const int T = hw_threads();
    std::vector<std::vector<int64_t>> cnt(T, std::vector<int64_t>(kNumBuckets, 0));
    parallel_for(n, T, [&](int t, int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i) {
        int b = popc3(packed + 3 * i);
        (*popc)[i] = static_cast<uint8_t>(b);
        cnt[t][b] += 1;
      }
    });
    for (auto& c : cnt)
      for (int b = 0; b < kNumBuckets; ++b) lay.count[b] += c[b];
    int64_t run = 0;
    for (int b = 0; b < kNumBuckets; ++b) {
      lay.pos_base[b] = run;
      run += (lay.count[b] + kBucketAlign - 1) / kBucketAlign * kBucketAlign;
    }
    lay.pos_base[kNumBuckets] = run;
    lay.n_tiles = run / kTile;
  } else {
    lay.count[0] = n;
    lay.n_tiles = (n + kBucketAlign - 1) / kBucketAlign * (kBucketAlign / kTile);
    lay.pos_base[0] = 0;
    for (int b = 1; b <= kNumBuckets; ++b) lay.pos_base[b] = lay.n_tiles * kTile;
  }
  lay.bytes = static_cast<size_t>(lay.n_tiles) * kTileBytes + static_cast<size_t>(lay.n_tiles) * kTile * 4 +
              2 * (kNumBuckets + 1) * sizeof(int32_t);
  return lay;
}

fps_status build_library(const uint64_t* packed, int64_t n, const int64_t* cids, const fps_load_desc* d,
                         Library** out) {
  for (int64_t i = 0; i < n; ++i)
    if (packed[3 * i + 2] >> (kBits - 128)) return FPS_ERR_INVALID_ARG;  // pad bits must be zero
  const bool bucketed = !(d->flags & FPS_LOAD_NO_BUCKETS);
  std::vector<uint8_t> popc;
  Layout lay = plan_layout(packed, n, bucketed, &popc);
  const bool want_fp8 = (d->flags & FPS_LOAD_TC_OPERAND) != 0;
  const bool want_fp4 = (d->flags & FPS_LOAD_TC_FP4) != 0;
  if (d->flags & FPS_LOAD_TC_INT8) return FPS_ERR_UNSUPPORTED;        // sm_103a has no tcgen05 kind::i8
  if ((want_fp8 || want_fp4) && !bucketed) return FPS_ERR_UNSUPPORTED;   // tensor tiles need popcount buckets
  size_t need = lay.bytes + (want_fp8 ? tc_operand_bytes(kTcFp8, lay.n_tiles) : 0) +
                (want_fp4 ? tc_operand_bytes(kTcFp4, lay.n_tiles) : 0);
  if (d->hbm_budget_bytes && need > d->hbm_budget_bytes) return FPS_ERR_BUDGET;

  Library* L = new (std::nothrow) Library();
  if (!L) return FPS_ERR_NOMEM;
  L->device = d->device;
  L->n = n;
  L->n_tiles = lay.n_tiles;
  L->bucketed = bucketed ? 1 : 0;
  if (cids) L->cids.assign(cids, cids + n);
  for (int b = 0; b < kNumBuckets; ++b) L->bucket_count[b] = bucketed ? lay.count[b] : 0;

  DeviceGuard g(d->device);
  if (!g.ok) {
    delete L;
    return FPS_ERR_CUDA;
  }
  if (cudaDeviceGetAttribute(&L->num_sms, cudaDevAttrMultiProcessorCount, d->device) != cudaSuccess) {
    cudaGetLastError();
    delete L;
    return FPS_ERR_CUDA;
  }

  // host staging of the tiled layout
  std::vector<uint64_t> words;
  std::vector<int32_t> perm;
  try {
    words.assign(static_cast<size_t>(lay.n_tiles) * kTile * kWords, 0);
    perm.assign(static_cast<size_t>(lay.n_tiles) * kTile, -1);
  } catch (const std::bad_alloc&) {
    delete L;
    return FPS_ERR_NOMEM;
  }
  auto place = [&](int64_t i, int64_t p) {
    int64_t t = p / kTile, r = p % kTile;
    uint64_t* base = &words[static_cast<size_t>(t) * kTile * kWords];
    base[r] = packed[3 * i];
    base[kTile + r] = packed[3 * i + 1];
    base[2 * kTile + r] = packed[3 * i + 2];
    perm[p] = static_cast<int32_t>(i);
  };
  const int T = hw_threads();
  if (bucketed) {
    // stable counting sort by popcount: per-thread offsets keep index order inside a bucket
    // parallel_for hands thread t the same index range in both passes
    std::vector<std::vector<int64_t>> cnt(T, std::vector<int64_t>(kNumBuckets, 0));
    parallel_for(n, T, [&](int t, int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i) cnt[t][popc[i]] += 1;
    });
    std::vector<std::vector<int64_t>> off(T, std::vector<int64_t>(kNumBuckets, 0));
    for (int b = 0; b < kNumBuckets; ++b) {
      int64_t run = lay.pos_base[b];
      for (int t = 0; t < T; ++t) {
        off[t][b] = run;
        run += cnt[t][b];
      }
    }
    parallel_for(n, T, [&](int t, int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i) place(i, off[t][popc[i]]++);
    });
  } else {
    parallel_for(n, T, [&](int, int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i) place(i, i);
    });
  }
  std::vector<int32_t> tile_off(kNumBuckets + 1, 0), bcount(kNumBuckets + 1, 0);
  for (int b = 0; b <= kNumBuckets; ++b) tile_off[b] = static_cast<int32_t>(lay.pos_base[b] / kTile);
  for (int b = 0; b < kNumBuckets; ++b) bcount[b] = static_cast<int32_t>(lay.count[b]);

  void *dw = nullptr, *dp = nullptr, *dto = nullptr, *dbc = nullptr;
  fps_status st = dev_alloc(L, &dw, words.size() * 8);
  if (st == FPS_OK) st = dev_alloc(L, &dp, perm.size() * 4);
  if (st == FPS_OK) st = dev_alloc(L, &dto, tile_off.size() * 4);
  if (st == FPS_OK) st = dev_alloc(L, &dbc, bcount.size() * 4);
  if (st == FPS_OK) {
    if (cudaMemcpy(dw, words.data(), words.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dp, perm.data(), perm.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dto, tile_off.data(), tile_off.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dbc, bcount.data(), bcount.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      st = FPS_ERR_CUDA;
    }
  }
  if (st != FPS_OK) {
    free_library(L);
    return st;
  }
  L->dev.words = static_cast<const uint64_t*>(dw);
  L->dev.perm = static_cast<const int32_t*>(dp);
  L->dev.tile_off = static_cast<const int32_t*>(dto);
  L->dev.bcount = static_cast<const int32_t*>(dbc);
  L->dev.n = n;
  L->dev.n_tiles = lay.n_tiles;
  L->dev.bucketed = L->bucketed;
  for (int fmt : {kTcFp8, kTcFp4}) {
    if (!(fmt == kTcFp8 ? want_fp8 : want_fp4)) continue;
    void* op = nullptr;
    st = dev_alloc(L, &op, tc_operand_bytes(fmt, lay.n_tiles));
    if (st == FPS_OK && (tc_pack_library(fmt, L->dev, static_cast<uint8_t*>(op), nullptr) != cudaSuccess ||
                         cudaDeviceSynchronize() != cudaSuccess)) {
      cudaGetLastError();
      st = FPS_ERR_CUDA;
    }
    if (st != FPS_OK) {
      free_library(L);
      return st;
    }
    (fmt == kTcFp8 ? L->tc_fp8 : L->tc_fp4) = static_cast<uint8_t*>(op);
  }
  *out = L;
  return FPS_OK;
}

// ------------------------------------------------------------------ workspaces
fps_status get_workspace(Library* L, cudaStream_t s, Workspace** out) {
  std::lock_guard<std::mutex> lock(L->mu);
  auto it = L->ws.find(s);
  if (it != L->ws.end()) {
    *out = it->second;
    return FPS_OK;
  }
  Workspace* w = new (std::nothrow) Workspace();
  if (!w) return FPS_ERR_NOMEM;
  w->cand_cap = scan_cand_capacity(L->num_sms);
  size_t st_bytes = (sizeof(ScanState) + 255) / 256 * 256;
  size_t io_bytes = (sizeof(HostIO) + 255) / 256 * 256;
  size_t bytes = 2 * st_bytes + io_bytes + 2 * w->cand_cap * sizeof(unsigned long long);
  if (cudaMalloc(&w->block, bytes) != cudaSuccess || cudaMallocHost(&w->io_host, sizeof(HostIO)) != cudaSuccess) {
    cudaGetLastError();
    if (w->block) cudaFree(w->block);
    delete w;
    return FPS_ERR_CUDA;
  }
  char* b = static_cast<char*>(w->block);
  w->st = reinterpret_cast<ScanState*>(b);
  w->io = reinterpret_cast<HostIO*>(b + st_bytes);
  w->cand = reinterpret_cast<unsigned long long*>(b + st_bytes + io_bytes);
  w->st2 = reinterpret_cast<ScanState*>(b + st_bytes + io_bytes + w->cand_cap * sizeof(unsigned long long));
  w->cand2 = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(w->st2) + st_bytes);
  if (cudaMemsetAsync(w->io, 0, sizeof(HostIO), s) != cudaSuccess || scan_state_init(w->st, s) != cudaSuccess ||
      scan_state_init(w->st2, s) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(w->block);
    cudaFreeHost(w->io_host);
    delete w;
    return FPS_ERR_CUDA;
  }
  L->ws[s] = w;
  *out = w;
  return FPS_OK;
}

fps_status check_k(int k) {
  if (k < 0) return FPS_ERR_INVALID_ARG;
  if (k > kKMax) return FPS_ERR_UNSUPPORTED;
  return FPS_OK;
}

// Read and clear the device error word of a workspace (stream already synchronised).
fps_status take_device_error(Workspace* w, cudaStream_t s) {
  uint32_t e = 0;
  if (cudaMemcpyAsync(&e, &w->io->err, sizeof e, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  if (!e) return FPS_OK;
  // a failed scan may leave its state dirty: clear error word and scan state
  if (cudaMemsetAsync(&w->io->err, 0, sizeof(uint32_t), s) != cudaSuccess || scan_state_init(w->st, s) != cudaSuccess ||
      scan_state_init(w->st2, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  if (e & DEVERR_TIMEOUT) return FPS_ERR_TIMEOUT;
  return FPS_ERR_OVERFLOW_INTERNAL;
}

double opt_timeout(const fps_search_opts* o) { return (o && o->timeout_s > 0) ? o->timeout_s : 2.0; }

// Host result slots [from, k) that no record fills hold -1 (index and distance).
void fill_unused(int32_t* out_index, int32_t* out_dist, int from, int k) {
  for (int i = from; i < k; ++i) {
    out_index[i] = -1;
    out_dist[i] = -1;
  }
}

// Host-IO single search through the workspace staging buffers.
fps_status search_one_host(Library* L, const uint64_t q[3], int k, int32_t* out_index, int32_t* out_dist,
                           int32_t* out_count, const fps_search_opts* opts, cudaStream_t s) {
  if (L->n == 0 || k == 0) {
    fill_unused(out_index, out_dist, 0, k);
    *out_count = 0;
    return FPS_OK;
  }
  Workspace* w = nullptr;
  fps_status st = get_workspace(L, s, &w);
  if (st != FPS_OK) return st;
  std::memcpy(w->io_host->query, q, 3 * sizeof(uint64_t));
  const int k_eff = static_cast<int>(std::min<int64_t>(k, L->n));
  if (cudaMemcpyAsync(w->io->query, w->io_host->query, 4 * sizeof(uint64_t), cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  // indices in res[0, k), distances in res[k, 2k) (the kernel writes -1 past k_eff)
  if (launch_scan_single(L->dev, w->io->query, k, w->st, w->cand, w->io->res, w->io->res + k, &w->io->count,
                         &w->io->err, L->num_sms, opt_timeout(opts), s) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  size_t bytes = offsetof(HostIO, res) - offsetof(HostIO, err) + 2 * sizeof(int32_t) * k;
  if (cudaMemcpyAsync(&w->io_host->err, &w->io->err, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  if (w->io_host->err) return take_device_error(w, s);
  const int c = w->io_host->count;
  std::memcpy(out_index, w->io_host->res, sizeof(int32_t) * c);
  std::memcpy(out_dist, w->io_host->res + k, sizeof(int32_t) * c);
  fill_unused(out_index, out_dist, c, k);
  *out_count = c;
  if (opts && opts->stats) {
    opts->stats->queries = 1;
    opts->stats->fallbacks = 0;
    opts->stats->device_fallbacks = 0;
    opts->stats->candidates = 0;
    opts->stats->path_used = FPS_PATH_POPC;
  }
  return FPS_OK;
}


// Grow a device (or pinned host) block to at least `need` bytes.  cudaFree waits for the
// device, so work still reading the old block has finished before it goes.
fps_status grow_block(void** block, size_t* have, size_t need, bool host) {
  if (*have >= need) return FPS_OK;
  if (*block) {
    if (host)
      cudaFreeHost(*block);
    else
      cudaFree(*block);
  }
  *block = nullptr;
  *have = 0;
  if ((host ? cudaMallocHost(block, need) : cudaMalloc(block, need)) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  *have = need;
  return FPS_OK;
}

// Grow the per-stream batch staging (device block and pinned host block).
fps_status batch_staging(Workspace* w, size_t dev_bytes, size_t host_bytes) {
  if (w->batch_bytes < dev_bytes) {
    if (w->batch_block) cudaFree(w->batch_block);
    w->batch_block = nullptr;
    w->batch_bytes = 0;
    if (cudaMalloc(&w->batch_block, dev_bytes) != cudaSuccess) {
      cudaGetLastError();
      return FPS_ERR_CUDA;
    }
    w->batch_bytes = dev_bytes;
  }
  if (w->batch_host_bytes < host_bytes) {
    if (w->batch_host) cudaFreeHost(w->batch_host);
    w->batch_host = nullptr;
    w->batch_host_bytes = 0;
    if (cudaMallocHost(&w->batch_host, host_bytes) != cudaSuccess) {
      cudaGetLastError();
      return FPS_ERR_CUDA;
    }
    w->batch_host_bytes = host_bytes;
  }
  return FPS_OK;
}

// Queries one after another through the single-query kernel (FPS_PATH_POPC); every
// search still streams the whole (unpruned) library.  All queries are in device memory
// before the first launch, so the launches after the first are programmatic dependents of
// their predecessor: search i+1 streams on the SMs that search i has released while
// search i merges.  Consecutive searches alternate between the workspace's two scan
// states; search i+2 reuses search i's state and can only start once search i+1's merge
// has waited for search i to finish, so a state is never shared by running grids.
fps_status batch_sequential(Library* L, Workspace* w, const uint64_t* dq, int Q, const int32_t* k, const int64_t* off,
                            int32_t* di, int32_t* dd, int32_t* dc, double tmo, cudaStream_t s) {
  for (int q = 0; q < Q; ++q) {   // empty results first, so the scan launches stay adjacent
    if (k[q] == 0 || L->n == 0) {
      // count 0; with no records every slot up to k holds -1 (all bytes 0xFF)
      if (cudaMemsetAsync(dc + q, 0, sizeof(int32_t), s) != cudaSuccess ||
          (k[q] > 0 && (cudaMemsetAsync(di + off[q], 0xFF, sizeof(int32_t) * k[q], s) != cudaSuccess ||
                        cudaMemsetAsync(dd + off[q], 0xFF, sizeof(int32_t) * k[q], s) != cudaSuccess))) {
        cudaGetLastError();
        return FPS_ERR_CUDA;
      }
    }
  }
  int launched = 0;
  for (int q = 0; q < Q; ++q) {
    if (k[q] == 0 || L->n == 0) continue;
    ScanState* st = (launched & 1) ? w->st2 : w->st;
    unsigned long long* cand = (launched & 1) ? w->cand2 : w->cand;
    if (launch_scan_single(L->dev, dq + 3 * q, k[q], st, cand, di + off[q], dd + off[q], dc + q, &w->io->err,
                           L->num_sms, tmo, s, launched > 0) != cudaSuccess) {
      cudaGetLastError();
      return FPS_ERR_CUDA;
    }
    ++launched;
  }
  return FPS_OK;
}

// Sub-allocation of one staging block: each section 256-byte aligned.
struct Carve {
  size_t at = 0;
  size_t take(size_t bytes) {
    size_t p = at;
    at += (bytes + 255) / 256 * 256;
    return p;
  }
};

// Candidate capacity of a query: 32 k + 8192 keys, never more than the library.
int64_t batch_cap(int k, int64_t n) {
  if (k <= 0) return 0;
  int64_t c = 32 * static_cast<int64_t>(k) + 8192;
  return c < n ? c : n;
}

// Many queries per launch with the batched kernels (pilot bound, scan, per-query select).
// Byte layout of one batch's staging block (device), mirrored for the parts that
// travel (the plan region goes host -> device, the output region back).
struct BatchLayout {
  size_t d_q, d_k, d_co, d_oo, d_tau, plan_end;
  size_t d_thr, d_hist, d_work, d_oi, d_od, d_oc, d_cnt, d_cand, out_begin, out_end, d_qop, bytes;
};

// qop_bytes: the tensor-core query operand (0 for the popcount batch)
BatchLayout batch_layout(int Q, int64_t total, int64_t cand_keys, bool dev_io, bool learned, size_t qop_bytes) {
  BatchLayout l{};
  Carve dv;
  l.d_q = dv.take(dev_io ? 0 : sizeof(uint64_t) * 3 * Q);
  l.d_k = dv.take(sizeof(int32_t) * Q);
  l.d_co = dv.take(sizeof(int64_t) * (Q + 1));
  l.d_oo = dv.take(sizeof(int64_t) * (Q + 1));
  l.d_tau = dv.take(learned && !dev_io ? sizeof(float) * Q : 0);
  l.plan_end = dv.at;
  l.d_thr = dv.take(sizeof(uint32_t) * Q);
  l.d_hist = dv.take(sizeof(uint32_t) * 168 * Q);
  l.d_work = dv.take(sizeof(uint32_t));
  l.d_oi = dv.take(dev_io ? 0 : sizeof(int32_t) * total);
  l.d_od = dv.take(dev_io ? 0 : sizeof(int32_t) * total);
  l.d_oc = dv.take(sizeof(int32_t) * Q);
  l.d_cnt = dv.take(sizeof(uint32_t) * Q);   // copied back with the counts (statistics)
  l.d_cand = dv.take(sizeof(unsigned long long) * static_cast<size_t>(cand_keys));
  l.out_begin = dev_io ? l.d_oc : l.d_oi;
  l.out_end = l.d_cand;
  l.d_qop = dv.take(qop_bytes);
  l.bytes = dv.at;
  return l;
}

std::vector<int64_t> batch_cand_offsets(const int32_t* k, int Q, int64_t n) {
  std::vector<int64_t> coff(static_cast<size_t>(Q) + 1, 0);
  for (int q = 0; q < Q; ++q) coff[q + 1] = coff[q] + batch_cap(k[q], n);
  return coff;
}

// Host side of the plan region: queries (host form), k, candidate and output offsets, predicted bounds.
void fill_plan(char* hb, const BatchLayout& l, const uint64_t* queries, int Q, const int32_t* k,
               const std::vector<int64_t>& coff, const int64_t* off, const float* tau, bool dev_io) {
  if (!dev_io) std::memcpy(hb + l.d_q, queries, sizeof(uint64_t) * 3 * Q);
  std::memcpy(hb + l.d_k, k, sizeof(int32_t) * Q);
  std::memcpy(hb + l.d_co, coff.data(), sizeof(int64_t) * (Q + 1));
  std::memcpy(hb + l.d_oo, off, sizeof(int64_t) * (Q + 1));
  if (tau && !dev_io) std::memcpy(hb + l.d_tau, tau, sizeof(float) * Q);
}

BatchDev batch_dev(char* db, const BatchLayout& l, int Q, const uint64_t* dev_queries, int32_t* dev_oi,
                   int32_t* dev_od, uint32_t* err) {
  BatchDev b{};
  b.Q = Q;
  b.queries = dev_queries ? dev_queries : reinterpret_cast<const uint64_t*>(db + l.d_q);
  b.k = reinterpret_cast<const int32_t*>(db + l.d_k);
  b.cand_off = reinterpret_cast<const int64_t*>(db + l.d_co);
  b.out_off = reinterpret_cast<const int64_t*>(db + l.d_oo);
  b.thr = reinterpret_cast<uint32_t*>(db + l.d_thr);
  b.cnt = reinterpret_cast<uint32_t*>(db + l.d_cnt);
  b.hist = reinterpret_cast<uint32_t*>(db + l.d_hist);
  b.cand = reinterpret_cast<unsigned long long*>(db + l.d_cand);
  b.out_idx = dev_oi ? dev_oi : reinterpret_cast<int32_t*>(db + l.d_oi);
  b.out_dist = dev_od ? dev_od : reinterpret_cast<int32_t*>(db + l.d_od);
  b.out_count = reinterpret_cast<int32_t*>(db + l.d_oc);
  b.err = err;
  return b;
}

bool is_tc_path(int path) { return path == FPS_PATH_TC_FP8 || path == FPS_PATH_TC_FP4; }
int tc_fmt_of(int path) { return path == FPS_PATH_TC_FP4 ? kTcFp4 : kTcFp8; }
const uint8_t* tc_operand_of(const Library* L, int path) {
  return path == FPS_PATH_TC_FP4 ? L->tc_fp4 : (path == FPS_PATH_TC_FP8 ? L->tc_fp8 : nullptr);
}
size_t qop_bytes_of(int path, int Q) { return is_tc_path(path) ? tc_query_operand_bytes(tc_fmt_of(path), Q) : 0; }
// The tile parameter a batched path runs with (param <= 0: its default).
int tile_param_of(int path, int param) {
  if (param > 0) return param;
  if (is_tc_path(path)) return tc_default_chunk(tc_fmt_of(path));
  return path == FPS_PATH_POPC_BATCH ? kPopcBatchDefaultQB : 0;
}

// The device work of one batch: bounds (sampled or predicted), scan, per-query select.
// path: FPS_PATH_POPC_BATCH, FPS_PATH_TC_FP8 or FPS_PATH_TC_FP4; param: its tile parameter.
cudaError_t enqueue_batch(Library* L, const BatchDev& b, char* db, const BatchLayout& l, int path, int param,
                          const float* tau_dev, double tmo, cudaStream_t s) {
  cudaError_t ce = batch_prepare(L->dev, b, tau_dev ? 0 : 1, s);
  if (ce == cudaSuccess && tau_dev) ce = batch_thr_from_tau(b, tau_dev, s);
  if (ce == cudaSuccess) {
    if (is_tc_path(path)) {
      const int fmt = tc_fmt_of(path);
      uint8_t* qop = reinterpret_cast<uint8_t*>(db + l.d_qop);
      ce = tc_pack_queries(fmt, b.queries, b.Q, qop, s);
      if (ce == cudaSuccess) ce = tc_scan(fmt, L->dev, b, tc_operand_of(L, path), qop, L->num_sms, param, tmo, s);
    } else {
      ce = batch_scan_popc(L->dev, b, L->num_sms, reinterpret_cast<uint32_t*>(db + l.d_work), param, s);
    }
  }
  if (ce == cudaSuccess) ce = batch_select(L->dev, b, s);
  return ce;
}

// After the output region is back on the host: statistics, exact re-runs of
// queries reported -2 (candidate overflow or a predicted bound too low), and
// the copy of host-form results into the caller's arrays.
fps_status finish_batch(Library* L, Workspace* w, const char* hb, const char* db, const BatchLayout& l,
                        const uint64_t* queries, int Q, const int32_t* k, const int64_t* off, int32_t* out_index,
                        int32_t* out_dist, int32_t* out_count, const fps_search_opts* opts, bool dev_io,
                        cudaStream_t s, int64_t* n_fallback) {
  const int32_t* hc = reinterpret_cast<const int32_t*>(hb + l.d_oc);
  const uint32_t* hcnt = reinterpret_cast<const uint32_t*>(hb + l.d_cnt);
  int64_t accepted = 0;
  for (int q = 0; q < Q; ++q) accepted += hcnt[q];
  if (opts && opts->stats) opts->stats->candidates = accepted;
  const double tmo = opt_timeout(opts);
  int64_t nf = 0;
  fps_status st = FPS_OK;
  for (int q = 0; q < Q; ++q) {
    if (hc[q] != -2) continue;
    ++nf;
    if (!dev_io) {
      int32_t c = 0;
      st = search_one_host(L, queries + 3 * q, k[q], out_index + off[q], out_dist + off[q], &c, opts, s);
      if (st != FPS_OK) return st;
      out_count[q] = c;
    }
  }
  if (dev_io) {
    if (cudaMemcpyAsync(out_count, db + l.d_oc, sizeof(int32_t) * Q, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
      cudaGetLastError();
      return FPS_ERR_CUDA;
    }
    // the fallback searches (if any) write their own counts after this copy
    for (int q = 0; q < Q && nf > 0; ++q) {
      if (hc[q] != -2) continue;
      if (launch_scan_single(L->dev, queries + 3 * q, k[q], w->st, w->cand, out_index + off[q], out_dist + off[q],
                             out_count + q, &w->io->err, L->num_sms, tmo, s) != cudaSuccess) {
        cudaGetLastError();
        return FPS_ERR_CUDA;
      }
    }
  } else {
    const int32_t* hi = reinterpret_cast<const int32_t*>(hb + l.d_oi);
    const int32_t* hd = reinterpret_cast<const int32_t*>(hb + l.d_od);
    for (int q = 0; q < Q; ++q) {
      if (hc[q] == -2) continue;
      out_count[q] = hc[q];
      std::memcpy(out_index + off[q], hi + off[q], sizeof(int32_t) * hc[q]);
      std::memcpy(out_dist + off[q], hd + off[q], sizeof(int32_t) * hc[q]);
      fill_unused(out_index + off[q], out_dist + off[q], hc[q], k[q]);
    }
  }
  *n_fallback = nf;
  return FPS_OK;
}

// Many queries per launch with the batched kernels (bounds, scan, per-query select).
fps_status batch_kernels(Library* L, Workspace* w, int path, int param, const uint64_t* queries, int Q,
                         const int32_t* k, const int64_t* off, int64_t total, int32_t* out_index, int32_t* out_dist,
                         int32_t* out_count, const fps_search_opts* opts, bool dev_io, cudaStream_t s,
                         int64_t* n_fallback, const float* learned_tau) {
  const bool learned = learned_tau != nullptr;
  std::vector<int64_t> coff = batch_cand_offsets(k, Q, L->n);
  const BatchLayout l = batch_layout(Q, total, coff[Q], dev_io, learned, qop_bytes_of(path, Q));
  fps_status st = batch_staging(w, l.bytes, l.plan_end > l.out_end ? l.plan_end : l.out_end);
  if (st != FPS_OK) return st;
  char* db = static_cast<char*>(w->batch_block);
  char* hb = static_cast<char*>(w->batch_host);
  fill_plan(hb, l, queries, Q, k, coff, off, learned_tau, dev_io);
  if (cudaMemcpyAsync(db, hb, l.plan_end, cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  const BatchDev b = batch_dev(db, l, Q, dev_io ? queries : nullptr, dev_io ? out_index : nullptr,
                               dev_io ? out_dist : nullptr, &w->io->err);
  const float* tau_dev = learned ? (dev_io ? learned_tau : reinterpret_cast<const float*>(db + l.d_tau)) : nullptr;
  if (enqueue_batch(L, b, db, l, path, param, tau_dev, opt_timeout(opts), s) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  // results (host form) or just the counts (device form) come back once
  if (cudaMemcpyAsync(hb + l.out_begin, db + l.out_begin, l.out_end - l.out_begin, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  st = take_device_error(w, s);
  if (st != FPS_OK) return st;
  return finish_batch(L, w, hb, db, l, queries, Q, k, off, out_index, out_dist, out_count, opts, dev_io, s,
                      n_fallback);
}

// Queries one after another through the single-query scan (FPS_PATH_POPC), host or device form.
fps_status run_sequential(Library* L, Workspace* w, const uint64_t* queries, int Q, const int32_t* k,
                          const int64_t* off, int64_t total, int32_t* out_index, int32_t* out_dist,
                          int32_t* out_count, double tmo, bool dev_io, cudaStream_t s) {
  if (dev_io) return batch_sequential(L, w, queries, Q, k, off, out_index, out_dist, out_count, tmo, s);
  // device staging: [queries Q*3][index total][dist total][count Q]; host mirror of the same
  const size_t qb = static_cast<size_t>(Q) * 3 * sizeof(uint64_t);
  const size_t rb = static_cast<size_t>(total) * sizeof(int32_t);
  const size_t cb = static_cast<size_t>(Q) * sizeof(int32_t);
  const size_t bytes = qb + 2 * rb + cb;
  fps_status st = batch_staging(w, bytes, bytes);
  if (st != FPS_OK) return st;
  char* hb = static_cast<char*>(w->batch_host);
  char* db = static_cast<char*>(w->batch_block);
  std::memcpy(hb, queries, qb);
  if (cudaMemcpyAsync(db, hb, qb, cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  int32_t* di = reinterpret_cast<int32_t*>(db + qb);
  int32_t* dd = reinterpret_cast<int32_t*>(db + qb + rb);
  int32_t* dc = reinterpret_cast<int32_t*>(db + qb + 2 * rb);
  st = batch_sequential(L, w, reinterpret_cast<const uint64_t*>(db), Q, k, off, di, dd, dc, tmo, s);
  if (st != FPS_OK) return st;
  if (cudaMemcpyAsync(hb + qb, db + qb, 2 * rb + cb, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  st = take_device_error(w, s);
  if (st != FPS_OK) return st;
  const int32_t* hi = reinterpret_cast<const int32_t*>(hb + qb);
  const int32_t* hd = reinterpret_cast<const int32_t*>(hb + qb + rb);
  const int32_t* hc = reinterpret_cast<const int32_t*>(hb + qb + 2 * rb);
  for (int q = 0; q < Q; ++q) {
    out_count[q] = hc[q];
    std::memcpy(out_index + off[q], hi + off[q], sizeof(int32_t) * hc[q]);
    std::memcpy(out_dist + off[q], hd + off[q], sizeof(int32_t) * hc[q]);
    fill_unused(out_index + off[q], out_dist + off[q], hc[q], k[q]);
  }
  return FPS_OK;
}

bool path_available(const Library* L, int path) {
  if (path == FPS_PATH_POPC || path == FPS_PATH_POPC_BATCH) return true;
  return tc_operand_of(L, path) != nullptr;
}

// One call on a resolved path (FPS_PATH_POPC, _POPC_BATCH, _TC_FP8 or _TC_FP4) with its
// tile parameter; *n_fallback counts the queries re-run by the exact single-query scan.
fps_status run_path(Library* L, Workspace* w, int path, int param, const uint64_t* queries, int Q, const int32_t* k,
                    const int64_t* off, int64_t total, int32_t* out_index, int32_t* out_dist, int32_t* out_count,
                    const fps_search_opts* opts, bool dev_io, cudaStream_t s, const float* tau,
                    int64_t* n_fallback) {
  *n_fallback = 0;
  if (path == FPS_PATH_POPC)
    return run_sequential(L, w, queries, Q, k, off, total, out_index, out_dist, out_count, opt_timeout(opts), dev_io,
                          s);
  return batch_kernels(L, w, path, param, queries, Q, k, off, total, out_index, out_dist, out_count, opts, dev_io, s,
                       n_fallback, tau);
}

std::string device_name(int device) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  return prop.name;
}

// Autotuner (FPS_PATH_AUTO): every batched kernel the library holds an operand for at
// its default tile shape (and, for at most 64 queries, the sequential single-query
// scan), then the fastest kernel at its other tile shapes; each run is the whole call
// and returns the same exact results, so the call's outputs are those of the last run.
fps_status autotune(Library* L, Workspace* w, const std::string& cls, const uint64_t* queries, int Q, const int32_t* k,
                    const int64_t* off, int64_t total, int32_t* out_index, int32_t* out_dist, int32_t* out_count,
                    const fps_search_opts* opts, bool dev_io, cudaStream_t s, const float* tau,
                    Library::Choice* chosen, int64_t* n_fallback) {
  std::vector<Library::Choice> cands;
  if (Q <= 64) cands.push_back({FPS_PATH_POPC, 0});
  for (int p : {FPS_PATH_POPC_BATCH, FPS_PATH_TC_FP8, FPS_PATH_TC_FP4})
    if (path_available(L, p)) cands.push_back({p, tile_param_of(p, 0)});
  double best_ms = 0.0;
  auto timed = [&](const Library::Choice& c) -> fps_status {
    int64_t nf = 0;
    auto t0 = std::chrono::steady_clock::now();
    fps_status st = run_path(L, w, c.path, c.param, queries, Q, k, off, total, out_index, out_dist, out_count, opts,
                             dev_io, s, tau, &nf);
    if (st == FPS_OK && cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      st = FPS_ERR_CUDA;
    }
    if (st != FPS_OK) return st;
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (chosen->path == 0 || ms < best_ms) {
      *chosen = c;
      best_ms = ms;
      *n_fallback = nf;
    }
    return FPS_OK;
  };
  *chosen = Library::Choice{};
  for (const auto& c : cands) {
    fps_status st = timed(c);
    if (st != FPS_OK) return st;
  }
  std::vector<int> shapes;
  if (chosen->path == FPS_PATH_POPC_BATCH) shapes = {32, 128};
  if (is_tc_path(chosen->path)) {
    const int d = tc_default_chunk(tc_fmt_of(chosen->path));
    shapes = {d / 2, 2 * d};
  }
  const int best_path = chosen->path;
  for (int p : shapes) {
    fps_status st = timed({best_path, p});
    if (st != FPS_OK) return st;
  }
  {
    std::lock_guard<std::mutex> lock(L->mu);
    L->tuned[cls] = *chosen;
  }
  const char* cache = std::getenv("FPS_TUNE_CACHE");
  if (cache && *cache) tune_cache_put(cache, device_name(L->device).c_str(), L->n, cls, chosen->path, chosen->param,
                                      best_ms);
  return FPS_OK;
}

fps_status search_batch_impl(Library* L, const uint64_t* queries, int Q, const int32_t* k, const int64_t* off,
                             int64_t total, int32_t* out_index, int32_t* out_dist, int32_t* out_count,
                             const fps_search_opts* opts, bool dev_io, cudaStream_t s) {
  if (Q == 0) return FPS_OK;
  Workspace* w = nullptr;
  fps_status st = get_workspace(L, s, &w);
  if (st != FPS_OK) return st;
  int path = opts ? opts->path : FPS_PATH_AUTO;
  const float* tau = nullptr;
  if (path == FPS_PATH_LEARNED) {
    if (!opts->tau) return FPS_ERR_INVALID_ARG;
    tau = opts->tau;                      // predicted bounds replace the pilot; the scan itself is tuned below
    path = FPS_PATH_AUTO;
  }
  if (!dev_io)
    for (int q = 0; q < Q; ++q)
      if (queries[3 * q + 2] >> (kBits - 128)) return FPS_ERR_INVALID_ARG;
  if (path != FPS_PATH_AUTO && path != FPS_PATH_POPC && path != FPS_PATH_POPC_BATCH && !is_tc_path(path))
    return FPS_ERR_UNSUPPORTED;   // FPS_PATH_TC_I8: sm_103a has no kind::i8
  // no records: every path answers count 0 and -1 in each query's k slots, which the
  // sequential path writes without launching a scan
  if (L->n == 0) path = FPS_PATH_POPC;
  int param = 0;
  int64_t nf = 0;
  if (path == FPS_PATH_AUTO) {
    int kmax = 0;
    for (int q = 0; q < Q; ++q) kmax = std::max(kmax, k[q]);
    const std::string cls = tune_class_name(Q, kmax, tau != nullptr);
    Library::Choice c{};
    bool known = false;
    {
      std::lock_guard<std::mutex> lock(L->mu);
      auto it = L->tuned.find(cls);
      if (it != L->tuned.end()) {
        c = it->second;
        known = true;
      }
    }
    const char* cache = std::getenv("FPS_TUNE_CACHE");
    if (!known && cache && *cache) {
      int cp = 0, cparam = 0;
      double ms = 0.0;
      if (tune_cache_get(cache, device_name(L->device).c_str(), L->n, cls, &cp, &cparam, &ms) &&
          path_available(L, cp) && (cp == FPS_PATH_POPC ? Q <= 64 : cp != FPS_PATH_AUTO)) {
        c = {cp, cparam};
        known = true;
        std::lock_guard<std::mutex> lock(L->mu);
        L->tuned[cls] = c;
      }
    }
    if (!known) {
      st = autotune(L, w, cls, queries, Q, k, off, total, out_index, out_dist, out_count, opts, dev_io, s, tau, &c,
                    &nf);
      if (st != FPS_OK) return st;
      if (opts && opts->stats) {
        opts->stats->queries = Q;
        opts->stats->fallbacks = nf;
        opts->stats->device_fallbacks = 0;
        opts->stats->path_used = c.path;
        opts->stats->tile_param = c.param;
      }
      return FPS_OK;
    }
    path = c.path;
    param = c.param;
  }
  if (!path_available(L, path)) return FPS_ERR_UNSUPPORTED;
  param = path == FPS_PATH_POPC ? 0 : tile_param_of(path, param);
  st = run_path(L, w, path, param, queries, Q, k, off, total, out_index, out_dist, out_count, opts, dev_io, s, tau,
                &nf);
  if (st == FPS_OK && opts && opts->stats) {
    opts->stats->queries = Q;
    opts->stats->fallbacks = nf;
    opts->stats->device_fallbacks = 0;
    if (path == FPS_PATH_POPC) opts->stats->candidates = 0;
    opts->stats->path_used = path;
    opts->stats->tile_param = param;
  }
  return st;
}

// A batch whose shape (Q, k, path) is fixed: own buffers and one captured CUDA
// graph (plan copy in, bounds, scan, select, results and error word out).
struct BatchPlan {
  Library* L = nullptr;
  int Q = 0;
  int path = FPS_PATH_POPC_BATCH, param = 0;   // batched kernel and its tile parameter
  bool learned = false;
  bool empty = false;        // library without records: no device state, results written on the host
  std::vector<int32_t> k;
  std::vector<int64_t> off, coff;
  int64_t total = 0;
  BatchLayout lay{};
  char* db = nullptr;        // device block
  char* hb = nullptr;        // pinned host mirror of the plan and output regions
  uint32_t* err = nullptr;   // device error word
  uint32_t* err_host = nullptr;
  cudaStream_t cap = nullptr;
  cudaStream_t cap_body = nullptr;   // captures the fallback loop's body
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // device-side exact fallback: its own scan state, candidate keys and search slot
  char* fb = nullptr;
  ScanState* fb_st = nullptr;
  ScanSlot* fb_slot = nullptr;
  unsigned long long* fb_cand = nullptr;
  uint32_t* fb_count_host = nullptr;  // queries the graph re-ran (pinned)
};

void free_plan(BatchPlan* P) {
  if (!P) return;
  DeviceGuard g(P->L ? P->L->device : 0);
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  if (P->cap) cudaStreamDestroy(P->cap);
  if (P->cap_body) cudaStreamDestroy(P->cap_body);
  if (P->fb) cudaFree(P->fb);
  if (P->fb_count_host) cudaFreeHost(P->fb_count_host);
  if (P->db) cudaFree(P->db);
  if (P->hb) cudaFreeHost(P->hb);
  if (P->err) cudaFree(P->err);
  if (P->err_host) cudaFreeHost(P->err_host);
  delete P;
}

// The exact fallback inside the graph: a first pick, then a WHILE node whose body scans the
// picked query (indirect launch of the single-query scan) and picks the next one, until no
// query with count -2 is left.  Captured on s (being captured); the body on P->cap_body.
cudaError_t plan_capture_fallback(BatchPlan* P, double tmo, cudaStream_t s) {
  const uint64_t* dq = reinterpret_cast<const uint64_t*>(P->db + P->lay.d_q);
  const int32_t* dk = reinterpret_cast<const int32_t*>(P->db + P->lay.d_k);
  const int64_t* doo = reinterpret_cast<const int64_t*>(P->db + P->lay.d_oo);
  int32_t* di = reinterpret_cast<int32_t*>(P->db + P->lay.d_oi);
  int32_t* dd = reinterpret_cast<int32_t*>(P->db + P->lay.d_od);
  int32_t* dc = reinterpret_cast<int32_t*>(P->db + P->lay.d_oc);
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) e = launch_fallback_pick(dq, dk, doo, di, dd, dc, P->Q, P->fb_slot, true, h, s);
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t loop = nullptr;
  e = cudaGraphAddNode(&loop, g, deps, nullptr, nd, &np);
  if (e != cudaSuccess) return e;
  cudaGraph_t body = np.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(P->cap_body, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t e2 = launch_scan_indirect(P->L->dev, P->fb_slot, P->fb_st, P->fb_cand, P->err, P->L->num_sms, tmo,
                                        P->cap_body);
  if (e2 == cudaSuccess) e2 = launch_fallback_pick(dq, dk, doo, di, dd, dc, P->Q, P->fb_slot, false, h, P->cap_body);
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(P->cap_body, &captured);
  if (e2 != cudaSuccess) return e2;
  if (e != cudaSuccess) return e;
  return cudaStreamUpdateCaptureDependencies(s, &loop, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// Enqueue the whole batch on stream s (once eagerly, then under capture).  The device-side
// fallback needs a graph (its loop is a conditional node), so only the captured run has it;
// the eager run's results are discarded.
cudaError_t plan_enqueue(BatchPlan* P, double tmo, cudaStream_t s, bool captured) {
  const BatchDev b = batch_dev(P->db, P->lay, P->Q, nullptr, nullptr, nullptr, P->err);
  const float* tau_dev = P->learned ? reinterpret_cast<const float*>(P->db + P->lay.d_tau) : nullptr;
  cudaError_t e = cudaMemcpyAsync(P->db, P->hb, P->lay.plan_end, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = enqueue_batch(P->L, b, P->db, P->lay, P->path, P->param, tau_dev, tmo, s);
  if (e == cudaSuccess && captured) e = plan_capture_fallback(P, tmo, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(P->hb + P->lay.out_begin, P->db + P->lay.out_begin, P->lay.out_end - P->lay.out_begin,
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(P->err_host, P->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && captured)
    e = cudaMemcpyAsync(P->fb_count_host, &P->fb_slot->nfallback, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  return e;
}

}  // namespace

// ===================================================================== C ABI
extern "C" {

const char* fps_status_string(fps_status st) {
  switch (st) {
    case FPS_OK: return "ok";
    case FPS_ERR_INVALID_ARG: return "invalid argument";
    case FPS_ERR_IO: return "cannot read library file";
    case FPS_ERR_PARSE: return "malformed library line";
    case FPS_ERR_BUDGET: return "library exceeds the device memory budget";
    case FPS_ERR_CUDA: return "CUDA runtime error";
    case FPS_ERR_TIMEOUT: return "device-side wait timed out";
    case FPS_ERR_OVERFLOW_INTERNAL: return "internal candidate buffer overflow";
    case FPS_ERR_UNSUPPORTED: return "unsupported request";
    case FPS_ERR_NOMEM: return "host out of memory";
  }
  return "unknown status";
}

fps_status fps_pack_query(const char* query166, uint64_t out[FPS_WORDS]) {
  if (!query166 || !out) return FPS_ERR_INVALID_ARG;
  uint64_t w[3] = {0, 0, 0};
  for (int j = 0; j < kBits; ++j) {
    char c = query166[j];
    if (c != '0' && c != '1') return FPS_ERR_INVALID_ARG;
    w[j >> 6] |= static_cast<uint64_t>(c - '0') << (j & 63);
  }
  out[0] = w[0];
  out[1] = w[1];
  out[2] = w[2];
  return FPS_OK;
}

fps_status fps_pack_text(const char* text, size_t text_len, uint32_t flags, uint64_t* out_packed, int64_t* out_cids,
                         size_t cap, size_t* out_n, size_t* err_line) {
  if ((!text && text_len) || !out_n) return FPS_ERR_INVALID_ARG;
  Parsed p;
  fps_status st = parse_text(text ? text : "", text_len, flags, &p, err_line);
  if (st != FPS_OK) return st;
  *out_n = static_cast<size_t>(p.n);
  if (!out_packed) return FPS_OK;
  if (static_cast<size_t>(p.n) > cap) return FPS_ERR_INVALID_ARG;
  std::memcpy(out_packed, p.packed.data(), p.packed.size() * sizeof(uint64_t));
  if (out_cids) std::memcpy(out_cids, p.cids.data(), p.cids.size() * sizeof(int64_t));
  return FPS_OK;
}

fps_status fps_library_load(const fps_load_desc* d, fps_library* out) {
  if (!d || !out) return FPS_ERR_INVALID_ARG;
  *out = nullptr;
  int sources = (d->path != nullptr) + (d->text != nullptr) + (d->packed != nullptr);
  if (sources != 1) return FPS_ERR_INVALID_ARG;
  Library* L = nullptr;
  fps_status st;
  if (d->packed) {
    if (d->n_packed >= (static_cast<size_t>(1) << 31) - 1) return FPS_ERR_UNSUPPORTED;
    st = build_library(d->packed, static_cast<int64_t>(d->n_packed), d->cids, d, &L);
  } else {
    std::vector<char> file;
    const char* text = d->text;
    size_t len = d->text_len;
    if (d->path) {
      FILE* f = std::fopen(d->path, "rb");
      if (!f) return FPS_ERR_IO;
      std::fseek(f, 0, SEEK_END);
      long sz = std::ftell(f);
      std::fseek(f, 0, SEEK_SET);
      if (sz < 0) {
        std::fclose(f);
        return FPS_ERR_IO;
      }
      try {
        file.resize(static_cast<size_t>(sz));
      } catch (const std::bad_alloc&) {
        std::fclose(f);
        return FPS_ERR_NOMEM;
      }
      size_t got = sz ? std::fread(file.data(), 1, file.size(), f) : 0;
      std::fclose(f);
      if (got != file.size()) return FPS_ERR_IO;
      text = file.data();
      len = file.size();
    }
    Parsed p;
    st = parse_text(text ? text : "", len, d->flags, &p, d->err_line);
    if (st != FPS_OK) return st;
    st = build_library(p.packed.data(), p.n, p.any_cid ? p.cids.data() : nullptr, d, &L);
  }
  if (st == FPS_OK) *out = reinterpret_cast<fps_library>(L);
  return st;
}

fps_status fps_release(fps_library lib) {
  if (!lib) return FPS_OK;
  Library* L = reinterpret_cast<Library*>(lib);
  free_library(L);
  return FPS_OK;
}

fps_status fps_library_info_get(fps_library lib, fps_library_info* info) {
  if (!lib || !info) return FPS_ERR_INVALID_ARG;
  Library* L = reinterpret_cast<Library*>(lib);
  std::memset(info, 0, sizeof *info);
  info->n_records = L->n;
  info->n_tiles = L->n_tiles;
  info->device_bytes = L->device_bytes;
  info->device = L->device;
  info->bucketed = L->bucketed;
  info->has_tc_operand = L->tc_fp8 ? 1 : 0;
  info->has_tc_fp4 = L->tc_fp4 ? 1 : 0;
  for (int b = 0; b < kNumBuckets; ++b) info->bucket_count[b] = L->bucket_count[b];
  return FPS_OK;
}

fps_status fps_library_cid(fps_library lib, int64_t index, int64_t* cid) {
  if (!lib || !cid) return FPS_ERR_INVALID_ARG;
  Library* L = reinterpret_cast<Library*>(lib);
  if (index < 0 || index >= L->n) return FPS_ERR_INVALID_ARG;
  *cid = L->cids.empty() ? index : L->cids[static_cast<size_t>(index)];
  return FPS_OK;
}

fps_status fps_search(fps_library lib, const char* query166, int k, int32_t* out_index, int32_t* out_dist,
                      int64_t* out_cid, int* out_count, void* cuda_stream) {
  if (!lib || !query166 || !out_count || (k > 0 && (!out_index || !out_dist))) return FPS_ERR_INVALID_ARG;
  fps_status st = check_k(k);
  if (st != FPS_OK) return st;
  uint64_t q[3];
  st = fps_pack_query(query166, q);
  if (st != FPS_OK) return st;
  Library* L = reinterpret_cast<Library*>(lib);
  DeviceGuard g(L->device);
  if (!g.ok) return FPS_ERR_CUDA;
  int32_t c = 0;
  st = search_one_host(L, q, k, out_index, out_dist, &c, nullptr, static_cast<cudaStream_t>(cuda_stream));
  if (st != FPS_OK) return st;
  if (out_cid)
    for (int i = 0; i < k; ++i) out_cid[i] = i >= c ? -1 : (L->cids.empty() ? out_index[i] : L->cids[out_index[i]]);
  *out_count = c;
  return FPS_OK;
}

fps_status fps_search_packed(fps_library lib, const uint64_t* query, int k, int32_t* out_index, int32_t* out_dist,
                             int32_t* out_count, const fps_search_opts* opts, void* cuda_stream) {
  if (!lib || !query || !out_count || (k > 0 && (!out_index || !out_dist))) return FPS_ERR_INVALID_ARG;
  fps_status st = check_k(k);
  if (st != FPS_OK) return st;
  Library* L = reinterpret_cast<Library*>(lib);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  DeviceGuard g(L->device);
  if (!g.ok) return FPS_ERR_CUDA;
  const bool dev_io = opts && (opts->flags & FPS_SEARCH_DEVICE_IO);
  if (!dev_io) {
    if (query[2] >> (kBits - 128)) return FPS_ERR_INVALID_ARG;
    return search_one_host(L, query, k, out_index, out_dist, out_count, opts, s);
  }
  if (L->n == 0 || k == 0) {   // no records: count 0, every slot -1 (all bytes 0xFF)
    if (cudaMemsetAsync(out_count, 0, sizeof(int32_t), s) != cudaSuccess ||
        (k > 0 && (cudaMemsetAsync(out_index, 0xFF, sizeof(int32_t) * k, s) != cudaSuccess ||
                   cudaMemsetAsync(out_dist, 0xFF, sizeof(int32_t) * k, s) != cudaSuccess))) {
      cudaGetLastError();
      return FPS_ERR_CUDA;
    }
    return FPS_OK;
  }
  Workspace* w = nullptr;
  st = get_workspace(L, s, &w);
  if (st != FPS_OK) return st;
  if (launch_scan_single(L->dev, query, k, w->st, w->cand, out_index, out_dist, out_count, &w->io->err, L->num_sms,
                         opt_timeout(opts), s) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  return FPS_OK;
}


fps_status fps_search_batch(fps_library lib, const uint64_t* queries, int Q, const int32_t* k,
                            const int64_t* out_offsets, int32_t* out_index, int32_t* out_dist, int32_t* out_count,
                            const fps_search_opts* opts, void* cuda_stream) {
  if (!lib || Q < 0 || (Q > 0 && (!queries || !k || !out_offsets || !out_index || !out_dist || !out_count)))
    return FPS_ERR_INVALID_ARG;
  int64_t total = 0;
  for (int q = 0; q < Q; ++q) {
    fps_status st = check_k(k[q]);
    if (st != FPS_OK) return st;
    if (out_offsets[q] < 0 || out_offsets[q + 1] - out_offsets[q] < k[q]) return FPS_ERR_INVALID_ARG;
    total = std::max<int64_t>(total, out_offsets[q + 1]);
  }
  Library* L = reinterpret_cast<Library*>(lib);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  DeviceGuard g(L->device);
  if (!g.ok) return FPS_ERR_CUDA;
  const bool dev_io = opts && (opts->flags & FPS_SEARCH_DEVICE_IO);
  return search_batch_impl(L, queries, Q, k, out_offsets, total, out_index, out_dist, out_count, opts, dev_io, s);
}

fps_status fps_search_shards(const fps_library* libs, int n_libs, const int64_t* index_base, const uint64_t* queries,
                             int Q, const int32_t* k, const int64_t* out_offsets, int32_t* out_index,
                             int32_t* out_dist, int32_t* out_count, const fps_search_opts* opts, int64_t* progress,
                             void* cuda_stream) {
  if (!libs || n_libs <= 0 || n_libs > kShardsMax || Q < 0 ||
      (Q > 0 && (!queries || !k || !out_offsets || !out_index || !out_dist || !out_count)))
    return FPS_ERR_INVALID_ARG;
  if (n_libs > FPS_SHARDS_MAX) return FPS_ERR_INVALID_ARG;
  std::vector<Library*> Ls(n_libs);
  std::vector<int64_t> base(n_libs);
  int64_t acc = 0;
  for (int i = 0; i < n_libs; ++i) {
    if (!libs[i]) return FPS_ERR_INVALID_ARG;
    Ls[i] = reinterpret_cast<Library*>(libs[i]);
    if (Ls[i]->device != Ls[0]->device) return FPS_ERR_INVALID_ARG;
    base[i] = index_base ? index_base[i] : acc;
    acc += Ls[i]->n;
    if (base[i] < 0 || base[i] + Ls[i]->n > static_cast<int64_t>(INT32_MAX)) return FPS_ERR_INVALID_ARG;
  }
  {  // the global index ranges must be disjoint
    std::vector<std::pair<int64_t, int64_t>> r;
    for (int i = 0; i < n_libs; ++i)
      if (Ls[i]->n > 0) r.emplace_back(base[i], base[i] + Ls[i]->n);
    std::sort(r.begin(), r.end());
    for (size_t i = 1; i < r.size(); ++i)
      if (r[i].first < r[i - 1].second) return FPS_ERR_INVALID_ARG;
  }
  int64_t total = 0;
  for (int q = 0; q < Q; ++q) {
    fps_status st = check_k(k[q]);
    if (st != FPS_OK) return st;
    if (out_offsets[q] < 0 || out_offsets[q + 1] - out_offsets[q] < k[q]) return FPS_ERR_INVALID_ARG;
    total = std::max<int64_t>(total, out_offsets[q + 1]);
  }
  if (Q == 0) return FPS_OK;
  Library* L0 = Ls[0];
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  DeviceGuard g(L0->device);
  if (!g.ok) return FPS_ERR_CUDA;
  const bool dev_io = opts && (opts->flags & FPS_SEARCH_DEVICE_IO);
  if (!dev_io)
    for (int q = 0; q < Q; ++q)
      if (queries[3 * q + 2] >> (kBits - 128)) return FPS_ERR_INVALID_ARG;
  int64_t* prog_dev = nullptr;
  if (progress && cudaHostGetDevicePointer(reinterpret_cast<void**>(&prog_dev), progress, 0) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_INVALID_ARG;   // not pinned, device-mapped host memory
  }
  Workspace* w = nullptr;
  fps_status st = get_workspace(L0, s, &w);
  if (st != FPS_OK) return st;
  // device staging: [offsets Q+1][k Q][queries Q*3 (host form)][per shard: index, dist (total each), count Q]
  //                 [merged index, dist, count (host form)]
  Carve cv;
  const size_t d_off = cv.take(sizeof(int64_t) * (Q + 1));
  const size_t d_k = cv.take(sizeof(int32_t) * Q);
  const size_t d_q = cv.take(dev_io ? 0 : sizeof(uint64_t) * 3 * Q);
  std::vector<size_t> d_si(n_libs), d_sd(n_libs), d_sc(n_libs);
  for (int i = 0; i < n_libs; ++i) {
    d_si[i] = cv.take(sizeof(int32_t) * std::max<int64_t>(total, 1));
    d_sd[i] = cv.take(sizeof(int32_t) * std::max<int64_t>(total, 1));
    d_sc[i] = cv.take(sizeof(int32_t) * Q);
  }
  const size_t d_mi = cv.take(dev_io ? 0 : sizeof(int32_t) * std::max<int64_t>(total, 1));
  const size_t d_md = cv.take(dev_io ? 0 : sizeof(int32_t) * std::max<int64_t>(total, 1));
  const size_t d_mc = cv.take(dev_io ? 0 : sizeof(int32_t) * Q);
  const size_t h_bytes = cv.at;   // pinned mirror of the same layout (offsets, queries, merged results)
  st = grow_block(&w->shard_block, &w->shard_bytes, cv.at, false);
  if (st == FPS_OK) st = grow_block(&w->shard_host, &w->shard_host_bytes, h_bytes, true);
  if (st != FPS_OK) return st;
  char* db = static_cast<char*>(w->shard_block);
  char* hb = static_cast<char*>(w->shard_host);
  std::memcpy(hb + d_off, out_offsets, sizeof(int64_t) * (Q + 1));
  std::memcpy(hb + d_k, k, sizeof(int32_t) * Q);
  if (!dev_io) std::memcpy(hb + d_q, queries, sizeof(uint64_t) * 3 * Q);
  if (cudaMemcpyAsync(db, hb, dev_io ? d_q : d_q + sizeof(uint64_t) * 3 * Q, cudaMemcpyHostToDevice, s) !=
      cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  const uint64_t* qdev = dev_io ? queries : reinterpret_cast<const uint64_t*>(db + d_q);
  fps_search_opts so{};
  if (opts) so = *opts;
  so.flags |= FPS_SEARCH_DEVICE_IO;
  fps_search_stats shard_stats{};
  so.stats = &shard_stats;
  int64_t fallbacks = 0, candidates = 0, path_used = 0;
  ShardLists sl{};
  sl.n = n_libs;
  for (int i = 0; i < n_libs; ++i) {
    int32_t* si = reinterpret_cast<int32_t*>(db + d_si[i]);
    int32_t* sd = reinterpret_cast<int32_t*>(db + d_sd[i]);
    int32_t* sc = reinterpret_cast<int32_t*>(db + d_sc[i]);
    shard_stats = fps_search_stats{};
    DeviceGuard gi(Ls[i]->device);
    st = search_batch_impl(Ls[i], qdev, Q, k, out_offsets, total, si, sd, sc, &so, true, s);
    if (st != FPS_OK) return st;
    fallbacks += shard_stats.fallbacks;
    candidates += shard_stats.candidates;
    path_used = shard_stats.path_used;
    if (prog_dev && launch_progress(prog_dev + i, Q, s) != cudaSuccess) {
      cudaGetLastError();
      return FPS_ERR_CUDA;
    }
    sl.idx[i] = si;
    sl.dist[i] = sd;
    sl.count[i] = sc;
    sl.base[i] = base[i];
  }
  int32_t* mi = dev_io ? out_index : reinterpret_cast<int32_t*>(db + d_mi);
  int32_t* md = dev_io ? out_dist : reinterpret_cast<int32_t*>(db + d_md);
  int32_t* mc = dev_io ? out_count : reinterpret_cast<int32_t*>(db + d_mc);
  if (launch_shard_merge(sl, Q, reinterpret_cast<const int64_t*>(db + d_off), reinterpret_cast<const int32_t*>(db + d_k),
                         mi, md, mc, s) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  if (!dev_io) {
    if (cudaMemcpyAsync(hb + d_mi, db + d_mi, d_mc + sizeof(int32_t) * Q - d_mi, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      return FPS_ERR_CUDA;
    }
    for (int i = 0; i < n_libs; ++i) {   // a device-side failure in any shard's searches
      Workspace* wi = nullptr;
      DeviceGuard gi(Ls[i]->device);
      st = get_workspace(Ls[i], s, &wi);
      if (st == FPS_OK) st = take_device_error(wi, s);
      if (st != FPS_OK) return st;
    }
    // k[q] slots per query (the merge wrote -1 past its count); slots past k stay the caller's
    const int32_t* hmi = reinterpret_cast<const int32_t*>(hb + d_mi);
    const int32_t* hmd = reinterpret_cast<const int32_t*>(hb + d_md);
    for (int q = 0; q < Q; ++q) {
      std::memcpy(out_index + out_offsets[q], hmi + out_offsets[q], sizeof(int32_t) * k[q]);
      std::memcpy(out_dist + out_offsets[q], hmd + out_offsets[q], sizeof(int32_t) * k[q]);
    }
    std::memcpy(out_count, hb + d_mc, sizeof(int32_t) * Q);
  }
  if (opts && opts->stats) {
    opts->stats->queries = Q;
    opts->stats->fallbacks = fallbacks;
    opts->stats->device_fallbacks = 0;
    opts->stats->candidates = candidates;
    opts->stats->path_used = path_used;
  }
  return FPS_OK;
}

fps_status fps_cluster_search(fps_library lib, const uint64_t* queries, int Q, int c_min, int c_max, int k,
                              int* out_c, int32_t* out_labels, int32_t* out_medoids, int64_t* out_scores,
                              int32_t* out_index, int32_t* out_dist, int32_t* out_count, void* cuda_stream) {
  if (!lib || !queries || Q < 1 || Q > FPS_CLUSTER_MAX_Q || c_min < 2 || c_max < c_min ||
      c_max > FPS_CLUSTER_MAX_C || !out_c || !out_labels || !out_medoids || !out_count ||
      (k > 0 && (!out_index || !out_dist)))
    return FPS_ERR_INVALID_ARG;
  fps_status st = check_k(k);
  if (st != FPS_OK) return st;
  for (int q = 0; q < Q; ++q)
    if (queries[3 * q + 2] >> (kBits - 128)) return FPS_ERR_INVALID_ARG;
  Library* L = reinterpret_cast<Library*>(lib);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  DeviceGuard g(L->device);
  if (!g.ok) return FPS_ERR_CUDA;
  const int c_hi = std::min(c_max, Q - 1);
  const int n_c = c_max - c_min + 1;
  // device scratch: queries, D, row sums, per count: labels, costs, medoids, round state;
  // seeds, round flags, sizes, scores
  Carve cv;
  const size_t d_q = cv.take(sizeof(uint64_t) * 3 * Q);
  const size_t d_D = cv.take(sizeof(int32_t) * static_cast<size_t>(Q) * Q);
  const size_t d_rs = cv.take(sizeof(int32_t) * Q);
  const size_t d_cost = cv.take(sizeof(int32_t) * static_cast<size_t>(Q) * n_c);
  const size_t d_lab = cv.take(sizeof(int32_t) * static_cast<size_t>(Q) * n_c);
  const size_t d_seed = cv.take(sizeof(int32_t) * kClusterMaxC);
  const size_t d_med = cv.take(sizeof(int32_t) * kClusterMaxC * n_c);
  const size_t d_state = cv.take(sizeof(int32_t) * 4 * n_c);
  const size_t d_any = cv.take(sizeof(int32_t) * kClusterIters);
  const size_t d_sizes = cv.take(sizeof(int32_t) * kClusterMaxC);
  const size_t d_score = cv.take(sizeof(unsigned long long) * n_c);
  // the scratch lives in the stream's workspace and only grows (no allocation per call)
  const size_t h_words = 4 * static_cast<size_t>(n_c);   // pinned: round state up, one round flag down
  Workspace* w = nullptr;
  st = get_workspace(L, s, &w);
  if (st == FPS_OK) st = grow_block(&w->cluster_block, &w->cluster_bytes, cv.at, false);
  if (st == FPS_OK) st = grow_block(&w->cluster_host, &w->cluster_host_bytes, sizeof(int32_t) * h_words, true);
  if (st != FPS_OK) return st;
  char* db = static_cast<char*>(w->cluster_block);
  int32_t* hflag = static_cast<int32_t*>(w->cluster_host);
  auto fail = [&](fps_status code) {
    cudaGetLastError();
    cudaStreamSynchronize(s);
    return code;
  };
  int32_t* D = reinterpret_cast<int32_t*>(db + d_D);
  int32_t* rs = reinterpret_cast<int32_t*>(db + d_rs);
  int32_t* seed = reinterpret_cast<int32_t*>(db + d_seed);
  int32_t* sizes = reinterpret_cast<int32_t*>(db + d_sizes);
  unsigned long long* score = reinterpret_cast<unsigned long long*>(db + d_score);
  if (cudaMemcpyAsync(db + d_q, queries, sizeof(uint64_t) * 3 * Q, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(score, 0, sizeof(unsigned long long) * n_c, s) != cudaSuccess ||
      cluster_qdist(reinterpret_cast<const uint64_t*>(db + d_q), Q, D, s) != cudaSuccess ||
      cluster_rowsum(D, Q, nullptr, rs, s) != cudaSuccess ||
      cluster_select(rs, Q, false, nullptr, 0, nullptr, 0, seed, s) != cudaSuccess)
    return fail(FPS_ERR_CUDA);
  // farthest-first seeds up to the largest count (the seeds of a count are a prefix of them);
  // rs serves as the distance to the nearest seed
  for (int t = 1; t < c_hi; ++t) {
    if (cluster_near(D, Q, seed + t - 1, t == 1, rs, s) != cudaSuccess ||
        cluster_select(rs, Q, true, seed, t, nullptr, 0, seed + t, s) != cudaSuccess)
      return fail(FPS_ERR_CUDA);
  }
  // k-medoids for every count at once: one host check per round (some count still moving)
  const int n_live = c_hi >= c_min ? c_hi - c_min + 1 : 0;
  ClusterRounds rr{D, Q, c_min, n_live, reinterpret_cast<int32_t*>(db + d_med), reinterpret_cast<int32_t*>(db + d_lab),
                   reinterpret_cast<int32_t*>(db + d_cost), reinterpret_cast<int32_t*>(db + d_state),
                   reinterpret_cast<int32_t*>(db + d_any)};
  for (size_t x = 0; x < h_words; ++x) hflag[x] = 0;
  for (int t = 0; t < n_live; ++t) hflag[4 * t] = 1;   // active, no rounds yet
  if (n_live > 0 &&
      (cudaMemcpyAsync(rr.state, hflag, sizeof(int32_t) * 4 * n_live, cudaMemcpyHostToDevice, s) != cudaSuccess ||
       cudaMemsetAsync(rr.any_active, 0, sizeof(int32_t) * kClusterIters, s) != cudaSuccess))
    return fail(FPS_ERR_CUDA);
  for (int t = 0; t < n_live; ++t)   // slot t starts from the first c_min + t seeds
    if (cudaMemcpyAsync(rr.med + kClusterMaxC * t, seed, sizeof(int32_t) * (c_min + t), cudaMemcpyDeviceToDevice,
                        s) != cudaSuccess)
      return fail(FPS_ERR_CUDA);
  for (int round = 0; round < kClusterIters && n_live > 0; ++round) {
    if (cluster_round(rr, round, s) != cudaSuccess ||
        cudaMemcpyAsync(hflag, rr.any_active + round, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail(FPS_ERR_CUDA);
    if (!hflag[0]) break;   // every count's medoids repeat, or its rounds are used up
  }
  if (cluster_final_assign(rr, s) != cudaSuccess) return fail(FPS_ERR_CUDA);
  for (int t = 0; t < n_live; ++t)
    if (cluster_silhouette(D, Q, rr.lab + static_cast<size_t>(Q) * t, c_min + t, sizes, score + t, s) != cudaSuccess)
      return fail(FPS_ERR_CUDA);
  std::vector<unsigned long long> sc(n_c, 0ull);
  if (cudaMemcpyAsync(sc.data(), score, sizeof(unsigned long long) * n_c, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(FPS_ERR_CUDA);
  int best = 1;
  long long best_score = 0;
  for (int c = c_min; c <= c_hi; ++c) {
    const long long v = static_cast<long long>(sc[c - c_min]);
    if (best == 1 || v > best_score) {
      best = c;
      best_score = v;
    }
  }
  if (out_scores)
    for (int c = c_min; c <= c_max; ++c)
      out_scores[c - c_min] = c <= c_hi ? static_cast<int64_t>(sc[c - c_min]) : INT64_MIN;
  std::vector<int32_t> med_h(kClusterMaxC, 0);
  if (best == 1) {   // fewer than c_min + 1 queries: one cluster around the most central query
    if (cudaMemcpyAsync(med_h.data(), seed, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail(FPS_ERR_CUDA);
    for (int q = 0; q < Q; ++q) out_labels[q] = 0;
  } else {
    const int slot = best - c_min;
    if (cudaMemcpyAsync(med_h.data(), reinterpret_cast<int32_t*>(db + d_med) + kClusterMaxC * slot,
                        sizeof(int32_t) * best, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(out_labels, reinterpret_cast<int32_t*>(db + d_lab) + static_cast<size_t>(Q) * slot,
                        sizeof(int32_t) * Q, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail(FPS_ERR_CUDA);
  }
  *out_c = best;
  for (int t = 0; t < best; ++t) out_medoids[t] = med_h[t];
  // every cluster searched with its medoid (one after another through the single-query scan)
  std::vector<uint64_t> mq(3 * static_cast<size_t>(best));
  std::vector<int32_t> kk(best, k);
  std::vector<int64_t> off(best + 1, 0);
  for (int t = 0; t < best; ++t) {
    std::memcpy(&mq[3 * t], queries + 3 * static_cast<size_t>(med_h[t]), 3 * sizeof(uint64_t));
    off[t + 1] = off[t] + k;
  }
  fps_search_opts o{};
  o.path = FPS_PATH_POPC;
  std::vector<int32_t> ti(std::max<int64_t>(off[best], 1)), td(std::max<int64_t>(off[best], 1));
  st = search_batch_impl(L, mq.data(), best, kk.data(), off.data(), off[best], ti.data(), td.data(), out_count, &o,
                         false, s);
  if (st != FPS_OK) return st;
  for (int t = 0; t < best && k > 0; ++t) {
    std::memcpy(out_index + static_cast<size_t>(t) * k, ti.data() + off[t], sizeof(int32_t) * k);   // -1 past the count
    std::memcpy(out_dist + static_cast<size_t>(t) * k, td.data() + off[t], sizeof(int32_t) * k);
  }
  return FPS_OK;
}

fps_status fps_merge_topk(const int32_t* idx, const int32_t* dist, const int64_t* part_off, int parts, int k,
                          int32_t* out_index, int32_t* out_dist, int* out_n) {
  if (parts < 0 || k < 0 || !part_off || !out_n || (k > 0 && (!out_index || !out_dist))) return FPS_ERR_INVALID_ARG;
  for (int p = 0; p < parts; ++p)
    if (part_off[p + 1] < part_off[p] || (part_off[p + 1] > part_off[p] && (!idx || !dist))) return FPS_ERR_INVALID_ARG;
  // a heap of the current head of every list, ordered by (distance, index)
  using Head = std::pair<uint64_t, int>;
  auto key = [&](int64_t e) {
    return (static_cast<uint64_t>(static_cast<uint32_t>(dist[e])) << 32) | static_cast<uint32_t>(idx[e]);
  };
  std::vector<Head> heap;
  std::vector<int64_t> pos(parts);
  for (int p = 0; p < parts; ++p) {
    pos[p] = part_off[p];
    if (pos[p] < part_off[p + 1]) heap.emplace_back(key(pos[p]), p);
  }
  auto cmp = [](const Head& a, const Head& b) { return a > b; };
  std::make_heap(heap.begin(), heap.end(), cmp);
  int n = 0;
  while (n < k && !heap.empty()) {
    std::pop_heap(heap.begin(), heap.end(), cmp);
    const int p = heap.back().second;
    heap.pop_back();
    out_index[n] = idx[pos[p]];
    out_dist[n] = dist[pos[p]];
    ++n;
    if (++pos[p] < part_off[p + 1]) {
      heap.emplace_back(key(pos[p]), p);
      std::push_heap(heap.begin(), heap.end(), cmp);
    }
  }
  fill_unused(out_index, out_dist, n, k);
  *out_n = n;
  return FPS_OK;
}

fps_status fps_batch_plan_create(fps_library lib, int Q, const int32_t* k, int path, int learned,
                                 fps_batch_plan* out) {
  if (!lib || !out || Q <= 0 || !k) return FPS_ERR_INVALID_ARG;
  *out = nullptr;
  Library* L = reinterpret_cast<Library*>(lib);
  int param = 0;
  if (path == FPS_PATH_AUTO) {
    // the batched kernel the autotuner chose for this size class, if it chose one already;
    // else the tensor cores when the library holds an operand for them
    int kmax = 0;
    for (int q = 0; q < Q; ++q) kmax = std::max(kmax, k[q]);
    {
      std::lock_guard<std::mutex> lock(L->mu);
      auto it = L->tuned.find(tune_class_name(Q, kmax, learned != 0));
      if (it != L->tuned.end() && it->second.path != FPS_PATH_POPC) {
        path = it->second.path;
        param = it->second.param;
      }
    }
    if (path == FPS_PATH_AUTO)
      path = L->tc_fp8 ? FPS_PATH_TC_FP8 : (L->tc_fp4 ? FPS_PATH_TC_FP4 : FPS_PATH_POPC_BATCH);
  }
  if (path != FPS_PATH_POPC_BATCH && !is_tc_path(path)) return FPS_ERR_UNSUPPORTED;
  if (!path_available(L, path)) return FPS_ERR_UNSUPPORTED;
  BatchPlan* P = new (std::nothrow) BatchPlan();
  if (!P) return FPS_ERR_NOMEM;
  P->L = L;
  P->Q = Q;
  P->path = path;
  P->param = tile_param_of(path, param);
  P->learned = learned != 0;
  P->k.assign(k, k + Q);
  P->off.assign(static_cast<size_t>(Q) + 1, 0);
  for (int q = 0; q < Q; ++q) {
    fps_status st = check_k(k[q]);
    if (st != FPS_OK) {
      free_plan(P);
      return st;
    }
    P->off[q + 1] = P->off[q] + k[q];
  }
  P->total = P->off[Q];
  if (L->n == 0) {
    P->empty = true;
    *out = reinterpret_cast<fps_batch_plan>(P);
    return FPS_OK;
  }
  P->coff = batch_cand_offsets(k, Q, L->n);
  P->lay = batch_layout(Q, P->total, P->coff[Q], false, P->learned, qop_bytes_of(P->path, Q));
  DeviceGuard g(L->device);
  const size_t hbytes = P->lay.plan_end > P->lay.out_end ? P->lay.plan_end : P->lay.out_end;
  if (!g.ok || cudaMalloc(&P->db, P->lay.bytes) != cudaSuccess || cudaMallocHost(&P->hb, hbytes) != cudaSuccess ||
      cudaMalloc(&P->err, 256) != cudaSuccess || cudaMallocHost(&P->err_host, sizeof(uint32_t)) != cudaSuccess ||
      cudaMemset(P->err, 0, 256) != cudaSuccess ||
      cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&P->cap_body, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    free_plan(P);
    return FPS_ERR_CUDA;
  }
  {
    // the fallback's scan state, slot and candidate keys
    const size_t st_bytes = (sizeof(ScanState) + 255) / 256 * 256;
    const size_t slot_bytes = (sizeof(ScanSlot) + 255) / 256 * 256;
    const size_t cand_bytes = scan_cand_capacity(L->num_sms) * sizeof(unsigned long long);
    if (cudaMalloc(&P->fb, st_bytes + slot_bytes + cand_bytes) != cudaSuccess ||
        cudaMallocHost(&P->fb_count_host, sizeof(uint32_t)) != cudaSuccess) {
      cudaGetLastError();
      free_plan(P);
      return FPS_ERR_CUDA;
    }
    P->fb_st = reinterpret_cast<ScanState*>(P->fb);
    P->fb_slot = reinterpret_cast<ScanSlot*>(P->fb + st_bytes);
    P->fb_cand = reinterpret_cast<unsigned long long*>(P->fb + st_bytes + slot_bytes);
    *P->fb_count_host = 0;
    if (scan_state_init(P->fb_st, P->cap) != cudaSuccess ||
        cudaMemsetAsync(P->fb_slot, 0, sizeof(ScanSlot), P->cap) != cudaSuccess ||
        scan_indirect_prepare() != cudaSuccess) {
      cudaGetLastError();
      free_plan(P);
      return FPS_ERR_CUDA;
    }
  }
  std::memset(P->hb, 0, hbytes);
  fill_plan(P->hb, P->lay, nullptr, Q, P->k.data(), P->coff, P->off.data(), nullptr, true);
  // one eager run (sets kernel attributes, checks the sequence), then capture the same sequence
  cudaError_t e = plan_enqueue(P, 2.0, P->cap, false);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->cap);
  if (e == cudaSuccess) e = cudaMemset(P->err, 0, 256);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e2 = plan_enqueue(P, 2.0, P->cap, true);
    e = cudaStreamEndCapture(P->cap, &P->graph);
    if (e2 != cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&P->exec, P->graph, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_plan(P);
    return FPS_ERR_CUDA;
  }
  *out = reinterpret_cast<fps_batch_plan>(P);
  return FPS_OK;
}

fps_status fps_batch_plan_run(fps_batch_plan plan, const uint64_t* queries, const float* tau, int32_t* out_index,
                              int32_t* out_dist, int32_t* out_count, fps_search_stats* stats, void* cuda_stream) {
  if (!plan || !queries || !out_index || !out_dist || !out_count) return FPS_ERR_INVALID_ARG;
  BatchPlan* P = reinterpret_cast<BatchPlan*>(plan);
  if (P->learned && !tau) return FPS_ERR_INVALID_ARG;
  for (int q = 0; q < P->Q; ++q)
    if (queries[3 * q + 2] >> (kBits - 128)) return FPS_ERR_INVALID_ARG;
  Library* L = P->L;
  if (P->empty) {
    for (int q = 0; q < P->Q; ++q) {
      out_count[q] = 0;
      fill_unused(out_index + P->off[q], out_dist + P->off[q], 0, P->k[q]);
    }
    if (stats) {
      *stats = fps_search_stats{};
      stats->queries = P->Q;
      stats->path_used = P->path;
      stats->tile_param = P->param;
    }
    return FPS_OK;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  DeviceGuard g(L->device);
  if (!g.ok) return FPS_ERR_CUDA;
  std::memcpy(P->hb + P->lay.d_q, queries, sizeof(uint64_t) * 3 * P->Q);
  if (P->learned) std::memcpy(P->hb + P->lay.d_tau, tau, sizeof(float) * P->Q);
  if (cudaGraphLaunch(P->exec, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  if (*P->err_host) {
    cudaMemset(P->err, 0, 256);
    return (*P->err_host & DEVERR_TIMEOUT) ? FPS_ERR_TIMEOUT : FPS_ERR_OVERFLOW_INTERNAL;
  }
  Workspace* w = nullptr;
  fps_status st = get_workspace(L, s, &w);
  if (st != FPS_OK) return st;
  fps_search_opts o{};
  o.stats = stats;
  int64_t nf = 0;
  st = finish_batch(L, w, P->hb, P->db, P->lay, queries, P->Q, P->k.data(), P->off.data(), out_index, out_dist,
                    out_count, &o, false, s, &nf);
  if (st == FPS_OK && stats) {
    stats->queries = P->Q;
    stats->fallbacks = nf + *P->fb_count_host;
    stats->device_fallbacks = *P->fb_count_host;
    stats->path_used = P->path;
    stats->tile_param = P->param;
  }
  return st;
}

fps_status fps_batch_plan_release(fps_batch_plan plan) {
  free_plan(reinterpret_cast<BatchPlan*>(plan));
  return FPS_OK;
}

fps_status fps_sync(fps_library lib, void* cuda_stream) {
  if (!lib) return FPS_ERR_INVALID_ARG;
  Library* L = reinterpret_cast<Library*>(lib);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  DeviceGuard g(L->device);
  if (!g.ok) return FPS_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  Workspace* w = nullptr;
  {
    std::lock_guard<std::mutex> lock(L->mu);
    auto it = L->ws.find(s);
    if (it == L->ws.end()) return FPS_OK;
    w = it->second;
  }
  return take_device_error(w, s);
}

}  // extern "C"
