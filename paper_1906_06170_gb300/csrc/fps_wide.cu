// Longer fingerprints (n bits, W = ceil(n / 64) words per record) and the
// Tanimoto measure: an exact top-k scan beside the 166-bit path.
//
// The paper searches 166 MACCS keys by Manhattan distance (Sec. 4.3) and names
// more features as future work (Sec. 5).  For n-bit records:
//   Manhattan: d(q, x) = popc(q XOR x), ranked ascending;
//   Tanimoto:  T(q, x) = c / u with c = popc(q AND x), u = popc(q OR x)
//              (1 when u = 0), ranked descending.
// Ties are ranked by ascending record index, so the answer is unique.
//
// Exact integer keys (smaller = better, unique per record):
//   Manhattan  key = d << 32 | index
//   Tanimoto   key = S << 32 | index,  S = 2^24 - floor(c 2^24 / u)  (S = 0 when u = 0)
// For n < 4096 two different fractions c/u differ by at least 1/n^2 > 2^-24,
// so floor(c 2^24 / u) orders them exactly and S is an exact rank of T.  The
// scan tests a record against the bound's S_b without dividing:
//   S <= S_b  <=>  c 2^24 >= (2^24 - S_b) u,
// and forms the key (one 64-bit division) only for records that pass.
//
// Layout in HBM: word-major tiles of 128 records, [tile][W][128] uint64, so a
// warp reads 256 contiguous bytes per (word, 32 records); each lane keeps 32
// loads (8 words of its 4 records) in flight.  One persistent block per SM
// (16 warps for k <= 128, 8 with the larger buffers above); warps claim
// 4-tile chunks from one counter (the next claim issued while the current
// chunk is scored), which lets faster SMs take more tiles.  Each warp keeps
// the keys under its bound in a shared buffer; when the buffer fills it sorts,
// keeps its best k and publishes the k-th key as a global bound (atomicMin: k
// records at or under it exist).  When its warps are done, every block sorts
// their survivors, keeps its k best and publishes its own k-th key.  The
// last block to finish gathers the survivors under the final bound, selects
// the k smallest keys (bitonic sort in shared memory, or bisection over the key
// when more survive than shared memory holds), recomputes c and u of the
// winners and writes them.
// No wait in this kernel depends on another block.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "fps_internal.h"

namespace fps {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kWTile = 128;               // records per tile
constexpr int kClaimTiles = 4;            // tiles per claim from the tile counter
constexpr int kMaxBlocks = 1024;          // grid size limit (one block per SM)
constexpr int kWarpsMax = 16;             // warps per block, at most (16 for k <= 128, 8 above)
constexpr int kMaxWords = FPS_WIDE_MAX_BITS / 64;

struct WideLib {
  const uint64_t* words;  // [n_tiles][W][128]
  const uint16_t* popc;   // [n_tiles * 128]: popc of each record (0 for padding)
  int64_t n;
  int64_t n_tiles;
  int W;
};

// The bound (read by every warp after every tile) and the tile counter (one
// atomic per claim) sit on separate 128-byte lines.
struct WideState {
  unsigned long long thr_key;   // global bound on the k-th key
  unsigned int ncand;           // unused (kept zero)
  unsigned int done;            // blocks finished
  unsigned int pad0[28];
  unsigned int next_tile;       // tile counter
  unsigned int pad1[31];
};
static_assert(sizeof(WideState) == 256, "scan state fills its 256-byte slot");

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// S = 2^24 - floor(c 2^24 / u), 0 for u = 0 (similarity 1)
__device__ __forceinline__ uint32_t tanimoto_rank(uint32_t c, uint32_t u) {
  if (u == 0u) return 0u;
  return (1u << 24) - static_cast<uint32_t>((static_cast<unsigned long long>(c) << 24) / u);
}

__device__ void warp_sort(unsigned long long* s, int n, int lane) {   // ascending, n a power of two
  for (int kk = 2; kk <= n; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < (n >> 1); i += 32) {
        const int pos = 2 * i - (i & (j - 1)), par = pos + j;
        const bool asc = (pos & kk) == 0;
        const unsigned long long a = s[pos], b = s[par];
        if ((a > b) == asc) {
          s[pos] = b;
          s[par] = a;
        }
      }
      __syncwarp();
    }
  }
}

__device__ void block_sort(unsigned long long* s, int n) {
  for (int kk = 2; kk <= n; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < (n >> 1); i += blockDim.x) {
        const int pos = 2 * i - (i & (j - 1)), par = pos + j;
        const bool asc = (pos & kk) == 0;
        const unsigned long long a = s[pos], b = s[par];
        if ((a > b) == asc) {
          s[pos] = b;
          s[par] = a;
        }
      }
      __syncthreads();
    }
  }
}

// Keys a block can sort in shared memory (the warp buffers' space, at least 8192 keys).
__host__ __device__ constexpr int merge_cap(int warps, int cap_per_warp) {
  return warps * cap_per_warp > 8192 ? warps * cap_per_warp : 8192;
}

__device__ __forceinline__ int pow2_at_least(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Keep the keys <= thr, sorted, at most k of them; returns the new count and
// tightens thr to the k-th key when k remain.
template <int CAP>
__device__ int compact_keys(unsigned long long* buf, int cnt, int k, unsigned long long& thr, int lane) {
  for (int i = cnt + lane; i < CAP; i += 32) buf[i] = ~0ull;
  __syncwarp();
  warp_sort(buf, CAP, lane);
  int keep = cnt < k ? cnt : k;
  if (keep == k && k > 0 && buf[k - 1] < thr) thr = buf[k - 1];
  int c = 0;   // keys above the (possibly tighter) bound drop out
  for (int base = 0; base < keep; base += 32) {
    const int i = base + lane;
    const bool in = i < keep && buf[i] <= thr;
    c += __popc(__ballot_sync(kFull, in));
  }
  __syncwarp();
  return c;
}

template <int METRIC, int WARPS, int CAP>
__global__ void __launch_bounds__(WARPS * 32, 1)
    wide_scan_kernel(WideLib L, const uint64_t* __restrict__ query, int k, WideState* st,
                     unsigned long long* __restrict__ cand, unsigned int* __restrict__ bcnt,
                     int32_t* __restrict__ out_idx, int32_t* __restrict__ out_num, int32_t* __restrict__ out_den,
                     int32_t* __restrict__ out_count) {
  extern __shared__ __align__(16) unsigned long long wsm[];    // WARPS * CAP keys (reused by the merges)
  __shared__ uint64_t sq[kMaxWords];
  __shared__ int s_last, s_cnt, s_wcnt[WARPS];
  __shared__ int s_bcnt[kMaxBlocks];
  __shared__ unsigned long long s_lo, s_hi;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int W = L.W;
  for (int w = tid; w < W; w += blockDim.x) sq[w] = query[w];
  __syncthreads();
  uint32_t pq = 0;   // popc of the query (Tanimoto: u = popc q + popc x - c)
  for (int w = 0; w < W; ++w) pq += __popcll(sq[w]);

  unsigned long long* buf = wsm + static_cast<size_t>(warp) * CAP;
  int cnt = 0;
  unsigned long long thr = ld_relaxed_u64(&st->thr_key);
  // tiles are claimed kClaimTiles at a time (one atomic per chunk on a single counter)
  const int64_t n_chunks = (L.n_tiles + kClaimTiles - 1) / kClaimTiles;
  unsigned int next = 0;
  if (lane == 0) next = atomicAdd(&st->next_tile, 1u);
  next = __shfl_sync(kFull, next, 0);
  int sub = 0;
  unsigned int chunk = next;
  if (lane == 0 && chunk < n_chunks) next = atomicAdd(&st->next_tile, 1u);   // the following chunk
  while (chunk < static_cast<unsigned int>(n_chunks)) {
    const int64_t t = static_cast<int64_t>(chunk) * kClaimTiles + sub;
    if (t >= L.n_tiles) break;
    const uint64_t* base = L.words + static_cast<size_t>(t) * W * kWTile;
    uint32_t a[4] = {0u, 0u, 0u, 0u}, b[4] = {0u, 0u, 0u, 0u};
    if (METRIC == FPS_METRIC_TANIMOTO) {
#pragma unroll
      for (int m = 0; m < 4; ++m) b[m] = pq + __ldcs(L.popc + t * kWTile + lane + 32 * m);
    }
    // 8 words x 4 records = 32 streaming loads issued before any of them is used
    for (int w0 = 0; w0 < W; w0 += 8) {
      uint64_t x[8][4];
#pragma unroll
      for (int ww = 0; ww < 8; ++ww) {
        const uint64_t* row = base + static_cast<size_t>(w0 + ww) * kWTile + lane;
#pragma unroll
        for (int m = 0; m < 4; ++m) x[ww][m] = (w0 + ww < W) ? __ldcs(row + 32 * m) : 0ull;
      }
#pragma unroll
      for (int ww = 0; ww < 8; ++ww) {
        const uint64_t qw = (w0 + ww < W) ? sq[w0 + ww] : 0ull;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          if (METRIC == FPS_METRIC_MANHATTAN)
            a[m] += __popcll(x[ww][m] ^ qw);
          else
            a[m] += __popcll(x[ww][m] & qw);
        }
      }
    }
    if (METRIC == FPS_METRIC_TANIMOTO) {
#pragma unroll
      for (int m = 0; m < 4; ++m) b[m] -= a[m];   // u = popc q + popc x - c
    }
    // the bound as a test without division: S <= S_b <=> c 2^24 >= (2^24 - S_b) u
    const uint32_t sb = static_cast<uint32_t>(thr >> 32);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int64_t r = t * kWTile + lane + 32 * m;
      bool pass = r < L.n;
      unsigned long long key = ~0ull;
      if (pass) {
        if (METRIC == FPS_METRIC_MANHATTAN) {
          pass = a[m] <= sb;
          key = (static_cast<unsigned long long>(a[m]) << 32) | static_cast<uint32_t>(r);
        } else {
          const unsigned long long fb = sb >= (1u << 24) ? 0ull : static_cast<unsigned long long>((1u << 24) - sb);
          pass = (static_cast<unsigned long long>(a[m]) << 24) >= fb * b[m];
          if (pass) key = (static_cast<unsigned long long>(tanimoto_rank(a[m], b[m])) << 32) | static_cast<uint32_t>(r);
        }
        pass = pass && key <= thr;
      }
      const uint32_t bal = __ballot_sync(kFull, pass);
      if (pass) buf[cnt + __popc(bal & ((1u << lane) - 1u))] = key;
      cnt += __popc(bal);
    }
    __syncwarp();
    if (cnt > CAP - kWTile) {
      cnt = compact_keys<CAP>(buf, cnt, k, thr, lane);
      if (lane == 0 && cnt == k) atomicMin(&st->thr_key, thr);
    }
    const unsigned long long g = ld_relaxed_u64(&st->thr_key);
    thr = g < thr ? g : thr;
    if (++sub == kClaimTiles) {
      sub = 0;
      chunk = __shfl_sync(kFull, next, 0);
      if (lane == 0 && chunk < n_chunks) next = atomicAdd(&st->next_tile, 1u);
    }
  }
  cnt = compact_keys<CAP>(buf, cnt, k, thr, lane);
  if (lane == 0 && cnt == k) atomicMin(&st->thr_key, thr);

  // ---- block merge: the 8 warps' survivors -> the block's k best, its k-th key published as a
  // bound; the block's slice of `cand` (8 FPS_K_MAX keys) is the staging area
  unsigned long long* slice = cand + static_cast<size_t>(blockIdx.x) * kWarpsMax * FPS_K_MAX;
  if (lane == 0) s_wcnt[warp] = cnt;
  __syncthreads();
  int off = 0, nb = 0;
  for (int w2 = 0; w2 < WARPS; ++w2) {
    off += w2 < warp ? s_wcnt[w2] : 0;
    nb += s_wcnt[w2];
  }
  for (int i = lane; i < cnt; i += 32) slice[off + i] = buf[i];
  __syncthreads();
  {
    const int p2 = pow2_at_least(nb > 1 ? nb : 1);
    for (int i = tid; i < p2; i += blockDim.x) wsm[i] = i < nb ? slice[i] : ~0ull;
    __syncthreads();
    block_sort(wsm, p2);
    const int kept = nb < k ? nb : k;
    if (tid == 0 && kept == k) atomicMin(&st->thr_key, wsm[k - 1]);
    for (int i = tid; i < kept; i += blockDim.x) slice[i] = wsm[i];
    if (tid == 0) bcnt[blockIdx.x] = static_cast<unsigned int>(kept);
  }

  // ---- the last block selects the k smallest survivors
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(&st->done, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int k_eff = static_cast<int>(k < L.n ? k : L.n);
  const int cap = merge_cap(WARPS, CAP);
  unsigned long long* s = wsm;
  // only keys under the final bound can be among the k smallest (k keys at or under it exist)
  const unsigned long long fthr = ld_relaxed_u64(&st->thr_key);
  auto survivor = [&](int b, int i) { return __ldcg(cand + static_cast<size_t>(b) * kWarpsMax * FPS_K_MAX + i); };
  // every block's count at once (a loop over blocks with a dependent load each would serialise
  // gridDim.x memory round trips), then one flattened pass over (block, slot)
  for (int b = tid; b < static_cast<int>(gridDim.x); b += blockDim.x)
    s_bcnt[b] = static_cast<int>(*reinterpret_cast<volatile unsigned int*>(bcnt + b));
  if (tid == 0) s_cnt = 0;
  __syncthreads();
  const int slots = static_cast<int>(gridDim.x) * k;   // a block keeps at most k keys
  for (int x = tid; x < slots; x += blockDim.x) {
    const int b = x / k, i = x - b * k;
    if (i >= s_bcnt[b]) continue;
    const unsigned long long key = survivor(b, i);
    if (key <= fthr) {
      const int p = atomicAdd(&s_cnt, 1);
      if (p < cap) s[p] = key;
    }
  }
  __syncthreads();
  int nsel = s_cnt;
  __syncthreads();
  if (nsel > cap) {
    // bisection on the key: the k_eff-th smallest key K, then the keys <= K (exactly k_eff: keys are unique)
    if (tid == 0) {
      s_lo = 0ull;
      s_hi = fthr;
    }
    __syncthreads();
    for (int it = 0; it < 64 && s_lo < s_hi; ++it) {
      const unsigned long long lo = s_lo, hi = s_hi, mid = lo + (hi - lo) / 2;
      if (tid == 0) s_cnt = 0;
      __syncthreads();
      int local = 0;
      for (int x = tid; x < slots; x += blockDim.x) {
        const int b = x / k, i = x - b * k;
        if (i < s_bcnt[b]) local += survivor(b, i) <= mid;
      }
      atomicAdd(&s_cnt, local);
      __syncthreads();
      if (tid == 0) {
        if (s_cnt >= k_eff)
          s_hi = mid;
        else
          s_lo = mid + 1;
      }
      __syncthreads();
    }
    const unsigned long long K = s_lo;
    if (tid == 0) s_cnt = 0;
    __syncthreads();
    for (int x = tid; x < slots; x += blockDim.x) {
      const int b = x / k, i = x - b * k;
      if (i >= s_bcnt[b]) continue;
      const unsigned long long key = survivor(b, i);
      if (key <= K) {
        const int p = atomicAdd(&s_cnt, 1);
        if (p < cap) s[p] = key;
      }
    }
    __syncthreads();
    nsel = s_cnt < cap ? s_cnt : cap;
  }
  __syncthreads();
  const int p2 = pow2_at_least(nsel > 1 ? nsel : 1);
  for (int i = nsel + tid; i < p2; i += blockDim.x) s[i] = ~0ull;
  __syncthreads();
  block_sort(s, p2);
  const int nout = k_eff < nsel ? k_eff : nsel;
  for (int i = tid; i < nout; i += blockDim.x) {
    const unsigned long long key = s[i];
    const int64_t r = static_cast<int64_t>(key & 0xFFFFFFFFull);
    out_idx[i] = static_cast<int32_t>(r);
    if (METRIC == FPS_METRIC_MANHATTAN) {
      out_num[i] = static_cast<int32_t>(key >> 32);
      out_den[i] = 1;
    } else {
      const uint64_t* rec = L.words + static_cast<size_t>(r / kWTile) * W * kWTile + (r % kWTile);
      uint32_t c = 0, u = 0;
      for (int w = 0; w < W; ++w) {
        const uint64_t x = rec[static_cast<size_t>(w) * kWTile];
        c += __popcll(x & sq[w]);
        u += __popcll(x | sq[w]);
      }
      out_num[i] = static_cast<int32_t>(c);
      out_den[i] = static_cast<int32_t>(u);
    }
  }
  for (int i = nout + tid; i < k; i += blockDim.x) {   // slots past min(k, N), up to k, hold -1
    out_idx[i] = -1;
    out_num[i] = -1;
    out_den[i] = -1;
  }
  if (tid == 0) {
    *out_count = nout;
    st->thr_key = ~0ull;   // ready for the next search on this state
    st->ncand = 0u;
    st->done = 0u;
    st->next_tile = 0u;
  }
}

__global__ void wide_state_init_kernel(WideState* st) {
  if (threadIdx.x == 0) {
    st->thr_key = ~0ull;
    st->ncand = 0u;
    st->done = 0u;
    st->next_tile = 0u;
  }
}

template <int METRIC, int WARPS, int CAP>
cudaError_t launch_wide(const WideLib& L, const uint64_t* q, int k, WideState* st, unsigned long long* cand,
                        unsigned int* bcnt, int32_t* oi, int32_t* on, int32_t* od, int32_t* oc, int num_sms,
                        cudaStream_t s) {
  auto kern = wide_scan_kernel<METRIC, WARPS, CAP>;
  const size_t smem = sizeof(unsigned long long) * merge_cap(WARPS, CAP);
  static std::atomic<uint64_t> configured{0};   // one per instantiation
  cudaError_t e = smem_attr_once(kern, smem, &configured);
  if (e != cudaSuccess) return e;
  if (num_sms > kMaxBlocks) return cudaErrorInvalidConfiguration;
  kern<<<num_sms, WARPS * 32, smem, s>>>(L, q, k, st, cand, bcnt, oi, on, od, oc);
  return cudaGetLastError();
}

constexpr int kSmallCapW = 256, kLargeCapW = 2048;

// ------------------------------------------------------------------- host
struct WideWs {
  WideState* st = nullptr;
  unsigned long long* cand = nullptr;   // per block: 8 FPS_K_MAX keys
  unsigned int* bcnt = nullptr;         // per block: survivors after the block merge
  uint64_t* q = nullptr;         // query (device)
  int32_t* out = nullptr;        // index, num, den (FPS_K_MAX each) + count (device)
  void* block = nullptr;
  int32_t* host = nullptr;       // pinned mirror of out
};

struct WideLibrary {
  int device = 0;
  int n_bits = 0;
  WideLib dev{};
  uint64_t* words = nullptr;
  uint16_t* popc = nullptr;
  size_t device_bytes = 0;
  int num_sms = 0;
  std::mutex mu;
  std::map<cudaStream_t, WideWs*> ws;
};

struct WideGuard {
  int prev = 0;
  bool ok = false;
  explicit WideGuard(int dev) {
    ok = cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess;
  }
  ~WideGuard() {
    if (ok) cudaSetDevice(prev);
  }
};

void free_wide(WideLibrary* L) {
  if (!L) return;
  WideGuard g(L->device);
  for (auto& kv : L->ws) {
    if (kv.second->block) cudaFree(kv.second->block);
    if (kv.second->host) cudaFreeHost(kv.second->host);
    delete kv.second;
  }
  if (L->words) cudaFree(L->words);
  if (L->popc) cudaFree(L->popc);
  delete L;
}

fps_status wide_workspace(WideLibrary* L, cudaStream_t s, WideWs** out) {
  std::lock_guard<std::mutex> lock(L->mu);
  auto it = L->ws.find(s);
  if (it != L->ws.end()) {
    *out = it->second;
    return FPS_OK;
  }
  WideWs* w = new (std::nothrow) WideWs();
  if (!w) return FPS_ERR_NOMEM;
  const size_t cand_keys = static_cast<size_t>(L->num_sms) * kWarpsMax * FPS_K_MAX;
  const size_t st_b = 256, q_b = sizeof(uint64_t) * kMaxWords, out_b = sizeof(int32_t) * (3 * FPS_K_MAX + 1);
  const size_t bytes = st_b + q_b + (out_b + 255) / 256 * 256 + cand_keys * sizeof(unsigned long long) +
                       sizeof(unsigned int) * static_cast<size_t>(L->num_sms);
  if (cudaMalloc(&w->block, bytes) != cudaSuccess || cudaMallocHost(&w->host, out_b) != cudaSuccess) {
    cudaGetLastError();
    if (w->block) cudaFree(w->block);
    delete w;
    return FPS_ERR_CUDA;
  }
  char* b = static_cast<char*>(w->block);
  w->st = reinterpret_cast<WideState*>(b);
  w->q = reinterpret_cast<uint64_t*>(b + st_b);
  w->out = reinterpret_cast<int32_t*>(b + st_b + q_b);
  w->cand = reinterpret_cast<unsigned long long*>(b + st_b + q_b + (out_b + 255) / 256 * 256);
  w->bcnt = reinterpret_cast<unsigned int*>(w->cand + cand_keys);
  wide_state_init_kernel<<<1, 32, 0, s>>>(w->st);
  if (cudaGetLastError() != cudaSuccess) {
    cudaFree(w->block);
    cudaFreeHost(w->host);
    delete w;
    return FPS_ERR_CUDA;
  }
  L->ws[s] = w;
  *out = w;
  return FPS_OK;
}

// Text of lines of n_bits '0'/'1' characters (a trailing '\r' dropped) -> W words per record.
fps_status wide_parse(const char* text, size_t len, int n_bits, std::vector<uint64_t>* out, int64_t* n_out,
                      size_t* err_line) {
  const int W = (n_bits + 63) / 64;
  int64_t n = 0;
  size_t p = 0;
  out->clear();
  while (p < len) {
    size_t e = p;
    while (e < len && text[e] != '\n') ++e;
    size_t l = e - p;
    if (l > 0 && text[p + l - 1] == '\r') --l;
    if (static_cast<int>(l) != n_bits) {
      if (err_line) *err_line = static_cast<size_t>(n + 1);
      return FPS_ERR_PARSE;
    }
    out->resize(out->size() + W, 0ull);
    uint64_t* w = out->data() + static_cast<size_t>(n) * W;
    for (int j = 0; j < n_bits; ++j) {
      const char c = text[p + j];
      if (c != '0' && c != '1') {
        if (err_line) *err_line = static_cast<size_t>(n + 1);
        return FPS_ERR_PARSE;
      }
      if (c == '1') w[j >> 6] |= 1ull << (j & 63);
    }
    ++n;
    p = e + 1;
  }
  *n_out = n;
  return FPS_OK;
}

}  // namespace
}  // namespace fps

using namespace fps;

extern "C" {

fps_status fps_wide_load(const char* text, size_t text_len, const uint64_t* packed, size_t n_packed, int n_bits,
                         int device, size_t hbm_budget_bytes, fps_wide_library* out, size_t* err_line) {
  if (!out || n_bits < 1 || n_bits > FPS_WIDE_MAX_BITS || (!text && !packed) || (text && packed))
    return FPS_ERR_INVALID_ARG;
  *out = nullptr;
  const int W = (n_bits + 63) / 64;
  std::vector<uint64_t> parsed;
  int64_t n = 0;
  const uint64_t* src = packed;
  if (text) {
    fps_status st = wide_parse(text, text_len, n_bits, &parsed, &n, err_line);
    if (st != FPS_OK) return st;
    src = parsed.data();
  } else {
    n = static_cast<int64_t>(n_packed);
    const int tail = n_bits & 63;
    if (tail)   // bits past n_bits must be zero
      for (int64_t r = 0; r < n; ++r)
        if (packed[r * W + W - 1] >> tail) return FPS_ERR_INVALID_ARG;
  }
  if (n >= static_cast<int64_t>(INT32_MAX)) return FPS_ERR_UNSUPPORTED;
  const int64_t n_tiles = (n + kWTile - 1) / kWTile;
  const size_t bytes = static_cast<size_t>(n_tiles > 0 ? n_tiles : 1) * W * kWTile * sizeof(uint64_t);
  const size_t pbytes = static_cast<size_t>(n_tiles > 0 ? n_tiles : 1) * kWTile * sizeof(uint16_t);
  if (hbm_budget_bytes && bytes + pbytes > hbm_budget_bytes) return FPS_ERR_BUDGET;
  WideLibrary* L = new (std::nothrow) WideLibrary();
  if (!L) return FPS_ERR_NOMEM;
  L->device = device;
  L->n_bits = n_bits;
  WideGuard g(device);
  if (!g.ok || cudaDeviceGetAttribute(&L->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    delete L;
    return FPS_ERR_CUDA;
  }
  // word-major tiles: [tile][word][128 records], padding records zero
  std::vector<uint64_t> tiled(bytes / sizeof(uint64_t), 0ull);
  std::vector<uint16_t> pc(pbytes / sizeof(uint16_t), 0);
  for (int64_t r = 0; r < n; ++r) {
    int p = 0;
    for (int w = 0; w < W; ++w) {
      const uint64_t x = src[static_cast<size_t>(r) * W + w];
      tiled[(static_cast<size_t>(r / kWTile) * W + w) * kWTile + (r % kWTile)] = x;
      p += __builtin_popcountll(x);
    }
    pc[static_cast<size_t>(r)] = static_cast<uint16_t>(p);
  }
  if (cudaMalloc(&L->words, bytes) != cudaSuccess || cudaMalloc(&L->popc, pbytes) != cudaSuccess ||
      cudaMemcpy(L->words, tiled.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(L->popc, pc.data(), pbytes, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    free_wide(L);
    return FPS_ERR_CUDA;
  }
  L->device_bytes = bytes + pbytes;
  L->dev = WideLib{L->words, L->popc, n, n_tiles, W};
  *out = reinterpret_cast<fps_wide_library>(L);
  return FPS_OK;
}

fps_status fps_wide_release(fps_wide_library lib) {
  free_wide(reinterpret_cast<WideLibrary*>(lib));
  return FPS_OK;
}

fps_status fps_wide_info(fps_wide_library lib, int64_t* n_records, int* n_bits, size_t* device_bytes) {
  if (!lib) return FPS_ERR_INVALID_ARG;
  WideLibrary* L = reinterpret_cast<WideLibrary*>(lib);
  if (n_records) *n_records = L->dev.n;
  if (n_bits) *n_bits = L->n_bits;
  if (device_bytes) *device_bytes = L->device_bytes;
  return FPS_OK;
}

fps_status fps_wide_search(fps_wide_library lib, const uint64_t* query, int k, int metric, int32_t* out_index,
                           int32_t* out_num, int32_t* out_den, int32_t* out_count, uint32_t flags,
                           void* cuda_stream) {
  if (!lib || !query || !out_count || k < 0 || (k > 0 && (!out_index || !out_num || !out_den)) ||
      (metric != FPS_METRIC_MANHATTAN && metric != FPS_METRIC_TANIMOTO))
    return FPS_ERR_INVALID_ARG;
  if (k > FPS_K_MAX) return FPS_ERR_UNSUPPORTED;
  WideLibrary* L = reinterpret_cast<WideLibrary*>(lib);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const bool dev_io = (flags & FPS_SEARCH_DEVICE_IO) != 0;
  const int W = L->dev.W;
  if (!dev_io && (L->n_bits & 63) && (query[W - 1] >> (L->n_bits & 63))) return FPS_ERR_INVALID_ARG;
  WideGuard g(L->device);
  if (!g.ok) return FPS_ERR_CUDA;
  if (L->dev.n == 0 || k == 0) {   // no records: count 0, every slot -1
    if (dev_io) {
      const size_t b = sizeof(int32_t) * k;
      if (cudaMemsetAsync(out_count, 0, sizeof(int32_t), s) != cudaSuccess ||
          (k > 0 && (cudaMemsetAsync(out_index, 0xFF, b, s) != cudaSuccess ||
                     cudaMemsetAsync(out_num, 0xFF, b, s) != cudaSuccess ||
                     cudaMemsetAsync(out_den, 0xFF, b, s) != cudaSuccess))) {
        cudaGetLastError();
        return FPS_ERR_CUDA;
      }
    } else {
      for (int i = 0; i < k; ++i) out_index[i] = out_num[i] = out_den[i] = -1;
      *out_count = 0;
    }
    return FPS_OK;
  }
  WideWs* w = nullptr;
  fps_status st = wide_workspace(L, s, &w);
  if (st != FPS_OK) return st;
  const uint64_t* dq = query;
  int32_t *oi = out_index, *on = out_num, *od = out_den, *oc = out_count;
  if (!dev_io) {
    if (cudaMemcpyAsync(w->q, query, sizeof(uint64_t) * W, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      cudaGetLastError();
      return FPS_ERR_CUDA;
    }
    dq = w->q;
    oi = w->out;
    on = w->out + FPS_K_MAX;
    od = w->out + 2 * FPS_K_MAX;
    oc = w->out + 3 * FPS_K_MAX;
  }
  cudaError_t e;
  const bool small = k <= kSmallCapW - kWTile;
  if (metric == FPS_METRIC_MANHATTAN)
    e = small ? launch_wide<FPS_METRIC_MANHATTAN, 16, kSmallCapW>(L->dev, dq, k, w->st, w->cand, w->bcnt, oi, on, od, oc, L->num_sms, s)
              : launch_wide<FPS_METRIC_MANHATTAN, 8, kLargeCapW>(L->dev, dq, k, w->st, w->cand, w->bcnt, oi, on, od, oc, L->num_sms, s);
  else
    e = small ? launch_wide<FPS_METRIC_TANIMOTO, 16, kSmallCapW>(L->dev, dq, k, w->st, w->cand, w->bcnt, oi, on, od, oc, L->num_sms, s)
              : launch_wide<FPS_METRIC_TANIMOTO, 8, kLargeCapW>(L->dev, dq, k, w->st, w->cand, w->bcnt, oi, on, od, oc, L->num_sms, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  if (dev_io) return FPS_OK;
  if (cudaMemcpyAsync(w->host, w->out, sizeof(int32_t) * (3 * FPS_K_MAX + 1), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  const int c = w->host[3 * FPS_K_MAX];
  std::memcpy(out_index, w->host, sizeof(int32_t) * k);   // the kernel wrote -1 past c
  std::memcpy(out_num, w->host + FPS_K_MAX, sizeof(int32_t) * k);
  std::memcpy(out_den, w->host + 2 * FPS_K_MAX, sizeof(int32_t) * k);
  *out_count = c;
  return FPS_OK;
}

}  // extern "C"
