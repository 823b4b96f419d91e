// Batched exact top-k: many queries per launch, each with its own k.
//
// Paper: Sec. 4.3 / Fig. 3 steps 3-6 for every query of a batch (the "batch"
// search of Sec. 4.4 without its unspecified clustering step).  Distances are
// the same integers as the single-query scan: d = sum_w popc(q_w ^ x_w).
//
// Three kernels share a per-query state (BatchDev):
//   batch_prepare_kernel  clears the state and, optionally, sets each query's
//                         starting bound to its exact k-th distance over a
//                         32 K-record sample of the library -- a valid upper
//                         bound of the true k-th distance (a subset's k-th
//                         smallest is never below the whole set's);
//   batch_popc_kernel     (CUDA-core popcount scan) accepts record x for query q
//                         iff d(q, x) <= thr[q]; accepted records are counted
//                         in hist[q] and appended (as distance and layout
//                         position) to q's candidate region;
//                         after accepting, the warp re-derives the bound (the
//                         smallest D with >= k accepted at distance <= D) and
//                         tightens thr[q].  Popcount buckets whose lower bound
//                         |popc q - b| exceeds thr[q] are skipped per query;
//   (with predicted starting bounds instead of the pilot, a query whose bound was
//   too low ends with fewer than k accepted records; the select kernel reports
//   it as -2 and the host re-runs it exactly)
//   batch_select_kernel   per query: hist is exact up to the final bound
//                         (every record at distance <= the true k-th distance
//                         was accepted and counted once), which gives the k-th
//                         distance T and the count below it; candidates below
//                         T plus the smallest indices at T, sorted, are the
//                         answer.  A query whose candidates overflowed its
//                         region is reported as -2 and re-run by the host with
//                         the single-query scan.
#include <cuda_runtime.h>

#include <cstdint>

#include "fps_internal.h"

namespace fps {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kPilotTiles = 256;         // 256 x 128 = 32 K sample records
constexpr int kSelThreads = 256;
constexpr int kSelFin = 2048;            // >= FPS_K_MAX, power of two
constexpr int kSelTies = 8192;           // tie keys sorted in shared memory

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_add_u32(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

__device__ void block_bitonic_sort(unsigned long long* s, int n) {
  for (int kk = 2; kk <= n; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < (n >> 1); i += blockDim.x) {
        int pos = 2 * i - (i & (j - 1));
        int par = pos + j;
        bool asc = (pos & kk) == 0;
        unsigned long long a = s[pos], b = s[par];
        if ((a > b) == asc) {
          s[pos] = b;
          s[par] = a;
        }
      }
      __syncthreads();
    }
  }
}

// Bucket of a tile and the number of records it holds (0 for padding tiles).
__device__ __forceinline__ void tile_bucket(const int* tile_off, const int* bcount, int bucketed, int64_t n,
                                            int64_t t, int* b_out, int* nvalid) {
  if (!bucketed) {
    *b_out = -1;
    int64_t rem = n - t * kTile;
    *nvalid = rem <= 0 ? 0 : (rem < kTile ? static_cast<int>(rem) : kTile);
    return;
  }
  int lo = 0, hi = kNumBuckets - 1;  // last bucket with tile_off[b] <= t
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (tile_off[mid] <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  *b_out = lo;
  int rem = bcount[lo] - static_cast<int>(t - tile_off[lo]) * kTile;
  *nvalid = rem <= 0 ? 0 : (rem < kTile ? rem : kTile);
}

// ------------------------------------------------------------------ prepare
__global__ void __launch_bounds__(256) batch_prepare_kernel(DevLib lib, BatchDev b, int use_pilot) {
  __shared__ uint32_t sh[168];
  const int q = blockIdx.x;
  for (int i = threadIdx.x; i < 168; i += blockDim.x) {
    b.hist[static_cast<size_t>(q) * 168 + i] = 0u;
    sh[i] = 0u;
  }
  if (threadIdx.x == 0) b.cnt[q] = 0u;
  if (!use_pilot) return;
  const int k = b.k[q];
  __syncthreads();
  const uint64_t q0 = b.queries[3 * q], q1 = b.queries[3 * q + 1], q2 = b.queries[3 * q + 2];
  const int64_t S = lib.n_tiles < kPilotTiles ? lib.n_tiles : kPilotTiles;
  for (int64_t i = threadIdx.x; i < S * kTile; i += blockDim.x) {
    int64_t t = (i / kTile) * lib.n_tiles / S;   // sample tiles spread over the whole layout
    int r = static_cast<int>(i % kTile);
    int64_t pos = t * kTile + r;
    if (__ldg(lib.perm + pos) < 0) continue;      // padding position
    const uint64_t* w = lib.words + t * (kWords * kTile);
    uint32_t d = __popcll(w[r] ^ q0) + __popcll(w[kTile + r] ^ q1) + __popcll(w[2 * kTile + r] ^ q2);
    atomicAdd(&sh[d], 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0, bound = 166u;
    for (int d = 0; d < kNumBuckets; ++d) {
      run += sh[d];
      if (k > 0 && run >= static_cast<uint32_t>(k)) {
        bound = static_cast<uint32_t>(d);
        break;
      }
    }
    b.thr[q] = bound;
  }
}

// --------------------------------------------------------- popcount scan
// Smallest D with >= k accepted records at distance <= D among bins 0..upto; 167 if none.
__device__ uint32_t warp_bound(const uint32_t* hist, int k, uint32_t upto, int lane) {
  uint32_t carry = 0, found = 167u;
  for (uint32_t base = 0; base <= upto && found == 167u; base += 32) {
    uint32_t bin = base + lane;
    uint32_t v = bin <= upto ? __ldcg(hist + bin) : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(kFull, v, o);
      if (lane >= o) v += t;
    }
    v += carry;
    uint32_t bal = __ballot_sync(kFull, v >= static_cast<uint32_t>(k) && bin <= upto);
    if (bal) found = base + __ffs(bal) - 1;
    carry = __shfl_sync(kFull, v, 31);
  }
  return found;
}

template <int QB>
__global__ void __launch_bounds__(256) batch_popc_kernel(DevLib lib, BatchDev b, int n_groups, int n_chunks,
                                                          uint32_t* work) {
  __shared__ uint64_t qw[QB][3];
  __shared__ int qpc[QB];
  __shared__ int qk[QB];
  __shared__ uint32_t qthr[QB];
  __shared__ int tile_off_s[kNumBuckets + 1];
  __shared__ int bcount_s[kNumBuckets + 1];
  __shared__ int s_item;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  if (lib.bucketed)
    for (int i = threadIdx.x; i < kNumBuckets + 1; i += blockDim.x) {
      tile_off_s[i] = lib.tile_off[i];
      bcount_s[i] = i < kNumBuckets ? lib.bcount[i] : 0;
    }
  const int n_items = n_groups * n_chunks;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = static_cast<int>(atomicAdd(work, 1u));
    __syncthreads();
    const int item = s_item;
    if (item >= n_items) break;
    const int g = item / n_chunks, c = item % n_chunks;
    for (int i = threadIdx.x; i < QB; i += blockDim.x) {
      int q = g * QB + i;
      bool on = q < b.Q && b.k[q] > 0;
      qk[i] = on ? b.k[q] : 0;
      uint64_t a0 = on ? b.queries[3 * q] : 0, a1 = on ? b.queries[3 * q + 1] : 0, a2 = on ? b.queries[3 * q + 2] : 0;
      qw[i][0] = a0;
      qw[i][1] = a1;
      qw[i][2] = a2;
      qpc[i] = __popcll(a0) + __popcll(a1) + __popcll(a2);
      qthr[i] = on ? ld_relaxed_u32(b.thr + q) : 0u;
    }
    __syncthreads();
    const int64_t t0 = lib.n_tiles * c / n_chunks, t1 = lib.n_tiles * (c + 1) / n_chunks;
    int64_t since_pull = 0;
    for (int64_t t = t0 + warp; t < t1; t += nwarps) {
      int bk, nvalid;
      tile_bucket(tile_off_s, bcount_s, lib.bucketed, lib.n, t, &bk, &nvalid);
      if (nvalid <= 0) continue;
      const uint64_t* w = lib.words + t * (kWords * kTile);
      uint64_t x0[4], x1[4], x2[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        int r = lane + 32 * m;
        x0[m] = __ldcs(w + r);
        x1[m] = __ldcs(w + kTile + r);
        x2[m] = __ldcs(w + 2 * kTile + r);
      }
      for (int i = 0; i < QB; ++i) {
        if (qk[i] == 0) continue;
        const uint32_t thr = *reinterpret_cast<volatile uint32_t*>(&qthr[i]);
        if (bk >= 0 && static_cast<uint32_t>(abs(bk - qpc[i])) > thr) continue;  // bucket lower bound
        const uint64_t a0 = qw[i][0], a1 = qw[i][1], a2 = qw[i][2];
        uint32_t d[4];
        bool hit = false;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          d[m] = __popcll(x0[m] ^ a0) + __popcll(x1[m] ^ a1) + __popcll(x2[m] ^ a2);
          hit |= (lane + 32 * m < nvalid) && d[m] <= thr;
        }
        if (!__any_sync(kFull, hit)) continue;
        // accept: count, append, then tighten the bound of this query
        const int q = g * QB + i;
        const int64_t off = b.cand_off[q], cap = b.cand_off[q + 1] - off;
        uint32_t* hq = b.hist + static_cast<size_t>(q) * 168;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          bool acc = (lane + 32 * m < nvalid) && d[m] <= thr;
          uint32_t bal = __ballot_sync(kFull, acc);
          if (!bal) continue;
          uint32_t base = 0;
          if (lane == __ffs(bal) - 1) base = atomicAdd(b.cnt + q, static_cast<uint32_t>(__popc(bal)));
          base = __shfl_sync(kFull, base, __ffs(bal) - 1);
          if (acc) {
            const uint32_t pos = static_cast<uint32_t>(t * kTile + lane + 32 * m);
            uint32_t slot = base + __popc(bal & lanemask_lt());
            if (slot < cap) b.cand[off + slot] = (static_cast<unsigned long long>(d[m]) << 32) | pos;
            uint32_t same = __match_any_sync(bal, d[m]);
            if ((same & lanemask_lt()) == 0) red_add_u32(hq + d[m], static_cast<uint32_t>(__popc(same)));
          }
        }
        __syncwarp();
        uint32_t D = warp_bound(hq, qk[i], thr, lane);
        if (D < thr && lane == 0) {
          atomicMin(b.thr + q, D);
          atomicMin(&qthr[i], D);
        }
        __syncwarp();
      }
      // fold in bounds tightened by other blocks now and then
      if (++since_pull == 16) {
        since_pull = 0;
        for (int i = lane; i < QB; i += 32) {
          int q = g * QB + i;
          if (qk[i] > 0) atomicMin(&qthr[i], ld_relaxed_u32(b.thr + q));
        }
      }
    }
  }
}

// ------------------------------------------------------------------- select
__global__ void __launch_bounds__(kSelThreads) batch_select_kernel(DevLib lib, BatchDev b) {
  extern __shared__ __align__(16) unsigned long long sm[];
  unsigned long long* fin = sm;
  unsigned long long* ties = sm + kSelFin;
  __shared__ uint32_t hs[168];
  __shared__ int s_T, s_cless, s_nfin, s_ntie, s_cnt;
  const int q = blockIdx.x;
  const int k = b.k[q];
  const int64_t ob = b.out_off[q];
  if (k <= 0 || lib.n == 0) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) {   // an empty library: every slot holds -1
      b.out_idx[ob + i] = -1;
      b.out_dist[ob + i] = -1;
    }
    if (threadIdx.x == 0) b.out_count[q] = 0;
    return;
  }
  const int k_eff = static_cast<int>(k < lib.n ? k : lib.n);
  const uint32_t cnt = b.cnt[q];
  const int64_t off = b.cand_off[q], cap = b.cand_off[q + 1] - off;
  if (static_cast<int64_t>(cnt) > cap) {
    if (threadIdx.x == 0) b.out_count[q] = -2;  // candidates were lost: exact fallback needed
    return;
  }
  for (int i = threadIdx.x; i < 168; i += blockDim.x) hs[i] = b.hist[static_cast<size_t>(q) * 168 + i];
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    int T = kNumBuckets;
    for (int d = 0; d < kNumBuckets; ++d) {
      if (run + hs[d] >= static_cast<uint32_t>(k_eff)) {
        T = d;
        break;
      }
      run += hs[d];
    }
    s_T = T;
    s_cless = static_cast<int>(run);
    s_nfin = 0;
    s_ntie = 0;
  }
  __syncthreads();
  const uint32_t T = static_cast<uint32_t>(s_T);
  const int cless = s_cless, need = k_eff - cless;
  // candidate keys hold layout positions: d << 32 | position -> d << 32 | library index
  unsigned long long* cq = b.cand + off;
  for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    unsigned long long key = cq[i];
    const int32_t idx = __ldg(lib.perm + static_cast<uint32_t>(key));
    key = (key & 0xFFFFFFFF00000000ull) | static_cast<uint32_t>(idx);
    cq[i] = key;
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    unsigned long long key = cq[i];
    uint32_t dd = static_cast<uint32_t>(key >> 32);
    if (dd < T) {
      int p = atomicAdd(&s_nfin, 1);
      if (p < kSelFin) fin[p] = key;
    } else if (dd == T) {
      int p = atomicAdd(&s_ntie, 1);
      if (p < kSelTies) ties[p] = key;
    }
  }
  __syncthreads();
  if (s_T >= kNumBuckets) {
    // fewer than k records were accepted: the starting bound was below the true
    // k-th distance (possible only with a predicted bound) -- exact fallback
    if (threadIdx.x == 0) b.out_count[q] = -2;
    return;
  }
  if (threadIdx.x == 0 && (s_nfin != cless || s_ntie < need)) atomicOr(b.err, DEVERR_INTERNAL);
  const int ntie = s_ntie;
  if (need > 0) {
    if (ntie <= kSelTies) {
      int p = next_pow2(ntie);
      for (int i = ntie + threadIdx.x; i < p; i += blockDim.x) ties[i] = ~0ull;
      __syncthreads();
      block_bitonic_sort(ties, p);
      for (int i = threadIdx.x; i < need; i += blockDim.x)
        if (cless + i < kSelFin) fin[cless + i] = ties[i];
    } else {
      uint32_t lo = 0, hi = 0x7FFFFFFFu;   // need-th smallest index at distance T
      while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        int local = 0;
        for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
          unsigned long long key = cq[i];
          local += (static_cast<uint32_t>(key >> 32) == T) && (static_cast<uint32_t>(key) <= mid);
        }
        atomicAdd(&s_cnt, local);
        __syncthreads();
        if (s_cnt >= need)
          hi = mid;
        else
          lo = mid + 1;
        __syncthreads();
      }
      if (threadIdx.x == 0) s_nfin = cless;
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
        unsigned long long key = cq[i];
        if (static_cast<uint32_t>(key >> 32) == T && static_cast<uint32_t>(key) <= lo) {
          int p = atomicAdd(&s_nfin, 1);
          if (p < kSelFin) fin[p] = key;
        }
      }
    }
  }
  __syncthreads();
  int p = next_pow2(k_eff);
  for (int i = k_eff + threadIdx.x; i < p; i += blockDim.x) fin[i] = ~0ull;
  __syncthreads();
  block_bitonic_sort(fin, p);
  for (int i = threadIdx.x; i < k; i += blockDim.x) {   // slots past k_eff hold -1
    b.out_idx[ob + i] = i < k_eff ? static_cast<int32_t>(fin[i] & 0xFFFFFFFFull) : -1;
    b.out_dist[ob + i] = i < k_eff ? static_cast<int32_t>(fin[i] >> 32) : -1;
  }
  if (threadIdx.x == 0) b.out_count[q] = k_eff;
}

}  // namespace

cudaError_t batch_prepare(const DevLib& lib, const BatchDev& b, int use_pilot, cudaStream_t s) {
  if (b.Q == 0) return cudaSuccess;
  batch_prepare_kernel<<<b.Q, 256, 0, s>>>(lib, b, use_pilot);
  return cudaGetLastError();
}

__global__ void thr_from_tau_kernel(BatchDev b, const float* tau) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= b.Q) return;
  const float t = ceilf(tau[q]);
  b.thr[q] = t <= 0.f ? 0u : (t >= 166.f ? 166u : static_cast<uint32_t>(t));
}

cudaError_t batch_thr_from_tau(const BatchDev& b, const float* tau, cudaStream_t s) {
  if (b.Q == 0) return cudaSuccess;
  thr_from_tau_kernel<<<(b.Q + 255) / 256, 256, 0, s>>>(b, tau);
  return cudaGetLastError();
}

template <int QB>
cudaError_t launch_batch_popc(const DevLib& lib, const BatchDev& b, int num_sms, uint32_t* work, cudaStream_t s) {
  const int grid = 2 * num_sms;
  const int n_groups = (b.Q + QB - 1) / QB;
  int n_chunks = (8 * grid + n_groups - 1) / n_groups;          // several items per block
  int64_t max_chunks = lib.n_tiles / 64 > 0 ? lib.n_tiles / 64 : 1;  // at least 64 tiles per chunk
  if (n_chunks > max_chunks) n_chunks = static_cast<int>(max_chunks);
  if (n_chunks < 1) n_chunks = 1;
  cudaError_t e = cudaMemsetAsync(work, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  batch_popc_kernel<QB><<<grid, 256, 0, s>>>(lib, b, n_groups, n_chunks, work);
  return cudaGetLastError();
}

cudaError_t batch_scan_popc(const DevLib& lib, const BatchDev& b, int num_sms, uint32_t* work, int qb,
                            cudaStream_t s) {
  if (b.Q == 0 || lib.n == 0) return cudaSuccess;
  if (qb <= 0) qb = kPopcBatchDefaultQB;
  if (qb == 32) return launch_batch_popc<32>(lib, b, num_sms, work, s);
  if (qb == 128) return launch_batch_popc<128>(lib, b, num_sms, work, s);
  return launch_batch_popc<64>(lib, b, num_sms, work, s);
}

cudaError_t batch_select(const DevLib& lib, const BatchDev& b, cudaStream_t s) {
  if (b.Q == 0) return cudaSuccess;
  const size_t smem = (kSelFin + kSelTies) * sizeof(unsigned long long);
  static std::atomic<uint64_t> configured{0};
  cudaError_t e = smem_attr_once(batch_select_kernel, smem, &configured);
  if (e != cudaSuccess) return e;
  batch_select_kernel<<<b.Q, kSelThreads, smem, s>>>(lib, b);
  return cudaGetLastError();
}

namespace {

// ------------------------------------------------------------- shard merge
// One warp per query: lane s holds the head of shard s's ascending list; each
// round the smallest key (distance << 32 | global index) over the lanes is
// written and its lane advances.  Indices of different shards never collide,
// so the keys are distinct and the order is the total (distance, index) order.
__global__ void shard_merge_kernel(ShardLists sl, int Q, const int64_t* __restrict__ off,
                                   const int32_t* __restrict__ k, int32_t* __restrict__ out_idx,
                                   int32_t* __restrict__ out_dist, int32_t* __restrict__ out_count) {
  const int lane = threadIdx.x & 31;
  const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (q >= Q) return;
  const int64_t o = off[q];
  const int kq = k[q];   // the slots from off[q] on may be more than k[q]; the results are not
  int cnt = 0, p = 0;
  if (lane < sl.n) cnt = sl.count[lane][q];
  auto key_at = [&](int i) -> unsigned long long {
    return (static_cast<unsigned long long>(static_cast<uint32_t>(sl.dist[lane][o + i])) << 32) |
           static_cast<uint32_t>(sl.base[lane] + sl.idx[lane][o + i]);
  };
  unsigned long long head = (lane < sl.n && p < cnt) ? key_at(p) : ~0ull;
  int n_out = 0;
  for (; n_out < kq; ++n_out) {
    unsigned long long m = head;
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) {
      const unsigned long long other = __shfl_xor_sync(kFull, m, sh);
      m = other < m ? other : m;
    }
    if (m == ~0ull) break;
    if (lane == 0) {
      out_idx[o + n_out] = static_cast<int32_t>(m & 0xFFFFFFFFull);
      out_dist[o + n_out] = static_cast<int32_t>(m >> 32);
    }
    if (head == m) {
      ++p;
      head = p < cnt ? key_at(p) : ~0ull;
    }
  }
  for (int i = n_out + lane; i < kq; i += 32) {   // slots past the merged count, up to k, hold -1
    out_idx[o + i] = -1;
    out_dist[o + i] = -1;
  }
  if (lane == 0) out_count[q] = n_out;
}

__global__ void progress_kernel(int64_t* slot, int64_t value) {
  if (threadIdx.x == 0) *reinterpret_cast<volatile int64_t*>(slot) = value;
}

}  // namespace

cudaError_t launch_shard_merge(const ShardLists& sl, int Q, const int64_t* off, const int32_t* k, int32_t* out_idx,
                               int32_t* out_dist, int32_t* out_count, cudaStream_t s) {
  if (Q <= 0) return cudaSuccess;
  const int warps = 8;
  shard_merge_kernel<<<(Q + warps - 1) / warps, 32 * warps, 0, s>>>(sl, Q, off, k, out_idx, out_dist, out_count);
  return cudaGetLastError();
}

cudaError_t launch_progress(int64_t* slot_dev, int64_t value, cudaStream_t s) {
  progress_kernel<<<1, 32, 0, s>>>(slot_dev, value);
  return cudaGetLastError();
}

}  // namespace fps

