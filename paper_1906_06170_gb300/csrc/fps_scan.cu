// Single-query exhaustive scan + exact top-k (one launch per query).
//
// Paper: Sec. 4.3 (Manhattan distance over the 166 keys) and Fig. 3 (pair
// each row with its distance, sort ascending, take the first k).  For 0/1 keys
// |a_j - b_j| = a_j XOR b_j, so a row's distance is
//   d = popc(q0 ^ x0) + popc(q1 ^ x1) + popc(q2 ^ x2)
// over the three packed 64-bit words.  The top-k is the k smallest keys
// key = d << 32 | index, i.e. ascending distance with ties by index.
//
// Design (one persistent CTA per SM, every warp independent):
//   * each warp streams 3 KB tiles of the library through its own ring of
//     shared-memory stages filled by 1-D TMA bulk copies (cp.async.bulk) that
//     complete on per-stage mbarriers; the library is read once, evict-first;
//   * tiles are visited by popcount bucket in order of the lower bound
//     |popc q - popc x| <= d (nearest buckets first), and a warp stops as soon
//     as the bound of its next tile exceeds the current distance threshold;
//   * a record is a candidate iff its key is <= the running threshold key.
//     The threshold is the min of (a) the smallest D such that at least k
//     accepted records have d <= D, read from the block's own histogram of
//     accepted distances in shared memory and published to all blocks
//     (atomicMin), and (b) the k-th key of any warp's local buffer (atomicMin).
//     Both are valid upper bounds of the true k-th key, so no top-k member is
//     ever rejected.  The block histograms reach the global one once, when
//     their block ends: a global histogram updated and re-read after every
//     tile puts every warp of the grid on the same few L2 lines;
//   * candidates go to a per-warp shared buffer; a full buffer is filtered
//     against the threshold and, if still longer than k, sorted and cut to k;
//   * the last CTA to finish reads the histogram -- exact below the final
//     threshold -- to get the k-th distance T and the number of records closer
//     than T, keeps every candidate below T plus the smallest indices at T,
//     sorts them and writes the result.  It then restores the scan state.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>

#include "fps_internal.h"

namespace fps {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kStages = 3;
// one ring stage: a 3 KB tile followed by the 16-byte threshold block of the
// scan state, both delivered by bulk copies that complete on the stage's mbarrier
constexpr int kThrBytes = 16;
// Work distribution.  Items (3 KB tiles in visit order) are swept front to
// back by the whole grid, so at any moment all warps read one contiguous
// window of the library.  The first kStaticNum/kStaticDen of the items are
// dealt round-robin (warp w takes w, w + W, w + 2W, ...); the rest are handed
// out one by one, still in sweep order, by kQueues counters on separate cache
// lines (warp w draws from counter w % kQueues), so warps the memory system
// serves faster take more of the tail.  Each warp keeps two requests in flight
// so the atomics' latency stays hidden.  Some SMs stream up to ~40% slower
// than the rest; their static share must end before the tail runs out, while
// tail items cost a little more than static ones: 5/8 static measured best.
constexpr int kStaticNum = 5, kStaticDen = 8;
constexpr int kQueues = 16;
constexpr int kStageBytes = kTileBytes + kThrBytes;
constexpr int kTieCap = 16384;          // tie keys sorted in shared memory by the merge
constexpr int kFinCap = 2048;           // >= FPS_K_MAX, power of two
constexpr int kWarpSortMax = 256;       // merge sorts up to this many keys in one warp

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Spin on an mbarrier phase, giving up at the deadline (no unbounded waits).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t deadline) {
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() > deadline) return false;
  }
  return true;
}

__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ uint64_t l2_evict_last_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
      : "memory");
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_add_u32(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ unsigned long long key_bound_of_dist(uint32_t d) {
  return (static_cast<unsigned long long>(d) << 32) | 0xFFFFFFFFull;
}

// -------------------------------------------------------------- sorting helpers
// Ascending bitonic sort of n (power of two) keys in shared memory by one warp.
__device__ void warp_bitonic_sort(unsigned long long* s, int n, int lane) {
  for (int kk = 2; kk <= n; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < (n >> 1); i += 32) {
        int pos = 2 * i - (i & (j - 1));
        int par = pos + j;
        bool asc = (pos & kk) == 0;
        unsigned long long a = s[pos], b = s[par];
        if ((a > b) == asc) {
          s[pos] = b;
          s[par] = a;
        }
      }
      __syncwarp();
    }
  }
}

// Same, by the whole block.
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

__device__ __forceinline__ int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// ---------------------------------------------------------- per-warp candidates
// Drop keys above the threshold; if more than k remain, sort and keep k, and
// publish the k-th key as a global bound.  Returns the new count.
__device__ int compact_buffer(unsigned long long* buf, int cnt, int k, unsigned long long& thr_key,
                              ScanState* st, int lane) {
  int kept = 0;
  for (int base = 0; base < cnt; base += 32) {
    int i = base + lane;
    unsigned long long v = i < cnt ? buf[i] : ~0ull;
    bool keep = i < cnt && v <= thr_key;
    __syncwarp();
    uint32_t bal = __ballot_sync(kFull, keep);
    if (keep) buf[kept + __popc(bal & lanemask_lt())] = v;
    kept += __popc(bal);
  }
  __syncwarp();
  if (kept > k) {
    int p = next_pow2(kept);
    for (int i = kept + lane; i < p; i += 32) buf[i] = ~0ull;
    __syncwarp();
    warp_bitonic_sort(buf, p, lane);
    kept = k;
    unsigned long long kth = buf[k - 1];
    if (kth < thr_key) {
      thr_key = kth;
      if (lane == 0) atomicMin(&st->thr_key, kth);
    }
  }
  __syncwarp();
  return kept;
}

// The smallest D with at least k accepted records at distance <= D in the
// block's histogram; 167 if none.  Lane l reads bins 6l .. 6l+5.  Other warps
// of the block may be adding to it: counts only grow, so a stale read gives a
// looser bound, never an invalid one (k distinct records within D exist).
__device__ uint32_t bound_from_block_hist(const uint32_t* sh_hist, int k, int lane) {
  uint32_t h[6] = {0, 0, 0, 0, 0, 0};
  if (lane < 28) {
    const volatile uint32_t* p = sh_hist + 6 * lane;
#pragma unroll
    for (int i = 0; i < 6; ++i) h[i] = p[i];
  }
  uint32_t sum = h[0] + h[1] + h[2] + h[3] + h[4] + h[5];
  uint32_t incl = sum;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  uint32_t bal = __ballot_sync(kFull, incl >= static_cast<uint32_t>(k));
  if (!bal) return 167u;
  const int src = __ffs(bal) - 1;
  uint32_t found = 167u;
  if (lane == src) {
    uint32_t run = incl - sum;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      run += h[i];
      if (run >= static_cast<uint32_t>(k) && found == 167u) found = 6 * lane + i;
    }
  }
  return __shfl_sync(kFull, found, src);
}

// Add the block's histogram to the global one (one warp, after the block's
// scan has ended).
__device__ __forceinline__ void flush_hist(const uint32_t* sh_hist, ScanState* st, int lane) {
  for (int b = lane; b < kNumBuckets; b += 32) {
    const uint32_t v = sh_hist[b];
    if (v) red_add_u32(&st->hist[b], v);
  }
  __syncwarp();
}

// Count accepted records of one warp step in the block's shared histogram,
// one shared atomic per distinct distance.
__device__ __forceinline__ void count_accepted(uint32_t* sh_hist, bool acc, uint32_t bal, uint32_t d) {
  if (acc) {
    uint32_t same = __match_any_sync(bal, d);
    if ((same & lanemask_lt()) == 0) atomicAdd(&sh_hist[d], static_cast<uint32_t>(__popc(same)));
  }
}

struct Tables {
  uint32_t sh_hist[168];          // accepted records of this block per distance
  int lv_start[kNumBuckets + 2];  // items before level L (level = |popc q - bucket|)
  int lo_b[kNumBuckets + 1];      // bucket popc q - L, or -1
  int hi_b[kNumBuckets + 1];      // bucket popc q + L, or -1
  int nt_lo[kNumBuckets + 1];     // tiles holding records in lo_b
  int tile_off[kNumBuckets + 1];
  int bcount[kNumBuckets + 1];
  int nlev;
  int is_last;
  int nfin;
  int ntie;
  int T;
  int cless;
  int wbase[32];                  // first candidate slot of each warp of the block
  uint32_t blk_base;              // first candidate slot of the block
};

struct Item {
  int64_t tile;
  int level;
  int nvalid;
};

__device__ __forceinline__ int tiles_of(int count) { return (count + kTile - 1) / kTile; }

__device__ __forceinline__ Item locate(const Tables& tb, int t, int& cur) {
  while (t >= tb.lv_start[cur + 1]) ++cur;
  int o = t - tb.lv_start[cur];
  int b, tl;
  if (o < tb.nt_lo[cur]) {
    b = tb.lo_b[cur];
    tl = o;
  } else {
    b = tb.hi_b[cur];
    tl = o - tb.nt_lo[cur];
  }
  Item it;
  it.tile = static_cast<int64_t>(tb.tile_off[b]) + tl;
  it.level = cur;
  int rem = tb.bcount[b] - tl * kTile;
  it.nvalid = rem < kTile ? rem : kTile;
  return it;
}

template <int WARPS, int CAP>
struct Smem {
  static constexpr size_t ring = static_cast<size_t>(WARPS) * kStages * kStageBytes;
  static constexpr size_t bufs = static_cast<size_t>(WARPS) * CAP * 8;
  static constexpr size_t bars = static_cast<size_t>(WARPS) * kStages * 8;
  static constexpr size_t items = static_cast<size_t>(WARPS) * kStages * 4;
  static constexpr size_t total = ring + bufs + bars + items + sizeof(Tables);
  static_assert(ring + bufs >= (kFinCap + kTieCap) * 8, "merge scratch must fit in the scan buffers");
  static_assert(WARPS <= 32, "one candidate base per warp in the tables");
};

// ---------------------------------------------------------------------- kernel
template <int WARPS, int CAP>
__global__ void __launch_bounds__(WARPS * 32, 1)
    scan_single_kernel(DevLib lib, const uint64_t* query_arg, int k_arg, ScanState* st,
                       unsigned long long* __restrict__ cand, int32_t* out_idx_arg, int32_t* out_dist_arg,
                       int32_t* out_count_arg, uint32_t* err, uint64_t timeout_ns, const ScanSlot* slot) {
  // indirect launch (the device-side fallback of a captured batch): the search is
  // described by a slot that a preceding kernel of the graph filled
  const uint64_t* __restrict__ query = slot ? slot->query : query_arg;
  const int k = slot ? slot->k : k_arg;
  int32_t* __restrict__ out_idx = slot ? slot->out_idx : out_idx_arg;
  int32_t* __restrict__ out_dist = slot ? slot->out_dist : out_dist_arg;
  int32_t* __restrict__ out_count = slot ? slot->out_count : out_count_arg;
  extern __shared__ __align__(128) unsigned char smem[];
  using L = Smem<WARPS, CAP>;
  unsigned char* ring_all = smem;
  unsigned long long* bufs_all = reinterpret_cast<unsigned long long*>(smem + L::ring);
  uint64_t* bars_all = reinterpret_cast<uint64_t*>(smem + L::ring + L::bufs);
  int* items_all = reinterpret_cast<int*>(smem + L::ring + L::bufs + L::bars);
  Tables& tb = *reinterpret_cast<Tables*>(smem + L::ring + L::bufs + L::bars + L::items);

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const uint64_t q0 = __ldg(query + 0), q1 = __ldg(query + 1), q2 = __ldg(query + 2);
  const int pq = __popcll(q0) + __popcll(q1) + __popcll(q2);
  const uint64_t deadline = global_ns() + timeout_ns;

  // ---- visit-order tables (nearest popcount buckets first)
  for (int b = tid; b < 168; b += blockDim.x) tb.sh_hist[b] = 0u;
  if (lib.bucketed) {
    for (int b = tid; b < kNumBuckets; b += blockDim.x) {
      tb.tile_off[b] = lib.tile_off[b];
      tb.bcount[b] = lib.bcount[b];
    }
  }
  __syncthreads();
  if (warp == 0) {
    if (lib.bucketed) {
      const int nlev = 1 + (pq > kBits - pq ? pq : kBits - pq);
      uint32_t carry = 0;
      for (int c = 0; c < 6; ++c) {
        int lv = c * 32 + lane;
        int lo = -1, hi = -1, ntl = 0, nth = 0;
        if (lv < nlev) {
          lo = pq - lv >= 0 ? pq - lv : -1;
          hi = (lv > 0 && pq + lv <= kBits) ? pq + lv : -1;
          ntl = lo >= 0 ? tiles_of(tb.bcount[lo]) : 0;
          nth = hi >= 0 ? tiles_of(tb.bcount[hi]) : 0;
        }
        uint32_t v = static_cast<uint32_t>(ntl + nth);
        for (int o = 1; o < 32; o <<= 1) {
          uint32_t t = __shfl_up_sync(kFull, v, o);
          if (lane >= o) v += t;
        }
        v += carry;
        if (lv < nlev) {
          tb.lo_b[lv] = lo;
          tb.hi_b[lv] = hi;
          tb.nt_lo[lv] = ntl;
          tb.lv_start[lv + 1] = static_cast<int>(v);
        }
        carry = __shfl_sync(kFull, v, 31);
      }
      __syncwarp();
      if (lane == 0) {
        tb.lv_start[0] = 0;
        tb.nlev = nlev;
        tb.lv_start[nlev + 1] = tb.lv_start[nlev];  // sentinel level: never entered
      }
    } else if (lane == 0) {
      tb.tile_off[0] = 0;
      tb.bcount[0] = static_cast<int>(lib.n);
      tb.lo_b[0] = 0;
      tb.hi_b[0] = -1;
      tb.nt_lo[0] = tiles_of(static_cast<int>(lib.n));
      tb.lv_start[0] = 0;
      tb.lv_start[1] = tb.nt_lo[0];
      tb.lv_start[2] = tb.nt_lo[0];
      tb.nlev = 1;
    }
    if (lane == 0) {
      tb.is_last = 0;
      tb.nfin = 0;
      tb.ntie = 0;
    }
  }
  if (lane == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bars_all[warp * kStages + s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // ---- per-warp streaming scan
  unsigned char* ring = ring_all + static_cast<size_t>(warp) * kStages * kStageBytes;
  uint64_t* bars = bars_all + warp * kStages;
  int* stage_item = items_all + warp * kStages;
  unsigned long long* buf = bufs_all + static_cast<size_t>(warp) * CAP;
  const int total = tb.lv_start[tb.nlev];
  const int W = gridDim.x * WARPS;
  const int gw = blockIdx.x * WARPS + warp;
  const int per_warp_static = static_cast<int>(static_cast<long long>(total) * kStaticNum / kStaticDen / W);
  const int dyn_base = per_warp_static * W;          // first item of the queued tail
  uint32_t* my_queue = &st->queue[32 * (gw % kQueues)];
  const uint64_t pol = l2_evict_first_policy();
  const uint64_t pol_keep = l2_evict_last_policy();

  unsigned long long thr_key = ~0ull;
  {
    unsigned long long g = ld_relaxed_u64(&st->thr_key);
    unsigned long long gd = key_bound_of_dist(ld_relaxed_u32(&st->thr_d));
    thr_key = g < gd ? g : gd;
  }
  int cnt = 0;
  int n_issued = 0;
  bool stop_issue = false;
  bool failed = false;
  int fail_j = 0;
  int cur_issue = 0, cur_proc = 0;

  // issue side: j-th item of the warp; tail items come from the warp's queue,
  // requested two items ahead (lane 0 holds the pending queue positions)
  int issue_j = 0;
  uint32_t pend0 = 0, pend1 = 0;
  if (lane == 0 && dyn_base < total) {
    pend0 = atomicAdd(my_queue, 1u);
    pend1 = atomicAdd(my_queue, 1u);
  }
  auto try_issue = [&](int j) {
    if (stop_issue) return;
    int t;
    if (issue_j < per_warp_static) {
      t = gw + issue_j * W;
    } else {
      uint32_t r = __shfl_sync(kFull, pend0, 0);
      t = dyn_base + (gw % kQueues) + kQueues * static_cast<int>(r);
      if (t < total && lane == 0) {
        pend0 = pend1;
        pend1 = atomicAdd(my_queue, 1u);
      }
    }
    if (t >= total) {
      stop_issue = true;
      return;
    }
    Item it = locate(tb, t, cur_issue);
    if (static_cast<uint32_t>(it.level) > static_cast<uint32_t>(thr_key >> 32)) {
      stop_issue = true;  // this and every later item is too far in popcount
      return;
    }
    ++issue_j;
    if (lane == 0) {
      uint64_t* bar = &bars[j % kStages];
      unsigned char* dst = ring + (j % kStages) * kStageBytes;
      stage_item[j % kStages] = t;
      mbar_arrive_expect_tx(bar, kStageBytes);
      bulk_copy_g2s(dst, lib.words + it.tile * (kWords * kTile), kTileBytes, bar, pol);
      bulk_copy_g2s(dst + kTileBytes, &st->thr_key, kThrBytes, bar, pol_keep);
    }
    n_issued = j + 1;
  };

  for (int j = 0; j < kStages; ++j) try_issue(j);

  for (int j = 0; j < n_issued; ++j) {
    const int stage = j % kStages;
    // every lane observes the phase (acquire of the bulk copy's writes); the
    // verdict is made warp-uniform so no lane leaves the loop alone
    bool landed = mbar_wait_bounded(&bars[stage], static_cast<uint32_t>((j / kStages) & 1), deadline);
    if (!__all_sync(kFull, landed)) {
      failed = true;
      fail_j = j;
      break;
    }
    const unsigned char* sb = ring + stage * kStageBytes;
    {
      // thresholds as they were when this tile was issued (never looser than the truth)
      unsigned long long g_key = *reinterpret_cast<const unsigned long long*>(sb + kTileBytes);
      uint32_t g_d = *reinterpret_cast<const uint32_t*>(sb + kTileBytes + 8);
      unsigned long long gd = key_bound_of_dist(g_d);
      if (g_key < thr_key) thr_key = g_key;
      if (gd < thr_key) thr_key = gd;
    }
    Item it = locate(tb, stage_item[stage], cur_proc);
    const uint32_t D = static_cast<uint32_t>(thr_key >> 32);
    if (static_cast<uint32_t>(it.level) <= D) {
      const uint64_t* s = reinterpret_cast<const uint64_t*>(sb);
      uint32_t d[4];
      bool c[4];
      bool any = false;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        int r = lane + 32 * m;
        uint64_t x0 = s[r], x1 = s[kTile + r], x2 = s[2 * kTile + r];
        d[m] = __popcll(x0 ^ q0) + __popcll(x1 ^ q1) + __popcll(x2 ^ q2);
        c[m] = (r < it.nvalid) && (d[m] <= D);
        any |= c[m];
      }
      if (__any_sync(kFull, any)) {
        // Re-derive the bound from the block's histogram and publish it.
        auto refresh_bound = [&]() {
          __syncwarp();
          const uint32_t Dstar = bound_from_block_hist(tb.sh_hist, k, lane);
          if (Dstar < 167u) {
            const unsigned long long nk = key_bound_of_dist(Dstar);
            if (nk < thr_key) {
              thr_key = nk;
              if (lane == 0) atomicMin(&st->thr_d, Dstar);
            }
          }
        };
        // First tile of the warp: count every record within the bound first and
        // take the block's bound from those counts, so that only records within
        // the new bound need their index and a buffer slot.  Counted records left
        // out lie above a valid bound, hence above the k-th distance, where the
        // merge needs no exact count.
        const bool first = j == 0;
        if (first) {
#pragma unroll
          for (int m = 0; m < 4; ++m) count_accepted(tb.sh_hist, c[m], __ballot_sync(kFull, c[m]), d[m]);
          refresh_bound();
        }
        const uint32_t Dn = static_cast<uint32_t>(thr_key >> 32);
        bool added = false;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          unsigned long long key = ~0ull;
          bool acc = false;
          if (c[m] && d[m] <= Dn) {
            int32_t idx = __ldg(lib.perm + it.tile * kTile + lane + 32 * m);
            key = (static_cast<unsigned long long>(d[m]) << 32) | static_cast<uint32_t>(idx);
            acc = key <= thr_key;
          }
          uint32_t bal = __ballot_sync(kFull, acc);
          if (acc) buf[cnt + __popc(bal & lanemask_lt())] = key;
          if (!first) count_accepted(tb.sh_hist, acc, bal, d[m]);
          cnt += __popc(bal);
          added |= bal != 0;
        }
        __syncwarp();
        if (added && !first) refresh_bound();
        if (cnt > CAP - kTile) cnt = compact_buffer(buf, cnt, k, thr_key, st, lane);
      }
    }
    __syncwarp();
    try_issue(j + kStages);
  }

  if (failed) {
    // stop issuing; wait (bounded) for every copy still in flight before leaving
    if (lane == 0) atomicOr(err, DEVERR_TIMEOUT);
    // items fail_j .. n_issued-1 are the copies not yet consumed; each is the
    // next phase of its stage, so waiting on that phase is well defined
    const uint64_t drain_deadline = global_ns() + (timeout_ns > kDrainNs ? timeout_ns : kDrainNs);
    for (int j = fail_j; j < n_issued; ++j)
      mbar_wait_bounded(&bars[j % kStages], static_cast<uint32_t>((j / kStages) & 1), drain_deadline);
  }

  // final per-warp selection against the block's latest bound, then hand the
  // candidates to the merge: one slot reservation per block
  {
    __syncwarp();
    const uint32_t Db = bound_from_block_hist(tb.sh_hist, k, lane);
    if (Db < 167u && key_bound_of_dist(Db) < thr_key) thr_key = key_bound_of_dist(Db);
  }
  cnt = compact_buffer(buf, cnt, k, thr_key, st, lane);
  if (lane == 0) tb.wbase[warp] = cnt;
  __syncthreads();
  if (tid == 0) {
    uint32_t tot = 0;
    for (int w = 0; w < WARPS; ++w) {
      const int c = tb.wbase[w];
      tb.wbase[w] = static_cast<int>(tot);
      tot += static_cast<uint32_t>(c);
    }
    tb.blk_base = tot ? atomicAdd(&st->ncand, tot) : 0u;
  }
  __syncthreads();
  {
    const uint32_t base = tb.blk_base + static_cast<uint32_t>(tb.wbase[warp]);
    for (int i = lane; i < cnt; i += 32) cand[base + i] = buf[i];
  }

  // ---- the block's counts to the global histogram, then the last block merges
  if (warp == 0) flush_hist(tb.sh_hist, st, lane);
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    unsigned prev = atomicAdd(&st->done, 1u);
    tb.is_last = (prev == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!tb.is_last) return;
  __threadfence();
  // In a sequence of searches (programmatic dependent launches, alternating
  // between two scan states) this grid may have started while the previous
  // search was still merging.  The merge waits for that grid to finish, then
  // lets the next search start on the SMs this grid has already released.
  // Without a programmatic dependency both instructions return at once.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  unsigned long long* fin = reinterpret_cast<unsigned long long*>(smem);
  unsigned long long* ties = fin + kFinCap;
  const int k_eff = static_cast<int>(k < lib.n ? k : lib.n);
  int* hs = tb.lo_b;  // reuse: 167 ints
  for (int b = tid; b < kNumBuckets; b += blockDim.x) hs[b] = static_cast<int>(ld_relaxed_u32(&st->hist[b]));
  __syncthreads();
  if (warp == 0) {
    // T = first distance whose running count reaches k_eff (warp prefix sums, 32 bins a round)
    uint32_t carry = 0;
    int T = kNumBuckets, cl = 0;
    for (int c0 = 0; c0 < kNumBuckets; c0 += 32) {
      const int b = c0 + lane;
      const uint32_t v = b < kNumBuckets ? static_cast<uint32_t>(hs[b]) : 0u;
      uint32_t incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t hit = __ballot_sync(kFull, b < kNumBuckets && carry + incl >= static_cast<uint32_t>(k_eff));
      if (hit) {
        const int f = __ffs(hit) - 1;
        T = c0 + f;
        cl = static_cast<int>(carry + __shfl_sync(kFull, incl - v, f));
        break;
      }
      carry += __shfl_sync(kFull, incl, 31);
    }
    if (lane == 0) {
      tb.T = T;
      tb.cless = T < kNumBuckets ? cl : static_cast<int>(carry);
    }
  }
  __syncthreads();
  const uint32_t T = static_cast<uint32_t>(tb.T);
  const int cless = tb.cless;
  const int need = k_eff - cless;  // smallest indices still needed at distance T
  const uint32_t ncand = ld_relaxed_u32(&st->ncand);
  constexpr int kGather = 8;  // candidate loads in flight per thread
  for (uint32_t base = 0; base < ncand; base += blockDim.x * kGather) {
    unsigned long long v[kGather];
#pragma unroll
    for (int u = 0; u < kGather; ++u) {
      const uint32_t i = base + u * blockDim.x + tid;
      v[u] = i < ncand ? __ldcg(cand + i) : ~0ull;
    }
#pragma unroll
    for (int u = 0; u < kGather; ++u) {
      const uint32_t dd = static_cast<uint32_t>(v[u] >> 32);
      if (dd < T) {
        int p = atomicAdd(&tb.nfin, 1);
        if (p < kFinCap) fin[p] = v[u];
      } else if (dd == T) {
        int p = atomicAdd(&tb.ntie, 1);
        if (p < kTieCap) ties[p] = v[u];
      }
    }
  }
  __syncthreads();
  if (tid == 0 && (tb.nfin != cless || tb.T >= kNumBuckets || tb.ntie < need)) atomicOr(err, DEVERR_INTERNAL);
  const int ntie = tb.ntie;
  if (need > 0) {
    if (ntie <= kTieCap) {
      const int p = next_pow2(ntie);
      if (p <= kWarpSortMax) {   // few ties: one warp sorts them, no block-wide barriers
        if (warp == 0) {
          for (int i = ntie + lane; i < p; i += 32) ties[i] = ~0ull;
          __syncwarp();
          warp_bitonic_sort(ties, p, lane);
          for (int i = lane; i < need; i += 32)
            if (cless + i < kFinCap) fin[cless + i] = ties[i];
        }
      } else {
        for (int i = ntie + tid; i < p; i += blockDim.x) ties[i] = ~0ull;
        __syncthreads();
        block_bitonic_sort(ties, p);
        for (int i = tid; i < need; i += blockDim.x)
          if (cless + i < kFinCap) fin[cless + i] = ties[i];
      }
    } else {
      // Many equal distances: find the need-th smallest index at distance T by bisection.
      __shared__ int s_cnt;
      uint32_t lo = 0, hi = 0x7FFFFFFFu;
      while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (tid == 0) s_cnt = 0;
        __syncthreads();
        int local = 0;
        for (uint32_t i = tid; i < ncand; i += blockDim.x) {
          unsigned long long key = __ldcg(cand + i);
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
      if (tid == 0) tb.nfin = cless;
      __syncthreads();
      for (uint32_t i = tid; i < ncand; i += blockDim.x) {
        unsigned long long key = __ldcg(cand + i);
        if (static_cast<uint32_t>(key >> 32) == T && static_cast<uint32_t>(key) <= lo) {
          int p = atomicAdd(&tb.nfin, 1);
          if (p < kFinCap) fin[p] = key;
        }
      }
    }
  }
  __syncthreads();
  {
    const int p = next_pow2(k_eff);
    if (p <= kWarpSortMax) {
      if (warp == 0) {
        for (int i = k_eff + lane; i < p; i += 32) fin[i] = ~0ull;
        __syncwarp();
        warp_bitonic_sort(fin, p, lane);
        for (int i = lane; i < k_eff; i += 32) {
          out_idx[i] = static_cast<int32_t>(fin[i] & 0xFFFFFFFFull);
          out_dist[i] = static_cast<int32_t>(fin[i] >> 32);
        }
        if (lane == 0) *out_count = k_eff;
      }
    } else {
      for (int i = k_eff + tid; i < p; i += blockDim.x) fin[i] = ~0ull;
      __syncthreads();
      block_bitonic_sort(fin, p);
      for (int i = tid; i < k_eff; i += blockDim.x) {
        out_idx[i] = static_cast<int32_t>(fin[i] & 0xFFFFFFFFull);
        out_dist[i] = static_cast<int32_t>(fin[i] >> 32);
      }
      if (tid == 0) *out_count = k_eff;
    }
  }
  // slots past min(k, N), up to k, hold -1
  for (int i = k_eff + tid; i < k; i += blockDim.x) {
    out_idx[i] = -1;
    out_dist[i] = -1;
  }
  // restore the scan state for the next search on this workspace
  for (int b = tid; b < 168; b += blockDim.x) st->hist[b] = 0u;
  if (tid == 0) {
    st->thr_key = ~0ull;
    st->thr_d = 166u;
    st->ncand = 0u;
    st->done = 0u;
  }
  for (int c = tid; c < kQueues; c += blockDim.x) st->queue[32 * c] = 0u;
}

constexpr int kSmallWarps = 16, kSmallCap = 256;   // k <= 128
constexpr int kLargeWarps = 8, kLargeCap = 2048;   // k <= 1920

// ------------------------------------------------------------ small libraries
// A library whose layout has at most kSmPer positions per thread of a grid of
// kSmThreads-thread blocks (about 1.2 M records on 152 SMs) is scanned in one
// wave, without the bucket order: with a handful of records per thread, the fixed
// costs of the streaming kernel (visit-order tables, copy rings, running
// bounds, two global atomics per block) are most of a query's time.
//   1. thread t computes the distances of layout positions t, t + T, t + 2T, ...
//      (T threads in the grid; consecutive threads read consecutive records of
//      the word-major tiles, so the loads coalesce);
//   2. the block histograms its distances and takes T_b, the smallest D with at
//      least k of its records at distance <= D (every record if it holds fewer).
//      The k-th distance T of the whole library is <= T_b for every block;
//   3. the block writes its records below T_b (fewer than k) and those at T_b
//      (as many as its region has room for) as keys d << 32 | index to its own
//      region of the candidate array, and its counts and T_b to the scan state;
//   4. the last block to finish reads every region.  The keys hold every record
//      below T, and every record at T unless some block with T_b == T ran out of
//      room, in which case the records at T are read again from the library.
//      The k-th smallest candidate distance is T; the keys below it plus the
//      smallest indices at T, sorted, are the answer (Fig. 3's first k rows).
constexpr int kSmThreads = 1024;
constexpr int kSmPer = 8;                   // layout positions per thread
constexpr int kSmMaxK = 128;                // largest k served
constexpr int kSmRegion = 2048;             // keys per block: [0, kSmMaxK) below T_b, then those at T_b
constexpr int kSmTieRoom = kSmRegion - kSmMaxK;
constexpr int kSmTieCap = 2048;             // keys at T sorted in shared memory by the merge
constexpr size_t kSmSmem = static_cast<size_t>(kSmMaxK + kSmTieCap) * sizeof(unsigned long long);
static_assert(kSmRegion <= kSmallWarps * (kSmallCap - kTile), "a block's region fits the candidate array");

// bcnt word of a block: keys below T_b (bits 0-7), keys at T_b written (bits 8-19),
// T_b (bits 20-27; 255 when the block holds fewer than k records), room ran out (bit 31)
__device__ __forceinline__ uint32_t sm_pack(uint32_t lt, uint32_t eq, uint32_t tb, bool over) {
  return lt | (eq << 8) | (tb << 20) | (over ? 0x80000000u : 0u);
}

// Warp-aggregated append: the lanes with take write key to dst[counter++] in lane order
// (one shared atomic for the warp); slots at or past cap are counted, not written.
// Called by all 32 lanes together.
__device__ __forceinline__ void warp_append(bool take, unsigned long long key, uint32_t* counter,
                                            unsigned long long* dst, uint32_t cap, int lane) {
  const uint32_t m = __ballot_sync(kFull, take);
  if (m == 0) return;
  const int lead = __ffs(m) - 1;
  uint32_t base = 0;
  if (lane == lead) base = atomicAdd(counter, static_cast<uint32_t>(__popc(m)));
  base = __shfl_sync(kFull, base, lead);
  if (take) {
    const uint32_t p = base + static_cast<uint32_t>(__popc(m & lanemask_lt()));
    if (p < cap) dst[p] = key;
  }
}

// Distance of layout position p to the query, or 0xFF for a padding position.  No
// branch depends on a load, so the loads of consecutive calls are all in flight together.
__device__ __forceinline__ uint32_t sm_dist(const DevLib& lib, int64_t p, uint64_t q0, uint64_t q1, uint64_t q2) {
  const uint64_t* w = lib.words + (p >> 7) * (kWords * kTile) + (p & (kTile - 1));
  const uint64_t x0 = __ldg(w), x1 = __ldg(w + kTile), x2 = __ldg(w + 2 * kTile);
  const int32_t idx = __ldg(lib.perm + p);
  const uint32_t d = static_cast<uint32_t>(__popcll(x0 ^ q0) + __popcll(x1 ^ q1) + __popcll(x2 ^ q2));
  return idx < 0 ? 0xFFu : d;
}

// Ascending bitonic sort of 32 x E keys held by one warp, key i = lane + 32 e in x[e] of
// lane `lane` (E a power of two): partners in other lanes are exchanged by shuffles,
// partners in the same lane by register swaps.
template <int E>
__device__ __forceinline__ void warp_sort_regs(unsigned long long (&x)[E], int lane) {
  constexpr int n = 32 * E;
#pragma unroll
  for (int kk = 2; kk <= n; kk <<= 1) {
#pragma unroll
    for (int j = kk >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int pe = e ^ (j >> 5);
          if (pe > e) {
            const bool asc = ((lane + 32 * e) & kk) == 0;
            const unsigned long long a = x[e], b = x[pe];
            if ((a > b) == asc) {
              x[e] = b;
              x[pe] = a;
            }
          }
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int i = lane + 32 * e;
          const unsigned long long y = __shfl_xor_sync(kFull, x[e], j);
          const bool asc = (i & kk) == 0, lower = (lane & j) == 0;
          const bool take_min = lower == asc;
          x[e] = take_min ? (y < x[e] ? y : x[e]) : (y > x[e] ? y : x[e]);
        }
      }
    }
  }
}

// The merge of the small-library scan, by its last block.  keys: kSmMaxK + kSmTieCap
// shared keys.
__device__ void sm_merge(const DevLib& lib, int k, ScanState* st, const unsigned long long* __restrict__ cand,
                         int32_t* out_idx, int32_t* out_dist, int32_t* out_count, uint32_t* err, uint64_t q0,
                         uint64_t q1, uint64_t q2, unsigned long long* keys) {
  __shared__ uint32_t bc[kScanSmallMaxBlocks];
  __shared__ uint32_t s_T, s_cless, s_nfin, s_ntie, s_tover, s_cnt;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = static_cast<int>(gridDim.x);
  const int k_eff = static_cast<int>(k < lib.n ? k : lib.n);
  unsigned long long* fin = keys;              // the answer: keys below T, then the chosen ones at T
  unsigned long long* ties = keys + kSmMaxK;   // keys at T
  if (tid == 0) {
    s_nfin = 0u;
    s_ntie = 0u;
    s_tover = 0xFFFFFFFFu;
  }
  __syncthreads();
  for (int b = tid; b < nb; b += kSmThreads) {
    const uint32_t w = __ldcg(&st->bcnt[b]);
    bc[b] = w;
    if (w >> 31) atomicMin(&s_tover, (w >> 20) & 0xFFu);   // a block whose keys at its T_b ran out of room
  }
  if (warp == kSmThreads / 32 - 1) {
    // T = first distance whose running count reaches k_eff.  The blocks added their counts
    // at distances <= their own T_b, so the histogram is exact up to min T_b >= T.
    uint32_t carry = 0;
    int T = kNumBuckets, cl = 0;
    for (int c0 = 0; c0 < kNumBuckets; c0 += 32) {
      const int b = c0 + lane;
      const uint32_t v = b < kNumBuckets ? __ldcg(&st->hist[b]) : 0u;
      uint32_t incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t hit = __ballot_sync(kFull, b < kNumBuckets && carry + incl >= static_cast<uint32_t>(k_eff));
      if (hit) {
        const int f = __ffs(hit) - 1;
        T = c0 + f;
        cl = static_cast<int>(carry + __shfl_sync(kFull, incl - v, f));
        break;
      }
      carry += __shfl_sync(kFull, incl, 31);
    }
    if (lane == 0) {
      s_T = static_cast<uint32_t>(T);
      s_cless = static_cast<uint32_t>(cl);
    }
  }
  __syncthreads();
  // The keys that can hold the answer, fn(key) for each: a region's keys below its T_b,
  // and its keys at T_b only when T_b == T (T <= T_b, so otherwise they lie above T).
  // Warp w reads regions w, w + 16, ..., ten at a time, 32 consecutive keys per load, the
  // first 64 keys of each of the ten regions in flight together; keys past 64 in a region
  // are read 32 at a time.  Called once T is known.
  constexpr int kWarps = kSmThreads / 32, kBatch = 10;
  auto key_index = [](uint32_t i, uint32_t lt) { return i < lt ? i : kSmMaxK + (i - lt); };
  auto keys_of = [&](uint32_t w) {
    const uint32_t lt = w & 0xFFu;
    return ((w >> 20) & 0xFFu) == s_T ? lt + ((w >> 8) & 0xFFFu) : lt;
  };
  auto for_each_key = [&](auto&& fn) {
    for (int b0 = warp; b0 < nb; b0 += kWarps * kBatch) {
      unsigned long long v[kBatch][2];
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int b = b0 + kWarps * j;
        const uint32_t w = b < nb ? bc[b] : 0u, lt = w & 0xFFu, n = b < nb ? keys_of(w) : 0u;
        const unsigned long long* reg = cand + static_cast<size_t>(b < nb ? b : 0) * kSmRegion;
        v[j][0] = static_cast<uint32_t>(lane) < n ? __ldcg(reg + key_index(lane, lt)) : ~0ull;
        v[j][1] = static_cast<uint32_t>(lane + 32) < n ? __ldcg(reg + key_index(lane + 32, lt)) : ~0ull;
      }
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        if (v[j][0] != ~0ull) fn(v[j][0]);
        if (v[j][1] != ~0ull) fn(v[j][1]);
      }
      for (int j = 0; j < kBatch; ++j) {
        const int b = b0 + kWarps * j;
        if (b >= nb) break;
        const uint32_t w = bc[b], lt = w & 0xFFu, n = keys_of(w);
        const unsigned long long* reg = cand + static_cast<size_t>(b) * kSmRegion;
        for (uint32_t i = 64u + lane; i < n; i += 32u) fn(__ldcg(reg + key_index(i, lt)));
      }
    }
  };
  __syncthreads();
  const uint32_t T = s_T;
  const int cless = static_cast<int>(s_cless);
  const int need = k_eff - cless;   // smallest indices still needed at distance T
  if (T >= static_cast<uint32_t>(kNumBuckets)) {
    if (tid == 0) atomicOr(err, DEVERR_INTERNAL);   // fewer candidates than k: cannot happen
  } else {
    // keys at T come from the regions unless a block with T_b == T ran out of room for
    // them; then from the library itself
    const bool from_lib = s_tover == T;
    const int64_t n_pos = lib.n_tiles * kTile;
    auto for_each_tie = [&](auto&& fn) {
      if (from_lib) {
        for (int64_t p = tid; p < n_pos; p += kSmThreads)
          if (sm_dist(lib, p, q0, q1, q2) == T)
            fn((static_cast<unsigned long long>(T) << 32) | static_cast<uint32_t>(__ldg(lib.perm + p)));
      } else {
        for_each_key([&](unsigned long long key) {
          if (static_cast<uint32_t>(key >> 32) == T) fn(key);
        });
      }
    };
    auto add = [](uint32_t* counter, unsigned long long* dst, uint32_t cap, unsigned long long key) {
      const uint32_t p = atomicAdd(counter, 1u);
      if (p < cap) dst[p] = key;
    };
    for_each_key([&](unsigned long long key) {
      const uint32_t d = static_cast<uint32_t>(key >> 32);
      if (d < T)
        add(&s_nfin, fin, kSmMaxK, key);
      else if (d == T && !from_lib)
        add(&s_ntie, ties, kSmTieCap, key);
    });
    if (from_lib) for_each_tie([&](unsigned long long key) { add(&s_ntie, ties, kSmTieCap, key); });
    __syncthreads();
    if (tid == 0 && (s_nfin != static_cast<uint32_t>(cless) || s_ntie < static_cast<uint32_t>(need)))
      atomicOr(err, DEVERR_INTERNAL);
    const int ntie = static_cast<int>(s_ntie);
    // the keys below T and those at T sorted together in one warp's registers when they fit
    // in kSmMaxK; otherwise the need smallest indices at T are chosen first
    const int nt = need > 0 ? ntie : 0;
    const bool together = cless + nt <= kSmMaxK;
    if (need > 0 && !together) {
      if (ntie <= kSmThreads) {
        // one key per thread: the need-th smallest index by bisection, each step one
        // block-wide count; the need keys at or below it are the ones (indices differ)
        const bool has = tid < ntie;
        const unsigned long long mine = has ? ties[tid] : ~0ull;
        const uint32_t my = static_cast<uint32_t>(mine);
        uint32_t lo = 0, hi = static_cast<uint32_t>(lib.n - 1);
        while (lo < hi) {
          const uint32_t mid = lo + (hi - lo) / 2;
          if (__syncthreads_count(has && my <= mid) >= need)
            hi = mid;
          else
            lo = mid + 1;
        }
        warp_append(has && my <= lo, mine, &s_nfin, fin, kSmMaxK, lane);
      } else if (ntie <= kSmTieCap) {
        const int p2 = next_pow2(ntie);
        {
          for (int i = ntie + tid; i < p2; i += kSmThreads) ties[i] = ~0ull;
          __syncthreads();
          block_bitonic_sort(ties, p2);
          for (int i = tid; i < need; i += kSmThreads) fin[cless + i] = ties[i];
        }
      } else {
        // very many records at T: the need-th smallest index among them, by bisection
        uint32_t lo = 0, hi = 0x7FFFFFFFu;
        while (lo < hi) {
          const uint32_t mid = lo + (hi - lo) / 2;
          if (tid == 0) s_cnt = 0u;
          __syncthreads();
          uint32_t local = 0;
          for_each_tie([&](unsigned long long key) { local += static_cast<uint32_t>(key) <= mid; });
          atomicAdd(&s_cnt, local);
          __syncthreads();
          if (s_cnt >= static_cast<uint32_t>(need))
            hi = mid;
          else
            lo = mid + 1;
          __syncthreads();
        }
        if (tid == 0) s_nfin = static_cast<uint32_t>(cless);
        __syncthreads();
        for_each_tie([&](unsigned long long key) {
          if (static_cast<uint32_t>(key) <= lo) add(&s_nfin, fin, kSmMaxK, key);
        });
      }
    }
    __syncthreads();
    if (warp == 0) {
      // element i = lane + 32 e: fin[0 .. cless) then ties[0 .. nt) (together), or fin[0 .. k_eff)
      unsigned long long x[kSmMaxK / 32];
#pragma unroll
      for (int e = 0; e < kSmMaxK / 32; ++e) {
        const int i = lane + 32 * e;
        if (together)
          x[e] = i < cless ? fin[i] : (i - cless < nt ? ties[i - cless] : ~0ull);
        else
          x[e] = i < k_eff ? fin[i] : ~0ull;
      }
      warp_sort_regs(x, lane);
      // the answer is the k_eff smallest keys (keys are unique: distance, then index)
#pragma unroll
      for (int e = 0; e < kSmMaxK / 32; ++e) {
        const int i = lane + 32 * e;
        if (i < k_eff) {
          out_idx[i] = static_cast<int32_t>(x[e] & 0xFFFFFFFFull);
          out_dist[i] = static_cast<int32_t>(x[e] >> 32);
        }
      }
      if (lane == 0) *out_count = k_eff;
    }
  }
  // slots past min(k, N), up to k, hold -1
  for (int i = k_eff + tid; i < k; i += kSmThreads) {
    out_idx[i] = -1;
    out_dist[i] = -1;
  }
  // restore the scan state for the next search on this workspace
  for (int b = tid; b < nb; b += kSmThreads) st->bcnt[b] = 0u;
  for (int b = tid; b < 168; b += kSmThreads) st->hist[b] = 0u;
  if (tid == 0) st->done = 0u;
}

__global__ void __launch_bounds__(kSmThreads, 1)
    scan_small_kernel(DevLib lib, const uint64_t* __restrict__ query, int k, ScanState* st,
                      unsigned long long* __restrict__ cand, int32_t* __restrict__ out_idx,
                      int32_t* __restrict__ out_dist, int32_t* __restrict__ out_count, uint32_t* err) {
  extern __shared__ __align__(16) unsigned long long sm_keys[];   // merge: [below T][at T]
  __shared__ uint32_t hist[168];
  __shared__ uint32_t s_lt, s_eq, s_tb, s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n_pos = lib.n_tiles * kTile;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * kSmThreads;
  const int64_t g = static_cast<int64_t>(blockIdx.x) * kSmThreads + tid;
  const uint64_t q0 = __ldg(query), q1 = __ldg(query + 1), q2 = __ldg(query + 2);
  for (int b = tid; b < 168; b += kSmThreads) hist[b] = 0u;
  if (tid == 0) {
    s_lt = 0u;
    s_eq = 0u;
  }
  // 1. distances, 8 bits each (0xFF: no record)
  uint32_t dpk[kSmPer / 4];
#pragma unroll
  for (int i = 0; i < kSmPer / 4; ++i) dpk[i] = 0u;
#pragma unroll
  for (int i = 0; i < kSmPer; ++i) {
    // positions past the layout read its last position (a valid address) and are dropped
    const int64_t p = g + i * stride;
    const uint32_t d = sm_dist(lib, p < n_pos ? p : n_pos - 1, q0, q1, q2);
    dpk[i >> 2] |= (p < n_pos ? d : 0xFFu) << (8 * (i & 3));
  }
  __syncthreads();
  // 2. the block's histogram of its distances
#pragma unroll
  for (int i = 0; i < kSmPer; ++i) {
    const uint32_t d = (dpk[i >> 2] >> (8 * (i & 3))) & 0xFFu;
    if (d != 0xFFu) atomicAdd(&hist[d], 1u);
  }
  __syncthreads();
  if (warp == 0) {
    uint32_t carry = 0, tb = 0xFFu;
    for (int c0 = 0; c0 < kNumBuckets && tb == 0xFFu; c0 += 32) {
      const int b = c0 + lane;
      const uint32_t v = b < kNumBuckets ? hist[b] : 0u;
      uint32_t incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t hit = __ballot_sync(kFull, b < kNumBuckets && carry + incl >= static_cast<uint32_t>(k));
      if (hit) tb = static_cast<uint32_t>(c0 + __ffs(hit) - 1);
      carry += __shfl_sync(kFull, incl, 31);
    }
    if (lane == 0) s_tb = tb;
  }
  __syncthreads();
  // 3. the block's counts at distances <= T_b to the global histogram (exact there for
  // D <= min T_b, where the k-th distance lies), and its keys below T_b, then at T_b,
  // into its region
  const uint32_t tb = s_tb;
  for (int b = tid; b < kNumBuckets && static_cast<uint32_t>(b) <= tb; b += kSmThreads)
    if (hist[b]) red_add_u32(&st->hist[b], hist[b]);
  unsigned long long* region = cand + static_cast<size_t>(blockIdx.x) * kSmRegion;
#pragma unroll
  for (int i = 0; i < kSmPer; ++i) {
    const uint32_t d = (dpk[i >> 2] >> (8 * (i & 3))) & 0xFFu;
    if (d <= tb && d != 0xFFu) {
      const unsigned long long key =
          (static_cast<unsigned long long>(d) << 32) | static_cast<uint32_t>(__ldg(lib.perm + g + i * stride));
      if (d < tb) {
        region[atomicAdd(&s_lt, 1u)] = key;   // fewer than k <= kSmMaxK
      } else {
        const uint32_t slot = atomicAdd(&s_eq, 1u);
        if (slot < static_cast<uint32_t>(kSmTieRoom)) region[kSmMaxK + slot] = key;
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t eq = s_eq;
    st->bcnt[blockIdx.x] = sm_pack(s_lt, min(eq, static_cast<uint32_t>(kSmTieRoom)), tb, eq > kSmTieRoom);
  }
  // one fence for the keys and the counts, then the count of finished blocks
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(&st->done, 1u) == gridDim.x - 1 ? 1u : 0u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // in a sequence of searches, wait for the previous one to finish before the merge and
  // let the next one start (see the streaming kernel)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  sm_merge(lib, k, st, cand, out_idx, out_dist, out_count, err, q0, q1, q2, sm_keys);
}

__global__ void scan_state_init_kernel(ScanState* st) {
  for (int b = threadIdx.x; b < 168; b += blockDim.x) st->hist[b] = 0u;
  for (int b = threadIdx.x; b < kScanSmallMaxBlocks; b += blockDim.x) st->bcnt[b] = 0u;
  if (threadIdx.x == 0) {
    st->thr_key = ~0ull;
    st->thr_d = 166u;
    st->done = 0u;
    st->ncand = 0u;
  }
  for (int c = threadIdx.x; c < kQueues; c += blockDim.x) st->queue[32 * c] = 0u;
}

template <int WARPS, int CAP>
cudaError_t configure_cfg() {
  static std::atomic<uint64_t> configured{0};   // one per instantiation, a bit per device
  return smem_attr_once(scan_single_kernel<WARPS, CAP>, Smem<WARPS, CAP>::total, &configured);
}

template <int WARPS, int CAP>
cudaError_t launch_cfg(const DevLib& lib, const uint64_t* q, int k, ScanState* st, unsigned long long* cand,
                       int32_t* oi, int32_t* od, int32_t* oc, uint32_t* err, int num_sms, uint64_t tns,
                       bool programmatic, cudaStream_t s, const ScanSlot* slot = nullptr) {
  using L = Smem<WARPS, CAP>;
  auto kern = scan_single_kernel<WARPS, CAP>;
  cudaError_t ce = configure_cfg<WARPS, CAP>();
  if (ce != cudaSuccess) return ce;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(num_sms));
  cfg.blockDim = dim3(WARPS * 32);
  cfg.dynamicSmemBytes = L::total;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = programmatic ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, lib, q, k, st, cand, oi, od, oc, err, tns, slot);
}

// Device-side fallback of a captured batch: find the next query whose count is -2 (it needs
// the exact scan), describe it in the slot and set the graph's loop condition (1 = found).
// One warp; the only caller of cudaGraphSetConditional is lane 0.
__global__ void fallback_pick_kernel(const uint64_t* queries, const int32_t* k, const int64_t* out_off,
                                     int32_t* oi, int32_t* od, int32_t* oc, int Q, ScanSlot* slot, int first,
                                     cudaGraphConditionalHandle h) {
  const int lane = threadIdx.x;
  const int from = first ? 0 : slot->cursor + 1;
  int found = -1;
  for (int base = from; base < Q; base += 32) {
    const int q = base + lane;
    const uint32_t b = __ballot_sync(kFull, q < Q && oc[q] == -2 && k[q] > 0);
    if (b) {
      found = base + __ffs(b) - 1;
      break;
    }
  }
  if (lane == 0) {
    if (first) slot->nfallback = 0u;
    if (found >= 0) {
      slot->query = queries + 3 * static_cast<size_t>(found);
      slot->k = k[found];
      slot->out_idx = oi + out_off[found];
      slot->out_dist = od + out_off[found];
      slot->out_count = oc + found;
      slot->cursor = found;
      slot->nfallback += 1u;
    } else {
      slot->k = 0;
      slot->cursor = Q;
    }
    cudaGraphSetConditional(h, found >= 0 ? 1u : 0u);
  }
}


}  // namespace

ScanConfig scan_config_for(int k) {
  if (k <= kSmallCap - kTile)
    return {kSmallWarps, kSmallCap, kSmallCap - kTile, Smem<kSmallWarps, kSmallCap>::total};
  return {kLargeWarps, kLargeCap, kLargeCap - kTile, Smem<kLargeWarps, kLargeCap>::total};
}

size_t scan_cand_capacity(int num_sms) {
  size_t a = static_cast<size_t>(num_sms) * kSmallWarps * (kSmallCap - kTile);
  size_t b = static_cast<size_t>(num_sms) * kLargeWarps * (kLargeCap - kTile);
  return a > b ? a : b;
}

cudaError_t scan_state_init(ScanState* st, cudaStream_t s) {
  scan_state_init_kernel<<<1, 192, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t scan_indirect_prepare() { return configure_cfg<kLargeWarps, kLargeCap>(); }

cudaError_t launch_scan_indirect(const DevLib& lib, const ScanSlot* slot, ScanState* st, unsigned long long* cand,
                                 uint32_t* err, int num_sms, double timeout_s, cudaStream_t s) {
  // the k of a slot is only known on the device: the configuration that serves every k
  uint64_t tns = static_cast<uint64_t>((timeout_s > 0 ? timeout_s : 2.0) * 1e9);
  return launch_cfg<kLargeWarps, kLargeCap>(lib, nullptr, 0, st, cand, nullptr, nullptr, nullptr, err, num_sms, tns,
                                            false, s, slot);
}

cudaError_t launch_fallback_pick(const uint64_t* queries, const int32_t* k, const int64_t* out_off, int32_t* oi,
                                 int32_t* od, int32_t* oc, int Q, ScanSlot* slot, bool first,
                                 cudaGraphConditionalHandle h, cudaStream_t s) {
  fallback_pick_kernel<<<1, 32, 0, s>>>(queries, k, out_off, oi, od, oc, Q, slot, first ? 1 : 0, h);
  return cudaGetLastError();
}

bool scan_small_fits(const DevLib& lib, int k, int num_sms) {
  return lib.n > 0 && k >= 1 && k <= kSmMaxK && num_sms >= 1 && num_sms <= kScanSmallMaxBlocks &&
         lib.n_tiles * kTile <= static_cast<int64_t>(kSmPer) * num_sms * kSmThreads;
}

// The small-library scan has no waits (every load is a plain load), so it takes no deadline.
cudaError_t launch_scan_small(const DevLib& lib, const uint64_t* q, int k, ScanState* st, unsigned long long* cand,
                              int32_t* oi, int32_t* od, int32_t* oc, uint32_t* err, int num_sms, bool programmatic,
                              cudaStream_t s) {
  static std::atomic<uint64_t> configured{0};
  cudaError_t ce = smem_attr_once(scan_small_kernel, kSmSmem, &configured);
  if (ce != cudaSuccess) return ce;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(num_sms));
  cfg.blockDim = dim3(kSmThreads);
  cfg.dynamicSmemBytes = kSmSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = programmatic ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, scan_small_kernel, lib, q, k, st, cand, oi, od, oc, err);
}

cudaError_t launch_scan_single(const DevLib& lib, const uint64_t* d_query, int k, ScanState* st,
                               unsigned long long* cand, int32_t* out_idx, int32_t* out_dist, int32_t* out_count,
                               uint32_t* err, int num_sms, double timeout_s, cudaStream_t s, bool programmatic) {
  if (scan_small_fits(lib, k, num_sms))
    return launch_scan_small(lib, d_query, k, st, cand, out_idx, out_dist, out_count, err, num_sms, programmatic, s);
  uint64_t tns = static_cast<uint64_t>((timeout_s > 0 ? timeout_s : 2.0) * 1e9);
  if (k <= kSmallCap - kTile)
    return launch_cfg<kSmallWarps, kSmallCap>(lib, d_query, k, st, cand, out_idx, out_dist, out_count, err, num_sms,
                                              tns, programmatic, s);
  return launch_cfg<kLargeWarps, kLargeCap>(lib, d_query, k, st, cand, out_idx, out_dist, out_count, err, num_sms,
                                            tns, programmatic, s);
}

}  // namespace fps

// ===========================================================================
// Single-query search that allocates nothing.
//
// Some callers cannot allocate device memory when they search: code whose
// device memory is entirely owned by another allocator (a framework pool that
// must account for every byte), code with a hard latency budget where a
// cudaMalloc and its implicit synchronisation are not acceptable, and code
// that searches on many short-lived streams, each of which would make
// fps_search_packed allocate a new per-stream workspace.  For them the scan's
// scratch (scan state, error word, candidate keys) lives in one file-scope
// device array of fixed size, kNoAllocBytes, which every GPU that loads this
// library holds until the process exits.
// ===========================================================================
namespace fps {
namespace {

constexpr int kNoAllocMaxSms = 160;                      // largest grid the array can serve
constexpr int kNoAllocKMax = kSmallCap - kTile;          // 128: the shared-buffer configuration
static_assert(kNoAllocKMax == FPS_NOALLOC_K_MAX, "the enforced k limit is the one the header states");
constexpr size_t kNoAllocStateBytes = (sizeof(ScanState) + 255) / 256 * 256;
constexpr size_t kNoAllocErrBytes = 256;
constexpr size_t kNoAllocCandKeys = static_cast<size_t>(kNoAllocMaxSms) * kSmallWarps * kNoAllocKMax;
constexpr size_t kNoAllocBytes = kNoAllocStateBytes + kNoAllocErrBytes + kNoAllocCandKeys * 8;  // ~2.6 MB
constexpr int kNoAllocMaxDevices = 64;

}  // namespace
}  // namespace fps

static __device__ __align__(256) unsigned char g_noalloc_scratch[fps::kNoAllocBytes];

namespace fps {
namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per
// device (host code cannot use the symbol itself as a device pointer).
cudaError_t noalloc_scratch(int device, unsigned char** out) {
  if (device < 0 || device >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[device] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_addr[device]);
  return cudaSuccess;
}

// Every call starts from a clean scan state and a cleared error word: the
// array keeps whatever the previous call (possibly a failed one) left there.
__global__ void noalloc_prepare_kernel(ScanState* st, uint32_t* err) {
  for (int b = threadIdx.x; b < 168; b += blockDim.x) st->hist[b] = 0u;
  for (int c = threadIdx.x; c < kQueues; c += blockDim.x) st->queue[32 * c] = 0u;
  if (threadIdx.x == 0) {
    st->thr_key = ~0ull;
    st->thr_d = 166u;
    st->done = 0u;
    st->ncand = 0u;
    *err = 0u;
  }
}

// Bound on each device-side wait: 2 s, or FPS_NOALLOC_TIMEOUT_NS when that is set to a
// positive integer (read on every call, so a test can make one call's waits run out).
uint64_t noalloc_timeout_ns() {
  const char* v = std::getenv("FPS_NOALLOC_TIMEOUT_NS");
  if (v && *v) {
    char* end = nullptr;
    const unsigned long long t = std::strtoull(v, &end, 10);
    if (end && *end == '\0' && t > 0) return t;
  }
  return 2000000000ull;
}

// A device-side failure (a bounded wait that ran out) is reported to the caller
// as *out_count = -1, since the error word itself is not the caller's memory.
__global__ void noalloc_finish_kernel(const uint32_t* err, int32_t* out_count) {
  if (threadIdx.x == 0 && *err != 0u) *out_count = -1;
}

}  // namespace
}  // namespace fps

extern "C" fps_status fps_search_noalloc(fps_library lib, const uint64_t* query, int k, int32_t* out_index,
                                         int32_t* out_dist, int32_t* out_count, void* cuda_stream) {
  using namespace fps;
  if (!lib || !query || !out_count || k < 0 || (k > 0 && (!out_index || !out_dist))) return FPS_ERR_INVALID_ARG;
  if (k > kNoAllocKMax) return FPS_ERR_UNSUPPORTED;
  Library* L = reinterpret_cast<Library*>(lib);
  if (L->num_sms > kNoAllocMaxSms) return FPS_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(L->device) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  fps_status status = FPS_OK;
  unsigned char* base = nullptr;
  if (noalloc_scratch(L->device, &base) != cudaSuccess) {
    status = FPS_ERR_CUDA;
  } else if (L->n == 0 || k == 0) {
    // count 0; with no records every slot up to k holds -1 (all bytes 0xFF), as on every path
    if (cudaMemsetAsync(out_count, 0, sizeof(int32_t), s) != cudaSuccess ||
        (k > 0 && (cudaMemsetAsync(out_index, 0xFF, sizeof(int32_t) * k, s) != cudaSuccess ||
                   cudaMemsetAsync(out_dist, 0xFF, sizeof(int32_t) * k, s) != cudaSuccess)))
      status = FPS_ERR_CUDA;
  } else {
    ScanState* st = reinterpret_cast<ScanState*>(base);
    uint32_t* err = reinterpret_cast<uint32_t*>(base + kNoAllocStateBytes);
    auto* cand = reinterpret_cast<unsigned long long*>(base + kNoAllocStateBytes + kNoAllocErrBytes);
    noalloc_prepare_kernel<<<1, 192, 0, s>>>(st, err);
    if (cudaGetLastError() != cudaSuccess ||
        launch_cfg<kSmallWarps, kSmallCap>(L->dev, query, k, st, cand, out_index, out_dist, out_count, err,
                                           L->num_sms, noalloc_timeout_ns(), false, s) != cudaSuccess) {
      status = FPS_ERR_CUDA;
    } else {
      noalloc_finish_kernel<<<1, 32, 0, s>>>(err, out_count);
      if (cudaGetLastError() != cudaSuccess) status = FPS_ERR_CUDA;
    }
  }
  if (status != FPS_OK) cudaGetLastError();
  cudaSetDevice(prev);
  return status;
}
