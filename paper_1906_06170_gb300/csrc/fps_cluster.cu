// Batch clustering search: kernels that cluster a batch of queries.
//
// The paper's interface clusters a batch of query fingerprints, picks the
// number of clusters by the silhouette ("contour") coefficient and lists the
// top 30 library molecules per cluster (Sec. 4.4, results after Fig. 1); it
// names no algorithm.  The procedure computed here, identical step by step to
// the oracle's, is:
//   D[i][j]       Manhattan distance between queries i and j (Sec. 4.3);
//   seeding       first medoid = the query with the smallest row sum of D,
//                 then farthest-first (largest distance to the nearest chosen
//                 medoid; chosen medoids excluded);
//   k-medoids     assign every query to its nearest medoid (ties: the medoid
//                 chosen first); new medoid of a cluster = its member with the
//                 smallest sum of distances to the cluster; repeat until the
//                 medoids repeat (at most kClusterIters rounds);
//   silhouette    per query floor(s * 2^32) with s = (b - a) / max(a, b) formed
//                 from integer sums (a: mean distance inside its cluster, b:
//                 the smallest mean distance to another non-empty cluster; 0
//                 for a singleton or max(a, b) = 0); a clustering's score is
//                 the sum over queries.
// Every tie goes to the smaller query index.  All arithmetic is integer, so
// the chosen count and the medoids equal the oracle's exactly.  The rounds of
// all counts run together, each kernel covering every count still moving; the
// host (fps_host.cpp) checks once per round whether any count goes on, then
// searches the library with the chosen count's medoids.
#include <cuda_runtime.h>

#include <cstdint>

#include "fps_internal.h"

namespace fps {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__global__ void qdist_kernel(const uint64_t* __restrict__ q, int Q, int32_t* __restrict__ D) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Q || j >= Q) return;
  const uint64_t* a = q + 3 * static_cast<size_t>(i);
  const uint64_t* b = q + 3 * static_cast<size_t>(j);
  D[static_cast<size_t>(i) * Q + j] = __popcll(a[0] ^ b[0]) + __popcll(a[1] ^ b[1]) + __popcll(a[2] ^ b[2]);
}

// One warp per row: row sums, or (lab != nullptr) sums over the row's own cluster.
__global__ void rowsum_kernel(const int32_t* __restrict__ D, int Q, const int32_t* __restrict__ lab,
                              int32_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= Q) return;
  const int32_t* row = D + static_cast<size_t>(i) * Q;
  const int li = lab ? lab[i] : 0;
  int32_t s = 0;
  for (int j = lane; j < Q; j += 32)
    if (!lab || lab[j] == li) s += row[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
  if (lane == 0) out[i] = s;
}

// near[i] = min(near[i], D[i][*m]) (first = 1: near[i] = D[i][*m])
__global__ void near_kernel(const int32_t* __restrict__ D, int Q, const int32_t* __restrict__ m, int first,
                            int32_t* __restrict__ near) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Q) return;
  const int32_t d = D[static_cast<size_t>(i) * Q + *m];
  near[i] = first ? d : (d < near[i] ? d : near[i]);
}

// Single block: smallest (mode 0) or largest (mode 1) value over i with
// keep(i), ties to the smaller i.  keep: lab == nullptr -> every i not among
// the first n_ex medoids in `ex`; else lab[i] == want.  Result: *out (or -1).
__global__ void select_kernel(const int32_t* __restrict__ val, int Q, int mode, const int32_t* __restrict__ ex,
                              int n_ex, const int32_t* __restrict__ lab, int want, int32_t* __restrict__ out) {
  __shared__ unsigned long long best[32];
  // packed (value + 2^31 or 2^31 - value, index): the smaller packed wins, so the value decides and then
  // the smaller index; values are distances or distance sums, far below 2^31
  unsigned long long mine = ~0ull;
  for (int i = threadIdx.x; i < Q; i += blockDim.x) {
    bool keep;
    if (lab) {
      keep = lab[i] == want;
    } else {
      keep = true;
      for (int t = 0; t < n_ex; ++t) keep = keep && ex[t] != i;
    }
    if (!keep) continue;
    const long long v = mode == 0 ? static_cast<long long>(val[i]) : -static_cast<long long>(val[i]);
    const unsigned long long packed = (static_cast<unsigned long long>(v + (1ll << 31)) << 32) |
                                      static_cast<unsigned long long>(static_cast<uint32_t>(i));
    mine = packed < mine ? packed : mine;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(kFull, mine, o);
    mine = other < mine ? other : mine;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) best[warp] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long b = ~0ull;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) b = best[w] < b ? best[w] : b;
    *out = b == ~0ull ? -1 : static_cast<int32_t>(b & 0xFFFFFFFFull);
  }
}

// ------------------------------------------- k-medoids rounds for every count at once
// Slot s clusters into c_min + s groups.  Each round runs the assignment, the
// within-cluster row sums and the medoid update of every slot still active;
// a slot stops when its medoids repeat (its labels then belong to them) or
// after kClusterIters rounds (its labels are then re-derived from the last
// medoids), exactly as one count at a time would.

// lab[s][i] = the nearest medoid of slot s (ties: the one chosen first).  final_pass: only
// the slots that ran out of rounds.
__global__ void assign_multi_kernel(ClusterRounds r, int final_pass) {
  const int s = blockIdx.y;
  const int32_t* st = r.state + 4 * s;
  if (final_pass ? st[2] == 0 : st[0] == 0) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= r.Q) return;
  const int c = r.c_min + s;
  const int32_t* med = r.med + kClusterMaxC * s;
  const int32_t* row = r.D + static_cast<size_t>(i) * r.Q;
  int bt = 0;
  int32_t bd = row[med[0]];
  for (int t = 1; t < c; ++t) {
    const int32_t d = row[med[t]];
    if (d < bd) {
      bd = d;
      bt = t;
    }
  }
  r.lab[static_cast<size_t>(s) * r.Q + i] = bt;
}

// cost[s][i] = sum of D[i][j] over the members j of i's cluster in slot s (one warp per row)
__global__ void rowsum_multi_kernel(ClusterRounds r) {
  const int s = blockIdx.y;
  if (r.state[4 * s] == 0) return;
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= r.Q) return;
  const int32_t* row = r.D + static_cast<size_t>(i) * r.Q;
  const int32_t* lab = r.lab + static_cast<size_t>(s) * r.Q;
  const int li = lab[i];
  int32_t sum = 0;
  for (int j = lane; j < r.Q; j += 32)
    if (lab[j] == li) sum += row[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
  if (lane == 0) r.cost[static_cast<size_t>(s) * r.Q + i] = sum;
}

// One block per slot: every cluster's member with the smallest cost (ties: smaller index;
// an empty cluster keeps its medoid), then the slot's state for the next round.
// any_active[round] = 1 if some slot goes on.
__global__ void medoid_multi_kernel(ClusterRounds r, int round) {
  const int s = blockIdx.x;
  int32_t* st = r.state + 4 * s;
  if (st[0] == 0) return;
  const int c = r.c_min + s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t* lab = r.lab + static_cast<size_t>(s) * r.Q;
  const int32_t* cost = r.cost + static_cast<size_t>(s) * r.Q;
  int32_t* med = r.med + kClusterMaxC * s;
  __shared__ int32_t nm[kClusterMaxC];
  __shared__ int changed;
  if (threadIdx.x == 0) changed = 0;
  __syncthreads();
  for (int t = warp; t < c; t += blockDim.x >> 5) {
    long long mine = LLONG_MAX;
    for (int i = lane; i < r.Q; i += 32)
      if (lab[i] == t) {
        const long long packed = (static_cast<long long>(cost[i]) << 32) | static_cast<long long>(i);
        mine = packed < mine ? packed : mine;
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long other = __shfl_xor_sync(kFull, mine, o);
      mine = other < mine ? other : mine;
    }
    if (lane == 0) {
      const int32_t m = mine == LLONG_MAX ? med[t] : static_cast<int32_t>(mine & 0xFFFFFFFFll);
      nm[t] = m;
      if (m != med[t]) atomicExch(&changed, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!changed) {
      st[0] = 0;                          // the medoids repeat: the labels belong to them
    } else {
      for (int t = 0; t < c; ++t) med[t] = nm[t];
      if (++st[1] == kClusterIters) {
        st[0] = 0;                        // out of rounds: labels of the new medoids follow
        st[2] = 1;
      } else {
        r.any_active[round] = 1;
      }
    }
  }
}

__global__ void sizes_kernel(const int32_t* __restrict__ lab, int Q, int c, int32_t* __restrict__ sizes) {
  __shared__ int32_t sh[kClusterMaxC];
  for (int t = threadIdx.x; t < c; t += blockDim.x) sh[t] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < Q; i += blockDim.x) atomicAdd(&sh[lab[i]], 1);
  __syncthreads();
  for (int t = threadIdx.x; t < c; t += blockDim.x) sizes[t] = sh[t];
}

// One warp per query: per-cluster sums of its row, then floor(s * 2^32) added to *score.
// Each lane adds its elements into its own column of shared counters indexed by the
// element's cluster (one add per element, no bank conflicts), then the columns are summed.
constexpr int kSilWarps = 8;
__global__ void __launch_bounds__(32 * kSilWarps)
    silhouette_kernel(const int32_t* __restrict__ D, int Q, const int32_t* __restrict__ lab, int c,
                      const int32_t* __restrict__ sizes, unsigned long long* __restrict__ score) {
  __shared__ int32_t acc[kSilWarps][kClusterMaxC][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * kSilWarps + w;
  if (i >= Q) return;   // whole warps only: the block has no block-wide barrier
#pragma unroll
  for (int t = 0; t < kClusterMaxC; ++t) acc[w][t][lane] = 0;
  const int32_t* row = D + static_cast<size_t>(i) * Q;
  for (int j = lane; j < Q; j += 32) acc[w][lab[j]][lane] += row[j];
  __syncwarp();
  int32_t mine = 0;   // lane t: the sum over cluster t
  if (lane < kClusterMaxC)
    for (int l = 0; l < 32; ++l) mine += acc[w][lane][l];
  int32_t sums[kClusterMaxC];
#pragma unroll
  for (int t = 0; t < kClusterMaxC; ++t) sums[t] = __shfl_sync(kFull, mine, t);
  if (lane != 0) return;
  const int A = lab[i];
  long long s_fixed = 0;
  if (sizes[A] > 1) {
    const long long SA = sums[A], na = sizes[A] - 1;
    long long SB = -1, nb = 1;
    for (int t = 0; t < c; ++t) {
      if (t == A || sizes[t] == 0) continue;
      if (SB < 0 || static_cast<long long>(sums[t]) * nb < SB * sizes[t]) {
        SB = sums[t];
        nb = sizes[t];
      }
    }
    if (SB >= 0) {
      const long long N = SB * na - SA * nb;                  // (b - a) na nb
      const long long M = SA * nb > SB * na ? SA * nb : SB * na;   // max(a, b) na nb
      if (M > 0) {
        const __int128 num = static_cast<__int128>(N) << 32;
        __int128 qq = num / M;                               // truncates toward zero
        if ((num % M) != 0 && num < 0) qq -= 1;              // floor
        s_fixed = static_cast<long long>(qq);
      }
    }
  }
  atomicAdd(score, static_cast<unsigned long long>(s_fixed));   // two's complement sum
}

}  // namespace

cudaError_t cluster_qdist(const uint64_t* q, int Q, int32_t* D, cudaStream_t s) {
  dim3 grid((Q + 255) / 256, Q);
  qdist_kernel<<<grid, 256, 0, s>>>(q, Q, D);
  return cudaGetLastError();
}

cudaError_t cluster_rowsum(const int32_t* D, int Q, const int32_t* lab, int32_t* out, cudaStream_t s) {
  rowsum_kernel<<<(Q + 7) / 8, 256, 0, s>>>(D, Q, lab, out);
  return cudaGetLastError();
}

cudaError_t cluster_near(const int32_t* D, int Q, const int32_t* m, bool first, int32_t* near, cudaStream_t s) {
  near_kernel<<<(Q + 255) / 256, 256, 0, s>>>(D, Q, m, first ? 1 : 0, near);
  return cudaGetLastError();
}

cudaError_t cluster_select(const int32_t* val, int Q, bool largest, const int32_t* ex, int n_ex, const int32_t* lab,
                           int want, int32_t* out, cudaStream_t s) {
  select_kernel<<<1, 1024, 0, s>>>(val, Q, largest ? 1 : 0, ex, n_ex, lab, want, out);
  return cudaGetLastError();
}

cudaError_t cluster_round(const ClusterRounds& r, int round, cudaStream_t s) {
  if (r.n_slots <= 0) return cudaSuccess;
  assign_multi_kernel<<<dim3((r.Q + 255) / 256, r.n_slots), 256, 0, s>>>(r, 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  rowsum_multi_kernel<<<dim3((r.Q + 7) / 8, r.n_slots), 256, 0, s>>>(r);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  medoid_multi_kernel<<<r.n_slots, 512, 0, s>>>(r, round);
  return cudaGetLastError();
}

cudaError_t cluster_final_assign(const ClusterRounds& r, cudaStream_t s) {
  if (r.n_slots <= 0) return cudaSuccess;
  assign_multi_kernel<<<dim3((r.Q + 255) / 256, r.n_slots), 256, 0, s>>>(r, 1);
  return cudaGetLastError();
}

cudaError_t cluster_silhouette(const int32_t* D, int Q, const int32_t* lab, int c, int32_t* sizes,
                               unsigned long long* score, cudaStream_t s) {
  sizes_kernel<<<1, 1024, 0, s>>>(lab, Q, c, sizes);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  silhouette_kernel<<<(Q + kSilWarps - 1) / kSilWarps, 32 * kSilWarps, 0, s>>>(D, Q, lab, c, sizes, score);
  return cudaGetLastError();
}

}  // namespace fps
