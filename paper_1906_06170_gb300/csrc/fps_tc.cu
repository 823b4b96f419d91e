// Batched scan on the 5th-generation tensor cores (tcgen05, TMEM).
//
// Paper: Sec. 4.3 -- Manhattan distance over 166 binary keys.  For 0/1 vectors
//   d(q, x) = sum_j |q_j - x_j| = popc(q) + popc(x) - 2 (q . x),
// so a batch of queries against the library is one dense contraction
// Q x K x N (K = 166 keys, padded to 192) followed by a per-element compare.
// Every product is 0 or 1 and every partial sum an integer <= 166, so any
// accumulator that holds the integers up to 166 exactly gives the exact q . x,
// and the distances equal the popcount path's.  Two operand formats:
//   FP8  kind::f8f6f4, E4M3 bytes (0x38 = 1.0), FP16 accumulators (every
//        integer up to 2048 is exact in FP16); tiles of 256 records;
//   FP4  kind::mxf4 (block-scaled), packed E2M1 nibbles (0x2 = 1.0, two keys
//        per byte), FP32 accumulators; every UE8M0 scale factor is 127
//        (2^0 = 1), so each product is still 0 or 1; tiles of 128 records,
//        so that three accumulators (TMEM columns 0, 128, 256) and the scale
//        factors fit the 512 columns.  Half the operand bytes of FP8 per key.
// (sm_103a has no tcgen05 kind::i8, so there is no INT8 variant.)
//
// CTA (one per SM, 14 warps):
//   warp 0  producer: 1-D bulk copies (cp.async.bulk) of the query tile A
//           (128 rows, double-buffered per work item) and of library tiles B
//           into a ring of stages, completing on mbarriers;
//   warps 1, 13  MMA issuers (warp 1 also allocates 512 TMEM columns): one
//           thread of each issues the MMAs of alternate library tiles (K = 192
//           in slices of 32 (FP8) or 64 (FP4) keys) into the tile's accumulator
//           (two for FP8, three for FP4, in turn) and commits to the stage-free
//           and accumulator-full barriers;
//   warps 2..9 epilogue: thread = query (TMEM lane), two warps per lane
//           quarter, each taking half of the tile's columns.  The test needs
//           one number per (query, group of columns), because a group lies
//           inside one popcount bucket:
//             d <= thr  <=>  acc >= ceil((popc q + popc x - thr) / 2),
//           taken as a max over the groups' bit patterns (non-negative FP16
//           and FP32 values order like unsigned integers).  FP8: the FP16
//           values are read (tcgen05.ld, pack::16b) with one wait and the
//           accumulator goes back to the MMA before the compare.  FP4: the
//           TMEM loads return the group maximum itself (tcgen05.ld.red), and
//           only a passing group is read as values, before the release (the
//           MMA meanwhile fills the other two accumulators).  A lane whose
//           group passes hands it (as FP16), with the bar, to a shared ring;
//   warps 10, 11 flushers, taking alternate 32-slot blocks of the ring: each
//           finishes the compare of up to 32 ring entries per round (one lane
//           per entry, 64 columns), takes each entry's candidate slots with one
//           returning atomic (all in flight together), then the warp appends
//           the round's accepted (distance, position) records to their queries'
//           candidate regions, 32 at a time, and counts them in the queries'
//           histograms (the shared batched state of fps_batch.cu); every 4
//           accepted records of a query it asks for the bound to be re-derived;
//   warp 12 refresher: re-derives a query's bound (smallest D with at least k
//           accepted records at distance <= D) with a warp-wide prefix sum over
//           its histogram and publishes it globally (atomicMin) and to the
//           epilogue through a per-row shared word.
// Operand layout (both operands, K-major, no swizzle): 8-row x 16-byte core
// matrices of 128 contiguous bytes; along K they follow each other (leading
// byte offset 128), along rows every 8-row group spans all K chunks (stride
// byte offset 128 x chunks).  The library operand is written in exactly this
// layout at load time, so a plain bulk copy lands a tile ready for the MMA.
// Work: items (query tile, chunk of library tiles) in chunk-major order, dealt
// round-robin, so the query tiles of a chunk run at the same time and the
// chunk is read from HBM once and from L2 by the rest.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "fps_internal.h"

namespace fps {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kTcQ = 128;                    // queries per CTA (M)
constexpr int kLbo = 128;                    // bytes between 16-byte K chunks
constexpr int kEpiWarps = 8;                 // two per TMEM lane quarter
constexpr int kFlushWarps = 2;               // drain the hand-off ring, alternate 32-slot blocks
constexpr int kFlushWarp0 = 2 + kEpiWarps;   // first flusher
constexpr int kRefWarp = kFlushWarp0 + kFlushWarps;   // re-derives query bounds from the histograms
constexpr int kMma2Warp = kRefWarp + 1;      // second MMA issuer (odd tiles; warp 1 takes the even ones)
constexpr int kThreads = 32 * (kMma2Warp + 1);
constexpr uint32_t kRefCap = 32;             // pending bound refreshes per flusher
constexpr uint32_t kRingCap = 192;           // epilogue hand-offs in flight per CTA
static_assert(kRingCap % (32 * kFlushWarps) == 0, "ring blocks alternate between the flushers");
constexpr uint32_t kTmemCols = 512;

// Operand formats.  kRows = records per library tile (the MMA's N), kKBytes =
// operand bytes per row (192 keys), kMmaK = keys per MMA, kBStages = library
// ring stages, kBParts = bulk copies per library tile.
struct Fp8 {
  static constexpr int kRows = 256;
  static constexpr int kKBytes = 192;
  static constexpr int kMmaK = 32;
  static constexpr int kBStages = 3;
  static constexpr int kBParts = 1;
  static constexpr bool kFp4 = false;
  static constexpr int kAccs = 2;                // accumulators in TMEM
  static constexpr uint32_t kAccStride = 256;   // TMEM columns between the two accumulators
};
struct Fp4 {
  static constexpr int kRows = 128;
  static constexpr int kKBytes = 96;
  static constexpr int kMmaK = 64;
  static constexpr int kBStages = 8;
  static constexpr int kBParts = 1;
  static constexpr bool kFp4 = true;
  static constexpr int kAccs = 3;               // three accumulators, at columns 0, 128 and 256
  static constexpr uint32_t kAccStride = 128;
  static constexpr uint32_t kSfaCol = 384;      // scale factors beside them (every byte 127: scale 1)
  static constexpr uint32_t kSfbCol = 448;
  static constexpr int kSfCols = 64;
};

template <class F>
struct Geom {
  static constexpr int kChunks = F::kKBytes / 16;           // 16-byte K chunks per row
  static constexpr int kSbo = kLbo * kChunks;               // bytes between 8-row groups
  static constexpr int kBTileBytes = F::kRows * F::kKBytes;
  static constexpr int kATileBytes = kTcQ * F::kKBytes;
  static constexpr int kMmas = 192 / F::kMmaK;              // MMAs per library tile
  static constexpr int kSliceBytes = F::kMmaK * F::kKBytes / 192;   // operand bytes of one K slice per row
  static_assert(kSliceBytes == 32, "each K slice spans two core matrices along K");
  static_assert((kBTileBytes / F::kBParts) % 16 == 0, "bulk copies move multiples of 16 bytes");
};

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
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
// Bounded wait: gives up timeout_ns after it started (no unbounded spins).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t deadline = global_ns() + timeout_ns;
  while (!mbar_try_wait(bar, parity))
    if (global_ns() > deadline) return false;
  return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// Same, with an L2 cache policy (createpolicy) for the copied lines.
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Hand-off words in shared memory: a release store publishes the writer's earlier
// stores, an acquire load orders the reader's later loads after it (no full fence).
__device__ __forceinline__ uint32_t ld_acquire_smem(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_smem(uint32_t* p, uint32_t v) {
  asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}

// Shared-memory matrix descriptor: K-major, no swizzle (layout type 0).
template <class F>
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>((kLbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((Geom<F>::kSbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;  // descriptor version for tcgen05
  return d;
}

// Instruction descriptors.
// kind::f8f6f4: dense, A = B = E4M3 (format 0 at bits 7 and 10), D = F16 (format 0 at
// bits 4-5; every sum is an integer <= 166, exact in FP16), both K-major, N >> 3 at
// bit 17, M >> 4 at bit 24.
// kind::mxf4 (block-scaled): dense, scale-factor ids 0 (bits 4-5, 29-30), A = B = E2M1
// (MXF4 format 1 at bits 7 and 10), both K-major, N >> 3 at bit 17, scale type UE8M0
// (bit 23), M >> 4 at bit 24, K = 64 per MMA (bit 31 clear); D is FP32.
template <class F>
__device__ __forceinline__ uint32_t instr_desc() {
  uint32_t d = 0;
  if constexpr (F::kFp4) {
    d |= 1u << 7;
    d |= 1u << 10;
    d |= 1u << 23;
  }
  d |= static_cast<uint32_t>(F::kRows >> 3) << 17;
  d |= static_cast<uint32_t>(kTcQ >> 4) << 24;
  return d;
}

template <class F>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc,
                                    uint32_t sfa, uint32_t sfb) {
  if constexpr (F::kFp4) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%5], [%6], p;\n}\n" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc), "r"(sfa), "r"(sfb)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

// 64 consecutive 16-bit TMEM columns of this thread's lane, two per register
// (pack::16b); valid only after tmem_wait_ld().
__device__ __forceinline__ void tmem_ld64h_nowait(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.pack::16b.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
}

// 32 consecutive 32-bit TMEM columns of this thread's lane (FP32 accumulators);
// valid only after tmem_wait_ld().
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
}

// Largest of 64 consecutive 32-bit TMEM columns of this thread's lane, taken by the TMEM
// loads themselves (tcgen05.ld.red: max over the loaded columns as unsigned integers;
// non-negative FP32 values order like their bit patterns).  Four loads of 16 columns; the
// loaded values are not needed, so all four write the same 16 scratch registers.  Valid
// only after tmem_wait_ld().
__device__ __forceinline__ uint32_t tmem_max64_nowait(uint32_t a) {
#define FPS_T16 "{t0, t1, t2, t3, t4, t5, t6, t7, t8, t9, t10, t11, t12, t13, t14, t15}"
  uint32_t m0, m1, m2, m3;
  asm volatile(
      "{\n .reg .b32 t<16>;\n"
      " tcgen05.ld.red.sync.aligned.32x32b.x16.max.u32 " FPS_T16 ", %0, [%4];\n"
      " tcgen05.ld.red.sync.aligned.32x32b.x16.max.u32 " FPS_T16 ", %1, [%5];\n"
      " tcgen05.ld.red.sync.aligned.32x32b.x16.max.u32 " FPS_T16 ", %2, [%6];\n"
      " tcgen05.ld.red.sync.aligned.32x32b.x16.max.u32 " FPS_T16 ", %3, [%7];\n}\n"
      : "=r"(m0), "=r"(m1), "=r"(m2), "=r"(m3)
      : "r"(a), "r"(a + 16), "r"(a + 32), "r"(a + 48)
      : "memory");
#undef FPS_T16
  return max(max(m0, m1), max(m2, m3));
}

// 32 consecutive TMEM columns of this thread's lane := w.
__device__ __forceinline__ void tmem_st32_fill(uint32_t taddr, uint32_t w) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
      "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
      "r"(w)
      : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void red_add_u32(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Byte offset of (row, key byte) inside a K-major no-swizzle operand tile.
template <class F>
__host__ __device__ __forceinline__ uint32_t op_offset(int row, int kb) {
  return static_cast<uint32_t>((row >> 3) * Geom<F>::kSbo + (kb >> 4) * kLbo + (row & 7) * 16 + (kb & 15));
}

// 16 FP8 operand bytes of one record: keys 16c .. 16c+15 as 0 / one (0x38).
__device__ __forceinline__ uint4 operand_chunk8(uint64_t w0, uint64_t w1, uint64_t w2, int c) {
  uint32_t out[4];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    uint32_t v = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int j = 16 * c + 4 * b + e;
      uint64_t w = j < 64 ? w0 : (j < 128 ? w1 : w2);
      uint32_t bit = (j < kBits) ? static_cast<uint32_t>((w >> (j & 63)) & 1ull) : 0u;
      v |= (bit ? 0x38u : 0u) << (8 * e);
    }
    out[b] = v;
  }
  return make_uint4(out[0], out[1], out[2], out[3]);
}

// 16 FP4 operand bytes of one record: keys 32c .. 32c+31, two per byte (key 32c + 2j in
// the low nibble of byte j, key 32c + 2j + 1 in its high nibble), E2M1 0 or one (0x2).
// Keys past 165 are zero bits of the packed record.
__device__ __forceinline__ uint4 operand_chunk4(uint64_t w0, uint64_t w1, uint64_t w2, int c) {
  const uint64_t w = c < 2 ? w0 : (c < 4 ? w1 : w2);
  const uint32_t bits = static_cast<uint32_t>(w >> (32 * (c & 1)));
  uint32_t out[4];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    uint32_t v = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) v |= ((bits >> (8 * b + e)) & 1u) << (4 * e + 1);
    out[b] = v;
  }
  return make_uint4(out[0], out[1], out[2], out[3]);
}

template <class F>
__device__ __forceinline__ uint4 operand_chunk(uint64_t w0, uint64_t w1, uint64_t w2, int c) {
  if constexpr (F::kFp4)
    return operand_chunk4(w0, w1, w2, c);
  else
    return operand_chunk8(w0, w1, w2, c);
}

// ------------------------------------------------------------- operand build
// Library operand: tensor tile T holds layout positions T * kRows .. + kRows - 1;
// positions past the layout (the last FP4 tile) are zero rows.
template <class F>
__global__ void tc_pack_library_kernel(DevLib lib, uint8_t* op, int64_t n_tc) {
  constexpr int kC = Geom<F>::kChunks;
  const int64_t n_pos = lib.n_tiles * kTile;
  const int64_t total = n_tc * F::kRows * kC;
  for (int64_t u = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; u < total;
       u += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t T = u / (F::kRows * kC);
    const int rem = static_cast<int>(u % (F::kRows * kC));
    const int g = rem / (8 * kC), rr = (rem % (8 * kC)) % 8, c = (rem % (8 * kC)) / 8;
    const int row = 8 * g + rr;
    const int64_t pos = T * F::kRows + row;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (pos < n_pos) {
      const uint64_t* w = lib.words + (pos / kTile) * (kWords * kTile) + (pos % kTile);
      v = operand_chunk<F>(w[0], w[kTile], w[2 * kTile], c);
    }
    *reinterpret_cast<uint4*>(op + T * Geom<F>::kBTileBytes + op_offset<F>(row, 16 * c)) = v;
  }
}

// Query operand: Q rounded up to 128-row tiles, rows past Q are zero.
template <class F>
__global__ void tc_pack_queries_kernel(const uint64_t* q, int Q, uint8_t* op, int q_tiles) {
  constexpr int kC = Geom<F>::kChunks;
  const int total = q_tiles * kTcQ * kC;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < total; u += gridDim.x * blockDim.x) {
    const int t = u / (kTcQ * kC), rem = u % (kTcQ * kC);
    const int g = rem / (8 * kC), rr = (rem % (8 * kC)) % 8, c = (rem % (8 * kC)) / 8;
    const int row = 8 * g + rr, qi = t * kTcQ + row;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (qi < Q) v = operand_chunk<F>(q[3 * qi], q[3 * qi + 1], q[3 * qi + 2], c);
    *reinterpret_cast<uint4*>(op + static_cast<size_t>(t) * Geom<F>::kATileBytes + op_offset<F>(row, 16 * c)) = v;
  }
}

// ------------------------------------------------------------------- scan
// One epilogue lane's group of up to 64 accumulators (a query against up to 64
// records) that passed the group-level test, as FP16, with what the flusher needs to
// finish the compare:
//   m0 = need (FP16 bit pattern) | valid columns << 16,
//   m1 = popc q + popc x | item sequence << 9,  pos0 = layout position of column 0,
//   coff, cap = the query's candidate region (first key, keys);
// seq = ring slot + 1 once written.
struct RingEntry {
  uint4 v[8];
  uint32_t q, m0, m1, pos0;
  uint32_t seq, cap;
  unsigned long long coff;
};
static_assert(sizeof(RingEntry) == 160, "ring entry layout");

template <class F>
struct TcSmem {
  uint8_t a[2][Geom<F>::kATileBytes];
  uint8_t b[F::kBStages][Geom<F>::kBTileBytes];
  uint64_t b_full[F::kBStages], b_empty[F::kBStages];
  uint64_t a_full[2], a_empty[2];
  uint64_t acc_full[F::kAccs], acc_empty[F::kAccs];
  // (A parity wait cannot tell a phase from the one two before it.  Every epilogue warp
  // takes every tile in order, so it waits for each accumulator's phases in order.  An MMA
  // issuer takes every other tile: it reaches tile t only after the release of tile
  // t - 2 - kAccs that its previous tile needed, which the in-order epilogue gives no
  // earlier than that of tile t - 2 kAccs, the phase before the one tile t waits for.  So
  // no wait ever runs two phases ahead.)
  uint64_t fin[2];                 // per MMA issuer: all of its MMAs complete
  uint32_t tmem_base;
  int bpos[kNumBuckets + 1];       // first layout position of each bucket
  int bend[kNumBuckets + 1];       // one past its last record
  RingEntry ring[kRingCap];
  // per query row: (item sequence << 32) | ~bound -- a 64-bit max keeps the newest
  // item and, within it, the smallest bound
  unsigned long long thr_w[kTcQ];
  uint32_t pend[kTcQ];             // accepted records per row (refresh every 4)
  uint2 ref_q[kFlushWarps][kRefCap];   // refresh requests (query, item sequence), one queue per flusher
  uint32_t r_tail;                 // ring slots claimed by the epilogue
  uint32_t f_head[kFlushWarps];    // next slot each flusher retires; slots below the minimum are free
  uint32_t epi_done;               // epilogue warps finished
  uint32_t ref_tail[kFlushWarps];  // refresh requests posted (per flusher)
  uint32_t ref_head[kFlushWarps];  // refresh requests done (refresher)
  uint32_t flush_done;             // flushers finished
};
static_assert(sizeof(TcSmem<Fp8>) + 1024 <= 232448, "shared memory per CTA");
static_assert(sizeof(TcSmem<Fp4>) + 1024 <= 232448, "shared memory per CTA");

// Every ring slot below this one is retired.  A flusher never passes a slot that
// is claimed and unwritten, so the minimum of the heads is at most any such slot.
template <class S>
__device__ __forceinline__ uint32_t ring_retired(const S& sm) {
  uint32_t m = ld_acquire_smem(&sm.f_head[0]);
#pragma unroll
  for (int f = 1; f < kFlushWarps; ++f) m = min(m, ld_acquire_smem(&sm.f_head[f]));
  return m;
}

// Epilogue side: claim a ring slot, wait (bounded) for room, write the entry
// (fill(e) writes its 64 FP16 values).
template <class S, class Fill>
__device__ __forceinline__ bool ring_push(S& sm, Fill&& fill, uint32_t q, uint32_t m0, uint32_t m1, uint32_t pos0,
                                          unsigned long long coff, uint32_t cap, uint64_t timeout_ns) {
  const uint32_t slot = atomicAdd(&sm.r_tail, 1u);
  if (slot - ring_retired(sm) >= kRingCap) {
    // the ring is full: wait without taking issue slots from the flushers
    const uint64_t deadline = global_ns() + timeout_ns;
    while (slot - ring_retired(sm) >= kRingCap) {
      if (global_ns() > deadline) return false;
      __nanosleep(64);
    }
  }
  RingEntry& e = sm.ring[slot % kRingCap];
  fill(e);
  *reinterpret_cast<uint4*>(&e.q) = make_uint4(q, m0, m1, pos0);
  e.cap = cap;
  e.coff = coff;
  st_release_smem(&e.seq, slot + 1);
  return true;
}

// Position of the (r+1)-th set bit of m (r < popc(m)).
__device__ __forceinline__ int nth_set_bit(uint32_t m, uint32_t r) {
  int pos = 0;
#pragma unroll
  for (int sh = 16; sh > 0; sh >>= 1) {
    const uint32_t low = static_cast<uint32_t>(__popc(m & ((1u << sh) - 1u)));
    if (r >= low) {
      r -= low;
      m >>= sh;
      pos += sh;
    }
  }
  return pos;
}

// Bucket of layout position p: the last bucket starting at or before p (empty
// buckets start where the next one does).
__device__ __forceinline__ int bucket_at(const int* bpos, int64_t p) {
  int lo = 0, hi = kNumBuckets - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (bpos[mid] <= p)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// FP32 accumulators of a group that passed, as FP16 pairs (column 2i low, 2i + 1 high);
// every value is an integer <= 166, exact in FP16.
__device__ __forceinline__ uint32_t half2_bits(uint32_t lo, uint32_t hi) {
  const __half2 h = __floats2half2_rn(__uint_as_float(lo), __uint_as_float(hi));
  return *reinterpret_cast<const uint32_t*>(&h);
}

// FP16 and FP32 bit patterns of an integer 1 <= n < 1024 (both exact), with integer
// arithmetic only: the exponent is the position of the top bit.
__device__ __forceinline__ uint32_t f16_bits_of(int n) {
  const int e = 31 - __clz(n);
  return (static_cast<uint32_t>(e + 15) << 10) | ((static_cast<uint32_t>(n) << (10 - e)) & 0x3FFu);
}
__device__ __forceinline__ uint32_t f32_bits_of(int n) {
  const int e = 31 - __clz(n);
  return (static_cast<uint32_t>(e + 127) << 23) | ((static_cast<uint32_t>(n) << (23 - e)) & 0x7FFFFFu);
}

// Largest of the 64 non-negative FP16 values held as 32 pairs: four independent
// max chains, then one fold (bit patterns of non-negative FP16 order like integers).
__device__ __forceinline__ uint32_t max64_half(const uint32_t (&w)[32]) {
  uint32_t m0 = __vimax3_u16x2(w[0], w[1], w[2]), m1 = __vimax3_u16x2(w[3], w[4], w[5]);
  uint32_t m2 = __vimax3_u16x2(w[6], w[7], w[8]), m3 = __vimax3_u16x2(w[9], w[10], w[11]);
#pragma unroll
  for (int e = 12; e < 28; e += 8) {
    m0 = __vimax3_u16x2(m0, w[e], w[e + 1]);
    m1 = __vimax3_u16x2(m1, w[e + 2], w[e + 3]);
    m2 = __vimax3_u16x2(m2, w[e + 4], w[e + 5]);
    m3 = __vimax3_u16x2(m3, w[e + 6], w[e + 7]);
  }
  m0 = __vimax3_u16x2(m0, w[28], w[29]);
  m1 = __vimax3_u16x2(m1, w[30], w[31]);
  const uint32_t m = __vimax3_u16x2(m0, m1, __vmaxu2(m2, m3));
  return max(m & 0xFFFFu, m >> 16);
}

template <class F>
__global__ void __launch_bounds__(kThreads, 1)
    tc_scan_kernel(DevLib lib, BatchDev b, const uint8_t* __restrict__ lib_op, const uint8_t* __restrict__ q_op,
                   int64_t n_tc, int n_qt, int chunk, uint64_t timeout_ns) {
  using G = Geom<F>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  TcSmem<F>& S = *reinterpret_cast<TcSmem<F>*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n_chunks = (n_tc + chunk - 1) / chunk;
  const int64_t n_items = n_chunks * n_qt;

  for (int i = threadIdx.x; i < kNumBuckets + 1; i += blockDim.x) {
    S.bpos[i] = lib.tile_off[i] * kTile;
    S.bend[i] = i < kNumBuckets ? lib.tile_off[i] * kTile + lib.bcount[i] : S.bpos[i];
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < F::kBStages; ++s) {
      mbar_init(&S.b_full[s], 1);
      mbar_init(&S.b_empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&S.a_full[i], 1);
      mbar_init(&S.a_empty[i], 2);   // both MMA issuers are done with the query tile
    }
    for (int i = 0; i < F::kAccs; ++i) {
      mbar_init(&S.acc_full[i], 1);
      mbar_init(&S.acc_empty[i], kEpiWarps);
    }
    mbar_init(&S.fin[0], 1);
    mbar_init(&S.fin[1], 1);
    S.r_tail = 0;
    for (int f = 0; f < kFlushWarps; ++f) {
      S.f_head[f] = 32u * f;
      S.ref_tail[f] = 0;
      S.ref_head[f] = 0;
    }
    S.epi_done = 0;
    S.flush_done = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (uint32_t i = threadIdx.x; i < kRingCap; i += blockDim.x) S.ring[i].seq = 0;
  for (int i = threadIdx.x; i < kTcQ; i += blockDim.x) {
    S.thr_w[i] = 0ull;
    S.pend[i] = 0u;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&S.tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;
  if constexpr (F::kFp4) {
    // unit scale factors: every byte of both scale-factor regions is 127 (2^0) in every lane
    if (warp >= 2 && warp < 6) {
      const uint32_t lane_base = tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16);
#pragma unroll
      for (int c = 0; c < F::kSfCols; c += 32) {
        tmem_st32_fill(lane_base + F::kSfaCol + c, 0x7F7F7F7Fu);
        tmem_st32_fill(lane_base + F::kSfbCol + c, 0x7F7F7F7Fu);
      }
      tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  const uint64_t deadline = timeout_ns;   // per wait
  const uint64_t drain = timeout_ns > kDrainNs ? timeout_ns : kDrainNs;   // own copies / MMAs in flight
  bool ok = true;

  if (warp == 0) {
    // ------------------------------------------------------------- producer
    if (lane == 0) {
      // library tiles are read by every query tile of their chunk: keep them in L2 (evict last)
      uint64_t pol_b;
      asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol_b));
      uint32_t bn = 0;  // library tiles issued so far
      uint32_t na = 0;  // query tiles issued so far
      for (int64_t j = 0; ok; ++j) {
        const int64_t item = blockIdx.x + j * gridDim.x;
        if (item >= n_items) break;
        const int qt = static_cast<int>(item % n_qt);
        const int64_t c = item / n_qt;
        const int ab = static_cast<int>(j & 1);
        if (!mbar_wait(&S.a_empty[ab], static_cast<uint32_t>(((j >> 1) & 1) ^ 1), deadline)) {
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(&S.a_full[ab], G::kATileBytes);
        bulk_g2s(S.a[ab], q_op + static_cast<size_t>(qt) * G::kATileBytes, G::kATileBytes, &S.a_full[ab]);
        ++na;
        const int64_t t0 = c * chunk, t1 = min(t0 + chunk, n_tc);
        for (int64_t T = t0; T < t1; ++T, ++bn) {
          const int s = static_cast<int>(bn % F::kBStages);
          const uint32_t use = bn / F::kBStages;
          if (!mbar_wait(&S.b_empty[s], (use & 1) ^ 1, deadline)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&S.b_full[s], G::kBTileBytes);
          const uint8_t* src = lib_op + T * G::kBTileBytes;
          constexpr int kPart = G::kBTileBytes / F::kBParts;
#pragma unroll
          for (int part = 0; part < F::kBParts; ++part)
            bulk_g2s_hint(S.b[s] + part * kPart, src + part * kPart, kPart, &S.b_full[s], pol_b);
        }
      }
      // wait (bounded) for copies still in flight before anyone leaves
      for (int s = 0; s < F::kBStages; ++s) {
        if (bn > static_cast<uint32_t>(s)) {
          uint32_t last_use = (bn - 1 - s) / F::kBStages;
          mbar_wait(&S.b_full[s], last_use & 1, drain);
        }
      }
      for (int a = 0; a < 2; ++a) {
        if (na > static_cast<uint32_t>(a)) {
          uint32_t last_use = (na - 1 - a) / 2;
          mbar_wait(&S.a_full[a], last_use & 1, drain);
        }
      }
      if (!ok) atomicOr(b.err, DEVERR_TIMEOUT);
    }
  } else if (warp == 1 || warp == kMma2Warp) {
    // ------------------------------------------------------------ MMA issue
    // Two issuing threads, one per accumulator: warp 1 takes the even tiles of the
    // CTA's sequence, warp kMma2Warp the odd ones.  Issuing a tcgen05.mma costs a
    // single thread tens of cycles, as does each barrier wait, so one thread alone
    // cannot keep the tensor pipe busy; with two, the MMAs of consecutive tiles are
    // issued in parallel and run back to back.
    const uint32_t mine = warp == 1 ? 0u : 1u;
    if (lane == 0) {
      const uint32_t idesc = instr_desc<F>();
      uint32_t sfa = 0, sfb = 0;
      if constexpr (F::kFp4) {
        sfa = tmem + F::kSfaCol;
        sfb = tmem + F::kSfbCol;
      }
      uint32_t bn = 0, tn = 0;  // library tiles consumed, accumulators produced
      for (int64_t j = 0; ok; ++j) {
        const int64_t item = blockIdx.x + j * gridDim.x;
        if (item >= n_items) break;
        const int64_t c = item / n_qt;
        const int ab = static_cast<int>(j & 1);
        if (!mbar_wait(&S.a_full[ab], static_cast<uint32_t>((j >> 1) & 1), deadline)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_base = smem_addr(S.a[ab]);
        const int64_t t0 = c * chunk, t1 = min(t0 + chunk, n_tc);
        for (int64_t T = t0; T < t1; ++T, ++bn, ++tn) {
          if ((tn & 1u) != mine) continue;
          const int s = static_cast<int>(bn % F::kBStages);
          const int acc = static_cast<int>(tn % F::kAccs);
          if (!mbar_wait(&S.acc_empty[acc], ((tn / F::kAccs) & 1) ^ 1, deadline) ||
              !mbar_wait(&S.b_full[s], (bn / F::kBStages) & 1, deadline)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t b_base = smem_addr(S.b[s]);
          const uint32_t d_tmem = tmem + static_cast<uint32_t>(acc) * F::kAccStride;
#pragma unroll
          for (int ks = 0; ks < G::kMmas; ++ks)
            mma<F>(d_tmem, smem_desc<F>(a_base + 256 * ks), smem_desc<F>(b_base + 256 * ks), idesc,
                   ks > 0 ? 1u : 0u, sfa, sfb);
          mma_commit(&S.b_empty[s]);
          mma_commit(&S.acc_full[acc]);
        }
        if (!ok) break;
        mma_commit(&S.a_empty[ab]);
      }
      if (!ok) atomicOr(b.err, DEVERR_TIMEOUT);
      // all MMAs issued by this thread complete before the final barrier
      mma_commit(&S.fin[mine]);
      mbar_wait(&S.fin[mine], 0, drain);
    }
  } else if (warp < kFlushWarp0) {
    // -------------------------------------------------------------- epilogue
    const int ew = warp - 2;
    const int quarter = warp & 3;                 // TMEM lanes 32*quarter .. +31
    const int half = ew >> 2;                     // which half of the tile's columns
    const int row = 32 * quarter + lane;          // query row inside the tile
    const uint32_t lane_addr = static_cast<uint32_t>(32 * quarter) << 16;
    uint32_t tn = 0;
    int bk = 0;                                   // bucket cursor (positions ascend within an item)
    for (int64_t j = 0; ok; ++j) {
      const int64_t item = blockIdx.x + j * gridDim.x;
      if (item >= n_items) break;
      const int qt = static_cast<int>(item % n_qt);
      const int64_t c = item / n_qt;
      const int q = qt * kTcQ + row;
      const bool live = q < b.Q && b.k[q] > 0;
      int pq = 0;
      uint32_t thr = 0;
      int64_t co = 0;      // the query's candidate region: first key, keys
      uint32_t ccap = 0;
      if (live) {
        pq = __popcll(b.queries[3 * q]) + __popcll(b.queries[3 * q + 1]) + __popcll(b.queries[3 * q + 2]);
        thr = ld_relaxed_u32(b.thr + q);
        co = b.cand_off[q];
        ccap = static_cast<uint32_t>(b.cand_off[q + 1] - co);
        atomicMax(&S.thr_w[row], (static_cast<unsigned long long>(j) << 32) | (0xFFFFFFFFu - thr));
      }
      // tile indices and layout positions fit 32 bits (positions index the int32 perm)
      const int t0 = static_cast<int>(c * chunk), t1 = static_cast<int>(min(c * chunk + chunk, n_tc));
      bk = bucket_at(S.bpos, static_cast<int64_t>(t0) * F::kRows);
      int nxt = bk + 1 < kNumBuckets ? S.bpos[bk + 1] : 0x7FFFFFFF;   // where the next bucket starts
      // the cursor moves only when a position reaches the next bucket (rarely: a few
      // hundred boundaries in the whole library)
      auto advance = [&](int p) {
        while (p >= nxt) {
          ++bk;
          nxt = bk + 1 < kNumBuckets ? S.bpos[bk + 1] : 0x7FFFFFFF;
        }
      };
      // other CTAs' refreshes of this query reach the row through the global bound,
      // re-read every 16 tiles (loaded 8 tiles before it is used); the refresher's
      // per-row word is read every 4 tiles
      uint32_t gthr = thr;
      for (int T = t0; T < t1; ++T, ++tn) {
        const int acc = static_cast<int>(tn % F::kAccs);
        const uint32_t acc_par = (tn / F::kAccs) & 1;
        if (live && ((T - t0) & 3) == 0) {   // the refresher may have tightened this row's bound
          const unsigned long long w = *reinterpret_cast<volatile unsigned long long*>(&S.thr_w[row]);
          if ((w >> 32) == static_cast<unsigned long long>(j)) {
            const uint32_t t = 0xFFFFFFFFu - static_cast<uint32_t>(w);
            thr = t < thr ? t : thr;
          }
          if (((T - t0) & 15) == 8) thr = gthr < thr ? gthr : thr;
          if (((T - t0) & 15) == 0) gthr = ld_relaxed_u32(b.thr + q);
        }
        const int tpos = T * F::kRows;            // layout position of the tile's column 0
        // a group of columns passes when acc >= ceil((pq + px - thr) / 2) for one of its
        // records: the largest accumulator against the bar of the group's bucket px
        auto bar_of = [&](int px, uint32_t& need16) {
          const int need = (pq + px - static_cast<int>(thr) + 1) >> 1;   // <= 166
          need16 = need <= 0 ? 0u : f16_bits_of(need);
          return need <= 0 ? 0u : f32_bits_of(need);
        };
        auto push = [&](auto&& fill, uint32_t need16, int px, int p0, int ncols) {
          int lim = S.bend[px] - p0;
          lim = lim < ncols ? lim : ncols;
          if (lim <= 0) return;
          if (!ring_push(S, fill, static_cast<uint32_t>(q), need16 | (static_cast<uint32_t>(lim) << 16),
                         static_cast<uint32_t>(pq + px) | (static_cast<uint32_t>(j) << 9), static_cast<uint32_t>(p0),
                         static_cast<unsigned long long>(co), ccap, deadline))
            ok = false;
        };
        if constexpr (!F::kFp4) {
          // FP8: a 256-record tile lies inside one bucket; this warp reads columns
          // 128 half .. +127 as two groups of 64 FP16 values (pack::16b)
          advance(tpos);
          const bool act = live && static_cast<uint32_t>(abs(bk - pq)) <= thr;
          const bool landed = mbar_wait(&S.acc_full[acc], acc_par, deadline);
          if (!__all_sync(kFull, landed)) {   // one verdict for the whole warp
            ok = false;
            break;
          }
          tc_fence_after();
          uint32_t v[2][32];
          if (__any_sync(kFull, act)) {
            const uint32_t col0 = static_cast<uint32_t>(acc) * F::kAccStride + static_cast<uint32_t>(half * 128);
            tmem_ld64h_nowait(tmem + lane_addr + col0, v[0]);
            tmem_ld64h_nowait(tmem + lane_addr + col0 + 64, v[1]);
            tmem_wait_ld();
          }
          // the values are in registers: hand the accumulator back to the MMA before comparing
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&S.acc_empty[acc]);
          if (act) {
            uint32_t need16;
            bar_of(bk, need16);
#pragma unroll
            for (int g = 0; g < 2; ++g) {
              // rare: some of these 64 records may be within the bound; the flusher
              // finishes the compare column by column
              if (max64_half(v[g]) >= need16) {
                auto fill = [&](RingEntry& e) {
#pragma unroll
                  for (int i = 0; i < 8; ++i)
                    e.v[i] = make_uint4(v[g][4 * i], v[g][4 * i + 1], v[g][4 * i + 2], v[g][4 * i + 3]);
                };
                push(fill, need16, bk, tpos + half * 128 + g * 64, 64);
              }
            }
          }
        } else {
          // FP4: a 128-record tile lies inside one bucket (buckets start at multiples of 256
          // records); this warp takes columns 64 half .. +63 as one group.  The group's maximum
          // comes from the TMEM loads themselves (tcgen05.ld.red); a group that passes (rare) is
          // read again as values and goes to the ring before the accumulator is released --
          // with three accumulators the MMA runs on while one warp hands off.
          advance(tpos);
          const bool act = live && static_cast<uint32_t>(abs(bk - pq)) <= thr;
          const bool landed = mbar_wait(&S.acc_full[acc], acc_par, deadline);
          if (!__all_sync(kFull, landed)) {   // one verdict for the whole warp
            ok = false;
            break;
          }
          tc_fence_after();
          if (__any_sync(kFull, act)) {
            uint32_t need16 = 0, need = 0;
            if (act) need = bar_of(bk, need16);
            const uint32_t base = tmem + lane_addr + static_cast<uint32_t>(acc) * F::kAccStride + 64u * half;
            const uint32_t m = tmem_max64_nowait(base);
            tmem_wait_ld();
            const bool pass = act && m >= need;
            if (__any_sync(kFull, pass)) {
              uint32_t h[32];   // FP16 pairs (column 2i low, 2i + 1 high), read 32 columns at a time
              {
                uint32_t v[32];
                tmem_ld32_nowait(base, v);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; ++i) h[i] = half2_bits(v[2 * i], v[2 * i + 1]);
              }
              {
                uint32_t v[32];
                tmem_ld32_nowait(base + 32, v);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; ++i) h[16 + i] = half2_bits(v[2 * i], v[2 * i + 1]);
              }
              if (pass) {
                auto fill = [&](RingEntry& e) {
#pragma unroll
                  for (int i = 0; i < 8; ++i) e.v[i] = make_uint4(h[4 * i], h[4 * i + 1], h[4 * i + 2], h[4 * i + 3]);
                };
                push(fill, need16, bk, tpos + 64 * half, 64);
              }
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&S.acc_empty[acc]);
        }
      }
      if (!ok) break;
    }
    if (!ok && lane == 0) atomicOr(b.err, DEVERR_TIMEOUT);
    __syncwarp();
    if (lane == 0) atomicAdd(&S.epi_done, 1u);
  } else if (warp < kRefWarp) {
    // --------------------------------------------------------------- flushers
    // Flusher f takes the ring's 32-slot blocks f, f + kFlushWarps, ...  Up to 32
    // ring entries per round, one lane per entry: the exact compare of the
    // entry's 64 columns and one returning atomic for its candidate slots, all
    // entries' atomics in flight together; then the round's accepted records are
    // written by the whole warp, 32 at a time (candidate, histogram count), and
    // a bound refresh is requested every 4 accepted records of a query.
    const int fw = warp - kFlushWarp0;
    uint32_t head = 32u * static_cast<uint32_t>(fw), rtail = 0;
    uint64_t idle_since = 0;
    // The ring entries of a round are released before the round's slot
    // reservations return: each lane keeps at most one accepted record of the
    // previous round (p_*), written once the owner entry's reservation (e_*)
    // is in, at the start of the next round or when the warp goes idle.
    bool pv = false;
    int p_own = 0;
    uint32_t p_r = 0, p_d = 0, p_pos = 0;
    uint32_t e_base = 0, e_cap = 0;
    long long e_coff = 0;
    auto write_pending = [&]() {
      const uint32_t obase = __shfl_sync(kFull, e_base, p_own);
      const uint32_t ocap = __shfl_sync(kFull, e_cap, p_own);
      const long long ocoff = __shfl_sync(kFull, e_coff, p_own);
      if (pv && obase + p_r < ocap) b.cand[ocoff + obase + p_r] = (static_cast<unsigned long long>(p_d) << 32) | p_pos;
      pv = false;
    };
    for (;;) {
      const uint32_t idx = head + static_cast<uint32_t>(lane);
      const bool ready = idx < ((head & ~31u) + 32u) &&   // within this flusher's current block
                         ld_acquire_smem(&S.ring[idx % kRingCap].seq) == idx + 1;
      const uint32_t bal = __ballot_sync(kFull, ready);
      const int n = bal == kFull ? 32 : __ffs(~bal) - 1;   // ready entries in a row from head
      if (n == 0) {
        write_pending();
        const bool epi_over = *reinterpret_cast<volatile uint32_t*>(&S.epi_done) == kEpiWarps;
        // every claimed slot of this flusher's blocks is below head
        if (epi_over && *reinterpret_cast<volatile uint32_t*>(&S.r_tail) <= head) break;
        // idle: wait for the epilogue (itself bounded); claimed-but-unwritten slots after
        // it finished get timeout_ns, and no idle spell may exceed 32 x timeout_ns
        const uint64_t now = global_ns();
        if (idle_since == 0) idle_since = now;
        if (now - idle_since > (epi_over ? timeout_ns : 32 * timeout_ns)) {
          if (lane == 0) atomicOr(b.err, DEVERR_TIMEOUT);
          break;
        }
        __nanosleep(128);
        continue;
      }
      idle_since = 0;
      const bool mine = lane < n;
      const RingEntry& e = S.ring[idx % kRingCap];
      uint32_t eq = 0, m0 = 0, m1 = 0, pos0 = 0, ecap = 0;
      unsigned long long ecoff = 0;
      uint32_t hlo = 0, hhi = 0;   // bit c of (hhi:hlo): column c passes
      if (mine) {
        const uint4 mt = *reinterpret_cast<const uint4*>(&e.q);
        eq = mt.x;
        m0 = mt.y;
        m1 = mt.z;
        pos0 = mt.w;
        ecap = e.cap;
        ecoff = e.coff;
        const uint32_t need16 = m0 & 0xFFFFu, need2 = need16 | (need16 << 16);
        // halves are below 0x8000: (w | 0x80008000) - need2 borrows across neither half and
        // leaves bit 15 (31) set exactly where the low (high) half is >= need
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const uint4 a4 = e.v[i];
          const uint32_t ww[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int r = 4 * i + u;   // word r holds columns 2r (low half) and 2r + 1 (high half)
            const uint32_t t = ((ww[u] | 0x80008000u) - need2) & 0x80008000u;
            const uint32_t two = ((t >> 15) & 1u) | ((t >> 30) & 2u);
            if (r < 16)
              hlo |= two << (2 * r);
            else
              hhi |= two << (2 * (r - 16));
          }
        }
        const int lim = static_cast<int>(m0 >> 16);   // valid columns, 1..64
        if (lim <= 32) {
          hhi = 0;
          if (lim < 32) hlo &= (1u << lim) - 1u;
        } else if (lim < 64) {
          hhi &= (1u << (lim - 32)) - 1u;
        }
      }
      const uint32_t cnt = static_cast<uint32_t>(__popc(hlo) + __popc(hhi));
      write_pending();   // the previous round's reservations are needed before they are replaced
      bool req = false;
      if (cnt > 0) {
        e_base = atomicAdd(b.cnt + eq, cnt);
        const uint32_t old = atomicAdd(&S.pend[eq % kTcQ], cnt);
        req = (old >> 2) != ((old + cnt) >> 2);
        e_coff = static_cast<long long>(ecoff);
        e_cap = ecap;
      }
      // this entry's first record among the round's accepted records
      uint32_t incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t off = incl - cnt;
      const uint32_t total = __shfl_sync(kFull, incl, 31);
      const bool defer = total <= 32;   // one record per lane: written next round
      __syncwarp();   // every lane may read every entry of the round (each owner acquired its own)
      for (uint32_t h0 = 0; h0 < total; h0 += 32) {
        const uint32_t h = h0 + static_cast<uint32_t>(lane);
        // owner: the last entry whose first record is <= h (it has records when h < total)
        int own = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const uint32_t o2 = __shfl_sync(kFull, off, own + step);
          if (o2 <= h) own += step;
        }
        const uint32_t r = h - __shfl_sync(kFull, off, own);
        const uint32_t olo = __shfl_sync(kFull, hlo, own), ohi = __shfl_sync(kFull, hhi, own);
        const uint32_t oq = __shfl_sync(kFull, eq, own), om1 = __shfl_sync(kFull, m1, own);
        const uint32_t opos = __shfl_sync(kFull, pos0, own);
        uint32_t d = 0, pos = 0;
        if (h < total) {
          const uint32_t nlo = static_cast<uint32_t>(__popc(olo));
          const int col = r < nlo ? nth_set_bit(olo, r) : 32 + nth_set_bit(ohi, r - nlo);
          const uint16_t* vals = reinterpret_cast<const uint16_t*>(S.ring[(head + own) % kRingCap].v);
          const int a = static_cast<int>(__half2float(__ushort_as_half(vals[col])));
          d = static_cast<uint32_t>(static_cast<int>(om1 & 0x1FFu) - 2 * a);
          pos = opos + static_cast<uint32_t>(col);
          red_add_u32(b.hist + static_cast<size_t>(oq) * 168 + d, 1u);
        }
        if (defer) {
          pv = h < total;
          p_own = own;
          p_r = r;
          p_d = d;
          p_pos = pos;
        } else {   // more records than lanes: wait for the reservations now
          const uint32_t obase = __shfl_sync(kFull, e_base, own);
          const uint32_t ocap = __shfl_sync(kFull, e_cap, own);
          const long long ocoff = __shfl_sync(kFull, e_coff, own);
          if (h < total && obase + r < ocap) b.cand[ocoff + obase + r] = (static_cast<unsigned long long>(d) << 32) | pos;
        }
      }
      __syncwarp();
      head += static_cast<uint32_t>(n);
      if ((head & 31u) == 0) head += 32u * (kFlushWarps - 1);   // over the other flushers' blocks
      if (lane == 0) st_release_smem(&S.f_head[fw], head);
      // post refresh requests while there is room (a dropped request only delays a bound)
      const uint32_t rb = __ballot_sync(kFull, req);
      if (rb) {
        uint32_t rh = 0;
        if (lane == 0) rh = *reinterpret_cast<volatile uint32_t*>(&S.ref_head[fw]);
        const uint32_t room = kRefCap - (rtail - __shfl_sync(kFull, rh, 0));   // one view for the warp
        const uint32_t rank = __popc(rb & ((1u << lane) - 1u));
        if (req && rank < room) S.ref_q[fw][(rtail + rank) % kRefCap] = make_uint2(eq, m1 >> 9);
        const uint32_t posted = min(static_cast<uint32_t>(__popc(rb)), room);
        __syncwarp();
        rtail += posted;
        if (lane == 0) st_release_smem(&S.ref_tail[fw], rtail);
      }
    }
    write_pending();
    __syncwarp();
    if (lane == 0) atomicAdd(&S.flush_done, 1u);
  } else if (warp == kRefWarp) {
    // -------------------------------------------------------------- refresher
    // bound = smallest D <= thr with at least k accepted records at distance <= D,
    // from the query's histogram (any subset of its counts gives a valid bound)
    // (one request from each flusher's queue in turn; two scalar queue heads, which an
    // array indexed by the queue number would have put in local memory)
    static_assert(kFlushWarps == 2, "the refresher polls two request queues");
    uint32_t rh0 = 0, rh1 = 0;
    uint64_t idle_since = 0;
    int f = 0;
    for (;;) {
      const uint32_t t0v = ld_acquire_smem(&S.ref_tail[0]), t1v = ld_acquire_smem(&S.ref_tail[1]);
      int src;
      if (f == 0)
        src = t0v != rh0 ? 0 : (t1v != rh1 ? 1 : -1);
      else
        src = t1v != rh1 ? 1 : (t0v != rh0 ? 0 : -1);
      if (src < 0) {
        const bool fl_over = *reinterpret_cast<volatile uint32_t*>(&S.flush_done) == kFlushWarps;
        if (fl_over && t0v == rh0 && t1v == rh1) break;
        const uint64_t now = global_ns();
        if (idle_since == 0) idle_since = now;
        if (now - idle_since > 64 * timeout_ns) {
          if (lane == 0) atomicOr(b.err, DEVERR_TIMEOUT);
          break;
        }
        __nanosleep(512);
        continue;
      }
      f = src ^ 1;
      idle_since = 0;
      const uint32_t head_src = src == 0 ? rh0 : rh1;
      const uint2 r = S.ref_q[src][head_src % kRefCap];
      const uint32_t rq = r.x, rj = r.y;
      const uint32_t kq = static_cast<uint32_t>(b.k[rq]);
      const uint32_t tcur = ld_relaxed_u32(b.thr + rq);
      const uint32_t* hist = b.hist + static_cast<size_t>(rq) * 168;
      uint32_t carry = 0, D = 167u;
      for (uint32_t base = 0; base <= tcur && base < 168u; base += 32) {
        const uint32_t e = base + lane;
        uint32_t x = (e <= tcur && e < 168u) ? __ldcg(hist + e) : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(kFull, x, o);
          if (lane >= o) x += y;
        }
        const uint32_t hit = __ballot_sync(kFull, e <= tcur && carry + x >= kq);
        if (hit) {
          D = base + static_cast<uint32_t>(__ffs(hit) - 1);
          break;
        }
        carry += __shfl_sync(kFull, x, 31);
      }
      if (lane == 0 && D < tcur) {
        atomicMin(b.thr + rq, D);
        atomicMax(&S.thr_w[rq % kTcQ], (static_cast<unsigned long long>(rj) << 32) | (0xFFFFFFFFu - D));
      }
      __syncwarp();
      if (src == 0)
        ++rh0;
      else
        ++rh1;
      if (lane == 0) *reinterpret_cast<volatile uint32_t*>(&S.ref_head[src]) = head_src + 1;
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}


template <class F>
int64_t tensor_tiles(int64_t n_tiles128) {
  return (n_tiles128 * kTile + F::kRows - 1) / F::kRows;
}

template <class F>
cudaError_t launch_tc(const DevLib& lib, const BatchDev& b, const uint8_t* lib_op, const uint8_t* q_op, int n_qt,
                      int num_sms, int chunk, double timeout_s, cudaStream_t s) {
  const int64_t n_tc = tensor_tiles<F>(lib.n_tiles);
  if (n_tc == 0 || n_qt == 0) return cudaSuccess;
  const size_t smem = sizeof(TcSmem<F>) + 1024;
  static std::atomic<uint64_t> configured{0};
  cudaError_t e = smem_attr_once(tc_scan_kernel<F>, smem, &configured);
  if (e != cudaSuccess) return e;
  const uint64_t tns = static_cast<uint64_t>((timeout_s > 0 ? timeout_s : 2.0) * 1e9);
  tc_scan_kernel<F><<<num_sms, kThreads, smem, s>>>(lib, b, lib_op, q_op, n_tc, n_qt, chunk, tns);
  return cudaGetLastError();
}

template <class F>
cudaError_t pack_library(const DevLib& lib, uint8_t* op, cudaStream_t s) {
  const int64_t n_tc = tensor_tiles<F>(lib.n_tiles);
  if (n_tc == 0) return cudaSuccess;
  tc_pack_library_kernel<F><<<4096, 256, 0, s>>>(lib, op, n_tc);
  return cudaGetLastError();
}

template <class F>
cudaError_t pack_queries(const uint64_t* q, int Q, uint8_t* op, cudaStream_t s) {
  const int q_tiles = (Q + kTcQ - 1) / kTcQ;
  if (q_tiles == 0) return cudaSuccess;
  const int total = q_tiles * kTcQ * Geom<F>::kChunks;
  tc_pack_queries_kernel<F><<<(total + 255) / 256, 256, 0, s>>>(q, Q, op, q_tiles);
  return cudaGetLastError();
}

}  // namespace

int64_t tc_tiles(int fmt, int64_t n_tiles128) {
  return fmt == kTcFp4 ? tensor_tiles<Fp4>(n_tiles128) : tensor_tiles<Fp8>(n_tiles128);
}

int tc_tile_rows(int fmt) { return fmt == kTcFp4 ? Fp4::kRows : Fp8::kRows; }

size_t tc_operand_bytes(int fmt, int64_t n_tiles128) {
  return fmt == kTcFp4 ? static_cast<size_t>(tensor_tiles<Fp4>(n_tiles128)) * Geom<Fp4>::kBTileBytes
                       : static_cast<size_t>(tensor_tiles<Fp8>(n_tiles128)) * Geom<Fp8>::kBTileBytes;
}

size_t tc_query_operand_bytes(int fmt, int Q) {
  const size_t tiles = static_cast<size_t>((Q + kTcQ - 1) / kTcQ);
  return tiles * (fmt == kTcFp4 ? Geom<Fp4>::kATileBytes : Geom<Fp8>::kATileBytes);
}

cudaError_t tc_pack_library(int fmt, const DevLib& lib, uint8_t* op, cudaStream_t s) {
  return fmt == kTcFp4 ? pack_library<Fp4>(lib, op, s) : pack_library<Fp8>(lib, op, s);
}

cudaError_t tc_pack_queries(int fmt, const uint64_t* q, int Q, uint8_t* op, cudaStream_t s) {
  return fmt == kTcFp4 ? pack_queries<Fp4>(q, Q, op, s) : pack_queries<Fp8>(q, Q, op, s);
}

cudaError_t tc_scan(int fmt, const DevLib& lib, const BatchDev& b, const uint8_t* lib_op, const uint8_t* q_op,
                    int num_sms, int chunk, double timeout_s, cudaStream_t s) {
  const int n_qt = (b.Q + kTcQ - 1) / kTcQ;
  if (chunk <= 0) chunk = tc_default_chunk(fmt);
  return fmt == kTcFp4 ? launch_tc<Fp4>(lib, b, lib_op, q_op, n_qt, num_sms, chunk, timeout_s, s)
                       : launch_tc<Fp8>(lib, b, lib_op, q_op, n_qt, num_sms, chunk, timeout_s, s);
}

// Library tiles per work item: 64 x 256 records (FP8), 128 x 128 records (FP4) -- about
// 16 K records, so that the query tiles of a chunk reuse it from L2.
int tc_default_chunk(int fmt) { return fmt == kTcFp4 ? 128 : 64; }

}  // namespace fps
