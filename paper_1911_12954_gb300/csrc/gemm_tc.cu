// gemm_tc.cu - tcgen05 / TMEM / TMA GEMM for the block-spin contraction (FP16x3 and TF32x3).
//
// C[m][n] = alpha * sum_s sum_k (Ahi Bhi + Ahi Blo + Alo Bhi)[m,n,k] over the segments s of
// one output, with A = Ahi + Alo and B = Bhi + Blo: either fp16 planes (hi, lo of 2^14 x;
// kind::f16, the default) or tf32 values stored in FP32 words (kind::tf32), both operands
// K-major in K panels (see tma_load). One launch computes every output of a group (the pure
// tensor and the impure ones of a step, GemmGroup): an output with two segments, such as
// S' = (A_S B_T^T + A_T B_S^T) / 2, runs its k loop over both operand pairs into one
// accumulator, so no output is read back. This is the O(D^15) block-spin contraction of the HOTRG step,
// where Sec. 2 of arXiv:1911.12954 places the D^(4d-1) cost of the method, carried out on
// the 5th-generation tensor cores with FP32 accumulation; the dropped Alo Blo term is below
// 2^-21 of each product.
//
// The tensor cores add each MMA's products into the FP32 accumulator with truncation,
// so an accumulator that runs over the whole K picks up a bias that grows linearly with
// K (measured 2.5e-4 relative at K = 32768). The kernels therefore promote the partial
// sum of every chunk of k (32 for tf32; 128, or 64 / 256 in the other variants, for fp16)
// from TMEM into FP32 registers, where the sums are rounded to nearest: the truncation
// bias is bounded by one chunk's worth. Each promotion reads the whole 128 x 256 FP32
// accumulator out of TMEM and holds the MMAs back for a few hundred cycles, so the chunk
// is as long as the accuracy allows (at D = 8, 64-k chunks cost 17 % of the MMA time and
// 128-k chunks 7 %).
//
// Two kernels share the promotion and epilogue code:
//
// gemm_tf32x3_kernel (one CTA per 128 x 256 tile): persistent, one CTA per SM, 10 warps.
//   warp 0 lane 0 : TMA producer. Per k-block (one swizzle row of 64 bytes: 32 fp16 or 16
//                   tf32 values), four tiles (Ahi, Alo: 128 rows; Bhi, Blo: 256 rows) land
//                   in one pipeline stage through cp.async.bulk.tensor (3D, K panels).
//   warp 1 lane 0 : MMA issuer. Per k-block, k-steps x 3 products of
//                   tcgen05.mma.cta_group::1.kind::tf32 or kind::f16 (M=128, N=256) into one of
//                   two TMEM chunk accumulators (2 x 256 of the 512 columns); commits free
//                   the stage and hand the chunk to the epilogue.
//   warps 2..9    : promotion + epilogue. Warp w reads TMEM lane quarter w % 4 and column
//                   half (w - 2) / 4 with tcgen05.ld 32x32b, adds the chunk into 128 FP32
//                   registers per thread, and after the last k-block of the tile writes
//                   alpha * acc + beta * C with guarded stores.
//
// gemm_pair_kernel (fp16 only; one CTA pair per 256 x 256 tile): the same roles in a cluster
//   of two CTAs on two SMs. Each CTA copies its own 128 rows of A and its own half (128 rows)
//   of the B tile into its own shared memory with plain TMA loads whose completion is counted
//   on the even CTA's mbarrier (.cta_group::2); the even CTA's MMA thread issues
//   tcgen05.mma.cta_group::2 (M = 256, N = 256), which reads A and B from both CTAs and writes
//   each CTA's 128 accumulator rows into its own TMEM. Its commits are addressed one barrier
//   at a time (the CTA's own and, through mapa, the partner's), and every copy lands in the
//   shared memory of the CTA that issued it. Every B row is fetched by one SM of the pair, so
//   the pair reads half the B bytes of two single-CTA tiles. Its k-blocks are 64 fp16 wide
//   (one 128-byte swizzle row per operand row, the padded row pitch of the K panels), 3
//   stages of 64 KB per CTA: with 64-byte rows the pair read 4x the DRAM bytes of the
//   single-CTA kernel at D_cut = 8 (559 GB against 134 GB per launch), with 128-byte rows
//   the same 134 GB, and its GEMM ran in 89 ms against 106 ms for single CTAs.
//
// Tiles are visited in groups of 16 M-tiles so the CTAs running at the same time share
// A and B k-blocks through L2.
// Every mbarrier wait is bounded (globaltimer, 4 s): on expiry the thread raises the
// timeout status word and leaves its loop; teardown still drains the copies and MMAs in
// flight (bounded) and frees TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"

namespace hotrg {

namespace tc {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int TMEM_COLS = 2 * BN;                       // two chunk accumulators
constexpr int GROUP_M = 16;
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr unsigned long long kWaitNs = 4000000000ull;

// Pipeline variants. One k-block = one swizzle row of ROWB bytes (128 B or 64 B) per
// operand row; F16 selects fp16 operands (kind::f16, K = 16 per MMA) instead of tf32
// (kind::tf32, K = 8). Either way an MMA k-step spans 32 bytes of the row. CHUNK is the
// k promoted from TMEM to registers at once. PAIR: the two-CTA form (B_BYTES is then this
// CTA's half of the B tile, and the MMA spans M = 2 BM rows).
template <int ROWB, bool F16, int CHUNK, bool PAIR = false>
struct Cfg {
  static constexpr bool kF16 = F16;
  static constexpr bool kPair = PAIR;
  static constexpr int ELT = F16 ? 2 : 4;
  static constexpr int BK = ROWB / ELT;                            // elements per k-block
  static constexpr int KSTEPS = ROWB / 32;                         // MMAs per product per k-block
  static constexpr int STAGES = PAIR ? (ROWB == 128 ? 3 : 6) : (ROWB == 128 ? 2 : 4);
  static constexpr int A_BYTES = BM * ROWB;
  static constexpr int B_BYTES = (PAIR ? BN / 2 : BN) * ROWB;
  static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int KB_PER_CHUNK = CHUNK / BK;
  static_assert(CHUNK % BK == 0, "a chunk is a whole number of k-blocks");
  static constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
  static_assert(SMEM_BYTES <= 232448, "shared memory per CTA");
  static constexpr uint64_t LAYOUT = ROWB == 128 ? 2 : 4;         // UMMA swizzle: 128 B or 64 B
  static constexpr uint32_t SBO = 8 * ROWB;                       // 8 rows of one swizzle row
  static constexpr int MMA_M = PAIR ? 2 * BM : BM;
  // instruction descriptor: D = F32; A = B = TF32 (2) or F16 (0); both K-major; N = 256, M
  static constexpr uint32_t IDESC = (1u << 4) | ((F16 ? 0u : 2u) << 7) | ((F16 ? 0u : 2u) << 10) |
                                    ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(MMA_M >> 4) << 24);
};
using CfgTF32 = Cfg<64, false, 32>;     // default tf32 pipeline: 4 stages of 16-wide k-blocks
using CfgTF32W = Cfg<128, false, 32>;   // tf32, 2 stages of 32-wide k-blocks
using CfgF16 = Cfg<64, true, 128>;      // fp16: 4 stages of 32-wide k-blocks, 128-k chunks
using CfgF16S = Cfg<64, true, 64>;      // fp16 with 64-k chunks
using CfgF16L = Cfg<64, true, 256>;     // fp16 with 256-k chunks
using CfgF16P = Cfg<128, true, 128, true>;  // fp16, CTA pairs, 3 stages of 64 KB, 128-k chunks

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
// Arrival on an mbarrier of any CTA of the cluster (shared::cluster address from mapa).
// Relaxed: the arrival only reports that this warp's TMEM loads have completed (wait::ld),
// and a release at cluster scope would first wait for the thread's earlier global stores
// (the previous tile's C rows) to become visible, which stalled the epilogue and with it the
// MMAs (D_cut = 8 GEMM 151 ms against 103 ms relaxed).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t caddr) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr) : "memory");
}
template <bool CLUSTER>
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  if constexpr (CLUSTER) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
  }
  return ok != 0;
}
// Bounded wait; false (and the timeout status raised) when it gives up. CLUSTER: the
// arrivals may come from the partner CTA (acquire at cluster scope).
template <bool CLUSTER = false>
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* status,
                                          unsigned long long limit_ns = kWaitNs) {
  if (mbar_try<CLUSTER>(b, parity)) return true;
  const unsigned long long t0 = now_ns();
  while (true) {
    if (mbar_try<CLUSTER>(b, parity)) return true;
    if (now_ns() - t0 > limit_ns) {
      atomicAdd(&status[kStTimeout], 1);
      return false;
    }
  }
}

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing arrives at
// (no copies, no MMAs in flight), gives up after limit_ns and raises the status word.
__global__ void wait_selftest_kernel(int* status, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_wait(&bar, 0, status, limit_ns);
  }
}

// Operands are stored in K panels: element (row, k) with k = p Kp + kin of tensor w sits at
// [((w P + p) rows + row) kps + kin] (kps = Kp rounded up to 4). The 4D tensor map is
// {Kp, rows, P, W}; a panel keeps the rows of one k range contiguous, so a box of 128 rows
// spans at most a few pages even when K is in the hundreds of thousands.
__device__ __forceinline__ void tma_load(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y, int z,
                                         int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
      "[%2];" ::"r"(su32(dst)),
      "l"((uint64_t)map), "r"(su32(bar)), "r"(x), "r"(y), "r"(z), "r"(w)
      : "memory");
}
// The same load into this CTA's shared memory, with its bytes counted on an mbarrier of
// either CTA of the pair (bar: shared::cluster address).
__device__ __forceinline__ void tma_load_pair(const CUtensorMap* map, uint32_t bar, void* dst, int x, int y, int z,
                                              int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(su32(dst)),
      "l"((uint64_t)map), "r"(bar), "r"(x), "r"(y), "r"(z), "r"(w)
      : "memory");
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %cluster_ctarank;" : "=r"(r));
  return r;
}
// shared::cluster address of the variable at shared::cta address `a` in CTA `rank`
__device__ __forceinline__ uint32_t mapa(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

// K-major operand in the canonical swizzled layout TMA writes: rows of one swizzle width,
// 8-row groups SBO bytes apart.
template <class C>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(C::SBO >> 4) << 32;                // stride byte offset: 8 rows
  d |= (uint64_t)1 << 46;                            // descriptor version (tcgen05)
  d |= C::LAYOUT << 61;                              // swizzle mode
  return d;
}

template <class CF>
__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  if constexpr (CF::kPair) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(CF::IDESC), "r"(accumulate)
        : "memory");
  } else if constexpr (CF::kF16) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(CF::IDESC), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(CF::IDESC), "r"(accumulate)
        : "memory");
  }
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
// Arrives on one mbarrier (shared::cluster address: this CTA's or the partner's) once the
// pair MMAs issued so far by this thread have completed.
__device__ __forceinline__ void mma_commit_pair(uint32_t caddr) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(caddr)
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int group, int& tm, int& tn) {
  const int per_group = group * tiles_n;
  const int g = t / per_group;
  const int first_m = g * group;
  const int gm = min(group, tiles_m - first_m);
  const int r = t - g * per_group;
  tm = first_m + r % gm;
  tn = r / gm;
}

// Adds one chunk accumulator (this warp's 32 TMEM lanes, its half of the 256 columns) into
// the thread's 128 FP32 registers.
__device__ __forceinline__ void promote_chunk(uint32_t taddr, float* acc) {
#pragma unroll
  for (int c = 0; c < BN / 64; ++c) {
    float v[32];
    tmem_ld32(taddr + (uint32_t)(c * 32), v);
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[c * 32 + j] += v[j];
  }
}

// Output factor of problem pb: its alpha, times 2^-(eA + eB) for operands scaled by their
// max-norm exponents.
__device__ __forceinline__ float out_alpha(const GemmGroup& g, int pb) {
  if (!g.amax_a) return g.p[pb].alpha;
  const int e = pb / g.per_elem;
  return ldexpf(g.p[pb].alpha, -(split_exponent(g.amax_a[e], kF16Top) + split_exponent(g.amax_b[e], kF16Top)));
}

// alpha * acc for one thread's 128 columns of row m (guarded).
__device__ __forceinline__ void store_row(float* __restrict__ C, int64_t ldc, int M, int N, int64_t m, int n0,
                                          const float* acc, float alpha) {
  if (m >= M) return;
  float* crow = C + m * ldc + n0;
  if (n0 + BN / 2 <= N && ((((uintptr_t)crow) & 15) == 0)) {
#pragma unroll
    for (int j = 0; j < BN / 2; j += 4)
      *(float4*)(crow + j) = make_float4(alpha * acc[j], alpha * acc[j + 1], alpha * acc[j + 2], alpha * acc[j + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < BN / 2; ++j)
      if (n0 + j < N) crow[j] = alpha * acc[j];
  }
}

template <class CF>
__global__ void __launch_bounds__(THREADS, 1)
    gemm_tf32x3_kernel(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                       const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo,
                       const __grid_constant__ GemmGroup grp, int64_t ldc, int M, int N, int Kp, int P,
                       int* status) {
  constexpr int STAGES = CF::STAGES, BK = CF::BK, A_BYTES = CF::A_BYTES, B_BYTES = CF::B_BYTES,
                STAGE_BYTES = CF::STAGE_BYTES, KPC = CF::KB_PER_CHUNK;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* full = bars;                 // [STAGES]
  uint64_t* empty = bars + STAGES;       // [STAGES]
  uint64_t* cfull = bars + 2 * STAGES;   // [2] chunk accumulator written
  uint64_t* cempty = cfull + 2;          // [2] chunk accumulator drained
  uint64_t* drain = cempty + 2;          // [1]
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_m = (M + BM - 1) / BM, tiles_n = (N + BN - 1) / BN;
  const int ntiles1 = tiles_m * tiles_n;          // tiles of one output
  const int ntiles = grp.nprob * ntiles1;         // outputs one after the other
  const int nkbp = (Kp + BK - 1) / BK;   // k-blocks per panel (the last one zero-filled past Kp)
  const int nkb = P * nkbp;              // k-blocks of one segment

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&cfull[a], 1);
      mbar_init(&cempty[a], 32 * EPI_WARPS);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ TMA producer
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mAhi) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mAlo) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mBhi) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mBlo) : "memory");
    int s = 0;
    uint32_t ph = 0;
    int nissued = 0;   // k-blocks issued; stage q has been filled (nissued - q + STAGES - 1) / STAGES times
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int pb = t / ntiles1;
      int tm, tn;
      tile_coords(t - pb * ntiles1, tiles_m, tiles_n, GROUP_M, tm, tn);
      const int nseg = grp.p[pb].nseg;
      for (int kb = 0; kb < nseg * nkb; ++kb) {
        if (!mbar_wait(&empty[s], ph ^ 1, status)) {
          ok = false;
          break;
        }
        uint8_t* st = smem + s * STAGE_BYTES;
        const int sg = kb >= nkb ? 1 : 0, kq = kb - sg * nkb;
        const int wa = grp.p[pb].a[sg], wb = grp.p[pb].b[sg];
        const int pn = kq / nkbp, kx = (kq - pn * nkbp) * BK;
        mbar_expect_tx(&full[s], STAGE_BYTES);
        tma_load(&mAhi, &full[s], st, kx, tm * BM, pn, wa);
        tma_load(&mAlo, &full[s], st + A_BYTES, kx, tm * BM, pn, wa);
        tma_load(&mBhi, &full[s], st + 2 * A_BYTES, kx, tn * BN, pn, wb);
        tma_load(&mBlo, &full[s], st + 2 * A_BYTES + B_BYTES, kx, tn * BN, pn, wb);
        ++nissued;
        if (++s == STAGES) {
          s = 0;
          ph ^= 1;
        }
      }
    }
    // make sure every copy issued has landed before the CTA can exit
    for (int q = 0; q < STAGES && q < nissued; ++q)
      mbar_wait(&full[q], (uint32_t)(((nissued - q + STAGES - 1) / STAGES - 1) & 1), status);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    int s = 0, cb = 0;
    uint32_t ph = 0, cph = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int nkbt = grp.p[t / ntiles1].nseg * nkb;
      for (int kb = 0; kb < nkbt; ++kb) {
        const bool first = kb % KPC == 0;
        const bool last = kb % KPC == KPC - 1 || kb == nkbt - 1;
        if ((first && !mbar_wait(&cempty[cb], cph ^ 1, status)) || !mbar_wait(&full[s], ph, status)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t d = tmem + (uint32_t)(cb * BN);
        const uint32_t base = su32(smem + s * STAGE_BYTES);
        const uint64_t ahi = smem_desc<CF>(base), alo = smem_desc<CF>(base + A_BYTES);
        const uint64_t bhi = smem_desc<CF>(base + 2 * A_BYTES), blo = smem_desc<CF>(base + 2 * A_BYTES + B_BYTES);
#pragma unroll
        for (int kk = 0; kk < CF::KSTEPS; ++kk) {
          const uint64_t off = (uint64_t)(kk * 32) >> 4;   // one k-step = 32 bytes along the swizzled row
          mma<CF>(d, alo + off, bhi + off, (first && kk == 0) ? 0u : 1u);
          mma<CF>(d, ahi + off, blo + off, 1);
          mma<CF>(d, ahi + off, bhi + off, 1);
        }
        mma_commit(&empty[s]);
        if (last) {
          mma_commit(&cfull[cb]);
          if (++cb == 2) {
            cb = 0;
            cph ^= 1;
          }
        }
        if (++s == STAGES) {
          s = 0;
          ph ^= 1;
        }
      }
    }
    // every MMA issued has completed once this commit arrives
    mma_commit(drain);
    mbar_wait(drain, 0, status);
  } else if (warp >= 2) {
    // ------------------------------------------------------------ promotion + epilogue
    const int q = warp & 3;                 // TMEM lane quarter this warp may access
    const int h = (warp - 2) >> 2;          // column half of the tile
    const int row = q * 32 + lane;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    int cb = 0;
    uint32_t cph = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int pb = t / ntiles1;
      int tm, tn;
      tile_coords(t - pb * ntiles1, tiles_m, tiles_n, GROUP_M, tm, tn);
      const int nchunk = (grp.p[pb].nseg * nkb + KPC - 1) / KPC;
      float acc[BN / 2];
#pragma unroll
      for (int j = 0; j < BN / 2; ++j) acc[j] = 0.f;
      for (int kc = 0; kc < nchunk; ++kc) {
        // warp-uniform outcome: tcgen05.ld below must be executed by all 32 lanes
        if (!__all_sync(0xffffffffu, mbar_wait(&cfull[cb], cph, status))) {
          ok = false;
          break;
        }
        fence_after();
        promote_chunk(tmem + lane_base + (uint32_t)(cb * BN + h * (BN / 2)), acc);
        fence_before();
        mbar_arrive(&cempty[cb]);
        if (++cb == 2) {
          cb = 0;
          cph ^= 1;
        }
      }
      if (!ok) break;
      store_row(grp.p[pb].C, ldc, M, N, (int64_t)tm * BM + row, tn * BN + h * (BN / 2), acc, out_alpha(grp, pb));
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// Two-CTA form (cluster of 2): CTA rank r holds rows r BM .. r BM + 127 of a 256-row tile
// (M tiles 2g and 2g + 1) and B rows r BN/2 .. r BN/2 + 127 of its N tile. Rank 0 (the even
// CTA) owns the full barriers of the copies, issues every MMA and collects the epilogue's
// "chunk drained" arrivals of both CTAs; each CTA's empty and chunk-full barriers are
// arrived at by rank 0's commits, one commit per barrier.
template <class CF>
__global__ void __launch_bounds__(THREADS, 1)
    gemm_pair_kernel(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                     const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo,
                     const __grid_constant__ GemmGroup grp, int64_t ldc, int M, int N, int Kp, int P,
                     int* status) {
  static_assert(CF::kPair && CF::kF16, "pair kernel: fp16 pair configuration");
  constexpr int STAGES = CF::STAGES, BK = CF::BK, A_BYTES = CF::A_BYTES, B_BYTES = CF::B_BYTES,
                STAGE_BYTES = CF::STAGE_BYTES, KPC = CF::KB_PER_CHUNK;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* full = bars;                 // [STAGES] rank 0's: both CTAs' copies of a stage landed
  uint64_t* empty = bars + STAGES;       // [STAGES] this CTA's stage may be refilled
  uint64_t* cfull = bars + 2 * STAGES;   // [2] this CTA's chunk accumulator written
  uint64_t* cempty = cfull + 2;          // [2] rank 0's: both CTAs drained the chunk accumulator
  uint64_t* drain = cempty + 2;          // [1]
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const int cid = blockIdx.x / 2, ncl = gridDim.x / 2;
  const int tiles_m = (M + BM - 1) / BM, tiles_n = (N + BN - 1) / BN;
  const int tiles_mg = (tiles_m + 1) / 2;               // 256-row tiles
  const int ntiles1 = tiles_mg * tiles_n;               // tiles of one output
  const int ntiles = grp.nprob * ntiles1;
  const int nkbp = (Kp + BK - 1) / BK;
  const int nkb = P * nkbp;                             // k-blocks of one segment

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);            // rank 0's producer arrival (it expects both CTAs' bytes)
      mbar_init(&empty[s], 1);           // rank 0's commit for this CTA
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&cfull[a], 1);
      mbar_init(&cempty[a], 2 * EPI_WARPS);   // one arrival per epilogue warp of either CTA
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    // the same TMEM columns in both CTAs (one warp of each CTA takes part)
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  fence_before();
  cluster_sync_all();   // both CTAs' barriers initialised and TMEM allocated before any use
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ TMA producer (both CTAs)
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mAhi) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mAlo) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mBhi) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mBlo) : "memory");
    const uint32_t full0 = mapa(su32(&full[0]), 0);   // rank 0's full barriers
    int s = 0;
    uint32_t ph = 0;
    int nissued = 0;   // k-blocks issued; stage q has been filled (nissued - q + STAGES - 1) / STAGES times
    bool ok = true;
    for (int t = cid; t < ntiles && ok; t += ncl) {
      const int pb = t / ntiles1;
      int tg, tn;
      tile_coords(t - pb * ntiles1, tiles_mg, tiles_n, GROUP_M / 2, tg, tn);
      const int tm = 2 * tg + (int)rank;
      const int yb = tn * BN + (int)rank * (BN / 2);
      const int nseg = grp.p[pb].nseg;
      for (int kb = 0; kb < nseg * nkb; ++kb) {
        if (!mbar_wait<true>(&empty[s], ph ^ 1, status)) {
          ok = false;
          break;
        }
        uint8_t* st = smem + s * STAGE_BYTES;
        const int sg = kb >= nkb ? 1 : 0, kq = kb - sg * nkb;
        const int wa = grp.p[pb].a[sg], wb = grp.p[pb].b[sg];
        const int pn = kq / nkbp, kx = (kq - pn * nkbp) * BK;
        if (rank == 0) mbar_expect_tx(&full[s], 2 * STAGE_BYTES);   // this CTA's and the partner's copies
        const uint32_t fb = full0 + (uint32_t)(s * sizeof(uint64_t));
        tma_load_pair(&mAhi, fb, st, kx, tm * BM, pn, wa);
        tma_load_pair(&mAlo, fb, st + A_BYTES, kx, tm * BM, pn, wa);
        tma_load_pair(&mBhi, fb, st + 2 * A_BYTES, kx, yb, pn, wb);
        tma_load_pair(&mBlo, fb, st + 2 * A_BYTES + B_BYTES, kx, yb, pn, wb);
        ++nissued;
        if (++s == STAGES) {
          s = 0;
          ph ^= 1;
        }
      }
    }
    // rank 0 sees every copy of both CTAs land on its own barriers before it can leave (the
    // partner waits for rank 0 at the closing cluster barrier)
    if (rank == 0)
      for (int q = 0; q < STAGES && q < nissued; ++q)
        mbar_wait(&full[q], (uint32_t)(((nissued - q + STAGES - 1) / STAGES - 1) & 1), status);
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ------------------------------------------------------------ MMA issuer (rank 0)
    const uint32_t empty1 = mapa(su32(&empty[0]), 1), cfull1 = mapa(su32(&cfull[0]), 1);
    int s = 0, cb = 0;
    uint32_t ph = 0, cph = 0;
    bool ok = true;
    for (int t = cid; t < ntiles && ok; t += ncl) {
      const int nkbt = grp.p[t / ntiles1].nseg * nkb;
      for (int kb = 0; kb < nkbt; ++kb) {
        const bool first = kb % KPC == 0;
        const bool last = kb % KPC == KPC - 1 || kb == nkbt - 1;
        if ((first && !mbar_wait<true>(&cempty[cb], cph ^ 1, status)) || !mbar_wait(&full[s], ph, status)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t d = tmem + (uint32_t)(cb * BN);
        const uint32_t base = su32(smem + s * STAGE_BYTES);   // the same offsets in both CTAs
        const uint64_t ahi = smem_desc<CF>(base), alo = smem_desc<CF>(base + A_BYTES);
        const uint64_t bhi = smem_desc<CF>(base + 2 * A_BYTES), blo = smem_desc<CF>(base + 2 * A_BYTES + B_BYTES);
#pragma unroll
        for (int kk = 0; kk < CF::KSTEPS; ++kk) {
          const uint64_t off = (uint64_t)(kk * 32) >> 4;
          mma<CF>(d, alo + off, bhi + off, (first && kk == 0) ? 0u : 1u);
          mma<CF>(d, ahi + off, blo + off, 1);
          mma<CF>(d, ahi + off, bhi + off, 1);
        }
        mma_commit_pair(su32(&empty[s]));
        mma_commit_pair(empty1 + (uint32_t)(s * sizeof(uint64_t)));
        if (last) {
          mma_commit_pair(su32(&cfull[cb]));
          mma_commit_pair(cfull1 + (uint32_t)(cb * sizeof(uint64_t)));
          if (++cb == 2) {
            cb = 0;
            cph ^= 1;
          }
        }
        if (++s == STAGES) {
          s = 0;
          ph ^= 1;
        }
      }
    }
    mma_commit_pair(su32(drain));
    mbar_wait(drain, 0, status);
  } else if (warp >= 2) {
    // ------------------------------------------------------------ promotion + epilogue (both CTAs)
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const uint32_t cempty0 = mapa(su32(&cempty[0]), 0);   // rank 0's drained barriers
    int cb = 0;
    uint32_t cph = 0;
    bool ok = true;
    for (int t = cid; t < ntiles && ok; t += ncl) {
      const int pb = t / ntiles1;
      int tg, tn;
      tile_coords(t - pb * ntiles1, tiles_mg, tiles_n, GROUP_M / 2, tg, tn);
      const int tm = 2 * tg + (int)rank;
      const int nchunk = (grp.p[pb].nseg * nkb + KPC - 1) / KPC;
      float acc[BN / 2];
#pragma unroll
      for (int j = 0; j < BN / 2; ++j) acc[j] = 0.f;
      for (int kc = 0; kc < nchunk; ++kc) {
        if (!__all_sync(0xffffffffu, mbar_wait<true>(&cfull[cb], cph, status))) {
          ok = false;
          break;
        }
        fence_after();
        promote_chunk(tmem + lane_base + (uint32_t)(cb * BN + h * (BN / 2)), acc);
        fence_before();
        __syncwarp();   // every lane's tcgen05.ld has completed (wait::ld) before the arrival
        if (lane == 0) mbar_arrive_cluster(cempty0 + (uint32_t)(cb * sizeof(uint64_t)));
        if (++cb == 2) {
          cb = 0;
          cph ^= 1;
        }
      }
      if (!ok) break;
      store_row(grp.p[pb].C, ldc, M, N, (int64_t)tm * BM + row, tn * BN + h * (BN / 2), acc, out_alpha(grp, pb));
    }
  }
  fence_before();
  __syncthreads();
  // neither CTA leaves (or frees TMEM) while rank 0's MMAs may still read its shared memory
  // or write its TMEM, or while arrivals addressed to it may still be in flight
  cluster_sync_all();
  if (warp == 0) {
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ---------------------------------------------------------------------------- FP64-grade GEMM
// gemm_oz_kernel: C = alpha A B^T in FP64 accuracy on the fp16 tensor cores (an Ozaki-type
// splitting; Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59 (2012), here with fixed-point
// slices). Each operand is given as kOzSlices = 5 planes of integers, x = sum_i v_i 2^-8(i+1)
// (|v_0| <= 256, |v_i| <= 128: |x| < 1 after the max-norm scale), so x_A x_B = sum_{i,j}
// v_i w_j 2^-8(i+j+2). The products with i + j <= 4 (15 of the 25; the rest lie below 2^-40 of
// the leading one) are formed, one TMEM accumulator per group g = i + j (5 x 96 columns).
// Within a chunk of 256 k the sums of groups 0 and 1 are integers below 2^24, exact in FP32
// whatever order and truncation the tensor cores use; group 2 lies below 2^-16 of the leading
// group (one FP32 rounding per chunk below 2^-40 of it, and only when its sum passes 2^24),
// groups 3 and 4 below 2^-24. After each chunk the epilogue adds groups 0..2 (times 1, 2^-8,
// 2^-16) into a float pair hi + lo (TwoSum), 2^-24 and 2^-32 times groups 3 and 4 into lo, and
// renormalises the pair; at the end it writes alpha 2^-(16 + eA + eB) (hi + lo) in FP64 (added
// to C when accumulating): no FP64 arithmetic in the k loop (a few FP64 operations per clock
// per SM on this chip).
//   Tile 128 x 96 per CTA, one CTA per SM; k-blocks of 32 fp16 (64-byte swizzle), 3 stages
//   of 10 planes (70 KB); warp 0 TMA, warp 1 MMA (15 products x 2 k-steps per k-block),
//   warps 2..13 promotion (warp w: TMEM lane quarter w % 4, 32 of the 96 columns).
constexpr int OZ_BN = 96;
constexpr int OZ_EPI_WARPS = 12;
constexpr int OZ_THREADS = 64 + 32 * OZ_EPI_WARPS;
constexpr int OZ_COLS = OZ_BN / (OZ_EPI_WARPS / 4);   // 32 columns per epilogue thread
constexpr int OZ_TMEM_COLS = 512;                       // 5 x 96 used
struct CfgOz {
  static constexpr bool kF16 = true;
  static constexpr bool kPair = false;
  static constexpr int ELT = 2;
  static constexpr int BK = 32;
  static constexpr int KSTEPS = 2;
  static constexpr int STAGES = 3;
  static constexpr int A_PLANE = BM * 64;                 // bytes of one plane's k-block
  static constexpr int B_PLANE = OZ_BN * 64;
  static constexpr int STAGE_BYTES = kOzSlices * (A_PLANE + B_PLANE);
  static constexpr int KB_PER_CHUNK = 256 / BK;
  static constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
  static_assert(SMEM_BYTES <= 232448, "shared memory per CTA");
  static constexpr uint64_t LAYOUT = 4;                   // 64-byte swizzle
  static constexpr uint32_t SBO = 8 * 64;
  // D = F32, A = B = F16, both K-major, N = 96, M = 128
  static constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(OZ_BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
};

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// hi + lo += x (Knuth's TwoSum; the error of the sum goes into lo)
__device__ __forceinline__ void two_sum_into(float& hi, float& lo, float x) {
  const float t = hi + x;
  const float bp = t - hi;
  lo += (hi - (t - bp)) + (x - bp);
  hi = t;
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
    gemm_oz_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
                   double* __restrict__ C, int64_t ldc, int M, int N, int Kp, int P, double alpha,
                   const unsigned* amax_a, const unsigned* amax_b, int accumulate, int* status) {
  using CF = CfgOz;
  constexpr int STAGES = CF::STAGES, BK = CF::BK, STAGE_BYTES = CF::STAGE_BYTES, KPC = CF::KB_PER_CHUNK;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* full = bars;                 // [STAGES]
  uint64_t* empty = bars + STAGES;       // [STAGES]
  uint64_t* cfull = bars + 2 * STAGES;   // chunk accumulators written
  uint64_t* cempty = cfull + 1;          // chunk accumulators drained
  uint64_t* drain = cempty + 1;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_m = (M + BM - 1) / BM, tiles_n = (N + OZ_BN - 1) / OZ_BN;
  const int ntiles = tiles_m * tiles_n;
  const int nkbp = (Kp + BK - 1) / BK;
  const int nkb = P * nkbp;
  const int nchunk = (nkb + KPC - 1) / KPC;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(cfull, 1);
    mbar_init(cempty, 32 * OZ_EPI_WARPS);
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(OZ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ TMA producer
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mB) : "memory");
    int s = 0, nissued = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      int tm, tn;
      tile_coords(t, tiles_m, tiles_n, GROUP_M, tm, tn);
      for (int kb = 0; kb < nkb; ++kb) {
        if (!mbar_wait(&empty[s], ph ^ 1, status)) {
          ok = false;
          break;
        }
        uint8_t* st = smem + s * STAGE_BYTES;
        const int pn = kb / nkbp, kx = (kb - pn * nkbp) * BK;
        mbar_expect_tx(&full[s], STAGE_BYTES);
#pragma unroll
        for (int q = 0; q < kOzSlices; ++q) {
          tma_load(&mA, &full[s], st + q * CF::A_PLANE, kx, tm * BM, pn, q);
          tma_load(&mB, &full[s], st + kOzSlices * CF::A_PLANE + q * CF::B_PLANE, kx, tn * OZ_BN, pn, q);
        }
        ++nissued;
        if (++s == STAGES) {
          s = 0;
          ph ^= 1;
        }
      }
    }
    for (int q = 0; q < STAGES && q < nissued; ++q)
      mbar_wait(&full[q], (uint32_t)(((nissued - q + STAGES - 1) / STAGES - 1) & 1), status);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    int s = 0;
    uint32_t ph = 0, cph = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      for (int kb = 0; kb < nkb; ++kb) {
        const bool first = kb % KPC == 0;
        const bool last = kb % KPC == KPC - 1 || kb == nkb - 1;
        if ((first && !mbar_wait(cempty, cph ^ 1, status)) || !mbar_wait(&full[s], ph, status)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t base = su32(smem + s * STAGE_BYTES);
#pragma unroll
        for (int kk = 0; kk < CF::KSTEPS; ++kk) {
          const uint64_t off = (uint64_t)(kk * 32) >> 4;
#pragma unroll
          for (int g = 0; g < kOzSlices; ++g) {
            const uint32_t d = tmem + (uint32_t)(g * OZ_BN);
#pragma unroll
            for (int i = 0; i <= g; ++i) {
              const uint64_t a = smem_desc<CF>(base + i * CF::A_PLANE) + off;
              const uint64_t b = smem_desc<CF>(base + kOzSlices * CF::A_PLANE + (g - i) * CF::B_PLANE) + off;
              mma<CF>(d, a, b, (first && kk == 0 && i == 0) ? 0u : 1u);
            }
          }
        }
        mma_commit(&empty[s]);
        if (last) {
          mma_commit(cfull);
          cph ^= 1;
        }
        if (++s == STAGES) {
          s = 0;
          ph ^= 1;
        }
      }
    }
    mma_commit(drain);
    mbar_wait(drain, 0, status);
  } else if (warp >= 2) {
    // ------------------------------------------------------------ promotion + epilogue
    const int q = warp & 3;                       // TMEM lane quarter
    const int cpart = (warp - 2) >> 2;            // which 32 of the 96 columns
    const int row = q * 32 + lane;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    uint32_t cph = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      int tm, tn;
      tile_coords(t, tiles_m, tiles_n, GROUP_M, tm, tn);
      float hi[OZ_COLS], lo[OZ_COLS];
#pragma unroll
      for (int j = 0; j < OZ_COLS; ++j) hi[j] = lo[j] = 0.f;
      for (int kc = 0; kc < nchunk; ++kc) {
        if (!__all_sync(0xffffffffu, mbar_wait(cfull, cph, status))) {
          ok = false;
          break;
        }
        fence_after();
#pragma unroll
        for (int g = 0; g < kOzSlices; ++g) {
          // 2^-8g: exact scalings of exact (groups 0, 1) or nearly exact (2..4) chunk sums
          const float sc = g == 0 ? 1.f : (g == 1 ? 0x1p-8f : (g == 2 ? 0x1p-16f : (g == 3 ? 0x1p-24f : 0x1p-32f)));
#pragma unroll
          for (int c16 = 0; c16 < OZ_COLS; c16 += 16) {
            float v[16];
            tmem_ld16(tmem + lane_base + (uint32_t)(g * OZ_BN + cpart * OZ_COLS + c16), v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              if (g < 3) two_sum_into(hi[c16 + j], lo[c16 + j], v[j] * sc);
              else lo[c16 + j] = fmaf(v[j], sc, lo[c16 + j]);
            }
          }
        }
        // renormalise each pair (FastTwoSum: |lo| back to half an ulp of hi), so that lo's own
        // roundings stay near 2^-48 of the sum over the whole k loop
#pragma unroll
        for (int j = 0; j < OZ_COLS; ++j) {
          const float s = hi[j] + lo[j];
          lo[j] = lo[j] - (s - hi[j]);
          hi[j] = s;
        }
        fence_before();
        mbar_arrive(cempty);
        cph ^= 1;
      }
      if (!ok) break;
      const int64_t m = (int64_t)tm * BM + row;
      const int n0 = tn * OZ_BN + cpart * OZ_COLS;
      if (m < M) {
        double* crow = C + m * ldc + n0;
        // alpha 2^-16, and 2^-(eA + eB) for the operands' max-norm scales
        const int es = amax_a ? split_exponent(*amax_a, kOzTop) + split_exponent(*amax_b, kOzTop) : 0;
        const double a16 = ldexp(alpha, -16 - es);
#pragma unroll
        for (int j = 0; j < OZ_COLS; ++j)
          if (n0 + j < N) crow[j] = a16 * ((double)hi[j] + (double)lo[j]) + (accumulate ? crow[j] : 0.0);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS) : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

template <class CF>
bool make_map(CUtensorMap* map, const void* ptr, int64_t rows, int64_t Kp, int64_t kps, int64_t P, int64_t W,
              int64_t wstride, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[4] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)P, (cuuint64_t)W};
  cuuint64_t strides[3] = {(cuuint64_t)(kps * CF::ELT), (cuuint64_t)(rows * kps * CF::ELT),
                           (cuuint64_t)(wstride * CF::ELT)};
  cuuint32_t box[4] = {(cuuint32_t)CF::BK, (cuuint32_t)box_rows, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(map, CF::kF16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)ptr,
                   dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CF::LAYOUT == 2 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Per-device launch set-up (SM count, shared-memory attributes, pair grid), done once per
// device while it is current and before any launch on it, so that no launch inside a stream
// capture does host-side set-up and a process driving several devices sets each one up.
constexpr int kMaxDevices = 64;
struct DeviceSetup {
  bool done = false;
  int sms = 0;
  int pair_grid = 0;   // 2 x the two-CTA clusters that can be resident at once (0: none)
};
DeviceSetup g_setup[kMaxDevices];

const DeviceSetup* device_setup() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  DeviceSetup& d = g_setup[dev];
  if (d.done) return &d;
  if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return nullptr;
  bool ok = cudaFuncSetAttribute(gemm_tf32x3_kernel<CfgTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)CfgTF32::SMEM_BYTES) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(gemm_tf32x3_kernel<CfgTF32W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)CfgTF32W::SMEM_BYTES) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(gemm_tf32x3_kernel<CfgF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)CfgF16::SMEM_BYTES) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(gemm_tf32x3_kernel<CfgF16S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)CfgF16S::SMEM_BYTES) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(gemm_tf32x3_kernel<CfgF16L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)CfgF16L::SMEM_BYTES) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(gemm_oz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)CfgOz::SMEM_BYTES) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return nullptr;
  }
  int n = 0;
  if (cudaFuncSetAttribute(gemm_pair_kernel<CfgF16P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)CfgF16P::SMEM_BYTES) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * 64);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = CfgF16P::SMEM_BYTES;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&n, gemm_pair_kernel<CfgF16P>, &cfg) != cudaSuccess) n = 0;
  }
  cudaGetLastError();
  d.pair_grid = 2 * n;
  d.done = true;
  return &d;
}

template <class CF>
cudaError_t launch_single(const void* Ahi, const void* Alo, const void* Bhi, const void* Blo, int64_t W, int64_t aws,
                          int64_t bws, int64_t Kp, int64_t kps, int64_t P, int64_t M, int64_t N, int64_t ldc,
                          const GemmGroup& g, int* status, cudaStream_t st, const DeviceSetup& dv) {
  CUtensorMap mAhi, mAlo, mBhi, mBlo;
  if (!make_map<CF>(&mAhi, Ahi, M, Kp, kps, P, W, aws, BM) || !make_map<CF>(&mAlo, Alo, M, Kp, kps, P, W, aws, BM) ||
      !make_map<CF>(&mBhi, Bhi, N, Kp, kps, P, W, bws, BN) || !make_map<CF>(&mBlo, Blo, N, Kp, kps, P, W, bws, BN))
    return cudaErrorInvalidValue;
  const int64_t tiles = g.nprob * ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  const int grid = (int)(tiles < dv.sms ? tiles : dv.sms);
  gemm_tf32x3_kernel<CF><<<grid, THREADS, CF::SMEM_BYTES, st>>>(mAhi, mAlo, mBhi, mBlo, g, ldc, (int)M, (int)N,
                                                               (int)Kp, (int)P, status);
  return cudaGetLastError();
}

cudaError_t launch_pair(const void* Ahi, const void* Alo, const void* Bhi, const void* Blo, int64_t W, int64_t aws,
                        int64_t bws, int64_t Kp, int64_t kps, int64_t P, int64_t M, int64_t N, int64_t ldc,
                        const GemmGroup& g, int* status, cudaStream_t st, const DeviceSetup& dv) {
  using CF = CfgF16P;
  CUtensorMap mAhi, mAlo, mBhi, mBlo;
  // each CTA copies its own 128 rows of A and its own 128-row half of the B tile
  if (!make_map<CF>(&mAhi, Ahi, M, Kp, kps, P, W, aws, BM) || !make_map<CF>(&mAlo, Alo, M, Kp, kps, P, W, aws, BM) ||
      !make_map<CF>(&mBhi, Bhi, N, Kp, kps, P, W, bws, BN / 2) ||
      !make_map<CF>(&mBlo, Blo, N, Kp, kps, P, W, bws, BN / 2))
    return cudaErrorInvalidValue;
  const int64_t pairs = g.nprob * ((M + 2 * BM - 1) / (2 * BM)) * ((N + BN - 1) / BN);
  int grid = dv.pair_grid;
  if (grid / 2 > pairs) grid = (int)(2 * pairs);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = CF::SMEM_BYTES;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, gemm_pair_kernel<CF>, mAhi, mAlo, mBhi, mBlo, g, ldc, (int)M, (int)N, (int)Kp,
                            (int)P, status);
}

}  // namespace tc

// Every output of the group g: C_p[M][N] (row stride ldc) = alpha_p * sum over its segments
// s of A_{a_s} B_{b_s}^T, with the W operand tensors of each plane in K panels (see
// tma_load): panel width Kp (kps = its stride), P panels, K = P Kp per segment; tensor w of
// a plane starts aws (A) or bws (B) elements after tensor w - 1. variant 0:
// tf32, k-blocks of 16, 64-byte swizzle, 4 stages; 1: tf32, k-blocks of 32, 128-byte
// swizzle, 2 stages; 2: fp16 operands (hi/lo planes of __half), k-blocks of 32, 64-byte
// swizzle, 4 stages, 128-k promotion chunks (kps % 8 == 0); 3: as 2 with 64-k chunks; 4: as
// 2 with 256-k chunks; 5: fp16 in CTA pairs (tcgen05.mma.cta_group::2, 256 x 256 tiles),
// k-blocks of 64 (kps % 64 == 0), 128-k chunks.
cudaError_t launch_gemm_group(const void* Ahi, const void* Alo, const void* Bhi, const void* Blo, int W, int64_t aws,
                              int64_t bws, int64_t Kp, int64_t kps, int64_t P, int64_t M, int64_t N, int64_t ldc,
                              const GemmGroup& g, int* status, cudaStream_t st, int variant) {
  using namespace tc;
  if (M <= 0 || N <= 0 || g.nprob == 0) return cudaSuccess;
  if (Kp <= 0 || P <= 0 || W < 1 || M > 0x7fffffff || N > 0x7fffffff || Kp * P > 0x7fffffff || ldc < N ||
      g.nprob < 0 || g.nprob > kMaxGemmProblems || (W > 1 && (aws < P * M * kps || bws < P * N * kps)))
    return cudaErrorInvalidValue;
  for (int q = 0; q < g.nprob; ++q) {
    const GemmProblem& pr = g.p[q];
    if (!pr.C || pr.nseg < 1 || pr.nseg > 2) return cudaErrorInvalidValue;
    for (int sg = 0; sg < pr.nseg; ++sg)
      if (pr.a[sg] < 0 || pr.a[sg] >= W || pr.b[sg] < 0 || pr.b[sg] >= W) return cudaErrorInvalidValue;
  }
  if ((g.amax_a == nullptr) != (g.amax_b == nullptr) || (g.amax_a && g.per_elem < 1)) return cudaErrorInvalidValue;
  const bool f16 = variant >= 2 && variant <= 5;
  if ((kps & (variant == 5 ? 63 : (f16 ? 7 : 3))) || kps < Kp) return cudaErrorInvalidValue;
  if ((((uintptr_t)Ahi) | ((uintptr_t)Alo) | ((uintptr_t)Bhi) | ((uintptr_t)Blo)) & 15) return cudaErrorInvalidValue;
  const DeviceSetup* dv = device_setup();
  if (!dv) return cudaErrorInitializationError;
  if (variant == 5) {
    // a device (or partition) that cannot co-schedule two-CTA clusters runs the same
    // products on single CTAs
    if (dv->pair_grid >= 2) return launch_pair(Ahi, Alo, Bhi, Blo, W, aws, bws, Kp, kps, P, M, N, ldc, g, status, st, *dv);
    return launch_single<CfgF16>(Ahi, Alo, Bhi, Blo, W, aws, bws, Kp, kps, P, M, N, ldc, g, status, st, *dv);
  }
  if (variant == 4) return launch_single<CfgF16L>(Ahi, Alo, Bhi, Blo, W, aws, bws, Kp, kps, P, M, N, ldc, g, status, st, *dv);
  if (variant == 3) return launch_single<CfgF16S>(Ahi, Alo, Bhi, Blo, W, aws, bws, Kp, kps, P, M, N, ldc, g, status, st, *dv);
  if (variant == 2) return launch_single<CfgF16>(Ahi, Alo, Bhi, Blo, W, aws, bws, Kp, kps, P, M, N, ldc, g, status, st, *dv);
  if (variant == 1) return launch_single<CfgTF32W>(Ahi, Alo, Bhi, Blo, W, aws, bws, Kp, kps, P, M, N, ldc, g, status, st, *dv);
  return launch_single<CfgTF32>(Ahi, Alo, Bhi, Blo, W, aws, bws, Kp, kps, P, M, N, ldc, g, status, st, *dv);
}

// FP64-grade GEMM (gemm_oz_kernel): C = alpha A B^T, A and B as kOzSlices integer planes in
// K panels, plane p of A at A + p aps elements (B: bps); kps % 8 == 0.
cudaError_t launch_gemm_oz(const void* A, const void* B, int64_t aps, int64_t bps, int64_t Kp, int64_t kps, int64_t P,
                           int64_t M, int64_t N, double* C, int64_t ldc, double alpha, const unsigned* amax_a,
                           const unsigned* amax_b, bool accumulate, int* status, cudaStream_t st) {
  using namespace tc;
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (!A || !B || !C || Kp <= 0 || P <= 0 || M > 0x7fffffff || N > 0x7fffffff || Kp * P > 0x7fffffff || ldc < N ||
      (kps & 7) || kps < Kp || aps < P * M * kps || bps < P * N * kps)
    return cudaErrorInvalidValue;
  if ((((uintptr_t)A) | ((uintptr_t)B)) & 15) return cudaErrorInvalidValue;
  const DeviceSetup* dv = device_setup();
  if (!dv) return cudaErrorInitializationError;
  CUtensorMap mA, mB;
  if (!make_map<CfgOz>(&mA, A, M, Kp, kps, P, kOzSlices, aps, BM) ||
      !make_map<CfgOz>(&mB, B, N, Kp, kps, P, kOzSlices, bps, OZ_BN))
    return cudaErrorInvalidValue;
  const int64_t tiles = ((M + BM - 1) / BM) * ((N + OZ_BN - 1) / OZ_BN);
  const int grid = (int)(tiles < dv->sms ? tiles : dv->sms);
  if ((amax_a == nullptr) != (amax_b == nullptr)) return cudaErrorInvalidValue;
  gemm_oz_kernel<<<grid, OZ_THREADS, CfgOz::SMEM_BYTES, st>>>(mA, mB, C, ldc, (int)M, (int)N, (int)Kp, (int)P, alpha,
                                                              amax_a, amax_b, accumulate ? 1 : 0, status);
  return cudaGetLastError();
}

// Sets the kernels' shared-memory attributes and caches the SM count and pair grid of the
// current device ahead of time, so no first launch does host-side set-up (which must not
// happen inside a stream capture).
void gemm_prepare() { tc::device_setup(); }

cudaError_t launch_wait_selftest(int* status, unsigned long long limit_ns, cudaStream_t st) {
  tc::wait_selftest_kernel<<<1, 32, 0, st>>>(status, limit_ns);
  return cudaGetLastError();
}

}  // namespace hotrg
