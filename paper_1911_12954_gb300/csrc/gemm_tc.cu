// gemm_tc.cu - tcgen05 / TMEM / TMA GEMM for the block-spin contraction (FP16x3 and TF32x3).
//
// C[m][n] = alpha * sum_k (Ahi Bhi + Ahi Blo + Alo Bhi)[m,n,k] + beta * C[m][n]
// with A = Ahi + Alo and B = Bhi + Blo: either fp16 planes (hi, lo of 2^14 x; kind::f16,
// the default) or tf32 values stored in FP32 words (kind::tf32), both operands K-major in
// K panels (see tma_load). This is the O(D^15) block-spin contraction of the HOTRG step,
// where Sec. 2 of arXiv:1911.12954 places the D^(4d-1) cost of the method, carried out on
// the 5th-generation tensor cores with FP32 accumulation; the dropped Alo Blo term is below
// 2^-21 of each product.
//
// The tensor cores add each MMA's products into the FP32 accumulator with truncation,
// so an accumulator that runs over the whole K picks up a bias that grows linearly with
// K (measured 2.5e-4 relative at K = 32768). The kernel therefore promotes the partial
// sum of every chunk of k (32 for tf32; 128, or 64 in the short-chunk variant, for fp16)
// from TMEM into FP32 registers, where the sums are rounded to nearest: the truncation
// bias is bounded by one chunk's worth. Each promotion reads the whole 128 x 256 FP32
// accumulator out of TMEM and holds the MMAs back for a few hundred cycles, so the chunk
// is as long as the accuracy allows (at D = 8, 64-k chunks cost 17 % of the MMA time and
// 128-k chunks 7 %).
//
// Structure: persistent kernel, one CTA per SM, 10 warps.
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
// k promoted from TMEM to registers at once.
template <int ROWB, bool F16, int CHUNK>
struct Cfg {
  static constexpr bool kF16 = F16;
  static constexpr int ELT = F16 ? 2 : 4;
  static constexpr int BK = ROWB / ELT;                            // elements per k-block
  static constexpr int KSTEPS = ROWB / 32;                         // MMAs per product per k-block
  static constexpr int STAGES = ROWB == 128 ? 2 : 4;
  static constexpr int A_BYTES = BM * ROWB;
  static constexpr int B_BYTES = BN * ROWB;
  static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int KB_PER_CHUNK = CHUNK / BK;
  static_assert(CHUNK % BK == 0, "a chunk is a whole number of k-blocks");
  static constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
  static constexpr uint64_t LAYOUT = ROWB == 128 ? 2 : 4;         // UMMA swizzle: 128 B or 64 B
  static constexpr uint32_t SBO = 8 * ROWB;                       // 8 rows of one swizzle row
  // instruction descriptor: D = F32; A = B = TF32 (2) or F16 (0); both K-major; N = 256, M = 128
  static constexpr uint32_t IDESC = (1u << 4) | ((F16 ? 0u : 2u) << 7) | ((F16 ? 0u : 2u) << 10) |
                                    ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
};
using CfgTF32 = Cfg<64, false, 32>;     // default tf32 pipeline: 4 stages of 16-wide k-blocks
using CfgTF32W = Cfg<128, false, 32>;   // tf32, 2 stages of 32-wide k-blocks
using CfgF16 = Cfg<64, true, 128>;      // fp16: 4 stages of 32-wide k-blocks, 128-k chunks
using CfgF16S = Cfg<64, true, 64>;      // fp16 with 64-k chunks
using CfgF16L = Cfg<64, true, 256>;     // fp16 with 256-k chunks

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
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; false (and the timeout status raised) when it gives up.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* status,
                                          unsigned long long limit_ns = kWaitNs) {
  if (mbar_try(b, parity)) return true;
  const unsigned long long t0 = now_ns();
  while (true) {
    if (mbar_try(b, parity)) return true;
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

// Operands are stored in K panels: element (row, k) with k = p Kp + kin sits at
// [(p rows + row) kps + kin] (kps = Kp rounded up to 4). The 3D tensor map is
// {Kp, rows, P}; a panel keeps the rows of one k range contiguous, so a box of 128 rows
// spans at most a few pages even when K is in the hundreds of thousands.
__device__ __forceinline__ void tma_load(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(su32(dst)),
      "l"((uint64_t)map), "r"(su32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// The same load delivered to the same shared-memory offset (and completing the same mbarrier
// offset) in every CTA of the cluster named by ctaMask.
__device__ __forceinline__ void tma_load_mc(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y, int z,
                                            uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster"
      " [%0], [%1, {%3, %4, %5}], [%2], %6;" ::"r"(su32(dst)),
      "l"((uint64_t)map), "r"(su32(bar)), "r"(x), "r"(y), "r"(z), "h"(mask)
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
  if constexpr (CF::kF16) {
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
// Arrives (once the MMAs issued so far have completed) on the mbarrier at this offset in
// every CTA of the cluster named by ctaMask.
__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                   su32(bar)),
               "h"(mask)
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

// CL = 2: clusters of two CTAs on vertically adjacent tiles (same N tile, M tiles 2g and
// 2g + 1). Each CTA loads its own A tile and one half of the shared B tile, multicast into
// both CTAs, so B is read from L2 once per pair; a stage is refilled only after both CTAs'
// MMAs have read it (their commits arrive on both CTAs' empty barriers).
template <class CF, int CL>
__global__ void __launch_bounds__(THREADS, 1)
    gemm_tf32x3_kernel(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                       const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo,
                       float* __restrict__ C, int64_t ldc, int M, int N, int Kp, int P, float alpha, float beta,
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
  const int rm = CL == 2 ? (int)cluster_rank() : 0;    // this CTA's M tile within the pair
  const int cid = blockIdx.x / CL, ncl = gridDim.x / CL;
  const int tiles_m = (M + BM - 1) / BM, tiles_n = (N + BN - 1) / BN;
  const int tiles_mg = (tiles_m + CL - 1) / CL;          // M tiles per cluster group
  const int ntiles = tiles_mg * tiles_n;
  const int nkbp = (Kp + BK - 1) / BK;   // k-blocks per panel (the last one zero-filled past Kp)
  const int nkb = P * nkbp;
  const int nchunk = (nkb + KPC - 1) / KPC;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], CL);      // the MMA commits of every CTA that reads this stage
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
  if (CL == 2) cluster_sync_all();   // the partner's barriers exist before any multicast
  else __syncthreads();
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
    int issued[STAGES] = {};
    bool ok = true;
    for (int t = cid; t < ntiles && ok; t += ncl) {
      int tg, tn;
      tile_coords(t, tiles_mg, tiles_n, GROUP_M / CL, tg, tn);
      const int tm = tg * CL + rm;
      for (int kb = 0; kb < nkb; ++kb) {
        if (!mbar_wait(&empty[s], ph ^ 1, status)) {
          ok = false;
          break;
        }
        uint8_t* st = smem + s * STAGE_BYTES;
        const int pn = kb / nkbp, kx = (kb - pn * nkbp) * BK;
        mbar_expect_tx(&full[s], STAGE_BYTES);   // own A + both halves of B
        tma_load(&mAhi, &full[s], st, kx, tm * BM, pn);
        tma_load(&mAlo, &full[s], st + A_BYTES, kx, tm * BM, pn);
        if (CL == 2) {
          const int half = B_BYTES / 2, yb = tn * BN + rm * (BN / 2);
          tma_load_mc(&mBhi, &full[s], st + 2 * A_BYTES + rm * half, kx, yb, pn, 3);
          tma_load_mc(&mBlo, &full[s], st + 2 * A_BYTES + B_BYTES + rm * half, kx, yb, pn, 3);
        } else {
          tma_load(&mBhi, &full[s], st + 2 * A_BYTES, kx, tn * BN, pn);
          tma_load(&mBlo, &full[s], st + 2 * A_BYTES + B_BYTES, kx, tn * BN, pn);
        }
        ++issued[s];
        if (++s == STAGES) {
          s = 0;
          ph ^= 1;
        }
      }
    }
    // make sure every copy issued has landed before the CTA can exit
    for (int q = 0; q < STAGES; ++q)
      if (issued[q] > 0) mbar_wait(&full[q], (uint32_t)((issued[q] - 1) & 1), status);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    int s = 0, cb = 0;
    uint32_t ph = 0, cph = 0;
    bool ok = true;
    for (int t = cid; t < ntiles && ok; t += ncl) {
      for (int kb = 0; kb < nkb; ++kb) {
        const bool first = kb % KPC == 0;
        const bool last = kb % KPC == KPC - 1 || kb == nkb - 1;
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
        if (CL == 2) mma_commit_mc(&empty[s], 3);
        else mma_commit(&empty[s]);
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
    for (int t = cid; t < ntiles && ok; t += ncl) {
      int tg, tn;
      tile_coords(t, tiles_mg, tiles_n, GROUP_M / CL, tg, tn);
      const int tm = tg * CL + rm;
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
#pragma unroll
        for (int c = 0; c < BN / 64; ++c) {
          float v[32];
          tmem_ld32(tmem + lane_base + (uint32_t)(cb * BN + h * (BN / 2) + c * 32), v);
#pragma unroll
          for (int j = 0; j < 32; ++j) acc[c * 32 + j] += v[j];
        }
        fence_before();
        mbar_arrive(&cempty[cb]);
        if (++cb == 2) {
          cb = 0;
          cph ^= 1;
        }
      }
      if (!ok) break;
      const int64_t m = (int64_t)tm * BM + row;
      const int n0 = tn * BN + h * (BN / 2);
      if (m < M) {
        float* crow = C + m * ldc + n0;
        if (n0 + BN / 2 <= N && ((((uintptr_t)crow) & 15) == 0)) {
#pragma unroll
          for (int j = 0; j < BN / 2; j += 4) {
            float4 o = make_float4(alpha * acc[j], alpha * acc[j + 1], alpha * acc[j + 2], alpha * acc[j + 3]);
            if (beta != 0.f) {
              const float4 old = *(const float4*)(crow + j);
              o.x += beta * old.x;
              o.y += beta * old.y;
              o.z += beta * old.z;
              o.w += beta * old.w;
            }
            *(float4*)(crow + j) = o;
          }
        } else {
#pragma unroll
          for (int j = 0; j < BN / 2; ++j)
            if (n0 + j < N) crow[j] = alpha * acc[j] + (beta != 0.f ? beta * crow[j] : 0.f);
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  // neither CTA leaves while the partner may still multicast into it or arrive on its barriers
  if (CL == 2) cluster_sync_all();
  if (warp == 0) {
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
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
bool make_map(CUtensorMap* map, const void* ptr, int64_t rows, int64_t Kp, int64_t kps, int64_t P, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)P};
  cuuint64_t strides[2] = {(cuuint64_t)(kps * CF::ELT), (cuuint64_t)(rows * kps * CF::ELT)};
  cuuint32_t box[3] = {(cuuint32_t)CF::BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CF::kF16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)ptr,
                   dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CF::LAYOUT == 2 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Grid of the 2-CTA cluster variant: twice the number of two-CTA clusters that can be
// resident at once (every SM that can pair up), found once per kernel before any capture.
template <class CF>
int cluster_grid() {
  static int grid = -1;
  if (grid >= 0) return grid;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2 * 64);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = CF::SMEM_BYTES;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaFuncSetAttribute(gemm_tf32x3_kernel<CF, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)CF::SMEM_BYTES) != cudaSuccess ||
      cudaOccupancyMaxActiveClusters(&n, gemm_tf32x3_kernel<CF, 2>, &cfg) != cudaSuccess)
    n = 0;
  cudaGetLastError();
  grid = 2 * n;
  return grid;
}

template <class CF, int CL>
cudaError_t launch_variant(const void* Ahi, const void* Alo, const void* Bhi, const void* Blo, int64_t Kp,
                           int64_t kps, int64_t P, float* C, int64_t ldc, int64_t M, int64_t N, float alpha,
                           float beta, int* status, cudaStream_t st) {
  CUtensorMap mAhi, mAlo, mBhi, mBlo;
  // with CL = 2 each CTA copies half of the B tile (BN / 2 rows) into both CTAs
  if (!make_map<CF>(&mAhi, Ahi, M, Kp, kps, P, BM) || !make_map<CF>(&mAlo, Alo, M, Kp, kps, P, BM) ||
      !make_map<CF>(&mBhi, Bhi, N, Kp, kps, P, BN / CL) || !make_map<CF>(&mBlo, Blo, N, Kp, kps, P, BN / CL))
    return cudaErrorInvalidValue;
  static int sms = 0;
  static bool attr = false;
  if (!attr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(gemm_tf32x3_kernel<CF, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)CF::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int64_t tiles_m = (M + BM - 1) / BM, tiles_n = (N + BN - 1) / BN;
  if (CL == 1) {
    const int64_t tiles = tiles_m * tiles_n;
    const int grid = (int)(tiles < sms ? tiles : sms);
    gemm_tf32x3_kernel<CF, CL><<<grid, THREADS, CF::SMEM_BYTES, st>>>(mAhi, mAlo, mBhi, mBlo, C, ldc, (int)M, (int)N,
                                                                     (int)Kp, (int)P, alpha, beta, status);
    return cudaGetLastError();
  }
  int grid = cluster_grid<CF>();
  if (grid < 2) return cudaErrorInvalidConfiguration;
  const int64_t pairs = (tiles_m + 1) / 2 * tiles_n;
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
  return cudaLaunchKernelEx(&cfg, gemm_tf32x3_kernel<CF, CL>, mAhi, mAlo, mBhi, mBlo, C, ldc, (int)M, (int)N, (int)Kp,
                            (int)P, alpha, beta, status);
}

}  // namespace tc

// C[M][N] (ldc) = alpha * A B^T + beta * C with A, B in K panels (see tma_load): panel
// width Kp (kps = its stride), P panels, K = P Kp. P = 1, kps = ld is the plain row-major
// K-major layout. variant 0 (default): tf32, k-blocks of 16, 64-byte swizzle, 4 stages;
// variant 1: tf32, k-blocks of 32, 128-byte swizzle, 2 stages; variant 2: fp16 operands
// (hi/lo planes of __half), k-blocks of 32, 64-byte swizzle, 4 stages, 128-k promotion
// chunks (kps % 8 == 0); variant 3: as 2 with 64-k chunks; variant 4: as 2 with 256-k chunks;
// variant 5: as 2 in clusters of two CTAs sharing (multicasting) the B tile.
cudaError_t launch_gemm_tf32x3_v(const void* Ahi, const void* Alo, const void* Bhi, const void* Blo, int64_t Kp,
                                 int64_t kps, int64_t P, float* C, int64_t ldc, int64_t M, int64_t N, float alpha,
                                 float beta, int* status, cudaStream_t st, int variant) {
  using namespace tc;
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (Kp <= 0 || P <= 0 || M > 0x7fffffff || N > 0x7fffffff || Kp * P > 0x7fffffff) return cudaErrorInvalidValue;
  const bool f16 = variant >= 2 && variant <= 5;
  if ((kps & (f16 ? 7 : 3)) || kps < Kp) return cudaErrorInvalidValue;
  if ((((uintptr_t)Ahi) | ((uintptr_t)Alo) | ((uintptr_t)Bhi) | ((uintptr_t)Blo)) & 15) return cudaErrorInvalidValue;
  if (variant == 5) {
    // a device (or partition) that cannot co-schedule two-CTA clusters runs the same sums on
    // single CTAs
    if (cluster_grid<CfgF16>() >= 2)
      return launch_variant<CfgF16, 2>(Ahi, Alo, Bhi, Blo, Kp, kps, P, C, ldc, M, N, alpha, beta, status, st);
    return launch_variant<CfgF16, 1>(Ahi, Alo, Bhi, Blo, Kp, kps, P, C, ldc, M, N, alpha, beta, status, st);
  }
  if (variant == 4)
    return launch_variant<CfgF16L, 1>(Ahi, Alo, Bhi, Blo, Kp, kps, P, C, ldc, M, N, alpha, beta, status, st);
  if (variant == 3)
    return launch_variant<CfgF16S, 1>(Ahi, Alo, Bhi, Blo, Kp, kps, P, C, ldc, M, N, alpha, beta, status, st);
  if (variant == 2)
    return launch_variant<CfgF16, 1>(Ahi, Alo, Bhi, Blo, Kp, kps, P, C, ldc, M, N, alpha, beta, status, st);
  if (variant == 1)
    return launch_variant<CfgTF32W, 1>(Ahi, Alo, Bhi, Blo, Kp, kps, P, C, ldc, M, N, alpha, beta, status, st);
  return launch_variant<CfgTF32, 1>(Ahi, Alo, Bhi, Blo, Kp, kps, P, C, ldc, M, N, alpha, beta, status, st);
}

// Sets the kernels' shared-memory attributes and caches the SM count ahead of time, so no
// first launch does host-side set-up (which must not happen inside a stream capture).
void gemm_prepare() {
  using namespace tc;
  static bool done = false;
  if (done) return;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  cudaFuncSetAttribute(gemm_tf32x3_kernel<CfgTF32, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)CfgTF32::SMEM_BYTES);
  cudaFuncSetAttribute(gemm_tf32x3_kernel<CfgTF32W, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)CfgTF32W::SMEM_BYTES);
  cudaFuncSetAttribute(gemm_tf32x3_kernel<CfgF16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)CfgF16::SMEM_BYTES);
  cudaFuncSetAttribute(gemm_tf32x3_kernel<CfgF16S, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)CfgF16S::SMEM_BYTES);
  cudaFuncSetAttribute(gemm_tf32x3_kernel<CfgF16L, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)CfgF16L::SMEM_BYTES);
  cluster_grid<CfgF16>();   // sets the cluster kernel's attribute and caches its grid
  done = true;
}

cudaError_t launch_wait_selftest(int* status, unsigned long long limit_ns, cudaStream_t st) {
  tc::wait_selftest_kernel<<<1, 32, 0, st>>>(status, limit_ns);
  return cudaGetLastError();
}

cudaError_t launch_gemm_tf32x3(const float* Ahi, const float* Alo, const float* Bhi, const float* Blo, int64_t Kp,
                               int64_t kps, int64_t P, float* C, int64_t ldc, int64_t M, int64_t N, float alpha,
                               float beta, int* status, cudaStream_t st) {
  // plain tf32 entry: pipeline variant 0
  return launch_gemm_tf32x3_v(Ahi, Alo, Bhi, Blo, Kp, kps, P, C, ldc, M, N, alpha, beta, status, st, 0);
}

}  // namespace hotrg
