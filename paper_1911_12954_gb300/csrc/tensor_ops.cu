// tensor_ops.cu - memory-bound tensor kernels of the HOTRG step.
//
//  * ttm_short / ttm_pair_f16 / ttm_long / ttm_long4 kernels, ttm_kernel: contraction of one
//                     or two legs of a tensor with an isometry (the half contractions
//                     T x U^a x U^b that build the operands of the block-spin GEMM, and the
//                     closing contractions with U^c, Fig. 1C), writing any output leg order,
//                     optionally split into fp16 (or tf32) hi + lo planes for the tensor-core
//                     path; one, two or four fibres per thread, the generic ttm_kernel for
//                     shapes the fibre forms do not take.
//  * init_kernel    : the 4D Ising site tensors T and S (Fig. 1A) and ln c_0.
//  * sumsq/normalise: c = ||T'||_F in FP64, ln c / 2^k accumulated (ln Z / V), T' /= c.
//  * trace_kernel   : Tr T (each leg joined to its primed partner), FP64.
//  * xind_kernel    : the degeneracy indicator X = (Tr M)^2 / Tr(M M) of the coarse tensor.
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace hotrg {

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Exact 8-bit slices of x (|x| < 1, FP64): r <- 256 r, v = rint(r), r <- r - v, five times;
// every step is exact in FP64 and every v an integer fp16 holds exactly (|v| <= 256).
__device__ __forceinline__ void oz_store(__half* out, int64_t plane, int64_t o, double x) {
  double r = x;
#pragma unroll
  for (int i = 0; i < kOzSlices; ++i) {
    r *= 256.0;
    const double v = rint(r);
    out[o + i * plane] = __float2half_rn((float)v);
    r -= v;
  }
}

// Power-of-two scale of a split pass: from the operand's largest magnitude (a max pass of the
// same contraction wrote it to amax) or, without one, the fixed 2^14 of the fp16 planes.
template <int MODE>
__device__ __forceinline__ double split_scale(const unsigned* amax) {
  if (MODE == kTTMSplitF16) return amax ? ldexp(1.0, split_exponent(*amax, kF16Top)) : (double)kF16Scale;
  if (MODE == kTTMSplitOz) return ldexp(1.0, amax ? split_exponent(*amax, kOzTop) : kOzTop);
  return 1.0;
}

// Largest magnitude seen by the threads of a block, times mul, merged into *amax (bits of a
// non-negative float, rounded up, so that the recorded value bounds mul times every output).
__device__ __forceinline__ void merge_max(unsigned* amax, double m, float mul) {
  float f = __double2float_ru(m * (double)mul);
  for (int off = 16; off > 0; off >>= 1) f = fmaxf(f, __shfl_down_sync(0xffffffffu, f, off));
  if ((threadIdx.x & 31) == 0 && f > 0.f && amax) atomicMax(amax, __float_as_uint(f));
}

// Output pointer of batch element e: the split modes write fp16 planes, whose strides count
// fp16 values; the others count elements of the output type.
template <typename TO, int MODE>
__device__ __forceinline__ TO* elem_out(TO* p, int64_t off) {
  if (!p) return p;
  if (MODE == kTTMSplitF16 || MODE == kTTMSplitOz) return (TO*)((__half*)p + off);
  return p + off;
}

template <typename TI, typename TU, typename TO, int MODE>
__global__ void __launch_bounds__(256) ttm_kernel(const TI* __restrict__ in, const TU* __restrict__ U,
                                                  TO* __restrict__ out, TO* __restrict__ out_lo,
                                                  TTMArgs a) {
  using Acc = typename std::conditional<sizeof(TI) == 8, double, float>::type;
  const int64_t eb = blockIdx.y;               // batch element
  unsigned* amax = a.amax ? a.amax + eb * a.amax_bs : nullptr;
  const Acc sscale = (Acc)split_scale<MODE>(amax);
  Acc tmax = 0;                                // largest |output| of this thread (max modes), in the
                                               // accumulator type: no FP64 work for FP32 data
  in += eb * a.in_bs;
  if (U) U += eb * a.u_bs;
  out = elem_out<TO, MODE>(out, eb * a.out_bs);
  out_lo = elem_out<TO, MODE>(out_lo, eb * a.out_bs);
  const int outer_dims = a.rank - a.rin;
  for (int64_t row = blockIdx.x; row < a.outer; row += gridDim.x) {
    int64_t r = row, in0 = 0, u0 = 0, o0 = 0;
    for (int d = outer_dims - 1; d >= 0; --d) {
      const int64_t n = a.dims[d];
      const int64_t i = r % n;
      r /= n;
      in0 += i * a.in_st[d];
      u0 += i * a.u_st[d];
      o0 += i * a.out_st[d];
    }
    for (int64_t e = threadIdx.x; e < a.inner; e += blockDim.x) {
      uint32_t q = (uint32_t)e;
      int64_t i1 = in0, u1 = u0, o1 = o0;
      for (int d = a.rank - 1; d >= outer_dims; --d) {
        const uint32_t n = (uint32_t)a.dims[d];
        const uint32_t i = q % n;
        q /= n;
        i1 += (int64_t)i * a.in_st[d];
        u1 += (int64_t)i * a.u_st[d];
        o1 += (int64_t)i * a.out_st[d];
      }
      Acc acc = 0;
      if (U == nullptr) {
        acc = (Acc)in[i1];
      } else {
        for (int j1 = 0; j1 < a.J1; ++j1) {
          const int64_t ib = i1 + j1 * a.in_sj1;
          const int64_t ub = u1 + j1 * a.u_sj1;
          for (int j2 = 0; j2 < a.J2; ++j2)
            acc = fma((Acc)U[ub + j2 * a.u_sj2], (Acc)in[ib + j2 * a.in_sj2], acc);
        }
      }
      acc *= (Acc)a.alpha;
      if (MODE == kTTMMaxAbs || MODE == kTTMStoreMax) tmax = fmax(tmax, fabs(acc));
      if (MODE == kTTMMaxAbs) {
      } else if (MODE == kTTMSplitTF32) {
        const float v = (float)acc;
        const float hi = tf32_round(v);
        out[o1] = (TO)hi;
        out_lo[o1] = (TO)tf32_round(v - hi);
      } else if (MODE == kTTMSplitF16) {
        const float v = (float)(acc * sscale);
        const __half hi = __float2half_rn(v);
        ((__half*)out)[o1] = hi;
        ((__half*)out_lo)[o1] = __float2half_rn(v - __half2float(hi));
      } else if (MODE == kTTMSplitOz) {
        oz_store((__half*)out, (__half*)out_lo - (__half*)out, o1, (double)acc * (double)sscale);
      } else if (MODE == kTTMAccumulate) {
        out[o1] = (TO)(acc + (Acc)a.beta * (Acc)out[o1]);
      } else {
        out[o1] = (TO)acc;
      }
    }
  }
  if (MODE == kTTMMaxAbs || MODE == kTTMStoreMax) merge_max(amax, (double)tmax, a.amax_mul);   // every thread gets here
}

// ---------------------------------------------------------------------------- fiber form
// The same contraction organised by input fibre: out[f, r] = alpha sum_j U[j, r] in[f, j]
// with f the multi-index of the untouched legs, j = (j1, j2) the contracted legs and
// r = (r1, r2) the new ones. One thread per fibre; consecutive threads take consecutive
// fibres, so reads and writes along the innermost fibre leg are coalesced, every input
// element is read once and every output written once. U (and the output offsets of the
// new index) sit in shared memory, read by all lanes of a warp at once (broadcast).
struct FiberArgs {
  int nf;                       // fibre dims (outermost first)
  int fdims[kMaxRank];
  int64_t fin[kMaxRank], fout[kMaxRank];
  int64_t nfib;
  int R1, R2;                   // new-index dims
  int64_t ru1, ru2, ro1, ro2;   // their U-column and output strides
  int J1, J2;                   // contracted dims
  int64_t ji1, ji2, ju1, ju2;   // their input and U-row strides
  double alpha;
  int nb;                       // batch elements (blockIdx.y), strides as in TTMArgs
  int64_t in_bs, u_bs, out_bs;
  unsigned* amax;               // as in TTMArgs
  float amax_mul;
  int amax_bs;
};

constexpr int kShortJ = 16;     // longest contraction of the short form
constexpr int kShortRB = 32;    // accumulators per block of the new index (short form)
constexpr int kLongRMax = 16;   // longest new index of the long form

__device__ __forceinline__ void fiber_offsets(const FiberArgs& a, uint32_t f, int64_t& io, int64_t& oo) {
  io = 0;
  oo = 0;
#pragma unroll
  for (int d = kMaxRank - 1; d >= 0; --d) {   // unrolled: the parameter arrays are indexed statically
    if (d < a.nf) {
      const uint32_t n = (uint32_t)a.fdims[d];
      const uint32_t i = f % n;
      f /= n;
      io += (int64_t)i * a.fin[d];
      oo += (int64_t)i * a.fout[d];
    }
  }
}

// acc already carries the split pass's power-of-two scale (folded into U by the caller)
template <typename R, int MODE>
__device__ __forceinline__ void fiber_store(R* out, R* out_lo, int64_t o, R acc) {
  if (MODE == kTTMSplitTF32) {
    const float v = (float)acc;
    const float hi = tf32_round(v);
    out[o] = (R)hi;
    out_lo[o] = (R)tf32_round(v - hi);
  } else if (MODE == kTTMSplitF16) {
    // fp16 hi + lo of 2^e x: the pair keeps 22 significant bits
    const float v = (float)acc;
    const __half hi = __float2half_rn(v);
    ((__half*)out)[o] = hi;
    ((__half*)out_lo)[o] = __float2half_rn(v - __half2float(hi));
  } else if (MODE == kTTMSplitOz) {
    oz_store((__half*)out, (__half*)out_lo - (__half*)out, o, (double)acc);
  } else {
    out[o] = acc;
  }
}

// Short contractions (J <= 16: the half contractions with U^a and U^b). The J inputs of a
// fibre stay in registers; the new index is produced in blocks of 32 accumulators, each U
// row of a block read as 16-byte vectors, so an output costs about J FMAs plus its store.
template <typename R, int MODE>
__global__ void __launch_bounds__(256) ttm_short_kernel(const R* __restrict__ in, const R* __restrict__ U,
                                                        R* __restrict__ out, R* __restrict__ out_lo, FiberArgs a) {
  in += blockIdx.y * a.in_bs;                  // batch element blockIdx.y
  U += blockIdx.y * a.u_bs;
  out = elem_out<R, MODE>(out, blockIdx.y * a.out_bs);
  out_lo = elem_out<R, MODE>(out_lo, blockIdx.y * a.out_bs);
  extern __shared__ __align__(16) unsigned char fsm[];
  const int J = a.J1 * a.J2, Rn = a.R1 * a.R2;
  const int Rp = (Rn + kShortRB - 1) / kShortRB * kShortRB;
  R* Us = (R*)fsm;                                       // [J][Rp], zero past Rn
  int64_t* roff = (int64_t*)(fsm + (size_t)J * Rp * sizeof(R));   // [Rp] output offset of r
  int64_t* joff = roff + Rp;                             // [J] input offset of j
  // the split's power-of-two scale (exact) is folded into U
  unsigned* amax = a.amax ? a.amax + blockIdx.y * a.amax_bs : nullptr;
  const R uscale = (R)split_scale<MODE>(amax);
  R tmax = 0;                                            // max modes: largest |output| (type R)
  for (int e = threadIdx.x; e < J * Rp; e += blockDim.x) {
    const int j = e / Rp, r = e % Rp;
    R v = 0;
    if (r < Rn) {
      const int j1 = j / a.J2, j2 = j % a.J2, r1 = r / a.R2, r2 = r % a.R2;
      v = U[j1 * a.ju1 + j2 * a.ju2 + r1 * a.ru1 + r2 * a.ru2] * uscale;
    }
    Us[e] = v;
  }
  for (int r = threadIdx.x; r < Rp; r += blockDim.x) roff[r] = r < Rn ? (r / a.R2) * a.ro1 + (r % a.R2) * a.ro2 : 0;
  for (int j = threadIdx.x; j < J; j += blockDim.x) joff[j] = (j / a.J2) * a.ji1 + (j % a.J2) * a.ji2;
  __syncthreads();
  const R alpha = (R)a.alpha;
  const bool scaled = a.alpha != 1.0;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < a.nfib; f += (int64_t)gridDim.x * blockDim.x) {
    int64_t io, oo;
    fiber_offsets(a, (uint32_t)f, io, oo);
    R x[kShortJ];
#pragma unroll
    for (int j = 0; j < kShortJ; ++j) x[j] = j < J ? in[io + joff[j]] : (R)0;
    for (int rb = 0; rb < Rn; rb += kShortRB) {
      R acc[kShortRB];
#pragma unroll
      for (int i = 0; i < kShortRB; ++i) acc[i] = 0;
#pragma unroll
      for (int j = 0; j < kShortJ; ++j) {
        if (j < J) {
          const R* u = Us + j * Rp + rb;
          if constexpr (sizeof(R) == 4) {
#pragma unroll
            for (int i = 0; i < kShortRB; i += 4) {
              const float4 q = *(const float4*)(u + i);
              acc[i] = fma((R)q.x, x[j], acc[i]);
              acc[i + 1] = fma((R)q.y, x[j], acc[i + 1]);
              acc[i + 2] = fma((R)q.z, x[j], acc[i + 2]);
              acc[i + 3] = fma((R)q.w, x[j], acc[i + 3]);
            }
          } else {
#pragma unroll
            for (int i = 0; i < kShortRB; i += 2) {
              const double2 q = *(const double2*)(u + i);
              acc[i] = fma((R)q.x, x[j], acc[i]);
              acc[i + 1] = fma((R)q.y, x[j], acc[i + 1]);
            }
          }
        }
      }
#pragma unroll
      for (int i = 0; i < kShortRB; ++i)
        if (rb + i < Rn) {
          const R v = scaled ? acc[i] * alpha : acc[i];
          if (MODE == kTTMMaxAbs || MODE == kTTMStoreMax) tmax = fmax(tmax, fabs(v));
          if (MODE != kTTMMaxAbs) fiber_store<R, MODE>(out, out_lo, oo + roff[rb + i], v);
        }
    }
  }
  if (MODE == kTTMMaxAbs || MODE == kTTMStoreMax) merge_max(amax, (double)tmax, a.amax_mul);   // every thread gets here
}

// The fp16 split of a short contraction, two fibres per thread: when the innermost fibre leg
// has output stride 1 and an even extent (and every other output stride is even), fibres
// 2f and 2f + 1 are neighbours in the output, so their hi (and lo) values go out as one
// 4-byte half2: a warp store fills a 128-byte line and each U row read serves two fibres.
// MAXONLY: the max pass of the same contraction (kTTMMaxAbs: nothing written, the largest
// |output| times a.amax_mul merged into a.amax[element]).
template <typename R, bool MAXONLY>
__global__ void __launch_bounds__(256) ttm_pair_f16_kernel(const R* __restrict__ in, const R* __restrict__ U,
                                                           R* __restrict__ out, R* __restrict__ out_lo, FiberArgs a) {
  constexpr int RB = 16;
  unsigned* amax = a.amax ? a.amax + blockIdx.y * a.amax_bs : nullptr;
  float tmax = 0.f;                            // MAXONLY: largest |output| of this thread
  in += blockIdx.y * a.in_bs;                  // batch element blockIdx.y
  U += blockIdx.y * a.u_bs;
  out = elem_out<R, kTTMSplitF16>(out, blockIdx.y * a.out_bs);
  out_lo = elem_out<R, kTTMSplitF16>(out_lo, blockIdx.y * a.out_bs);
  extern __shared__ __align__(16) unsigned char fsm[];
  const int J = a.J1 * a.J2, Rn = a.R1 * a.R2;
  const int Rp = (Rn + kShortRB - 1) / kShortRB * kShortRB;
  R* Us = (R*)fsm;                                       // [J][Rp], zero past Rn, times the split scale
  int64_t* roff = (int64_t*)(fsm + (size_t)J * Rp * sizeof(R));
  int64_t* joff = roff + Rp;
  for (int e = threadIdx.x; e < J * Rp; e += blockDim.x) {
    const int j = e / Rp, r = e % Rp;
    R v = 0;
    if (r < Rn) {
      const int j1 = j / a.J2, j2 = j % a.J2, r1 = r / a.R2, r2 = r % a.R2;
      v = U[j1 * a.ju1 + j2 * a.ju2 + r1 * a.ru1 + r2 * a.ru2] * (R)(MAXONLY ? 1.0 : split_scale<kTTMSplitF16>(amax));
    }
    Us[e] = v;
  }
  for (int r = threadIdx.x; r < Rp; r += blockDim.x) roff[r] = r < Rn ? (r / a.R2) * a.ro1 + (r % a.R2) * a.ro2 : 0;
  for (int j = threadIdx.x; j < J; j += blockDim.x) joff[j] = (j / a.J2) * a.ji1 + (j % a.J2) * a.ji2;
  __syncthreads();
  const int64_t step_in = a.fin[a.nf - 1];     // input offset from fibre 2f to 2f + 1
  const int64_t npair = a.nfib / 2;
  __half* hi_out = (__half*)out;
  __half* lo_out = (__half*)out_lo;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < npair; f += (int64_t)gridDim.x * blockDim.x) {
    int64_t io, oo;
    fiber_offsets(a, (uint32_t)(2 * f), io, oo);   // oo is even: a 4-byte aligned half2 slot
    R x0[kShortJ], x1[kShortJ];
#pragma unroll
    for (int j = 0; j < kShortJ; ++j) {
      x0[j] = j < J ? in[io + joff[j]] : (R)0;
      x1[j] = j < J ? in[io + step_in + joff[j]] : (R)0;
    }
    for (int rb = 0; rb < Rn; rb += RB) {
      R a0[RB], a1[RB];
#pragma unroll
      for (int i = 0; i < RB; ++i) a0[i] = a1[i] = 0;
#pragma unroll
      for (int j = 0; j < kShortJ; ++j) {
        if (j < J) {
          const R* u = Us + j * Rp + rb;
#pragma unroll
          for (int i = 0; i < RB; i += 4) {
            const float4 q = *(const float4*)(u + i);
            a0[i] = fmaf(q.x, x0[j], a0[i]);
            a0[i + 1] = fmaf(q.y, x0[j], a0[i + 1]);
            a0[i + 2] = fmaf(q.z, x0[j], a0[i + 2]);
            a0[i + 3] = fmaf(q.w, x0[j], a0[i + 3]);
            a1[i] = fmaf(q.x, x1[j], a1[i]);
            a1[i + 1] = fmaf(q.y, x1[j], a1[i + 1]);
            a1[i + 2] = fmaf(q.z, x1[j], a1[i + 2]);
            a1[i + 3] = fmaf(q.w, x1[j], a1[i + 3]);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        if (MAXONLY) {
          if (rb + i < Rn) tmax = fmaxf(tmax, fmaxf(fabsf(a0[i]), fabsf(a1[i])));
        } else if (rb + i < Rn) {
          const int64_t o = oo + roff[rb + i];
          const __half h0 = __float2half_rn(a0[i]), h1 = __float2half_rn(a1[i]);
          const __half l0 = __float2half_rn(a0[i] - __half2float(h0));
          const __half l1 = __float2half_rn(a1[i] - __half2float(h1));
          *(__half2*)(hi_out + o) = __halves2half2(h0, h1);
          *(__half2*)(lo_out + o) = __halves2half2(l0, l1);
        }
      }
    }
  }
  if (MAXONLY) merge_max(amax, (double)tmax, a.amax_mul);   // every thread of the block gets here
}

// Long contractions (J > 16 with a short new index, Rn <= 16: the closing passes with U^c).
// The outputs of a fibre stay in RB registers; its J inputs stream through in (j1, j2)
// order, eight loads issued before their FMAs so that several are in flight per thread.
template <typename R, int RB>
__global__ void __launch_bounds__(256) ttm_long_kernel(const R* __restrict__ in, const R* __restrict__ U,
                                                       R* __restrict__ out, FiberArgs a) {
  in += blockIdx.y * a.in_bs;                  // batch element blockIdx.y
  U += blockIdx.y * a.u_bs;
  out += blockIdx.y * a.out_bs;
  extern __shared__ __align__(16) unsigned char fsm[];
  const int J = a.J1 * a.J2, Rn = a.R1 * a.R2;
  R* Us = (R*)fsm;                                       // [J][RB], zero past Rn
  int64_t* roff = (int64_t*)(fsm + (size_t)J * RB * sizeof(R));   // [RB]
  for (int e = threadIdx.x; e < J * RB; e += blockDim.x) {
    const int j = e / RB, r = e % RB;
    R v = 0;
    if (r < Rn) {
      const int j1 = j / a.J2, j2 = j % a.J2, r1 = r / a.R2, r2 = r % a.R2;
      v = U[j1 * a.ju1 + j2 * a.ju2 + r1 * a.ru1 + r2 * a.ru2];
    }
    Us[e] = v;
  }
  for (int r = threadIdx.x; r < RB; r += blockDim.x) roff[r] = r < Rn ? (r / a.R2) * a.ro1 + (r % a.R2) * a.ro2 : 0;
  __syncthreads();
  const R alpha = (R)a.alpha;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < a.nfib; f += (int64_t)gridDim.x * blockDim.x) {
    int64_t io, oo;
    fiber_offsets(a, (uint32_t)f, io, oo);
    R acc[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[r] = 0;
    for (int j1 = 0; j1 < a.J1; ++j1) {
      const R* src = in + io + j1 * a.ji1;
      const R* u = Us + (size_t)j1 * a.J2 * RB;
      int j2 = 0;
      for (; j2 + 8 <= a.J2; j2 += 8) {
        R xv[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) xv[q] = src[(int64_t)(j2 + q) * a.ji2];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const R* uq = u + (j2 + q) * RB;
#pragma unroll
          for (int r = 0; r < RB; ++r) acc[r] = fma(uq[r], xv[q], acc[r]);
        }
      }
      for (; j2 < a.J2; ++j2) {
        const R xv = src[(int64_t)j2 * a.ji2];
        const R* uq = u + j2 * RB;
#pragma unroll
        for (int r = 0; r < RB; ++r) acc[r] = fma(uq[r], xv, acc[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < RB; ++r)
      if (r < Rn) out[oo + roff[r]] = acc[r] * alpha;
  }
}

// The long form four fibres per thread: when the innermost fibre leg has input and output
// stride 1 and an extent divisible by 4 (every other stride a multiple of 4), fibres 4f..4f+3
// are neighbours in both tensors, so each contracted index is one 16-byte load and each
// output one 16-byte store.
template <int RB>
__global__ void __launch_bounds__(256) ttm_long4_kernel(const float* __restrict__ in, const float* __restrict__ U,
                                                        float* __restrict__ out, FiberArgs a) {
  in += blockIdx.y * a.in_bs;                  // batch element blockIdx.y
  U += blockIdx.y * a.u_bs;
  out += blockIdx.y * a.out_bs;
  extern __shared__ __align__(16) unsigned char fsm[];
  const int J = a.J1 * a.J2, Rn = a.R1 * a.R2;
  float* Us = (float*)fsm;                               // [J][RB], zero past Rn
  int64_t* roff = (int64_t*)(fsm + (size_t)J * RB * sizeof(float));
  for (int e = threadIdx.x; e < J * RB; e += blockDim.x) {
    const int j = e / RB, r = e % RB;
    float v = 0;
    if (r < Rn) {
      const int j1 = j / a.J2, j2 = j % a.J2, r1 = r / a.R2, r2 = r % a.R2;
      v = U[j1 * a.ju1 + j2 * a.ju2 + r1 * a.ru1 + r2 * a.ru2];
    }
    Us[e] = v;
  }
  for (int r = threadIdx.x; r < RB; r += blockDim.x) roff[r] = r < Rn ? (r / a.R2) * a.ro1 + (r % a.R2) * a.ro2 : 0;
  __syncthreads();
  const float alpha = (float)a.alpha;
  const int64_t nquad = a.nfib / 4;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nquad; f += (int64_t)gridDim.x * blockDim.x) {
    int64_t io, oo;
    fiber_offsets(a, (uint32_t)(4 * f), io, oo);   // both multiples of 4: 16-byte aligned
    float4 acc[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int j1 = 0; j1 < a.J1; ++j1) {
      const float* src = in + io + j1 * a.ji1;
      const float* u = Us + (size_t)j1 * a.J2 * RB;
      int j2 = 0;
      for (; j2 + 4 <= a.J2; j2 += 4) {
        float4 xv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) xv[q] = *(const float4*)(src + (int64_t)(j2 + q) * a.ji2);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float* uq = u + (j2 + q) * RB;
#pragma unroll
          for (int r = 0; r < RB; ++r) {
            const float w = uq[r];
            acc[r].x = fmaf(w, xv[q].x, acc[r].x);
            acc[r].y = fmaf(w, xv[q].y, acc[r].y);
            acc[r].z = fmaf(w, xv[q].z, acc[r].z);
            acc[r].w = fmaf(w, xv[q].w, acc[r].w);
          }
        }
      }
      for (; j2 < a.J2; ++j2) {
        const float4 xv = *(const float4*)(src + (int64_t)j2 * a.ji2);
        const float* uq = u + j2 * RB;
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          const float w = uq[r];
          acc[r].x = fmaf(w, xv.x, acc[r].x);
          acc[r].y = fmaf(w, xv.y, acc[r].y);
          acc[r].z = fmaf(w, xv.z, acc[r].z);
          acc[r].w = fmaf(w, xv.w, acc[r].w);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RB; ++r)
      if (r < Rn)
        *(float4*)(out + oo + roff[r]) =
            make_float4(acc[r].x * alpha, acc[r].y * alpha, acc[r].z * alpha, acc[r].w * alpha);
  }
}

// Fibres 4f..4f+3 are neighbours with 16-byte aligned starts in input and output.
inline bool quadable(const FiberArgs& f, const void* in, const void* out) {
  if (f.nf < 1 || f.fin[f.nf - 1] != 1 || f.fout[f.nf - 1] != 1 || (f.fdims[f.nf - 1] & 3)) return false;
  for (int d = 0; d < f.nf - 1; ++d)
    if ((f.fin[d] & 3) || (f.fout[d] & 3)) return false;
  if ((f.ji1 & 3) || (f.ji2 & 3) || (f.ro1 & 3) || (f.ro2 & 3)) return false;
  if (f.nb > 1 && ((f.in_bs & 3) || (f.out_bs & 3))) return false;     // every element 16-byte aligned
  return ((((uintptr_t)in) | ((uintptr_t)out)) & 15) == 0;
}

inline size_t short_smem(int J, int Rn, size_t rsize) {
  const size_t Rp = (size_t)(Rn + kShortRB - 1) / kShortRB * kShortRB;
  return (size_t)J * Rp * rsize + (Rp + (size_t)J) * sizeof(int64_t);
}
inline int long_rb(int Rn) { return Rn <= 8 ? 8 : kLongRMax; }
inline size_t long_smem(int J, int Rn, size_t rsize) {
  return (size_t)J * long_rb(Rn) * rsize + (size_t)long_rb(Rn) * sizeof(int64_t);
}
constexpr size_t kFiberSmemMax = 48 * 1024;

// Converts a TTMArgs into the fibre form when it fits; false otherwise.
bool to_fiber(const TTMArgs& a, size_t rsize, FiberArgs& f) {
  f = FiberArgs{};
  int nr = 0;
  f.R1 = f.R2 = 1;
  f.ru1 = f.ru2 = f.ro1 = f.ro2 = 0;
  f.nfib = 1;
  for (int i = 0; i < a.rank; ++i) {
    if (a.u_st[i] != 0) {
      if (a.in_st[i] != 0 || nr == 2) return false;
      if (nr == 0) {
        f.R1 = (int)a.dims[i];
        f.ru1 = a.u_st[i];
        f.ro1 = a.out_st[i];
      } else {
        f.R2 = (int)a.dims[i];
        f.ru2 = a.u_st[i];
        f.ro2 = a.out_st[i];
      }
      ++nr;
    } else {
      f.fdims[f.nf] = (int)a.dims[i];
      f.fin[f.nf] = a.in_st[i];
      f.fout[f.nf] = a.out_st[i];
      f.nfib *= a.dims[i];
      ++f.nf;
    }
  }
  f.J1 = a.J1;
  f.J2 = a.J2;
  f.ji1 = a.in_sj1;
  f.ji2 = a.in_sj2;
  f.ju1 = a.u_sj1;
  f.ju2 = a.u_sj2;
  f.alpha = a.alpha;
  f.nb = a.nb;
  f.in_bs = a.in_bs;
  f.u_bs = a.u_bs;
  f.out_bs = a.out_bs;
  f.amax = a.amax;
  f.amax_mul = a.amax_mul;
  f.amax_bs = a.amax_bs;
  const int J = a.J1 * a.J2, Rn = f.R1 * f.R2;
  if (f.nf == 0 || f.nfib > 0x7fffffffLL) return false;   // fibre index decoded in 32 bits
  if (J <= kShortJ) return Rn <= 256 && short_smem(J, Rn, rsize) <= kFiberSmemMax;
  return Rn <= kLongRMax && long_smem(J, Rn, rsize) <= kFiberSmemMax;
}

// Fibres 2f, 2f + 1 share a 4-byte aligned half2 slot: innermost fibre leg of even extent and
// output stride 1, every other output stride (fibre legs and new index) even, planes 4-byte aligned.
inline bool pairable(const FiberArgs& f, const void* out, const void* out_lo) {
  if (f.nf < 1 || f.fout[f.nf - 1] != 1 || (f.fdims[f.nf - 1] & 1)) return false;
  for (int d = 0; d < f.nf - 1; ++d)
    if (f.fout[d] & 1) return false;
  if ((f.ro1 & 1) || (f.ro2 & 1)) return false;
  if (f.nb > 1 && (f.out_bs & 1)) return false;                       // every element's half2 slots aligned
  return ((((uintptr_t)out) | ((uintptr_t)out_lo)) & 3) == 0;
}

template <typename R>
cudaError_t launch_fiber(const R* in, const R* U, R* out, R* out_lo, const FiberArgs& f, int mode, cudaStream_t st) {
  const int J = f.J1 * f.J2, Rn = f.R1 * f.R2;
  // blocks per batch element: the whole launch stays near 16 blocks per SM
  const int64_t cap = std::max<int64_t>(8, 152 * 16 / f.nb);
  int64_t blocks = (f.nfib + 255) / 256;
  if (blocks > cap) blocks = cap;
  const dim3 g((unsigned)blocks, f.nb);
  if (J > kShortJ) {               // long form (plain store only)
    if (mode != kTTMStore) return cudaErrorInvalidValue;
    const size_t smem = long_smem(J, Rn, sizeof(R));
    if constexpr (sizeof(R) == 4) {
      if (quadable(f, in, out)) {
        int64_t qblocks = (f.nfib / 4 + 255) / 256;
        if (qblocks > cap) qblocks = cap;
        const dim3 gq((unsigned)qblocks, f.nb);
        if (long_rb(Rn) == 8) ttm_long4_kernel<8><<<gq, 256, smem, st>>>(in, U, out, f);
        else ttm_long4_kernel<kLongRMax><<<gq, 256, smem, st>>>(in, U, out, f);
        return cudaGetLastError();
      }
    }
    if (long_rb(Rn) == 8) ttm_long_kernel<R, 8><<<g, 256, smem, st>>>(in, U, out, f);
    else ttm_long_kernel<R, kLongRMax><<<g, 256, smem, st>>>(in, U, out, f);
    return cudaGetLastError();
  }
  const size_t smem = short_smem(J, Rn, sizeof(R));
  if constexpr (sizeof(R) == 4) {
    // the fp16 split, and its max pass, two fibres per thread (the max pass writes nothing:
    // the split's output layout decides, so that both passes take the same kernel)
    if ((mode == kTTMSplitF16 || (mode == kTTMMaxAbs && f.amax)) && f.alpha == 1.0 && pairable(f, out, out_lo)) {
      int64_t pblocks = (f.nfib / 2 + 255) / 256;
      if (pblocks > cap) pblocks = cap;
      const dim3 gp((unsigned)pblocks, f.nb);
      if (mode == kTTMMaxAbs) ttm_pair_f16_kernel<R, true><<<gp, 256, smem, st>>>(in, U, out, out_lo, f);
      else ttm_pair_f16_kernel<R, false><<<gp, 256, smem, st>>>(in, U, out, out_lo, f);
      return cudaGetLastError();
    }
  }
  if (mode == kTTMSplitTF32) ttm_short_kernel<R, kTTMSplitTF32><<<g, 256, smem, st>>>(in, U, out, out_lo, f);
  else if (mode == kTTMSplitF16) ttm_short_kernel<R, kTTMSplitF16><<<g, 256, smem, st>>>(in, U, out, out_lo, f);
  else if (mode == kTTMSplitOz) ttm_short_kernel<R, kTTMSplitOz><<<g, 256, smem, st>>>(in, U, out, out_lo, f);
  else if (mode == kTTMMaxAbs) ttm_short_kernel<R, kTTMMaxAbs><<<g, 256, smem, st>>>(in, U, out, out_lo, f);
  else if (mode == kTTMStoreMax) ttm_short_kernel<R, kTTMStoreMax><<<g, 256, smem, st>>>(in, U, out, out_lo, f);
  else ttm_short_kernel<R, kTTMStore><<<g, 256, smem, st>>>(in, U, out, out_lo, f);
  return cudaGetLastError();
}

template <typename TI, typename TU, typename TO>
cudaError_t launch_ttm(const TI* in, const TU* U, TO* out, TO* out_lo, const TTMArgs& a, int mode,
                       cudaStream_t st) {
  if (a.outer <= 0 || a.inner <= 0) return cudaSuccess;
  if (a.inner > 0x7fffffffLL) return cudaErrorInvalidValue;
  if constexpr (std::is_same<TI, TU>::value && std::is_same<TI, TO>::value) {
    FiberArgs f;
    if (U != nullptr && mode != kTTMAccumulate && to_fiber(a, sizeof(TI), f) &&
        (f.J1 * f.J2 <= kShortJ || mode == kTTMStore))
      return launch_fiber<TI>(in, U, out, out_lo, f, mode, st);
  }
  if (a.nb < 1) return cudaErrorInvalidValue;
  const int64_t bcap = std::max<int64_t>(8, 152 * 64 / a.nb);
  const dim3 blocks((unsigned)(a.outer < bcap ? a.outer : bcap), a.nb);
  const int threads = a.inner >= 256 ? 256 : (int)((a.inner + 31) / 32 * 32);
  switch (mode) {
    case kTTMStore:
      ttm_kernel<TI, TU, TO, kTTMStore><<<blocks, threads, 0, st>>>(in, U, out, out_lo, a);
      break;
    case kTTMSplitTF32:
      ttm_kernel<TI, TU, TO, kTTMSplitTF32><<<blocks, threads, 0, st>>>(in, U, out, out_lo, a);
      break;
    case kTTMSplitF16:
      ttm_kernel<TI, TU, TO, kTTMSplitF16><<<blocks, threads, 0, st>>>(in, U, out, out_lo, a);
      break;
    case kTTMSplitOz:
      ttm_kernel<TI, TU, TO, kTTMSplitOz><<<blocks, threads, 0, st>>>(in, U, out, out_lo, a);
      break;
    case kTTMMaxAbs:
      ttm_kernel<TI, TU, TO, kTTMMaxAbs><<<blocks, threads, 0, st>>>(in, U, out, out_lo, a);
      break;
    case kTTMStoreMax:
      ttm_kernel<TI, TU, TO, kTTMStoreMax><<<blocks, threads, 0, st>>>(in, U, out, out_lo, a);
      break;
    default:
      ttm_kernel<TI, TU, TO, kTTMAccumulate><<<blocks, threads, 0, st>>>(in, U, out, out_lo, a);
  }
  return cudaGetLastError();
}

template cudaError_t launch_ttm<double, double, double>(const double*, const double*, double*, double*,
                                                        const TTMArgs&, int, cudaStream_t);
template cudaError_t launch_ttm<float, float, float>(const float*, const float*, float*, float*,
                                                     const TTMArgs&, int, cudaStream_t);
template cudaError_t launch_ttm<double, double, float>(const double*, const double*, float*, float*,
                                                       const TTMArgs&, int, cudaStream_t);
template cudaError_t launch_ttm<float, double, double>(const float*, const double*, double*, double*,
                                                       const TTMArgs&, int, cudaStream_t);

// ---------------------------------------------------------------------------- site tensors
// T[i1..i8] = sum_s w_s prod_j W[s][i_j], S = sum_s sigma_s w_s prod_j W[s][i_j];
// w_s = exp(beta h sigma_s), sigma = (+1, -1), W as in Fig. 1A's tensor network of the
// Ising model. One block per batch element, 256 threads = 256 entries. Writes the
// normalised tensors and ln c_0 = ln ||T||_F.
template <typename R>
__global__ void __launch_bounds__(256) init_kernel(const double* __restrict__ beta, const double* __restrict__ h,
                                                   R* T, R* S, int64_t slot, double* lnz_acc) {
  const int b = blockIdx.x;
  const double be = beta[b], hb = h[b];
  const double ch = sqrt(cosh(be)), sh = sqrt(sinh(be));
  const int i = threadIdx.x;
  double t = 0, s = 0;
  for (int sp = 0; sp < 2; ++sp) {
    const double sig = sp == 0 ? 1.0 : -1.0;
    const double w = exp(be * hb * sig);
    double p = 1.0;
    for (int leg = 0; leg < 8; ++leg) {
      const int bit = (i >> (7 - leg)) & 1;          // leg 0 is the slowest index
      p *= bit == 0 ? ch : sig * sh;
    }
    t += w * p;
    s += sig * w * p;
  }
  __shared__ double red[256];
  red[i] = t * t;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (i < off) red[i] += red[i + off];
    __syncthreads();
  }
  const double c = sqrt(red[0]);
  T[b * slot + i] = (R)(t / c);
  if (S != nullptr) S[b * slot + i] = (R)(s / c);
  if (i == 0) lnz_acc[b] = log(c);
}

template <typename R>
cudaError_t launch_init(const double* beta, const double* h, R* T, R* S, int64_t slot, double* lnz_acc,
                        int batch, cudaStream_t st) {
  init_kernel<R><<<batch, 256, 0, st>>>(beta, h, T, S, slot, lnz_acc);
  return cudaGetLastError();
}
template cudaError_t launch_init<double>(const double*, const double*, double*, double*, int64_t, double*,
                                         int, cudaStream_t);
template cudaError_t launch_init<float>(const double*, const double*, float*, float*, int64_t, double*, int,
                                        cudaStream_t);

// ---------------------------------------------------------------------------- norm
// Pass 1: each block writes the FP64 sum of squares of its grid-stride share.
constexpr int kNormBlocks = kNormPartials;

template <typename R>
__global__ void __launch_bounds__(256) sumsq_kernel(const R* __restrict__ x, int64_t n, int64_t xstride,
                                                    double* partial) {
  x += blockIdx.y * xstride;                   // batch element blockIdx.y
  partial += blockIdx.y * gridDim.x;
  double acc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)x[i];
    acc = fma(v, v, acc);
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  __shared__ double w[8];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int j = 0; j < 8; ++j) s += w[j];
    partial[blockIdx.x] = s;
  }
}

// Pass 2 (one block): c = sqrt(sum), ln Z accumulator += ln(c) / 2^(k+1), record ln c in
// rec_b[k] where k = *step is the number of steps done before this one (read on the
// device, so a captured step replays correctly at any k).
__global__ void norm_finish_kernel(const double* __restrict__ partial, int np, const int* __restrict__ step,
                                   double* c_out, double* lnz_acc, DevRecord* rec_b, int* status) {
  // batch element blockIdx.x
  partial += blockIdx.x * np;
  c_out += blockIdx.x;
  lnz_acc += blockIdx.x;
  rec_b += blockIdx.x * kMaxSteps;
  __shared__ double red[256];
  double s = 0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += partial[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int k = *step;
    const double c = sqrt(red[0]);
    double* ln_c_rec = &rec_b[k < kMaxSteps ? k : kMaxSteps - 1].ln_c;
    if (!(c > 0.0) || !isfinite(c)) {
      atomicAdd(&status[kStNonFinite], 1);
      *c_out = 1.0;
      *ln_c_rec = nan("");
    } else {
      *c_out = c;
      *lnz_acc += log(c) * ldexp(1.0, -(k + 1));
      *ln_c_rec = log(c);
    }
  }
}

// ---------------------------------------------------------------------------- split statistics
__global__ void __launch_bounds__(256) plane_stats_kernel(const __half* __restrict__ p, int64_t nrows, int64_t Kp,
                                                          int64_t kps, unsigned long long* out) {
  unsigned long long nz = 0, ns = 0;
  unsigned mx = 0;
  const int64_t n = nrows * Kp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / Kp;
    const unsigned a = __half_as_ushort(p[r * kps + (i - r * Kp)]) & 0x7fffu;   // magnitude bits
    nz += a == 0u;
    ns += (a != 0u && a < 0x0400u);
    mx = max(mx, a);
  }
  for (int off = 16; off > 0; off >>= 1) {
    nz += __shfl_down_sync(0xffffffffu, nz, off);
    ns += __shfl_down_sync(0xffffffffu, ns, off);
    mx = max(mx, __shfl_down_sync(0xffffffffu, mx, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[0], nz);
    atomicAdd(&out[1], ns);
    atomicMax(&out[2], (unsigned long long)mx);
  }
}

cudaError_t launch_plane_stats(const void* plane, int64_t nrows, int64_t Kp, int64_t kps, unsigned long long* out,
                               cudaStream_t st) {
  if (nrows <= 0 || Kp <= 0) return cudaSuccess;
  if (Kp > kps) return cudaErrorInvalidValue;
  int64_t blocks = (nrows * Kp + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  plane_stats_kernel<<<(unsigned)blocks, 256, 0, st>>>((const __half*)plane, nrows, Kp, kps, out);
  return cudaGetLastError();
}

// Advances the device step counter at the end of a step.
__global__ void step_end_kernel(int* step) {
  if (threadIdx.x == 0) *step += 1;
}

cudaError_t launch_step_end(int* step, cudaStream_t st) {
  step_end_kernel<<<1, 32, 0, st>>>(step);
  return cudaGetLastError();
}

template <typename R>
__global__ void __launch_bounds__(256) scale_kernel(R* __restrict__ x, int64_t n, int64_t xstride,
                                                    const double* __restrict__ c) {
  x += blockIdx.y * xstride;                   // batch element blockIdx.y
  const R inv = (R)(1.0 / c[blockIdx.y]);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= inv;
}

template <typename R>
cudaError_t launch_norm(const R* x, int64_t n, int nb, int64_t xstride, double* partial, const int* step,
                        double* c_out, double* lnz_acc, DevRecord* rec_b, int* status, cudaStream_t st) {
  sumsq_kernel<R><<<dim3(kNormBlocks, nb), 256, 0, st>>>(x, n, xstride, partial);
  norm_finish_kernel<<<nb, 256, 0, st>>>(partial, kNormBlocks, step, c_out, lnz_acc, rec_b, status);
  return cudaGetLastError();
}
template <typename R>
cudaError_t launch_scale(R* x, int64_t n, int nb, int64_t xstride, const double* c, cudaStream_t st) {
  if (n <= 0 || nb <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  scale_kernel<R><<<dim3((unsigned)blocks, nb), 256, 0, st>>>(x, n, xstride, c);
  return cudaGetLastError();
}
template cudaError_t launch_norm<double>(const double*, int64_t, int, int64_t, double*, const int*, double*, double*,
                                         DevRecord*, int*, cudaStream_t);
template cudaError_t launch_norm<float>(const float*, int64_t, int, int64_t, double*, const int*, double*, double*,
                                        DevRecord*, int*, cudaStream_t);
template cudaError_t launch_scale<double>(double*, int64_t, int, int64_t, const double*, cudaStream_t);
template cudaError_t launch_scale<float>(float*, int64_t, int, int64_t, const double*, cudaStream_t);

// ---------------------------------------------------------------------------- trace
// Tr T = sum_{x,y,z,t} T[x,x,y,y,z,z,t,t] in FP64; one block per batch element.
template <typename R>
__global__ void __launch_bounds__(256) trace_kernel(const R* __restrict__ T, int64_t slot, int Dx, int Dy, int Dz,
                                                    int Dt, double* out) {
  const R* t = T + blockIdx.x * slot;
  // strides of the primed legs; the unprimed leg of direction nu has D_nu times that
  const int64_t szp = (int64_t)Dt * Dt, syp = (int64_t)Dz * Dz * szp, sxp = (int64_t)Dy * Dy * syp;
  const int64_t n = (int64_t)Dx * Dy * Dz * Dt;
  double acc = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    int64_t r = i;
    const int64_t it = r % Dt; r /= Dt;
    const int64_t iz = r % Dz; r /= Dz;
    const int64_t iy = r % Dy; r /= Dy;
    const int64_t ix = r;
    const int64_t off = ix * (Dx + 1) * sxp + iy * (Dy + 1) * syp + iz * (Dz + 1) * szp + it * (Dt + 1);
    acc += (double)t[off];
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

template <typename R>
cudaError_t launch_trace(const R* T, int64_t slot, const int* dims, int batch, double* out, cudaStream_t st) {
  trace_kernel<R><<<batch, 256, 0, st>>>(T, slot, dims[0], dims[1], dims[2], dims[3], out);
  return cudaGetLastError();
}
template cudaError_t launch_trace<double>(const double*, int64_t, const int*, int, double*, cudaStream_t);
template cudaError_t launch_trace<float>(const float*, int64_t, const int*, int, double*, cudaStream_t);

// ---------------------------------------------------------------------------- X indicator
// Degeneracy indicator of the coarse tensor (Sec. 3.1 locates T_c with it): M[i][j] = T with
// leg nu = i, leg nu' = j and each other direction traced, X = (Tr M)^2 / Tr(M M). One block
// per batch element; one warp per entry of M (lanes stride over the traced directions),
// FP64 sums.
template <typename R>
__global__ void __launch_bounds__(256) xind_kernel(const R* __restrict__ T, int64_t slot, int Dx, int Dy, int Dz,
                                                   int Dt, int nu, double* out) {
  const R* t = T + blockIdx.x * slot;
  const int D[4] = {Dx, Dy, Dz, Dt};
  int64_t st[8], s = 1;
  for (int leg = 7; leg >= 0; --leg) {
    st[leg] = s;
    s *= D[leg / 2];
  }
  int od[3];
  int64_t ost[3];   // diagonal stride (leg + its primed partner) of the traced directions
  int q = 0;
  for (int n = 0; n < 4; ++n)
    if (n != nu) {
      od[q] = D[n];
      ost[q] = st[2 * n] + st[2 * n + 1];
      ++q;
    }
  const int Dn = D[nu];
  const int64_t nrest = (int64_t)od[0] * od[1] * od[2];
  __shared__ double M[kMaxLeg * kMaxLeg];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int e = w; e < Dn * Dn; e += nw) {
    const int i = e / Dn, j = e % Dn;
    const int64_t base = i * st[2 * nu] + j * st[2 * nu + 1];
    double acc = 0;
    for (int64_t r = lane; r < nrest; r += 32) {
      const int64_t r2 = r % od[2], r1 = (r / od[2]) % od[1], r0 = r / ((int64_t)od[2] * od[1]);
      acc += (double)t[base + r0 * ost[0] + r1 * ost[1] + r2 * ost[2]];
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) M[e] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0, tr2 = 0;
    for (int i = 0; i < Dn; ++i) {
      tr += M[i * Dn + i];
      for (int j = 0; j < Dn; ++j) tr2 += M[i * Dn + j] * M[j * Dn + i];
    }
    out[blockIdx.x] = tr * tr / tr2;
  }
}

template <typename R>
cudaError_t launch_xind(const R* T, int64_t slot, const int* dims, int batch, int nu, double* out, cudaStream_t st) {
  if (nu < 0 || nu > 3 || dims[nu] > kMaxLeg) return cudaErrorInvalidValue;
  xind_kernel<R><<<batch, 256, 0, st>>>(T, slot, dims[0], dims[1], dims[2], dims[3], nu, out);
  return cudaGetLastError();
}
template cudaError_t launch_xind<double>(const double*, int64_t, const int*, int, int, double*, cudaStream_t);
template cudaError_t launch_xind<float>(const float*, int64_t, const int*, int, int, double*, cudaStream_t);

}  // namespace hotrg
