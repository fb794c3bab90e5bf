// gram.cu - Gram (environment) matrices of the HOSVD of two adjacent tensors (Fig. 1B).
//
// For a step along mu and a transverse leg l (nu or nu'), the Gram matrix of the pair
// tensor M = T1 -mu- T2 on its fused (T1.l, T2.l) leg factorises into two half-Grams of
// the single tensor, each a symmetric rank-K update with rows (l, mu-leg):
//   A1[(a,k),(b,k')] = sum_rest T[a@l, k@mu', rest] T[b@l, k'@mu', rest]
//   A2[(a,k),(b,k')] = sum_rest T[a@l, k@mu , rest] T[b@l, k'@mu , rest]
//   G[(a1 a2),(b1 b2)] = sum_{k,k'} A1[(a1,k),(b1,k')] A2[(a2,k),(b2,k')].
// gram_kernel computes 64x64 tiles of one half-Gram over one chunk of the summed index
// (split-K: K = D^6 is long, R = D_l D_mu is short), products in the storage precision
// summed per 32-term slice with FMA, then the slice sums accumulated: in FP64 for FP64
// tensors, for FP32 ones as an unevaluated pair of floats (hi + lo, Knuth's TwoSum) that
// adds them without a further rounding and without the FP64 pipe (a few FP64 operations
// per clock per SM on this chip, against 128 FP32 FMAs). For FP32 tensors each slice sum
// is therefore rounded once in FP32 (2^-24 of the slice's magnitude), and a Gram entry's
// error is bounded by 2^-24 times the sum of its slices' magnitudes, whatever K is, where
// one FP32 running sum over K = D^6 terms would add an error that grows with K.
// gram_reduce adds the chunks of every job in a fixed order (deterministic, one launch);
// gram_merge forms G in FP64.
#include <type_traits>

#include "common.cuh"

namespace hotrg {

constexpr int kGT = 64;   // output tile
constexpr int kGK = 32;   // k slice held in shared memory

// hi + lo += x exactly up to the rounding of lo (TwoSum of hi and x).
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float t = hi + x;
  const float bp = t - hi;
  const float err = (hi - (t - bp)) + (x - bp);
  hi = t;
  lo += err;
}

template <typename R>
__global__ void __launch_bounds__(256) gram_kernel(const __grid_constant__ GramPack jobs, int njobs, int Rmax,
                                                   int nchunks) {
  const int bidx = blockIdx.z / njobs;        // batch element
  const GramJob& jb = jobs.j[blockIdx.z - bidx * njobs];
  const int Rn = jb.D1 * jb.D2;
  const int ntile = (Rn + kGT - 1) / kGT;
  const int ti = blockIdx.y / ((Rmax + kGT - 1) / kGT);
  const int tj = blockIdx.y % ((Rmax + kGT - 1) / kGT);
  if (ti >= ntile || tj >= ntile) return;
  const bool diag = ti == tj;                 // both operand tiles are the same rows
  const R* T = (const R*)jb.T + bidx * jobs.sT;
  const int64_t kchunk = (jb.K + nchunks - 1) / nchunks;
  const int64_t k0 = blockIdx.x * kchunk;
  const int64_t k1 = min(jb.K, k0 + kchunk);

  __shared__ R Xi[kGK][kGT + 1];
  __shared__ R Xj[kGK][kGT + 1];
  __shared__ int64_t roff[kGK];
  __shared__ int64_t rowi[kGT], rowj[kGT];

  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  if (tid < kGT) {
    const int i = ti * kGT + tid;
    rowi[tid] = i < Rn ? (i / jb.D2) * jb.s1 + (i % jb.D2) * jb.s2 : -1;
  } else if (tid < 2 * kGT) {
    const int j = tj * kGT + (tid - kGT);
    rowj[tid - kGT] = j < Rn ? (j / jb.D2) * jb.s1 + (j % jb.D2) * jb.s2 : -1;
  }
  using Pair = typename std::conditional<sizeof(R) == 8, double, float>::type;
  Pair acc[4][4], accl[4][4];     // accl: low parts of the float pairs (unused for FP64)
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) acc[a][b] = accl[a][b] = 0;
  const R(*Xb)[kGT + 1] = diag ? Xi : Xj;

  for (int64_t kb = k0; kb < k1; kb += kGK) {
    __syncthreads();
    if (tid < kGK) {
      // K = prod of six bond dimensions <= 16^6 < 2^32: the summed index decodes in 32 bits
      uint32_t k = (uint32_t)(kb + tid);
      int64_t off = 0;
      if (kb + tid < k1) {
        for (int d = jb.nrest - 1; d >= 0; --d) {
          const uint32_t n = (uint32_t)jb.rdims[d];
          const uint32_t i = k % n;
          k /= n;
          off += (int64_t)i * jb.rst[d];
        }
        roff[tid] = off;
      } else {
        roff[tid] = -1;
      }
    }
    __syncthreads();
    for (int e = tid; e < kGK * kGT; e += 256) {
      const int r = e / kGK, kk = e % kGK;   // consecutive threads: consecutive summed index
      const int64_t ro = roff[kk];
      const int64_t oi = rowi[r];
      Xi[kk][r] = (ro >= 0 && oi >= 0) ? T[oi + ro] : (R)0;
      if (!diag) {
        const int64_t oj = rowj[r];
        Xj[kk][r] = (ro >= 0 && oj >= 0) ? T[oj + ro] : (R)0;
      }
    }
    __syncthreads();
    if (diag && ty > tx) continue;   // mirrored from the thread (tx, ty) at the end
    R part[4][4];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) part[a][b] = 0;
#pragma unroll 8
    for (int kk = 0; kk < kGK; ++kk) {
      R vi[4], vj[4];
      for (int a = 0; a < 4; ++a) vi[a] = Xi[kk][ty * 4 + a];
      for (int b = 0; b < 4; ++b) vj[b] = Xb[kk][tx * 4 + b];
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) part[a][b] = fma(vi[a], vj[b], part[a][b]);
    }
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        if constexpr (sizeof(R) == 8) acc[a][b] += part[a][b];
        else two_sum_acc(acc[a][b], accl[a][b], part[a][b]);
      }
  }
  // on a diagonal tile only the blocks ty <= tx were summed; the block (ty, tx) also gives
  // (tx, ty) as its transpose (the same products in the same order: bit-identical)
  if (diag && ty > tx) return;
  double* out = jb.partial + bidx * jobs.sPart + (int64_t)blockIdx.x * Rn * Rn;
  for (int a = 0; a < 4; ++a) {
    const int i = ti * kGT + ty * 4 + a;
    if (i >= Rn) continue;
    for (int b = 0; b < 4; ++b) {
      const int j = tj * kGT + tx * 4 + b;
      if (j >= Rn) continue;
      const double v = (double)acc[a][b] + (double)accl[a][b];
      out[(int64_t)i * Rn + j] = v;
      if (diag && ty < tx) out[(int64_t)j * Rn + i] = v;
    }
  }
}

template <typename R>
cudaError_t launch_gram(const GramPack& jobs, int njobs, int Rmax, int nchunks, cudaStream_t st) {
  const int nt = (Rmax + kGT - 1) / kGT;
  dim3 grid(nchunks, nt * nt, njobs * jobs.batch);
  gram_kernel<R><<<grid, 256, 0, st>>>(jobs, njobs, Rmax, nchunks);
  return cudaGetLastError();
}
template cudaError_t launch_gram<double>(const GramPack&, int, int, int, cudaStream_t);
template cudaError_t launch_gram<float>(const GramPack&, int, int, int, cudaStream_t);

// out_i[e] = sum_c partial_i[c][e] for every job i of the pack (and batch element), in one
// launch; job i of element b goes to out[(b njobs + i) out_stride]. A block takes 32
// consecutive entries of one job; its 8 warps add interleaved chunk subsets (warp w: chunks
// c = w mod 8, in increasing c) and the 8 warp sums are added in warp order, so the result
// does not depend on scheduling.
__global__ void __launch_bounds__(256) gram_reduce_kernel(const __grid_constant__ GramPack jobs, int njobs,
                                                          int nchunks, int64_t out_stride, double* __restrict__ out) {
  const int bidx = blockIdx.y / njobs;
  const GramJob& jb = jobs.j[blockIdx.y - bidx * njobs];
  const double* partial = jb.partial + bidx * jobs.sPart;
  const int64_t RR = (int64_t)jb.D1 * jb.D2 * jb.D1 * jb.D2;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __shared__ double red[8][32];
  for (int64_t e0 = (int64_t)blockIdx.x * 32; e0 < RR; e0 += (int64_t)gridDim.x * 32) {
    const int64_t e = e0 + lane;
    double s = 0;
    if (e < RR)
      for (int c = w; c < nchunks; c += 8) s += partial[(int64_t)c * RR + e];
    red[w][lane] = s;
    __syncthreads();
    if (w == 0 && e < RR) {
      double t = 0;
      for (int q = 0; q < 8; ++q) t += red[q][lane];
      out[(int64_t)blockIdx.y * out_stride + e] = t;
    }
    __syncthreads();
  }
}

cudaError_t launch_gram_reduce(const GramPack& jobs, int njobs, int nchunks, int64_t RRmax, int64_t out_stride,
                               double* out, cudaStream_t st) {
  int64_t blocks = (RRmax + 31) / 32;
  if (blocks > 1024) blocks = 1024;
  gram_reduce_kernel<<<dim3((unsigned)blocks, (unsigned)(njobs * jobs.batch)), 256, 0, st>>>(jobs, njobs, nchunks,
                                                                                             out_stride, out);
  return cudaGetLastError();
}

// G[(a1 a2),(b1 b2)] = sum_{k,k'} A1[(a1,k),(b1,k')] A2[(a2,k),(b2,k')], FP64.
__global__ void gram_merge_kernel(const double* __restrict__ A1, const double* __restrict__ A2, int Dn, int Dk,
                                  double* __restrict__ G) {
  const int n = Dn * Dn;
  const int Rk = Dn * Dk;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int row = e / n, col = e % n;
    const int a1 = row / Dn, a2 = row % Dn, b1 = col / Dn, b2 = col % Dn;
    double s = 0;
    for (int k = 0; k < Dk; ++k)
      for (int kp = 0; kp < Dk; ++kp)
        s = fma(A1[(int64_t)(a1 * Dk + k) * Rk + b1 * Dk + kp], A2[(int64_t)(a2 * Dk + k) * Rk + b2 * Dk + kp], s);
    G[e] = s;
  }
}

cudaError_t launch_gram_merge(const double* A1, const double* A2, int Dn, int Dk, double* G, cudaStream_t st) {
  const int n2 = Dn * Dn * Dn * Dn;
  gram_merge_kernel<<<(n2 + 255) / 256, 256, 0, st>>>(A1, A2, Dn, Dk, G);
  return cudaGetLastError();
}

// One launch for the six Gram matrices of every batch element: blockIdx.y = b * 6 + i * 2 +
// side (same arithmetic and order as gram_merge_kernel).
__global__ void gram_merge_batch_kernel(const double* __restrict__ half, int64_t RRs, int Dn0, int Dn1, int Dn2,
                                        int Dk, double* __restrict__ G, int64_t nn) {
  const int q = blockIdx.y % 6, bidx = blockIdx.y / 6;
  const int i = q / 2;
  const int Dn = i == 0 ? Dn0 : (i == 1 ? Dn1 : Dn2);
  const double* A1 = half + ((int64_t)bidx * 12 + q * 2) * RRs;
  const double* A2 = A1 + RRs;
  double* Gq = G + ((int64_t)bidx * 6 + q) * nn;
  const int n = Dn * Dn;
  const int Rk = Dn * Dk;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int row = e / n, col = e % n;
    const int a1 = row / Dn, a2 = row % Dn, b1 = col / Dn, b2 = col % Dn;
    double s = 0;
    for (int k = 0; k < Dk; ++k)
      for (int kp = 0; kp < Dk; ++kp)
        s = fma(A1[(int64_t)(a1 * Dk + k) * Rk + b1 * Dk + kp], A2[(int64_t)(a2 * Dk + k) * Rk + b2 * Dk + kp], s);
    Gq[e] = s;
  }
}

cudaError_t launch_gram_merge_batch(const double* half, int64_t RRs, const int Dn[3], int Dk, double* G, int64_t nn,
                                    int batch, cudaStream_t st) {
  int nmax = 0;
  for (int i = 0; i < 3; ++i) nmax = nmax > Dn[i] * Dn[i] ? nmax : Dn[i] * Dn[i];
  const int blocks = (nmax * nmax + 255) / 256;
  gram_merge_batch_kernel<<<dim3(blocks, 6 * batch), 256, 0, st>>>(half, RRs, Dn[0], Dn[1], Dn[2], Dk, G, nn);
  return cudaGetLastError();
}

}  // namespace hotrg
