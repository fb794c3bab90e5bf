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
// accumulated in FP64 per 32-term slice; gram_reduce adds the chunks in a fixed order
// (deterministic); gram_merge forms G in FP64.
#include "common.cuh"

namespace hotrg {

constexpr int kGT = 64;   // output tile
constexpr int kGK = 32;   // k slice held in shared memory

template <typename R>
__global__ void __launch_bounds__(256) gram_kernel(const __grid_constant__ GramPack jobs, int Rmax, int nchunks) {
  const GramJob& jb = jobs.j[blockIdx.z];
  const int Rn = jb.D1 * jb.D2;
  const int ntile = (Rn + kGT - 1) / kGT;
  const int ti = blockIdx.y / ((Rmax + kGT - 1) / kGT);
  const int tj = blockIdx.y % ((Rmax + kGT - 1) / kGT);
  if (ti >= ntile || tj >= ntile) return;
  const R* T = (const R*)jb.T;
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
  double acc[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

  for (int64_t kb = k0; kb < k1; kb += kGK) {
    __syncthreads();
    if (tid < kGK) {
      int64_t k = kb + tid, off = 0;
      if (k < k1) {
        for (int d = jb.nrest - 1; d >= 0; --d) {
          const int64_t i = k % jb.rdims[d];
          k /= jb.rdims[d];
          off += i * jb.rst[d];
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
      const int64_t oi = rowi[r], oj = rowj[r];
      Xi[kk][r] = (ro >= 0 && oi >= 0) ? T[oi + ro] : (R)0;
      Xj[kk][r] = (ro >= 0 && oj >= 0) ? T[oj + ro] : (R)0;
    }
    __syncthreads();
    R part[4][4];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) part[a][b] = 0;
#pragma unroll 8
    for (int kk = 0; kk < kGK; ++kk) {
      R vi[4], vj[4];
      for (int a = 0; a < 4; ++a) vi[a] = Xi[kk][ty * 4 + a];
      for (int b = 0; b < 4; ++b) vj[b] = Xj[kk][tx * 4 + b];
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) part[a][b] = fma(vi[a], vj[b], part[a][b]);
    }
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) acc[a][b] += (double)part[a][b];
  }
  double* out = jb.partial + (int64_t)blockIdx.x * Rn * Rn;
  for (int a = 0; a < 4; ++a) {
    const int i = ti * kGT + ty * 4 + a;
    if (i >= Rn) continue;
    for (int b = 0; b < 4; ++b) {
      const int j = tj * kGT + tx * 4 + b;
      if (j < Rn) out[(int64_t)i * Rn + j] = acc[a][b];
    }
  }
}

template <typename R>
cudaError_t launch_gram(const GramPack& jobs, int njobs, int Rmax, int nchunks, cudaStream_t st) {
  const int nt = (Rmax + kGT - 1) / kGT;
  dim3 grid(nchunks, nt * nt, njobs);
  gram_kernel<R><<<grid, 256, 0, st>>>(jobs, Rmax, nchunks);
  return cudaGetLastError();
}
template cudaError_t launch_gram<double>(const GramPack&, int, int, int, cudaStream_t);
template cudaError_t launch_gram<float>(const GramPack&, int, int, int, cudaStream_t);

// out[e] = sum_c partial[c][e], chunks added in increasing c.
__global__ void gram_reduce_kernel(const double* __restrict__ partial, int nchunks, int64_t RR,
                                   double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < RR; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0;
    for (int c = 0; c < nchunks; ++c) s += partial[c * RR + e];
    out[e] = s;
  }
}

cudaError_t launch_gram_reduce(const double* partial, int nchunks, int64_t RR, double* out, cudaStream_t st) {
  int64_t blocks = (RR + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  gram_reduce_kernel<<<(unsigned)blocks, 256, 0, st>>>(partial, nchunks, RR, out);
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

}  // namespace hotrg
