// gemm_simt.cu - CUDA-core GEMM for the FP64 reference mode and the FP32 mode.
//
// C[m][n] = alpha * sum_k A[m*lda + k] B[n*ldb + k] + beta * C[m*ldc + n]: both operands
// K-major (the layout the block-spin contraction builds, the same one the tensor-core
// path consumes). 128x64 output tile per CTA, 256 threads with an 8x4 register tile,
// 16-wide k slices staged in shared memory. FP64 mode uses DFMA; FP32 mode FFMA with FP32
// accumulation. Ragged M, N and K edges are guarded.
#include "common.cuh"

namespace hotrg {

constexpr int kBM = 128, kBN = 64, kBK = 16;

template <typename R>
__global__ void __launch_bounds__(256) gemm_simt_kernel(const R* __restrict__ A, int64_t lda, const R* __restrict__ B,
                                                        int64_t ldb, R* __restrict__ C, int64_t ldc, int64_t M,
                                                        int64_t N, int64_t K, R alpha, R beta) {
  __shared__ R As[kBK][kBM + 4];
  __shared__ R Bs[kBK][kBN + 4];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;   // 16 x 16 threads; rows ty*8.., cols tx*4..
  const int64_t m0 = (int64_t)blockIdx.y * kBM, n0 = (int64_t)blockIdx.x * kBN;
  R acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;

  for (int64_t k0 = 0; k0 < K; k0 += kBK) {
    // A tile: 128 x 16 = 2048 elements, 8 per thread; k fastest for coalescing
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int e = tid + r * 256;
      const int row = e / kBK, kk = e % kBK;
      const int64_t gm = m0 + row, gk = k0 + kk;
      As[kk][row] = (gm < M && gk < K) ? A[gm * lda + gk] : (R)0;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + r * 256;
      const int col = e / kBK, kk = e % kBK;
      const int64_t gn = n0 + col, gk = k0 + kk;
      Bs[kk][col] = (gn < N && gk < K) ? B[gn * ldb + gk] : (R)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      R a[8], b[4];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = As[kk][ty * 8 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t gm = m0 + ty * 8 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      R* c = C + gm * ldc + gn;
      *c = beta == (R)0 ? alpha * acc[i][j] : alpha * acc[i][j] + beta * *c;
    }
  }
}

template <typename R>
cudaError_t launch_gemm_simt(const R* A, int64_t lda, const R* B, int64_t ldb, R* C, int64_t ldc, int64_t M,
                             int64_t N, int64_t K, double alpha, double beta, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const int64_t gy = (M + kBM - 1) / kBM, gx = (N + kBN - 1) / kBN;
  if (gy > 65535 || gx > 0x7fffffffLL) return cudaErrorInvalidValue;
  dim3 grid((unsigned)gx, (unsigned)gy);
  gemm_simt_kernel<R><<<grid, 256, 0, st>>>(A, lda, B, ldb, C, ldc, M, N, K, (R)alpha, (R)beta);
  return cudaGetLastError();
}
template cudaError_t launch_gemm_simt<double>(const double*, int64_t, const double*, int64_t, double*, int64_t,
                                              int64_t, int64_t, int64_t, double, double, cudaStream_t);
template cudaError_t launch_gemm_simt<float>(const float*, int64_t, const float*, int64_t, float*, int64_t, int64_t,
                                             int64_t, int64_t, double, double, cudaStream_t);

}  // namespace hotrg
