// common.cuh - shared types of the HOTRG CUDA library (internal header).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>

namespace hotrg {

constexpr int kMaxRank = 10;      // legs of the largest intermediate (D^10 operands)
constexpr int kMaxLeg = 16;       // largest bond dimension (dcut_max)
constexpr int kMaxGramN = kMaxLeg * kMaxLeg;  // largest Gram matrix side (D_nu^2)
constexpr int kMaxSteps = 64;     // steps recorded per batch element
constexpr int kJacobiMaxSweeps = 60;
constexpr int kJacobiSmemN = 96;  // the eigensolver keeps A and V in shared memory up to this n (no work buffer)

// Device-side status words (in the caller's workspace), read back at sync points.
enum StatusWord { kStNoConv = 0, kStNonFinite = 1, kStTimeout = 2, kStWords = 4 };

// Tensor-times-matrix descriptor: out[o] = alpha * sum_{j1<J1, j2<J2}
//   U[u(o) + j1*u_sj1 + j2*u_sj2] * in[i(o) + j1*in_sj1 + j2*in_sj2]  (+ beta * out[o])
// where o runs over `rank` output dims (iteration order: dims[0] outermost); the last
// `rin` dims form the inner loop of one block. i(o), u(o), out offset are linear in the
// output multi-index with the given strides. U == nullptr means U = 1 (a permutation).
struct TTMArgs {
  int rank;
  int rin;
  int J1, J2;
  int64_t dims[kMaxRank];
  int64_t in_st[kMaxRank];
  int64_t u_st[kMaxRank];
  int64_t out_st[kMaxRank];
  int64_t in_sj1, in_sj2, u_sj1, u_sj2;
  int64_t outer, inner;
  double alpha, beta;
  // nb batch elements in one launch: element e reads in + e in_bs and U + e u_bs and writes
  // out + e out_bs (output strides count fp16 values in the fp16 split modes)
  int nb;
  int64_t in_bs, u_bs, out_bs;
  // split modes: an upper bound of the operand's magnitudes (bits of a non-negative float)
  // that sets its power-of-two scale (nullptr: the fixed scale); kTTMMaxAbs and kTTMStoreMax:
  // where the pass accumulates amax_mul times its largest |output| (atomicMax, rounded up).
  // One word per batch element: element e uses amax[e amax_bs].
  unsigned* amax;
  float amax_mul;
  int amax_bs;
};

enum TTMMode {
  kTTMStore = 0,
  kTTMSplitTF32 = 1,
  kTTMAccumulate = 2,
  kTTMSplitF16 = 3,
  kTTMSplitOz = 4,
  kTTMMaxAbs = 5,    // computes the outputs, keeps only their largest magnitude (a.amax)
  kTTMStoreMax = 6   // kTTMStore, and accumulates the largest |output| as kTTMMaxAbs does
};
// Per-operand power-of-two scale of the split modes (max-norm scaling): with m the largest
// magnitude of the operand and m < 2^ex (frexp), the operand is multiplied by 2^(top - ex),
// so its largest entry lies in [2^(top-1), 2^top): top = 15 for the fp16 hi/lo planes (fp16's
// largest finite value is 65504), 0 for the integer slices (which need |x| < 1). m = 0 gives
// the exponent top. The product of two such operands carries 2^(eA + eB), which the GEMM
// removes. Computed identically by the split passes and the GEMM epilogues.
__host__ __device__ inline int split_exponent(unsigned mbits, int top) {
  if (mbits == 0u) return top;
  const int ex = (int)((mbits >> 23) & 0xffu) - 126;   // m = f 2^ex, f in [0.5, 1)
  return top - ex;
}
constexpr int kF16Top = 15;
constexpr int kOzTop = 0;
// FP64-grade tensor-core mode (Ozaki-type splitting): an FP64 operand x with |x| < 1 (after
// its max-norm scale) is stored as kOzSlices fp16 planes of integers v_i, x = sum_i v_i
// 2^(-8 (i + 1)) up to 2^-41; |v_0| <= 256, |v_i| <= 128 for i >= 1. Plane p of an operand
// starts p times the plane size after plane 0 (the split pass takes the plane size as
// out_lo - out).
constexpr int kOzSlices = 5;
// Scale applied to operands stored as fp16 hi/lo pairs: |x| <= 1 (normalised tensors
// contracted with isometries) becomes <= 2^14, inside fp16's normal range with room for
// the products; the GEMM undoes it with alpha * 2^-28.
constexpr float kF16Scale = 16384.0f;

// One half-Gram job: A[(i1 i2), (j1 j2)] = sum_rest T[i1@l1, i2@l2, rest] T[j1, j2, rest].
struct GramJob {
  const void* T;
  int D1, D2;               // sizes of the two row legs
  int64_t s1, s2;           // their strides in T
  int nrest;                // number of summed legs (6 for a rank-8 tensor)
  int64_t rdims[8];         // summed leg sizes (outermost first)
  int64_t rst[8];           // summed leg strides
  int64_t K;                // product of rdims
  double* partial;          // [nchunks][R][R]
};

// One symmetric eigenproblem for the Jacobi kernel.
struct EigJob {
  const double* G;          // n x n, row-major, symmetric
  double* work;             // 2 n^2 doubles of global scratch (used when n is large)
  double* lam;              // n eigenvalues, descending
  double* U;                // n x chi, first chi eigenvectors in canonical gauge
  double* eps;              // sum of the discarded eigenvalues (index >= chi)
  int* degenerate;          // 1 if the cut at chi falls inside a cluster
  int n, chi;
};

// Side choice for one transverse direction: candidates from the nu and nu' Gram matrices.
struct SelectJob {
  const double* U[2];      // candidate isometries (n x chi), nu side and nu' side
  const double* lam0;      // spectrum of the nu side (absolute tie floor)
  const double* eps[2];    // discarded eigenvalue sums
  const int* degen[2];     // cut inside a cluster
  double* U64;             // chosen isometry, FP64, n x chi (after Gram-Schmidt)
  void* Ur;                // chosen isometry in the storage precision
  int n, chi;
  double* rec_eps;         // step record: eps of both sides
  int* rec_primed;         // step record: side taken
  int* rec_degen;          // step record: degenerate cut on the side taken
  // when rec_b != nullptr the record fields above are ignored and the kernel writes
  // rec_b[*step].{eps,primed,degen}[nu] (step counter read on the device)
  struct DevRecord* rec_b;
  const int* step;
  int nu;
};

// Step record as kept on the device for each batch element and step.
struct DevRecord {
  double eps[4][2];
  double ln_c;
  int primed[4];
  int degen[4];
};

// Job packs passed to kernels by value (kernel parameter space), so a step needs no
// host-to-device copies of job descriptors and can be captured in a CUDA graph. A pack
// describes the jobs of batch element 0; with batch > 1 one launch also runs them for
// elements 1 .. batch - 1, every pointer of element b advanced by b times its stride
// (counted in elements of the pointed-to type). batch = 1 is the plain pack.
constexpr int kMaxGramJobs = 12;
constexpr int kMaxEigJobs = 6;
constexpr int kMaxSelectJobs = 3;
struct GramPack {
  GramJob j[kMaxGramJobs];
  int batch = 1;
  int64_t sT = 0;           // tensor (storage elements)
  int64_t sPart = 0;        // split-K partials (doubles)
};
struct EigPack {
  EigJob j[kMaxEigJobs];
  int batch = 1;
  int64_t sG = 0, sWork = 0, sLam = 0, sU = 0, sEps = 0, sDeg = 0;
};
struct SelectPack {
  SelectJob j[kMaxSelectJobs];
  int batch = 1;
  int64_t sU = 0;           // candidate isometries (doubles)
  int64_t sLam = 0, sEps = 0, sDeg = 0;
  int64_t sU64 = 0;         // chosen isometry, FP64
  int64_t sUr = 0;          // chosen isometry, storage precision (elements)
  int64_t sRec = 0;         // step records (DevRecord)
};

// Message returned by hotrg_last_error for this host thread.
void set_last_error(const char* msg);

// Host-side launchers (defined in the .cu files, called by the orchestrator).
template <typename TI, typename TU, typename TO>
cudaError_t launch_ttm(const TI* in, const TU* U, TO* out, TO* out_lo, const TTMArgs& a, int mode,
                       cudaStream_t st);

template <typename R>
cudaError_t launch_gram(const GramPack& jobs, int njobs, int Rmax, int nchunks, cudaStream_t st);
cudaError_t launch_gram_reduce(const GramPack& jobs, int njobs, int nchunks, int64_t RRmax, int64_t out_stride,
                               double* out, cudaStream_t st);
cudaError_t launch_gram_merge(const double* A1, const double* A2, int Dn, int Dk, double* G,
                              cudaStream_t st);
// The six Gram matrices (3 transverse directions x 2 sides) of each of `batch` elements in
// one launch: half-Grams at half[((b * 12) + (i * 2 + side) * 2 + h) * RRs] (h = 0: k on
// T1's mu' leg, 1: k on T2's mu leg), G at G[((b * 6) + i * 2 + side) * nn], Dn[i] the bond
// dimension of direction i, Dk that of mu.
cudaError_t launch_gram_merge_batch(const double* half, int64_t RRs, const int Dn[3], int Dk, double* G, int64_t nn,
                                    int batch, cudaStream_t st);
cudaError_t launch_jacobi(const EigPack& jobs, int njobs, int nmax, double cluster_tau, int* status,
                          cudaStream_t st, int max_sweeps = kJacobiMaxSweeps, double tie_rel = 1e-8);
cudaError_t launch_wait_selftest(int* status, unsigned long long limit_ns, cudaStream_t st);
// FP64-grade product on the fp16 tensor cores: C[M][N] (double, row stride ldc) =
// alpha A B^T with A, B given as kOzSlices integer planes each (K panels as in
// launch_gemm_group; plane p of A at A + p aps elements, of B at B + p bps), each operand
// sliced after scaling by 2^split_exponent(*amax, kOzTop) (amax_a, amax_b; nullptr: no scale);
// accumulate: C += alpha A B^T.
cudaError_t launch_gemm_oz(const void* A, const void* B, int64_t aps, int64_t bps, int64_t Kp, int64_t kps, int64_t P,
                           int64_t M, int64_t N, double* C, int64_t ldc, double alpha, const unsigned* amax_a,
                           const unsigned* amax_b, bool accumulate, int* status, cudaStream_t st);
// One output of a grouped block-spin GEMM: C = alpha * sum_{s < nseg} A_{a[s]} B_{b[s]}^T,
// where A_w, B_w are the w-th operand tensors of the launch (the k loop runs over the nseg
// segments one after the other, each the full K).
struct GemmProblem {
  float* C;
  float alpha;
  int nseg;
  int a[2], b[2];
};
constexpr int kMaxGemmProblems = 96;   // 32 temperatures x 3 tensors per launch
struct GemmGroup {
  GemmProblem p[kMaxGemmProblems];
  int nprob;
  // fp16 operands scaled by their max-norm exponents (split_exponent(amax[e], kF16Top), one
  // word per batch element e, problem pb of element pb / per_elem): the epilogue multiplies by
  // 2^-(eA + eB); nullptr: the operands carry no such scale
  const unsigned* amax_a;
  const unsigned* amax_b;
  int per_elem;
};
// Tensor-core GEMM over W operand tensors per plane (hi, lo), each [P][rows][kps] in K
// panels, tensor w of a plane aws (A) or bws (B) elements after tensor w - 1; every problem
// has M rows, N columns and row stride ldc. variant selects the pipeline (gemm_tc.cu).
cudaError_t launch_gemm_group(const void* Ahi, const void* Alo, const void* Bhi, const void* Blo, int W, int64_t aws,
                              int64_t bws, int64_t Kp, int64_t kps, int64_t P, int64_t M, int64_t N, int64_t ldc,
                              const GemmGroup& g, int* status, cudaStream_t st, int variant);

template <typename R>
cudaError_t launch_select(const SelectPack& jobs, int njobs, double side_rel, cudaStream_t st);
template <typename R>
cudaError_t launch_init(const double* beta, const double* h, R* T, R* S, int64_t slot, double* lnz_acc,
                        int batch, cudaStream_t st);
template <typename R>
cudaError_t launch_norm(const R* x, int64_t n, int nb, int64_t xstride, double* partial, const int* step,
                        double* c_out, double* lnz_acc,
                        DevRecord* rec_b, int* status, cudaStream_t st);
cudaError_t launch_step_end(int* step, cudaStream_t st);
// Counts over one fp16 plane in K panels (nrows rows of kps values, the first Kp of each
// read): out[0] += zero entries, out[1] += entries in fp16's subnormal range (nonzero, below
// 2^-14), out[2] = max(out[2], bits of the largest magnitude).
cudaError_t launch_plane_stats(const void* plane, int64_t nrows, int64_t Kp, int64_t kps, unsigned long long* out,
                               cudaStream_t st);
void jacobi_prepare();
void gemm_prepare();
template <typename R>
cudaError_t launch_scale(R* x, int64_t n, int nb, int64_t xstride, const double* c, cudaStream_t st);
template <typename R>
cudaError_t launch_trace(const R* T, int64_t slot, const int* dims, int batch, double* out, cudaStream_t st);
template <typename R>
cudaError_t launch_xind(const R* T, int64_t slot, const int* dims, int batch, int nu, double* out, cudaStream_t st);
constexpr int kNormPartials = 2 * 152;

template <typename R>
cudaError_t launch_gemm_simt(const R* A, int64_t lda, const R* B, int64_t ldb, R* C, int64_t ldc,
                             int64_t M, int64_t N, int64_t K, double alpha, double beta,
                             cudaStream_t st);

}  // namespace hotrg
