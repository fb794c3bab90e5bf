// jacobi.cu - FP64 symmetric eigensolver for the HOSVD Gram matrices (Fig. 1B) and the
// choice of the truncating isometry.
//
// jacobi_kernel: one CTA per matrix. Cyclic two-sided Jacobi in round-robin (tournament)
// order: each round rotates n/2 disjoint index pairs at once, so every 2x2 block of A is
// updated by exactly one thread and the rounds need only block barriers. The tournament runs
// separately inside each connected component of A's nonzero pattern (exact zeros between
// components stay exact zeros), which quarters the work when the Gram matrix splits by Z2
// charge. A pair is
// rotated when |a_pq| > max(1e-18 ||G||_F, 2^-52 sqrt|a_pp a_qq|); a sweep without
// rotations ends the loop, and max_sweeps sweeps (kJacobiMaxSweeps unless the context
// overrides it) raise the no-convergence status
// (results are still written). Then: eigenvalues sorted descending, the discarded sum
// eps = sum_{j >= chi} lambda_j, and the first chi eigenvectors in the canonical gauge:
// eigenvalues closer than cluster_tau * lambda_0 form a cluster (cluster_tau is set
// above the rounding noise of the Gram matrix: 1e-10 when the tensors are FP64, 1e-6
// when they are stored in FP32); inside a cluster the
// basis is built by repeatedly taking the unit vector e_i with the longest projection on
// the not-yet-covered part of the cluster's eigenspace (lowest i within a relative
// tie_rel of the longest: 1e-8 for FP64 tensors, 1e-4 for FP32-stored ones, whose noise
// would otherwise break exact symmetric ties at random) and normalising that projection. This gauge depends only on the
// eigenspaces, so it does not depend on the eigensolver.
//
// select_kernel: per transverse direction, the side (nu or nu') with the smaller
// discarded sum (a difference within side_rel (eps + eps') + 1e-13 lambda_0 is a tie and
// goes to nu; side_rel = 1e-9 for FP64 tensors, 1e-6 for FP32 ones), then modified Gram-Schmidt in FP64 on the kept vectors, and copies of U in
// FP64 and in the storage precision.
#include <math.h>

#include "common.cuh"

namespace hotrg {

constexpr int kJT = 512;            // threads per Jacobi CTA (16 warps: latency, not FP64 throughput, bounds a round)
constexpr int kSmemJacobiN = kJacobiSmemN;    // A and V in shared memory up to this n

__device__ __forceinline__ void rr_pair(int r, int i, int m, int& p, int& q) {
  if (i == 0) {
    p = r;
    q = m - 1;
  } else {
    p = (r + i) % (m - 1);
    q = (r - i + (m - 1)) % (m - 1);
  }
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
}

// e-th entry (row-major) of the upper triangle, diagonal included, of an h x h grid.
__device__ __forceinline__ void tri_index(int e, int h, int& P, int& Q) {
  // rows start at s(P) = P h - P (P - 1) / 2; invert with a float square root, then fix up
  const float b = 2.0f * h + 1.0f;
  int r = (int)((b - sqrtf(b * b - 8.0f * (float)e)) * 0.5f);
  r = r < 0 ? 0 : (r > h - 1 ? h - 1 : r);
  while (r > 0 && r * h - r * (r - 1) / 2 > e) --r;
  while (r + 1 < h && (r + 1) * h - (r + 1) * r / 2 <= e) ++r;
  P = r;
  Q = r + (e - (r * h - r * (r - 1) / 2));
}

__device__ double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  __syncthreads();
  return s;
}

__global__ void __launch_bounds__(kJT) jacobi_kernel(const __grid_constant__ EigPack jobs, int njobs, int use_smem,
                                                     double cluster_tau, double tie_rel, int max_sweeps,
                                                     int* status) {
  extern __shared__ double dyn[];
  // one slot per rotation pair of a round: at most n (ceil(m_c / 2) <= m_c per component)
  __shared__ double cs[kMaxGramN], sn[kMaxGramN];
  __shared__ int pp[kMaxGramN], qq[kMaxGramN];
  __shared__ double lam[kMaxGramN], nrm[kMaxGramN];
  __shared__ int perm[kMaxGramN], cstart[kMaxGramN + 1];
  __shared__ double red[kJT / 32];
  __shared__ int rotated, ncl, pivot;
  __shared__ int comp[kMaxGramN];          // component label: its smallest index
  __shared__ int mem[kMaxGramN];           // indices grouped by component
  __shared__ int cbeg[kMaxGramN + 1];      // component c: mem[cbeg[c] .. cbeg[c + 1])
  __shared__ int poff[kMaxGramN + 1];      // first pair slot of component c
  __shared__ int toff[kMaxGramN + 1];      // first 2x2 block of component c
  __shared__ int voff[kMaxGramN + 1];      // first V-update item of component c
  __shared__ int ncomp, rmax, changed;
  __shared__ double pivval;

  // job blockIdx.x % njobs of batch element blockIdx.x / njobs
  const int64_t bidx = blockIdx.x / njobs;
  EigJob jb = jobs.j[blockIdx.x - bidx * njobs];
  jb.G += bidx * jobs.sG;
  if (jb.work) jb.work += bidx * jobs.sWork;
  jb.lam += bidx * jobs.sLam;
  jb.U += bidx * jobs.sU;
  jb.eps += bidx * jobs.sEps;
  jb.degenerate += bidx * jobs.sDeg;
  const int n = jb.n, chi = jb.chi;
  const int tid = threadIdx.x;
  double* A = use_smem ? dyn : jb.work;   // use_smem: every job of the launch has n <= kSmemJacobiN
  double* V = A + (int64_t)n * n;

  double fro = 0;
  for (int e = tid; e < n * n; e += kJT) {
    // the upper triangle of G, mirrored (the merged Gram is symmetric up to summation order)
    const int gi = e / n, gj = e % n;
    const double g = jb.G[gi <= gj ? e : gj * n + gi];
    A[e] = g;
    V[e] = (e / n == e % n) ? 1.0 : 0.0;
    fro += g * g;
  }
  fro = sqrt(block_sum(fro, red));
  const double tol_abs = 1e-18 * fro;
  const double tol_rel = 2.220446049250313e-16;

  // ---- connected components of the nonzero pattern of A. A rotation of a pair inside one
  // component leaves the entries between components exactly zero (and the rows of V outside
  // the component too), so each component is diagonalised by its own round-robin tournament
  // and the rest is skipped, exactly. With h = 0 the Gram matrices of the Ising tensors split
  // this way by the Z2 charge of the fused index (two halves: a quarter of the FP64 work);
  // a connected matrix takes the plain tournament, operation for operation.
  for (int i = tid; i < n; i += kJT) comp[i] = i;
  while (true) {
    __syncthreads();
    if (tid == 0) changed = 0;
    __syncthreads();
    for (int i = tid; i < n; i += kJT) {
      int lab = comp[i];
      for (int j = 0; j < n; ++j)
        if (A[i * n + j] != 0.0 && comp[j] < lab) lab = comp[j];
      if (lab < comp[i]) {
        comp[i] = lab;
        changed = 1;
      }
    }
    __syncthreads();
    if (!changed) break;
  }
  if (tid == 0) {
    // components in the order of their smallest member; members in increasing index
    int nc = 0;
    for (int i = 0; i < n; ++i)
      if (comp[i] == i) perm[i] = nc++;   // perm: label -> component number (scratch here)
    for (int c = 0; c <= nc; ++c) cbeg[c] = 0;
    for (int i = 0; i < n; ++i) ++cbeg[perm[comp[i]] + 1];
    for (int c = 0; c < nc; ++c) cbeg[c + 1] += cbeg[c];
    for (int c = 0; c < nc; ++c) cstart[c] = cbeg[c];   // fill cursor (scratch here)
    for (int i = 0; i < n; ++i) mem[cstart[perm[comp[i]]]++] = i;
    poff[0] = toff[0] = voff[0] = 0;
    int rm = 1;
    for (int c = 0; c < nc; ++c) {
      const int mc = cbeg[c + 1] - cbeg[c], mp = mc + (mc & 1), np = mp / 2;
      poff[c + 1] = poff[c] + np;
      toff[c + 1] = toff[c] + np * (np + 1) / 2;
      voff[c + 1] = voff[c] + mc * np;
      rm = max(rm, mp - 1);
    }
    ncomp = nc;
    rmax = rm;
  }
  __syncthreads();
  const int nc = ncomp, npairs = poff[nc], nblk = toff[nc], nvu = voff[nc], rounds = rmax;

  int sweep = 0;
  for (; sweep < max_sweeps && n > 1; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < rounds; ++r) {
      for (int sl = tid; sl < npairs; sl += kJT) {
        int c = 0;
        while (poff[c + 1] <= sl) ++c;
        const int mc = cbeg[c + 1] - cbeg[c], mp = mc + (mc & 1);
        int lp, lq;
        rr_pair(r % (mp - 1), sl - poff[c], mp, lp, lq);
        const int p = mem[cbeg[c] + lp], q = lq < mc ? mem[cbeg[c] + lq] : -1;
        double cr = 1.0, sr = 0.0;
        if (q >= 0) {
          const double apq = A[p * n + q], app = A[p * n + p], aqq = A[q * n + q];
          if (fabs(apq) > fmax(tol_abs, tol_rel * sqrt(fabs(app * aqq)))) {
            // tan of the rotation angle, the smaller root of t^2 + 2 tau t - 1 = 0; one
            // division, one square root and one reciprocal square root on the round's
            // critical path (tau^2 would overflow beyond 1e154: t -> 1 / (2 tau) there)
            const double tau = (aqq - app) / (2.0 * apq);
            const double at = fabs(tau);
            const double t = at > 1e150 ? 0.5 / tau : (tau >= 0 ? 1.0 : -1.0) / (at + sqrt(fma(tau, tau, 1.0)));
            cr = rsqrt(fma(t, t, 1.0));
            sr = t * cr;
            rotated = 1;
          }
        }
        cs[sl] = cr;
        sn[sl] = sr;
        pp[sl] = p;
        qq[sl] = q;
      }
      __syncthreads();
      // A <- J^T A J, one 2x2 block (pair P rows, pair Q columns) per thread iteration, P and Q
      // of one component, P <= Q only: the block (Q, P) is written as the transpose, so A
      // stays exactly symmetric and the FP64 work (the scarce pipe on this chip) is halved
      for (int e = tid; e < nblk; e += kJT) {
        int c = 0;
        while (toff[c + 1] <= e) ++c;
        int P, Q;
        tri_index(e - toff[c], poff[c + 1] - poff[c], P, Q);
        P += poff[c];
        Q += poff[c];
        const double c1 = cs[P], s1 = sn[P], c2 = cs[Q], s2 = sn[Q];
        if (s1 == 0.0 && s2 == 0.0) continue;
        const int p1 = pp[P], q1 = qq[P], p2 = pp[Q], q2 = qq[Q];
        const bool hq1 = q1 >= 0, hq2 = q2 >= 0;
        const double a = A[p1 * n + p2];
        const double b = hq2 ? A[p1 * n + q2] : 0.0;
        const double cc = hq1 ? A[q1 * n + p2] : 0.0;
        const double d = (hq1 && hq2) ? A[q1 * n + q2] : 0.0;
        // rows
        const double ra = c1 * a - s1 * cc, rb = c1 * b - s1 * d;
        const double rc = s1 * a + c1 * cc, rd = s1 * b + c1 * d;
        // columns
        double na = c2 * ra - s2 * rb, nb = s2 * ra + c2 * rb;
        double nc2 = c2 * rc - s2 * rd, nd = s2 * rc + c2 * rd;
        if (P == Q && s1 != 0.0) {
          nb = 0.0;
          nc2 = 0.0;
        }
        A[p1 * n + p2] = na;
        if (hq2) A[p1 * n + q2] = nb;
        if (hq1) A[q1 * n + p2] = nc2;
        if (hq1 && hq2) A[q1 * n + q2] = nd;
        if (P != Q) {
          A[p2 * n + p1] = na;
          if (hq2) A[q2 * n + p1] = nb;
          if (hq1) A[p2 * n + q1] = nc2;
          if (hq1 && hq2) A[q2 * n + q1] = nd;
        }
      }
      // V <- V J, rows of the pair's component only (the others are zero in its columns)
      for (int e = tid; e < nvu; e += kJT) {
        int c = 0;
        while (voff[c + 1] <= e) ++c;
        const int np = poff[c + 1] - poff[c], t = e - voff[c];
        const int row = mem[cbeg[c] + t / np], Q = poff[c] + t % np;
        const double sv = sn[Q];
        if (sv == 0.0) continue;
        const double cv = cs[Q];
        const int p = pp[Q], q = qq[Q];
        const double vp = V[row * n + p], vq = V[row * n + q];
        V[row * n + p] = cv * vp - sv * vq;
        V[row * n + q] = sv * vp + cv * vq;
      }
      __syncthreads();
    }
    if (rotated == 0) break;
    __syncthreads();
  }
  if (tid == 0 && sweep >= max_sweeps && n > 1) atomicAdd(&status[kStNoConv], 1);

  // ---- sort descending (rank = number of larger eigenvalues, ties by index)
  for (int i = tid; i < n; i += kJT) nrm[i] = A[i * n + i];
  __syncthreads();
  for (int i = tid; i < n; i += kJT) {
    // ranked by (value, index) with a NaN taken as -inf: a strict total order, so perm is a
    // permutation whatever the input (a non-finite tensor is reported by the normalisation)
    const double li = nrm[i], ki = li == li ? li : -INFINITY;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double lj = nrm[j], kj = lj == lj ? lj : -INFINITY;
      rank += (kj > ki) || (kj == ki && j < i);
    }
    perm[rank] = i;
    lam[rank] = li;
  }
  __syncthreads();
  for (int i = tid; i < n; i += kJT) jb.lam[i] = lam[i];
  if (tid == 0) {
    double e = 0;
    for (int j = chi; j < n; ++j) e += lam[j];
    *jb.eps = e;
    int nc = 0;
    cstart[nc++] = 0;
    for (int j = 1; j < n; ++j)
      if (lam[j - 1] - lam[j] > cluster_tau * fabs(lam[0])) cstart[nc++] = j;
    cstart[nc] = n;
    ncl = nc;
    int deg = 0;
    for (int c = 0; c < nc; ++c)
      if (cstart[c] < chi && chi < cstart[c + 1]) deg = 1;
    *jb.degenerate = deg;
  }
  __syncthreads();

  // ---- canonical gauge for the first chi columns, written to U (n x chi)
  for (int c = 0; c < ncl; ++c) {
    const int s0 = cstart[c], e0 = cstart[c + 1];
    if (s0 >= chi) break;
    for (int i = tid; i < n; i += kJT) {   // |P_cluster e_i|^2
      double b = 0;
      for (int j = s0; j < e0; ++j) {
        const double v = V[i * n + perm[j]];
        b = fma(v, v, b);
      }
      nrm[i] = b;
    }
    __syncthreads();
    const int tend = min(e0, chi);
    for (int t = s0; t < tend; ++t) {
      double mx = 0;
      for (int i = tid; i < n; i += kJT) mx = fmax(mx, nrm[i]);
      for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
      if ((tid & 31) == 0) red[tid >> 5] = mx;
      __syncthreads();
      if (tid == 0) {
        double m2 = 0;
        for (int w = 0; w < kJT / 32; ++w) m2 = fmax(m2, red[w]);
        int ip = 0;
        for (int i = 0; i < n; ++i)
          if (nrm[i] >= (1.0 - tie_rel) * m2) {
            ip = i;
            break;
          }
        pivot = ip;
        pivval = nrm[ip];
      }
      __syncthreads();
      const int ip = pivot;
      const double inv = 1.0 / sqrt(pivval);
      for (int i = tid; i < n; i += kJT) {
        double g = 0;
        for (int j = s0; j < e0; ++j) g = fma(V[i * n + perm[j]], V[ip * n + perm[j]], g);
        for (int u = s0; u < t; ++u) g -= jb.U[i * chi + u] * jb.U[ip * chi + u];
        jb.U[i * chi + t] = g * inv;
      }
      __threadfence_block();
      __syncthreads();
      for (int i = tid; i < n; i += kJT) {
        const double g = jb.U[i * chi + t];
        nrm[i] -= g * g;
      }
      __syncthreads();
    }
    __syncthreads();
  }
}

// The shared-memory attribute is set once per device: by jacobi_prepare (called when a
// workspace is attached, ahead of any stream capture) or at the first launch on a device.
constexpr int kJacobiMaxDevices = 64;
bool g_jacobi_attr[kJacobiMaxDevices] = {};

cudaError_t jacobi_attr_for_current_device() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kJacobiMaxDevices) return cudaErrorInvalidDevice;
  if (g_jacobi_attr[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           2 * kSmemJacobiN * kSmemJacobiN * (int)sizeof(double));
  if (e == cudaSuccess) g_jacobi_attr[dev] = true;
  return e;
}

void jacobi_prepare() { jacobi_attr_for_current_device(); }

cudaError_t launch_jacobi(const EigPack& jobs, int njobs, int nmax, double cluster_tau, int* status,
                          cudaStream_t st, int max_sweeps, double tie_rel) {
  const int smem_n = nmax <= kSmemJacobiN ? nmax : 0;
  const size_t smem = (size_t)2 * smem_n * smem_n * sizeof(double);
  const cudaError_t e = jacobi_attr_for_current_device();
  if (e != cudaSuccess) return e;
  jacobi_kernel<<<njobs * jobs.batch, kJT, smem, st>>>(jobs, njobs, smem_n > 0 ? 1 : 0, cluster_tau, tie_rel,
                                                      max_sweeps, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------- side choice
template <typename R>
__global__ void __launch_bounds__(256) select_kernel(const __grid_constant__ SelectPack jobs, int njobs,
                                                     double side_rel) {
  // job blockIdx.x % njobs of batch element blockIdx.x / njobs
  const int64_t bidx = blockIdx.x / njobs;
  SelectJob jb = jobs.j[blockIdx.x - bidx * njobs];
  jb.U[0] += bidx * jobs.sU;
  jb.U[1] += bidx * jobs.sU;
  jb.lam0 += bidx * jobs.sLam;
  jb.eps[0] += bidx * jobs.sEps;
  jb.eps[1] += bidx * jobs.sEps;
  jb.degen[0] += bidx * jobs.sDeg;
  jb.degen[1] += bidx * jobs.sDeg;
  jb.U64 += bidx * jobs.sU64;
  jb.Ur = (R*)jb.Ur + bidx * jobs.sUr;
  if (jb.rec_b) jb.rec_b += bidx * jobs.sRec;
  __shared__ double red[8];
  __shared__ int side;
  const int n = jb.n, chi = jb.chi, tid = threadIdx.x;
  if (tid == 0) {
    const double e0 = *jb.eps[0], e1 = *jb.eps[1];
    side = (e0 - e1 > side_rel * (fabs(e0) + fabs(e1)) + 1e-13 * fabs(jb.lam0[0])) ? 1 : 0;
    double* re = jb.rec_eps;
    int* rp = jb.rec_primed;
    int* rd = jb.rec_degen;
    if (jb.rec_b != nullptr) {           // record slot of the current step, read on the device
      const int k = *jb.step < kMaxSteps ? *jb.step : kMaxSteps - 1;
      re = jb.rec_b[k].eps[jb.nu];
      rp = &jb.rec_b[k].primed[jb.nu];
      rd = &jb.rec_b[k].degen[jb.nu];
    }
    re[0] = e0;
    re[1] = e1;
    *rp = side;
    *rd = *jb.degen[side];
  }
  __syncthreads();
  const double* src = jb.U[side];
  for (int e = tid; e < n * chi; e += blockDim.x) jb.U64[e] = src[e];
  __syncthreads();
  // modified Gram-Schmidt, FP64
  for (int j = 0; j < chi; ++j) {
    for (int i = 0; i < j; ++i) {
      double d = 0;
      for (int r = tid; r < n; r += blockDim.x) d = fma(jb.U64[r * chi + i], jb.U64[r * chi + j], d);
      d = block_sum(d, red);
      for (int r = tid; r < n; r += blockDim.x) jb.U64[r * chi + j] -= d * jb.U64[r * chi + i];
      __syncthreads();
    }
    double q = 0;
    for (int r = tid; r < n; r += blockDim.x) q = fma(jb.U64[r * chi + j], jb.U64[r * chi + j], q);
    q = block_sum(q, red);
    const double inv = 1.0 / sqrt(q);
    for (int r = tid; r < n; r += blockDim.x) jb.U64[r * chi + j] *= inv;
    __syncthreads();
  }
  R* ur = (R*)jb.Ur;
  for (int e = tid; e < n * chi; e += blockDim.x) ur[e] = (R)jb.U64[e];
}

template <typename R>
cudaError_t launch_select(const SelectPack& jobs, int njobs, double side_rel, cudaStream_t st) {
  select_kernel<R><<<njobs * jobs.batch, 256, 0, st>>>(jobs, njobs, side_rel);
  return cudaGetLastError();
}
template cudaError_t launch_select<double>(const SelectPack&, int, double, cudaStream_t);
template cudaError_t launch_select<float>(const SelectPack&, int, double, cudaStream_t);

}  // namespace hotrg
