// hotrg.cu - C ABI and step orchestration of the HOTRG library (include/hotrg.h).
//
// One coarse-graining step along mu (Fig. 1 of arXiv:1911.12954), for each batch
// element, as a fixed sequence of stream-ordered launches with no host synchronisation:
//   1. Gram halves on both sides of the three transverse legs (12 split-K jobs, one
//      launch), chunk reduction, merge into six D_nu^2 x D_nu^2 FP64 Gram matrices.
//   2. Jacobi eigensolver on the six matrices (one launch), canonical gauge, then the
//      side choice + Gram-Schmidt per direction (one launch).
//   3. Block-spin contraction (the O(D^15) part, Sec. 2): the transverse direction whose
//      closing is cheapest is c, the others a and b. For each slice of X (new a leg):
//        A[(X Y c1 c1' mu1), (a2 b2 a1' b1' k)] = T1 x_{a1} U^a x_{b1} U^b   (two passes)
//        B[(X' Y' c2 c2' mu2'), (a2 b2 a1' b1' k)] = T2 x_{a2'} U^a x_{b2'} U^b
//        C = A B^T                                                        (the GEMM)
//        T'[X, X', Y, Y', Z, Z', mu1, mu2'] = C x_{(c1 c2)} U^c x_{(c1' c2')} U^c
//      Impure tensors: S' = (C(S,T) + C(T,S)) / 2, M_1 = C(S,S), M' = (C(M,T) + C(T,M)) / 2.
//   4. c = ||T'||_F (FP64), ln c / 2^k accumulated, T', S', M' divided by c.
// Tensors are stored row-major over legs [x, x', y, y', z, z', t, t'].
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "hotrg.h"

using namespace hotrg;

namespace {

thread_local std::string g_last_error;

}  // namespace

void hotrg::set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

namespace {

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Sizes of one step (elements), derived from the bond dimensions before the step.
struct StepPlan {
  int mu, a, b, c;
  int D[4];
  int chi[4];
  int newD[4];
  int64_t E, Enew;        // tensor elements before / after
  int64_t rowsA_full;     // xs = chi_a
  int64_t rowsB;          // chi_a chi_b Dc^2 Dmu
  int64_t K;              // Da^2 Db^2 Dmu = P Kp
  // GEMM operands in K panels: element (row, k = p Kp + kin) at [(p rows + row) kps + kin];
  // the panel holds the last `ksuf` of the summed legs (a2, b2, a1', b1', k)
  int ksuf;
  int64_t Kp, kps, P;
  int xs;                 // X values per slice (rows of A and C)
  int xs2;                // X' values per slice (rows of B, columns of C)
  // Gram
  int R[4];               // rows of the half-Gram per direction = D_nu D_mu
  int Rmax, nmax, nchunks;
  int batch;              // batch elements whose isometry stages run together
  int ne;                 // batch elements contracted together (one group of launches)
  int gemm_opt;           // tensor-core GEMM pipeline option of this step (-1: the context's)
  bool tuned;             // closing direction and pipeline taken from the autotuner's cache
  double main_flops, total_flops;
};

struct Layout {
  // persistent
  size_t status, step, lnz, cval, trace, rec, beta, hfield, U64, Ur, tensors;
  int64_t cap;            // elements per tensor slot
  size_t persistent_end;
};

}  // namespace

struct hotrg_ctx {
  int batch = 1, dcut_max = 2, prec = HOTRG_FP64, impure = 0;
  int impure_active = 0;
  size_t rsize = 8;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  int64_t cap_planned = 0;
  Layout L{};
  bool ready = false;        // workspace laid out
  bool initialised = false;  // tensors exist
  int sticky = 0;
  int k = 0;
  int dims[4] = {2, 2, 2, 2};
  int mu_hist[kMaxSteps];
  int slices_hist[kMaxSteps][2];
  int dims_hist[kMaxSteps][4];
  int cur = 0;               // which tensor buffer holds the current tensors
  int last_chi[4] = {0, 0, 0, 0};
  int last_Dold[4] = {0, 0, 0, 0};
  int last_mu = -1;
  std::vector<double> h_host;
  int jacobi_sweeps = kJacobiMaxSweeps;
  int gemm_variant = 0;
  bool use_graphs = false;
  bool autotune = false;
  int group_max = 0;           // most temperatures contracted together (0: as many as fit)
  int maxnorm = 1;             // FP16X3 operand scaling: a ScaleMode (0: the fixed 2^14)
  StepPlan last_plan{};        // plan of the last step (its last block's operands stay in scratch)
  int last_kstep = -1;         // steps done before it (-1: none since the last init)
  int group_hist[kMaxSteps];   // temperatures contracted together at each step
  int c_hist[kMaxSteps];       // closing direction of each step
  int opt_hist[kMaxSteps];     // GEMM pipeline option of each step (-1: CUDA cores)
  int tuned_hist[kMaxSteps];   // plan from the autotuner's cache
  uint64_t tune_timed = 0;     // step shapes timed by this context
  uint64_t tune_hits = 0;      // steps whose plan came from the cache
  struct GraphEntry {
    cudaGraphExec_t exec;
    uint64_t launches;
  };
  std::map<std::string, GraphEntry> graphs;   // captured steps, keyed by everything a step's launches depend on
  // launch accounting
  uint64_t launches = 0;
  bool profiling = false;
  std::vector<cudaEvent_t> ev;   // pairs (start, stop) of timed GEMM launches
  size_t ev_used = 0;
  uint64_t gemm_launches = 0;
  double gemm_flops = 0;
  void drop_graphs() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second.exec);
    graphs.clear();
  }
  ~hotrg_ctx() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    drop_graphs();
  }
};

namespace {

hotrg_status cuda_fail(hotrg_ctx* ctx, cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  if (ctx) ctx->sticky = HOTRG_ECUDA;
  return HOTRG_ECUDA;
}

#define CK(call, where)                                   \
  do {                                                    \
    cudaError_t e__ = (call);                             \
    if (e__ != cudaSuccess) return cuda_fail(ctx, e__, where); \
  } while (0)


// A launcher call that issues `n` kernels.
#define LK(n, call, where)                                \
  do {                                                    \
    CK(call, where);                                      \
    ctx->launches += (n);                                 \
  } while (0)

// Largest element offset a TTM launch touches in its input, isometry and output (all
// strides are non-negative); launches that would leave their buffers are refused.
struct Extent {
  int64_t in, u, out;
};
Extent ttm_extent(const TTMArgs& a) {
  Extent e{0, 0, 0};
  for (int i = 0; i < a.rank; ++i) {
    e.in += (a.dims[i] - 1) * a.in_st[i];
    e.u += (a.dims[i] - 1) * a.u_st[i];
    e.out += (a.dims[i] - 1) * a.out_st[i];
  }
  e.in += (a.J1 - 1) * a.in_sj1 + (a.J2 - 1) * a.in_sj2;
  e.u += (a.J1 - 1) * a.u_sj1 + (a.J2 - 1) * a.u_sj2;
  return e;
}

thread_local int64_t g_lim_in = -1, g_lim_u = -1, g_lim_out = -1;  // elements available

template <typename R>
inline cudaError_t launch_ttm_r(const R* in, const R* U, R* out, R* lo, const TTMArgs& a, int mode, cudaStream_t st) {
  const Extent e = ttm_extent(a);
  for (int i = 0; i < a.rank; ++i)
    if (a.in_st[i] < 0 || a.u_st[i] < 0 || a.out_st[i] < 0) return cudaErrorInvalidValue;
  if (e.in >= g_lim_in || (U && e.u >= g_lim_u) || e.out >= g_lim_out) {
    g_last_error = "TTM launch refused: extent outside its buffer";
    return cudaErrorInvalidValue;
  }
  // batch elements must not overlap: each element's stride covers one element's buffer
  if (a.nb > 1 && (a.in_bs < g_lim_in || (U && a.u_bs < g_lim_u) || a.out_bs < g_lim_out)) {
    g_last_error = "TTM launch refused: batch stride shorter than one element's buffer";
    return cudaErrorInvalidValue;
  }
  return launch_ttm<R, R, R>(in, U, out, lo, a, mode, st);
}

// Per-element strides of a group of batch elements contracted together (element e of the
// group at base + e * stride, in elements of each buffer's type; operand planes in operand
// elements).
struct ElemStrides {
  int ne = 1;
  int64_t T = 0;     // tensors (current and next buffer): the slot capacity
  int64_t U = 0;     // isometries
  int64_t O1 = 0;    // first half-contraction pass
  int64_t op = 0;    // GEMM operand planes (all tensors of one element)
  int64_t C = 0;     // GEMM outputs (all tensors of one element)
  int64_t O3 = 0;    // first closing pass
};

// Phases of an operand build (build_A, build_B): the first half-contraction pass into O1, the
// max pass of the second (largest |operand| into the scratch word, for max-norm scaling), the
// second pass writing the operand planes.
enum BuildPhase { kPass1 = 1, kPassMax = 2, kPass2 = 4 };

// How an operand side's max-norm scale is found (the word amax of the side):
//  * kScaleBound (fp16 planes): the first pass records sqrt(J) times its largest |output|,
//    J the length of the second pass's contraction. The second pass computes A[f, r] =
//    sum_j U[j, r] O1[f, j] with U[., r] part of a column of an isometry (norm <= 1), so by
//    Cauchy-Schwarz |A[f, r]| <= ||O1[f, .]||_2 <= sqrt(J) max |O1|: a bound of the operand's
//    largest magnitude at no extra pass, at most log2(sqrt(J)) bits above it;
//  * kScaleExact (FP64-grade integer slices, whose precision is fixed-point relative to the
//    scale): a max pass computes the second pass's outputs once more and records their
//    exact largest magnitude.
enum ScaleMode { kScaleNone = 0, kScaleBound = 1, kScaleExact = 2 };

inline TTMArgs batched(TTMArgs t, int ne, int64_t in_bs, int64_t u_bs, int64_t out_bs) {
  t.nb = ne;
  t.in_bs = in_bs;
  t.u_bs = u_bs;
  t.out_bs = out_bs;
  return t;
}
inline void ttm_limits(int64_t in, int64_t u, int64_t out) {
  g_lim_in = in;
  g_lim_u = u;
  g_lim_out = out;
}

int64_t tensor_elems(const int D[4]) {
  int64_t e = 1;
  for (int n = 0; n < 4; ++n) e *= (int64_t)D[n] * D[n];
  return e;
}

// Tensor-core modes split each operand into hi + lo planes; operand element size in bytes.
inline bool tc_mode(int prec) { return prec == HOTRG_TF32X3 || prec == HOTRG_FP16X3; }
// tensors stored in FP64 (FP64 and FP64-grade tensor-core modes)
inline bool f64_store(int prec) { return prec == HOTRG_FP64 || prec == HOTRG_FP64OZ; }
// GEMM operands in K panels with 128-byte rows (every tensor-core mode)
inline bool panel_mode(int prec) { return tc_mode(prec) || prec == HOTRG_FP64OZ; }
// operand planes: hi + lo (FP16X3, TF32X3), the integer slices (FP64OZ), or one
inline int operand_planes(int prec) { return tc_mode(prec) ? 2 : (prec == HOTRG_FP64OZ ? kOzSlices : 1); }
// TTM pass that writes the GEMM operand planes
inline int split_mode(int prec) {
  return prec == HOTRG_FP16X3 ? kTTMSplitF16 : (prec == HOTRG_FP64OZ ? kTTMSplitOz : kTTMSplitTF32);
}
inline size_t operand_size(int prec) {
  return prec == HOTRG_FP64 ? 8 : ((prec == HOTRG_FP16X3 || prec == HOTRG_FP64OZ) ? 2 : 4);
}

double plan_main_flops(const int D[4], const int chi[4], int mu, int a, int b, int c) {
  const double rows = (double)chi[a] * chi[b] * D[c] * D[c] * D[mu];
  const double K = (double)D[a] * D[a] * D[b] * D[b] * D[mu];
  return 2.0 * rows * rows * K;
}

// force_c >= 0 (a transverse direction) fixes the closing direction; otherwise the one
// with the fewest flops is taken.
StepPlan make_plan(const int D[4], int mu, int dcut, int prec, int batch = 1, int force_c = -1) {
  StepPlan p{};
  p.mu = mu;
  p.batch = batch;
  p.ne = 1;
  p.gemm_opt = -1;
  for (int n = 0; n < 4; ++n) {
    p.D[n] = D[n];
    p.chi[n] = (n == mu) ? D[n] : std::min(D[n] * D[n], dcut);
    p.newD[n] = p.chi[n];
  }
  int tr[3], t = 0;
  for (int n = 0; n < 4; ++n)
    if (n != mu) tr[t++] = n;
  // closing direction: the one that minimises the main contraction (ties: last)
  double best = -1;
  int bc = tr[2];
  for (int i = 0; i < 3; ++i) {
    const int c = tr[i];
    int ab[2], q = 0;
    for (int j = 0; j < 3; ++j)
      if (j != i) ab[q++] = tr[j];
    const double f = plan_main_flops(D, p.chi, mu, ab[0], ab[1], c);
    if (force_c >= 0 ? c == force_c : (best < 0 || f <= best)) {
      best = f;
      bc = c;
    }
  }
  p.c = bc;
  int q = 0, ab[2];
  for (int i = 0; i < 3; ++i)
    if (tr[i] != bc) ab[q++] = tr[i];
  p.a = ab[0];
  p.b = ab[1];
  p.E = tensor_elems(D);
  p.Enew = tensor_elems(p.newD);
  const int Da = D[p.a], Db = D[p.b], Dc = D[p.c], Dm = D[mu];
  p.rowsB = (int64_t)p.chi[p.a] * p.chi[p.b] * Dc * Dc * Dm;
  p.rowsA_full = p.rowsB;
  p.K = (int64_t)Da * Da * Db * Db * Dm;
  {
    // tensor-core operands: the widest panel of trailing summed legs up to 4096 values, so
    // one box of 128 rows stays within 2 MB; CUDA-core operands: one panel, plain rows
    const int64_t kd[5] = {Da, Db, Da, Db, Dm};
    int64_t prod = 1;
    p.ksuf = 0;
    for (int q = 1; q <= 5; ++q) {
      const int64_t next = prod * kd[5 - q];
      if (panel_mode(prec) && next > 4096 && q > 1) break;
      prod = next;
      p.ksuf = q;
    }
    p.Kp = prod;
    // tensor-core operands: panel rows start on 128-byte boundaries, so the 64-byte rows the
    // GEMM's copies fetch never straddle an L2 line (unaligned strides cost D = 10 and 13 a
    // third of their throughput); CUDA-core operands: 16-byte rows
    const int64_t al = panel_mode(prec) ? 128 / (int64_t)operand_size(prec) : 4;
    p.kps = (p.Kp + al - 1) / al * al;
    p.P = p.K / p.Kp;
  }
  p.xs = p.chi[p.a];
  p.xs2 = p.chi[p.a];
  p.Rmax = 0;
  p.nmax = 0;
  for (int n = 0; n < 4; ++n) {
    p.R[n] = D[n] * Dm;
    if (n != mu) {
      p.Rmax = std::max(p.Rmax, p.R[n]);
      p.nmax = std::max(p.nmax, D[n] * D[n]);
    }
  }
  const int64_t Kg = p.E / p.Rmax;
  int64_t nc = (Kg + 511) / 512;
  if (nc > 256) nc = 256;
  if (nc < 1) nc = 1;
  // keep the split-K partials of all batch elements under 256 MB
  const int64_t per = (int64_t)batch * kMaxGramJobs * p.Rmax * p.Rmax * 8;
  while (nc > 1 && nc * per > (256LL << 20)) nc /= 2;
  p.nchunks = (int)nc;
  p.main_flops = best;
  // every other product of the step, counted as 2 flops per multiply-add
  const double Ed = (double)p.E, rA = (double)p.rowsA_full, rB = (double)p.rowsB, Kd = (double)p.K;
  double f = best;
  f += 2.0 * Da * p.chi[p.a] * Ed + 2.0 * Db * rA * Kd;            // A = T x U^a x U^b
  f += 2.0 * Da * p.chi[p.a] * Ed + 2.0 * Db * rB * Kd;            // B = T x U^a x U^b
  f += 2.0 * p.chi[p.c] * rA * rB + 2.0 * Dc * Dc * (double)p.Enew; // closing with U^c twice
  for (int n = 0; n < 4; ++n)
    if (n != mu) f += 8.0 * p.R[n] * Ed + 2.0 * 2.0 * pow((double)D[n], 4) * Dm * Dm;  // Gram
  p.total_flops = f;
  return p;
}

int ntensors(int impure) { return (impure & HOTRG_IMPURE_SIGMASIGMA) ? 3 : ((impure & HOTRG_IMPURE_SIGMA) ? 2 : 1); }

// Scratch bytes of one step with slice sizes xs (new X) and xs2 (new X').
struct Scratch {
  size_t gpart, npart, gA, G, jwork, lam, eps, degen, Uside;
  size_t O1A, A, Alo, O1B, B, Blo, C, O3;
  size_t amax;            // operand magnitude bounds of the current A and B per element (max-norm scaling)
  size_t stats;           // counters of hotrg_split_stats
  size_t total;
};

Scratch scratch_layout(const StepPlan& p, int xs, int xs2, int prec, int impure, size_t rs) {
  Scratch s{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  const int nt = ntensors(impure);
  // isometry stage: one copy per batch element (all elements run it together)
  const size_t nb = (size_t)p.batch;
  s.gpart = take(nb * kMaxGramJobs * p.nchunks * p.Rmax * p.Rmax * 8);
  s.npart = take(nb * kNormPartials * 8);
  s.gA = take(nb * kMaxGramJobs * p.Rmax * p.Rmax * 8);
  s.G = take(nb * 6 * p.nmax * p.nmax * 8);
  s.jwork = take(p.nmax > kJacobiSmemN ? nb * 6 * 2 * p.nmax * p.nmax * 8 : 0);
  s.lam = take(nb * 6 * p.nmax * 8);
  s.eps = take(nb * 6 * 8);
  s.degen = take(nb * 6 * 4);
  s.Uside = take(nb * 6 * p.nmax * kMaxLeg * 8);
  const int64_t rowsA = (int64_t)xs * p.chi[p.b] * p.D[p.c] * p.D[p.c] * p.D[p.mu];
  const int64_t rowsB = (int64_t)xs2 * p.chi[p.b] * p.D[p.c] * p.D[p.c] * p.D[p.mu];
  const bool split = tc_mode(prec);
  const size_t os = operand_size(prec) * (prec == HOTRG_FP64OZ ? kOzSlices : 1);   // the slices of one operand
  // contraction: one copy per element of a group (p.ne elements contracted together)
  const size_t ne = (size_t)p.ne;
  s.O1A = take(ne * nt * xs * p.E * rs);              // first pass of every tensor's A
  s.A = take(ne * nt * p.P * rowsA * p.kps * os);
  s.Alo = split ? take(ne * nt * p.P * rowsA * p.kps * os) : 0;
  s.O1B = take(ne * nt * xs2 * p.E * rs);
  s.B = take(ne * nt * p.P * rowsB * p.kps * os);
  s.Blo = split ? take(ne * nt * p.P * rowsB * p.kps * os) : 0;
  s.C = take(ne * nt * rowsA * rowsB * rs);
  s.O3 = take(ne * (size_t)(rowsA * rowsB / (p.D[p.c] * p.D[p.c]) * p.chi[p.c]) * rs);
  s.amax = take(2 * ne * nt * sizeof(unsigned));   // A side, then B side: per element (and tensor)
  s.stats = take(4 * 3 * sizeof(unsigned long long));   // hotrg_split_stats counters
  s.total = off;
  return s;
}

Layout persistent_layout(int batch, int64_t cap, int impure, size_t rs) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  L.status = take(kStWords * 4);
  L.step = take(sizeof(int));
  L.lnz = take(batch * 8);
  L.cval = take(batch * 8);
  L.trace = take(4 * batch * 8);   // Tr T, Tr S, Tr M, X indicator
  L.rec = take((size_t)batch * kMaxSteps * sizeof(DevRecord));
  L.beta = take(batch * 8);
  L.hfield = take(batch * 8);
  L.U64 = take((size_t)batch * 4 * kMaxGramN * kMaxLeg * 8);
  L.Ur = take((size_t)batch * 4 * kMaxGramN * kMaxLeg * rs);
  L.cap = cap;
  L.tensors = take((size_t)ntensors(impure) * 2 * batch * cap * rs);
  L.persistent_end = off;
  return L;
}

// canonical row-major strides of a rank-8 tensor with bond dims D
void canon_strides(const int D[4], int64_t st[8]) {
  int64_t s = 1;
  for (int leg = 7; leg >= 0; --leg) {
    st[leg] = s;
    s *= D[leg / 2];
  }
}

template <typename R>
R* tensor_ptr(hotrg_ctx* ctx, int which, int buf, int b) {
  R* base = (R*)(ctx->ws + ctx->L.tensors);
  return base + (((int64_t)which * 2 + buf) * ctx->batch + b) * ctx->L.cap;
}

// Build a TTMArgs. `dims` in output iteration order, with per-dim strides.
struct Dim {
  int64_t n, in, u, out;
};
TTMArgs make_ttm(const std::vector<Dim>& d, int J1, int64_t in_sj1, int64_t u_sj1, int J2, int64_t in_sj2,
                 int64_t u_sj2, double alpha, double beta) {
  TTMArgs a{};
  a.rank = (int)d.size();
  a.J1 = J1;
  a.J2 = J2;
  a.in_sj1 = in_sj1;
  a.u_sj1 = u_sj1;
  a.in_sj2 = in_sj2;
  a.u_sj2 = u_sj2;
  a.alpha = alpha;
  a.beta = beta;
  a.nb = 1;
  a.amax_mul = 1.0f;
  a.amax_bs = 1;
  for (int i = 0; i < a.rank; ++i) {
    a.dims[i] = d[i].n;
    a.in_st[i] = d[i].in;
    a.u_st[i] = d[i].u;
    a.out_st[i] = d[i].out;
  }
  // inner part: trailing dims while the product stays <= 2^16 (at least one dim)
  int64_t inner = 1;
  int rin = 0;
  for (int i = a.rank - 1; i >= 0; --i) {
    if (rin > 0 && inner * d[i].n > 65536) break;
    inner *= d[i].n;
    ++rin;
  }
  a.rin = rin;
  a.inner = inner;
  int64_t outer = 1;
  for (int i = 0; i < a.rank - rin; ++i) outer *= d[i].n;
  a.outer = outer;
  return a;
}

// Row-major strides of a list of sizes.
std::vector<int64_t> rm_strides(const std::vector<int64_t>& n) {
  std::vector<int64_t> s(n.size());
  int64_t acc = 1;
  for (int i = (int)n.size() - 1; i >= 0; --i) {
    s[i] = acc;
    acc *= n[i];
  }
  return s;
}

// Output strides of the 10 legs of a GEMM operand (rows: the 5 row legs, then the summed
// legs a2, b2, a1', b1', k) in the K-panel layout with `rows` rows per panel.
void operand_strides(const StepPlan& p, const std::vector<int64_t>& rn, int64_t out[10]) {
  const std::vector<int64_t> rs = rm_strides(rn);
  int64_t rows = 1;
  for (int64_t x : rn) rows *= x;
  for (int i = 0; i < 5; ++i) out[i] = rs[i] * p.kps;
  const int Da = p.D[p.a], Db = p.D[p.b], Dm = p.D[p.mu];
  const int64_t kd[5] = {Da, Db, Da, Db, Dm};
  const int split = 5 - p.ksuf;  // legs [0, split) select the panel, [split, 5) lie inside it
  int64_t inner = 1;
  for (int j = 4; j >= split; --j) {
    out[5 + j] = inner;
    inner *= kd[j];
  }
  int64_t outer = rows * p.kps;
  for (int j = split - 1; j >= 0; --j) {
    out[5 + j] = outer;
    outer *= kd[j];
  }
}

template <typename R>
hotrg_status build_A(hotrg_ctx* ctx, const StepPlan& p, const R* P, const R* Ua, const R* Ub, int x0, int xs,
                     R* O1, R* A, R* Alo, cudaStream_t st, const ElemStrides& es, unsigned* amax, int amax_bs,
                     int scale, int phases) {
  const int mu = p.mu, a = p.a, b = p.b, c = p.c;
  const int Da = p.D[a], Db = p.D[b], Dc = p.D[c], Dm = p.D[mu];
  const int ca = p.chi[a], cb = p.chi[b];
  int64_t ts[8];
  canon_strides(p.D, ts);
  // O1[X, b1, c1, c1', mu1, a2, a1', b1', k] = sum_a1 U^a[a1, a2, X] P[...]
  const std::vector<int64_t> on = {xs, Db, Dc, Dc, Dm, Da, Da, Db, Dm};
  const std::vector<int64_t> os = rm_strides(on);
  {
    std::vector<Dim> d = {
        {xs, 0, 1, os[0]},                       // X   (U col X, offset x0 on U)
        {Db, ts[2 * b], 0, os[1]},               // b1
        {Dc, ts[2 * c], 0, os[2]},               // c1
        {Dc, ts[2 * c + 1], 0, os[3]},           // c1'
        {Dm, ts[2 * mu], 0, os[4]},              // mu1
        {Da, 0, ca, os[5]},                      // a2
        {Da, ts[2 * a + 1], 0, os[6]},           // a1'
        {Db, ts[2 * b + 1], 0, os[7]},           // b1'
        {Dm, ts[2 * mu + 1], 0, os[8]},          // k = T1.mu'
    };
    TTMArgs t = batched(make_ttm(d, Da, ts[2 * a], (int64_t)Da * ca, 1, 0, 0, 1.0, 0.0), es.ne, es.T, es.U, es.O1);
    ttm_limits(p.E, (int64_t)Da * Da * ca - x0, (int64_t)xs * p.E);
    const bool bound = amax && scale == kScaleBound;   // the second pass contracts b1: J = Db
    if (bound) {
      t.amax = amax;
      t.amax_mul = sqrtf((float)Db);
      t.amax_bs = amax_bs;
    }
    if (phases & kPass1) LK(1, launch_ttm_r<R>(P, Ua + x0, O1, nullptr, t, bound ? kTTMStoreMax : kTTMStore, st), "ttm A1");
  }
  // A[(X Y c1 c1' mu1), (a2 b2 a1' b1' k)] = sum_b1 U^b[b1, b2, Y] O1[X, b1, ...]
  {
    int64_t o[10];
    operand_strides(p, {xs, cb, Dc, Dc, Dm}, o);
    std::vector<Dim> d = {
        {xs, os[0], 0, o[0]},   // X
        {cb, 0, 1, o[1]},       // Y
        {Dc, os[2], 0, o[2]},   // c1
        {Dc, os[3], 0, o[3]},   // c1'
        {Dm, os[4], 0, o[4]},   // mu1
        {Da, os[5], 0, o[5]},   // a2
        {Db, 0, cb, o[6]},      // b2
        {Da, os[6], 0, o[7]},   // a1'
        {Db, os[7], 0, o[8]},   // b1'
        {Dm, os[8], 0, o[9]},   // k
    };
    TTMArgs t = make_ttm(d, Db, os[1], (int64_t)Db * cb, 1, 0, 0, 1.0, 0.0);
    const int mode = !Alo ? kTTMStore : split_mode(ctx->prec);
    ttm_limits((int64_t)xs * p.E, (int64_t)Db * Db * cb, p.P * ((int64_t)xs * cb * Dc * Dc * Dm) * p.kps);
    t = batched(t, es.ne, es.O1, es.U, es.op);
    t.amax = amax;   // max-norm scaling (nullptr: none): the max pass writes it, the split reads it
    t.amax_bs = amax_bs;
    if ((phases & kPassMax) && amax && scale == kScaleExact)
      LK(1, launch_ttm_r<R>(O1, Ub, A, Alo, t, kTTMMaxAbs, st), "ttm A max");
    if (phases & kPass2) LK(1, launch_ttm_r<R>(O1, Ub, A, Alo, t, mode, st), "ttm A2");
  }
  return HOTRG_OK;
}

template <typename R>
hotrg_status build_B(hotrg_ctx* ctx, const StepPlan& p, const R* Q, const R* Ua, const R* Ub, int x0, int xs,
                     R* O1, R* B, R* Blo, cudaStream_t st, const ElemStrides& es, unsigned* amax, int amax_bs,
                     int scale, int phases) {
  const int mu = p.mu, a = p.a, b = p.b, c = p.c;
  const int Da = p.D[a], Db = p.D[b], Dc = p.D[c], Dm = p.D[mu];
  const int ca = p.chi[a], cb = p.chi[b];
  int64_t ts[8];
  canon_strides(p.D, ts);
  // O1[X', b2', c2, c2', mu2', a2, b2, a1', k] = sum_a2' U^a[a1', a2', X'] Q[...], X' in [x0, x0 + xs)
  const std::vector<int64_t> on = {xs, Db, Dc, Dc, Dm, Da, Db, Da, Dm};
  const std::vector<int64_t> os = rm_strides(on);
  {
    std::vector<Dim> d = {
        {xs, 0, 1, os[0]},                       // X'  (U col X', offset x0 on U)
        {Db, ts[2 * b + 1], 0, os[1]},           // b2'
        {Dc, ts[2 * c], 0, os[2]},               // c2
        {Dc, ts[2 * c + 1], 0, os[3]},           // c2'
        {Dm, ts[2 * mu + 1], 0, os[4]},          // mu2'
        {Da, ts[2 * a], 0, os[5]},               // a2
        {Db, ts[2 * b], 0, os[6]},               // b2
        {Da, 0, (int64_t)Da * ca, os[7]},        // a1'
        {Dm, ts[2 * mu], 0, os[8]},              // k = T2.mu
    };
    TTMArgs t = batched(make_ttm(d, Da, ts[2 * a + 1], ca, 1, 0, 0, 1.0, 0.0), es.ne, es.T, es.U, es.O1);
    ttm_limits(p.E, (int64_t)Da * Da * ca - x0, (int64_t)xs * p.E);
    const bool bound = amax && scale == kScaleBound;   // the second pass contracts b1': J = Db
    if (bound) {
      t.amax = amax;
      t.amax_mul = sqrtf((float)Db);
      t.amax_bs = amax_bs;
    }
    if (phases & kPass1) LK(1, launch_ttm_r<R>(Q, Ua + x0, O1, nullptr, t, bound ? kTTMStoreMax : kTTMStore, st), "ttm B1");
  }
  {
    int64_t o[10];
    operand_strides(p, {xs, cb, Dc, Dc, Dm}, o);
    std::vector<Dim> d = {
        {xs, os[0], 0, o[0]},                   // X'
        {cb, 0, 1, o[1]},                       // Y'
        {Dc, os[2], 0, o[2]},                   // c2
        {Dc, os[3], 0, o[3]},                   // c2'
        {Dm, os[4], 0, o[4]},                   // mu2'
        {Da, os[5], 0, o[5]},                   // a2
        {Db, os[6], 0, o[6]},                   // b2
        {Da, os[7], 0, o[7]},                   // a1'
        {Db, 0, (int64_t)Db * cb, o[8]},        // b1'
        {Dm, os[8], 0, o[9]},                   // k
    };
    TTMArgs t = make_ttm(d, Db, os[1], cb, 1, 0, 0, 1.0, 0.0);
    const int mode = !Blo ? kTTMStore : split_mode(ctx->prec);
    ttm_limits((int64_t)xs * p.E, (int64_t)Db * Db * cb, p.P * ((int64_t)xs * cb * Dc * Dc * Dm) * p.kps);
    t = batched(t, es.ne, es.O1, es.U, es.op);
    t.amax = amax;   // max-norm scaling (nullptr: none): the max pass writes it, the split reads it
    t.amax_bs = amax_bs;
    if ((phases & kPassMax) && amax && scale == kScaleExact)
      LK(1, launch_ttm_r<R>(O1, Ub, B, Blo, t, kTTMMaxAbs, st), "ttm B max");
    if (phases & kPass2) LK(1, launch_ttm_r<R>(O1, Ub, B, Blo, t, mode, st), "ttm B2");
  }
  return HOTRG_OK;
}

// T'[slice] = C x_{(c1 c2)} U^c x_{(c1' c2')} U^c, written into the canonical layout.
template <typename R>
hotrg_status close_C(hotrg_ctx* ctx, const StepPlan& p, const R* C, const R* Uc, int x0, int xs, int x20, int xs2,
                     R* O3, R* Tn, cudaStream_t st, const ElemStrides& es) {
  const int mu = p.mu, a = p.a, b = p.b, c = p.c;
  const int Dc = p.D[c], Dm = p.D[mu];
  const int cb = p.chi[b], cc = p.chi[c];
  // C block: rows m = (X, Y, c1, c1', mu1), X in [x0, x0 + xs); columns n = (X', Y', c2, c2', mu2'),
  // X' in [x20, x20 + xs2); row-major with N = its column count
  const int64_t N = (int64_t)xs2 * cb * Dc * Dc * Dm;
  const std::vector<int64_t> mn = {xs, cb, Dc, Dc, Dm};
  const std::vector<int64_t> ms = rm_strides(mn);
  const std::vector<int64_t> nn = {xs2, cb, Dc, Dc, Dm};
  const std::vector<int64_t> ns = rm_strides(nn);
  // O3[Z, X, Y, c1', mu1, X', Y', c2', mu2']
  const std::vector<int64_t> on = {cc, xs, cb, Dc, Dm, xs2, cb, Dc, Dm};
  const std::vector<int64_t> os = rm_strides(on);
  {
    std::vector<Dim> d = {
        {cc, 0, 1, os[0]},              // Z
        {xs, ms[0] * N, 0, os[1]},      // X
        {cb, ms[1] * N, 0, os[2]},      // Y
        {Dc, ms[3] * N, 0, os[3]},      // c1'
        {Dm, ms[4] * N, 0, os[4]},      // mu1
        {xs2, ns[0], 0, os[5]},         // X'
        {cb, ns[1], 0, os[6]},          // Y'
        {Dc, ns[3], 0, os[7]},          // c2'
        {Dm, ns[4], 0, os[8]},          // mu2'
    };
    TTMArgs t = make_ttm(d, Dc, ms[2] * N, (int64_t)Dc * cc, Dc, ns[2], cc, 1.0, 0.0);
    ttm_limits((int64_t)xs * cb * Dc * Dc * Dm * N, (int64_t)Dc * Dc * cc, on[0] * os[0]);
    LK(1, launch_ttm_r<R>(C, Uc, O3, nullptr, batched(t, es.ne, es.C, es.U, es.O3), kTTMStore, st), "ttm close1");
  }
  {
    int64_t tn[8];
    canon_strides(p.newD, tn);
    // output iteration in canonical order of the new tensor, restricted to the X slice
    int64_t sizes[8], in_st[8], u_st[8];
    for (int n = 0; n < 4; ++n) {
      for (int pr = 0; pr < 2; ++pr) {
        const int leg = 2 * n + pr;
        int64_t sz = p.newD[n], in = 0, u = 0;
        if (n == a) {
          if (pr == 0) {
            sz = xs;
            in = os[1];
          } else {
            sz = xs2;
            in = os[5];
          }
        } else if (n == b) {
          in = pr == 0 ? os[2] : os[6];
        } else if (n == c) {
          if (pr == 0) in = os[0];
          else u = 1;                       // Z' from U^c column
        } else {                            // mu
          in = pr == 0 ? os[4] : os[8];
        }
        sizes[leg] = sz;
        in_st[leg] = in;
        u_st[leg] = u;
      }
    }
    std::vector<Dim> d;
    for (int leg = 0; leg < 8; ++leg) d.push_back({sizes[leg], in_st[leg], u_st[leg], tn[leg]});
    TTMArgs t = make_ttm(d, Dc, os[3], (int64_t)Dc * cc, Dc, os[7], cc, 1.0, 0.0);
    R* out = Tn + (int64_t)x0 * tn[2 * a] + (int64_t)x20 * tn[2 * a + 1];
    ttm_limits(on[0] * os[0], (int64_t)Dc * Dc * cc, p.Enew - (int64_t)x0 * tn[2 * a] - (int64_t)x20 * tn[2 * a + 1]);
    LK(1, launch_ttm_r<R>(O3, Uc, out, nullptr, batched(t, es.ne, es.O3, es.U, es.T), kTTMStore, st), "ttm close2");
  }
  return HOTRG_OK;
}

// Records a profiling event pair around one GEMM launch (eager steps only).
struct GemmTimer {
  hotrg_ctx* ctx;
  cudaStream_t st;
  cudaEvent_t e1 = nullptr;
  hotrg_status start() {
    if (!ctx->profiling || ctx->use_graphs) return HOTRG_OK;
    while (ctx->ev.size() < ctx->ev_used + 2) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e), "event create");
      ctx->ev.push_back(e);
    }
    cudaEvent_t e0 = ctx->ev[ctx->ev_used];
    e1 = ctx->ev[ctx->ev_used + 1];
    ctx->ev_used += 2;
    CK(cudaEventRecord(e0, st), "event record");
    return HOTRG_OK;
  }
  hotrg_status stop(double flops) {
    ctx->launches += 1;
    if (!e1) return HOTRG_OK;
    CK(cudaEventRecord(e1, st), "event record");
    ctx->gemm_launches += 1;
    ctx->gemm_flops += flops;
    return HOTRG_OK;
  }
};

// CUDA-core GEMM (FP64 and FP32 modes): C = alpha A B^T + beta C, one product per launch.
template <typename R>
hotrg_status gemm_simt(hotrg_ctx* ctx, const R* A, const R* B, const StepPlan& p, R* C, int64_t M, int64_t N,
                       double alpha, double beta, cudaStream_t st) {
  if (p.P != 1) return HOTRG_EUNSUPPORTED;
  GemmTimer tm{ctx, st};
  hotrg_status r = tm.start();
  if (r != HOTRG_OK) return r;
  CK(launch_gemm_simt<R>(A, p.kps, B, p.kps, C, N, M, N, p.K, alpha, beta, st), "gemm simt");
  return tm.stop(2.0 * (double)M * (double)N * (double)p.K);
}

// FP16X3 pipelines by option value: 0 = CTA pairs (tcgen05.mma.cta_group::2, 256 x 256 tiles),
// 128-k promotion chunks; 1 = one CTA, 64-k chunks; 2 = one CTA, 256-k chunks; 3 = one CTA,
// 128-k chunks.
constexpr int kF16Variant[4] = {5, 3, 4, 2};

// Tensor-core modes: every output of the group in one launch. The W operand tensors of a
// plane start Asz / Bsz operand elements apart.
hotrg_status gemm_tc(hotrg_ctx* ctx, const void* A, const void* Alo, const void* B, const void* Blo, int W,
                     int64_t Asz, int64_t Bsz, const StepPlan& p, const GemmGroup& g, int64_t M, int64_t N,
                     cudaStream_t st) {
  GemmTimer tm{ctx, st};
  hotrg_status r = tm.start();
  if (r != HOTRG_OK) return r;
  const int opt = p.gemm_opt >= 0 ? p.gemm_opt : ctx->gemm_variant;
  const int variant = ctx->prec == HOTRG_FP16X3 ? kF16Variant[opt] : opt;
  CK(launch_gemm_group(A, Alo, B, Blo, W, Asz, Bsz, p.Kp, p.kps, p.P, M, N, N, g, (int*)(ctx->ws + ctx->L.status),
                       st, variant),
     ctx->prec == HOTRG_FP16X3 ? "gemm f16x3" : "gemm tf32x3");
  double segs = 0;
  for (int q = 0; q < g.nprob; ++q) segs += g.p[q].nseg;
  return tm.stop(2.0 * (double)M * (double)N * (double)p.K * segs);
}

// Step 1 and 2 for every batch element in one set of launches: Gram halves (12 split-K
// jobs per element), chunk reduction, merge into the six Gram matrices, Jacobi (six
// matrices per element) and the side choice with Gram-Schmidt (three directions per
// element). The isometries land in each element's persistent slot (L.U64, L.Ur).
template <typename R>
hotrg_status isometry_stage(hotrg_ctx* ctx, const StepPlan& p, const Scratch& sc, char* sb, cudaStream_t st) {
  const int mu = p.mu;
  const int nb = p.batch;
  int* status = (int*)(ctx->ws + ctx->L.status);
  const int* dstep = (const int*)(ctx->ws + ctx->L.step);
  int64_t ts[8];
  canon_strides(p.D, ts);
  int dirs[3], nd = 0;
  for (int n = 0; n < 4; ++n)
    if (n != mu) dirs[nd++] = n;
  // ---------------------------------------------------------------- 1. Gram
  GramPack gp{};
  int nj = 0;
  double* gpart = (double*)(sb + sc.gpart);
  double* gA = (double*)(sb + sc.gA);
  const int64_t RR = (int64_t)p.Rmax * p.Rmax;
  for (int i = 0; i < 3; ++i) {
    const int n = dirs[i];
    for (int side = 0; side < 2; ++side) {
      for (int half = 0; half < 2; ++half) {   // half 0: k on mu' (T1), 1: k on mu (T2)
        GramJob& j = gp.j[nj];
        j.T = tensor_ptr<R>(ctx, 0, ctx->cur, 0);
        const int leg = 2 * n + side;
        const int kleg = half == 0 ? 2 * mu + 1 : 2 * mu;
        j.D1 = p.D[n];
        j.D2 = p.D[mu];
        j.s1 = ts[leg];
        j.s2 = ts[kleg];
        j.nrest = 0;
        j.K = 1;
        for (int l = 0; l < 8; ++l) {
          if (l == leg || l == kleg) continue;
          j.rdims[j.nrest] = p.D[l / 2];
          j.rst[j.nrest] = ts[l];
          j.K *= p.D[l / 2];
          ++j.nrest;
        }
        j.partial = gpart + (int64_t)nj * p.nchunks * RR;
        ++nj;
      }
    }
  }
  gp.batch = nb;
  gp.sT = ctx->L.cap;                                   // tensor slots of consecutive elements
  gp.sPart = (int64_t)kMaxGramJobs * p.nchunks * RR;
  LK(1, launch_gram<R>(gp, nj, p.Rmax, p.nchunks, st), "gram");
  LK(1, launch_gram_reduce(gp, nj, p.nchunks, RR, RR, gA, st), "gram reduce");
  double* G = (double*)(sb + sc.G);
  const int64_t nn = (int64_t)p.nmax * p.nmax;
  const int Dn[3] = {p.D[dirs[0]], p.D[dirs[1]], p.D[dirs[2]]};
  LK(1, launch_gram_merge_batch(gA, RR, Dn, p.D[mu], G, nn, nb, st), "gram merge");
  // ---------------------------------------------------------------- 2. eigen + side
  EigPack ep{};
  double* lam = (double*)(sb + sc.lam);
  double* eps = (double*)(sb + sc.eps);
  int* degen = (int*)(sb + sc.degen);
  double* Uside = (double*)(sb + sc.Uside);
  double* jwork = (double*)(sb + sc.jwork);
  const bool big = p.nmax > kJacobiSmemN;
  int nmax = 0;
  for (int i = 0; i < 3; ++i) {
    for (int side = 0; side < 2; ++side) {
      const int e = i * 2 + side;
      EigJob& j = ep.j[e];
      j.n = p.D[dirs[i]] * p.D[dirs[i]];
      j.chi = p.chi[dirs[i]];
      j.G = G + (int64_t)e * nn;
      j.work = big ? jwork + (int64_t)e * 2 * nn : nullptr;
      j.lam = lam + (int64_t)e * p.nmax;
      j.eps = eps + e;
      j.degenerate = degen + e;
      j.U = Uside + (int64_t)e * p.nmax * kMaxLeg;
      nmax = std::max(nmax, j.n);
    }
  }
  ep.batch = nb;
  ep.sG = 6 * nn;
  ep.sWork = big ? 6 * 2 * nn : 0;
  ep.sLam = 6 * (int64_t)p.nmax;
  ep.sU = 6 * (int64_t)p.nmax * kMaxLeg;
  ep.sEps = 6;
  ep.sDeg = 6;
  const bool fp64 = f64_store(ctx->prec);
  LK(1, launch_jacobi(ep, 6, nmax, fp64 ? 1e-10 : 1e-6, status, st, ctx->jacobi_sweeps, fp64 ? 1e-8 : 1e-4),
     "jacobi");
  SelectPack sp{};
  double* U64 = (double*)(ctx->ws + ctx->L.U64);
  R* Ur = (R*)(ctx->ws + ctx->L.Ur);
  DevRecord* rec = (DevRecord*)(ctx->ws + ctx->L.rec);
  for (int i = 0; i < 3; ++i) {
    const int n = dirs[i];
    SelectJob& j = sp.j[i];
    j.U[0] = ep.j[i * 2].U;
    j.U[1] = ep.j[i * 2 + 1].U;
    j.lam0 = ep.j[i * 2].lam;
    j.eps[0] = ep.j[i * 2].eps;
    j.eps[1] = ep.j[i * 2 + 1].eps;
    j.degen[0] = ep.j[i * 2].degenerate;
    j.degen[1] = ep.j[i * 2 + 1].degenerate;
    j.U64 = U64 + (int64_t)n * kMaxGramN * kMaxLeg;
    j.Ur = Ur + (int64_t)n * kMaxGramN * kMaxLeg;
    j.n = ep.j[i * 2].n;
    j.chi = ep.j[i * 2].chi;
    j.rec_eps = nullptr;
    j.rec_primed = nullptr;
    j.rec_degen = nullptr;
    j.rec_b = rec;
    j.step = dstep;
    j.nu = n;
  }
  sp.batch = nb;
  sp.sU = ep.sU;
  sp.sLam = ep.sLam;
  sp.sEps = ep.sEps;
  sp.sDeg = ep.sDeg;
  sp.sU64 = 4 * (int64_t)kMaxGramN * kMaxLeg;
  sp.sUr = 4 * (int64_t)kMaxGramN * kMaxLeg;
  sp.sRec = kMaxSteps;
  LK(1, launch_select<R>(sp, 3, fp64 ? 1e-9 : 1e-6, st), "select");
  return HOTRG_OK;
}

// What one contract_group call runs: the whole contraction (default), or a timing probe of
// the first slice block only: its tensor passes without the GEMM, or its GEMM alone on the
// first gemm_rows rows (operands left in place by a tensor-pass probe of the same plan).
struct Probe {
  bool first_block = false;
  bool ttm = true;
  bool gemm = true;
  int64_t gemm_rows = 0;
};

// Step 3 for the ne batch elements e0 .. e0 + ne - 1 together: the half contractions, the
// block-spin GEMM and the closing isometries, slice block by slice block, into the elements'
// next tensors (not yet normalised), every launch covering the whole group (the tensor passes
// index the element by blockIdx.y, the tensor-core GEMM takes every (element, tensor) output
// as one problem of its group). Reads each element's isometries from its persistent slot.
template <typename R>
hotrg_status contract_group(hotrg_ctx* ctx, const StepPlan& p, int e0, int ne, cudaStream_t st,
                            const Probe& pr = Probe()) {
  const Scratch sc = scratch_layout(p, p.xs, p.xs2, ctx->prec, ctx->impure_active, ctx->rsize);
  char* sb = ctx->ws + ctx->L.persistent_end;
  const int mu = p.mu;
  const int kstep = ctx->k;  // steps done before this one
  const int nt = ntensors(ctx->impure_active);
  const bool split = tc_mode(ctx->prec);
  const size_t osz = operand_size(ctx->prec);
  const int64_t rowsA = (int64_t)p.xs * p.chi[p.b] * p.D[p.c] * p.D[p.c] * p.D[mu];
  const int64_t rowsB = (int64_t)p.xs2 * p.chi[p.b] * p.D[p.c] * p.D[p.c] * p.D[mu];
  const int ca = p.chi[p.a];
  const bool b_sliced = p.xs2 < ca;
  if (ne < 1 || ne > p.ne || nt * ne > kMaxGemmProblems) return HOTRG_EINVAL;
  {
    R* Ur = (R*)(ctx->ws + ctx->L.Ur) + (int64_t)e0 * 4 * kMaxGramN * kMaxLeg;
    const R* Ua = Ur + (int64_t)p.a * kMaxGramN * kMaxLeg;
    const R* Ub = Ur + (int64_t)p.b * kMaxGramN * kMaxLeg;
    const R* Uc = Ur + (int64_t)p.c * kMaxGramN * kMaxLeg;
    // ---------------------------------------------------------------- 3. contraction
    R* O1A = (R*)(sb + sc.O1A);
    R* O1B = (R*)(sb + sc.O1B);
    // operand planes, addressed in bytes (fp16 operands are half the storage type's size);
    // FP64OZ: the kOzSlices planes of one operand follow each other (plane 1 in place of lo)
    const bool oz = ctx->prec == HOTRG_FP64OZ;
    const int64_t Asz = p.P * rowsA * p.kps, Bsz = p.P * rowsB * p.kps, Csz = rowsA * rowsB;
    char* Abuf = sb + sc.A;
    char* Alob = split ? sb + sc.Alo : (oz ? Abuf + Asz * (int64_t)osz : nullptr);
    char* Bbuf = sb + sc.B;
    char* Blob = split ? sb + sc.Blo : (oz ? Bbuf + Bsz * (int64_t)osz : nullptr);
    auto opnd = [&](char* base, int64_t elems) { return base ? (R*)(base + elems * (int64_t)osz) : (R*)nullptr; };
    R* Cbuf = (R*)(sb + sc.C);
    R* O3 = (R*)(sb + sc.O3);
    const R* src[3];
    R* dst[3];
    for (int w = 0; w < nt; ++w) {
      src[w] = tensor_ptr<R>(ctx, w, ctx->cur, e0);
      dst[w] = tensor_ptr<R>(ctx, w, 1 - ctx->cur, e0);
    }
    // element strides of the group (the scratch holds p.ne copies of every contraction buffer)
    const int64_t planes = oz ? kOzSlices : 1;
    ElemStrides esA, esB, esC;
    esA.ne = esB.ne = esC.ne = ne;
    esA.T = esB.T = esC.T = ctx->L.cap;
    esA.U = esB.U = esC.U = 4 * (int64_t)kMaxGramN * kMaxLeg;
    const int64_t O1Asz = (int64_t)p.xs * p.E, O1Bsz = (int64_t)p.xs2 * p.E;   // one tensor's first pass
    esA.O1 = nt * O1Asz;
    esB.O1 = nt * O1Bsz;
    // max-norm scaling of the fp16 planes and of the integer slices: one magnitude bound per
    // operand side over every tensor of the group (the segments of an output share 2^(eA+eB))
    const int scale = ctx->prec == HOTRG_FP16X3 ? ctx->maxnorm : (oz ? kScaleExact : kScaleNone);
    // (one word per element, so an element's scales do not depend on the group it runs in;
    // FP64OZ: one per element and tensor, each product being its own launch, so that the
    // impure tensors' slices keep their own precision)
    const int tw = oz ? nt : 1;               // words per element and side
    unsigned* amaxA = scale != kScaleNone ? (unsigned*)(sb + sc.amax) : nullptr;
    unsigned* amaxB = scale != kScaleNone ? amaxA + p.ne * tw : nullptr;
    // the first step's M operands are never read (M_1 = A(S) B(S)^T): not built
    const int nbuild = (kstep == 0 && nt >= 3) ? 2 : nt;
    esA.op = nt * Asz * planes;
    esB.op = nt * Bsz * planes;
    esC.C = nt * Csz;
    esC.O3 = rowsA * rowsB / ((int64_t)p.D[p.c] * p.D[p.c]) * p.chi[p.c];
    // Padding columns of a panel (kin >= Kp) are never read: the tensor maps stop at Kp and
    // the CUDA-core GEMM at K, so the operand buffers need no clearing.
    // every tensor's first pass, then (exact scaling) the max pass of every tensor, then the
    // second passes, which read the side's bound; the bound starts from zero before the
    // passes that record it
    auto clear_phase = [&](int ph) { return ph == (scale == kScaleBound ? kPass1 : kPassMax); };
    auto buildB = [&](int x20, int xs2) -> hotrg_status {
      for (int ph : {kPass1, kPassMax, kPass2}) {
        if (ph == kPassMax && scale != kScaleExact) continue;
        if (amaxB && clear_phase(ph)) CK(cudaMemsetAsync(amaxB, 0, ne * tw * sizeof(unsigned), st), "amax clear");
        for (int w = 0; w < nbuild; ++w) {
          hotrg_status s = build_B<R>(ctx, p, src[w], Ua, Ub, x20, xs2, O1B + w * O1Bsz, opnd(Bbuf, w * Bsz * planes),
                                      opnd(Blob, w * Bsz * planes), st, esB, amaxB ? amaxB + (tw > 1 ? w : 0) : nullptr,
                                      tw, scale, ph);
          if (s != HOTRG_OK) return s;
        }
      }
      return HOTRG_OK;
    };
    if (!b_sliced && pr.ttm) {
      hotrg_status s = buildB(0, ca);
      if (s != HOTRG_OK) return s;
    }
    const int xend = pr.first_block ? std::min(p.xs, ca) : ca;
    const int x2end = pr.first_block ? std::min(p.xs2, ca) : ca;
    for (int x0 = 0; x0 < xend; x0 += p.xs) {
      const int xs = std::min(p.xs, ca - x0);
      const int64_t rA_full = (int64_t)xs * p.chi[p.b] * p.D[p.c] * p.D[p.c] * p.D[mu];
      const int64_t rA = pr.gemm_rows > 0 ? std::min(rA_full, pr.gemm_rows) : rA_full;
      for (int ph : {kPass1, kPassMax, kPass2}) {
        if (!pr.ttm) break;
        if (ph == kPassMax && scale != kScaleExact) continue;
        if (amaxA && clear_phase(ph)) CK(cudaMemsetAsync(amaxA, 0, ne * tw * sizeof(unsigned), st), "amax clear");
        for (int w = 0; w < nbuild; ++w) {
          hotrg_status s = build_A<R>(ctx, p, src[w], Ua, Ub, x0, xs, O1A + w * O1Asz, opnd(Abuf, w * Asz * planes),
                                      opnd(Alob, w * Asz * planes), st, esA, amaxA ? amaxA + (tw > 1 ? w : 0) : nullptr,
                                      tw, scale, ph);
          if (s != HOTRG_OK) return s;
        }
      }
      for (int x20 = 0; x20 < x2end; x20 += p.xs2) {
        const int xs2 = std::min(p.xs2, ca - x20);
        const int64_t rB = (int64_t)xs2 * p.chi[p.b] * p.D[p.c] * p.D[p.c] * p.D[mu];
        if (b_sliced && pr.ttm) {
          hotrg_status s = buildB(x20, xs2);
          if (s != HOTRG_OK) return s;
        }
        hotrg_status s = HOTRG_OK;
        if (!pr.gemm) {
          // tensor-pass probe: no product
        } else if (split) {
          // every output of the block in one launch: C_T = A_T B_T^T, C_S = (A_S B_T^T + A_T B_S^T) / 2,
          // and M_1 = A_S B_S^T (the nearest-neighbour pair inside the first block) or
          // C_M = (A_M B_T^T + A_T B_M^T) / 2; operand tensor (e, w) of the group is tensor
          // e nt + w of the launch
          // fp16 operands carry 2^(eA + eB), which the epilogue removes (amax_a, amax_b), or,
          // without max-norm scaling, the fixed 2^14 each
          const double un = (ctx->prec == HOTRG_FP16X3 && !amaxA) ? 1.0 / ((double)kF16Scale * kF16Scale) : 1.0;
          GemmGroup g{};
          g.amax_a = amaxA;
          g.amax_b = amaxB;
          g.per_elem = nt;
          g.nprob = nt * ne;
          for (int e = 0; e < ne; ++e) {
            const int w0 = e * nt;
            R* Ce = Cbuf + (int64_t)w0 * Csz;
            g.p[w0] = GemmProblem{(float*)Ce, (float)un, 1, {w0, 0}, {w0, 0}};
            if (nt >= 2) g.p[w0 + 1] = GemmProblem{(float*)(Ce + Csz), (float)(0.5 * un), 2, {w0 + 1, w0}, {w0, w0 + 1}};
            if (nt >= 3)
              g.p[w0 + 2] = kstep == 0
                                ? GemmProblem{(float*)(Ce + 2 * Csz), (float)un, 1, {w0 + 1, 0}, {w0 + 1, 0}}
                                : GemmProblem{(float*)(Ce + 2 * Csz), (float)(0.5 * un), 2, {w0 + 2, w0}, {w0, w0 + 2}};
          }
          s = gemm_tc(ctx, Abuf, Alob, Bbuf, Blob, nt * ne, Asz, Bsz, p, g, rA, rB, st);
          if (s != HOTRG_OK) return s;
        } else if (oz) {   // FP64 accuracy, element by element, one product per launch
          for (int e = 0; e < ne && s == HOTRG_OK; ++e) {
            // operand tensor w of element e: its kOzSlices planes, Asz (Bsz) values each
            auto prod = [&](int wa, int wb, int out, double alpha, bool acc) -> hotrg_status {
              GemmTimer tm{ctx, st};
              hotrg_status r = tm.start();
              if (r != HOTRG_OK) return r;
              CK(launch_gemm_oz(Abuf + (e * esA.op + wa * Asz * planes) * (int64_t)osz,
                                Bbuf + (e * esB.op + wb * Bsz * planes) * (int64_t)osz, Asz, Bsz, p.Kp, p.kps, p.P,
                                rA, rB, (double*)(Cbuf + e * esC.C + out * Csz), rB, alpha, amaxA + e * tw + wa,
                                amaxB + e * tw + wb,
                                acc, (int*)(ctx->ws + ctx->L.status), st),
                 "gemm oz");
              return tm.stop(2.0 * (double)rA * (double)rB * (double)p.K);
            };
            s = prod(0, 0, 0, 1.0, false);                                    // C_T
            if (s == HOTRG_OK && nt >= 2) {                                    // C_S
              s = prod(1, 0, 1, 0.5, false);
              if (s == HOTRG_OK) s = prod(0, 1, 1, 0.5, true);
            }
            if (s == HOTRG_OK && nt >= 3) {
              if (kstep == 0) {
                s = prod(1, 1, 2, 1.0, false);                                 // M_1 = A(S) B(S)^T
              } else {                                                         // C_M
                s = prod(2, 0, 2, 0.5, false);
                if (s == HOTRG_OK) s = prod(0, 2, 2, 0.5, true);
              }
            }
          }
          if (s != HOTRG_OK) return s;
        } else for (int e = 0; e < ne; ++e) {
          R* Cbuf = (R*)(sb + sc.C) + e * esC.C;     // this element's outputs
          auto Ap = [&](int w) { return opnd(Abuf, e * esA.op + w * Asz); };
          auto Bp = [&](int w) { return opnd(Bbuf, e * esB.op + w * Bsz); };
          // C_T = A(T) B(T)^T
          s = gemm_simt<R>(ctx, Ap(0), Bp(0), p, Cbuf, rA, rB, 1.0, 0.0, st);
          if (s != HOTRG_OK) return s;
          if (nt >= 2) {  // C_S = (A(S) B(T)^T + A(T) B(S)^T) / 2
            s = gemm_simt<R>(ctx, Ap(1), Bp(0), p, Cbuf + Csz, rA, rB, 0.5, 0.0, st);
            if (s != HOTRG_OK) return s;
            s = gemm_simt<R>(ctx, Ap(0), Bp(1), p, Cbuf + Csz, rA, rB, 0.5, 1.0, st);
            if (s != HOTRG_OK) return s;
          }
          if (nt >= 3) {
            if (kstep == 0) {  // M_1 = A(S) B(S)^T: the nearest-neighbour pair inside the first block
              s = gemm_simt<R>(ctx, Ap(1), Bp(1), p, Cbuf + 2 * Csz, rA, rB, 1.0, 0.0, st);
              if (s != HOTRG_OK) return s;
            } else {           // M' = (A(M) B(T)^T + A(T) B(M)^T) / 2
              s = gemm_simt<R>(ctx, Ap(2), Bp(0), p, Cbuf + 2 * Csz, rA, rB, 0.5, 0.0, st);
              if (s != HOTRG_OK) return s;
              s = gemm_simt<R>(ctx, Ap(0), Bp(2), p, Cbuf + 2 * Csz, rA, rB, 0.5, 1.0, st);
              if (s != HOTRG_OK) return s;
            }
          }
        }
        for (int w = 0; w < nt && pr.ttm; ++w) {
          s = close_C<R>(ctx, p, Cbuf + w * Csz, Uc, x0, xs, x20, xs2, O3, dst[w], st, esC);
          if (s != HOTRG_OK) return s;
        }
      }
    }
  }
  return HOTRG_OK;
}

template <typename R>
hotrg_status do_step(hotrg_ctx* ctx, const StepPlan& p) {
  cudaStream_t st = ctx->stream;
  const Scratch sc = scratch_layout(p, p.xs, p.xs2, ctx->prec, ctx->impure_active, ctx->rsize);
  char* sb = ctx->ws + ctx->L.persistent_end;
  int* status = (int*)(ctx->ws + ctx->L.status);
  const int nt = ntensors(ctx->impure_active);
  const int* dstep = (const int*)(ctx->ws + ctx->L.step);
  hotrg_status s = isometry_stage<R>(ctx, p, sc, sb, st);
  if (s != HOTRG_OK) return s;
  for (int e0 = 0; e0 < ctx->batch; e0 += p.ne) {
    s = contract_group<R>(ctx, p, e0, std::min(p.ne, ctx->batch - e0), st);
    if (s != HOTRG_OK) return s;
  }
  // ---------------------------------------------------------------- 4. normalise (every element)
  DevRecord* rec = (DevRecord*)(ctx->ws + ctx->L.rec);
  double* lnz = (double*)(ctx->ws + ctx->L.lnz);
  double* cval = (double*)(ctx->ws + ctx->L.cval);
  const int64_t cap = ctx->L.cap;
  LK(2, launch_norm<R>(tensor_ptr<R>(ctx, 0, 1 - ctx->cur, 0), p.Enew, ctx->batch, cap, (double*)(sb + sc.npart), dstep,
                       cval, lnz, rec, status, st),
     "norm");
  for (int w = 0; w < nt; ++w)
    LK(1, launch_scale<R>(tensor_ptr<R>(ctx, w, 1 - ctx->cur, 0), p.Enew, ctx->batch, cap, cval, st), "scale");
  LK(1, launch_step_end((int*)(ctx->ws + ctx->L.step), st), "step end");
  return HOTRG_OK;
}

hotrg_status check_ready(hotrg_ctx* ctx) {
  if (!ctx) return HOTRG_EINVAL;
  if (!ctx->ready) return HOTRG_EWORKSPACE;
  return HOTRG_OK;
}

hotrg_status sync_and_status(hotrg_ctx* ctx) {
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "stream sync");
  int st[kStWords];
  e = cudaMemcpy(st, ctx->ws + ctx->L.status, sizeof(st), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "status read");
  if (st[kStTimeout]) ctx->sticky = HOTRG_ETIMEOUT;
  else if (st[kStNonFinite]) ctx->sticky = HOTRG_ENONFINITE;
  else if (st[kStNoConv]) ctx->sticky = HOTRG_ENOCONV;
  return ctx->sticky ? (hotrg_status)ctx->sticky : HOTRG_OK;
}

// Group size and slice sizes (X for A and C rows, X' for B rows and C columns). Per element
// (one temperature at a time): the slice pair that fits the workspace with the fewest GEMM
// blocks, then the largest X' slice. Grouped (ne >= 2 temperatures contracted together, each
// launch of the contraction covering the whole group): B unsliced and the largest X slice
// that fits. The plan with fewer groups x blocks (launches of the contraction) wins, ties to
// the larger group; a group holds at most kMaxGemmProblems / tensors temperatures (the
// outputs of one grouped GEMM launch). False if nothing fits.
bool choose_slices(const hotrg_ctx* ctx, StepPlan& p) {
  const size_t avail = ctx->ws_bytes - ctx->L.persistent_end;
  const int ca = p.chi[p.a];
  const int nt = ntensors(ctx->impure_active);
  StepPlan q = p;
  q.ne = 1;
  int best_xs = 0, best_xs2 = 0;
  int64_t best_blocks = -1;
  for (int xs = ca; xs >= 1; --xs) {
    for (int xs2 = ca; xs2 >= 1; --xs2) {
      if (scratch_layout(q, xs, xs2, ctx->prec, ctx->impure_active, ctx->rsize).total > avail) continue;
      const int64_t blocks = (int64_t)((ca + xs - 1) / xs) * ((ca + xs2 - 1) / xs2);
      if (best_blocks < 0 || blocks < best_blocks || (blocks == best_blocks && xs2 > best_xs2)) {
        best_blocks = blocks;
        best_xs = xs;
        best_xs2 = xs2;
      }
      break;  // smaller xs2 only adds blocks for this xs
    }
  }
  int best_ne = 1;
  int64_t best_cost = best_blocks < 0 ? -1 : (int64_t)ctx->batch * best_blocks;
  int ne_max = std::min(ctx->batch, kMaxGemmProblems / nt);
  if (ctx->group_max > 0) ne_max = std::min(ne_max, ctx->group_max);
  for (int ne = 2; ne <= ne_max; ++ne) {
    q.ne = ne;
    for (int xs = ca; xs >= 1; --xs) {
      if (scratch_layout(q, xs, ca, ctx->prec, ctx->impure_active, ctx->rsize).total > avail) continue;
      const int64_t cost = (int64_t)((ctx->batch + ne - 1) / ne) * ((ca + xs - 1) / xs);
      if (best_cost < 0 || cost <= best_cost) {
        best_cost = cost;
        best_ne = ne;
        best_xs = xs;
        best_xs2 = ca;
      }
      break;
    }
  }
  if (best_cost < 0) return false;
  p.ne = best_ne;
  p.xs = best_xs;
  p.xs2 = best_xs2;
  return true;
}

// ---------------------------------------------------------------------------- autotuner
// The plan choices that leave the method's arithmetic unchanged up to rounding are timed on
// the GPU and the fastest is kept, per device and step shape: the closing direction c (which
// transverse direction the last two isometry passes close; it fixes the shapes of the half
// contractions and of the GEMM) and the tensor-core pipeline (FP16X3: CTA pairs or single
// CTAs, which give bit-identical products; TF32X3: 16- or 32-wide k-blocks). The promotion
// chunk changes the truncation bias of the tensor-core accumulator, so it is not a candidate.
struct TuneChoice {
  int c;
  int opt;
  float ms;
};
std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune;   // keyed by device and step shape

std::string tune_key(const hotrg_ctx* ctx, int dir, int dcut) {
  int dev = -1;
  cudaGetDevice(&dev);
  char key[160];
  snprintf(key, sizeof(key), "dev%d prec%d b%d t%d D%d,%d,%d,%d mu%d cut%d ws%zu", dev, ctx->prec, ctx->batch,
           ntensors(ctx->impure_active), ctx->dims[0], ctx->dims[1], ctx->dims[2], ctx->dims[3], dir, dcut,
           ctx->ws_bytes);
  return key;
}

bool tune_lookup(const std::string& key, TuneChoice* out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return false;
  *out = it->second;
  return true;
}

// Ranks the candidate plans of the step hotrg_step(ctx, dir, dcut) would run next, with timing
// probes on the real operands of batch element 0 (the isometry stage runs once): for each
// closing direction the tensor passes of its first slice block (times its number of blocks),
// and the GEMM pipelines on the first 2048 rows of the planner's first block; a plan's
// estimate is its tensor-pass time plus its GEMM flops at the measured rate of the fastest
// pipeline. Probes write scratch and the (not normalised) next tensor, which the real step
// overwrites; the ln Z accumulator, the step counter and the current tensors do not change.
// A probe costs about one slice block, not a whole step. Not callable inside a capture.
template <typename R>
hotrg_status tune_step(hotrg_ctx* ctx, int dir, int dcut, TuneChoice* best_out) {
  cudaStream_t st = ctx->stream;
  StepPlan p0 = make_plan(ctx->dims, dir, dcut, ctx->prec, ctx->batch);
  if (!choose_slices(ctx, p0)) return HOTRG_EWORKSPACE;
  const Scratch sc0 = scratch_layout(p0, p0.xs, p0.xs2, ctx->prec, ctx->impure_active, ctx->rsize);
  hotrg_status s = isometry_stage<R>(ctx, p0, sc0, ctx->ws + ctx->L.persistent_end, st);
  if (s != HOTRG_OK) return s;
  std::vector<int> opts;
  if (ctx->prec == HOTRG_FP16X3) opts = {0, 3};        // CTA pairs, single CTAs (128-k chunks both)
  else if (ctx->prec == HOTRG_TF32X3) opts = {0, 1};
  else opts = {-1};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "tune event");
  CK(cudaEventCreate(&e1), "tune event");
  const bool prof = ctx->profiling;
  ctx->profiling = false;
  const uint64_t l0 = ctx->launches;
  auto timed = [&](const StepPlan& pl, const Probe& pr, float* ms) -> hotrg_status {
    cudaError_t e = cudaEventRecord(e0, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tune timing");
    hotrg_status r = contract_group<R>(ctx, pl, 0, 1, st, pr);
    if (r != HOTRG_OK) return r;
    e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    return e == cudaSuccess ? HOTRG_OK : cuda_fail(ctx, e, "tune timing");
  };
  const int nprod = ntensors(ctx->impure_active) == 1 ? 1 : (ctx->k == 0 ? 4 : 5);   // products per block
  double est_ttm[4] = {-1, -1, -1, -1}, flops[4] = {0, 0, 0, 0};
  for (int c = 0; c < 4 && s == HOTRG_OK; ++c) {
    if (c == dir || c == p0.c) continue;   // the planner's direction last: its operands stay for the GEMM probe
    StepPlan pc = make_plan(ctx->dims, dir, dcut, ctx->prec, ctx->batch, c);
    if (!choose_slices(ctx, pc)) continue;
    Probe pr;
    pr.first_block = true;
    pr.gemm = false;
    float ms = 0;
    s = timed(pc, pr, &ms);
    const int ca = pc.chi[pc.a];
    est_ttm[c] = (double)ms * ((ca + pc.xs - 1) / pc.xs) * ((ca + pc.xs2 - 1) / pc.xs2);
    flops[c] = nprod * pc.main_flops;
  }
  float best_g = -1.f;
  int best_opt = opts[0];
  if (s == HOTRG_OK) {
    Probe pr;
    pr.first_block = true;
    pr.gemm = false;
    float ms = 0;
    s = timed(p0, pr, &ms);
    const int ca = p0.chi[p0.a];
    est_ttm[p0.c] = (double)ms * ((ca + p0.xs - 1) / p0.xs) * ((ca + p0.xs2 - 1) / p0.xs2);
    flops[p0.c] = nprod * p0.main_flops;
  }
  const int64_t rows0 = (int64_t)std::min(p0.xs, p0.chi[p0.a]) * p0.chi[p0.b] * p0.D[p0.c] * p0.D[p0.c] * p0.D[dir];
  const int64_t cols0 = (int64_t)std::min(p0.xs2, p0.chi[p0.a]) * p0.chi[p0.b] * p0.D[p0.c] * p0.D[p0.c] * p0.D[dir];
  const int64_t probe_rows = std::min<int64_t>(rows0, 2048);
  for (int opt : opts) {
    if (s != HOTRG_OK) break;
    StepPlan pg = p0;
    pg.gemm_opt = opt;
    Probe pr;
    pr.first_block = true;
    pr.ttm = false;
    pr.gemm_rows = probe_rows;
    float ms = 0;
    s = timed(pg, pr, &ms);
    // ties (within 1 %) go to the default pipeline
    if (best_g < 0 || ms < 0.99f * best_g) {
      best_g = ms;
      best_opt = opt;
    }
  }
  ctx->launches = l0;
  ctx->profiling = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != HOTRG_OK) return s;
  hotrg_status st2 = sync_and_status(ctx);
  if (st2 != HOTRG_OK) return st2;
  // GEMM rate of the best pipeline on the probe (flops of every product of the block)
  const double probe_flops = 2.0 * (double)probe_rows * (double)cols0 * (double)p0.K * nprod;
  const double rate = best_g > 0 ? probe_flops / best_g : 0.0;   // flops per ms
  TuneChoice best{p0.c, best_opt, -1.f};
  double best_est = -1;
  for (int c = 0; c < 4; ++c) {
    if (est_ttm[c] < 0) continue;
    const double est = est_ttm[c] + (rate > 0 ? flops[c] / rate : 0.0);
    const bool is_default = c == p0.c;
    if (best_est < 0 || est < 0.99 * best_est || (is_default && est <= 1.01 * best_est)) {
      best_est = est;
      best.c = c;
    }
  }
  best.ms = (float)best_est;
  *best_out = best;
  return HOTRG_OK;
}

size_t persistent_bytes(const hotrg_ctx* ctx, int64_t cap) {
  return persistent_layout(ctx->batch, cap, ctx->impure, ctx->rsize).persistent_end;
}

}  // namespace

extern "C" {

const char* hotrg_status_string(int s) {
  switch (s) {
    case HOTRG_OK: return "ok";
    case HOTRG_EINVAL: return "invalid argument";
    case HOTRG_EWORKSPACE: return "workspace missing or too small";
    case HOTRG_ECUDA: return "CUDA error";
    case HOTRG_ENOCONV: return "eigensolver did not converge";
    case HOTRG_ENONFINITE: return "non-finite or non-positive norm";
    case HOTRG_ETIMEOUT: return "device-side wait timed out";
    case HOTRG_ESTATE: return "call out of order or context in error state";
    case HOTRG_EUNSUPPORTED: return "unsupported precision or size";
    default: return "unknown status";
  }
}

const char* hotrg_last_error(void) { return g_last_error.c_str(); }

hotrg_status hotrg_create(hotrg_ctx** out, int batch, int dcut_max, int prec, int impure_mask) {
  if (!out || batch < 1 || batch > 4096 || dcut_max < 2 || dcut_max > kMaxLeg) return HOTRG_EINVAL;
  if (prec != HOTRG_FP64 && prec != HOTRG_FP32 && prec != HOTRG_TF32X3 && prec != HOTRG_FP16X3 &&
      prec != HOTRG_FP64OZ)
    return HOTRG_EINVAL;
  if (impure_mask < 0 || impure_mask > 3 || impure_mask == HOTRG_IMPURE_SIGMASIGMA) return HOTRG_EINVAL;
  hotrg_ctx* c = new hotrg_ctx();
  c->batch = batch;
  c->dcut_max = dcut_max;
  c->prec = prec;
  c->impure = impure_mask;
  c->impure_active = impure_mask;
  c->rsize = f64_store(prec) ? 8 : 4;
  *out = c;
  return HOTRG_OK;
}

hotrg_status hotrg_destroy(hotrg_ctx* ctx) {
  delete ctx;
  return HOTRG_OK;
}

hotrg_status hotrg_workspace_size(hotrg_ctx* ctx, int nsteps, const int* dirs, const int* dcuts, const int* dims0,
                                  size_t* bytes) {
  if (!ctx || !bytes || nsteps < 0 || (nsteps > 0 && (!dirs || !dcuts))) return HOTRG_EINVAL;
  int D[4] = {2, 2, 2, 2};
  if (dims0)
    for (int n = 0; n < 4; ++n) {
      if (dims0[n] < 1 || dims0[n] > kMaxLeg) return HOTRG_EINVAL;
      D[n] = dims0[n];
    }
  size_t scratch = 0;
  int64_t cap = tensor_elems(D);
  // room for the largest useful group of temperatures contracted together (unsliced); a
  // smaller workspace makes the planner take smaller groups or slices
  int ne_full = std::min(ctx->batch, kMaxGemmProblems / ntensors(ctx->impure));
  if (ctx->group_max > 0) ne_full = std::min(ne_full, ctx->group_max);
  if (nsteps == 0) {
    int Dm[4] = {ctx->dcut_max, ctx->dcut_max, ctx->dcut_max, ctx->dcut_max};
    StepPlan p = make_plan(Dm, 0, ctx->dcut_max, ctx->prec, ctx->batch);
    p.ne = ne_full;
    scratch = scratch_layout(p, p.xs, p.xs2, ctx->prec, ctx->impure, ctx->rsize).total;
    cap = std::max(cap, tensor_elems(Dm));
  } else {
    for (int i = 0; i < nsteps; ++i) {
      if (dirs[i] < 0 || dirs[i] > 3 || dcuts[i] < 1 || dcuts[i] > ctx->dcut_max) return HOTRG_EINVAL;
      StepPlan p = make_plan(D, dirs[i], dcuts[i], ctx->prec, ctx->batch);
      p.ne = ne_full;
      scratch = std::max(scratch, scratch_layout(p, p.xs, p.xs2, ctx->prec, ctx->impure, ctx->rsize).total);
      for (int n = 0; n < 4; ++n) {
        D[n] = p.newD[n];
        if (D[n] > kMaxLeg) return HOTRG_EINVAL;
      }
      cap = std::max(cap, tensor_elems(D));
    }
  }
  ctx->cap_planned = cap;
  *bytes = persistent_bytes(ctx, cap) + scratch;
  return HOTRG_OK;
}

hotrg_status hotrg_set_workspace(hotrg_ctx* ctx, void* dev_ptr, size_t bytes) {
  if (!ctx || !dev_ptr || ((uintptr_t)dev_ptr & 255)) return HOTRG_EINVAL;
  int64_t cap = ctx->cap_planned;
  if (cap == 0) {
    int64_t d = ctx->dcut_max;
    cap = d * d * d * d * d * d * d * d;
  }
  Layout L = persistent_layout(ctx->batch, cap, ctx->impure, ctx->rsize);
  if (L.persistent_end > bytes) return HOTRG_EWORKSPACE;
  ctx->drop_graphs();
  jacobi_prepare();
  gemm_prepare();
  ctx->ws = (char*)dev_ptr;
  ctx->ws_bytes = bytes;
  ctx->L = L;
  ctx->ready = true;
  ctx->initialised = false;
  return HOTRG_OK;
}

hotrg_status hotrg_set_stream(hotrg_ctx* ctx, void* s) {
  if (!ctx) return HOTRG_EINVAL;
  if (ctx->use_graphs && s == nullptr) return HOTRG_EINVAL;   // the legacy stream cannot be captured
  ctx->stream = (cudaStream_t)s;
  return HOTRG_OK;
}

hotrg_status hotrg_init_tensor(hotrg_ctx* ctx, const double* beta, const double* h) {
  hotrg_status r = check_ready(ctx);
  if (r != HOTRG_OK) return r;
  if (!beta || !h) return HOTRG_EINVAL;
  for (int b = 0; b < ctx->batch; ++b)
    if (!(beta[b] >= 0.0) || !isfinite(beta[b]) || !isfinite(h[b])) return HOTRG_EINVAL;
  if (ctx->L.cap < 256) return HOTRG_EWORKSPACE;
  cudaStream_t st = ctx->stream;
  CK(cudaMemsetAsync(ctx->ws + ctx->L.status, 0, kStWords * 4, st), "init status");
  CK(cudaMemsetAsync(ctx->ws + ctx->L.step, 0, sizeof(int), st), "init step");
  CK(cudaMemsetAsync(ctx->ws + ctx->L.rec, 0, (size_t)ctx->batch * kMaxSteps * sizeof(DevRecord), st), "init rec");
  CK(cudaMemcpyAsync(ctx->ws + ctx->L.beta, beta, ctx->batch * 8, cudaMemcpyHostToDevice, st), "beta");
  CK(cudaMemcpyAsync(ctx->ws + ctx->L.hfield, h, ctx->batch * 8, cudaMemcpyHostToDevice, st), "h");
  ctx->impure_active = ctx->impure;
  ctx->cur = 0;
  const double* db = (const double*)(ctx->ws + ctx->L.beta);
  const double* dh = (const double*)(ctx->ws + ctx->L.hfield);
  double* lnz = (double*)(ctx->ws + ctx->L.lnz);
  if (f64_store(ctx->prec))
    LK(1, launch_init<double>(db, dh, tensor_ptr<double>(ctx, 0, 0, 0),
                           ctx->impure ? tensor_ptr<double>(ctx, 1, 0, 0) : nullptr, ctx->L.cap, lnz, ctx->batch, st),
       "init");
  else
    LK(1, launch_init<float>(db, dh, tensor_ptr<float>(ctx, 0, 0, 0),
                          ctx->impure ? tensor_ptr<float>(ctx, 1, 0, 0) : nullptr, ctx->L.cap, lnz, ctx->batch, st),
       "init");
  // the beta/h uploads read host memory that may go away: make them complete now
  CK(cudaStreamSynchronize(st), "init sync");
  ctx->h_host.assign(h, h + ctx->batch);
  for (int n = 0; n < 4; ++n) ctx->dims[n] = 2;
  ctx->k = 0;
  ctx->sticky = 0;
  ctx->initialised = true;
  ctx->last_mu = -1;
  ctx->last_kstep = -1;
  return HOTRG_OK;
}

hotrg_status hotrg_set_tensor(hotrg_ctx* ctx, int b, const int dims[4], const double* T_host) {
  hotrg_status r = check_ready(ctx);
  if (r != HOTRG_OK) return r;
  if (!dims || !T_host || b < 0 || b >= ctx->batch) return HOTRG_EINVAL;
  for (int n = 0; n < 4; ++n)
    if (dims[n] < 1 || dims[n] > ctx->dcut_max) return HOTRG_EINVAL;
  const int64_t E = tensor_elems(dims);
  if (E > ctx->L.cap) return HOTRG_EWORKSPACE;
  if (ctx->initialised && ctx->k > 0 && b > 0) return HOTRG_ESTATE;
  if (b > 0 && ctx->initialised)
    for (int n = 0; n < 4; ++n)
      if (dims[n] != ctx->dims[n]) return HOTRG_EINVAL;
  double nrm2 = 0;
  for (int64_t i = 0; i < E; ++i) nrm2 += T_host[i] * T_host[i];
  const double c = sqrt(nrm2);
  if (!(c > 0) || !isfinite(c)) return HOTRG_EINVAL;
  cudaStream_t st = ctx->stream;
  CK(cudaStreamSynchronize(st), "set_tensor sync");
  if (b == 0) {
    CK(cudaMemset(ctx->ws + ctx->L.status, 0, kStWords * 4), "status");
    CK(cudaMemset(ctx->ws + ctx->L.step, 0, sizeof(int)), "step");
    CK(cudaMemset(ctx->ws + ctx->L.rec, 0, (size_t)ctx->batch * kMaxSteps * sizeof(DevRecord)), "rec");
    ctx->cur = 0;
  }
  if (f64_store(ctx->prec)) {
    std::vector<double> tmp(E);
    for (int64_t i = 0; i < E; ++i) tmp[i] = T_host[i] / c;
    CK(cudaMemcpy(tensor_ptr<double>(ctx, 0, ctx->cur, b), tmp.data(), E * 8, cudaMemcpyHostToDevice), "upload");
  } else {
    std::vector<float> tmp(E);
    for (int64_t i = 0; i < E; ++i) tmp[i] = (float)(T_host[i] / c);
    CK(cudaMemcpy(tensor_ptr<float>(ctx, 0, ctx->cur, b), tmp.data(), E * 4, cudaMemcpyHostToDevice), "upload");
  }
  const double lc = log(c);
  CK(cudaMemcpy((double*)(ctx->ws + ctx->L.lnz) + b, &lc, 8, cudaMemcpyHostToDevice), "lnz");
  ctx->impure_active = 0;
  for (int n = 0; n < 4; ++n) ctx->dims[n] = dims[n];
  ctx->k = 0;
  ctx->sticky = 0;
  ctx->initialised = true;
  ctx->last_mu = -1;
  ctx->last_kstep = -1;
  ctx->h_host.assign(ctx->batch, 0.0);
  return HOTRG_OK;
}

hotrg_status hotrg_step(hotrg_ctx* ctx, int dir, int dcut) {
  hotrg_status r = check_ready(ctx);
  if (r != HOTRG_OK) return r;
  if (dir < 0 || dir > 3 || dcut < 1 || dcut > ctx->dcut_max) return HOTRG_EINVAL;
  if (!ctx->initialised || ctx->sticky) return HOTRG_ESTATE;
  if (ctx->k >= kMaxSteps) return HOTRG_ESTATE;
  StepPlan p = make_plan(ctx->dims, dir, dcut, ctx->prec, ctx->batch);
  for (int n = 0; n < 4; ++n)
    if (p.newD[n] > kMaxLeg) return HOTRG_EINVAL;
  if (p.Enew > ctx->L.cap) return HOTRG_EWORKSPACE;
  // the autotuner's plan for this shape (timed now if the context tunes and it is new)
  if (ctx->autotune) {
    const std::string key = tune_key(ctx, dir, dcut);
    TuneChoice tc{};
    bool hit = tune_lookup(key, &tc);
    if (hit) {
      ctx->tune_hits += 1;
    } else {
      hotrg_status ts = f64_store(ctx->prec) ? tune_step<double>(ctx, dir, dcut, &tc)
                                                : tune_step<float>(ctx, dir, dcut, &tc);
      if (ts != HOTRG_OK) return ts;
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune[key] = tc;
      ctx->tune_timed += 1;
    }
    p = make_plan(ctx->dims, dir, dcut, ctx->prec, ctx->batch, tc.c);
    p.gemm_opt = tc.opt;
    p.tuned = hit;
  }
  if (!choose_slices(ctx, p)) return HOTRG_EWORKSPACE;
  hotrg_status s = HOTRG_OK;
  if (!ctx->use_graphs) {
    s = f64_store(ctx->prec) ? do_step<double>(ctx, p) : do_step<float>(ctx, p);
    if (s != HOTRG_OK) return s;
  } else {
    // Everything the step's launches depend on: the plan (dims, direction, cut, slices),
    // which buffer holds the tensors, whether it is the first step (M_1 = C(S,S)) and the
    // impure tensors in use. ln c / 2^k and the record slot come from the device counter.
    char key[256];
    snprintf(key, sizeof(key), "%d %d %d %d %d %d %d %d %d %d %d %d %d %d %d", dir, dcut, ctx->dims[0],
             ctx->dims[1], ctx->dims[2], ctx->dims[3], ctx->cur, ctx->k == 0, ctx->impure_active, p.xs, p.xs2,
             ctx->batch, p.c, p.gemm_opt, p.ne);
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) {
      const uint64_t l0 = ctx->launches;
      CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
      s = f64_store(ctx->prec) ? do_step<double>(ctx, p) : do_step<float>(ctx, p);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
      if (s != HOTRG_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
      cudaGraphExec_t exec = nullptr;
      e = cudaGraphInstantiate(&exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "instantiate");
      it = ctx->graphs.emplace(key, hotrg_ctx::GraphEntry{exec, ctx->launches - l0}).first;
      ctx->launches = l0;
    }
    CK(cudaGraphLaunch(it->second.exec, ctx->stream), "graph launch");
    ctx->launches += it->second.launches;
  }
  ctx->last_plan = p;
  ctx->last_kstep = ctx->k;
  ctx->mu_hist[ctx->k] = dir;
  ctx->c_hist[ctx->k] = p.c;
  ctx->opt_hist[ctx->k] = tc_mode(ctx->prec) ? (p.gemm_opt >= 0 ? p.gemm_opt : ctx->gemm_variant) : -1;
  ctx->tuned_hist[ctx->k] = p.tuned ? 1 : 0;
  ctx->group_hist[ctx->k] = p.ne;
  ctx->slices_hist[ctx->k][0] = (p.chi[p.a] + p.xs - 1) / p.xs;
  ctx->slices_hist[ctx->k][1] = (p.chi[p.a] + p.xs2 - 1) / p.xs2;
  for (int n = 0; n < 4; ++n) {
    ctx->dims_hist[ctx->k][n] = p.newD[n];
    ctx->dims[n] = p.newD[n];
    ctx->last_chi[n] = p.chi[n];
    ctx->last_Dold[n] = p.D[n];
  }
  ctx->last_mu = dir;
  ctx->cur = 1 - ctx->cur;
  ctx->k += 1;
  return HOTRG_OK;
}

static hotrg_status traces(hotrg_ctx* ctx, int which, std::vector<double>& out) {
  const double* dtr = (const double*)(ctx->ws + ctx->L.trace);
  if (f64_store(ctx->prec))
    LK(1, launch_trace<double>(tensor_ptr<double>(ctx, which, ctx->cur, 0), ctx->L.cap, ctx->dims, ctx->batch,
                            (double*)dtr + which * ctx->batch, ctx->stream),
       "trace");
  else
    LK(1, launch_trace<float>(tensor_ptr<float>(ctx, which, ctx->cur, 0), ctx->L.cap, ctx->dims, ctx->batch,
                           (double*)dtr + which * ctx->batch, ctx->stream),
       "trace");
  hotrg_status s = sync_and_status(ctx);
  if (s != HOTRG_OK) return s;
  out.resize(ctx->batch);
  CK(cudaMemcpy(out.data(), dtr + which * ctx->batch, ctx->batch * 8, cudaMemcpyDeviceToHost), "trace read");
  return HOTRG_OK;
}

hotrg_status hotrg_lnZ(hotrg_ctx* ctx, double* out) {
  hotrg_status r = check_ready(ctx);
  if (r != HOTRG_OK) return r;
  if (!out) return HOTRG_EINVAL;
  if (!ctx->initialised) return HOTRG_ESTATE;
  std::vector<double> tr, acc(ctx->batch);
  r = traces(ctx, 0, tr);
  if (r != HOTRG_OK) return r;
  CK(cudaMemcpy(acc.data(), ctx->ws + ctx->L.lnz, ctx->batch * 8, cudaMemcpyDeviceToHost), "lnz read");
  hotrg_status res = HOTRG_OK;
  for (int b = 0; b < ctx->batch; ++b) {
    if (!(tr[b] > 0) || !isfinite(tr[b])) {
      out[b] = nan("");
      res = HOTRG_ENONFINITE;
    } else {
      out[b] = acc[b] + log(tr[b]) * ldexp(1.0, -ctx->k);
    }
  }
  return res;
}

hotrg_status hotrg_x_indicator(hotrg_ctx* ctx, int nu, double* X) {
  hotrg_status r = check_ready(ctx);
  if (r != HOTRG_OK) return r;
  if (!X || nu < 0 || nu > 3) return HOTRG_EINVAL;
  if (!ctx->initialised) return HOTRG_ESTATE;
  double* dx = (double*)(ctx->ws + ctx->L.trace) + 3 * ctx->batch;
  if (f64_store(ctx->prec))
    LK(1, launch_xind<double>(tensor_ptr<double>(ctx, 0, ctx->cur, 0), ctx->L.cap, ctx->dims, ctx->batch, nu, dx,
                           ctx->stream),
       "x indicator");
  else
    LK(1, launch_xind<float>(tensor_ptr<float>(ctx, 0, ctx->cur, 0), ctx->L.cap, ctx->dims, ctx->batch, nu, dx,
                          ctx->stream),
       "x indicator");
  hotrg_status s = sync_and_status(ctx);
  if (s != HOTRG_OK) return s;
  CK(cudaMemcpy(X, dx, ctx->batch * 8, cudaMemcpyDeviceToHost), "x indicator read");
  for (int b = 0; b < ctx->batch; ++b)
    if (!isfinite(X[b])) return HOTRG_ENONFINITE;
  return HOTRG_OK;
}

hotrg_status hotrg_impure_magnetization(hotrg_ctx* ctx, double* m) {
  hotrg_status r = check_ready(ctx);
  if (r != HOTRG_OK) return r;
  if (!m) return HOTRG_EINVAL;
  if (!ctx->initialised || !(ctx->impure_active & HOTRG_IMPURE_SIGMA)) return HOTRG_ESTATE;
  std::vector<double> t, s;
  if ((r = traces(ctx, 0, t)) != HOTRG_OK) return r;
  if ((r = traces(ctx, 1, s)) != HOTRG_OK) return r;
  for (int b = 0; b < ctx->batch; ++b) m[b] = s[b] / t[b];
  return HOTRG_OK;
}

hotrg_status hotrg_impure_energy(hotrg_ctx* ctx, double* e, double* ss) {
  hotrg_status r = check_ready(ctx);
  if (r != HOTRG_OK) return r;
  if (!ctx->initialised || !(ctx->impure_active & HOTRG_IMPURE_SIGMASIGMA) || ctx->k < 1) return HOTRG_ESTATE;
  std::vector<double> t, s, mm;
  if ((r = traces(ctx, 0, t)) != HOTRG_OK) return r;
  if ((r = traces(ctx, 1, s)) != HOTRG_OK) return r;
  if ((r = traces(ctx, 2, mm)) != HOTRG_OK) return r;
  for (int b = 0; b < ctx->batch; ++b) {
    const double sig2 = mm[b] / t[b];
    if (ss) ss[b] = sig2;
    if (e) e[b] = -4.0 * sig2 - ctx->h_host[b] * s[b] / t[b];
  }
  return HOTRG_OK;
}

hotrg_status hotrg_step_info(hotrg_ctx* ctx, int b, int step, hotrg_step_record* rec) {
  hotrg_status r = check_ready(ctx);
  if (r != HOTRG_OK) return r;
  if (!rec || b < 0 || b >= ctx->batch || step < 1 || step > ctx->k) return HOTRG_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  DevRecord d;
  CK(cudaMemcpy(&d, (DevRecord*)(ctx->ws + ctx->L.rec) + (int64_t)b * kMaxSteps + (step - 1), sizeof(d),
                cudaMemcpyDeviceToHost),
     "record read");
  memset(rec, 0, sizeof(*rec));
  rec->mu = ctx->mu_hist[step - 1];
  for (int n = 0; n < 4; ++n) {
    rec->dims[n] = ctx->dims_hist[step - 1][n];
    rec->primed[n] = d.primed[n];
    rec->degenerate[n] = d.degen[n];
    rec->eps[n][0] = d.eps[n][0];
    rec->eps[n][1] = d.eps[n][1];
  }
  rec->ln_c = d.ln_c;
  rec->slices[0] = ctx->slices_hist[step - 1][0];
  rec->slices[1] = ctx->slices_hist[step - 1][1];
  rec->closing = ctx->c_hist[step - 1];
  rec->gemm_option = ctx->opt_hist[step - 1];
  rec->tuned = ctx->tuned_hist[step - 1];
  rec->group = ctx->group_hist[step - 1];
  return HOTRG_OK;
}

hotrg_status hotrg_state(const hotrg_ctx* ctx, int* steps_done, int dims[4]) {
  if (!ctx) return HOTRG_EINVAL;
  if (steps_done) *steps_done = ctx->k;
  if (dims)
    for (int n = 0; n < 4; ++n) dims[n] = ctx->dims[n];
  return HOTRG_OK;
}

hotrg_status hotrg_copy_tensor(hotrg_ctx* ctx, int which, int b, double* host, size_t n) {
  hotrg_status r = check_ready(ctx);
  if (r != HOTRG_OK) return r;
  if (!host || b < 0 || b >= ctx->batch || which < 0 || which > 2) return HOTRG_EINVAL;
  if (which >= ntensors(ctx->impure_active)) return HOTRG_ESTATE;
  if (which == 2 && ctx->k < 1) return HOTRG_ESTATE;
  const int64_t E = tensor_elems(ctx->dims);
  if ((int64_t)n < E) return HOTRG_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  if (f64_store(ctx->prec)) {
    CK(cudaMemcpy(host, tensor_ptr<double>(ctx, which, ctx->cur, b), E * 8, cudaMemcpyDeviceToHost), "copy");
  } else {
    std::vector<float> tmp(E);
    CK(cudaMemcpy(tmp.data(), tensor_ptr<float>(ctx, which, ctx->cur, b), E * 4, cudaMemcpyDeviceToHost), "copy");
    for (int64_t i = 0; i < E; ++i) host[i] = tmp[i];
  }
  return HOTRG_OK;
}

hotrg_status hotrg_copy_isometry(hotrg_ctx* ctx, int b, int nu, double* host, size_t n) {
  hotrg_status r = check_ready(ctx);
  if (r != HOTRG_OK) return r;
  if (!host || b < 0 || b >= ctx->batch || nu < 0 || nu > 3 || ctx->last_mu < 0 || nu == ctx->last_mu)
    return HOTRG_EINVAL;
  const int chi = ctx->last_chi[nu];
  const int Dold = ctx->last_Dold[nu];
  const int64_t cnt = (int64_t)Dold * Dold * chi;
  if ((int64_t)n < cnt) return HOTRG_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  const double* U64 = (const double*)(ctx->ws + ctx->L.U64) + ((int64_t)b * 4 + nu) * kMaxGramN * kMaxLeg;
  CK(cudaMemcpy(host, U64, cnt * 8, cudaMemcpyDeviceToHost), "copy U");
  return HOTRG_OK;
}

hotrg_status hotrg_set_option(hotrg_ctx* ctx, int option, int value) {
  if (!ctx) return HOTRG_EINVAL;
  switch (option) {
    case HOTRG_OPT_JACOBI_SWEEPS:
      if (value < 1 || value > kJacobiMaxSweeps) return HOTRG_EINVAL;
      ctx->jacobi_sweeps = value;
      ctx->drop_graphs();
      return HOTRG_OK;
    case HOTRG_OPT_GEMM_VARIANT:
      if (value < 0 || value > (ctx->prec == HOTRG_FP16X3 ? 3 : 1)) return HOTRG_EINVAL;
      ctx->gemm_variant = value;
      ctx->drop_graphs();
      return HOTRG_OK;
    case HOTRG_OPT_GRAPHS:
      if (value < 0 || value > 1) return HOTRG_EINVAL;
      if (value && ctx->stream == nullptr) return HOTRG_EINVAL;
      ctx->use_graphs = value != 0;
      return HOTRG_OK;
    case HOTRG_OPT_AUTOTUNE:
      if (value < 0 || value > 1) return HOTRG_EINVAL;
      ctx->autotune = value != 0;
      return HOTRG_OK;
    case HOTRG_OPT_GROUP:
      if (value < 0 || value > kMaxGemmProblems) return HOTRG_EINVAL;
      ctx->group_max = value;
      return HOTRG_OK;
    case HOTRG_OPT_MAXNORM:
      if (value < kScaleNone || value > kScaleExact) return HOTRG_EINVAL;
      ctx->maxnorm = value;
      ctx->drop_graphs();
      return HOTRG_OK;
    default:
      return HOTRG_EINVAL;
  }
}

hotrg_status hotrg_split_stats(hotrg_ctx* ctx, hotrg_split_counts* out) {
  hotrg_status r = check_ready(ctx);
  if (r != HOTRG_OK) return r;
  if (!out) return HOTRG_EINVAL;
  if (ctx->prec != HOTRG_FP16X3) return HOTRG_EUNSUPPORTED;
  if (!ctx->initialised || ctx->last_kstep < 0) return HOTRG_ESTATE;
  const StepPlan& p = ctx->last_plan;
  const int nt = ntensors(ctx->impure_active);
  const int nbuild = (ctx->last_kstep == 0 && nt >= 3) ? 2 : nt;
  const Scratch sc = scratch_layout(p, p.xs, p.xs2, ctx->prec, ctx->impure_active, ctx->rsize);
  char* sb = ctx->ws + ctx->L.persistent_end;
  // the last group, the last slice block of A and (sliced) of B
  const int ca = p.chi[p.a];
  const int ne = ctx->batch - (ctx->batch - 1) / p.ne * p.ne;
  const int xs = ca - (ca - 1) / p.xs * p.xs, xs2 = ca - (ca - 1) / p.xs2 * p.xs2;
  const int64_t per_x = (int64_t)p.chi[p.b] * p.D[p.c] * p.D[p.c] * p.D[p.mu];
  const int64_t rowsA = (int64_t)p.xs * per_x, rowsB = (int64_t)p.xs2 * per_x;
  const int64_t Asz = p.P * rowsA * p.kps, Bsz = p.P * rowsB * p.kps;   // fp16 values per operand tensor
  unsigned long long* cnt = (unsigned long long*)(sb + sc.stats);   // [A hi, A lo, B hi, B lo][3]
  cudaStream_t st = ctx->stream;
  CK(cudaMemsetAsync(cnt, 0, 12 * sizeof(unsigned long long), st), "stats clear");
  for (int e = 0; e < ne; ++e)
    for (int w = 0; w < nbuild; ++w) {
      const int64_t ta = (int64_t)(e * nt + w) * Asz * 2, tb = (int64_t)(e * nt + w) * Bsz * 2;   // bytes
      CK(launch_plane_stats(sb + sc.A + ta, p.P * xs * per_x, p.Kp, p.kps, cnt + 0, st), "stats");
      CK(launch_plane_stats(sb + sc.Alo + ta, p.P * xs * per_x, p.Kp, p.kps, cnt + 3, st), "stats");
      CK(launch_plane_stats(sb + sc.B + tb, p.P * xs2 * per_x, p.Kp, p.kps, cnt + 6, st), "stats");
      CK(launch_plane_stats(sb + sc.Blo + tb, p.P * xs2 * per_x, p.Kp, p.kps, cnt + 9, st), "stats");
    }
  unsigned long long h[12];
  CK(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, st), "stats read");
  CK(cudaStreamSynchronize(st), "stats sync");
  const uint64_t nA = (uint64_t)ne * nbuild * p.P * xs * per_x * p.Kp;
  const uint64_t nB = (uint64_t)ne * nbuild * p.P * xs2 * per_x * p.Kp;
  auto half_value = [](unsigned long long bits) {   // magnitude bits of a finite fp16
    const int ex = (int)(bits >> 10) & 31, m = (int)(bits & 1023);
    return ex == 0 ? ldexp((double)m, -24) : ldexp(1.0 + m / 1024.0, ex - 15);
  };
  out->entries = nA + nB;
  out->hi_zero = h[0] + h[6];
  out->hi_subnormal = h[1] + h[7];
  out->lo_zero = h[3] + h[9];
  out->lo_subnormal = h[4] + h[10];
  out->hi_max[0] = half_value(h[2]);
  out->hi_max[1] = half_value(h[8]);
  return HOTRG_OK;
}

hotrg_status hotrg_autotune(hotrg_ctx* ctx, int dir, int dcut) {
  hotrg_status r = check_ready(ctx);
  if (r != HOTRG_OK) return r;
  if (dir < 0 || dir > 3 || dcut < 1 || dcut > ctx->dcut_max) return HOTRG_EINVAL;
  if (!ctx->initialised || ctx->sticky) return HOTRG_ESTATE;
  StepPlan p = make_plan(ctx->dims, dir, dcut, ctx->prec, ctx->batch);
  for (int n = 0; n < 4; ++n)
    if (p.newD[n] > kMaxLeg) return HOTRG_EINVAL;
  if (p.Enew > ctx->L.cap) return HOTRG_EWORKSPACE;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(ctx->stream, &cs), "capture query");
  if (cs != cudaStreamCaptureStatusNone) return HOTRG_ESTATE;
  TuneChoice tc{};
  r = f64_store(ctx->prec) ? tune_step<double>(ctx, dir, dcut, &tc) : tune_step<float>(ctx, dir, dcut, &tc);
  if (r != HOTRG_OK) return r;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[tune_key(ctx, dir, dcut)] = tc;
  ctx->tune_timed += 1;
  return HOTRG_OK;
}

hotrg_status hotrg_tune_stats(const hotrg_ctx* ctx, uint64_t* timed, uint64_t* hits) {
  if (!ctx) return HOTRG_EINVAL;
  if (timed) *timed = ctx->tune_timed;
  if (hits) *hits = ctx->tune_hits;
  return HOTRG_OK;
}

hotrg_status hotrg_selftest_wait(hotrg_ctx* ctx, int limit_ms) {
  hotrg_status r = check_ready(ctx);
  if (r != HOTRG_OK) return r;
  if (limit_ms < 1 || limit_ms > 1000) return HOTRG_EINVAL;
  int* status = (int*)(ctx->ws + ctx->L.status);
  LK(1, launch_wait_selftest(status, (unsigned long long)limit_ms * 1000000ull, ctx->stream), "selftest");
  return sync_and_status(ctx);
}

hotrg_status hotrg_profile_enable(hotrg_ctx* ctx, int enable) {
  if (!ctx) return HOTRG_EINVAL;
  if (ctx->ready) CK(cudaStreamSynchronize(ctx->stream), "sync");
  ctx->profiling = enable != 0;
  ctx->ev_used = 0;
  ctx->launches = 0;
  ctx->gemm_launches = 0;
  ctx->gemm_flops = 0;
  return HOTRG_OK;
}

hotrg_status hotrg_profile_read(hotrg_ctx* ctx, hotrg_profile* out) {
  if (!ctx || !out) return HOTRG_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  double ms = 0;
  for (size_t i = 0; i + 1 < ctx->ev_used; i += 2) {
    float t = 0;
    CK(cudaEventElapsedTime(&t, ctx->ev[i], ctx->ev[i + 1]), "event elapsed");
    ms += t;
  }
  out->launches = ctx->launches;
  out->gemm_launches = ctx->gemm_launches;
  out->gemm_ms = ms;
  out->gemm_flops = ctx->gemm_flops;
  return HOTRG_OK;
}

hotrg_status hotrg_step_flops(const hotrg_ctx* ctx, int dir, int dcut, double* main_flops, double* total_flops) {
  if (!ctx || dir < 0 || dir > 3 || dcut < 1) return HOTRG_EINVAL;
  StepPlan p = make_plan(ctx->dims, dir, dcut, ctx->prec);
  if (main_flops) *main_flops = p.main_flops;
  if (total_flops) *total_flops = p.total_flops;
  return HOTRG_OK;
}

}  // extern "C"
