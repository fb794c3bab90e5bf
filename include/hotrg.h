/*
 * hotrg.h - C ABI of the GB300 (sm_103a) HOTRG library for the 4D Ising model.
 *
 * What it computes (arXiv:1911.12954, Sec. 2, Fig. 1; impure-tensor observables of
 * Sec. 3.1): the higher-order tensor renormalisation group. A site tensor
 * T[x,x',y,y',z,z',t,t'] (unprimed leg of direction nu points to -nu, primed to +nu)
 * is coarse-grained along a direction mu by merging two neighbouring tensors; every
 * transverse direction nu gets an isometry U^nu (D_nu^2 -> chi_nu = min(D_nu^2, D_cut))
 * from the HOSVD of the pair, and the O(D^15) block-spin contraction produces the new
 * tensor, which is normalised by its Frobenius norm c. After k steps the lattice has
 * V = 2^k sites and ln Z / V = sum_i ln(c_i) / 2^i + ln(Tr T_k) / 2^k.
 *
 * Conventions shared by every call:
 *  - A context holds `batch` independent runs (one per temperature); everything is per
 *    batch element b in [0, batch).
 *  - Device memory and the CUDA stream belong to the caller. The library never calls
 *    cudaMalloc; it carves the caller's workspace (hotrg_set_workspace) and launches
 *    on the caller's stream (hotrg_set_stream; default: the legacy default stream).
 *  - Every call returns a hotrg_status and never aborts. Calls that return host values
 *    synchronise the stream and report device-side errors (eigensolver not converged,
 *    non-finite norm, timeout) raised by earlier asynchronous steps. After an error the
 *    context is sticky (HOTRG_ESTATE) until hotrg_init_tensor or hotrg_set_tensor.
 *  - Host arrays passed in are read before the call returns; host arrays passed out
 *    are written before it returns. Layout of a tensor on the host: row-major FP64
 *    over legs [x, x', y, y', z, z', t, t'] with sizes (Dx, Dx, Dy, Dy, Dz, Dz, Dt, Dt).
 */
#ifndef HOTRG_H
#define HOTRG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hotrg_ctx hotrg_ctx; /* opaque, created by hotrg_create, host-owned */

typedef enum {
  HOTRG_OK = 0,
  HOTRG_EINVAL = -1,      /* bad argument (null pointer, dir, dcut, batch index, sizes) */
  HOTRG_EWORKSPACE = -2,  /* no workspace set, or too small for the requested step      */
  HOTRG_ECUDA = -3,       /* a CUDA runtime call failed (message: hotrg_last_error)     */
  HOTRG_ENOCONV = -4,     /* Jacobi eigensolver hit its sweep limit                     */
  HOTRG_ENONFINITE = -5,  /* a norm or trace was not finite / not positive             */
  HOTRG_ETIMEOUT = -6,    /* a bounded device-side wait gave up                         */
  HOTRG_ESTATE = -7,      /* call out of order, or context sticky after an error        */
  HOTRG_EUNSUPPORTED = -8 /* precision or size not built into this library              */
} hotrg_status;

/* Arithmetic of the block-spin contraction and the Gram build.
 * HOTRG_FP64  : FP64 everywhere (DFMA).                                     reference
 * HOTRG_FP32  : FP32 SIMT FMA, FP32 accumulation; tensors stored in FP32.
 * HOTRG_TF32X3: tcgen05 tensor cores, each FP32 operand split into tf32 hi + lo,
 *               products hi*hi + hi*lo + lo*hi accumulated in FP32 (TMEM, promoted
 *               to FP32 registers every 32 k).
 * HOTRG_FP16X3: the same three products on fp16 hi + lo planes of 2^e x, e a power of two
 *               per operand from its magnitude (max-norm scaling, HOTRG_OPT_MAXNORM),
 *               removed in the GEMM epilogue (kind::f16: twice the tensor rate and half
 *               the operand bytes of TF32X3).
 * HOTRG_FP64OZ: FP64-grade block-spin product on the fp16 tensor cores (Ozaki-type
 *               splitting): tensors stored in FP64, each GEMM operand scaled by a power of
 *               two below 1 in magnitude (from its exact largest entry) and split into 5
 *               planes of exact 8-bit integer slices, the 15 leading slice products summed
 *               exactly per 256-k chunk (FP32 in TMEM) and across chunks as float pairs;
 *               error below 2^-40 of the operands' largest magnitudes per product term.
 *               Pure and impure tensors: the reference for the mixed modes at large D_cut,
 *               where the DFMA product of HOTRG_FP64 takes about 25 min per step (D_cut =
 *               10).
 * In every mode the Gram matrices are accumulated in FP64 (float pairs of FP32 slice
 * sums for FP32-stored tensors), and the eigensolver, the isometries, the norm and
 * ln Z / V are FP64. */
typedef enum {
  HOTRG_FP64 = 0,
  HOTRG_FP32 = 1,
  HOTRG_TF32X3 = 2,
  HOTRG_FP16X3 = 3,
  HOTRG_FP64OZ = 4
} hotrg_precision;

/* Impure tensors propagated with the pure one (same isometries, same c):
 * SIGMA: S (one sigma inserted) -> magnetisation <sigma> = Tr S / Tr T.
 * SIGMASIGMA: M (sigma_n sigma_{n+mu0}, mu0 = first step's direction) -> <sigma sigma>;
 * requires SIGMA. */
enum { HOTRG_IMPURE_NONE = 0, HOTRG_IMPURE_SIGMA = 1, HOTRG_IMPURE_SIGMASIGMA = 2 };

/* Per-step record kept for every batch element (FP64). */
typedef struct {
  int mu;            /* direction of the step: 0..3 = x, y, z, t                      */
  int dims[4];       /* bond dimensions after the step                               */
  int primed[4];     /* per transverse nu: 1 if the nu' side of the HOSVD was taken    */
  double eps[4][2];  /* per transverse nu: discarded eigenvalue sum, nu and nu' side   */
  double ln_c;       /* ln of the Frobenius norm of the new tensor before normalising */
  int degenerate[4]; /* per transverse nu: the cut fell inside an eigenvalue cluster   */
  int slices[2];     /* slices of the new a leg taken for A (rows) and for B (rows) when
                        the workspace was smaller than the unsliced plan (1 = unsliced) */
  int closing;       /* transverse direction closed by the last two isometry passes    */
  int gemm_option;   /* HOTRG_OPT_GEMM_VARIANT value of the block-spin GEMM (-1: the
                        CUDA-core GEMM of the FP64 and FP32 modes)                      */
  int tuned;         /* 1 if closing and gemm_option came from the autotuner's cache    */
  int group;         /* batch elements contracted together (each launch of the
                        contraction covered this many temperatures)                     */
} hotrg_step_record;

/* Create a context for `batch` runs with bond dimensions up to `dcut_max`
 * (2 <= dcut_max <= 16), precision `prec` and impure mask. No device memory is
 * touched. Errors: EINVAL. */
hotrg_status hotrg_create(hotrg_ctx** out, int batch, int dcut_max, int prec, int impure_mask);

/* Release the context (not the caller's workspace). Accepts NULL. */
hotrg_status hotrg_destroy(hotrg_ctx* ctx);

/* Plan a run and return the bytes of device workspace it needs: the steps `dirs[i]`,
 * `dcuts[i]` (i < nsteps) from the 2x2x2x2 initial tensor or, when dims0 != NULL, from a
 * tensor of bond dimensions dims0[4] given to hotrg_set_tensor. With nsteps == 0 the
 * bound covers any step whose bond dimensions are all <= dcut_max. The plan fixes the
 * per-tensor capacity used by the next hotrg_set_workspace. The returned size lets every
 * step contract unsliced; a smaller workspace (at least the persistent part plus one
 * X slice) makes hotrg_step slice the new a-leg instead. Errors: EINVAL. */
hotrg_status hotrg_workspace_size(hotrg_ctx* ctx, int nsteps, const int* dirs, const int* dcuts,
                                  const int* dims0, size_t* bytes);

/* Give the library `bytes` bytes of device memory at `dev_ptr` (256-byte aligned),
 * owned by the caller, kept until the next call of this function or hotrg_destroy.
 * Errors: EINVAL (null or misaligned pointer). */
hotrg_status hotrg_set_workspace(hotrg_ctx* ctx, void* dev_ptr, size_t bytes);

/* Launch all later work on `cuda_stream` (a cudaStream_t, caller-owned; NULL =
 * legacy default stream). */
hotrg_status hotrg_set_stream(hotrg_ctx* ctx, void* cuda_stream);

/* Site tensors of the 4D Ising model (Fig. 1A; H = -sum s s' - h sum s):
 * T[i1..i8] = sum_s e^{beta h s} prod_j W[s, i_j], W = [[sqrt(cosh b), sqrt(sinh b)],
 * [sqrt(cosh b), -sqrt(sinh b)]]; S the same with an extra factor s. beta[b], h[b] are
 * host arrays of length batch (beta >= 0). Resets the step counter, ln Z accumulator,
 * records and sticky error. Asynchronous. Errors: EINVAL, EWORKSPACE, ECUDA. */
hotrg_status hotrg_init_tensor(hotrg_ctx* ctx, const double* beta, const double* h);

/* Replace the pure tensor of batch element b by the host tensor `T_host` with bond
 * dimensions dims[4] (each <= dcut_max; layout in the header comment); the stored
 * tensor is T_host / ||T_host||_F and ln ||T_host|| starts the accumulator. Disables
 * impure tensors for the context. For kernel-level tests. Synchronous. */
hotrg_status hotrg_set_tensor(hotrg_ctx* ctx, int b, const int dims[4], const double* T_host);

/* One coarse-graining step along `dir` (0..3) with cut `dcut` (>= 1, <= dcut_max),
 * for every batch element: Gram matrices on both sides of the three transverse bond
 * pairs (FP64 accumulation), Jacobi eigendecomposition (FP64, on the GPU), isometries
 * from the side with the smaller discarded eigenvalue sum, the block-spin contraction
 * in the context's precision, normalisation by ||T'||_F and ln c / 2^k accumulated in
 * FP64. Impure tensors follow with the same isometries and c. Asynchronous on the
 * stream; device-side failures are reported by the next synchronising call.
 * Errors: EINVAL, EWORKSPACE, ESTATE, ECUDA. */
hotrg_status hotrg_step(hotrg_ctx* ctx, int dir, int dcut);

/* ln Z / V of the 2^k-site periodic lattice after the k steps done so far, per batch
 * element (host array of length batch). Synchronises. */
hotrg_status hotrg_lnZ(hotrg_ctx* ctx, double* lnZ_over_V);

/* <sigma> = Tr S_k / Tr T_k per batch element. Needs HOTRG_IMPURE_SIGMA. */
hotrg_status hotrg_impure_magnetization(hotrg_ctx* ctx, double* m);

/* <sigma_n sigma_{n+mu0}> = Tr M_k / Tr T_k and E/V = -4 <sigma sigma> - h <sigma>
 * per batch element (k >= 1). Needs HOTRG_IMPURE_SIGMASIGMA. Either pointer may be
 * NULL. */
hotrg_status hotrg_impure_energy(hotrg_ctx* ctx, double* e, double* sigma_sigma);

/* Degeneracy indicator X of the current tensor along direction nu (0..3 = x, y, z, t), per
 * batch element (host array of length batch): M[i][j] = T with leg nu = i, leg nu' = j and
 * every other direction traced, X = (Tr M)^2 / Tr(M M). Sec. 3.1 of arXiv:1911.12954 locates
 * T_c from X (citing Gu and Wen for the definition, restated here): after many steps X is 1
 * in the symmetric phase and 2 when Z2 is broken. FP64 sums on the device. Valid after any
 * number of steps (k = 0 included). Synchronises. Errors: EINVAL (nu, NULL), ESTATE (not
 * initialised), ENONFINITE (Tr(M M) = 0 or a non-finite tensor). */
hotrg_status hotrg_x_indicator(hotrg_ctx* ctx, int nu, double* X);

/* Record of step `step` (1-based, <= steps done) of batch element b. Synchronises. */
hotrg_status hotrg_step_info(hotrg_ctx* ctx, int b, int step, hotrg_step_record* rec);

/* Number of steps done since the last init/set_tensor; current bond dimensions. */
hotrg_status hotrg_state(const hotrg_ctx* ctx, int* steps_done, int dims[4]);

/* Copy tensor `which` (0 = T, 1 = S, 2 = M) of batch element b to the host as FP64,
 * normalised as stored; `n` = capacity of `host` in elements (must be >= Dx^2 Dy^2
 * Dz^2 Dt^2). Synchronises. */
hotrg_status hotrg_copy_tensor(hotrg_ctx* ctx, int which, int b, double* host, size_t n);

/* Copy the isometry U^nu of the last step (b, nu transverse) to the host as FP64,
 * row-major [(i1*D_nu + i2)][chi_nu]; `n` = capacity. Synchronises. */
hotrg_status hotrg_copy_isometry(hotrg_ctx* ctx, int b, int nu, double* host, size_t n);

/* Algorithmic floating-point operations of the next step along `dir` with `dcut` from
 * the current bond dimensions D, per batch element and per tensor product (2 flops per
 * multiply-add). main = 2 (chi_a chi_b D_c^2 D_mu)^2 (D_a^2 D_b^2 D_mu), the block-spin
 * contraction (2 D^15 when every dimension is D), with c the transverse direction that
 * makes it smallest; total adds the isometry applications, the closing contractions and
 * the Gram build. Host-only, no device access. */
hotrg_status hotrg_step_flops(const hotrg_ctx* ctx, int dir, int dcut, double* main_flops,
                              double* total_flops);

/* Tuning and test options of a context (host-side; take effect from the next step).
 * HOTRG_OPT_JACOBI_SWEEPS: sweep limit of the eigensolver, 1..60 (default 60); reaching it
 *   raises HOTRG_ENOCONV at the next synchronising call (used to test that path).
 * HOTRG_OPT_GEMM_VARIANT: tensor-core GEMM pipeline. TF32X3: 0 = 4 stages of 16-wide
 *   k-blocks (default), 1 = 2 stages of 32-wide k-blocks. FP16X3: 0 = partial sums promoted
 *   from the tensor-core accumulator to FP32 registers every 128 k, each 256 x 256 tile
 *   computed by a pair of CTAs on two SMs (tcgen05.mma.cta_group::2; each CTA loads half of
 *   the B tile) (default); 1 = every 64 k (slower, a smaller truncation bias), 2 = every
 *   256 k (faster, a larger one), 3 = every 128 k, one CTA per 128 x 256 tile (1..3 one CTA
 *   per tile).
 * HOTRG_OPT_GRAPHS: 1 = capture each distinct step (plan, buffer, first step or not) once
 *   into a CUDA graph and replay it (every kernel of the step for every batch element in
 *   one graph launch); needs a non-default stream (hotrg_set_stream). Per-GEMM profiling
 *   events are not recorded in this mode.
 * HOTRG_OPT_AUTOTUNE: 1 = every step takes its closing direction and GEMM pipeline from the
 *   autotuner's cache (hotrg_autotune), timing a step shape it has not seen before the step
 *   runs (outside any capture; with HOTRG_OPT_GRAPHS, tune every shape with
 *   hotrg_autotune before the first captured step). 0 (default) = the planner's choice:
 *   the closing direction with the fewest flops and the option's pipeline.
 * HOTRG_OPT_GROUP: most batch elements contracted together, 0..96 (0, the default: as many
 *   as the planner finds best). The isometry stage and the normalisation always run once
 *   for the whole batch; the contraction runs group by group, every launch covering the
 *   group (tensor passes over all its elements, one grouped GEMM for all its outputs). The
 *   planner compares one element at a time (slices with the fewest GEMM blocks) with groups
 *   that fit the workspace with B unsliced, and takes the fewest launches; results do not
 *   depend on the grouping (every element's arithmetic is the same, its operand scales
 *   included).
 * HOTRG_OPT_MAXNORM: FP16X3 operand scaling. Each operand side of each batch element is
 *   multiplied by a power of two 2^e with B 2^e in [2^14, 2^15), B a bound of its largest
 *   magnitude m, so that no entry overflows the fp16 planes; the GEMM epilogue multiplies by
 *   2^-(eA + eB) (exact). 1 (default) = B recorded by the first half-contraction pass, no
 *   extra pass: sqrt(D_b) times that pass's largest |output|, a bound of every operand entry
 *   by Cauchy-Schwarz (the second pass applies part of an isometry column); the largest
 *   entry then sits at most log2(B / m) + 1 bits below 2^15. 2 = B = m, from a max pass
 *   that computes the second pass's outputs once more (largest entry in [2^14, 2^15)).
 *   0 = the fixed 2^14 of every operand. Other precisions ignore it (FP64OZ always scales
 *   by the exact largest magnitude, from a max pass).
 * Errors: EINVAL. */
enum {
  HOTRG_OPT_JACOBI_SWEEPS = 1,
  HOTRG_OPT_GEMM_VARIANT = 2,
  HOTRG_OPT_GRAPHS = 3,
  HOTRG_OPT_AUTOTUNE = 4,
  HOTRG_OPT_GROUP = 5,
  HOTRG_OPT_MAXNORM = 6
};
hotrg_status hotrg_set_option(hotrg_ctx* ctx, int option, int value);

/* Autotuner: times, on the GPU and on the run's current tensors, every plan of the step
 * hotrg_step(ctx, dir, dcut) would run next that computes the same contraction: each
 * closing direction (the transverse direction whose isometries are applied last; it sets
 * the shapes of the half contractions and of the block-spin GEMM, Sec. 2) and, in the
 * tensor-core modes, each pipeline that gives the same products (FP16X3: CTA pairs or one
 * CTA per tile; TF32X3: 16- or 32-wide k-blocks). The fastest (ties to the planner's
 * choice) is cached for this device and step shape (bond dimensions, direction, cut,
 * precision, batch, tensors, workspace size) for the life of the process and used by
 * every context with HOTRG_OPT_AUTOTUNE set. The run does not advance: the current
 * tensors, ln Z and the step counter are unchanged. Synchronises the stream; not allowed
 * while the stream is being captured (ESTATE). Errors: EINVAL, EWORKSPACE, ESTATE,
 * ECUDA and the device-side statuses. */
hotrg_status hotrg_autotune(hotrg_ctx* ctx, int dir, int dcut);

/* Shapes this context has timed (hotrg_autotune or HOTRG_OPT_AUTOTUNE) and steps whose plan
 * it took from the cache. Errors: EINVAL. */
hotrg_status hotrg_tune_stats(const hotrg_ctx* ctx, uint64_t* timed, uint64_t* hits);

/* Failure-detection self-test: on the context's stream, one thread waits, with the same
 * bounded wait the tensor-core GEMM uses on its mbarriers, on a barrier that nothing
 * signals, for limit_ms (1..1000) milliseconds. The wait gives up, raises the timeout status
 * word in the workspace and the kernel returns; no copies or MMAs are in flight in it. The
 * call synchronises and returns HOTRG_ETIMEOUT like any device-side timeout; the context is
 * sticky until hotrg_init_tensor / hotrg_set_tensor, and the CUDA context stays usable. */
hotrg_status hotrg_selftest_wait(hotrg_ctx* ctx, int limit_ms);

/* Launch accounting of one context, for benchmarks. */
typedef struct {
  uint64_t launches;      /* CUDA kernels this context launched since the last reset         */
  uint64_t gemm_launches; /* launches of the block-spin GEMM (the O(D^15) product)            */
  double gemm_ms;         /* their summed device time, CUDA events on the context's stream   */
  double gemm_flops;      /* their summed algorithmic flops, 2 M N K each                    */
} hotrg_profile;

/* enable != 0: from now on record a CUDA event pair around every GEMM launch (host-side
 * events, no device memory); any call resets the counters. */
hotrg_status hotrg_profile_enable(hotrg_ctx* ctx, int enable);

/* Counters since the last hotrg_profile_enable. Synchronises the stream. */
hotrg_status hotrg_profile_read(hotrg_ctx* ctx, hotrg_profile* out);

/* Rounding statistics of the FP16X3 split (max-norm scaling, HOTRG_OPT_MAXNORM), over the
 * operands of the last block-spin GEMM of the last step (the A and B planes still in the
 * workspace: every tensor of the last group of batch elements, the last slice block of
 * each side). An operand entry x is stored as hi = fp16(2^e x), lo = fp16(2^e x - hi). */
typedef struct {
  uint64_t entries;       /* operand entries counted (A and B)                                */
  uint64_t hi_zero;       /* entries whose hi is zero                                         */
  uint64_t hi_subnormal;  /* entries whose hi is nonzero and below 2^-14 (fp16 subnormal)     */
  uint64_t lo_zero;       /* entries whose lo is zero (hi holds 2^e x exactly)                */
  uint64_t lo_subnormal;  /* entries whose lo is nonzero and below 2^-14: bits lost           */
  double hi_max[2];       /* largest |hi| of the A and of the B operands (below 2^15)        */
} hotrg_split_counts;

/* Counts over the last step's operands (reads the workspace; synchronises the stream).
 * Errors: EUNSUPPORTED unless the precision is FP16X3; ESTATE before the first step after
 * hotrg_init_tensor / hotrg_set_tensor. */
hotrg_status hotrg_split_stats(hotrg_ctx* ctx, hotrg_split_counts* out);

/* HOSVD isometry of one transverse direction, for callers that cannot allocate device
 * memory. The paper has no counterpart: this is an allocation-free form of the isometry
 * stage of hotrg_step for code that runs inside another framework's memory pool or
 * under a fixed memory budget, plugins handed only their input and output buffers, and
 * threads that must not enter the allocator while other GPU work is in flight.
 *
 * Input: T_dev, a device FP64 tensor with bond dimensions dims[4] in the library's
 * layout (header comment); step direction mu, transverse direction nu (mu != nu), cut
 * dcut. Output (device memory, caller-owned): U_dev, the isometry as in
 * hotrg_copy_isometry (row-major [(i1 D_nu + i2)][chi], chi = min(D_nu^2, dcut)),
 * eps_dev[2], the discarded eigenvalue sums of the nu and nu' sides, primed_dev[0], 1
 * if the nu' side was taken. Same kernels, tolerances and canonical gauge as the FP64
 * mode of hotrg_step. Runs on `stream` (cudaStream_t, NULL = legacy default) and
 * returns after the results are written (synchronises the stream).
 *
 * It allocates nothing: all intermediates live in one fixed device array of 8 MiB
 * inside the library, held by every GPU that loads the library until the process
 * exits. Limit: every bond dimension <= 8 (larger ones return HOTRG_EINVAL with the
 * reason in hotrg_last_error); any dcut >= 1 (chi <= D_nu^2 <= 64). The first call on a
 * device looks up that array's device address (make it before any stream capture). Calls
 * share the array, so calls that overlap on the GPU race; each call clears the status
 * words it uses. A NaN or infinity in T_dev gives HOTRG_ENONFINITE (U_dev and eps_dev
 * then hold no usable values).
 * Errors: EINVAL, ECUDA, ENOCONV, ENONFINITE. */
hotrg_status hotrg_isometry_noalloc(const double* T_dev, const int dims[4], int mu, int nu, int dcut,
                                    double* U_dev, double* eps_dev, int* primed_dev, void* stream);

/* Text of a status code, and the last CUDA error message seen by this thread. */
const char* hotrg_status_string(int status);
const char* hotrg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HOTRG_H */
