// noalloc.cu - HOSVD isometry of one transverse direction without any device allocation.
//
// Some callers cannot allocate device memory at all: code running inside another
// framework's memory pool or under a strict memory budget, plugins handed only their
// input and output buffers, or a host thread that must not call into the allocator
// while other work is in flight. hotrg_isometry_noalloc serves them. It runs the same
// kernels as the isometry stage of hotrg_step (split-K Gram halves, chunk reduction,
// Gram merge, FP64 Jacobi with the canonical gauge, side choice + Gram-Schmidt), but
// every intermediate lives in one file-scope __device__ array of kNoAllocBytes bytes
// instead of in a caller workspace. Every GPU that loads the library keeps that array
// until the process exits.
//
// Host code cannot use the array's name as a device address (it names a host-side
// stand-in), so the first call on each device looks its device address up with
// cudaGetSymbolAddress while that device is current and caches it. Because of this
// set-up, the first call on a device should come before any stream capture.
//
// All calls share the array and it keeps the previous call's contents: the call clears
// the status words it counts into, and calls that overlap on the GPU (two streams, two
// host threads) race on it.
//
// Limits: bond dimensions up to 8 (the Gram matrices are then at most 64 x 64 and fit the
// array); any dcut >= 1 (chi = min(D_nu^2, dcut) <= 64 columns, which the candidate and
// output regions are sized for). A tensor with a NaN or infinity gives non-finite Gram
// eigenvalues, which the call reports as HOTRG_ENONFINITE.
#include <math.h>

#include <string>

#include "common.cuh"
#include "hotrg.h"

namespace hotrg {

// Largest bond dimension the array is sized for: the Gram matrices of a direction with
// D_nu <= 8 next to a step direction with D_mu <= 8 (R = D_nu D_mu <= 64, n = D_nu^2 <= 64).
constexpr int kNoAllocMaxLeg = 8;
constexpr int kNoAllocR = kNoAllocMaxLeg * kNoAllocMaxLeg;   // half-Gram side
constexpr int kNoAllocN = kNoAllocMaxLeg * kNoAllocMaxLeg;   // Gram side
constexpr int kNoAllocChunks = 32;                           // split-K chunks per half-Gram
constexpr size_t kNoAllocBytes = 8u << 20;                   // 8 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

constexpr int kMaxDevices = 64;
void* g_scratch_dev[kMaxDevices] = {};

constexpr size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// Offsets inside the array (bytes).
struct NoAllocLayout {
  size_t status, part, half, G, lam, eps, degen, Ucand, recs, U64r, total;
};

constexpr NoAllocLayout layout() {
  NoAllocLayout L{};
  size_t o = 0;
  L.status = o;  o = up256(o + kStWords * sizeof(int));
  L.part = o;    o = up256(o + (size_t)4 * kNoAllocChunks * kNoAllocR * kNoAllocR * sizeof(double));
  L.half = o;    o = up256(o + (size_t)4 * kNoAllocR * kNoAllocR * sizeof(double));
  L.G = o;       o = up256(o + (size_t)2 * kNoAllocN * kNoAllocN * sizeof(double));
  L.lam = o;     o = up256(o + (size_t)2 * kNoAllocN * sizeof(double));
  L.eps = o;     o = up256(o + 2 * sizeof(double));
  L.degen = o;   o = up256(o + 2 * sizeof(int));
  L.Ucand = o;   o = up256(o + (size_t)2 * kNoAllocN * kNoAllocN * sizeof(double));   // chi <= n
  L.recs = o;    o = up256(o + sizeof(DevRecord));
  L.U64r = o;    o = up256(o + (size_t)kNoAllocN * kNoAllocN * sizeof(double));
  L.total = o;
  return L;
}
static_assert(layout().total <= kNoAllocBytes, "no-alloc scratch layout exceeds the array");

hotrg_status fail(hotrg_status s, const std::string& msg) {
  set_last_error(msg.c_str());
  return s;
}

}  // namespace
}  // namespace hotrg

using namespace hotrg;

extern "C" hotrg_status hotrg_isometry_noalloc(const double* T_dev, const int dims[4], int mu, int nu, int dcut,
                                               double* U_dev, double* eps_dev, int* primed_dev, void* stream) {
  if (!T_dev || !dims || !U_dev || !eps_dev || !primed_dev)
    return fail(HOTRG_EINVAL, "hotrg_isometry_noalloc: null pointer");
  if (mu < 0 || mu > 3 || nu < 0 || nu > 3 || mu == nu || dcut < 1)
    return fail(HOTRG_EINVAL, "hotrg_isometry_noalloc: bad mu, nu or dcut");
  for (int n = 0; n < 4; ++n)
    if (dims[n] < 1 || dims[n] > kNoAllocMaxLeg)
      return fail(HOTRG_EINVAL, "hotrg_isometry_noalloc: bond dimension " + std::to_string(dims[n]) +
                                    " exceeds the limit of the fixed scratch array (" +
                                    std::to_string(kNoAllocMaxLeg) + ")");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(HOTRG_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(HOTRG_EUNSUPPORTED, "hotrg_isometry_noalloc: device index");
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(HOTRG_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_dev[dev] = p;
  }
  unsigned char* base = (unsigned char*)g_scratch_dev[dev];
  constexpr NoAllocLayout L = layout();
  int* status = (int*)(base + L.status);

  const int Dn = dims[nu], Dm = dims[mu];
  const int n = Dn * Dn, chi = n < dcut ? n : dcut, R = Dn * Dm;
  int64_t ts[8], s = 1;
  for (int leg = 7; leg >= 0; --leg) {
    ts[leg] = s;
    s *= dims[leg / 2];
  }
  const int64_t E = s;
  int64_t nch = (E / R + 511) / 512;
  if (nch > kNoAllocChunks) nch = kNoAllocChunks;
  if (nch < 1) nch = 1;

#define NA_CK(call, what)                                                              \
  do {                                                                                 \
    cudaError_t e__ = (call);                                                          \
    if (e__ != cudaSuccess) return fail(HOTRG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e__)); \
  } while (0)

  NA_CK(cudaMemsetAsync(status, 0, kStWords * sizeof(int), st), "clear status");
  // Gram halves: (side, half) -> rows (leg of nu on that side, mu' leg for T1 / mu leg for T2)
  GramPack gp{};
  double* part = (double*)(base + L.part);
  double* half = (double*)(base + L.half);
  for (int side = 0; side < 2; ++side) {
    for (int h = 0; h < 2; ++h) {
      GramJob& j = gp.j[side * 2 + h];
      const int leg = 2 * nu + side, kleg = h == 0 ? 2 * mu + 1 : 2 * mu;
      j.T = T_dev;
      j.D1 = Dn;
      j.D2 = Dm;
      j.s1 = ts[leg];
      j.s2 = ts[kleg];
      j.nrest = 0;
      j.K = 1;
      for (int l = 0; l < 8; ++l) {
        if (l == leg || l == kleg) continue;
        j.rdims[j.nrest] = dims[l / 2];
        j.rst[j.nrest] = ts[l];
        j.K *= dims[l / 2];
        ++j.nrest;
      }
      j.partial = part + (int64_t)(side * 2 + h) * kNoAllocChunks * kNoAllocR * kNoAllocR;
    }
  }
  NA_CK(launch_gram<double>(gp, 4, R, (int)nch, st), "gram");
  NA_CK(launch_gram_reduce(gp, 4, (int)nch, (int64_t)R * R, (int64_t)kNoAllocR * kNoAllocR, half, st), "gram reduce");
  double* G = (double*)(base + L.G);
  for (int side = 0; side < 2; ++side)
    NA_CK(launch_gram_merge(half + (int64_t)(side * 2) * kNoAllocR * kNoAllocR,
                            half + (int64_t)(side * 2 + 1) * kNoAllocR * kNoAllocR, Dn, Dm,
                            G + (int64_t)side * kNoAllocN * kNoAllocN, st),
          "gram merge");
  EigPack ep{};
  for (int side = 0; side < 2; ++side) {
    EigJob& j = ep.j[side];
    j.n = n;
    j.chi = chi;
    j.G = G + (int64_t)side * kNoAllocN * kNoAllocN;
    j.work = nullptr;  // n <= 64: the eigensolver keeps A and V in shared memory
    j.lam = (double*)(base + L.lam) + side * kNoAllocN;
    j.eps = (double*)(base + L.eps) + side;
    j.degenerate = (int*)(base + L.degen) + side;
    j.U = (double*)(base + L.Ucand) + (int64_t)side * kNoAllocN * kNoAllocN;
  }
  NA_CK(launch_jacobi(ep, 2, n, 1e-10, status, st), "jacobi");
  SelectPack sp{};
  DevRecord* rec = (DevRecord*)(base + L.recs);
  SelectJob& sj = sp.j[0];
  sj.U[0] = ep.j[0].U;
  sj.U[1] = ep.j[1].U;
  sj.lam0 = ep.j[0].lam;
  sj.eps[0] = ep.j[0].eps;
  sj.eps[1] = ep.j[1].eps;
  sj.degen[0] = ep.j[0].degenerate;
  sj.degen[1] = ep.j[1].degenerate;
  sj.U64 = U_dev;
  sj.Ur = (double*)(base + L.U64r);
  sj.n = n;
  sj.chi = chi;
  sj.rec_eps = eps_dev;
  sj.rec_primed = primed_dev;
  sj.rec_degen = &rec->degen[0];
  sj.rec_b = nullptr;             // explicit record pointers above
  sj.step = nullptr;
  sj.nu = nu;
  NA_CK(launch_select<double>(sp, 1, 1e-9, st), "select");
  int host_status[kStWords];
  double host_lam[2 * kNoAllocN];
  NA_CK(cudaMemcpyAsync(host_status, status, sizeof(host_status), cudaMemcpyDeviceToHost, st), "status read");
  NA_CK(cudaMemcpyAsync(host_lam, base + L.lam, sizeof(host_lam), cudaMemcpyDeviceToHost, st), "spectrum read");
  NA_CK(cudaStreamSynchronize(st), "sync");
#undef NA_CK
  // a NaN or infinity anywhere in T reaches a diagonal entry of a Gram matrix, which no
  // rotation clears: the spectra show it
  for (int side = 0; side < 2; ++side)
    for (int i = 0; i < n; ++i)
      if (!isfinite(host_lam[side * kNoAllocN + i]))
        return fail(HOTRG_ENONFINITE, "hotrg_isometry_noalloc: non-finite Gram spectrum (NaN or infinity in T)");
  if (host_status[kStNoConv]) return fail(HOTRG_ENOCONV, "hotrg_isometry_noalloc: Jacobi sweep limit reached");
  return HOTRG_OK;
}
