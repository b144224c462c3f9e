// qp_pcg_solve_taps_static: the taps-backend PCG solve for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running while another component holds the device-memory budget
// (a serving process that reserved all free memory for its own pool), code that must not change the device's
// allocation state during a latency-critical phase, or embedders whose memory is owned by another runtime.
// This entry point serves them: it builds nothing in the heap of the device and calls no cudaMalloc,
// cudaFree or allocating library routine. Every intermediate the solve needs (the coefficient tables, the
// diagonal preconditioner, the PCG vectors, the reduction partials and the solver state) lives in one
// file-scope __device__ array of fixed size, which every GPU that loads this library holds until the process
// exits. The caller passes the right-hand sides and the solution buffer, as for qp_pcg_solve.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "qp_internal.cuh"

namespace qp {

constexpr size_t kStaticScratchBytes = (size_t)QP_STATIC_SCRATCH_BYTES;

// The shared scratch. Host code must not pass its name to a kernel (in host code it is a host-side stand-in,
// not a device address); the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {

std::mutex g_static_mutex;
void* g_static_addr[64] = {};   // device address of g_static_scratch per device id, set on first use

// Device address of the scratch on the current device (looked up once per device, with it current).
unsigned char* static_scratch_address() {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) raise(QP_ERR_UNSUPPORTED, "device ordinal beyond 63");
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      raise(QP_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") + cudaGetErrorString(e));
    }
    g_static_addr[dev] = p;
  }
  return static_cast<unsigned char*>(g_static_addr[dev]);
}

// Bump allocator over the static scratch (256-byte aligned pieces); raises when the request does not fit.
struct Carve {
  unsigned char* base;
  size_t used = 0;
  template <typename T> T* take(size_t count) {
    const size_t bytes = (count * sizeof(T) + 255) / 256 * 256;
    if (used + bytes > kStaticScratchBytes)
      raise(QP_ERR_INVALID_ARG, "problem too large for the static scratch of qp_pcg_solve_taps_static (" +
                                    std::to_string(kStaticScratchBytes) + " bytes)");
    T* p = reinterpret_cast<T*>(base + used);
    used += bytes;
    return p;
  }
};


// Host description built without heap memory: geometry plus the merged, Hermitian-checked taps, sorted as
// [mean][star taps per axis][multi-axis taps] (the device layout of PlanDev).
struct HostTaps {
  PlanDev pd;
  double2 c64[MAXT * 6];
  float2 c32[MAXT * 6];
  StarParams star;
  bool real = true;
};

void build_host(int d, int n, const double* P, const int* N, const qp_coeff* c, HostTaps& ht) {
  if (d < 1 || d > MAXD || n < d || n > MAXN) raise(QP_ERR_INVALID_ARG, "need 1 <= d <= 3 and d <= n <= 6");
  if (!P || !N || !c) raise(QP_ERR_INVALID_ARG, "P, N and coeff must be non-null");
  if (c->repr != QP_REPR_TAPS) raise(QP_ERR_INVALID_ARG, "qp_pcg_solve_taps_static takes a tap coefficient");
  if (c->kind < QP_COEF_SCALAR || c->kind > QP_COEF_SYM) raise(QP_ERR_INVALID_ARG, "unknown coefficient kind");
  if (c->ntaps < 1 || c->ntaps > MAXT || !c->tap_k || !c->tap_val) raise(QP_ERR_INVALID_ARG, "bad tap list");
  PlanDev& pd = ht.pd;
  std::memset(&pd, 0, sizeof(pd));
  ht.real = true;
  int64_t D = 1;
  for (int j = 0; j < n; ++j) {
    if (N[j] < 2 || N[j] > 1024) raise(QP_ERR_INVALID_ARG, "every N_j must be in 2..1024");
    D *= N[j];
  }
  if (D > (int64_t(1) << 30)) raise(QP_ERR_INVALID_ARG, "D must be <= 2^30");
  pd.n = n;
  pd.d = d;
  pd.D = (int)D;
  pd.kind = c->kind;
  pd.ncomp = c->kind == QP_COEF_SCALAR ? 1 : (c->kind == QP_COEF_DIAG ? d : d * (d + 1) / 2);
  pd.backend = QP_BACKEND_TAPS;
  int st = 1;
  for (int j = n - 1; j >= 0; --j) {
    pd.N[j] = N[j];
    pd.Nst[j] = N[j];
    pd.nyq[j] = -1;
    pd.stride[j] = st;
    pd.div[j] = make_fastdiv((uint32_t)N[j]);
    st *= N[j];
  }
  pd.hspec = 0;
  pd.Hl = (N[n - 1] + 1) / 2;
  for (int j = n; j < MAXN; ++j) {
    pd.N[j] = 1;
    pd.Nst[j] = 1;
    pd.nyq[j] = -1;
    pd.stride[j] = (int)D;
    pd.div[j] = make_fastdiv(1);
  }
  for (int a = 0; a < d; ++a)
    for (int j = 0; j < n; ++j) {
      if (!std::isfinite(P[a * n + j])) raise(QP_ERR_INVALID_ARG, "P has a non-finite entry");
      pd.P[a][j] = P[a * n + j];
      pd.P32[a][j] = (float)P[a * n + j];
    }
  // merge duplicate modes (fixed-size arrays)
  const int nc = pd.ncomp;
  int mode[MAXT][MAXN];
  double val[MAXT][12];
  int G = 0;
  for (int t = 0; t < c->ntaps; ++t) {
    int m[MAXN] = {0, 0, 0, 0, 0, 0};
    for (int j = 0; j < n; ++j) {
      m[j] = c->tap_k[t * n + j];
      if (2 * std::abs(m[j]) >= N[j]) raise(QP_ERR_INVALID_ARG, "tap mode component |m_j| must be < N_j/2");
      if (std::abs(m[j]) > 127) raise(QP_ERR_INVALID_ARG, "tap mode component |m_j| must be <= 127");
    }
    int id = -1;
    for (int s = 0; s < G && id < 0; ++s) {
      bool eq = true;
      for (int j = 0; j < n; ++j) eq = eq && mode[s][j] == m[j];
      if (eq) id = s;
    }
    if (id < 0) {
      id = G++;
      for (int j = 0; j < MAXN; ++j) mode[id][j] = m[j];
      for (int q = 0; q < 12; ++q) val[id][q] = 0.0;
    }
    for (int q = 0; q < 2 * nc; ++q) {
      const double x = c->tap_val[t * 2 * nc + q];
      if (!std::isfinite(x)) raise(QP_ERR_INVALID_ARG, "tap value is not finite");
      val[id][q] += x;
    }
  }
  double vmax = 0.0;
  for (int s = 0; s < G; ++s)
    for (int q = 0; q < 2 * nc; ++q) vmax = std::fmax(vmax, std::fabs(val[s][q]));
  int mean = -1;
  for (int s = 0; s < G; ++s) {
    int partner = -1, nz = 0;
    for (int j = 0; j < n; ++j) nz += mode[s][j] != 0;
    if (nz == 0) mean = s;
    for (int u = 0; u < G && partner < 0; ++u) {
      bool eq = true;
      for (int j = 0; j < n; ++j) eq = eq && mode[u][j] == -mode[s][j];
      if (eq) partner = u;
    }
    if (partner < 0) raise(QP_ERR_INVALID_ARG, "tap list is not Hermitian-paired: mode -m missing");
    for (int q = 0; q < nc; ++q) {
      if (std::fabs(val[s][2 * q] - val[partner][2 * q]) > 1e-12 * vmax ||
          std::fabs(val[s][2 * q + 1] + val[partner][2 * q + 1]) > 1e-12 * vmax)
        raise(QP_ERR_INVALID_ARG, "tap values must satisfy A~_{-m} = conj(A~_m) (real coefficient)");
      if (val[s][2 * q + 1] != 0.0) ht.real = false;
    }
  }
  if (mean < 0) raise(QP_ERR_NOT_ELLIPTIC, "the coefficient has no mean (m = 0) tap");
  if (!mean_tap_spd(c->kind, d, val[mean]))
    raise(QP_ERR_NOT_ELLIPTIC, "the coefficient's mean A~_0 is not positive definite");
  int order[MAXT];
  int no = 0;
  order[no++] = mean;
  for (int j = 0; j < n; ++j) {
    pd.star_begin[j] = no;
    for (int s = 0; s < G; ++s) {
      int nz = 0, ax = -1;
      for (int q = 0; q < n; ++q)
        if (mode[s][q] != 0) {
          ++nz;
          ax = q;
        }
      if (s != mean && nz == 1 && ax == j) order[no++] = s;
    }
  }
  pd.star_begin[n] = no;
  for (int s = 0; s < G; ++s) {
    int nz = 0;
    for (int q = 0; q < n; ++q) nz += mode[s][q] != 0;
    if (s != mean && nz > 1) order[no++] = s;
  }
  for (int j = n + 1; j <= MAXN; ++j) pd.star_begin[j] = pd.star_begin[n];
  for (int s = 0; s < G; ++s) {
    for (int j = 0; j < MAXN; ++j) pd.m[s][j] = (signed char)mode[order[s]][j];
    for (int q = 0; q < nc; ++q) {
      ht.c64[s * nc + q] = make_double2(val[order[s]][2 * q], val[order[s]][2 * q + 1]);
      ht.c32[s * nc + q] = make_float2((float)val[order[s]][2 * q], (float)val[order[s]][2 * q + 1]);
    }
  }
  pd.ntaps = G;
  pd.real_coef = ht.real ? 1 : 0;
  make_star(pd, ht.c64, ht.c32, ht.star);
}

}  // namespace

}  // namespace qp

using namespace qp;

extern "C" qp_status qp_pcg_solve_taps_static(int d, int n, const double* P, const int* N, const qp_coeff* coeff,
                                              int nrhs, const void* F, void* U, const qp_solve_opts* opts,
                                              qp_solve_info* info, void* stream) {
  try {
    if (!F || !U || !opts) raise(QP_ERR_INVALID_ARG, "F, U and opts must be non-null");
    if (((uintptr_t)F | (uintptr_t)U) & 15u) raise(QP_ERR_INVALID_ARG, "F and U must be 16-byte aligned");
    if (nrhs < 1 || nrhs > MAXR) raise(QP_ERR_INVALID_ARG, "nrhs must be 1..4");
    if (opts->mode != QP_MODE_FP64) raise(QP_ERR_INVALID_ARG, "qp_pcg_solve_taps_static runs the FP64 mode only");
    if (!(opts->tol >= 0.0) || opts->maxit < 1) raise(QP_ERR_INVALID_ARG, "tol must be >= 0 and maxit >= 1");
    if (opts->precond != QP_PRECOND_JACOBI && opts->precond != QP_PRECOND_FROBENIUS)
      raise(QP_ERR_INVALID_ARG, "unknown preconditioner");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    static thread_local HostTaps ht;   // about 60 KB: kept off the stack
    build_host(d, n, P, N, coeff, ht);
    const int D = ht.pd.D;
    const int nc = ht.pd.ncomp, G = ht.pd.ntaps;
    const int64_t chunk = chunk_modes(D);
    const int nchunks = (int)((D + chunk - 1) / chunk);
    const int run = (N[n - 1] % 2 == 0) ? 2 : 1;   // stencil run along the last axis
    const int nblk_diag = (int)std::min<int64_t>((D + BLOCK - 1) / BLOCK, 152 * 8);

    // carve the static scratch (size checks before any device work)
    Carve cv{static_scratch_address()};
    PlanDev* d_pd = cv.take<PlanDev>(1);
    StarParams* d_star = cv.take<StarParams>(1);
    double2* d_c64 = cv.take<double2>((size_t)G * nc);
    float2* d_c32 = cv.take<float2>((size_t)G * nc);
    double* jac64 = cv.take<double>(D);
    double* frob64 = cv.take<double>(D);
    float* jac32 = cv.take<float>(D);
    float* frob32 = cv.take<float>(D);
    double2* r = cv.take<double2>((size_t)nrhs * D);
    double2* h = cv.take<double2>((size_t)nrhs * D);
    double2* w = cv.take<double2>((size_t)nrhs * D);
    double* partials = cv.take<double>((size_t)NSLOT * nchunks + 2 * (size_t)nblk_diag);
    RhsSt* st = cv.take<RhsSt>(MAXR);
    unsigned* counters = cv.take<unsigned>(64);   // [0] ucount, [1] kcount, [2] diag counter
    int* ndone = cv.take<int>(16);
    double* small = cv.take<double>(16);

    // the scratch keeps the previous call's contents: reset what must start at zero
    CK(cudaMemsetAsync(counters, 0, 64 * sizeof(unsigned), s));
    CK(cudaMemsetAsync(ndone, 0, 16 * sizeof(int), s));
    CK(cudaMemsetAsync(st, 0, MAXR * sizeof(RhsSt), s));
    ht.pd.coef64 = d_c64;
    ht.pd.coef32 = d_c32;
    ht.pd.star = ht.pd.star1 ? d_star : nullptr;
    CK(cudaMemcpyAsync(d_pd, &ht.pd, sizeof(PlanDev), cudaMemcpyHostToDevice, s));
    if (ht.pd.star1) CK(cudaMemcpyAsync(d_star, &ht.star, sizeof(StarParams), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_c64, ht.c64, (size_t)G * nc * sizeof(double2), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_c32, ht.c32, (size_t)G * nc * sizeof(float2), cudaMemcpyHostToDevice, s));
    launch_diag(d_pd, G * nc, D, jac64, frob64, jac32, frob32, partials, counters + 2, small, nblk_diag,
                opts->precond == QP_PRECOND_FROBENIUS, s);
    CK_LAUNCH();
    double chk[2] = {0.0, 0.0};
    CK(cudaMemcpyAsync(chk, small, sizeof(chk), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double pmax = 0.0;
    for (int a = 0; a < d; ++a)
      for (int j = 0; j < n; ++j) pmax = std::fmax(pmax, std::fabs(P[a * n + j]));
    if (!(std::sqrt(std::fmax(chk[0], 0.0)) > 1e-12 * pmax))
      raise(QP_ERR_SINGULAR_P, "min over k != 0 of |P k| is ~0: P is not a projection on this grid");
    if (!(chk[1] > 0.0)) raise(QP_ERR_NOT_ELLIPTIC, "the Jacobi diagonal q(k) is not positive");

    // one unit (this plan and its right-hand sides), described in the kernel parameters
    BatchDev bd;
    std::memset(&bd, 0, sizeof(bd));
    UnitDev& un = bd.pu;
    un.plan = d_pd;
    un.D = D;
    un.nrhs = nrhs;
    un.chunk = (int)chunk;
    un.run = run;
    un.chunk0 = 0;
    un.nchunk = nchunks;
    un.F = static_cast<const double2*>(F);
    un.U = static_cast<double2*>(U);
    un.r = r;
    un.h = h;
    un.w = w;
    un.minv64 = opts->precond == QP_PRECOND_FROBENIUS ? frob64 : jac64;
    un.minv32 = opts->precond == QP_PRECOND_FROBENIUS ? frob32 : jac32;
    bd.nunits = 1;
    bd.nchunks = nchunks;
    bd.nslots = nrhs;
    bd.single = 1;
    bd.units = nullptr;
    bd.st = st;
    bd.chunk_unit = nullptr;
    bd.partials = partials;
    bd.ucount = counters;
    bd.kcount = counters + 1;
    bd.ndone = ndone;
    bd.tol2 = opts->tol * opts->tol;
    bd.otol2 = bd.tol2;
    bd.maxit = opts->maxit;
    bd.max_outer = 1;

    // warm start from U: w = Q U, r = F - w, then Algorithm 2 with the host polling the done count, then the
    // FP64 true residual. Like qp_pcg_solve, a right-hand side whose recursive residual met the tolerance while
    // its true residual did not (the two drift apart at tight tolerances) is solved again from its current U, at
    // most twice; iterations add up over the attempts.
    const bool realc = ht.real;
    // FP64 applies of a single star-1 unit take the kernel-parameter form only with stored weights, which this
    // entry point has no room for: its kernels read the plan's star data from shared memory
    const StarParams* st1 = nullptr;
    RhsSt hst[MAXR];
    int iters_before[MAXR] = {0, 0, 0, 0};
    for (int attempt = 0; attempt < 3; ++attempt) {
      launch_level_reset(bd, 0, s);
      launch_apply(bd, realc, G * nc, nrhs, LEVEL_FP64, EPI_NONE, false, 0, nchunks, st1, ht.pd.kind, s);
      launch_pcg_init(bd, nrhs, LEVEL_FP64, true, 0, nchunks, s);
      CK_LAUNCH();
      int done = 0, launched = 0, burst = 4;
      for (;;) {
        CK(cudaMemcpyAsync(&done, ndone, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (done >= nrhs) break;
        if (launched > opts->maxit + 64) raise(QP_ERR_CUDA, "PCG loop exceeded its cap without the device count");
        for (int i = 0; i < burst; ++i) {
          launch_apply(bd, realc, G * nc, nrhs, LEVEL_FP64, EPI_DOT_HW, false, 0, nchunks, st1, ht.pd.kind, s);
          launch_pcg_update(bd, nrhs, LEVEL_FP64, 0, nchunks, s);
          launch_pcg_hupdate(bd, nrhs, LEVEL_FP64, nchunks, s);
        }
        CK_LAUNCH();
        launched += burst;
        burst = std::min(burst * 2, 32);
      }
      launch_apply(bd, realc, G * nc, nrhs, LEVEL_FP64, EPI_RESIDUAL, false, 0, nchunks, st1, ht.pd.kind, s);
      CK_LAUNCH();
      CK(cudaMemcpyAsync(hst, st, MAXR * sizeof(RhsSt), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      bool again = false;
      for (int k = 0; k < nrhs; ++k) {
        hst[k].iters += iters_before[k];
        iters_before[k] = hst[k].iters;
        const double rel = hst[k].of2 > 0.0 ? std::sqrt(hst[k].orr / hst[k].of2) : 0.0;
        if (hst[k].status == QP_OK && rel > opts->tol) again = true;
      }
      if (!again) break;
    }
    // U(k = 0) = 0
    for (int k = 0; k < nrhs; ++k)
      CK(cudaMemsetAsync(static_cast<double2*>(U) + (size_t)k * D, 0, sizeof(double2), s));
    qp_status worst = QP_OK;
    for (int k = 0; k < nrhs; ++k) {
      const double rel = hst[k].of2 > 0.0 ? std::sqrt(hst[k].orr / hst[k].of2) : 0.0;
      int status = hst[k].status;
      if (status == QP_OK && rel > opts->tol) status = QP_ERR_NO_CONVERGENCE;
      if (hst[k].of2 == 0.0)   // F = 0: U = 0
        CK(cudaMemsetAsync(static_cast<double2*>(U) + (size_t)k * D, 0, (size_t)D * sizeof(double2), s));
      if (info) {
        info[k].status = status;
        info[k].iterations = hst[k].iters;
        info[k].outer_iterations = 0;
        info[k].rel_residual = rel;
      }
      if (status != QP_OK && (worst == QP_OK || status == QP_ERR_BREAKDOWN)) worst = (qp_status)status;
    }
    CK(cudaStreamSynchronize(s));
    if (worst != QP_OK) raise(worst, "at least one right-hand side did not reach the tolerance");
  } catch (const QpError& e) {
    set_last_error(e.msg);
    return e.s;
  }
  set_last_error("");
  return QP_OK;
}
