// C ABI of libqp: plan construction (Sec. 2.3 grids; Sec. 4.2 compressed tap storage; Sec. 4.3 diagonal
// preconditioners), the stiffness apply, PCG (Algorithm 2) in FP64 or as an FP32 inner solve inside FP64
// iterative refinement, the corrector right-hand sides and the homogenized coefficient (Sec. 5.2), for one
// plan or a batch of plans. Host code only orchestrates: every arithmetic step runs in this library's kernels.
//
// A solve is recorded once per (units, mode, preconditioner, tolerances) as a CUDA graph whose PCG loop (and,
// in refinement mode, the outer loop around it) is a conditional WHILE node driven by the kernels' own
// convergence flags, so a whole solve is one graph launch and one host read of the final state.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "qp_fft.cuh"
#include "qp_internal.cuh"

using namespace qp;

namespace qp {
static std::atomic<uint64_t> g_launches{0};
static thread_local int t_capturing = 0;
void count_launch(int n) {
  if (!t_capturing) g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed);
}
}  // namespace qp

namespace {

thread_local std::string g_err;

}  // namespace

void qp::set_last_error(const std::string& msg) { g_err = msg; }

namespace {

template <typename T> struct Vecs {
  cplx<T>* r = nullptr;
  cplx<T>* h = nullptr;
  cplx<T>* w = nullptr;
  cplx<T>* F = nullptr;   // FP64: right-hand sides; FP32: scaled refinement right-hand side
  cplx<T>* X = nullptr;   // FP64: solutions; FP32: inner correction
};

}  // namespace

struct Solver;

struct qp_plan {
  int d = 0, n = 0, kind = 0, ncomp = 0, backend = 0, max_rhs = 0, nblk = 0, precisions = 3, D = 0, exec = 0;
  int64_t Dfull = 0;             // product of the N_j (D is the stored length: D_h for a half-spectrum plan)
  int spectrum = QP_SPECTRUM_FULL;
  int N[MAXN] = {};
  double P[MAXD][MAXN] = {};
  double min_abs_lambda = 0.0;
  int64_t bytes = 0;
  std::vector<void*> dev_allocs;
  std::vector<std::pair<void*, size_t>> host_allocs;
  cudaStream_t create_stream = nullptr;   // plan buffers are allocated in this stream's order

  PlanDev host_pd{};           // host copy of the device plan description
  StarParams star_host{};      // star-1 stencil data (host_pd.star1), passed by value to single-plan kernels
  void* w64 = nullptr;         // star-1 plans: stored FP64 weights (star_host.w64), or null
  StarParams* star_dev = nullptr;   // device copy of star_host (host_pd.star), read by batches of several plans
  PlanDev* pd = nullptr;       // device copy
  bool real_coef = false;
  int coef_count = 0;          // ntaps * ncomp

  FftPlan* fft = nullptr;      // FFT backend

  double* jac64 = nullptr;
  double* frob64 = nullptr;
  bool frob_ready = false;          // the Frobenius diagonal is built (on first use)
  float* jac32 = nullptr;
  float* frob32 = nullptr;

  Vecs<double> v64;
  Vecs<float> v32;
  double* scratch = nullptr;        // set-up reductions (partials)
  unsigned* counter = nullptr;
  double* small = nullptr;          // device scratch for host-read results (a*, set-up checks)
  double* h_small = nullptr;        // pinned host mirror
  Solver* solver = nullptr;         // graph cache for single-plan solves

  void* dalloc(size_t bytes_) {
    void* p = dev_alloc(bytes_, create_stream);
    dev_allocs.push_back(p);
    bytes += (int64_t)bytes_;
    return p;
  }
  void* halloc(size_t bytes_) {
    void* p = pinned_alloc(bytes_);
    host_allocs.push_back({p, bytes_});
    return p;
  }
  ~qp_plan();
};

// ------------------------------------------------------------------------------------------------ solver

namespace {

struct Key {
  int mode, precond, nrhs, warm, maxit, max_outer;
  double tol, inner_tol;
  bool operator<(const Key& o) const {
    return std::tie(mode, precond, nrhs, warm, maxit, max_outer, tol, inner_tol) <
           std::tie(o.mode, o.precond, o.nrhs, o.warm, o.maxit, o.max_outer, o.tol, o.inner_tol);
  }
};

struct Entry {
  BatchDev bd{};
  int nblk = 0;
  std::vector<void*> allocs;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int fixed_nodes = 0, body_nodes = 0, outer_nodes = 0;
  int pgrid = 0;          // > 0: the solve is one persistent launch of this many blocks
  size_t psmem = 0;
  int psk = 0;            // persistent kernel's stencil source (0 shared plan, 1/2 star-1 scalar/diagonal)
  ~Entry() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (void* p : allocs) dev_free(p);
  }
};

}  // namespace

// A set of units (plans with their right-hand sides) and the recorded solve graphs for them.
struct Solver {
  std::vector<qp_plan*> plans;
  std::map<Key, std::unique_ptr<Entry>> cache;
  RhsSt* st = nullptr;                   // device [nunits * MAXR]
  RhsSt* h_st = nullptr;                 // pinned mirror
  unsigned* ucount = nullptr;
  unsigned* kcount = nullptr;
  int* ndone = nullptr;
  unsigned* pbar = nullptr;              // persistent solve: grid barrier words
  int* perr = nullptr;                   // persistent solve: barrier time-out flag
  int* h_perr = nullptr;                 // pinned mirror
  cudaStream_t cap = nullptr;
  bool graphs_ok = true;
  std::vector<void*> allocs;

  cudaStream_t s0 = nullptr;   // allocations are ordered on the stream of the call that created the solver

  Solver(const std::vector<qp_plan*>& ps, cudaStream_t s) : plans(ps), s0(s) {
    const size_t nu = plans.size();
    st = (RhsSt*)alloc(nu * MAXR * sizeof(RhsSt));
    ucount = (unsigned*)alloc(nu * sizeof(unsigned));
    kcount = (unsigned*)alloc(64);
    ndone = (int*)alloc(64);
    pbar = (unsigned*)alloc(64);
    perr = (int*)alloc(64);
    CK(cudaMemsetAsync(st, 0, nu * MAXR * sizeof(RhsSt), s));
    CK(cudaMemsetAsync(ucount, 0, nu * sizeof(unsigned), s));
    CK(cudaMemsetAsync(kcount, 0, 64, s));
    CK(cudaMemsetAsync(ndone, 0, 64, s));
    h_st = (RhsSt*)pinned_alloc(nu * MAXR * sizeof(RhsSt));
    h_perr = (int*)pinned_alloc(sizeof(int));
  }
  ~Solver() {
    cache.clear();
    if (cap) cudaStreamDestroy(cap);
    pinned_free(h_st, plans.size() * MAXR * sizeof(RhsSt));
    pinned_free(h_perr, sizeof(int));
    for (void* p : allocs) dev_free(p);
  }
  void* alloc(size_t b) {
    void* p = dev_alloc(b, s0);
    allocs.push_back(p);
    return p;
  }
  // the capture stream of graph recording, created on first use (persistent solves never record a graph)
  cudaStream_t capture_stream() {
    if (!cap) CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    return cap;
  }
};

qp_plan::~qp_plan() {
  cudaDeviceSynchronize();   // no work of any stream may still use the plan's buffers
  delete solver;
  if (fft) fft_plan_destroy(fft);
  for (void* p : dev_allocs) dev_free(p);
  for (auto& h : host_allocs) pinned_free(h.first, h.second);
  dev_trim();
}

struct qp_batch {
  std::vector<qp_plan*> plans;
  Solver* solver = nullptr;
  double* small = nullptr;     // device a* outputs (2 d^2 per plan)
  double* h_small = nullptr;
  size_t small_bytes = 0;
  PlanJob* jobs = nullptr;     // device table of the taps plans' right-hand-side / a* jobs
  int njobs = 0, jobs_mc = 1;  // their count and largest coefficient table (ntaps * ncomp)
  ~qp_batch() {
    cudaDeviceSynchronize();
    delete solver;
    dev_free(small);
    dev_free(jobs);
    pinned_free(h_small, small_bytes);
    dev_trim();
  }
};

namespace {

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int ncomp_of(int kind, int d) {
  if (kind == QP_COEF_SCALAR) return 1;
  if (kind == QP_COEF_DIAG) return d;
  return d * (d + 1) / 2;
}

bool is_23(int N) {
  while (N % 2 == 0) N /= 2;
  while (N % 3 == 0) N /= 3;
  return N == 1;
}

// ------------------------------------------------------------------------------------------------ plan set-up

// half: half-spectrum storage (QP_SPECTRUM_HALF): the last axis keeps k_{n-1} = 0 .. ceil(N/2) - 1 and vectors hold
// D_h = N_1 .. N_{n-1} ceil(N_n / 2) entries (p->D); p->Dfull keeps the product of all N_j.
void build_geometry(qp_plan* p, int d, int n, const double* P, const int* N, bool half) {
  if (d < 1 || d > MAXD) raise(QP_ERR_INVALID_ARG, "d must be 1..3");
  if (n < d || n > MAXN) raise(QP_ERR_INVALID_ARG, "n must satisfy d <= n <= 6");
  if (!P || !N) raise(QP_ERR_INVALID_ARG, "P and N must be non-null host arrays");
  p->d = d;
  p->n = n;
  int64_t Dfull = 1;
  for (int j = 0; j < n; ++j) {
    if (N[j] < 2 || N[j] > 1024) raise(QP_ERR_INVALID_ARG, "every N_j must be in 2..1024");
    Dfull *= N[j];
  }
  if (Dfull > (int64_t(1) << 30)) raise(QP_ERR_INVALID_ARG, "D = prod N_j must be <= 2^30");
  PlanDev& pd = p->host_pd;
  std::memset(&pd, 0, sizeof(pd));
  pd.n = n;
  pd.d = d;
  pd.hspec = half ? 1 : 0;
  pd.Hl = (N[n - 1] + 1) / 2;
  int st = 1;
  for (int j = n - 1; j >= 0; --j) {
    pd.N[j] = N[j];
    p->N[j] = N[j];
    pd.Nst[j] = (half && j == n - 1) ? pd.Hl : N[j];
    pd.nyq[j] = (half && j < n - 1 && N[j] % 2 == 0) ? N[j] / 2 : -1;
    pd.stride[j] = st;
    pd.div[j] = make_fastdiv((uint32_t)pd.Nst[j]);
    st *= pd.Nst[j];
  }
  const int64_t D = st;
  p->D = (int)D;
  p->Dfull = Dfull;
  pd.D = (int)D;
  for (int j = n; j < MAXN; ++j) {
    pd.N[j] = 1;
    pd.Nst[j] = 1;
    pd.nyq[j] = -1;
    pd.stride[j] = (int)D;
    pd.div[j] = make_fastdiv(1);
  }
  double pmax = 0.0;
  for (int a = 0; a < d; ++a)
    for (int j = 0; j < n; ++j) {
      if (!std::isfinite(P[a * n + j])) raise(QP_ERR_INVALID_ARG, "P has a non-finite entry");
      p->P[a][j] = P[a * n + j];
      pd.P[a][j] = P[a * n + j];
      pd.P32[a][j] = (float)P[a * n + j];
      pmax = std::max(pmax, std::fabs(P[a * n + j]));
    }
  if (pmax == 0.0) raise(QP_ERR_SINGULAR_P, "P is zero");
  p->nblk = (int)std::min<int64_t>((D + BLOCK - 1) / BLOCK, 152 * 8);
}

// Merges duplicate modes, checks the Hermitian pairing A~_{-m} = conj(A~_m), |m_j| < N_j / 2 and the mean,
// and sorts the taps as [mean][star taps per axis][multi-axis taps] (Alg. 1's stored A~ and index pairs).
void build_taps(qp_plan* p, const qp_coeff* c) {
  const int n = p->n, d = p->d, nc = p->ncomp;
  if (c->ntaps < 1 || c->ntaps > MAXT) raise(QP_ERR_INVALID_ARG, "ntaps must be 1..256");
  if (!c->tap_k || !c->tap_val) raise(QP_ERR_INVALID_ARG, "tap_k and tap_val must be non-null host arrays");
  std::map<std::vector<int>, int> index;
  std::vector<std::vector<int>> modes;
  std::vector<std::vector<double>> vals;   // 2*nc per tap
  for (int t = 0; t < c->ntaps; ++t) {
    std::vector<int> m(n);
    for (int j = 0; j < n; ++j) {
      m[j] = c->tap_k[t * n + j];
      if (2 * std::abs(m[j]) >= p->N[j]) raise(QP_ERR_INVALID_ARG, "tap mode component |m_j| must be < N_j/2");
      if (std::abs(m[j]) > 127) raise(QP_ERR_INVALID_ARG, "tap mode component |m_j| must be <= 127");
    }
    for (int q = 0; q < 2 * nc; ++q)
      if (!std::isfinite(c->tap_val[t * 2 * nc + q])) raise(QP_ERR_INVALID_ARG, "tap value is not finite");
    auto it = index.find(m);
    int id;
    if (it == index.end()) {
      id = (int)modes.size();
      index[m] = id;
      modes.push_back(m);
      vals.push_back(std::vector<double>(2 * nc, 0.0));
    } else {
      id = it->second;
    }
    for (int q = 0; q < 2 * nc; ++q) vals[id][q] += c->tap_val[t * 2 * nc + q];
  }
  double vmax = 0.0;
  for (auto& v : vals)
    for (double x : v) vmax = std::max(vmax, std::fabs(x));
  const int G = (int)modes.size();
  bool real_coef = true;
  int mean = -1;
  for (int t = 0; t < G; ++t) {
    std::vector<int> neg(n);
    bool zero = true;
    for (int j = 0; j < n; ++j) {
      neg[j] = -modes[t][j];
      zero = zero && modes[t][j] == 0;
    }
    if (zero) mean = t;
    auto it = index.find(neg);
    if (it == index.end()) raise(QP_ERR_INVALID_ARG, "tap list is not Hermitian-paired: mode -m missing");
    for (int q = 0; q < nc; ++q) {
      const double re = vals[t][2 * q], im = vals[t][2 * q + 1];
      const double pre = vals[it->second][2 * q], pim = vals[it->second][2 * q + 1];
      if (std::fabs(re - pre) > 1e-12 * vmax || std::fabs(im + pim) > 1e-12 * vmax)
        raise(QP_ERR_INVALID_ARG, "tap values must satisfy A~_{-m} = conj(A~_m) (real coefficient)");
      if (im != 0.0) real_coef = false;
    }
  }
  if (mean < 0) raise(QP_ERR_NOT_ELLIPTIC, "the coefficient has no mean (m = 0) tap");
  if (!mean_tap_spd(p->kind, d, vals[mean].data()))
    raise(QP_ERR_NOT_ELLIPTIC, "the coefficient's mean A~_0 is not positive definite");
  // sorted order: mean, star taps by axis, multi-axis taps
  std::vector<int> order;
  order.push_back(mean);
  PlanDev& pd = p->host_pd;
  for (int j = 0; j < n; ++j) {
    pd.star_begin[j] = (int)order.size();
    for (int t = 0; t < G; ++t) {
      if (t == mean) continue;
      int nz = 0, ax = -1;
      for (int q = 0; q < n; ++q)
        if (modes[t][q] != 0) {
          ++nz;
          ax = q;
        }
      if (nz == 1 && ax == j) order.push_back(t);
    }
  }
  pd.star_begin[n] = (int)order.size();
  for (int t = 0; t < G; ++t) {
    if (t == mean) continue;
    int nz = 0;
    for (int q = 0; q < n; ++q) nz += modes[t][q] != 0;
    if (nz > 1) order.push_back(t);
  }
  for (int j = n + 1; j <= MAXN; ++j) pd.star_begin[j] = pd.star_begin[n];
  std::vector<double2> coef64((size_t)G * nc);
  std::vector<float2> coef32((size_t)G * nc);
  for (int s = 0; s < G; ++s) {
    const int t = order[s];
    for (int j = 0; j < MAXN; ++j) pd.m[s][j] = (signed char)(j < n ? modes[t][j] : 0);
    for (int q = 0; q < nc; ++q) {
      coef64[(size_t)s * nc + q] = make_double2(vals[t][2 * q], vals[t][2 * q + 1]);
      coef32[(size_t)s * nc + q] = make_float2((float)vals[t][2 * q], (float)vals[t][2 * q + 1]);
    }
  }
  auto up = [&](const void* src, size_t bytes_) {
    void* dst = p->dalloc(bytes_);
    CK(cudaMemcpyAsync(dst, src, bytes_, cudaMemcpyHostToDevice, p->create_stream));   // pageable: staged
    return dst;
  };
  pd.coef64 = (const double2*)up(coef64.data(), coef64.size() * sizeof(double2));
  pd.coef32 = (const float2*)up(coef32.data(), coef32.size() * sizeof(float2));
  pd.ntaps = G;
  pd.real_coef = real_coef ? 1 : 0;
  p->real_coef = real_coef;
  p->coef_count = G * nc;
  make_star(pd, coef64.data(), coef32.data(), p->star_host);
  if (pd.star1) {
    p->star_dev = (StarParams*)up(&p->star_host, sizeof(StarParams));
    pd.star = p->star_dev;
  }
}

// FP64 weights of a star-1 plan stored per (tap slot, mode). The compressed format of Sec. 4.2 keeps the nonzero
// entries Q_ij of the stiffness matrix; on this GPU, where FP64 arithmetic runs at 1/64 of the FP32 rate, reading
// them once per apply is cheaper than forming them, so every FP64 apply of the plan reads them (single-plan
// kernels through the kernel-parameter StarParams, batches of several plans through its device copy). They are
// formed by the stencil's own arithmetic, so stored and formed weights agree bit for bit. Built when the plan has
// FP64 vectors and the table takes at most a quarter of the free device memory.
void build_star_weights(qp_plan* p, cudaStream_t s) {
  const PlanDev& pd = p->host_pd;
  if (!pd.star1 || !(p->precisions & 1) || pd.Nst[pd.n - 1] % 2 != 0) return;
  const size_t bytes = (size_t)(1 + 2 * pd.n) * (size_t)p->D * (p->real_coef ? sizeof(double) : sizeof(double2));
  size_t fr = 0, tot = 0;
  CK(cudaMemGetInfo(&fr, &tot));
  if (bytes > fr / 4) return;
  p->w64 = p->dalloc(bytes);
  p->star_host.w64 = p->w64;
  p->star_host.wreal = p->real_coef ? 1 : 0;
  launch_star_weights(p->star_host, p->real_coef, p->kind, p->D, p->w64, s);
  CK_LAUNCH();
  // the device copy of the StarParams (read by batches of several plans) points at the table too
  CK(cudaMemcpyAsync(p->star_dev, &p->star_host, sizeof(StarParams), cudaMemcpyHostToDevice, s));
}

// The same for a plan with general taps (not star-1): its FP64 entries Q_ij per (sorted tap, mode), [ntaps][D], formed
// by the general stencil's own arithmetic, read by every FP64 apply of the plan (single or batched). Built when the
// plan has FP64 vectors, stores the full spectrum and the table takes at most a quarter of the free device memory.
int last_axis_run(const qp_plan* p);

void build_gen_weights(qp_plan* p, cudaStream_t s) {
  PlanDev& pd = p->host_pd;
  if (pd.star1 || p->backend != QP_BACKEND_TAPS || !(p->precisions & 1) || pd.hspec) return;
  const size_t bytes = (size_t)pd.ntaps * (size_t)p->D * (p->real_coef ? sizeof(double) : sizeof(double2));
  size_t fr = 0, tot = 0;
  CK(cudaMemGetInfo(&fr, &tot));
  if (bytes > fr / 4) return;
  void* w = p->dalloc(bytes);
  launch_gen_weights(p->pd, p->real_coef, p->coef_count, p->D, last_axis_run(p), w, s);
  CK_LAUNCH();
  pd.wgen = w;
  pd.wgen_real = p->real_coef ? 1 : 0;
  CK(cudaMemcpyAsync(p->pd, &pd, sizeof(PlanDev), cudaMemcpyHostToDevice, s));
}

// QP_BACKEND_AUTO with a tap coefficient: the stencil and the FFT backend are both exact for it (the taps are a
// trigonometric polynomial), so the FP32 applies of both (max_rhs right-hand sides, the FFT one on its autotuned
// schedule) are timed once per (geometry, kind, taps, max_rhs) on this GPU and the faster is kept; the choice is
// cached for the process. The stencil costs about one multiply-add per tap and mode, the FFT passes about
// log D of them, so dense tap lists go to the FFT. Returns the backend; for QP_BACKEND_FFT, p->fft holds the FFT
// plan with the coefficient already transformed. The plan's tap tables and device description must be uploaded.
std::mutex g_backend_mu;
std::map<std::string, int> g_backend_cache;

int tune_backend(qp_plan* p, cudaStream_t s) {
  const PlanDev& pd = p->host_pd;
  std::string key = std::to_string(pd.d) + "/" + std::to_string(pd.kind) + "/" + std::to_string(pd.ntaps) + "/" +
                    std::to_string(p->max_rhs) + "/" + std::to_string(p->real_coef);
  for (int j = 0; j < pd.n; ++j) key += "/" + std::to_string(pd.N[j]);
  int cached = -1;
  {
    std::lock_guard<std::mutex> lk(g_backend_mu);
    auto it = g_backend_cache.find(key);
    if (it != g_backend_cache.end()) cached = it->second;
  }
  if (cached == QP_BACKEND_TAPS) return QP_BACKEND_TAPS;
  FftPlan* f = fft_plan_create(pd, p->precisions, p->max_rhs, s);
  try {
    fft_set_taps(f, pd, p->pd, s);
    if (cached == QP_BACKEND_FFT) {
      p->fft = f;
      return QP_BACKEND_FFT;
    }
    fft_autotune(f, pd, p->pd, s);
    const int nr = p->max_rhs;
    const size_t bytes = (size_t)nr * p->D * sizeof(float2);
    float2* h = p->v32.h;
    float2* w = p->v32.w;
    CK(cudaMemsetAsync(h, 0, bytes, s));
    const StarParams* st1 = pd.star1 ? &p->star_host : nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float ms[2] = {0.f, 0.f};
    for (int b = 0; b < 2; ++b) {
      auto run = [&]() {
        if (b == 0) launch_apply_plain<float>(p->pd, p->real_coef, p->coef_count, p->D, nr, h, w,
                                              pd.N[pd.n - 1] % 2 == 0 ? 2 : 1, st1, p->kind, s);
        else fft_apply<float>(f, pd, p->pd, h, w, nr, s);
      };
      run();
      CK(cudaEventRecord(e0, s));
      for (int rep = 0; rep < 3; ++rep) run();
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      CK_LAUNCH();
      CK(cudaEventElapsedTime(&ms[b], e0, e1));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const int choice = (ms[1] < 0.9f * ms[0]) ? QP_BACKEND_FFT : QP_BACKEND_TAPS;
    {
      std::lock_guard<std::mutex> lk(g_backend_mu);
      g_backend_cache[key] = choice;
    }
    if (choice == QP_BACKEND_FFT) {
      p->fft = f;
      return QP_BACKEND_FFT;
    }
  } catch (...) {
    cudaStreamSynchronize(s);
    fft_plan_destroy(f);
    throw;
  }
  CK(cudaStreamSynchronize(s));
  fft_plan_destroy(f);
  return QP_BACKEND_TAPS;
}

void alloc_workspace(qp_plan* p) {
  const size_t D = (size_t)p->D, R = (size_t)p->max_rhs;
  p->jac64 = (double*)p->dalloc(D * sizeof(double));
  p->frob64 = (double*)p->dalloc(D * sizeof(double));
  p->jac32 = (float*)p->dalloc(D * sizeof(float));
  p->frob32 = (float*)p->dalloc(D * sizeof(float));
  p->v64.r = (double2*)p->dalloc(R * D * sizeof(double2));
  p->v64.w = (double2*)p->dalloc(R * D * sizeof(double2));
  p->v64.F = (double2*)p->dalloc(R * D * sizeof(double2));
  p->v64.X = (double2*)p->dalloc(R * D * sizeof(double2));
  if (p->precisions & 1) p->v64.h = (double2*)p->dalloc(R * D * sizeof(double2));
  if (p->precisions & 2) {
    p->v32.r = (float2*)p->dalloc(R * D * sizeof(float2));
    p->v32.h = (float2*)p->dalloc(R * D * sizeof(float2));
    p->v32.w = (float2*)p->dalloc(R * D * sizeof(float2));
    p->v32.F = (float2*)p->dalloc(R * D * sizeof(float2));
    p->v32.X = (float2*)p->dalloc(R * D * sizeof(float2));
  }
  p->scratch = (double*)p->dalloc((size_t)4 * p->nblk * sizeof(double) + 64);
  p->counter = (unsigned*)p->dalloc(64);
  p->small = (double*)p->dalloc(256 * sizeof(double));
  CK(cudaMemsetAsync(p->counter, 0, 64, p->create_stream));
  CK(cudaMemsetAsync(p->small, 0, 256 * sizeof(double), p->create_stream));
  p->h_small = (double*)p->halloc(256 * sizeof(double));
}

// ------------------------------------------------------------------------------------------------ recording

// Modes per thread step of the stencil kernels for this plan: runs of 2 along the last axis when its length is
// even (the run then never crosses a row), else 1. (Longer runs cut index work further but need more registers
// per thread; on GB300 the occupancy they cost outweighed it.)
int last_axis_run(const qp_plan* p) { return (p->host_pd.Nst[p->host_pd.n - 1] % 2 == 0) ? 2 : 1; }

// Everything a solve needs about its units on the host side.
struct Units {
  std::vector<qp_plan*> plans;
  std::vector<int> nrhs;
  bool all_real = true;
  int max_coef = 1;
  int max_rhs = 1;
  bool direct = false;    // launch kernels directly (host-driven loops) instead of recording a graph
  int exec = QP_EXEC_GRAPH;  // QP_EXEC_AUTO / PERSISTENT: a single taps unit may run as one persistent launch
  int run = 2;               // shortest stencil run of the units (the persistent form needs 2)
};

// One stiffness apply over all units at a level: the FFT passes of FFT-backend units (they write w), then the
// batch stencil/epilogue kernel.
void record_apply(const Units& us, const Entry& en, int level, int epi, int refine, unsigned long long cond,
                  cudaStream_t s) {
  for (size_t u = 0; u < us.plans.size(); ++u) {
    if (refine == REFINE_ZERO_U) break;   // Q U = 0: no FFT passes either
    qp_plan* p = us.plans[u];
    if (p->backend != QP_BACKEND_FFT) continue;
    const int nr = us.nrhs[u];
    if (level == LEVEL_FP32) fft_apply<float>(p->fft, p->host_pd, p->pd, p->v32.h, p->v32.w, nr, s);
    else if (epi == EPI_DOT_HW) fft_apply<double>(p->fft, p->host_pd, p->pd, p->v64.h, p->v64.w, nr, s);
    else fft_apply<double>(p->fft, p->host_pd, p->pd, p->v64.X, p->v64.w, nr, s);
  }
  // a single star-1 unit with an even last axis takes its stencil data as a kernel parameter (FP64: only with
  // its stored weights)
  const qp_plan* p0 = us.plans.size() == 1 ? us.plans[0] : nullptr;
  const bool st = p0 && p0->backend == QP_BACKEND_TAPS && p0->host_pd.star1 && last_axis_run(p0) == 2 &&
                  (level == LEVEL_FP32 || p0->w64);
  launch_apply(en.bd, us.all_real, us.max_coef, us.max_rhs, level, epi, refine, cond, en.nblk,
               st ? &p0->star_host : nullptr, p0 ? p0->kind : 0, s);
  CK_LAUNCH();
}

// Phase timing (qp_set_phase_timing): while it is on, solves run in the host-driven form, one PCG iteration per
// host check (no launch after convergence), with CUDA events on the solve's stream around each kernel group; the
// durations are added up per phase once the solve's stream has been synchronised.
std::atomic<int> g_phase_timing{0};
std::mutex g_phase_mu;
double g_phase_ms[QP_NPHASE] = {};
int64_t g_phase_count[QP_NPHASE] = {};
struct PendingPhase {
  int phase;
  cudaEvent_t a, b;
};
thread_local std::vector<PendingPhase> t_pending;

template <typename Fn>
void timed(int phase, cudaStream_t s, Fn fn) {
  if (!g_phase_timing.load(std::memory_order_relaxed)) {
    fn();
    return;
  }
  PendingPhase pp{phase, nullptr, nullptr};
  CK(cudaEventCreate(&pp.a));
  CK(cudaEventCreate(&pp.b));
  CK(cudaEventRecord(pp.a, s));
  fn();
  CK(cudaEventRecord(pp.b, s));
  t_pending.push_back(pp);
}

// Adds the recorded phases of this thread's last solve (its stream synchronised) to the totals.
void resolve_phases() {
  if (t_pending.empty()) return;
  std::lock_guard<std::mutex> lk(g_phase_mu);
  for (auto& pp : t_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pp.a, pp.b) == cudaSuccess) {
      g_phase_ms[pp.phase] += ms;
      g_phase_count[pp.phase] += 1;
    }
    cudaEventDestroy(pp.a);
    cudaEventDestroy(pp.b);
  }
  t_pending.clear();
}

void body_pcg(const Units& us, const Entry& en, int level, unsigned long long cond, cudaStream_t s) {
  const bool l32 = level == LEVEL_FP32;
  timed(l32 ? QP_PHASE_APPLY32 : QP_PHASE_APPLY64, s,
        [&] { record_apply(us, en, level, EPI_DOT_HW, REFINE_NONE, cond, s); });
  timed(l32 ? QP_PHASE_UPDATE32 : QP_PHASE_UPDATE64, s,
        [&] { launch_pcg_update(en.bd, us.max_rhs, level, cond, en.nblk, s); });
  timed(l32 ? QP_PHASE_HUPDATE32 : QP_PHASE_HUPDATE64, s,
        [&] { launch_pcg_hupdate(en.bd, us.max_rhs, level, en.nblk, s); });
  CK_LAUNCH();
}

void zero_solutions(const Units& us, cudaStream_t s) {
  for (size_t u = 0; u < us.plans.size(); ++u)
    CK(cudaMemsetAsync(us.plans[u]->v64.X, 0, (size_t)us.nrhs[u] * us.plans[u]->D * sizeof(double2), s));
}

// U(k = 0) = 0 for every right-hand side (the excluded mean mode).
void zero_mean_mode(const Units& us, cudaStream_t s) {
  for (size_t u = 0; u < us.plans.size(); ++u)
    for (int r = 0; r < us.nrhs[u]; ++r)
      CK(cudaMemsetAsync(us.plans[u]->v64.X + (size_t)r * us.plans[u]->D, 0, sizeof(double2), s));
}

// Appends the capture of "fn" to graph g after the nodes "deps"; returns the leaf nodes of the capture.
template <typename Fn>
std::vector<cudaGraphNode_t> capture_into(cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, cudaStream_t cap,
                                          Fn fn) {
  CK(cudaStreamBeginCaptureToGraph(cap, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                   cudaStreamCaptureModeRelaxed));
  t_capturing = 1;
  try {
    fn(cap);
  } catch (...) {
    t_capturing = 0;
    cudaGraph_t tmp;
    cudaStreamEndCapture(cap, &tmp);
    throw;
  }
  t_capturing = 0;
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* leaves = nullptr;
  size_t nleaves = 0;
  CK(cudaStreamGetCaptureInfo(cap, &cs, nullptr, nullptr, &leaves, nullptr, &nleaves));
  std::vector<cudaGraphNode_t> out(leaves, leaves + nleaves);
  cudaGraph_t g2;
  CK(cudaStreamEndCapture(cap, &g2));
  return out;
}

// Adds a WHILE node after deps on handle h; returns (node, body graph).
std::pair<cudaGraphNode_t, cudaGraph_t> add_while(cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps,
                                                  cudaGraphConditionalHandle h) {
  // cudaGraphNodeParams holds a union whose members are not default-constructible in C++: zeroed storage
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  std::memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(raw);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &cp));
  return {node, cp.conditional.phGraph_out[0]};
}

int count_kernel_nodes(cudaGraph_t g) {
  size_t n = 0;
  CK(cudaGraphGetNodes(g, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  CK(cudaGraphGetNodes(g, nodes.data(), &n));
  int k = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    CK(cudaGraphNodeGetType(nd, &t));
    if (t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

// Records the solve:
//  FP64 mode:   [zero U] reset, [warm: w = Q U], init, WHILE{ apply+(h,w); update; hupdate }, true residual.
//  refinement:  [zero U] outer reset, r64 = F - Q U (FP64, decides convergence; = F without a warm start),
//               WHILE_outer{ F32 = r64/|r64|; reset; init32; WHILE_inner{ apply32; update32; hupdate32 };
//               U += |r64| c32; r64 = F - Q U }.
void build_graph(const Units& us, Entry& en, const Key& key, cudaStream_t cap) {
  cudaGraph_t g;
  CK(cudaGraphCreate(&g, 0));
  en.graph = g;
  if (key.mode == QP_MODE_FP64) {
    cudaGraphConditionalHandle hc;
    CK(cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault));
    auto pre = capture_into(g, {}, cap, [&](cudaStream_t s) {
      if (!key.warm) zero_solutions(us, s);
      launch_level_reset(en.bd, 0, s);
      if (key.warm) record_apply(us, en, LEVEL_FP64, EPI_NONE, REFINE_NONE, 0, s);
      launch_pcg_init(en.bd, us.max_rhs, LEVEL_FP64, key.warm != 0, hc, en.nblk, s);
      CK_LAUNCH();
    });
    auto wl = add_while(g, pre, hc);
    capture_into(wl.second, {}, cap, [&](cudaStream_t s) { body_pcg(us, en, LEVEL_FP64, hc, s); });
    capture_into(g, {wl.first}, cap, [&](cudaStream_t s) {
      record_apply(us, en, LEVEL_FP64, EPI_RESIDUAL, REFINE_NONE, 0, s);
      zero_mean_mode(us, s);
    });
    en.body_nodes = count_kernel_nodes(wl.second);
  } else {
    cudaGraphConditionalHandle ho;
    CK(cudaGraphConditionalHandleCreate(&ho, g, 1, cudaGraphCondAssignDefault));
    // the first true residual before the loop (U = 0 without a warm start: r64 = F, no apply), then per
    // outer iteration: inner FP32 solve, accumulation, true residual
    auto pre = capture_into(g, {}, cap, [&](cudaStream_t s) {
      if (!key.warm) zero_solutions(us, s);
      launch_level_reset(en.bd, 1, s);
      record_apply(us, en, LEVEL_FP64, EPI_RESIDUAL, key.warm ? REFINE_ON : REFINE_ZERO_U, ho, s);
    });
    auto wo = add_while(g, pre, ho);
    cudaGraph_t ob = wo.second;
    cudaGraphConditionalHandle hi;
    CK(cudaGraphConditionalHandleCreate(&hi, ob, 1, cudaGraphCondAssignDefault));
    auto b1 = capture_into(ob, {}, cap, [&](cudaStream_t s) {
      launch_refine_prep(en.bd, en.nblk, s);
      launch_level_reset(en.bd, 0, s);
      launch_pcg_init(en.bd, us.max_rhs, LEVEL_FP32, false, hi, en.nblk, s);
      CK_LAUNCH();
    });
    auto wi = add_while(ob, b1, hi);
    capture_into(wi.second, {}, cap, [&](cudaStream_t s) { body_pcg(us, en, LEVEL_FP32, hi, s); });
    capture_into(ob, {wi.first}, cap, [&](cudaStream_t s) {
      launch_refine_accum(en.bd, en.nblk, s);
      record_apply(us, en, LEVEL_FP64, EPI_RESIDUAL, REFINE_ON, ho, s);
      CK_LAUNCH();
    });
    capture_into(g, {wo.first}, cap, [&](cudaStream_t s) { zero_mean_mode(us, s); });
    en.body_nodes = count_kernel_nodes(wi.second);
    en.outer_nodes = count_kernel_nodes(ob);
  }
  en.fixed_nodes = count_kernel_nodes(g);
  CK(cudaGraphInstantiate(&en.exec, g, 0));
}

// The same sequence driven by a host loop that reads the device "done" counters (no graph).
void run_direct(const Units& us, Entry& en, const Key& key, int nslots, cudaStream_t s) {
  auto read_done = [&](int which) {
    int h = 0;
    CK(cudaMemcpyAsync(&h, en.bd.ndone + which, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return h;
  };
  const bool timing = g_phase_timing.load(std::memory_order_relaxed) != 0;
  auto pcg_loop = [&](int level) {
    int it = 0, chunk = timing ? 1 : 4;
    while (read_done(0) < nslots) {
      for (int i = 0; i < chunk; ++i) body_pcg(us, en, level, 0, s);
      it += chunk;
      if (!timing) chunk = std::min(chunk * 2, 32);
      if (it > key.maxit + 64) raise(QP_ERR_CUDA, "PCG loop exceeded its cap without the device flag");
    }
  };
  if (key.mode == QP_MODE_FP64) {
    timed(QP_PHASE_OTHER, s, [&] {
      if (!key.warm) zero_solutions(us, s);
      launch_level_reset(en.bd, 0, s);
    });
    if (key.warm) timed(QP_PHASE_RESIDUAL64, s, [&] { record_apply(us, en, LEVEL_FP64, EPI_NONE, REFINE_NONE, 0, s); });
    timed(QP_PHASE_INIT64, s, [&] { launch_pcg_init(en.bd, us.max_rhs, LEVEL_FP64, key.warm != 0, 0, en.nblk, s); });
    pcg_loop(LEVEL_FP64);
    timed(QP_PHASE_RESIDUAL64, s, [&] { record_apply(us, en, LEVEL_FP64, EPI_RESIDUAL, REFINE_NONE, 0, s); });
  } else {
    timed(QP_PHASE_OTHER, s, [&] {
      if (!key.warm) zero_solutions(us, s);
      launch_level_reset(en.bd, 1, s);
    });
    timed(QP_PHASE_RESIDUAL64, s, [&] {
      record_apply(us, en, LEVEL_FP64, EPI_RESIDUAL, key.warm ? REFINE_ON : REFINE_ZERO_U, 0, s);
    });
    for (int outer = 0; outer < 64; ++outer) {
      if (read_done(1) >= nslots) break;
      timed(QP_PHASE_REFINE, s, [&] { launch_refine_prep(en.bd, en.nblk, s); });
      timed(QP_PHASE_INIT32, s, [&] {
        launch_level_reset(en.bd, 0, s);
        launch_pcg_init(en.bd, us.max_rhs, LEVEL_FP32, false, 0, en.nblk, s);
      });
      pcg_loop(LEVEL_FP32);
      timed(QP_PHASE_REFINE, s, [&] { launch_refine_accum(en.bd, en.nblk, s); });
      timed(QP_PHASE_RESIDUAL64, s, [&] { record_apply(us, en, LEVEL_FP64, EPI_RESIDUAL, REFINE_ON, 0, s); });
      CK_LAUNCH();
    }
  }
  timed(QP_PHASE_OTHER, s, [&] { zero_mean_mode(us, s); });
}

// Builds (or finds) the entry for these units and key: device unit/chunk tables and the recorded graph.
Entry& get_entry(Solver* sv, const Units& us, const Key& key, cudaStream_t s) {
  auto it = sv->cache.find(key);
  if (it != sv->cache.end()) return *it->second;
  std::unique_ptr<Entry> en(new Entry());
  const int nu = (int)us.plans.size();
  int64_t E = 0;
  int nslots = 0;
  for (int u = 0; u < nu; ++u) {
    E += us.plans[u]->D;
    nslots += us.nrhs[u];
  }
  (void)E;
  std::vector<UnitDev> units(nu);
  std::vector<int> chunk_unit;
  for (int u = 0; u < nu; ++u) {
    qp_plan* p = us.plans[u];
    UnitDev& x = units[u];
    std::memset(&x, 0, sizeof(x));
    x.plan = p->pd;
    x.D = p->D;
    x.nrhs = us.nrhs[u];
    // chunks dispatched in index order (one block per chunk, or for the FP32 star-1 batch kernel a grid of the
    // resident blocks walking c, c + grid, ...) so that the resident blocks cover a contiguous window of modes
    // (neighbour reads along outer axes then hit L2); the chunk depends on D only (chunk_modes), so the
    // reduction order of a unit does not depend on its batch or on which block walks the chunk
    const int64_t chunk = chunk_modes(p->D);
    x.chunk = (int)chunk;
    x.run = last_axis_run(p);
    x.fft = p->backend == QP_BACKEND_FFT ? 1 : 0;
    x.hspec = p->host_pd.hspec;
    x.Hl = p->host_pd.Hl;
    x.hdiv = make_fastdiv((uint32_t)p->host_pd.Hl);
    x.chunk0 = (int)chunk_unit.size();
    x.nchunk = (int)((p->D + chunk - 1) / chunk);
    for (int c = 0; c < x.nchunk; ++c) chunk_unit.push_back(u);
    x.F = p->v64.F;
    x.U = p->v64.X;
    x.r = p->v64.r;
    x.h = p->v64.h;
    x.w = p->v64.w;
    x.F32 = p->v32.F;
    x.U32 = p->v32.X;
    x.r32 = p->v32.r;
    x.h32 = p->v32.h;
    x.w32 = p->v32.w;
    x.minv64 = key.precond == QP_PRECOND_FROBENIUS ? p->frob64 : p->jac64;
    x.minv32 = key.precond == QP_PRECOND_FROBENIUS ? p->frob32 : p->jac32;
  }
  const int nchunks = (int)chunk_unit.size();
  auto up = [&](const void* src, size_t bytes_) {
    void* dst = dev_alloc(bytes_, s);
    en->allocs.push_back(dst);
    CK(cudaMemcpyAsync(dst, src, bytes_, cudaMemcpyHostToDevice, s));   // pageable source: staged before return
    return dst;
  };
  BatchDev& bd = en->bd;
  bd.nunits = nu;
  bd.nchunks = nchunks;
  bd.nslots = nslots;
  bd.units = (const UnitDev*)up(units.data(), units.size() * sizeof(UnitDev));
  bd.single = nu == 1 ? 1 : 0;
  {
    // the FP32 apply of a single star-1 unit (even last axis) sweeps upwards, the general batch kernel downwards
    const qp_plan* p0 = nu == 1 ? us.plans[0] : nullptr;
    const bool star = p0 && p0->backend == QP_BACKEND_TAPS && p0->host_pd.star1 && last_axis_run(p0) == 2;
    bd.apply_down = star ? 0 : 1;
  }
  bd.hspec_any = 0;
  for (const UnitDev& x : units) bd.hspec_any |= x.hspec;
  bd.pu = units[0];
  bd.st = sv->st;
  bd.chunk_unit = (const int*)up(chunk_unit.data(), chunk_unit.size() * sizeof(int));
  {
    void* pp = dev_alloc((size_t)NSLOT_PERSIST * nchunks * sizeof(double), s);
    en->allocs.push_back(pp);
    bd.partials = (double*)pp;
  }
  bd.ucount = sv->ucount;
  bd.kcount = sv->kcount;
  bd.ndone = sv->ndone;
  bd.tol2 = (key.mode == QP_MODE_FP64 ? key.tol : key.inner_tol);
  bd.tol2 *= bd.tol2;
  bd.otol2 = key.tol * key.tol;
  bd.maxit = key.maxit;
  bd.max_outer = key.max_outer;
  en->nblk = nchunks;
  if ((us.exec == QP_EXEC_AUTO || us.exec == QP_EXEC_PERSISTENT) && nu == 1 && !us.direct && us.run == 2) {
    // every block of a cooperative launch is resident: at most the occupancy limit, at most one per chunk.
    // AUTO takes the persistent form only when every chunk has its own resident block (small and medium
    // problems, where launch and synchronisation latency dominate); larger solves keep the graph, whose
    // kernels run at higher occupancy.
    const size_t smem = persistent_smem(us.max_coef);
    const qp_plan* p0 = us.plans[0];
    const int sk = (p0->backend == QP_BACKEND_TAPS && p0->host_pd.star1 && p0->w64)
                       ? (p0->kind == QP_COEF_DIAG ? 2 : 1) : 0;
    int capn = 0;
    try {
      capn = persistent_capacity(us.all_real, us.max_rhs, sk, sk ? &p0->star_host : nullptr, smem);
    } catch (const QpError&) {
      cudaGetLastError();
      capn = 0;
    }
    if (capn > 0 && (us.exec == QP_EXEC_PERSISTENT || nchunks <= capn)) {
      en->pgrid = std::min(capn, nchunks);
      en->psmem = smem;
      en->psk = sk;
    }
  }
  if (en->pgrid == 0 && sv->graphs_ok && !us.direct) {
    try {
      build_graph(us, *en, key, sv->capture_stream());
    } catch (const QpError&) {
      // graphs with conditional nodes are unavailable: host-driven loops for this solver from now on
      cudaGetLastError();
      if (en->exec) cudaGraphExecDestroy(en->exec);
      if (en->graph) cudaGraphDestroy(en->graph);
      en->exec = nullptr;
      en->graph = nullptr;
      sv->graphs_ok = false;
    }
  }
  Entry& ref = *en;
  sv->cache[key] = std::move(en);
  return ref;
}

// Limit of one grid-barrier wait in the persistent solve (a wait covers one phase of the slowest block).
std::atomic<double> g_barrier_timeout{2.0};

struct SolveResult {
  std::vector<int> iters, outer, status;
  std::vector<double> rel, f2;
};

// One solve of all units (their F in v64.F, solutions in v64.X); reads back the state.
void run_solve(Solver* sv, const Units& us, const Key& key, cudaStream_t s, SolveResult& res) {
  Entry& en = get_entry(sv, us, key, s);
  int nslots = 0;
  for (int r : us.nrhs) nslots += r;
  if (g_phase_timing.load(std::memory_order_relaxed)) {
    run_direct(us, en, key, nslots, s);   // the same kernels, one timed group at a time
  } else if (en.pgrid > 0) {
    launch_persistent(en.bd, us.all_real, us.max_rhs, en.psk, en.psk ? &us.plans[0]->star_host : nullptr, key.mode,
                      key.warm != 0, sv->pbar, sv->perr, g_barrier_timeout.load(), en.pgrid, en.psmem, s);
    CK(cudaMemcpyAsync(sv->h_perr, sv->perr, sizeof(int), cudaMemcpyDeviceToHost, s));
  } else if (en.exec) {
    CK(cudaGraphLaunch(en.exec, s));
  } else {
    run_direct(us, en, key, nslots, s);
  }
  const size_t nu = us.plans.size();
  CK(cudaMemcpyAsync(sv->h_st, sv->st, nu * MAXR * sizeof(RhsSt), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  resolve_phases();
  const bool ran_persistent = en.pgrid > 0 && !g_phase_timing.load(std::memory_order_relaxed);
  if (ran_persistent && *sv->h_perr != 0)
    raise(QP_ERR_TIMEOUT, "persistent solve: a grid-barrier wait exceeded its limit");
  res = SolveResult();
  int max_it = 0, max_outer = 0, sum_inner_max = 0;
  for (size_t u = 0; u < nu; ++u)
    for (int r = 0; r < us.nrhs[u]; ++r) {
      const RhsSt& x = sv->h_st[u * MAXR + r];
      res.rel.push_back(x.of2 > 0.0 ? std::sqrt(x.orr / x.of2) : 0.0);
      res.f2.push_back(x.of2);
      if (key.mode == QP_MODE_FP64) {
        res.iters.push_back(x.iters);
        res.outer.push_back(0);
        res.status.push_back(x.status);
        max_it = std::max(max_it, x.iters);
      } else {
        res.iters.push_back(x.inner_total);
        res.outer.push_back(x.outer);
        res.status.push_back(x.ostatus);
        sum_inner_max = std::max(sum_inner_max, x.inner_total);
        max_outer = std::max(max_outer, x.outer);
      }
    }
  if (en.exec && !g_phase_timing.load(std::memory_order_relaxed)) {   // the graph ran: count its kernel nodes
    if (key.mode == QP_MODE_FP64) count_launch(en.fixed_nodes + en.body_nodes * std::max(1, max_it));
    else count_launch(en.fixed_nodes + en.outer_nodes * std::max(0, max_outer - 1) +
                      en.body_nodes * (sum_inner_max + max_outer));
  }
}

// The full solve with restarts (FP64 mode: the recursive residual can drift from the true one) and the
// F = 0 convention (U = 0).
void solve_units(Solver* sv, const Units& us, const qp_solve_opts& o, bool warm, cudaStream_t s, SolveResult& res) {
  Key key{o.mode, o.precond, 0, warm ? 1 : 0, o.maxit, o.max_outer > 0 ? o.max_outer : 12, o.tol,
          o.inner_tol > 0.0 ? o.inner_tol : 1e-5};
  for (int r : us.nrhs) key.nrhs = key.nrhs * 8 + r;
  run_solve(sv, us, key, s, res);
  if (o.mode == QP_MODE_FP64) {
    for (int attempt = 0; attempt < 2; ++attempt) {
      bool again = false;
      for (size_t i = 0; i < res.status.size(); ++i)
        if (res.status[i] == QP_OK && res.rel[i] > o.tol) again = true;
      if (!again) break;
      SolveResult r2;
      Key k2 = key;
      k2.warm = 1;
      run_solve(sv, us, k2, s, r2);
      for (size_t i = 0; i < res.status.size(); ++i) r2.iters[i] += res.iters[i];
      res = r2;
    }
    for (size_t i = 0; i < res.status.size(); ++i)
      if (res.status[i] == QP_OK && res.rel[i] > o.tol) res.status[i] = QP_ERR_NO_CONVERGENCE;
  }
  size_t i = 0;
  for (size_t u = 0; u < us.plans.size(); ++u)
    for (int r = 0; r < us.nrhs[u]; ++r, ++i)
      if (res.f2[i] == 0.0)
        CK(cudaMemsetAsync(us.plans[u]->v64.X + (size_t)r * us.plans[u]->D, 0, us.plans[u]->D * sizeof(double2), s));
}

Units single_units(qp_plan* p, int nrhs) {
  Units us;
  us.plans = {p};
  us.nrhs = {nrhs};
  us.all_real = p->backend == QP_BACKEND_FFT ? true : p->real_coef;
  us.max_coef = std::max(1, p->coef_count);
  us.max_rhs = nrhs;
  us.direct = p->exec == QP_EXEC_DIRECT;
  us.exec = (p->backend == QP_BACKEND_TAPS && p->spectrum == QP_SPECTRUM_FULL) ? p->exec : QP_EXEC_GRAPH;
  us.run = last_axis_run(p);
  return us;
}

void check_opts(const qp_solve_opts* o, const qp_plan* p) {
  if (!o) raise(QP_ERR_INVALID_ARG, "opts must be non-null");
  if (!(o->tol >= 0.0) || o->maxit < 1) raise(QP_ERR_INVALID_ARG, "tol must be >= 0 and maxit >= 1");
  if (o->precond != QP_PRECOND_JACOBI && o->precond != QP_PRECOND_FROBENIUS)
    raise(QP_ERR_INVALID_ARG, "unknown preconditioner");
  if (o->mode != QP_MODE_FP64 && o->mode != QP_MODE_FP32_REFINE) raise(QP_ERR_INVALID_ARG, "unknown mode");
  if (p && o->mode == QP_MODE_FP64 && !(p->precisions & 1))
    raise(QP_ERR_INVALID_ARG, "plan was created without the FP64 solve workspace");
  if (p && o->mode == QP_MODE_FP32_REFINE && !(p->precisions & 2))
    raise(QP_ERR_INVALID_ARG, "plan was created without the FP32 solve workspace");
}

// Builds the diagonal a solve is about to use if the plan does not hold it yet (the FFT backend's Frobenius
// diagonal, on first request).
void prepare_precond(qp_plan* p, int precond, cudaStream_t s) {
  if (precond != QP_PRECOND_FROBENIUS || p->frob_ready) return;
  if (p->spectrum == QP_SPECTRUM_HALF)
    raise(QP_ERR_UNSUPPORTED, "the Frobenius-optimal diagonal is not built for half-spectrum plans (Jacobi is)");
  if (p->backend == QP_BACKEND_TAPS) {
    launch_diag(p->pd, p->coef_count, p->D, p->jac64, p->frob64, p->jac32, p->frob32, p->scratch, p->counter,
                p->small, p->nblk, true, s);
    CK_LAUNCH();
  } else {
    fft_frobenius(p->fft, p->host_pd, p->pd, p->frob64, p->frob32, s);
  }
  p->frob_ready = true;
}

void corrector_rhs(qp_plan* p, int j0, int nrhs, double2* F, cudaStream_t s) {
  CK(cudaMemsetAsync(F, 0, (size_t)nrhs * p->D * sizeof(double2), s));
  if (p->backend == QP_BACKEND_TAPS) launch_rhs_taps(p->pd, p->coef_count, j0, nrhs, p->D, F, s);
  else fft_rhs(p->fft, p->host_pd, p->pd, j0, nrhs, F, s);
  CK_LAUNCH();
}

// a* into dst (device, 2 d^2 doubles: re, im per entry).
void astar_launch(qp_plan* p, const double2* U, double* dst, cudaStream_t s) {
  if (p->backend == QP_BACKEND_TAPS) launch_astar_taps(p->pd, p->coef_count, p->D, U, dst, s);
  else fft_astar(p->fft, p->host_pd, p->pd, U, dst, s);
  CK_LAUNCH();
}

void astar_reduce(qp_plan* p, const double2* U, double* Are, double* Aim, cudaStream_t s) {
  astar_launch(p, U, p->small, s);
  const int dd = p->d * p->d;
  CK(cudaMemcpyAsync(p->h_small, p->small, 2 * dd * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int q = 0; q < dd; ++q) {
    if (Are) Are[q] = p->h_small[2 * q];
    if (Aim) Aim[q] = p->h_small[2 * q + 1];
  }
}

qp_status worst(const SolveResult& r) {
  qp_status w = QP_OK;
  for (int st : r.status)
    if (st != QP_OK && (w == QP_OK || st == QP_ERR_BREAKDOWN)) w = (qp_status)st;
  return w;
}

void fill_info(const SolveResult& r, size_t off, int count, qp_solve_info* info) {
  if (!info) return;
  for (int k = 0; k < count; ++k) {
    info[k].status = r.status[off + k];
    info[k].iterations = r.iters[off + k];
    info[k].outer_iterations = r.outer[off + k];
    info[k].rel_residual = r.rel[off + k];
  }
}

}  // namespace

#define API_BEGIN try {
#define API_END                                              \
  }                                                          \
  catch (const QpError& e) {                                 \
    g_err = e.msg;                                           \
    return e.s;                                              \
  }                                                          \
  catch (const std::exception& e) {                          \
    g_err = e.what();                                        \
    return QP_ERR_CUDA;                                      \
  }                                                          \
  g_err.clear();                                             \
  return QP_OK;

extern "C" {

const char* qp_last_error(void) { return g_err.c_str(); }

uint64_t qp_launch_count(void) { return qp::g_launches.load(std::memory_order_relaxed); }

qp_status qp_plan_diagonal(qp_plan* p, int precond, double* out, void* stream) {
  API_BEGIN
  if (!p || !out) raise(QP_ERR_INVALID_ARG, "plan and out must be non-null");
  if (precond != QP_PRECOND_JACOBI && precond != QP_PRECOND_FROBENIUS) raise(QP_ERR_INVALID_ARG, "unknown preconditioner");
  cudaStream_t s = S(stream);
  prepare_precond(p, precond, s);
  const double* src = precond == QP_PRECOND_FROBENIUS ? p->frob64 : p->jac64;
  CK(cudaMemcpyAsync(out, src, (size_t)p->D * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  API_END
}

qp_status qp_l2qp_error(qp_plan* p, int nrhs, const void* U, const void* Uref, double* out, void* stream) {
  API_BEGIN
  if (!p || !U || !out) raise(QP_ERR_INVALID_ARG, "plan, U and out must be non-null");
  if (nrhs < 1 || nrhs > MAXR) raise(QP_ERR_INVALID_ARG, "nrhs must be 1..QP_MAX_RHS");
  if (((uintptr_t)U | (uintptr_t)Uref) & 15u) raise(QP_ERR_INVALID_ARG, "U and Uref must be 16-byte aligned");
  cudaStream_t s = S(stream);
  launch_l2_norms(p->D, nrhs, (const double2*)U, (const double2*)Uref, p->scratch, p->nblk, p->small,
                  p->host_pd.hspec ? p->host_pd.Hl : 0, s);
  CK_LAUNCH();
  CK(cudaMemcpyAsync(p->h_small, p->small, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int r = 0; r < nrhs; ++r) out[r] = p->h_small[r];
  API_END
}

qp_status qp_fft_tune_cache_save(const char* path, int* entries) {
  API_BEGIN
  if (!path) raise(QP_ERR_INVALID_ARG, "path must be non-null");
  const int n = fft_tune_cache_save(path);
  if (n < 0) raise(QP_ERR_INVALID_ARG, std::string("cannot write the tuning cache to ") + path);
  if (entries) *entries = n;
  API_END
}

qp_status qp_fft_tune_cache_load(const char* path, int* entries) {
  API_BEGIN
  if (!path) raise(QP_ERR_INVALID_ARG, "path must be non-null");
  const int n = fft_tune_cache_load(path);
  if (n == -2) raise(QP_ERR_UNSUPPORTED, std::string("the tuning cache ") + path + " was timed on another GPU");
  if (n < 0) raise(QP_ERR_INVALID_ARG, std::string("cannot read a tuning cache from ") + path);
  if (entries) *entries = n;
  API_END
}

qp_status qp_fft_tune_cache_clear(void) {
  API_BEGIN
  fft_tune_cache_clear();
  API_END
}

qp_status qp_set_fft_autotune(int enabled) {
  API_BEGIN
  fft_set_autotune(enabled != 0);
  API_END
}

qp_status qp_fft_schedule(const qp_plan* p, int precision, int* index, int* count, double* ms, char* text,
                          int text_len) {
  API_BEGIN
  if (!p) raise(QP_ERR_INVALID_ARG, "plan must be non-null");
  if (p->backend != QP_BACKEND_FFT || !p->fft) raise(QP_ERR_UNSUPPORTED, "the plan has no FFT backend");
  if (precision != QP_FP64 && precision != QP_FP32) raise(QP_ERR_INVALID_ARG, "precision must be QP_FP64 or QP_FP32");
  std::string t;
  float m = -1.f;
  const int idx = fft_schedule_get(p->fft, precision == QP_FP64, t, m);
  if (index) *index = idx;
  if (count) *count = fft_schedule_count(p->fft, precision == QP_FP64);
  if (ms) *ms = (double)m;
  if (text && text_len > 0) {
    const size_t nb = std::min<size_t>(t.size(), (size_t)text_len - 1);
    std::memcpy(text, t.data(), nb);
    text[nb] = 0;
  }
  API_END
}

qp_status qp_fft_set_schedule(qp_plan* p, int precision, int index) {
  API_BEGIN
  if (!p) raise(QP_ERR_INVALID_ARG, "plan must be non-null");
  if (p->backend != QP_BACKEND_FFT || !p->fft) raise(QP_ERR_UNSUPPORTED, "the plan has no FFT backend");
  if (precision != QP_FP64 && precision != QP_FP32) raise(QP_ERR_INVALID_ARG, "precision must be QP_FP64 or QP_FP32");
  fft_schedule_set(p->fft, precision == QP_FP64, index);
  API_END
}

qp_status qp_set_phase_timing(int enabled) {
  API_BEGIN
  std::lock_guard<std::mutex> lk(g_phase_mu);
  for (int i = 0; i < QP_NPHASE; ++i) {
    g_phase_ms[i] = 0.0;
    g_phase_count[i] = 0;
  }
  g_phase_timing.store(enabled ? 1 : 0);
  API_END
}

qp_status qp_phase_times(double* ms, int64_t* launches, int count) {
  API_BEGIN
  if (count < 0) raise(QP_ERR_INVALID_ARG, "count must be >= 0");
  std::lock_guard<std::mutex> lk(g_phase_mu);
  for (int i = 0; i < count; ++i) {
    if (ms) ms[i] = i < QP_NPHASE ? g_phase_ms[i] : 0.0;
    if (launches) launches[i] = i < QP_NPHASE ? g_phase_count[i] : 0;
  }
  API_END
}

qp_status qp_memory_pool_stats(int64_t* reserved_bytes, int64_t* used_bytes, uint64_t* allocations) {
  API_BEGIN
  pool_stats(reserved_bytes, used_bytes, allocations);
  API_END
}

qp_status qp_set_memory_cache(int64_t bytes) {
  API_BEGIN
  set_cache_bytes(bytes);
  API_END
}

qp_status qp_set_barrier_timeout(double seconds) {
  API_BEGIN
  if (!(seconds > 0.0 && seconds <= 3600.0)) raise(QP_ERR_INVALID_ARG, "barrier timeout must be in (0, 3600] s");
  g_barrier_timeout.store(seconds);
  API_END
}

qp_status qp_plan_create(int d, int n, const double* P, const int* N, const qp_coeff* coeff, const qp_options* opt,
                         void* stream, qp_plan** out) {
  API_BEGIN
  if (!out) raise(QP_ERR_INVALID_ARG, "out must be non-null");
  *out = nullptr;
  if (!coeff) raise(QP_ERR_INVALID_ARG, "coeff must be non-null");
  std::unique_ptr<qp_plan> p(new qp_plan());
  cudaStream_t s = S(stream);
  p->create_stream = s;
  p->spectrum = opt ? opt->spectrum : QP_SPECTRUM_FULL;
  if (p->spectrum != QP_SPECTRUM_FULL && p->spectrum != QP_SPECTRUM_HALF) raise(QP_ERR_INVALID_ARG, "unknown spectrum");
  const bool half = p->spectrum == QP_SPECTRUM_HALF;
  if (half && (coeff->repr != QP_REPR_TAPS || (opt && opt->backend == QP_BACKEND_FFT)))
    raise(QP_ERR_UNSUPPORTED, "the half-spectrum storage needs a tap coefficient on the taps backend");
  build_geometry(p.get(), d, n, P, N, half);
  if (coeff->kind < QP_COEF_SCALAR || coeff->kind > QP_COEF_SYM) raise(QP_ERR_INVALID_ARG, "unknown coefficient kind");
  p->kind = coeff->kind;
  p->ncomp = ncomp_of(coeff->kind, d);
  p->host_pd.kind = p->kind;
  p->host_pd.ncomp = p->ncomp;
  const int backend_req = opt ? opt->backend : QP_BACKEND_AUTO;
  p->max_rhs = (opt && opt->max_rhs > 0) ? opt->max_rhs : d;
  if (p->max_rhs > MAXR) raise(QP_ERR_INVALID_ARG, "max_rhs must be <= 4");
  p->precisions = (opt && opt->precisions) ? (opt->precisions & 3) : 3;
  p->exec = opt ? opt->exec : QP_EXEC_AUTO;
  if (p->exec < QP_EXEC_AUTO || p->exec > QP_EXEC_PERSISTENT) raise(QP_ERR_INVALID_ARG, "unknown exec mode");
  if (coeff->repr == QP_REPR_TAPS) {
    p->backend = (backend_req == QP_BACKEND_FFT) ? QP_BACKEND_FFT : QP_BACKEND_TAPS;
  } else if (coeff->repr == QP_REPR_GRID) {
    if (backend_req == QP_BACKEND_TAPS) raise(QP_ERR_INVALID_ARG, "a grid coefficient needs the FFT backend");
    if (!coeff->grid) raise(QP_ERR_INVALID_ARG, "grid must be a non-null device pointer");
    if ((uintptr_t)coeff->grid & 7u) raise(QP_ERR_INVALID_ARG, "grid must be 8-byte aligned");
    p->backend = QP_BACKEND_FFT;
  } else {
    raise(QP_ERR_INVALID_ARG, "unknown coefficient representation");
  }
  p->host_pd.backend = p->backend;
  if (p->backend == QP_BACKEND_FFT)
    for (int j = 0; j < n; ++j)
      if (!fft_supported(N[j])) raise(QP_ERR_UNSUPPORTED, "the FFT backend does not transform N_j = " + std::to_string(N[j]));
  if (coeff->repr == QP_REPR_TAPS) build_taps(p.get(), coeff);
  alloc_workspace(p.get());
  p->pd = (PlanDev*)p->dalloc(sizeof(PlanDev));
  bool fft_ok = true;
  for (int j = 0; j < n; ++j) fft_ok = fft_ok && fft_supported(N[j]);
  // (only dense tap lists on grids large enough to time reliably: below that the stencil is taken outright)
  if (p->backend == QP_BACKEND_TAPS && backend_req == QP_BACKEND_AUTO && fft_ok && (p->precisions & 2) && !half &&
      fft_autotune_on() && p->host_pd.ntaps >= 64 && p->D >= 65536) {
    CK(cudaMemcpyAsync(p->pd, &p->host_pd, sizeof(PlanDev), cudaMemcpyHostToDevice, s));
    p->backend = tune_backend(p.get(), s);
    if (p->backend == QP_BACKEND_FFT) {   // the stencil's own data is not used from here on
      p->host_pd.backend = QP_BACKEND_FFT;
      p->host_pd.star1 = 0;
      p->host_pd.star = nullptr;
    }
  }
  if (p->backend == QP_BACKEND_TAPS) {
    CK(cudaMemcpyAsync(p->pd, &p->host_pd, sizeof(PlanDev), cudaMemcpyHostToDevice, s));
    launch_diag(p->pd, p->coef_count, p->D, p->jac64, p->frob64, p->jac32, p->frob32, p->scratch, p->counter,
                p->small, p->nblk, false, s);
    CK_LAUNCH();
    build_star_weights(p.get(), s);
    build_gen_weights(p.get(), s);
  } else {
    CK(cudaMemcpyAsync(p->pd, &p->host_pd, sizeof(PlanDev), cudaMemcpyHostToDevice, s));
    if (!p->fft) {   // (AUTO with taps that the FFT backend applies faster: made and transformed already)
      p->fft = fft_plan_create(p->host_pd, p->precisions, p->max_rhs, s);
      if (coeff->repr == QP_REPR_GRID) fft_set_grid(p->fft, p->host_pd, p->pd, coeff->grid, s);
      else fft_set_taps(p->fft, p->host_pd, p->pd, s);
    }
    fft_autotune(p->fft, p->host_pd, p->pd, s);
    fft_diag(p->fft, &p->host_pd, p->pd, p->jac64, p->frob64, p->jac32, p->frob32, p->small, s);
    CK_LAUNCH();
  }
  CK(cudaMemcpyAsync(p->h_small, p->small, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double pmax = 0.0;
  for (int a = 0; a < d; ++a)
    for (int j = 0; j < n; ++j) pmax = std::max(pmax, std::fabs(p->P[a][j]));
  p->min_abs_lambda = std::sqrt(std::max(p->h_small[0], 0.0));
  if (!(p->min_abs_lambda > 1e-12 * pmax))
    raise(QP_ERR_SINGULAR_P, "min over k != 0 of |P k| is ~0: the columns of P are not Q-linearly independent "
                             "on this grid");
  if (!(p->h_small[1] > 0.0)) raise(QP_ERR_NOT_ELLIPTIC, "the Jacobi diagonal q(k) is not positive");
  if (p->backend == QP_BACKEND_FFT && !(p->h_small[2] > 0.0))
    raise(QP_ERR_NOT_ELLIPTIC, "the coefficient is not positive definite at some grid node");
  *out = p.release();
  API_END
}

qp_status qp_plan_destroy(qp_plan* plan) {
  API_BEGIN
  delete plan;
  API_END
}

qp_status qp_plan_query(const qp_plan* p, qp_plan_info* info) {
  API_BEGIN
  if (!p || !info) raise(QP_ERR_INVALID_ARG, "plan and info must be non-null");
  info->D = p->Dfull;
  info->stored = p->D;
  info->spectrum = p->spectrum;
  info->backend = p->backend;
  info->ntaps = p->host_pd.ntaps;
  info->max_rhs = p->max_rhs;
  info->min_abs_lambda = p->min_abs_lambda;
  info->device_bytes = p->bytes + (p->fft ? fft_plan_bytes(p->fft) : 0);
  info->star = p->host_pd.star1;
  info->stored_weights = (p->w64 != nullptr || p->host_pd.wgen != nullptr) ? 1 : 0;
  API_END
}

qp_status qp_apply_stiffness(qp_plan* p, int nrhs, const void* U, void* QU, int precision, void* stream) {
  API_BEGIN
  if (!p) raise(QP_ERR_INVALID_ARG, "plan must be non-null");
  if (nrhs < 1 || nrhs > p->max_rhs) raise(QP_ERR_INVALID_ARG, "nrhs must be 1..max_rhs");
  if (!U || !QU || U == QU) raise(QP_ERR_INVALID_ARG, "U and QU must be distinct non-null device pointers");
  if (((uintptr_t)U | (uintptr_t)QU) & 15u) raise(QP_ERR_INVALID_ARG, "U and QU must be 16-byte aligned");
  if (precision != QP_FP64 && precision != QP_FP32) raise(QP_ERR_INVALID_ARG, "precision must be QP_FP64 or QP_FP32");
  cudaStream_t s = S(stream);
  if (p->backend == QP_BACKEND_TAPS) {
    const StarParams* st1 = (p->host_pd.star1 && (precision == QP_FP32 || p->w64)) ? &p->star_host : nullptr;
    if (precision == QP_FP64)
      launch_apply_plain<double>(p->pd, p->real_coef, p->coef_count, p->D, nrhs, (const double2*)U, (double2*)QU,
                                 last_axis_run(p), st1, p->kind, s);
    else
      launch_apply_plain<float>(p->pd, p->real_coef, p->coef_count, p->D, nrhs, (const float2*)U, (float2*)QU,
                                last_axis_run(p), st1, p->kind, s);
  } else {
    if (precision == QP_FP64) fft_apply<double>(p->fft, p->host_pd, p->pd, (const double2*)U, (double2*)QU, nrhs, s);
    else fft_apply<float>(p->fft, p->host_pd, p->pd, (const float2*)U, (float2*)QU, nrhs, s);
  }
  CK_LAUNCH();
  API_END
}

qp_status qp_corrector_rhs(qp_plan* p, int j0, int nrhs, void* F, void* stream) {
  API_BEGIN
  if (!p || !F) raise(QP_ERR_INVALID_ARG, "plan and F must be non-null");
  if (j0 < 0 || nrhs < 1 || j0 + nrhs > p->d) raise(QP_ERR_INVALID_ARG, "need 0 <= j0 and j0 + nrhs <= d");
  if ((uintptr_t)F & 15u) raise(QP_ERR_INVALID_ARG, "F must be 16-byte aligned");
  corrector_rhs(p, j0, nrhs, (double2*)F, S(stream));
  API_END
}

qp_status qp_pcg_solve(qp_plan* p, int nrhs, const void* F, void* U, const qp_solve_opts* opts, qp_solve_info* info,
                       void* stream) {
  API_BEGIN
  if (!p || !F || !U) raise(QP_ERR_INVALID_ARG, "plan, F and U must be non-null");
  if (nrhs < 1 || nrhs > p->max_rhs) raise(QP_ERR_INVALID_ARG, "nrhs must be 1..max_rhs");
  check_opts(opts, p);
  cudaStream_t s = S(stream);
  prepare_precond(p, opts->precond, s);
  const size_t bytes = (size_t)nrhs * p->D * sizeof(double2);
  CK(cudaMemcpyAsync(p->v64.F, F, bytes, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(p->v64.X, U, bytes, cudaMemcpyDeviceToDevice, s));
  if (!p->solver) p->solver = new Solver({p}, s);
  Units us = single_units(p, nrhs);
  SolveResult r;
  solve_units(p->solver, us, *opts, true, s, r);
  CK(cudaMemcpyAsync(U, p->v64.X, bytes, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  fill_info(r, 0, nrhs, info);
  qp_status w = worst(r);
  if (w != QP_OK) raise(w, "at least one right-hand side did not reach the tolerance");
  API_END
}

qp_status qp_homogenized_reduce(qp_plan* p, const void* U, double* Are, double* Aim, void* stream) {
  API_BEGIN
  if (!p || !U || !Are) raise(QP_ERR_INVALID_ARG, "plan, U and Astar_re must be non-null");
  if ((uintptr_t)U & 15u) raise(QP_ERR_INVALID_ARG, "U must be 16-byte aligned");
  astar_reduce(p, (const double2*)U, Are, Aim, S(stream));
  API_END
}

qp_status qp_homogenized(qp_plan* p, const qp_solve_opts* opts, double* Are, double* Aim, qp_solve_info* infos,
                         void* stream) {
  API_BEGIN
  if (!p || !Are) raise(QP_ERR_INVALID_ARG, "plan and Astar_re must be non-null");
  check_opts(opts, p);
  if (p->max_rhs < p->d) raise(QP_ERR_INVALID_ARG, "qp_homogenized needs a plan with max_rhs >= d");
  cudaStream_t s = S(stream);
  prepare_precond(p, opts->precond, s);
  corrector_rhs(p, 0, p->d, p->v64.F, s);
  if (!p->solver) p->solver = new Solver({p}, s);
  Units us = single_units(p, p->d);
  SolveResult r;
  solve_units(p->solver, us, *opts, false, s, r);
  astar_reduce(p, p->v64.X, Are, Aim, s);
  fill_info(r, 0, p->d, infos);
  qp_status w = worst(r);
  if (w != QP_OK) raise(w, "at least one corrector did not reach the tolerance");
  API_END
}

qp_status qp_fft(int n, const int* N, int count, void* data, int sign, int precision, void* stream) {
  API_BEGIN
  if (n < 1 || n > MAXN || !N || !data || count < 1) raise(QP_ERR_INVALID_ARG, "bad n, N, count or data");
  if (sign != 1 && sign != -1) raise(QP_ERR_INVALID_ARG, "sign must be +1 or -1");
  int64_t D = 1;
  for (int j = 0; j < n; ++j) {
    if (N[j] < 2 || N[j] > 1024 || !is_23(N[j])) raise(QP_ERR_INVALID_ARG, "N_j must be 2..1024, products of 2, 3");
    if (!fft_supported(N[j])) raise(QP_ERR_UNSUPPORTED, "FFT size " + std::to_string(N[j]) + " is not built");
    D *= N[j];
  }
  if (D * count > (int64_t(1) << 31)) raise(QP_ERR_INVALID_ARG, "too many elements");
  if (precision != QP_FP64 && precision != QP_FP32) raise(QP_ERR_INVALID_ARG, "bad precision");
  if ((uintptr_t)data & (precision == QP_FP64 ? 15u : 7u))
    raise(QP_ERR_INVALID_ARG, "data must be aligned to its complex element (16 bytes FP64, 8 bytes FP32)");
  fft_standalone(n, N, count, data, sign, precision, S(stream));
  CK_LAUNCH();
  API_END
}

qp_status qp_batch_create(int count, qp_plan* const* plans, qp_batch** out) {
  API_BEGIN
  if (!out || !plans || count < 1) raise(QP_ERR_INVALID_ARG, "bad batch arguments");
  *out = nullptr;
  std::unique_ptr<qp_batch> b(new qp_batch());
  int tot = 0;
  for (int i = 0; i < count; ++i) {
    if (!plans[i]) raise(QP_ERR_INVALID_ARG, "null plan in batch");
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) raise(QP_ERR_INVALID_ARG, "a plan appears twice in the batch");
    if (plans[i]->max_rhs < plans[i]->d) raise(QP_ERR_INVALID_ARG, "every plan needs max_rhs >= d");
    b->plans.push_back(plans[i]);
    tot += 2 * plans[i]->d * plans[i]->d;
  }
  b->solver = new Solver(b->plans, nullptr);
  b->small = (double*)dev_alloc(tot * sizeof(double), nullptr);
  b->small_bytes = tot * sizeof(double);
  b->h_small = (double*)pinned_alloc(b->small_bytes);
  // the taps plans' right-hand sides and a* reductions run as one launch each over all of them
  std::vector<PlanJob> jobs;
  int off = 0;
  for (qp_plan* p : b->plans) {
    if (p->backend == QP_BACKEND_TAPS) {
      jobs.push_back(PlanJob{p->pd, p->D, p->d, p->v64.F, p->v64.X, b->small + off});
      b->jobs_mc = std::max(b->jobs_mc, p->coef_count);
    }
    off += 2 * p->d * p->d;
  }
  b->njobs = (int)jobs.size();
  if (b->njobs) {
    b->jobs = (PlanJob*)dev_alloc(jobs.size() * sizeof(PlanJob), nullptr);
    CK(cudaMemcpy(b->jobs, jobs.data(), jobs.size() * sizeof(PlanJob), cudaMemcpyHostToDevice));
  }
  CK(cudaStreamSynchronize(nullptr));
  *out = b.release();
  API_END
}

qp_status qp_batch_homogenized(qp_batch* b, const qp_solve_opts* opts, double* Astar_all, qp_solve_info* infos,
                               void* stream) {
  API_BEGIN
  if (!b || !Astar_all) raise(QP_ERR_INVALID_ARG, "batch and Astar_all must be non-null");
  for (qp_plan* p : b->plans) check_opts(opts, p);
  cudaStream_t s = S(stream);
  for (qp_plan* p : b->plans) prepare_precond(p, opts->precond, s);
  Units us;
  us.plans = b->plans;
  for (qp_plan* p : b->plans) {
    us.nrhs.push_back(p->d);
    us.max_rhs = std::max(us.max_rhs, p->d);
    us.direct = us.direct || p->exec == QP_EXEC_DIRECT;
    us.run = std::min(us.run, last_axis_run(p));
    if (p->backend == QP_BACKEND_TAPS) {
      us.all_real = us.all_real && p->real_coef;
      us.max_coef = std::max(us.max_coef, p->coef_count);
    } else {
      corrector_rhs(p, 0, p->d, p->v64.F, s);
    }
  }
  if (b->njobs) {
    launch_rhs_taps_multi(b->jobs, b->njobs, b->jobs_mc, s);
    CK_LAUNCH();
  }
  SolveResult r;
  solve_units(b->solver, us, *opts, false, s, r);
  int off = 0;
  for (qp_plan* p : b->plans) {
    if (p->backend != QP_BACKEND_TAPS) astar_launch(p, p->v64.X, b->small + off, s);
    off += 2 * p->d * p->d;
  }
  if (b->njobs) {
    launch_astar_taps_multi(b->jobs, b->njobs, b->jobs_mc, s);
    CK_LAUNCH();
  }
  CK(cudaMemcpyAsync(b->h_small, b->small, off * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int q = 0, o2 = 0;
  size_t slot = 0;
  for (qp_plan* p : b->plans) {
    for (int i = 0; i < p->d * p->d; ++i) Astar_all[q++] = b->h_small[o2 + 2 * i];
    o2 += 2 * p->d * p->d;
    fill_info(r, slot, p->d, infos ? infos + slot : nullptr);
    slot += p->d;
  }
  qp_status w = worst(r);
  if (w != QP_OK) raise(w, "at least one corrector did not reach the tolerance");
  API_END
}

qp_status qp_batch_destroy(qp_batch* b) {
  API_BEGIN
  delete b;
  API_END
}

}  // extern "C"
