// Internal declarations shared by the CUDA translation units of libqp (not part of the C ABI).
#pragma once
#include <algorithm>

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qp.h"

namespace qp {

// Error carried from any translation unit to the C ABI boundary (converted to a qp_status there).
struct QpError {
  qp_status s;
  std::string msg;
};

[[noreturn]] inline void raise(qp_status s, const std::string& msg) { throw QpError{s, msg}; }

inline void ck(cudaError_t e, const char* what, int line) {
  if (e == cudaSuccess) return;
  const qp_status s = (e == cudaErrorMemoryAllocation) ? QP_ERR_OOM : QP_ERR_CUDA;
  raise(s, std::string(what) + " (line " + std::to_string(line) + "): " + cudaGetErrorString(e));
}
#define CK(call) ::qp::ck((call), #call, __LINE__)
#define CK_LAUNCH() ::qp::ck(cudaGetLastError(), "kernel launch", __LINE__)

// Number of kernels this library has launched in the process (read through qp_launch_count()). Kernels that
// run inside a CUDA graph are added by the host after each graph launch from the iteration counts.
void count_launch(int n = 1);

// Sets the text qp_last_error() returns on this host thread.
void set_last_error(const std::string& msg);

constexpr int MAXN = QP_MAX_N_AXES;
constexpr int MAXD = QP_MAX_D;
constexpr int MAXR = QP_MAX_RHS;
constexpr int MAXT = QP_MAX_TAPS;
constexpr int BLOCK = 256;           // threads per block of every elementwise / stencil kernel
constexpr int NQ = 4;                // reduction quantities per right-hand side
constexpr int NSLOT = MAXR * NQ;     // partial slots per chunk
// residual epilogue: plain, with the refinement bookkeeping, or with it and U = 0 (Q U not computed)
enum { REFINE_NONE = 0, REFINE_ON = 1, REFINE_ZERO_U = 2 };
// the persistent solve keeps consecutive reductions in disjoint slots: init [0,12), (h,w) [12,16),
// update [16,24), true residual [24,32)
constexpr int NSLOT_PERSIST = 2 * NSLOT;

template <typename T> struct V2;
template <> struct V2<double> { using type = double2; };
template <> struct V2<float> { using type = float2; };
template <typename T> using cplx = typename V2<T>::type;

// Division by a runtime divisor d <= 2^30 of dividends x < 2^31 without a hardware divide: with
// L = ceil(log2 d), p = 31 + L and m = ceil(2^p / d) (< 2^32), floor(x / d) = (x * m) >> p exactly
// (Granlund & Montgomery, "Division by invariant integers using multiplication", PLDI 1994).
struct FastDiv {
  uint32_t d;
  uint32_t m;
  uint32_t p;
};

// Modes per chunk of a unit (a chunk is reduced by one block), a function of D only, so that a unit reduces in the
// same order alone or batched:
//   D < 32,768: 256 (small units need the blocks: 1,024 modes took 0.51 ms with 256, 0.58 with 512);
//   32,768 <= D < 65,536: 512, so that the stencil's runs of two modes keep every thread of a block busy;
//   65,536 <= D < 622,592: one chunk per SM (152 chunks of 2 ceil(D / 304) modes), which evens the FP64 work of
//     the persistent solve over all SMs (cfg1: 1.12 ms with 256 chunks of 256, 0.98 with 128 of 512, 0.94 with
//     152 of 432; the batched cfg3: 24.5, 20.0, 17.9 ms);
//   D >= 622,592: about 8 chunks per SM, at most 65,536 modes, so that a large unit's chunked kernels run in about
//     one wave of resident blocks (16^6 modes: 1214 chunks of 13,824; a cap of 8192 gave 2048 chunks, 1.7 waves).
inline int64_t chunk_modes(int64_t D) {
  constexpr int64_t SMS = 152;
  if (D < 32768) return BLOCK;
  if (D < 65536) return 2 * BLOCK;
  if (D < SMS * 4096) return 2 * ((D + 2 * SMS - 1) / (2 * SMS));
  return std::max<int64_t>(2 * BLOCK, std::min<int64_t>(65536, (D / (SMS * 8) + BLOCK - 1) / BLOCK * BLOCK));
}

// Is the mean tap A~_0 of a coefficient positive definite? vals: its components as (re, im) pairs in the kind's
// layout (scalar: a; diagonal: a_11..a_dd; symmetric: the upper triangle row by row); the real parts form the d x d
// matrix, tested by a Cholesky factorisation.
inline bool mean_tap_spd(int kind, int d, const double* vals) {
  double M[MAXD][MAXD] = {};
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      int comp = -1;
      if (kind == QP_COEF_SCALAR) comp = (a == b) ? 0 : -1;
      else if (kind == QP_COEF_DIAG) comp = (a == b) ? a : -1;
      else {
        const int lo = a < b ? a : b, hi = a < b ? b : a;
        comp = lo * d - lo * (lo - 1) / 2 + (hi - lo);
      }
      M[a][b] = comp >= 0 ? vals[2 * comp] : 0.0;
    }
  double L[MAXD][MAXD] = {};
  for (int i = 0; i < d; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = M[i][j];
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      if (i == j) {
        if (!(s > 0.0)) return false;
        L[i][i] = __builtin_sqrt(s);
      } else {
        L[i][j] = s / L[j][j];
      }
    }
  return true;
}

inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t L = 0;
  while ((1ull << L) < d) ++L;
  const uint32_t p = 31 + L;
  const uint64_t m = ((1ull << p) + d - 1) / d;
  return FastDiv{d, (uint32_t)m, p};
}

// Everything the star-1 stencil reads besides the vectors: the geometry, P, and the coefficients of the mean
// tap and of the taps m = +e_j, m = -e_j of every axis, at fixed offsets. A kernel that serves one plan takes it
// by value as a kernel parameter (read from the constant bank, so that the stencil's only L1 traffic is the
// vectors); a kernel over several plans reads the plan's device copy.
struct alignas(16) StarParams {
  double2 c64[MAXN][2][MAXD];   // [axis j][0: m = +e_j, 1: m = -e_j][component]
  double2 c064[MAXD];           // the mean tap
  double P64[MAXD][MAXN];
  float2 c32[MAXN][2][MAXD];
  float2 c032[MAXD];
  float P32[MAXD][MAXN];
  FastDiv div[MAXN];
  int N[MAXN], stride[MAXN];
  int woff[MAXN];               // (N_j - 1) stride_j
  int half[MAXN];               // ceil(N_j / 2)
  int has[MAXN];                // 1: the axis has the taps m = +-e_j
  int n, d;
  int wreal, pad_;              // 1: w64 holds real weights (8 bytes each; real tap values), else complex (16 bytes)
  const void* w64;              // the plan's stored FP64 weights (see star_slots), or null
  const void* pad_ptr_;
  // FP32 form of the taps as Hermitian pairs (the tap -e_j of a real coefficient holds the conjugate of the tap
  // +e_j): per axis j and component a < d of the lambda products, the tap +e_j's coefficient (a scalar coefficient
  // repeats it for every a) and that coefficient times P_aj; the mean tap's (real) coefficient per a
  float2 hc32[MAXN][MAXD];
  float2 hcp32[MAXN][MAXD];
  float c0r32[MAXD];
  int pad2_;
  // storage (PlanDev.Nst, nyq, hspec, Hl)
  int Nst[MAXN];
  int nyq[MAXN];
  int hspec, Hl, pad3_, pad4_;
};
static_assert(sizeof(StarParams) % 16 == 0, "StarParams is uploaded and passed as 16-byte words");

// Device description of one plan's geometry and (for the taps backend) its taps, sorted as
// [mean tap][star taps of axis 0] .. [star taps of axis n-1][taps with several nonzero axes].
struct alignas(16) PlanDev {
  int n, d, D, kind;
  int ncomp, ntaps, real_coef, backend;
  int N[MAXN];
  int stride[MAXN];
  FastDiv div[MAXN];
  int star_begin[MAXN + 1];   // star taps of axis j: [star_begin[j], star_begin[j+1]); multi-axis: [star_begin[n], ntaps)
  double P[MAXD][MAXN];
  float P32[MAXD][MAXN];
  const double2* coef64;      // [ntaps][ncomp], sorted order
  const float2* coef32;
  // star-1 form (star1 != 0): a scalar or diagonal coefficient with taps only at m = 0 and m = +-e_j, every
  // axis with taps of length >= 2; its stencil data in "star" (device)
  int star1, pad_star;
  const StarParams* star;
  signed char m[MAXT][MAXN];  // sorted tap modes
  // storage: Nst[j] entries along axis j (N[j], except ceil(N_{n-1} / 2) for the last axis of a half-spectrum plan,
  // which stores k_{n-1} = 0 .. Hl - 1 at index k_{n-1}); nyq[j]: the storage index of the dropped Nyquist mode
  // k_j = -N_j/2 of a half-spectrum plan (N_j even, j < n - 1), else -1
  int Nst[MAXN];
  int nyq[MAXN];
  int hspec, Hl, pad_h0, pad_h1;   // hspec: half-spectrum storage (QP_SPECTRUM_HALF); Hl = ceil(N_{n-1} / 2)
  // the stored FP64 stiffness entries of a plan with general taps, [tap (sorted)][D] (real: double, else double2),
  // which FP64 applies read instead of forming the weights; null if not stored
  const void* wgen;
  int wgen_real, pad_w0, pad_w1, pad_w2;
};
static_assert(sizeof(PlanDev) % 16 == 0, "PlanDev is copied to shared memory in 16-byte words");

// Sets PlanDev.star1 from the sorted taps (m, star_begin, N, stride, kind, backend must be set) and, for a
// star-1 plan, fills sp from the geometry and the sorted tap values c64 / c32 ([ntaps][ncomp]).
inline void make_star(PlanDev& pd, const double2* c64, const float2* c32, StarParams& sp) {
  pd.star1 = 0;
  sp = StarParams{};
  if (pd.backend != QP_BACKEND_TAPS || pd.star_begin[pd.n] != pd.ntaps) return;   // multi-axis taps
  if (pd.kind != QP_COEF_SCALAR && pd.kind != QP_COEF_DIAG) return;
  const int nc = pd.ncomp;
  for (int j = 0; j < pd.n; ++j) {
    int tp = -1, tm = -1;
    for (int t = pd.star_begin[j]; t < pd.star_begin[j + 1]; ++t) {
      if (pd.m[t][j] == 1 && tp < 0) tp = t;
      else if (pd.m[t][j] == -1 && tm < 0) tm = t;
      else return;                                   // |m_j| > 1 or a repeated mode
    }
    if ((tp < 0) != (tm < 0)) return;
    if (tp >= 0 && pd.N[j] < 2) return;
    sp.has[j] = tp >= 0 ? 1 : 0;
    for (int q = 0; q < nc && tp >= 0; ++q) {
      sp.c64[j][0][q] = c64[tp * nc + q];
      sp.c64[j][1][q] = c64[tm * nc + q];
      sp.c32[j][0][q] = c32[tp * nc + q];
      sp.c32[j][1][q] = c32[tm * nc + q];
    }
  }
  for (int q = 0; q < nc; ++q) {
    sp.c064[q] = c64[q];
    sp.c032[q] = c32[q];
  }
  for (int a = 0; a < pd.d; ++a) {
    const int q = pd.kind == QP_COEF_DIAG ? a : 0;
    sp.c0r32[a] = (float)c64[q].x;
    for (int j = 0; j < pd.n; ++j) {
      const double2 c = sp.c64[j][0][q];
      sp.hc32[j][a] = make_float2((float)c.x, (float)c.y);
      sp.hcp32[j][a] = make_float2((float)(c.x * pd.P[a][j]), (float)(c.y * pd.P[a][j]));
    }
  }
  for (int j = 0; j < MAXN; ++j) {
    sp.N[j] = pd.N[j];
    sp.stride[j] = pd.stride[j];
    sp.div[j] = pd.div[j];
    sp.woff[j] = (pd.N[j] - 1) * pd.stride[j];
    sp.half[j] = (pd.N[j] + 1) / 2;
    for (int a = 0; a < MAXD; ++a) {
      sp.P64[a][j] = pd.P[a][j];
      sp.P32[a][j] = pd.P32[a][j];
    }
  }
  sp.n = pd.n;
  sp.d = pd.d;
  for (int j = 0; j < MAXN; ++j) {
    sp.Nst[j] = pd.Nst[j];
    sp.nyq[j] = pd.nyq[j];
  }
  sp.hspec = pd.hspec;
  sp.Hl = pd.Hl;
  pd.star1 = 1;
}

// One solve unit: a plan and its nrhs right-hand sides (contiguous nrhs x D vectors).
struct UnitDev {
  const PlanDev* plan;
  int D, nrhs, chunk0, nchunk;
  int chunk;           // modes per chunk: a function of D only, so a unit reduces in the same order alone or batched
  int run;             // stencil run along the last axis: 2 when its length is even, else 1
  int fft;             // 1: FFT-backend unit (its applies write w in FFT passes; the batch kernels add only the
                       // epilogue and need no plan in shared memory)
  int hspec;           // 1: half-spectrum storage; a mode with k_{n-1} > 0 stands for itself and its mirror, so
                       // it weighs 2 in every inner product (its storage index e has e mod Hl != 0)
  int Hl, pad_u0;
  FastDiv hdiv;        // division by Hl
  const double2* F;   // right-hand side (FP64)
  double2* U;         // solution (FP64)
  double2* r;         // FP64 PCG residual
  double2* h;         // FP64 PCG direction
  double2* w;         // FP64 Q h, or the FP64 true residual F - Q U
  float2* F32;        // refinement: scaled FP32 right-hand side
  float2* U32;        // refinement: FP32 correction
  float2* r32;
  float2* h32;
  float2* w32;
  const double* minv64;   // diagonal preconditioner M (z = M r)
  const float* minv32;
};

// Per right-hand-side state (device).
struct RhsSt {
  double f2, rz, hw, rr, beta, alpha;     // PCG level (alpha = rz / hw, set once per iteration)
  double of2, orr, scale, prev_rel;       // refinement outer level (FP64 true residual)
  double inv_scale, pad0;                 // ||F - Q U|| of the last outer step (1 / scale)
  int iters, done, status, inner_total;
  int outer, odone, ostatus, upend;       // upend: converged in this iteration, its U += alpha h still to come
};

struct BatchDev {
  int nunits, nchunks, nslots, hspec_any;   // hspec_any: some unit has half-spectrum storage
  int single, apply_down, pad_[2];      // single: one unit, whose description is "pu" (kernel parameter);
                                        // apply_down: the batch's apply walks its chunks downwards (general kernel)
  UnitDev pu;
  const UnitDev* units;
  RhsSt* st;                            // [nunits * MAXR]
  const int* chunk_unit;                // [nchunks]
  double* partials;                     // [NSLOT][nchunks] ([NSLOT_PERSIST][nchunks] for the persistent solve)
  unsigned* ucount;                     // [nunits] chunk arrivals per unit
  unsigned* kcount;                     // [1] units finalized by the current kernel
  int* ndone;                           // [2]: right-hand sides done at the PCG level, at the outer level
  double tol2, otol2;                   // PCG-level and outer (refinement) tolerances, squared
  int maxit, max_outer;
};

enum { EPI_DOT_HW = 0, EPI_RESIDUAL = 1, EPI_NONE = 2 };
enum { LEVEL_FP64 = 0, LEVEL_FP32 = 1 };   // which vector set a PCG kernel works on

// ---- taps backend kernels (qp_taps.cu)
// Apply over every chunk of the batch (taps units only; FFT units get their w from the FFT passes and only
// the epilogue here). level LEVEL_FP64: EPI_DOT_HW reads h and writes w; EPI_RESIDUAL reads U and writes
// w = F - Q U; LEVEL_FP32: EPI_DOT_HW reads h32 and writes w32. refine: EPI_RESIDUAL runs the outer
// (refinement) bookkeeping. cond (0 = none): the graph conditional of the loop this apply belongs to; it is
// set to 0 by the call that completes the count of finished right-hand sides.
// realc: every taps plan in the batch has real tap values; mc: largest ntaps * ncomp over its taps plans.
// maxr: the largest nrhs of the batch's units. st1: for a batch of one star-1 unit with an even last axis, its
// StarParams (host memory, passed by value), else null; kind: that unit's coefficient kind.
void launch_apply(const BatchDev& b, bool realc, int mc, int maxr, int level, int epi, int refine,
                  unsigned long long cond, int nblk, const StarParams* st1, int kind, cudaStream_t s);
// Standalone apply of one plan: w = Q h for nrhs vectors (no reductions); st1, kind as launch_apply.
template <typename T>
void launch_apply_plain(const PlanDev* plan_dev, bool realc, int mc, int D, int nrhs, const cplx<T>* h, cplx<T>* w,
                        int run, const StarParams* st1, int kind, cudaStream_t s);
// Writes a general-taps plan's FP64 weights per (sorted tap, mode) to out: [ntaps][D] complex (double when realc);
// run: the plan's stencil run (2 for an even stored last axis, else 1).
void launch_gen_weights(const PlanDev* plan_dev, bool realc, int mc, int D, int run, void* out, cudaStream_t s);
// Writes a star-1 plan's FP64 weights per (tap slot, mode) to out: [1 + 2n][D] complex (double when realc).
void launch_star_weights(const StarParams& st, bool realc, int kind, int D, void* out, cudaStream_t s);
// with_frob: also the Frobenius-optimal diagonal (else frob / frob32 are not written).
void launch_diag(const PlanDev* plan_dev, int mc, int D, double* jac, double* frob, float* jac32, float* frob32,
                 double* partials, unsigned* counter, double* out, int nblk, bool with_frob, cudaStream_t s);
void launch_rhs_taps(const PlanDev* plan_dev, int mc, int j0, int nrhs, int D, double2* F, cudaStream_t s);
void launch_astar_taps(const PlanDev* plan_dev, int mc, int D, const double2* U, double* out, cudaStream_t s);
// One taps plan's part of a batch's corrector right-hand sides and a* reduction (one block each).
struct PlanJob {
  const PlanDev* plan;
  int D, nrhs;
  double2* F;          // its right-hand sides (zeroed beforehand)
  const double2* U;    // its corrector solutions
  double* out;         // its a*: 2 d^2 doubles
};
void launch_rhs_taps_multi(const PlanJob* jobs, int njobs, int mc, cudaStream_t s);
void launch_astar_taps_multi(const PlanJob* jobs, int njobs, int mc, cudaStream_t s);

// ---- PCG kernels (qp_pcg.cu)
void launch_level_reset(const BatchDev& b, int which, cudaStream_t s);
// maxr: the largest nrhs of the batch's units (selects the kernel instantiation).
void launch_pcg_init(const BatchDev& b, int maxr, int level, bool warm, unsigned long long cond, int nblk,
                     cudaStream_t s);
void launch_pcg_update(const BatchDev& b, int maxr, int level, unsigned long long cond, int nblk, cudaStream_t s);
void launch_pcg_hupdate(const BatchDev& b, int maxr, int level, int nblk, cudaStream_t s);
void launch_refine_prep(const BatchDev& b, int nblk, cudaStream_t s);
void launch_refine_accum(const BatchDev& b, int nblk, cudaStream_t s);
// Library memory (qp_mem.cu): device blocks from a stream-ordered pool that keeps freed blocks cached (dev_free
// must come after the device work using the block has completed), page-locked host blocks from a size-class cache.
void* dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void* p);
void dev_trim();
void set_cache_bytes(int64_t bytes);   // < 0: the default (an eighth of the device memory, at least 1 GiB)
void pool_stats(int64_t* reserved, int64_t* used, uint64_t* allocs);
void* pinned_alloc(size_t bytes);
void pinned_free(void* p, size_t bytes);

// ||U_r - Uref_r||_2 over the Fourier coefficients (qp_norms.cu)
void launch_l2_norms(int D, int nrhs, const double2* U, const double2* Uref, double* part, int nblk, double* out,
                     int hl, cudaStream_t s);

// persistent solve of one taps unit (qp_persistent.cu): the kernel's argument
struct PersistArgs {
  BatchDev b;          // b.single: one unit in b.pu, its state in b.st[0 .. MAXR)
  unsigned* bar;       // [0] arrivals, [1] generation (zeroed before the launch)
  int* err;            // set on a barrier timeout (zeroed before the launch)
  int mode;            // QP_MODE_FP64 or QP_MODE_FP32_REFINE
  int warm;            // start from the U held in the plan (else U = 0)
  unsigned long long timeout_ns;
  StarParams star;     // the unit's star-1 stencil data (kernels with sk != 0)
};
size_t persistent_smem(int coef_count);
// sk: 0 the plan's stencil from shared memory; 1 / 2 a star-1 plan with a scalar / diagonal coefficient and
// stored FP64 weights (its StarParams st passed by value).
// A star-1 plan of one of the fixed geometries compiled in: (n, d) = (6, 3), (4, 2), (2, 1), taps on every axis,
// nr = d right-hand sides; n gets the number of axes.
inline bool fixed_geometry(const StarParams& st, int nr, int& n) {
  n = st.n;
  if (!((n == 6 && st.d == 3) || (n == 4 && st.d == 2) || (n == 2 && st.d == 1)) || nr != st.d) return false;
  for (int j = 0; j < n; ++j)
    if (!st.has[j]) return false;
  return true;
}

int persistent_capacity(bool realc, int nr, int sk, const StarParams* st, size_t smem);
void launch_persistent(const BatchDev& b, bool realc, int nr, int sk, const StarParams* st, int mode, bool warm,
                       unsigned* bar, int* err, double timeout_s, int grid, size_t smem, cudaStream_t s);

}  // namespace qp
