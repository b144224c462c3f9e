/*
 * qp.h - C ABI of the GB300 (sm_103a) projection-method solver for quasiperiodic elliptic problems and
 * quasiperiodic homogenization (Jiang, Li, Zhang & Zhang, arXiv 2404.06841).
 *
 * A d-dimensional quasiperiodic coefficient A(x) = A(P^T x) is lifted to its parent function on the torus
 * T^n (Sec. 2.1). On N_1 x .. x N_n Fourier modes k (storage index k mod N_j per axis, C order, last axis
 * fastest: Sec. 3.1.2, eq. conversion) the discrete scheme (Sec. 3.1.1, eq. n-discrete_equation, and App. D
 * for a matrix coefficient) is the linear system Q U = F with
 *
 *     (Q U)(k) = sum_ab lambda_a(k) sum_k' A~^{ab}_{k -N k'} lambda_b(k') U(k'),   lambda(k) = P k,
 *
 * which the library solves by preconditioned CG (Sec. 4.3, Algorithm 2) and turns into the homogenized
 * coefficient A*_ij = M{ e_i^T A (e_j + grad u_j) } (Sec. 5.2, eq. homcoefficient).
 *
 * Conventions shared by every entry point:
 *  - Complex vectors are interleaved (re, im): complex128 for QP_FP64, complex64 for QP_FP32. A set of
 *    nrhs vectors is nrhs x D contiguous (vector r starts at element r*D). D = N_1 * .. * N_n.
 *  - Pointers named "device" must be device memory of the current CUDA device (for example torch tensors);
 *    pointers named "host" are ordinary host memory. The caller owns every pointer it passes.
 *  - "stream" is a cudaStream_t (NULL = legacy default stream). Every call is asynchronous on that stream
 *    unless it writes a host output (info, Astar), in which case it synchronises the stream before returning.
 *  - The mode k = 0 is not an unknown (Sec. 3.1.1: the test space has zero mean): entry k = 0 of a
 *    right-hand side is ignored and entry k = 0 of a solution is returned as 0. Row k = 0 of Q U is 0.
 *  - Errors: no exception crosses the ABI. A non-zero qp_status is returned, qp_last_error() describes it
 *    (per host thread), and outputs are unspecified. Arguments are validated before any device work.
 */
#ifndef QP_H
#define QP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QP_OK = 0,
  QP_ERR_INVALID_ARG = 1,     /* bad d, n, N, pointer, tap list, option */
  QP_ERR_SINGULAR_P = 2,      /* some k != 0 of K_N^n has |P k| below 1e-12 |P|: P is not a projection */
  QP_ERR_NOT_ELLIPTIC = 3,    /* the coefficient's mean (Jacobi diagonal) is not positive */
  QP_ERR_BREAKDOWN = 4,       /* PCG met (h, Q h) <= 0 or a NaN */
  QP_ERR_NO_CONVERGENCE = 5,  /* maxit reached before the tolerance */
  QP_ERR_TIMEOUT = 6,         /* a bounded device wait gave up */
  QP_ERR_UNSUPPORTED = 7,     /* valid request that the library does not implement */
  QP_ERR_OOM = 8,             /* device allocation failed */
  QP_ERR_CUDA = 9             /* any other CUDA runtime error */
} qp_status;

enum { QP_COEF_SCALAR = 0, QP_COEF_DIAG = 1, QP_COEF_SYM = 2 };
enum { QP_REPR_TAPS = 0, QP_REPR_GRID = 1 };
enum { QP_BACKEND_AUTO = 0, QP_BACKEND_TAPS = 1, QP_BACKEND_FFT = 2 };
enum { QP_FP64 = 0, QP_FP32 = 1 };
enum { QP_PRECOND_JACOBI = 0, QP_PRECOND_FROBENIUS = 1 };
enum { QP_MODE_FP64 = 0, QP_MODE_FP32_REFINE = 1 };
enum { QP_EXEC_AUTO = 0, QP_EXEC_DIRECT = 1, QP_EXEC_GRAPH = 2, QP_EXEC_PERSISTENT = 3 };
enum { QP_SPECTRUM_FULL = 0, QP_SPECTRUM_HALF = 1 };
enum { QP_MAX_N_AXES = 6, QP_MAX_D = 3, QP_MAX_RHS = 4, QP_MAX_TAPS = 256 };

typedef struct qp_plan qp_plan;     /* opaque; owns every internal device buffer */
typedef struct qp_batch qp_batch;   /* opaque; a set of plans solved together */

/* The coefficient A(theta): real, d x d symmetric, uniformly elliptic (Sec. 2.2).
 * kind: QP_COEF_SCALAR (A = a I, 1 component), QP_COEF_DIAG (d components a_11..a_dd),
 *       QP_COEF_SYM (d(d+1)/2 components: the upper triangle row by row, 11, 12, .., 1d, 22, .., dd).
 * repr: QP_REPR_TAPS - Fourier modes (taps): tap_k host int32 [ntaps x n], every |m_j| < N_j / 2 and <= 127;
 *       tap_val host double [ntaps x ncomp x 2] (re, im) with A~_{-m} = conj(A~_m) (so A is real).
 *       Values are the Fourier coefficients of Sec. 3.1.1; a mode listed twice is summed.
 *       QP_REPR_GRID - samples A(y_j) at y_j = 2 pi j / N: grid is DEVICE double [ncomp x D], C order, 8-byte
 *       aligned (else QP_ERR_INVALID_ARG); the plan copies it. Its Fourier coefficients are taken by the DFT with 1/D (Sec. 3.1.1). */
typedef struct {
  int kind;
  int repr;
  int ntaps;
  const int32_t* tap_k;
  const double* tap_val;
  const double* grid;
} qp_coeff;

typedef struct {
  int backend;      /* QP_BACKEND_*: AUTO takes FFT for a grid coefficient; for a tap coefficient the TAPS stencil,
                       except that a dense tap list (>= 64 taps) on >= 65,536 modes that the FFT backend can
                       transform has both backends' FP32 applies timed once per shape and keeps the faster */
  int max_rhs;      /* right-hand sides solved together, 1..QP_MAX_RHS; 0 = d */
  int precisions;   /* workspace: bit 0 = FP64 solve, bit 1 = FP32 (refinement inner) solve; 0 = both */
  int exec;         /* how a solve is driven (the iterates are bitwise the same in every mode):
                       QP_EXEC_GRAPH: one CUDA-graph launch whose loops are conditional WHILE nodes (three kernels
                       per PCG iteration); QP_EXEC_PERSISTENT: one cooperative launch of a persistent kernel that
                       meets at grid barriers (taps backend, single-plan solves, even last-axis length; others use
                       the graph); QP_EXEC_DIRECT: the graph's kernels launched one by one, the host polling
                       convergence (for profilers and callers that cannot launch graphs); QP_EXEC_AUTO (0,
                       default): PERSISTENT where it applies and every chunk of modes gets its own resident block,
                       else GRAPH. A persistent solve whose barrier wait exceeds its limit returns QP_ERR_TIMEOUT. */
  int spectrum;     /* QP_SPECTRUM_FULL (0, default): the scheme on K_N^n as written (Sec. 2.3, 3.1.1), complex vectors
                       of D = N_1 .. N_n entries. QP_SPECTRUM_HALF (not in the paper; opt-in): the scheme restricted to
                       the Nyquist-free modes K'_N = {k : |k_j| < N_j / 2} (for an even N_j the mode k_j = -N_j/2 is
                       dropped; for odd N_j nothing is), a set closed under k -> -k on which the solution of a real
                       problem satisfies U(-k) = conj(U(k)); vectors then store only the modes with k_n >= 0:
                       D_h = N_1 .. N_{n-1} x ceil(N_n / 2) entries, the last axis holding k_n = 0 .. ceil(N_n/2) - 1
                       at index k_n, the others in the usual storage order (index k_j mod N_j). A mode with k_n < 0
                       is the conjugate of its mirror -k; entries at a dropped mode (some k_j = -N_j/2, j < n) are
                       ignored on input and 0 on output; the k_n = 0 plane holds both k and -k, which a real
                       problem keeps conjugate (inputs should). About half the bytes per PCG iteration; the discrete
                       result differs from the full scheme's by the Nyquist modes' share (a* is larger or equal:
                       a smaller trial space). Taps backend with a tap coefficient, Jacobi preconditioner;
                       solves run as CUDA graphs (not persistent). qp_plan_query reports the stored length. */
} qp_options;

typedef struct {
  double tol;         /* stop when ||F - Q U||_2 <= tol ||F||_2 (Fourier coefficients; Parseval) */
  int maxit;          /* PCG iteration cap (all inner iterations in refinement mode) */
  int precond;        /* QP_PRECOND_JACOBI (diagonal of Q) or QP_PRECOND_FROBENIUS (eq. preconditioner; built on
                         first use, see qp_plan_diagonal) */
  int mode;           /* QP_MODE_FP64: FP64 vectors and operator; QP_MODE_FP32_REFINE: FP32 inner PCG in an
                         FP64 iterative-refinement loop (FP64 true residual, FP64 dot products) */
  double inner_tol;   /* refinement: relative tolerance of each inner FP32 solve (0 = 1e-5) */
  int max_outer;      /* refinement: outer-iteration cap (0 = 12) */
} qp_solve_opts;

typedef struct {
  int status;            /* qp_status of this right-hand side */
  int iterations;        /* PCG iterations (FP64 mode) or inner FP32 iterations (refinement) */
  int outer_iterations;  /* FP64 true-residual evaluations in refinement mode (0 in FP64 mode) */
  double rel_residual;   /* ||F - Q U||_2 / ||F||_2 recomputed in FP64 at exit (0 for F = 0) */
} qp_solve_info;

typedef struct {
  int64_t D;             /* N_1 * .. * N_n */
  int backend;           /* QP_BACKEND_TAPS or QP_BACKEND_FFT, as chosen */
  int ntaps;             /* distinct Fourier modes of the coefficient (taps backend) */
  int max_rhs;
  double min_abs_lambda; /* min over k != 0 of |P k| */
  int64_t device_bytes;  /* device memory the plan holds */
  int star;              /* 1: taps only at m = 0 and m = +-e_j with a scalar or diagonal coefficient (the star-1
                            stencil of the taps backend) */
  int stored_weights;    /* 1: the plan stores the FP64 stiffness entries Q_ij per (tap, mode) (Sec. 4.2's
                            compressed format Q~), which single-plan FP64 applies read instead of forming */
  int spectrum;          /* QP_SPECTRUM_FULL or QP_SPECTRUM_HALF */
  int64_t stored;        /* entries of each vector the plan's calls take: D, or D_h for QP_SPECTRUM_HALF */
} qp_plan_info;

/* Creates a plan: validates d (1..3), n (d..6), P (host double d x n, row-major, Sec. 2.1 projection
 * matrix), N (host int[n], 2..1024 each, products of 2 and 3 for the FFT backend), the coefficient, and builds
 * the per-axis lambda tables, the coefficient representation, the Jacobi diagonal (Sec. 4.3; the Frobenius-optimal
 * one, eq. preconditioner, is built on first use), for a star-1 taps plan its stored FP64 entries Q_ij (see
 * qp_plan_info), and for the FFT backend its autotuned apply schedule. Work runs on "stream"; the call
 * synchronises it. */
qp_status qp_plan_create(int d, int n, const double* P, const int* N, const qp_coeff* coeff,
                         const qp_options* opt, void* stream, qp_plan** out);
/* Waits for all work on the device (no stream may still use the plan), then returns the plan's device memory to
 * the library's pool (blocks are kept cached for the next plans up to the cache size of qp_set_memory_cache, by
 * default an eighth of the device's memory and at least 1 GiB; the rest goes back to the device). */
qp_status qp_plan_destroy(qp_plan* plan);
qp_status qp_plan_query(const qp_plan* plan, qp_plan_info* info);

/* QU = Q U (eq. n-discrete_equation; compressed mat-vec of Sec. 4.2 on the taps backend, or gradient ->
 * inverse n-dim DFT -> pointwise A(y) -> forward DFT -> divergence on the FFT backend).
 * U, QU: device, nrhs x D complex (complex128 for QP_FP64, complex64 for QP_FP32), each 16-byte aligned (the
 * kernels move two complex64 values per access); must not overlap. A misaligned pointer gives QP_ERR_INVALID_ARG. */
qp_status qp_apply_stiffness(qp_plan* plan, int nrhs, const void* U, void* QU, int precision, void* stream);

/* F = the corrector right-hand sides F_j(k) = i sum_a lambda_a(k) A~^{aj}_k, F_j(0) = 0, for
 * j = j0 .. j0+nrhs-1 (0-based; Sec. 5.2 eq. corrector, App. D f_1 = d alpha/dx_1). F: device complex128
 * nrhs x D, 16-byte aligned (a misaligned pointer gives QP_ERR_INVALID_ARG). */
qp_status qp_corrector_rhs(qp_plan* plan, int j0, int nrhs, void* F, void* stream);

/* Solves Q U = F for nrhs right-hand sides with PCG (Algorithm 2, z = M r). F: device complex128 nrhs x D.
 * U: device complex128 nrhs x D, in: initial guess (warm start), out: solution. info: host, nrhs entries.
 * Returns QP_OK only if every right-hand side met opts->tol; otherwise the worst status. */
qp_status qp_pcg_solve(qp_plan* plan, int nrhs, const void* F, void* U, const qp_solve_opts* opts,
                       qp_solve_info* info, void* stream);

/* Astar = the torus average A*_ij = A~^{ij}_0 + i sum_k sum_b A~^{ib}_{-k} lambda_b(k) U_j(k)
 * (eq. homcoefficient written in Fourier terms) from the d corrector solutions U (device complex128 d x D,
 * 16-byte aligned; a misaligned pointer gives QP_ERR_INVALID_ARG). Astar_re, Astar_im: host double d x d row-major (Astar_im may be NULL). FP64 throughout. */
qp_status qp_homogenized_reduce(qp_plan* plan, const void* U, double* Astar_re, double* Astar_im, void* stream);

/* The whole homogenization: the d corrector right-hand sides, their PCG solves (FP64 or FP32 + FP64
 * refinement per opts->mode), and the reduction above. Astar_re/Astar_im: host d x d; infos: host, d entries. */
qp_status qp_homogenized(qp_plan* plan, const qp_solve_opts* opts, double* Astar_re, double* Astar_im,
                         qp_solve_info* infos, void* stream);

/* Unnormalised in-place n-dimensional complex DFT of "count" contiguous arrays of shape N[0..n-1]:
 * X(k) = sum_j x(j) exp(sign * 2 pi i k.j / N), sign = -1 (forward) or +1 (inverse, without 1/D).
 * data: device complex128 (QP_FP64) or complex64 (QP_FP32), aligned to its element (16 or 8 bytes; else
 * QP_ERR_INVALID_ARG). N_j products of 2 and 3, 2..1024. */
qp_status qp_fft(int n, const int* N, int count, void* data, int sign, int precision, void* stream);

/* Batched homogenization: every corrector of every plan is solved in the same launches (one unit per
 * (plan, corrector)); plans may differ in d, n, N and coefficient. Astar_all: host, sum over plans of d*d
 * doubles (plan order, row-major each); infos: host, one per unit in plan order. */
qp_status qp_batch_create(int count, qp_plan* const* plans, qp_batch** out);
qp_status qp_batch_homogenized(qp_batch* batch, const qp_solve_opts* opts, double* Astar_all,
                               qp_solve_info* infos, void* stream);
qp_status qp_batch_destroy(qp_batch* batch);

/* Size in bytes of the device scratch that qp_pcg_solve_taps_static works in. */
#define QP_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)

/* FP64 PCG solve of Q U = F for a tap coefficient without a plan and without allocating device memory; the
 * paper has no counterpart (it concerns how a caller provides GPU memory, not the method). For callers that
 * cannot call cudaMalloc, for example because another component owns the device-memory budget. All of its
 * intermediates (coefficient tables, the diagonal preconditioner, the PCG vectors r, h, Q h, reduction
 * partials and solver state) live in one static device array of QP_STATIC_SCRATCH_BYTES that every GPU that
 * loads this library holds until the process exits; it never calls cudaMalloc, cudaFree or an allocating
 * library routine. Arguments as qp_plan_create (d, n, P, N, coeff; taps only) and qp_pcg_solve (nrhs, F, U
 * with U as the initial guess, opts with mode QP_MODE_FP64, info). Needs about (24 + 48 nrhs) D bytes plus
 * the tap tables; larger problems return QP_ERR_INVALID_ARG ("too large for the static scratch") before any
 * device work. It checks its inputs as qp_plan_create does (QP_ERR_NOT_ELLIPTIC for a mean tap that is not positive
 * definite) and, like qp_pcg_solve, solves again from the current U (at most twice) a right-hand side whose true
 * residual misses the tolerance after its recursive residual met it. The first call on a device looks up the array's device address (cudaGetSymbolAddress), so
 * make that first call before any stream capture. All calls share the one array: calls whose GPU work
 * overlaps (other streams or threads) race and give wrong results; serialise them. Each call clears what
 * must start at zero, so a call never depends on what the previous call left there. Synchronises stream. */
qp_status qp_pcg_solve_taps_static(int d, int n, const double* P, const int* N, const qp_coeff* coeff, int nrhs,
                                   const void* F, void* U, const qp_solve_opts* opts, qp_solve_info* info,
                                   void* stream);

/* The diagonal preconditioner of a solve, z = M r (Sec. 4.3): QP_PRECOND_JACOBI gives M(k) = 1/q(k), q the diagonal
 * of Q; QP_PRECOND_FROBENIUS gives the Frobenius-optimal M(k) = q(k)/||Q e_k||^2 (eq. preconditioner): on the taps
 * backend from the O(gD) column sums, on the FFT backend from FFT cross-correlations of lambda_a lambda_a' with
 * A~^{ab} conj(A~^{a'b'}) (d^4 + d(d+1) FP64 n-dim DFTs plus ~(5 + d(d+1)/2) x 16 B x D of temporary device memory);
 * on either backend done once, on this call or the first Frobenius solve. M(0) = 0 (the excluded mode). out: device
 * double[stored length] (D; D_h for a QP_SPECTRUM_HALF plan, which has the Jacobi diagonal only, 0 at dropped modes).
 * Synchronises stream. */
qp_status qp_plan_diagonal(qp_plan* plan, int precond, double* out, void* stream);

/* Error of a computed solution in the L^2_QP norm (Sec. 5.1, e_N = ||u_N - u||): by the Parseval identity of that
 * norm (Sec. 2.2, eq. parseval) it is the l^2 norm of the Fourier coefficients, out[r] = ||U_r - Uref_r||_2 over
 * K_N^n. U, Uref: device complex128, nrhs x D, 16-byte aligned (1 <= nrhs <= QP_MAX_RHS; Uref NULL gives ||U_r||). out: host
 * double[nrhs]. When Uref holds the exact solution's coefficients on K_N^n, modes of the exact solution outside
 * K_N^n (truncation) add the sum of their |coefficient|^2 to out[r]^2; the caller adds that part. Deterministic
 * FP64 reduction; synchronises stream. */
qp_status qp_l2qp_error(qp_plan* plan, int nrhs, const void* U, const void* Uref, double* out, void* stream);

/* The library's device-memory pool on the current device (plans, solvers and batches take their buffers from it):
 * reserved_bytes = memory the pool holds from the device, used_bytes = memory in live buffers, allocations = pool
 * allocations served so far in this process (all devices). Any output may be NULL. */
qp_status qp_memory_pool_stats(int64_t* reserved_bytes, int64_t* used_bytes, uint64_t* allocations);

/* Freed pool memory kept cached for later plans when a plan or batch is destroyed (process-wide): bytes >= 0 keeps
 * at most that much (0 returns every freed block to the device at once); bytes < 0 restores the default, an eighth
 * of the device's memory and at least 1 GiB. The pool is trimmed to the new size at once. */
qp_status qp_set_memory_cache(int64_t bytes);

/* Phase timing of solves, for profiling (not in the paper). While it is enabled, qp_pcg_solve, qp_homogenized and
 * qp_batch_homogenized run in the host-driven form (the kernels of the graph form, launched one PCG iteration at a
 * time and with no launch after convergence; the iterates are bitwise the same) with CUDA events on the solve's
 * stream around each group of kernels, and add each group's duration to its phase:
 *   QP_PHASE_APPLY32 / APPLY64: the stiffness apply of a PCG iteration (FP32 inner level / FP64 level) with its
 *     (h, Q h) reduction (FFT-backend plans: the FFT passes and the reduction);
 *   QP_PHASE_UPDATE32 / UPDATE64: the alpha step and the reductions for beta (r -= alpha Q h, ...);
 *   QP_PHASE_HUPDATE32 / HUPDATE64: the new search direction h = M r + beta h (and the U update);
 *   QP_PHASE_INIT32 / INIT64: the PCG initialisation of a (inner) solve;
 *   QP_PHASE_RESIDUAL64: FP64 applies of U (true residuals, warm starts);
 *   QP_PHASE_REFINE: the refinement steps (FP32 right-hand side 2^-e r with 2^e <= ||r|| < 2^(e+1), U += 2^e c);
 *   QP_PHASE_OTHER: zeroing and state resets.
 * qp_set_phase_timing(enabled) also clears the totals. qp_phase_times: for phases 0 .. count - 1 the summed
 * milliseconds (ms) and the number of timed groups (launches); either output may be NULL. Process-wide. */
enum { QP_PHASE_APPLY32 = 0, QP_PHASE_UPDATE32 = 1, QP_PHASE_HUPDATE32 = 2, QP_PHASE_INIT32 = 3,
       QP_PHASE_REFINE = 4, QP_PHASE_APPLY64 = 5, QP_PHASE_UPDATE64 = 6, QP_PHASE_HUPDATE64 = 7,
       QP_PHASE_INIT64 = 8, QP_PHASE_RESIDUAL64 = 9, QP_PHASE_OTHER = 10, QP_NPHASE = 11 };
qp_status qp_set_phase_timing(int enabled);
qp_status qp_phase_times(double* ms, int64_t* launches, int count);

/* Description of the last error on this host thread ("" if none). The string stays valid until the next call. */
const char* qp_last_error(void);

/* Number of CUDA kernels this library has launched in this process so far (all threads, all plans). */
uint64_t qp_launch_count(void);

/* FFT-backend apply schedules (an autotuner of this library; not in the paper, which has no FFT backend on a GPU).
 * The apply runs its n-dim transforms as passes over groups of consecutive axes staged in shared-memory tiles.
 * At plan creation every feasible schedule (one group, every split into two or three groups, each at tile
 * budgets of 48, 100 and 200 KB) and the per-axis path are timed on this GPU (CUDA events on the plan's
 * stream, max_rhs right-hand sides, for each precision in the plan's workspace) and the fastest is kept; the
 * choice is cached per (geometry, coefficient kind, max_rhs, precision) for the process, so later plans of the
 * same shape are not re-timed. Schedules differ only in the rounding order of the transforms.
 * qp_set_fft_autotune(0): later plans take the balanced-split heuristic instead (process-wide; cached choices
 * still apply). qp_fft_schedule: the schedule in use for precision (QP_FP64 / QP_FP32): its candidate index
 * (-1: the heuristic's), the number of candidates, its timed ms per apply (the timing of the plan that chose it
 * when the choice came from the cache; -1 if untimed) and a description
 * (text, text_len bytes with the terminating 0; any output may be NULL). qp_fft_set_schedule: use candidate
 * index (0 .. count - 1) from now on. Both return QP_ERR_UNSUPPORTED for a taps-backend plan. With the autotuner off,
 * QP_BACKEND_AUTO also stops timing the stencil against the FFT backend for tap coefficients (taps are kept). */
qp_status qp_set_fft_autotune(int enabled);
/* The autotuner's process-wide cache of FFT schedules (chosen candidate and every candidate's timing per geometry,
 * coefficient kind, max_rhs and precision) to and from a text file, so that a later process on the same kind of GPU
 * reuses the choices instead of timing again: save writes every entry (entries: how many; QP_ERR_INVALID_ARG when
 * the file cannot be written); load merges the file's entries into the cache (QP_ERR_INVALID_ARG for an unreadable
 * or malformed file, QP_ERR_UNSUPPORTED when it was written on another GPU model; nothing is merged then). A loaded
 * entry applies to later plans of its shape whose candidate list has the same length. clear empties the cache. */
qp_status qp_fft_tune_cache_save(const char* path, int* entries);
qp_status qp_fft_tune_cache_load(const char* path, int* entries);
qp_status qp_fft_tune_cache_clear(void);
qp_status qp_fft_schedule(const qp_plan* plan, int precision, int* index, int* count, double* ms, char* text,
                          int text_len);
qp_status qp_fft_set_schedule(qp_plan* plan, int precision, int index);

/* Limit, in seconds, of each grid-barrier wait of a persistent solve (QP_EXEC_PERSISTENT / AUTO); default 2.
 * A wait covers one phase (one stiffness apply or one vector update) of the slowest block, so the limit only
 * has to exceed the longest phase. A solve that exceeds it returns QP_ERR_TIMEOUT with its outputs undefined;
 * the device stays usable. Process-wide; 0 < seconds <= 3600, else QP_ERR_INVALID_ARG. */
qp_status qp_set_barrier_timeout(double seconds);

#ifdef __cplusplus
}
#endif
#endif /* QP_H */
