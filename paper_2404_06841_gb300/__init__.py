"""Python binding of libqp (include/qp.h): the GB300 projection-method solver for quasiperiodic elliptic
problems and quasiperiodic homogenization (arXiv 2404.06841).

Argument marshalling only. Every function has the C name and forwards to the shared library; tensors are
PyTorch CUDA tensors (complex128 / complex64, contiguous) passed by device pointer, on the current CUDA stream
unless ``stream`` is given. There is no fallback: if libqp.so is missing or fails to load, importing this
package raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqp.so")

QP_OK, QP_ERR_INVALID_ARG, QP_ERR_SINGULAR_P, QP_ERR_NOT_ELLIPTIC, QP_ERR_BREAKDOWN = 0, 1, 2, 3, 4
QP_ERR_NO_CONVERGENCE, QP_ERR_TIMEOUT, QP_ERR_UNSUPPORTED, QP_ERR_OOM, QP_ERR_CUDA = 5, 6, 7, 8, 9
STATUS_NAMES = {0: "QP_OK", 1: "QP_ERR_INVALID_ARG", 2: "QP_ERR_SINGULAR_P", 3: "QP_ERR_NOT_ELLIPTIC",
                4: "QP_ERR_BREAKDOWN", 5: "QP_ERR_NO_CONVERGENCE", 6: "QP_ERR_TIMEOUT", 7: "QP_ERR_UNSUPPORTED",
                8: "QP_ERR_OOM", 9: "QP_ERR_CUDA"}
QP_COEF_SCALAR, QP_COEF_DIAG, QP_COEF_SYM = 0, 1, 2
QP_REPR_TAPS, QP_REPR_GRID = 0, 1
QP_BACKEND_AUTO, QP_BACKEND_TAPS, QP_BACKEND_FFT = 0, 1, 2
QP_FP64, QP_FP32 = 0, 1
QP_PRECOND_JACOBI, QP_PRECOND_FROBENIUS = 0, 1
QP_MODE_FP64, QP_MODE_FP32_REFINE = 0, 1
QP_EXEC_AUTO, QP_EXEC_DIRECT, QP_EXEC_GRAPH, QP_EXEC_PERSISTENT = 0, 1, 2, 3
QP_SPECTRUM_FULL, QP_SPECTRUM_HALF = 0, 1
QP_PHASE_APPLY32, QP_PHASE_UPDATE32, QP_PHASE_HUPDATE32, QP_PHASE_INIT32, QP_PHASE_REFINE = 0, 1, 2, 3, 4
QP_PHASE_APPLY64, QP_PHASE_UPDATE64, QP_PHASE_HUPDATE64, QP_PHASE_INIT64, QP_PHASE_RESIDUAL64 = 5, 6, 7, 8, 9
QP_PHASE_OTHER, QP_NPHASE = 10, 11
KIND_CODES = {"scalar": QP_COEF_SCALAR, "diag": QP_COEF_DIAG, "sym": QP_COEF_SYM}

# Every symbol include/qp.h declares (checked by the test suite).
EXPORTS = ("qp_plan_create", "qp_plan_destroy", "qp_plan_query", "qp_apply_stiffness", "qp_corrector_rhs",
           "qp_pcg_solve", "qp_homogenized_reduce", "qp_homogenized", "qp_fft", "qp_batch_create",
           "qp_batch_homogenized", "qp_batch_destroy", "qp_last_error", "qp_launch_count",
           "qp_pcg_solve_taps_static", "qp_set_barrier_timeout", "qp_l2qp_error", "qp_plan_diagonal",
           "qp_set_fft_autotune", "qp_fft_schedule", "qp_fft_set_schedule", "qp_memory_pool_stats",
           "qp_set_memory_cache", "qp_set_phase_timing", "qp_phase_times", "qp_fft_tune_cache_save",
           "qp_fft_tune_cache_load", "qp_fft_tune_cache_clear")
PHASES = ("apply32", "update32", "hupdate32", "init32", "refine", "apply64", "update64", "hupdate64", "init64",
          "residual64", "other")


class qp_coeff(C.Structure):
    _fields_ = [("kind", C.c_int), ("repr", C.c_int), ("ntaps", C.c_int), ("tap_k", C.POINTER(C.c_int32)),
                ("tap_val", C.POINTER(C.c_double)), ("grid", C.c_void_p)]


class qp_options(C.Structure):
    _fields_ = [("backend", C.c_int), ("max_rhs", C.c_int), ("precisions", C.c_int), ("exec", C.c_int),
                ("spectrum", C.c_int)]


class qp_solve_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int), ("precond", C.c_int), ("mode", C.c_int),
                ("inner_tol", C.c_double), ("max_outer", C.c_int)]


class qp_solve_info(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("outer_iterations", C.c_int),
                ("rel_residual", C.c_double)]

    def as_dict(self):
        return {"status": STATUS_NAMES.get(self.status, self.status), "iterations": self.iterations,
                "outer_iterations": self.outer_iterations, "rel_residual": self.rel_residual}


class qp_plan_info(C.Structure):
    _fields_ = [("D", C.c_int64), ("backend", C.c_int), ("ntaps", C.c_int), ("max_rhs", C.c_int),
                ("min_abs_lambda", C.c_double), ("device_bytes", C.c_int64), ("star", C.c_int),
                ("stored_weights", C.c_int), ("spectrum", C.c_int), ("stored", C.c_int64)]


class QPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def load_library(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise ImportError("libqp.so is not built (%s); run __graft_entry__.build() or "
                          "python -m paper_2404_06841_gb300.build" % path)
    lib = C.CDLL(path)
    vp, i, dp, ip = C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int)
    sig = {
        "qp_plan_create": [i, i, dp, ip, C.POINTER(qp_coeff), C.POINTER(qp_options), vp, C.POINTER(vp)],
        "qp_plan_destroy": [vp],
        "qp_plan_query": [vp, C.POINTER(qp_plan_info)],
        "qp_apply_stiffness": [vp, i, vp, vp, i, vp],
        "qp_corrector_rhs": [vp, i, i, vp, vp],
        "qp_pcg_solve": [vp, i, vp, vp, C.POINTER(qp_solve_opts), C.POINTER(qp_solve_info), vp],
        "qp_homogenized_reduce": [vp, vp, dp, dp, vp],
        "qp_homogenized": [vp, C.POINTER(qp_solve_opts), dp, dp, C.POINTER(qp_solve_info), vp],
        "qp_fft": [i, ip, i, vp, i, i, vp],
        "qp_batch_create": [i, C.POINTER(vp), C.POINTER(vp)],
        "qp_batch_homogenized": [vp, C.POINTER(qp_solve_opts), dp, C.POINTER(qp_solve_info), vp],
        "qp_batch_destroy": [vp],
        "qp_pcg_solve_taps_static": [i, i, dp, ip, C.POINTER(qp_coeff), i, vp, vp, C.POINTER(qp_solve_opts),
                                     C.POINTER(qp_solve_info), vp],
        "qp_set_barrier_timeout": [C.c_double],
        "qp_l2qp_error": [vp, i, vp, vp, dp, vp],
        "qp_plan_diagonal": [vp, i, vp, vp],
        "qp_set_fft_autotune": [i],
        "qp_fft_tune_cache_save": [C.c_char_p, C.POINTER(C.c_int)],
        "qp_fft_tune_cache_load": [C.c_char_p, C.POINTER(C.c_int)],
        "qp_fft_tune_cache_clear": [],
        "qp_fft_schedule": [vp, i, ip, ip, dp, C.c_char_p, i],
        "qp_fft_set_schedule": [vp, i, i],
        "qp_memory_pool_stats": [C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_uint64)],
        "qp_set_memory_cache": [C.c_int64],
        "qp_set_phase_timing": [i],
        "qp_phase_times": [dp, C.POINTER(C.c_int64), i],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.qp_last_error.argtypes = []
    lib.qp_last_error.restype = C.c_char_p
    lib.qp_launch_count.argtypes = []
    lib.qp_launch_count.restype = C.c_uint64
    return lib


_lib = load_library()


def _check(status):
    if status != QP_OK:
        raise QPError(status, _lib.qp_last_error().decode())


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensors passed to libqp must be contiguous")
    return C.c_void_p(t.data_ptr())


class Plan:
    """Owns a qp_plan*; destroyed with qp_plan_destroy (explicitly or when collected)."""

    def __init__(self, handle, d, n, N, keep):
        self.handle = handle
        self.d, self.n, self.N = d, n, tuple(N)
        self.D = int(np.prod(N))
        self.shape = tuple(N)
        self.spectrum = QP_SPECTRUM_FULL
        self._keep = keep

    def __del__(self):
        try:
            if self.handle:
                qp_plan_destroy(self)
        except Exception:
            pass


def _coeff_struct(coeff, d, keep):
    """coeff: an object with kind ('scalar'|'diag'|'sym'), taps_k/taps_val (numpy) or grid (numpy/torch)."""
    c = qp_coeff()
    c.kind = KIND_CODES[coeff.kind] if isinstance(coeff.kind, str) else int(coeff.kind)
    if getattr(coeff, "taps_k", None) is not None:
        k = np.ascontiguousarray(coeff.taps_k, dtype=np.int32)
        v = np.ascontiguousarray(np.asarray(coeff.taps_val, dtype=np.complex128)).view(np.float64)
        v = np.ascontiguousarray(v)
        keep += [k, v]
        c.repr = QP_REPR_TAPS
        c.ntaps = int(k.shape[0])
        c.tap_k = k.ctypes.data_as(C.POINTER(C.c_int32))
        c.tap_val = v.ctypes.data_as(C.POINTER(C.c_double))
        c.grid = None
    else:
        import torch
        g = coeff.grid
        if not isinstance(g, torch.Tensor):
            g = torch.from_numpy(np.ascontiguousarray(g, dtype=np.float64))
        g = g.to(device="cuda", dtype=torch.float64).contiguous()
        keep.append(g)
        c.repr = QP_REPR_GRID
        c.ntaps = 0
        c.grid = g.data_ptr()
    return c


def qp_plan_create(d, n, P, N, coeff, backend=QP_BACKEND_AUTO, max_rhs=0, precisions=0, exec_mode=QP_EXEC_AUTO,
                   spectrum=QP_SPECTRUM_FULL, stream=None) -> Plan:
    """A plan; ``plan.D`` is the length of the vectors its calls take (the half-spectrum storage's D_h for
    spectrum=QP_SPECTRUM_HALF), ``plan.shape`` their shape as an array (last axis ceil(N/2) long for that storage)."""
    P = np.ascontiguousarray(P, dtype=np.float64).reshape(-1)
    Narr = np.ascontiguousarray(N, dtype=np.int32).reshape(-1)
    if d >= 1 and n >= 1 and (P.size != d * n or Narr.size != n):
        raise ValueError("P must hold d*n entries and N n entries")
    keep = [P, Narr]
    c = _coeff_struct(coeff, d, keep)
    opt = qp_options(int(backend), int(max_rhs), int(precisions), int(exec_mode), int(spectrum))
    out = C.c_void_p()
    _check(_lib.qp_plan_create(d, n, P.ctypes.data_as(C.POINTER(C.c_double)), Narr.ctypes.data_as(C.POINTER(C.c_int)),
                               C.byref(c), C.byref(opt), _stream(stream), C.byref(out)))
    plan = Plan(out, d, n, [int(x) for x in Narr], keep=[])
    if spectrum == QP_SPECTRUM_HALF:
        plan.spectrum = QP_SPECTRUM_HALF
        plan.shape = plan.N[:-1] + ((plan.N[-1] + 1) // 2,)
        plan.D = int(np.prod(plan.shape))
    return plan


def qp_plan_destroy(plan: Plan):
    if plan.handle:
        h = plan.handle
        plan.handle = None
        _check(_lib.qp_plan_destroy(h))


def qp_plan_query(plan: Plan) -> dict:
    info = qp_plan_info()
    _check(_lib.qp_plan_query(plan.handle, C.byref(info)))
    return {"D": info.D, "backend": {1: "taps", 2: "fft"}.get(info.backend, info.backend), "ntaps": info.ntaps,
            "max_rhs": info.max_rhs, "min_abs_lambda": info.min_abs_lambda, "device_bytes": info.device_bytes,
            "star": bool(info.star), "stored_weights": bool(info.stored_weights), "spectrum": info.spectrum,
            "stored": info.stored}


def qp_apply_stiffness(plan: Plan, U, QU, precision=QP_FP64, nrhs=None, stream=None):
    if nrhs is None:
        nrhs = U.numel() // plan.D
    _check(_lib.qp_apply_stiffness(plan.handle, int(nrhs), _ptr(U), _ptr(QU), int(precision), _stream(stream)))


def qp_corrector_rhs(plan: Plan, j0, nrhs, F, stream=None):
    _check(_lib.qp_corrector_rhs(plan.handle, int(j0), int(nrhs), _ptr(F), _stream(stream)))


def _opts(tol, maxit, precond, mode, inner_tol, max_outer):
    return qp_solve_opts(float(tol), int(maxit), int(precond), int(mode), float(inner_tol), int(max_outer))


def qp_pcg_solve(plan: Plan, F, U, tol=1e-10, maxit=1000, precond=QP_PRECOND_JACOBI, mode=QP_MODE_FP64,
                 inner_tol=0.0, max_outer=0, nrhs=None, stream=None, raise_on_error=True):
    if nrhs is None:
        nrhs = F.numel() // plan.D
    infos = (qp_solve_info * nrhs)()
    o = _opts(tol, maxit, precond, mode, inner_tol, max_outer)
    st = _lib.qp_pcg_solve(plan.handle, int(nrhs), _ptr(F), _ptr(U), C.byref(o), infos, _stream(stream))
    if raise_on_error:
        _check(st)
    return [x.as_dict() for x in infos]


def qp_homogenized_reduce(plan: Plan, U, stream=None):
    d = plan.d
    re = np.zeros(d * d)
    im = np.zeros(d * d)
    _check(_lib.qp_homogenized_reduce(plan.handle, _ptr(U), re.ctypes.data_as(C.POINTER(C.c_double)),
                                      im.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream)))
    return (re + 1j * im).reshape(d, d)


def qp_homogenized(plan: Plan, tol=1e-10, maxit=1000, precond=QP_PRECOND_JACOBI, mode=QP_MODE_FP64,
                   inner_tol=0.0, max_outer=0, stream=None, raise_on_error=True):
    """Returns (A* complex d x d, [info per corrector])."""
    d = plan.d
    re = np.zeros(d * d)
    im = np.zeros(d * d)
    infos = (qp_solve_info * d)()
    o = _opts(tol, maxit, precond, mode, inner_tol, max_outer)
    st = _lib.qp_homogenized(plan.handle, C.byref(o), re.ctypes.data_as(C.POINTER(C.c_double)),
                             im.ctypes.data_as(C.POINTER(C.c_double)), infos, _stream(stream))
    if raise_on_error:
        _check(st)
    return (re + 1j * im).reshape(d, d), [x.as_dict() for x in infos]


def qp_fft(data, N, sign=-1, precision=None, count=None, stream=None):
    """In-place unnormalised n-dim DFT of ``count`` contiguous arrays of shape N (sign -1 forward, +1 inverse)."""
    import torch
    N = [int(x) for x in N]
    if precision is None:
        precision = QP_FP64 if data.dtype == torch.complex128 else QP_FP32
    if count is None:
        count = data.numel() // int(np.prod(N))
    Narr = (C.c_int * len(N))(*N)
    _check(_lib.qp_fft(len(N), Narr, int(count), _ptr(data), int(sign), int(precision), _stream(stream)))


class Batch:
    def __init__(self, handle, plans):
        self.handle = handle
        self.plans = plans

    def __del__(self):
        try:
            if self.handle:
                qp_batch_destroy(self)
        except Exception:
            pass


def qp_batch_create(plans) -> Batch:
    arr = (C.c_void_p * len(plans))(*[p.handle.value if isinstance(p.handle, C.c_void_p) else p.handle
                                      for p in plans])
    out = C.c_void_p()
    _check(_lib.qp_batch_create(len(plans), arr, C.byref(out)))
    return Batch(out, list(plans))


def qp_batch_homogenized(batch: Batch, tol=1e-10, maxit=1000, precond=QP_PRECOND_JACOBI, mode=QP_MODE_FP32_REFINE,
                         inner_tol=0.0, max_outer=0, stream=None, raise_on_error=True):
    tot = sum(p.d * p.d for p in batch.plans)
    units = sum(p.d for p in batch.plans)
    A = np.zeros(tot)
    infos = (qp_solve_info * units)()
    o = _opts(tol, maxit, precond, mode, inner_tol, max_outer)
    st = _lib.qp_batch_homogenized(batch.handle, C.byref(o), A.ctypes.data_as(C.POINTER(C.c_double)), infos,
                                   _stream(stream))
    if raise_on_error:
        _check(st)
    out, off = [], 0
    for p in batch.plans:
        out.append(A[off:off + p.d * p.d].reshape(p.d, p.d))
        off += p.d * p.d
    return out, [x.as_dict() for x in infos]


def qp_batch_destroy(batch: Batch):
    if batch.handle:
        h = batch.handle
        batch.handle = None
        _check(_lib.qp_batch_destroy(h))


def qp_pcg_solve_taps_static(d, n, P, N, coeff, F, U, tol=1e-10, maxit=1000, precond=QP_PRECOND_JACOBI,
                             nrhs=None, stream=None, raise_on_error=True):
    """The allocation-free FP64 solve (no plan; all intermediates in the library's static device scratch)."""
    P = np.ascontiguousarray(P, dtype=np.float64).reshape(-1)
    Narr = np.ascontiguousarray(N, dtype=np.int32).reshape(-1)
    keep = [P, Narr]
    c = _coeff_struct(coeff, d, keep)
    if nrhs is None:
        nrhs = F.numel() // int(np.prod(Narr))
    infos = (qp_solve_info * nrhs)()
    o = _opts(tol, maxit, precond, QP_MODE_FP64, 0.0, 0)
    st = _lib.qp_pcg_solve_taps_static(d, n, P.ctypes.data_as(C.POINTER(C.c_double)),
                                       Narr.ctypes.data_as(C.POINTER(C.c_int)), C.byref(c), int(nrhs), _ptr(F),
                                       _ptr(U), C.byref(o), infos, _stream(stream))
    if raise_on_error:
        _check(st)
    return [x.as_dict() for x in infos]


def qp_last_error() -> str:
    return _lib.qp_last_error().decode()


def qp_launch_count() -> int:
    return int(_lib.qp_launch_count())


def qp_plan_diagonal(plan: Plan, precond=QP_PRECOND_JACOBI, stream=None):
    """The preconditioner diagonal M (z = M r) as a device float64 tensor of the plan's grid shape."""
    import torch
    out = torch.empty(plan.shape, dtype=torch.float64, device="cuda")
    _check(_lib.qp_plan_diagonal(plan.handle, int(precond), _ptr(out), _stream(stream)))
    return out


def qp_l2qp_error(plan: Plan, U, Uref=None, stream=None) -> np.ndarray:
    """e_r = ||U_r - Uref_r|| in the L^2_QP norm (the l^2 norm of the Fourier coefficients, Parseval), per
    right-hand side. U, Uref: contiguous device complex128 tensors holding nrhs x D entries."""
    nrhs = U.numel() // plan.D
    if nrhs * plan.D != U.numel() or (Uref is not None and Uref.numel() != U.numel()):
        raise QPError(QP_ERR_INVALID_ARG, "U and Uref must hold nrhs x D entries each")
    out = np.zeros(nrhs, dtype=np.float64)
    _check(_lib.qp_l2qp_error(plan.handle, int(nrhs), _ptr(U), _ptr(Uref),
                              out.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream)))
    return out


def qp_set_fft_autotune(enabled: bool) -> None:
    """Process-wide: time the FFT apply's candidate schedules at plan creation (default) or take the heuristic."""
    _check(_lib.qp_set_fft_autotune(1 if enabled else 0))


def qp_fft_schedule(plan: Plan, precision=QP_FP32) -> dict:
    """The FFT-backend apply schedule in use: candidate index, candidate count, timed ms per apply, description."""
    idx, cnt, ms = C.c_int(0), C.c_int(0), C.c_double(0.0)
    buf = C.create_string_buffer(256)
    _check(_lib.qp_fft_schedule(plan.handle, int(precision), C.byref(idx), C.byref(cnt), C.byref(ms), buf, 256))
    return {"index": idx.value, "count": cnt.value, "ms": ms.value, "text": buf.value.decode()}


def qp_fft_tune_cache_save(path: str) -> int:
    """Writes the autotuner's schedule cache to a text file; returns the entries written."""
    n = C.c_int(0)
    _check(_lib.qp_fft_tune_cache_save(str(path).encode(), C.byref(n)))
    return n.value


def qp_fft_tune_cache_load(path: str) -> int:
    """Merges a schedule cache file (written on the same GPU model) into the process's cache; returns its entries."""
    n = C.c_int(0)
    _check(_lib.qp_fft_tune_cache_load(str(path).encode(), C.byref(n)))
    return n.value


def qp_fft_tune_cache_clear() -> None:
    """Empties the autotuner's schedule cache (later plans are timed again, or take the heuristic when off)."""
    _check(_lib.qp_fft_tune_cache_clear())


def qp_fft_set_schedule(plan: Plan, precision, index: int) -> None:
    _check(_lib.qp_fft_set_schedule(plan.handle, int(precision), int(index)))


def qp_memory_pool_stats() -> dict:
    """The library's device-memory pool on the current device: reserved and used bytes, allocations served."""
    res, use, n = C.c_int64(0), C.c_int64(0), C.c_uint64(0)
    _check(_lib.qp_memory_pool_stats(C.byref(res), C.byref(use), C.byref(n)))
    return {"reserved_bytes": res.value, "used_bytes": use.value, "allocations": n.value}


def qp_set_memory_cache(nbytes: int) -> None:
    """Freed pool memory kept cached after a destroy (bytes; 0 returns all of it; < 0 restores the default)."""
    _check(_lib.qp_set_memory_cache(int(nbytes)))


def qp_set_phase_timing(enabled: bool) -> None:
    """Per-phase CUDA-event timing of solves (host-driven form while on); also clears the totals."""
    _check(_lib.qp_set_phase_timing(1 if enabled else 0))


def qp_phase_times() -> dict:
    """{phase name: (milliseconds, timed launches)} accumulated since qp_set_phase_timing."""
    n = len(PHASES)
    ms = (C.c_double * n)()
    cnt = (C.c_int64 * n)()
    _check(_lib.qp_phase_times(ms, cnt, n))
    return {name: (ms[i], cnt[i]) for i, name in enumerate(PHASES)}


def qp_set_barrier_timeout(seconds: float) -> None:
    """Limit of each grid-barrier wait of a persistent solve (process-wide; default 2 s)."""
    _check(_lib.qp_set_barrier_timeout(float(seconds)))


def plan_from_instance(inst, **kw) -> Plan:
    """Convenience: a plan for a ``qp_workloads.Instance``."""
    return qp_plan_create(inst.d, inst.n, inst.P, inst.N, inst.coeff, **kw)
