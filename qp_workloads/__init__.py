"""Seeded synthetic inputs for the quasiperiodic projection-method solver.

This module is shared by the FP64 oracle (test infrastructure) and by the CUDA path. It only draws and
describes inputs: projection matrices P, grid sizes N, the coefficient's Fourier modes ("taps") and the
coefficient's samples on the torus grid. It holds none of the method's arithmetic: no stiffness operator, no
transform of the solution, no solver, no homogenized-coefficient formula.

Conventions (used by both consumers):

* The coefficient A(theta) is a real, d x d, symmetric, uniformly elliptic field on the torus T^n
  (Sec. 2.2, elliptic problem; Sec. 5.2, corrector problem). It is stored as ``ncomp`` real components:
  ``scalar``: A = a I (1 component); ``diag``: A = diag(a_1..a_d) (d components);
  ``sym``: the upper triangle row by row, (11, 12, .., 1d, 22, .., dd) (d(d+1)/2 components).
* Taps: ``taps_k`` (g, n) int32 Fourier modes m and ``taps_val`` (g, ncomp) complex128 values A~_m with
  A(theta) = sum_m A~_m exp(i m.theta). A real field needs A~_{-m} = conj(A~_m); every generator here
  emits both members of each pair.
* Grid: ``grid`` (ncomp, N_1, .., N_n) float64, samples A(y_j) at y_j = 2 pi j / N (Sec. 2.3), C order
  with the last torus axis fastest.
* Every random draw goes through ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

SQRT2, SQRT3, SQRT5 = math.sqrt(2.0), math.sqrt(3.0), math.sqrt(5.0)
GOLDEN = (1.0 + SQRT5) / 2.0

KINDS = ("scalar", "diag", "sym")


def ncomp(kind: str, d: int) -> int:
    """Number of stored real components of the coefficient for ``kind`` in dimension d."""
    if kind == "scalar":
        return 1
    if kind == "diag":
        return d
    if kind == "sym":
        return d * (d + 1) // 2
    raise ValueError(f"unknown coefficient kind {kind!r}")


def sym_pairs(d: int):
    """(a, b) index pairs of the stored upper triangle, row by row."""
    return [(a, b) for a in range(d) for b in range(a, d)]


@dataclass
class Coefficient:
    kind: str
    taps_k: np.ndarray | None = None     # (g, n) int32
    taps_val: np.ndarray | None = None   # (g, ncomp) complex128
    grid: np.ndarray | None = None       # (ncomp, *N) float64

    @property
    def repr(self) -> str:
        return "taps" if self.taps_k is not None else "grid"


@dataclass
class Instance:
    """One quasiperiodic homogenization problem: projection P (d x n), grid N (n,), coefficient."""
    name: str
    P: np.ndarray
    N: tuple
    coeff: Coefficient
    tol: float = 1e-10
    meta: dict = field(default_factory=dict)

    @property
    def d(self) -> int:
        return int(self.P.shape[0])

    @property
    def n(self) -> int:
        return int(self.P.shape[1])

    @property
    def D(self) -> int:
        return int(np.prod(self.N))


# --------------------------------------------------------------------------------------------- helpers

def taps_from_dict(modes: dict, n: int, nc: int):
    """Pack {mode tuple: complex array (nc,)} into (taps_k, taps_val), mode order sorted for determinism."""
    keys = sorted(modes.keys())
    k = np.array(keys, dtype=np.int32).reshape(len(keys), n)
    v = np.array([np.asarray(modes[key], dtype=np.complex128).reshape(nc) for key in keys],
                 dtype=np.complex128).reshape(len(keys), nc)
    return k, v


def _add_mode(modes: dict, m, val, nc):
    key = tuple(int(x) for x in m)
    if key not in modes:
        modes[key] = np.zeros(nc, dtype=np.complex128)
    modes[key] = modes[key] + np.asarray(val, dtype=np.complex128)


def sample_on_grid(N, taps_k, taps_val) -> np.ndarray:
    """Evaluate the trigonometric polynomial sum_m val_m exp(i m.y) at the grid nodes y_j = 2 pi j / N.

    Direct evaluation, one separable product of per-axis exponentials per mode (input construction only).
    Returns the real part, shape (ncomp, *N); the imaginary part vanishes for Hermitian-paired taps.
    """
    N = tuple(int(x) for x in N)
    nc = taps_val.shape[1]
    out = np.zeros((nc,) + N, dtype=np.complex128)
    for m, val in zip(taps_k, taps_val):
        field_ = np.ones((), dtype=np.complex128)
        for j, Nj in enumerate(N):
            e = np.exp(1j * 2.0 * np.pi * ((int(m[j]) * np.arange(Nj)) % Nj) / Nj)
            field_ = np.multiply.outer(field_, e)
        for c in range(nc):
            out[c] += val[c] * field_
    return np.ascontiguousarray(out.real)


def unit_modes(n: int, radius: int = 1):
    """All nonzero integer modes m with |m|_inf <= radius, sorted."""
    rng_ = range(-radius, radius + 1)
    return [m for m in itertools.product(rng_, repeat=n) if any(m)]


def positive_half(modes):
    """One representative per +-pair: the mode whose first nonzero coordinate is positive."""
    out = []
    for m in modes:
        first = next(x for x in m if x != 0)
        if first > 0:
            out.append(m)
    return out


def manufactured_modes(n: int, kmax: int, seed: int):
    """Manufactured solution U^: modes |k|_inf <= kmax, k != 0, complex N(0,1) amplitudes.

    Returns (modes (M, n) int64, amps (M,) complex128).
    """
    rng = np.random.default_rng(seed)
    modes = np.array(unit_modes(n, kmax), dtype=np.int64)
    amps = rng.standard_normal(len(modes)) + 1j * rng.standard_normal(len(modes))
    return modes, amps


# --------------------------------------------------------------------------------------------- configs

P_CFG1 = np.array([[1.0, SQRT2, 0.0, 0.0], [0.0, 0.0, 1.0, SQRT3]])
P_CFG4 = np.array([[1.0, SQRT2, 0, 0, 0, 0], [0, 0, 1.0, SQRT3, 0, 0], [0, 0, 0, 0, 1.0, SQRT5]], dtype=float)


def cos_sum_taps(n: int, c0: float, amp: float):
    """Scalar a(theta) = c0 + amp * sum_j cos(theta_j): 1 + 2n taps."""
    modes = {}
    _add_mode(modes, (0,) * n, [c0], 1)
    for j in range(n):
        e = [0] * n
        e[j] = 1
        _add_mode(modes, e, [amp / 2], 1)
        e[j] = -1
        _add_mode(modes, e, [amp / 2], 1)
    return taps_from_dict(modes, n, 1)


def cfg0(N: int = 32) -> Instance:
    """d=1 lifted to n=2, P=(1, sqrt 2), a = 3 + cos th1 + cos th2 (5 taps), Jacobi-PCG to 1e-12."""
    k, v = cos_sum_taps(2, 3.0, 1.0)
    return Instance("cfg0_d1n2_N%d" % N, np.array([[1.0, SQRT2]]), (N, N), Coefficient("scalar", k, v),
                    tol=1e-12, meta={"manufactured_seed": 0, "manufactured_kmax": 4})


def cfg1(N: int = 16) -> Instance:
    """d=2 lifted to n=4, P=[[1,sqrt2,0,0],[0,0,1,sqrt3]], A = (5 + sum_j cos th_j) I2 (9 taps), tol 1e-10."""
    k, v = cos_sum_taps(4, 5.0, 1.0)
    return Instance("cfg1_d2n4_N%d" % N, P_CFG1.copy(), (N,) * 4, Coefficient("scalar", k, v),
                    tol=1e-10, meta={"manufactured_seed": 1, "manufactured_kmax": 4})


def spd_field_taps(n: int, d: int, seed: int, sigma: float = 0.1, mean: float = 2.75, radius: int = 1):
    """Symmetric d x d trig-polynomial field S = mean*I + sum_{0<|m|_inf<=radius} S^_m e^{i m.theta}.

    Real and imaginary parts of each upper-triangle entry of S^_m are N(0, sigma); S^_{-m} = conj(S^_m).
    """
    rng = np.random.default_rng(seed)
    nc = d * (d + 1) // 2
    modes = {}
    mean_val = np.array([mean if a == b else 0.0 for (a, b) in sym_pairs(d)], dtype=np.complex128)
    _add_mode(modes, (0,) * n, mean_val, nc)
    for m in positive_half(unit_modes(n, radius)):
        s = sigma * (rng.standard_normal(nc) + 1j * rng.standard_normal(nc))
        _add_mode(modes, m, s, nc)
        _add_mode(modes, tuple(-x for x in m), np.conj(s), nc)
    return taps_from_dict(modes, n, nc)


def clamp_spd_grid(d: int, grid_sym: np.ndarray, lo: float, hi: float):
    """At every node, S = Q L Q^T -> Q clamp(L, lo, hi) Q^T. Returns (grid, fraction of clamped nodes)."""
    pairs = sym_pairs(d)
    shp = grid_sym.shape[1:]
    S = np.zeros(shp + (d, d))
    for c, (a, b) in enumerate(pairs):
        S[..., a, b] = grid_sym[c]
        S[..., b, a] = grid_sym[c]
    L, Qm = np.linalg.eigh(S)
    clamped = np.any((L < lo) | (L > hi), axis=-1)
    Lc = np.clip(L, lo, hi)
    A = np.einsum("...ik,...k,...jk->...ij", Qm, Lc, Qm)
    out = np.stack([A[..., a, b] for (a, b) in pairs])
    return np.ascontiguousarray(out), float(clamped.mean())


def cfg2(N: int = 32, seed: int = 2) -> Instance:
    """d=2, n=4, cfg1's P, full SPD 2x2 coefficient A = Q clamp(L) Q^T from an 81-tap symmetric field, on the grid."""
    k, v = spd_field_taps(4, 2, seed)
    S = sample_on_grid((N,) * 4, k, v)
    grid, frac = clamp_spd_grid(2, S, 0.5, 5.0)
    return Instance("cfg2_d2n4_N%d_sym" % N, P_CFG1.copy(), (N,) * 4, Coefficient("sym", grid=grid),
                    tol=1e-10, meta={"seed": seed, "clamped_fraction": frac, "field_taps_k": k,
                                     "field_taps_val": v})


def random_cosine_scalar_taps(n: int, seed: int, T: int = 4):
    """a = c0 + sum_{t<T} rho_t cos(m_t.theta + phi_t), m_t from 0<|m|_inf<=1, rho~U[0,.5], phi~U[0,2pi),
    c0 = 0.5 + sum rho_t (so min a >= 0.5)."""
    rng = np.random.default_rng(seed)
    cand = unit_modes(n, 1)
    modes = {}
    rhos = []
    for _ in range(T):
        m = cand[int(rng.integers(len(cand)))]
        rho = float(rng.uniform(0.0, 0.5))
        phi = float(rng.uniform(0.0, 2.0 * np.pi))
        rhos.append(rho)
        _add_mode(modes, m, [0.5 * rho * np.exp(1j * phi)], 1)
        _add_mode(modes, tuple(-x for x in m), [0.5 * rho * np.exp(-1j * phi)], 1)
    _add_mode(modes, (0,) * n, [0.5 + sum(rhos)], 1)
    return taps_from_dict(modes, n, 1)


def cfg3():
    """64 instances: 32 with d=1, n=2, P=(1, alpha); 32 with d=2, n=4 (cfg1's P). Instance i uses seed 3000+i."""
    out = []
    i = 0
    for alpha, aname in ((SQRT2, "sqrt2"), (SQRT3, "sqrt3"), (SQRT5, "sqrt5"), (GOLDEN, "golden")):
        for N in (64, 128, 256, 512):
            for rep in range(2):
                k, v = random_cosine_scalar_taps(2, 3000 + i)
                out.append(Instance("cfg3_%02d_d1n2_%s_N%d" % (i, aname, N), np.array([[1.0, alpha]]), (N, N),
                                    Coefficient("scalar", k, v), tol=1e-10, meta={"seed": 3000 + i}))
                i += 1
    for N in (8, 12, 16, 24):
        for rep in range(8):
            k, v = random_cosine_scalar_taps(4, 3000 + i)
            out.append(Instance("cfg3_%02d_d2n4_N%d" % (i, N), P_CFG1.copy(), (N,) * 4,
                                Coefficient("scalar", k, v), tol=1e-10, meta={"seed": 3000 + i}))
            i += 1
    return out


def cfg4(N: int = 16, seed: int = 4) -> Instance:
    """d=3, n=6, A = diag(a_i), a_i = 4 + sum_j 0.5 cos(theta_j + phi_ij), phi ~ U[0, 2pi) (13 taps)."""
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=(3, 6))
    modes = {}
    _add_mode(modes, (0,) * 6, [4.0, 4.0, 4.0], 3)
    for j in range(6):
        e = [0] * 6
        e[j] = 1
        _add_mode(modes, e, 0.25 * np.exp(1j * phi[:, j]), 3)
        e[j] = -1
        _add_mode(modes, e, 0.25 * np.exp(-1j * phi[:, j]), 3)
    k, v = taps_from_dict(modes, 6, 3)
    return Instance("cfg4_d3n6_N%d_diag" % N, P_CFG4.copy(), (N,) * 6, Coefficient("diag", k, v),
                    tol=1e-10, meta={"seed": seed, "phi": phi})


def paper_elliptic_u1(N: int = 128) -> Instance:
    """The first elliptic example of Sec. 5.1.1 (Table 2): alpha_1(x) = cos(2 pi x) + cos(2 pi sqrt2 x) + 6, lifted
    with P = 2 pi (1, sqrt2) to 6 + cos th1 + cos th2, and the exact solution u_1(x) = sin(2 pi x) + sin(2 pi sqrt2 x),
    lifted to sin th1 + sin th2, whose Fourier coefficients are -i/2 at (1, 0), (0, 1) and +i/2 at (-1, 0), (0, -1).
    meta["u_modes"], meta["u_amps"]: those modes and coefficients."""
    k, v = cos_sum_taps(2, 6.0, 1.0)
    modes = np.array([(1, 0), (-1, 0), (0, 1), (0, -1)], dtype=np.int64)
    amps = np.array([-0.5j, 0.5j, -0.5j, 0.5j])
    return Instance("tab2_alpha1_u1_N%d" % N, 2.0 * math.pi * np.array([[1.0, SQRT2]]), (N, N),
                    Coefficient("scalar", k, v), tol=1e-14, meta={"u_modes": modes, "u_amps": amps})


def modes_on_grid(N, modes, amps) -> np.ndarray:
    """Dense array on K_N^n (storage index k mod N_j) holding the given Fourier coefficients."""
    out = np.zeros(tuple(N), dtype=np.complex128)
    for m, a in zip(modes, amps):
        out[tuple(int(x) % int(Nj) for x, Nj in zip(m, N))] += a
    return out


# --------------------------------------------------------------------------------------------- test inputs

def random_P(d: int, n: int, seed: int) -> np.ndarray:
    """A d x n projection with generic (almost surely Q-linearly independent) real columns."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.5, 1.5, size=(d, n)) * rng.choice([-1.0, 1.0], size=(d, n))


def random_taps(d: int, n: int, kind: str, seed: int, radius: int = 1, nmodes: int | None = None,
                margin: float = 0.5, sigma: float = 0.3):
    """Random Hermitian-paired taps with |m|_inf <= radius, made uniformly elliptic by the mean term.

    The mean is margin + (sum over nonzero modes of the entry magnitudes), so that every eigenvalue of A(theta)
    stays >= margin for all theta (Gershgorin on the oscillating part).
    """
    rng = np.random.default_rng(seed)
    nc = ncomp(kind, d)
    half = positive_half(unit_modes(n, radius))
    if nmodes is not None and nmodes < len(half):
        idx = rng.choice(len(half), size=nmodes, replace=False)
        half = [half[i] for i in sorted(idx)]
    modes = {}
    bound = 0.0
    for m in half:
        s = sigma * (rng.standard_normal(nc) + 1j * rng.standard_normal(nc))
        _add_mode(modes, m, s, nc)
        _add_mode(modes, tuple(-x for x in m), np.conj(s), nc)
        bound += 2.0 * float(np.abs(s).sum())
    if kind == "sym":
        mean = np.array([margin + bound if a == b else 0.0 for (a, b) in sym_pairs(d)])
        offd = 0.1 * rng.standard_normal(nc)
        mean = mean + np.array([0.0 if a == b else offd[c] for c, (a, b) in enumerate(sym_pairs(d))])
        mean = mean + np.array([abs(offd).sum() if a == b else 0.0 for (a, b) in sym_pairs(d)])
    else:
        mean = np.full(nc, margin + bound)
    _add_mode(modes, (0,) * n, mean, nc)
    return taps_from_dict(modes, n, nc)


def random_star_instance(d: int, n: int, N, kind: str = "scalar", seed: int = 0, axes=None, real: bool = False,
                         margin: float = 0.5, sigma: float = 0.3) -> Instance:
    """Random instance whose taps sit only at m = 0 and m = +-e_j for j in ``axes`` (default: every axis);
    ``real`` makes every tap value real (an even coefficient). Elliptic by the same Gershgorin mean as
    random_taps."""
    rng = np.random.default_rng(seed)
    N = tuple(int(x) for x in ((N,) * n if np.isscalar(N) else N))
    nc = ncomp(kind, d)
    axes = list(range(n)) if axes is None else list(axes)
    modes = {}
    bound = 0.0
    for j in axes:
        s = sigma * rng.standard_normal(nc) + (0.0 if real else 1j * sigma * rng.standard_normal(nc))
        e = [0] * n
        e[j] = 1
        _add_mode(modes, e, s, nc)
        e[j] = -1
        _add_mode(modes, e, np.conj(s), nc)
        bound += 2.0 * float(np.abs(s).sum())
    _add_mode(modes, (0,) * n, np.full(nc, margin + bound), nc)
    k, v = taps_from_dict(modes, n, nc)
    P = random_P(d, n, seed + 7919)
    return Instance("star_d%dn%d_%s_s%d" % (d, n, kind, seed), P, N, Coefficient(kind, k, v))


def random_instance(d: int, n: int, N, kind: str = "scalar", repr_: str = "taps", seed: int = 0,
                    P: np.ndarray | None = None, radius: int = 1, nmodes: int | None = None,
                    nonlinear: bool = False) -> Instance:
    """Random test instance. ``repr_='grid'`` samples the taps on the grid; ``nonlinear`` then adds
    s*(exp(x) - 1 - x) >= 0, x = (g - mean)/s, to every diagonal entry g, so the coefficient has full Fourier
    support (no finite tap list) and stays uniformly elliptic (diagonal entries only grow)."""
    if np.isscalar(N):
        N = (int(N),) * n
    N = tuple(int(x) for x in N)
    if P is None:
        P = random_P(d, n, seed + 7919)
    k, v = random_taps(d, n, kind, seed, radius=radius, nmodes=nmodes)
    name = "rand_d%dn%d_%s_%s_s%d" % (d, n, kind, repr_, seed)
    if repr_ == "taps":
        return Instance(name, np.asarray(P, float), N, Coefficient(kind, k, v))
    g = sample_on_grid(N, k, v)
    if nonlinear:
        g = g.copy()
        diag_idx = [0] if kind == "scalar" else (list(range(d)) if kind == "diag" else
                                                 [c for c, (a, b) in enumerate(sym_pairs(d)) if a == b])
        for c in diag_idx:
            s = max(float(np.abs(g[c] - g[c].mean()).max()), 1e-3)
            x = (g[c] - g[c].mean()) / s
            g[c] = g[c] + s * (np.exp(x) - 1.0 - x)
    return Instance(name, np.asarray(P, float), N, Coefficient(kind, grid=np.ascontiguousarray(g)),
                    meta={"taps_k": k, "taps_val": v, "nonlinear": nonlinear})
