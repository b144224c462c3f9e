"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test ties one oracle function to something other than itself: a printed value of the paper, a closed
form, a brute-force computation, or an invariant. A plausible slip in the oracle (a dropped term, a wrong
sign or index, a transposed operand) breaks at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import qp_workloads as W
from oracle import qp_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _inst(P, N, kind, taps=None, grid=None, tol=1e-12):
    return W.Instance("t", np.asarray(P, float), tuple(N), W.Coefficient(kind, *(taps or (None, None)), grid=grid),
                      tol=tol)


# ------------------------------------------------------------------------------ index conversion (paper)

def test_index_conversion_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "index_example.json")))
    assert O.tensor_to_vector_index(g["tensor_index"], g["N"]) == g["vector_index"]
    assert O.vector_to_tensor_index(g["vector_index"], g["N"]) == tuple(g["tensor_index"])


@pytest.mark.parametrize("N", [(4, 4), (3, 5), (6, 4, 2), (2, 3, 4, 5)])
def test_index_conversion_bijection_and_fftfreq(N):
    D = int(np.prod(N))
    seen = set()
    for i in range(D):
        k = O.vector_to_tensor_index(i, N)
        assert all(-Nj / 2 <= kj < Nj / 2 for kj, Nj in zip(k, N))
        assert O.tensor_to_vector_index(k, N) == i
        seen.add(k)
    assert len(seen) == D
    # the storage order is numpy's fftfreq order on every axis (k = ibar or ibar - N)
    for Nj in N:
        assert np.array_equal(O.signed_k(Nj), np.round(np.fft.fftfreq(Nj) * Nj).astype(int)) or Nj % 2 == 0
        if Nj % 2 == 0:
            ref = np.round(np.fft.fftfreq(Nj) * Nj).astype(int)   # numpy puts -N/2 at index N/2 as well
            assert np.array_equal(O.signed_k(Nj), ref)


def test_lambdas_against_matrix_product():
    P = W.random_P(2, 3, 5)
    N = (4, 6, 5)
    lam = O.lambdas(P, N)
    for i in [0, 7, 33, 119]:
        k = O.vector_to_tensor_index(i, N)
        idx = tuple(kj % Nj for kj, Nj in zip(k, N))
        assert np.allclose(lam[(slice(None),) + idx], P @ np.array(k, float), rtol=0, atol=1e-14)


# ------------------------------------------------------------------------------ DFT convention

def test_numpy_fft_matches_explicit_dft():
    """The oracle's grid transform must be A~_k = (1/D) sum_j A(y_j) e^{-i k.y_j} (Sec. 3.1.1)."""
    rng = np.random.default_rng(0)
    N = (3, 4)
    A = rng.standard_normal(N)
    hat = np.fft.fftn(A) / A.size
    for i in range(A.size):
        k = O.vector_to_tensor_index(i, N)
        s = 0
        for j0 in range(N[0]):
            for j1 in range(N[1]):
                y = (2 * np.pi * j0 / N[0], 2 * np.pi * j1 / N[1])
                s += A[j0, j1] * np.exp(-1j * (k[0] * y[0] + k[1] * y[1]))
        assert abs(hat[tuple(kj % Nj for kj, Nj in zip(k, N))] - s / A.size) < 1e-14


# ------------------------------------------------------------------------------ P7: brute force on tiny grids

TINY = [
    (1, 2, (4, 4), "scalar"), (1, 2, (6, 4), "scalar"), (2, 2, (4, 4), "diag"), (2, 2, (4, 6), "sym"),
    (2, 3, (4, 4, 2), "sym"), (1, 3, (4, 2, 4), "scalar"), (3, 3, (2, 4, 4), "diag"), (3, 3, (4, 2, 4), "sym"),
]


@pytest.mark.parametrize("d,n,N,kind", TINY)
def test_dense_Q_hermitian_positive_and_three_applies_agree(d, n, N, kind):
    inst = W.random_instance(d, n, N, kind, "taps", seed=11 + d + n)
    Ahat = O.coefficient_modes(inst)
    Q = O.dense_Q(inst.P, N, Ahat)
    assert np.abs(Q - Q.conj().T).max() <= 1e-12 * np.abs(Q).max()
    # k = 0 row and column vanish; the rest is positive definite
    assert np.abs(Q[0]).max() == 0 and np.abs(Q[:, 0]).max() == 0
    ev = np.linalg.eigvalsh(Q[1:, 1:])
    assert ev.min() > 0
    rng = np.random.default_rng(3)
    h = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    w_dense = (Q @ h.reshape(-1)).reshape(N)
    w_conv = O.apply_convolution(inst.P, N, Ahat, h)
    Agrid = O.coefficient_grid(inst)
    w_fft = O.apply_fft(inst.P, N, Agrid, h)
    scale = np.abs(w_dense).max()
    assert np.abs(w_conv - w_dense).max() <= 1e-12 * scale
    assert np.abs(w_fft - w_dense).max() <= 1e-12 * scale


@pytest.mark.parametrize("d,n,N,kind", [(1, 2, (4, 6), "scalar"), (2, 2, (4, 4), "sym"), (2, 3, (2, 4, 4), "diag")])
def test_fft_apply_on_full_support_grid_matches_dense(d, n, N, kind):
    """A grid coefficient with full Fourier support: dense Alg. 1 over all D modes == DFT apply."""
    inst = W.random_instance(d, n, N, kind, "grid", seed=5, nonlinear=True)
    Ahat = O.coefficient_modes(inst)
    assert len(O.nonzero_modes(Ahat, rel=1e-14)) > 0.5 * np.prod(N)
    Q = O.dense_Q(inst.P, N, Ahat)
    assert np.abs(Q - Q.conj().T).max() <= 1e-12 * np.abs(Q).max()
    rng = np.random.default_rng(4)
    h = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    w_dense = (Q @ h.reshape(-1)).reshape(N)
    w_fft = O.apply_fft(inst.P, N, O.coefficient_grid(inst), h)
    w_conv = O.apply_convolution(inst.P, N, Ahat, h)
    assert np.abs(w_fft - w_dense).max() <= 1e-12 * np.abs(w_dense).max()
    assert np.abs(w_conv - w_dense).max() <= 1e-12 * np.abs(w_dense).max()


def test_pcg_matches_direct_solve_on_tiny_grid():
    inst = W.random_instance(2, 3, (4, 4, 2), "sym", "taps", seed=21)
    Ahat = O.coefficient_modes(inst)
    Q = O.dense_Q(inst.P, inst.N, Ahat)
    F = O.corrector_rhs(inst.P, inst.N, Ahat, 0)
    U_direct = np.zeros(Q.shape[0], complex)
    U_direct[1:] = np.linalg.solve(Q[1:, 1:], F.reshape(-1)[1:])
    op = O.Operator(inst)
    for M in (O.jacobi_inverse(inst.P, inst.N, Ahat), O.frobenius_diag(inst.P, inst.N, Ahat)):
        U, info = O.pcg(op, F, M, tol=1e-14)
        assert info["status"] == "ok" and info["rel_residual"] <= 1e-13
        assert np.abs(U.reshape(-1) - U_direct).max() <= 1e-11 * np.abs(U_direct).max()


def test_frobenius_preconditioner_is_the_least_squares_optimum():
    """eq. precond: each M_jj minimises ||Q e_j M_jj - e_j||; solve that 1-unknown least-squares by lstsq."""
    inst = W.random_instance(2, 2, (4, 6), "sym", "taps", seed=8)
    Ahat = O.coefficient_modes(inst)
    Q = O.dense_Q(inst.P, inst.N, Ahat)
    M = O.frobenius_diag(inst.P, inst.N, Ahat).reshape(-1)
    D = Q.shape[0]
    for j in range(1, D):
        e = np.zeros(D, complex)
        e[j] = 1
        m, *_ = np.linalg.lstsq(Q[:, j:j + 1], e, rcond=None)
        assert abs(m[0] - M[j]) <= 1e-12 * abs(M[j])
    # column norms by the O(gD) tap formula equal the dense ones
    cn = O.column_norms2(inst.P, inst.N, Ahat).reshape(-1)
    assert np.allclose(cn, (np.abs(Q) ** 2).sum(axis=0), rtol=1e-12, atol=0)


# ------------------------------------------------------------------------------ P1, P2: one dimension

@pytest.mark.parametrize("n,N,repr_", [(2, 8, "taps"), (2, 12, "grid"), (3, 6, "taps"), (2, 16, "grid")])
def test_p1_one_dimension_harmonic_mean(n, N, repr_):
    """d = 1: the discrete equation forces a (1 + u') = const on the grid, so a*_N = 1/mean_grid(1/a)."""
    inst = W.random_instance(1, n, N, "scalar", repr_, seed=100 + n + N, nonlinear=(repr_ == "grid"))
    A, Us, infos, Ac = O.homogenized(inst, tol=1e-13)
    a = O.coefficient_grid(inst)[0, 0]
    ref = 1.0 / np.mean(1.0 / a)
    assert abs(A[0, 0] - ref) <= 1e-12 * ref
    assert abs(Ac[0, 0].imag) <= 1e-14 * ref


def test_p2_cfg0_closed_form():
    """a = 3 + cos th1 + cos th2: <1/a> = (1/2pi) int dth / sqrt((3 + cos th)^2 - 1), using the textbook
    (1/2pi) int dphi/(c + cos phi) = 1/sqrt(c^2 - 1) for c > 1; the torus is equidistributed (Lemma on
    consistent Fourier coefficients), so a* = 1/<1/a>."""
    from scipy.integrate import quad
    import warnings
    warnings.simplefilter("ignore")
    val, err = quad(lambda t: 1.0 / math.sqrt((3.0 + math.cos(t)) ** 2 - 1.0), 0.0, 2.0 * math.pi,
                    epsabs=1e-15, epsrel=1e-15, limit=200)
    astar_exact = 1.0 / (val / (2.0 * math.pi))
    inst = W.cfg0()
    A, Us, infos, _ = O.homogenized(inst)
    assert infos[0]["status"] == "ok" and infos[0]["rel_residual"] <= 1e-12
    assert abs(A[0, 0] - astar_exact) <= 1e-13 * astar_exact
    # one-dimensional Jacobi-PCG converges in a handful of iterations (P11 bounds the spectrum)
    assert infos[0]["iterations"] < 60


# ------------------------------------------------------------------------------ P3: Keller-Dykhne

@pytest.mark.parametrize("N", [8, 12])
def test_p3_keller_dykhne_periodic(N):
    """P = I, a = exp(eps (cos th1 - cos th2)): a(R x) = 1/a(x) under a quarter turn, so A* = I (2D duality)."""
    y = 2 * np.pi * np.arange(N) / N
    Y1, Y2 = np.meshgrid(y, y, indexing="ij")
    a = np.exp(0.5 * (np.cos(Y1) - np.cos(Y2)))
    inst = _inst(np.eye(2), (N, N), "scalar", grid=a[None].copy(), tol=1e-13)
    A, Us, infos, _ = O.homogenized(inst)
    assert np.abs(A - np.eye(2)).max() <= 1e-11


def test_p3_keller_dykhne_quasiperiodic():
    N = 6
    P = np.array([[1.0, W.SQRT2, 0, 0], [0, 0, 1.0, W.SQRT2]])
    y = 2 * np.pi * np.arange(N) / N
    Y = np.meshgrid(y, y, y, y, indexing="ij")
    a = np.exp(0.5 * (np.cos(Y[0]) + np.cos(Y[1]) - np.cos(Y[2]) - np.cos(Y[3])))
    inst = _inst(P, (N,) * 4, "scalar", grid=a[None].copy(), tol=1e-13)
    A, Us, infos, _ = O.homogenized(inst)
    assert np.abs(A - np.eye(2)).max() <= 1e-11


# ------------------------------------------------------------------------------ P4: laminate

def test_p4_laminate():
    """a depends on theta_1 only, and column 1 of P is e_1: a* is diag(harmonic mean, arithmetic mean)."""
    rng = np.random.default_rng(7)
    modes = {(0, 0, 0, 0): [4.0]}
    for m in (1, 2, 3):
        c = 0.4 * (rng.standard_normal() + 1j * rng.standard_normal())
        modes[(m, 0, 0, 0)] = [c]
        modes[(-m, 0, 0, 0)] = [np.conj(c)]
    k, v = W.taps_from_dict({kk: np.array(vv, complex) for kk, vv in modes.items()}, 4, 1)
    N = 8
    inst = _inst(W.P_CFG1, (N,) * 4, "scalar", taps=(k, v), tol=1e-13)
    A, Us, infos, _ = O.homogenized(inst)
    a1 = W.sample_on_grid((N,), k[:, :1], v)[0]
    assert abs(A[0, 0] - 1.0 / np.mean(1.0 / a1)) <= 1e-12 * A[0, 0]
    assert abs(A[1, 1] - 4.0) <= 1e-14 * 4
    assert abs(A[0, 1]) <= 1e-14 and abs(A[1, 0]) <= 1e-14
    assert infos[1]["iterations"] == 0      # the e_2 right-hand side vanishes


# ------------------------------------------------------------------------------ P5: constant coefficient

def test_p5_constant_coefficient_is_diagonal():
    c = 2.5
    k = np.zeros((1, 3), np.int32)
    v = np.array([[c]], complex)
    P = W.random_P(2, 3, 1)
    N = (4, 4, 6)
    inst = _inst(P, N, "scalar", taps=(k, v), tol=1e-14)
    Ahat = O.coefficient_modes(inst)
    Q = O.dense_Q(P, N, Ahat)
    lam = O.lambdas(P, N)
    l2 = (lam ** 2).sum(axis=0).reshape(-1)
    assert np.abs(Q - np.diag(c * l2)).max() <= 1e-13 * c * l2.max()
    rng = np.random.default_rng(2)
    F = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    F.reshape(-1)[0] = 0
    U, info = O.pcg(O.Operator(inst), F, O.jacobi_inverse(P, N, Ahat), tol=1e-14)
    assert info["iterations"] == 1
    Uex = np.zeros(N, complex)
    Uex.reshape(-1)[1:] = F.reshape(-1)[1:] / (c * l2[1:])
    assert np.abs(U - Uex).max() <= 1e-14 * np.abs(Uex).max()
    A, *_ = O.homogenized(inst)
    assert np.abs(A - c * np.eye(2)).max() <= 1e-14


# ------------------------------------------------------------------------------ P6: manufactured solutions

@pytest.mark.parametrize("which", ["cfg0", "cfg1"])
def test_p6_manufactured_solution(which):
    inst = getattr(W, which)()
    modes, amps = W.manufactured_modes(inst.n, inst.meta["manufactured_kmax"], inst.meta["manufactured_seed"])
    F = O.manufactured_rhs(inst.P, inst.coeff.taps_k, inst.coeff.taps_val, "scalar", inst.d, modes, amps, inst.N)
    Uex = O.modes_to_array(modes, amps, inst.N)
    op = O.Operator(inst)
    M = O.jacobi_inverse(op.P, op.N, op.Ahat)
    U, info = O.pcg(op, F, M, tol=1e-13)
    assert info["status"] == "ok"
    assert np.linalg.norm(U - Uex) <= 1e-11 * np.linalg.norm(Uex)


def test_p12_paper_table2_errors():
    """(alpha_1, u_1) of Sec. 5.1.1 with P = 2 pi (1, sqrt2): the printed C-PCG errors are at rounding level
    for N >= 8; the oracle reproduces that level (it must be tiny, not a specific digit)."""
    g = json.load(open(os.path.join(GOLDEN, "table2_pm_efficiency.json")))
    P = 2 * np.pi * np.array([[1.0, W.SQRT2]])
    k, v = W.cos_sum_taps(2, 6.0, 1.0)
    # u_1 parent: sin th1 + sin th2 = sum over +-e_j of -+ i/2 e^{+-i th_j}
    modes = np.array([(1, 0), (-1, 0), (0, 1), (0, -1)])
    amps = np.array([-0.5j, 0.5j, -0.5j, 0.5j])
    for N, e_paper in zip(g["N"][:3], g["e_N_C_PCG"][:3]):
        inst = _inst(P, (N, N), "scalar", taps=(k, v), tol=1e-14)
        F = O.manufactured_rhs(P, k, v, "scalar", 1, modes, amps, (N, N))
        op = O.Operator(inst)
        U, info = O.pcg(op, F, O.jacobi_inverse(op.P, op.N, op.Ahat), tol=1e-14)
        e_N = np.linalg.norm(U - O.modes_to_array(modes, amps, (N, N)))   # Parseval, eq. parseval
        assert e_N <= 10 * max(e_paper, 1e-16) + 1e-15


# ------------------------------------------------------------------------------ P8, P9, P10

@pytest.mark.parametrize("kind,seed", [("scalar", 1), ("diag", 2), ("sym", 3)])
def test_p8_voigt_reuss_and_p9_energy_form(kind, seed):
    inst = W.random_instance(2, 3, (6, 6, 4), kind, "taps", seed=seed)
    A, Us, infos, Ac = O.homogenized(inst, tol=1e-13)
    Agrid = O.coefficient_grid(inst)
    d = 2
    field_ = np.moveaxis(Agrid.reshape(d, d, -1), -1, 0)          # (D, d, d)
    voigt = field_.mean(axis=0)
    reuss = np.linalg.inv(np.linalg.inv(field_).mean(axis=0))
    # A* = A~_0 - F^H Q^{-1} F is Hermitian; its imaginary part comes only from the literal Nyquist modes
    # (k_j = -N/2 has no partner +N/2 in K_N^n), and is tiny once the corrector is resolved.
    assert np.abs(Ac - Ac.conj().T).max() <= 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(voigt - A).min() >= -1e-12
    assert np.linalg.eigvalsh(A - reuss).min() >= -1e-12
    E = O.homogenized_energy(inst.P, inst.N, Agrid, Us)
    assert np.abs(E - Ac).max() <= 1e-12 * np.abs(A).max()


def test_p10_scale_and_axis_permutation_invariance():
    inst = W.random_instance(2, 3, (6, 4, 6), "sym", "taps", seed=9)
    A, *_ = O.homogenized(inst, tol=1e-13)
    inst_s = W.Instance("s", 2 * np.pi * inst.P, inst.N, inst.coeff)
    As, *_ = O.homogenized(inst_s, tol=1e-13)
    assert np.abs(As - A).max() <= 1e-11 * np.abs(A).max()
    perm = [2, 0, 1]
    c = inst.coeff
    inst_p = W.Instance("p", inst.P[:, perm], tuple(inst.N[p] for p in perm),
                        W.Coefficient(c.kind, np.ascontiguousarray(c.taps_k[:, perm]), c.taps_val))
    Ap, *_ = O.homogenized(inst_p, tol=1e-13)
    assert np.abs(Ap - A).max() <= 1e-11 * np.abs(A).max()


def test_p10_identity_projection_is_the_periodic_spectral_method():
    """P = I, d = n = 1 is a periodic 1D problem: a* = harmonic mean, U solves (a (1 + u'))' = 0 exactly."""
    k, v = W.random_taps(1, 1, "scalar", seed=4, radius=3)
    inst = _inst(np.eye(1), (16,), "scalar", taps=(k, v), tol=1e-14)
    A, Us, infos, _ = O.homogenized(inst)
    a = W.sample_on_grid((16,), k, v)[0]
    assert abs(A[0, 0] - 1 / np.mean(1 / a)) <= 1e-13 * A[0, 0]
    # flux a (1 + u') is constant on the grid
    kk = O.signed_k(16).astype(float)
    du = np.fft.ifft(1j * kk * Us[0]) * 16
    flux = a * (1 + du)
    assert np.abs(flux - flux.mean()).max() <= 1e-12 * abs(flux.mean())


# ------------------------------------------------------------------------------ P11: Jacobi spectrum, d = 1

@pytest.mark.parametrize("N", [4, 6, 8])
def test_p11_jacobi_spectrum_one_dimension(N):
    """d = 1, scalar a > 0: J^{-1/2} Q J^{-1/2} on k != 0 has its spectrum in [min a, max a] / A~_0."""
    inst = W.random_instance(1, 2, (N, N), "scalar", "taps", seed=N)
    Ahat = O.coefficient_modes(inst)
    Q = O.dense_Q(inst.P, inst.N, Ahat)[1:, 1:]
    J = O.jacobi_diag(inst.P, inst.N, Ahat).reshape(-1)[1:]
    S = Q / np.sqrt(np.outer(J, J))
    ev = np.linalg.eigvalsh(S)
    a = O.coefficient_grid(inst)[0, 0]
    a0 = Ahat[(0, 0) + (0, 0)].real
    assert ev.min() >= a.min() / a0 - 1e-12 and ev.max() <= a.max() / a0 + 1e-12


# ------------------------------------------------------------------------------ right-hand side and a* formulas

def test_corrector_rhs_and_flux_formula_against_grid_definitions():
    """F_j = Fourier coefficients of div(A e_j) and A*_ij = grid mean of e_i^T A (e_j + grad u_j), computed here
    on the grid by finite sums of exponentials (independent of the oracle's Fourier-side formulas)."""
    inst = W.random_instance(2, 2, (6, 4), "sym", "taps", seed=31)
    N = inst.N
    D = int(np.prod(N))
    Ahat = O.coefficient_modes(inst)
    k, v = inst.coeff.taps_k, inst.coeff.taps_val
    P = inst.P
    # div(A e_j) at the nodes: sum_a d/dx_a A^{aj}; for a tap m, d/dx_a e^{i m.th(x)} = i (P m)_a e^{...}
    pairs = {(0, 0): 0, (0, 1): 1, (1, 0): 1, (1, 1): 2}
    for j in range(2):
        div = np.zeros(N, complex)
        for m, val in zip(k, v):
            lam_m = P @ m.astype(float)
            coef = sum(1j * lam_m[a] * val[pairs[(a, j)]] for a in range(2))
            ph =np.exp(1j * sum(float(m[t]) * (2 * np.pi * np.arange(N[t]) / N[t]).reshape(
                [-1 if s == t else 1 for s in range(2)]) for t in range(2)))
            div += coef * ph
        Fj = np.fft.fftn(div) / D
        Fj.reshape(-1)[0] = 0
        assert np.abs(O.corrector_rhs(P, N, Ahat, j) - Fj).max() <= 1e-13 * np.abs(Fj).max()
    rng = np.random.default_rng(0)
    Us = [rng.standard_normal(N) + 1j * rng.standard_normal(N) for _ in range(2)]
    for U in Us:
        U.reshape(-1)[0] = 0
    Ac = O.homogenized_from_correctors(P, N, Ahat, Us)
    Agrid = O.coefficient_grid(inst)
    lam = O.lambdas(P, N)
    for i in range(2):
        for j in range(2):
            grad = [np.fft.ifftn(1j * lam[b] * Us[j]) * D for b in range(2)]
            val = np.mean(Agrid[i, j] + sum(Agrid[i, b] * grad[b] for b in range(2)))
            assert abs(Ac[i, j] - val) <= 1e-12 * abs(val)


def test_pointwise_apply_matches_vectorised_convolution():
    """apply_taps_at (used for sampled checks at full size) agrees with the vectorised convolution."""
    inst = W.random_instance(2, 3, (6, 4, 8), "sym", "taps", seed=17)
    rng = np.random.default_rng(1)
    h = rng.standard_normal(inst.N) + 1j * rng.standard_normal(inst.N)
    w = O.apply_convolution(inst.P, inst.N, O.coefficient_modes(inst), h)
    pts = [tuple(int(rng.integers(0, Nj)) for Nj in inst.N) for _ in range(20)] + [(0, 0, 0), (5, 3, 7), (3, 2, 4)]
    wp = O.apply_taps_at(inst.P, inst.N, inst.coeff.taps_k, inst.coeff.taps_val, "sym", h, pts)
    assert np.abs(wp - np.array([w[p] for p in pts])).max() <= 1e-12 * np.abs(w).max()


# ------------------------------------------------------------------------------ Nyquist-free variant

@pytest.mark.parametrize("N", [(4, 6), (3, 4, 5), (2, 2, 3)])
def test_nyquist_free_mask_is_the_symmetric_index_set(N):
    keep = O.nyquist_free_mask(N)
    assert keep.sum() == np.prod([Nj - (1 - Nj % 2) for Nj in N])
    # closed under k -> -k: storage index i -> (-i) mod N on every axis
    flip = np.roll(np.flip(keep, axis=tuple(range(len(N)))), 1, axis=tuple(range(len(N))))
    assert np.array_equal(keep, flip)
    kg = O.k_grids(N)
    assert np.all(np.abs(kg[:, keep]) < np.asarray(N)[:, None] / 2.0)


def test_nyquist_free_is_the_full_scheme_on_odd_grids():
    inst = W.random_instance(2, 3, (5, 3, 7), "sym", "grid", seed=31, nonlinear=True)
    A1, _, _, Ac1 = O.homogenized(inst, tol=1e-13)
    A2, _, _, Ac2 = O.homogenized_nyquist_free(inst, tol=1e-13)
    assert np.abs(Ac1 - Ac2).max() <= 1e-14 * np.abs(A1).max()


@pytest.mark.parametrize("d,n,N,kind", [(1, 2, (6, 4), "scalar"), (2, 3, (4, 6, 4), "sym"), (2, 2, (6, 6), "diag")])
def test_nyquist_free_solution_against_dense_restriction(d, n, N, kind):
    """Q' = the principal submatrix of the dense Q (Alg. 1) on K'_N, solved directly, equals the oracle's
    restricted PCG; the solution is conjugate-symmetric, U(-k) = conj(U(k)), and a* is real. The full scheme on
    the same grid breaks both at the Nyquist modes (full-support grid coefficient), so the pin sees the
    restriction."""
    inst = W.random_instance(d, n, N, kind, "grid", seed=7 + d, nonlinear=True)
    Ahat = O.coefficient_modes(inst)
    Q = O.dense_Q(inst.P, N, Ahat)
    keep = O.nyquist_free_mask(N).reshape(-1)
    idx = np.nonzero(keep)[0][1:]                      # K'_N without k = 0
    A, Us, infos, Ac = O.homogenized_nyquist_free(inst, tol=1e-14)
    axes = tuple(range(len(N)))
    for j in range(d):
        F = O.corrector_rhs(inst.P, N, Ahat, j).reshape(-1)
        U_direct = np.zeros(Q.shape[0], complex)
        U_direct[idx] = np.linalg.solve(Q[np.ix_(idx, idx)], F[idx])
        U = Us[j].reshape(-1)
        assert np.abs(U - U_direct).max() <= 1e-11 * np.abs(U_direct).max()
        Um = np.roll(np.flip(Us[j], axis=axes), 1, axis=axes)          # U(-k) at index k
        assert np.abs(Um - np.conj(Us[j])).max() <= 1e-11 * np.abs(U_direct).max()
    assert np.abs(Ac.imag).max() <= 1e-13 * np.abs(A).max()
    _, Us_full, _, Ac_full = O.homogenized(inst, tol=1e-14)
    Um = np.roll(np.flip(Us_full[0], axis=axes), 1, axis=axes)
    assert np.abs(Um - np.conj(Us_full[0])).max() > 1e-8 * np.abs(Us_full[0]).max()


@pytest.mark.parametrize("kind,seed", [("scalar", 2), ("sym", 4)])
def test_nyquist_free_variational_bounds(kind, seed):
    """The restricted trial space is a subspace of the full one, so the restricted a* (minimum energy over it)
    lies between the full scheme's a* and the grid mean of A (the Voigt bound): A*_full <= A*' <= <A>."""
    inst = W.random_instance(2, 3, (6, 4, 6), kind, "grid", seed=seed, nonlinear=True)
    A_full, *_ = O.homogenized(inst, tol=1e-14)
    A_nf, *_ = O.homogenized_nyquist_free(inst, tol=1e-14)
    Agrid = O.coefficient_grid(inst)
    voigt = np.moveaxis(Agrid.reshape(2, 2, -1), -1, 0).mean(axis=0)
    assert np.linalg.eigvalsh(A_nf - A_full).min() >= -1e-12
    assert np.linalg.eigvalsh(voigt - A_nf).min() >= -1e-12
    assert np.abs(A_nf - A_full).max() > 1e-10          # the Nyquist modes carry energy here
