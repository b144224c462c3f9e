"""Plain FP64 CPU oracle of the projection method's hot path (Jiang, Li, Zhang & Zhang, arXiv 2404.06841).

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or run this module. The CUDA library never calls it and shares no code with it; the
two meet only in the seeded inputs of ``qp_workloads``.

What it computes, each step written out from the paper, in double precision, slow and obvious:

* index sets and the tensor-vector index conversion (Sec. 2.3 K_N^n; Sec. 3.1.2 eqs. conversion and
  inverse_convert);
* Fourier exponents lambda_k = P k (Sec. 2.1, eq. continuous_FS);
* the coefficient's discrete Fourier coefficients A~ (Sec. 3.1.1, taken from grid samples with the 1/D
  normalisation of Sec. 2.3);
* the stiffness operator of the discrete scheme, eq. n-discrete_equation, generalised to a matrix
  coefficient as in App. D (Q = sum_ab diag(lambda_a) C(A~^{ab}) diag(lambda_b)), three independent ways:
  entry by entry (Alg. 1, tiny grids), as an explicit wraparound convolution over the coefficient's nonzero
  modes (the compressed mat-vec of Sec. 4.2), and through the n-dimensional DFT (the multilevel circulant
  structure of Sec. 4.1 is diagonalised by it);
* the diagonal preconditioners: Jacobi (the diagonal of Q) and the Frobenius-optimal one of eq. precond /
  eq. preconditioner (Sec. 4.3);
* C-PCG, Algorithm 2;
* the corrector right-hand side (Sec. 5.2 eq. corrector; App. D, f_1 = d alpha / d x_1) and the homogenized
  coefficient of eq. homcoefficient, as a torus (grid) average;
* the Nyquist-free variant of the scheme (not in the paper: the definition behind the library's half-spectrum
  storage): the same Galerkin scheme restricted to the modes with no k_j = -N_j/2, a set closed under k -> -k.

Readings of places where the paper is silent or garbled (each is also listed in the design notes):
Nyquist modes k_j = -N/2 are kept with lambda = P k literally; k = 0 is excluded (U_0 = 0, row 0 of Q h is 0);
"solve M z = r" is read z = M r (M approximates Q^{-1}, eq. precond); q_ij^2 is |q_ij|^2 for complex Q;
inner products are Hermitian, (x, y) = sum conj(x) y; PCG stops on the recursive residual
||r||_2 <= tol ||F||_2 over Fourier coefficients (Parseval, eq. parseval) and reports the true residual.

Parity status: every function here is pinned by tests/test_oracle_pins.py (closed forms, brute force,
invariants and the paper's printed values).
"""
from __future__ import annotations

import itertools
import time

import numpy as np


# ------------------------------------------------------------------------------------ index conventions

def signed_k(Nj: int) -> np.ndarray:
    """k for storage index ibar = 0..Nj-1: ibar if ibar < Nj/2 else ibar - Nj (Sec. 3.1.2, eq. inverse_convert)."""
    ibar = np.arange(Nj)
    return np.where(ibar < Nj / 2.0, ibar, ibar - Nj).astype(np.int64)


def tensor_to_vector_index(kvec, N) -> int:
    """Sec. 3.1.2, eq. conversion: i = sum_k ibar_k prod_{t>k} N_t with ibar_k = i_k mod N_k."""
    i = 0
    for k, (ik, Nk) in enumerate(zip(kvec, N)):
        ibar = int(ik) % int(Nk)
        i += ibar * int(np.prod(N[k + 1:], dtype=np.int64))
    return i


def vector_to_tensor_index(i: int, N) -> tuple:
    """Sec. 3.1.2, eq. inverse_convert: ibar_k = floor((i mod prod_{t>=k} N_t) / prod_{t>k} N_t), then
    i_k = ibar_k if ibar_k < N_k/2 else ibar_k - N_k."""
    out = []
    for k, Nk in enumerate(N):
        hi = int(np.prod(N[k:], dtype=np.int64))
        lo = int(np.prod(N[k + 1:], dtype=np.int64))
        ibar = (i % hi) // lo
        out.append(ibar if ibar < Nk / 2.0 else ibar - Nk)
    return tuple(out)


def k_grids(N):
    """The n integer arrays k_j over the whole tensor, shape (n, *N), storage in fftfreq order."""
    return np.stack(np.meshgrid(*[signed_k(int(Nj)) for Nj in N], indexing="ij"))


def lambdas(P, N) -> np.ndarray:
    """Fourier exponents lambda_a(k) = sum_j P_aj k_j over the grid, shape (d, *N) (Sec. 2.1; Sec. 2.3)."""
    P = np.asarray(P, dtype=np.float64)
    kg = k_grids(N).astype(np.float64)
    return np.einsum("aj,j...->a...", P, kg)


# ------------------------------------------------------------------------------------ coefficient

def _pairs(kind: str, d: int):
    """Stored component c -> list of (a, b) entries it fills in the symmetric d x d coefficient."""
    if kind == "scalar":
        return [[(a, a) for a in range(d)]]
    if kind == "diag":
        return [[(a, a)] for a in range(d)]
    if kind == "sym":
        out = []
        for a in range(d):
            for b in range(a, d):
                out.append([(a, b)] if a == b else [(a, b), (b, a)])
        return out
    raise ValueError(kind)


def coefficient_modes(inst) -> np.ndarray:
    """A~^{ab}_k for k in K_N^n, shape (d, d, *N) complex, storage index = k mod N.

    Taps are scattered to their index m mod N. Grid samples are transformed as in Sec. 3.1.1:
    A~_k = (1/D) sum_j A(y_j) exp(-i k.y_j).
    """
    d, N = inst.d, tuple(inst.N)
    D = int(np.prod(N))
    out = np.zeros((d, d) + N, dtype=np.complex128)
    c = inst.coeff
    pairs = _pairs(c.kind, d)
    if c.taps_k is not None:
        for m, val in zip(c.taps_k, c.taps_val):
            idx = tuple(int(mj) % int(Nj) for mj, Nj in zip(m, N))
            for comp, entries in enumerate(pairs):
                for (a, b) in entries:
                    out[(a, b) + idx] += val[comp]
    else:
        for comp, entries in enumerate(pairs):
            hat = np.fft.fftn(c.grid[comp]) / D
            for (a, b) in entries:
                out[(a, b)] += hat
    return out


def coefficient_grid(inst) -> np.ndarray:
    """A^{ab}(y_j) on the grid, shape (d, d, *N) real. Taps are summed at the nodes directly."""
    d, N = inst.d, tuple(inst.N)
    c = inst.coeff
    pairs = _pairs(c.kind, d)
    if c.grid is not None:
        g = c.grid
    else:
        g = np.zeros((len(pairs),) + N, dtype=np.complex128)
        ys = [2.0 * np.pi * np.arange(int(Nj)) / int(Nj) for Nj in N]
        Y = np.meshgrid(*ys, indexing="ij")
        for m, val in zip(c.taps_k, c.taps_val):
            ph = np.exp(1j * sum(float(mj) * Yj for mj, Yj in zip(m, Y)))
            for comp in range(len(pairs)):
                g[comp] += val[comp] * ph
        g = g.real
    out = np.zeros((d, d) + N, dtype=np.float64)
    for comp, entries in enumerate(pairs):
        for (a, b) in entries:
            out[(a, b)] += g[comp]
    return out


def nonzero_modes(Ahat: np.ndarray, rel: float = 0.0):
    """Storage indices (tuples) where any A~^{ab} is nonzero."""
    mag = np.abs(Ahat).reshape((-1,) + Ahat.shape[2:]).max(axis=0)
    thr = rel * float(mag.max()) if rel > 0 else 0.0
    return [tuple(int(x) for x in idx) for idx in zip(*np.nonzero(mag > thr))]


# ------------------------------------------------------------------------------------ stiffness operator

def dense_Q(P, N, Ahat) -> np.ndarray:
    """Q = A o W entry by entry, Alg. 1 (compressed storage rule): for row i <- k_V and column j <- k_U,
    A_ij = A~_{k_V -N k_U}, W_ij = (P k_V)^T (P k_U); for a matrix coefficient (App. D)
    Q_ij = sum_ab lambda_a(k_V) A~^{ab}_{k_V -N k_U} lambda_b(k_U). Tiny grids only (D x D dense)."""
    N = tuple(int(x) for x in N)
    D = int(np.prod(N))
    P = np.asarray(P, dtype=np.float64)
    d = P.shape[0]
    ks = [vector_to_tensor_index(i, N) for i in range(D)]
    lam = [P @ np.array(k, dtype=np.float64) for k in ks]
    Q = np.zeros((D, D), dtype=np.complex128)
    for i in range(D):
        for j in range(D):
            kA = tuple((ks[i][t] - ks[j][t]) % N[t] for t in range(len(N)))
            s = 0.0 + 0.0j
            for a in range(d):
                for b in range(d):
                    s += lam[i][a] * Ahat[(a, b) + kA] * lam[j][b]
            Q[i, j] = s
    return Q


def apply_convolution(P, N, Ahat, h, modes=None) -> np.ndarray:
    """w = Q h as an explicit wraparound convolution over the coefficient's nonzero modes m (Sec. 4.2):
    w(k) = sum_ab lambda_a(k) sum_m A~^{ab}_m lambda_b(k -N m) h(k -N m).

    ``h`` has shape (*N) complex (storage index = k mod N). np.roll by m along every axis realises k -N m.
    """
    N = tuple(int(x) for x in N)
    lam = lambdas(P, N)
    d = lam.shape[0]
    if modes is None:
        modes = nonzero_modes(Ahat)
    axes = tuple(range(len(N)))
    w = np.zeros(N, dtype=np.complex128)
    g = [lam[b] * h for b in range(d)]                      # lambda_b h
    for m in modes:
        shift = tuple(int(x) for x in m)
        rolled = [np.roll(g[b], shift, axis=axes) for b in range(d)]
        for a in range(d):
            acc = np.zeros(N, dtype=np.complex128)
            for b in range(d):
                coef = Ahat[(a, b) + shift]
                if coef != 0:
                    acc += coef * rolled[b]
            w += lam[a] * acc
    return w


def apply_fft(P, N, Agrid, h) -> np.ndarray:
    """w = Q h through the n-dimensional DFT: gradient i lambda_b h, inverse DFT to the grid, pointwise product
    with A^{ab}(y_j), forward DFT, divergence -i lambda_a. The i and -i cancel:
    w = sum_a lambda_a fftn( sum_b A^{ab}(y) ifftn(lambda_b h) ) with numpy's normalisation (ifftn carries 1/D).
    Equal to apply_convolution when A~ = fftn(A)/D (the DFT diagonalises the multilevel circulant A, Sec. 4.1)."""
    N = tuple(int(x) for x in N)
    lam = lambdas(P, N)
    d = lam.shape[0]
    grads = [np.fft.ifftn(lam[b] * h) for b in range(d)]
    w = np.zeros(N, dtype=np.complex128)
    for a in range(d):
        flux = np.zeros(N, dtype=np.complex128)
        for b in range(d):
            flux += Agrid[a, b] * grads[b]
        w += lam[a] * np.fft.fftn(flux)
    return w


def apply_taps_at(P, N, taps_k, taps_val, kind, h, points) -> np.ndarray:
    """w(k) of eq. n-discrete_equation at the given storage points only, one plain sum per point:
    w(k) = sum over taps m of sum_ab lambda_a(k) A~^{ab}_m lambda_b(k -N m) h(k -N m), lambda = P k.
    ``h`` may be any array indexable by storage tuples (e.g. a memory-mapped full-size vector); ``points`` is a
    list of storage index tuples. For sampled checks at sizes the vectorised operator cannot hold."""
    P = np.asarray(P, dtype=np.float64)
    d = P.shape[0]
    N = tuple(int(x) for x in N)
    pairs = _pairs(kind, d)
    mats = []
    for val in taps_val:
        Am = np.zeros((d, d), dtype=np.complex128)
        for comp, entries in enumerate(pairs):
            for (a, b) in entries:
                Am[a, b] += val[comp]
        mats.append(Am)
    out = np.zeros(len(points), dtype=np.complex128)
    for q, idx in enumerate(points):
        k = np.array([signed_k(Nj)[i] for i, Nj in zip(idx, N)], dtype=np.float64)
        lk = P @ k
        s = 0.0 + 0.0j
        for m, Am in zip(taps_k, mats):
            idx2 = tuple((int(i) - int(mj)) % Nj for i, mj, Nj in zip(idx, m, N))
            k2 = np.array([signed_k(Nj)[i] for i, Nj in zip(idx2, N)], dtype=np.float64)
            s += (lk @ Am @ (P @ k2)) * h[idx2]
        out[q] = s
    return out


class Operator:
    """The stiffness operator of one instance, applied by convolution (taps) or by the DFT (grid)."""

    def __init__(self, inst, method: str | None = None):
        self.inst = inst
        self.P = np.asarray(inst.P, dtype=np.float64)
        self.N = tuple(int(x) for x in inst.N)
        self.Ahat = coefficient_modes(inst)
        if method is None:
            method = "conv" if inst.coeff.taps_k is not None else "fft"
        self.method = method
        if method == "fft":
            self.Agrid = coefficient_grid(inst)
        else:
            self.modes = nonzero_modes(self.Ahat)
        self.lam = lambdas(self.P, self.N)

    def __call__(self, h):
        if self.method == "fft":
            return apply_fft(self.P, self.N, self.Agrid, h)
        return apply_convolution(self.P, self.N, self.Ahat, h, self.modes)


# ------------------------------------------------------------------------------------ preconditioners

def jacobi_diag(P, N, Ahat) -> np.ndarray:
    """q_kk = sum_ab lambda_a(k) A~^{ab}_0 lambda_b(k), the diagonal of Q (real for Hermitian Q)."""
    lam = lambdas(P, N)
    d = lam.shape[0]
    zero = (0,) * len(N)
    q = np.zeros(lam.shape[1:], dtype=np.float64)
    for a in range(d):
        for b in range(d):
            q += (lam[a] * Ahat[(a, b) + zero] * lam[b]).real
    return q


def column_norms2(P, N, Ahat, modes=None) -> np.ndarray:
    """||Q e_j||_2^2 for every column j <- k_U: column j holds, at row k_V = k_U +N m, the entry
    sum_ab lambda_a(k_V) A~^{ab}_m lambda_b(k_U); sum |.|^2 over the nonzero modes m (Prop. in Sec. 4.3, O(gD))."""
    N = tuple(int(x) for x in N)
    lam = lambdas(P, N)
    d = lam.shape[0]
    if modes is None:
        modes = nonzero_modes(Ahat)
    axes = tuple(range(len(N)))
    out = np.zeros(N, dtype=np.float64)
    for m in modes:
        neg = tuple(-int(x) for x in m)
        lamV = [np.roll(lam[a], neg, axis=axes) for a in range(d)]      # lambda_a(k_U +N m) at index k_U
        e = np.zeros(N, dtype=np.complex128)
        for a in range(d):
            for b in range(d):
                coef = Ahat[(a, b) + tuple(int(x) for x in m)]
                if coef != 0:
                    e += lamV[a] * coef * lam[b]
        out += np.abs(e) ** 2
    return out


def frobenius_diag(P, N, Ahat, modes=None) -> np.ndarray:
    """M = diag(q_jj / ||Q e_j||^2), eq. preconditioner; M_00 = 0 (0/0 at k = 0, the excluded mode)."""
    q = jacobi_diag(P, N, Ahat)
    cn = column_norms2(P, N, Ahat, modes)
    out = np.zeros_like(q)
    nz = cn > 0
    out[nz] = q[nz] / cn[nz]
    return out


def jacobi_inverse(P, N, Ahat) -> np.ndarray:
    """The Jacobi preconditioner as z = M r with M = diag(1/q_kk), and M_00 = 0."""
    q = jacobi_diag(P, N, Ahat)
    out = np.zeros_like(q)
    nz = q != 0
    out[nz] = 1.0 / q[nz]
    flat = out.reshape(-1)
    flat[0] = 0.0
    return out


# ------------------------------------------------------------------------------------ C-PCG (Algorithm 2)

def hdot(x, y) -> complex:
    """Hermitian inner product (x, y) = sum conj(x) y."""
    return complex(np.vdot(x.reshape(-1), y.reshape(-1)))


def pcg(apply, F, Mdiag, tol: float, maxit: int = 10000, U0=None):
    """Algorithm 2 (C-PCG) with z = M r, stopping when ||r_j|| <= tol ||F||.

    Returns (U, info) with info = {iterations, rel_residual (true, recomputed), status}.
    The k = 0 entry of F is ignored and U_0 = 0 (Sec. 3.1.1, the test space excludes the mean).
    """
    F = np.array(F, dtype=np.complex128)
    F.reshape(-1)[0] = 0.0
    nF = np.sqrt(hdot(F, F).real)
    U = np.zeros_like(F) if U0 is None else np.array(U0, dtype=np.complex128)
    U.reshape(-1)[0] = 0.0
    if nF == 0.0:
        return np.zeros_like(F), {"iterations": 0, "rel_residual": 0.0, "status": "ok"}
    r = F - apply(U)
    z = Mdiag * r
    h = z.copy()
    rz = hdot(r, z).real
    it = 0
    status = "no_convergence"
    if np.sqrt(hdot(r, r).real) <= tol * nF:
        status = "ok"
    else:
        while it < maxit:
            w = apply(h)
            hw = hdot(h, w).real
            if not hw > 0.0:
                status = "breakdown"
                break
            alpha = rz / hw
            U = U + alpha * h
            r = r - alpha * w
            it += 1
            if np.sqrt(hdot(r, r).real) <= tol * nF:
                status = "ok"
                break
            z = Mdiag * r
            rz_new = hdot(r, z).real
            beta = rz_new / rz
            rz = rz_new
            h = z + beta * h
    U.reshape(-1)[0] = 0.0
    rt = F - apply(U)
    return U, {"iterations": it, "rel_residual": float(np.sqrt(hdot(rt, rt).real) / nF), "status": status}


# ------------------------------------------------------------------------------------ homogenization

def corrector_rhs(P, N, Ahat, j: int) -> np.ndarray:
    """F_j(k) = i sum_a lambda_a(k) A~^{aj}_k, F_j(0) = 0: the Fourier coefficients of div(A e_j), the
    right-hand side of the corrector problem -div(A (e_j + grad u)) = 0 (Sec. 5.2 eq. corrector; App. D)."""
    lam = lambdas(P, N)
    d = lam.shape[0]
    F = np.zeros(lam.shape[1:], dtype=np.complex128)
    for a in range(d):
        F += 1j * lam[a] * Ahat[a, j]
    F.reshape(-1)[0] = 0.0
    return F


def homogenized_from_correctors(P, N, Ahat, U_list) -> np.ndarray:
    """A*_ij = M{ e_i^T A (e_j + grad u_j) } (eq. homcoefficient) as the grid mean, written in Fourier terms:
    A*_ij = A~^{ij}_0 + sum_k sum_b A~^{ib}_{-k} (i lambda_b(k)) U_j(k). Returns the complex d x d matrix."""
    N = tuple(int(x) for x in N)
    lam = lambdas(P, N)
    d = lam.shape[0]
    axes = tuple(range(len(N)))
    zero = (0,) * len(N)
    out = np.zeros((d, d), dtype=np.complex128)
    for i in range(d):
        for j in range(d):
            s = Ahat[(i, j) + zero]
            for b in range(d):
                # A~_{-k} at storage index of k: reverse every axis and roll by one (index (-i) mod N).
                Aneg = np.roll(np.flip(Ahat[i, b], axis=axes), 1, axis=axes)
                s += np.sum(Aneg * 1j * lam[b] * U_list[j])
            out[i, j] = s
    return out


def homogenized_energy(P, N, Agrid, U_list) -> np.ndarray:
    """Energy form <(e_i + grad u_i)^T A (e_j + grad u_j)> on the grid (equal to the flux form at the discrete
    solution by Galerkin orthogonality). Gradients by the inverse DFT of i lambda U."""
    N = tuple(int(x) for x in N)
    lam = lambdas(P, N)
    d = lam.shape[0]
    grads = []
    for j in range(d):
        gj = [np.fft.ifftn(1j * lam[b] * U_list[j]) * np.prod(N) for b in range(d)]
        gj[j] = gj[j] + 1.0
        grads.append(gj)
    out = np.zeros((d, d), dtype=np.complex128)
    for i in range(d):
        for j in range(d):
            s = 0.0
            for a in range(d):
                for b in range(d):
                    s = s + np.conj(grads[i][a]) * Agrid[a, b] * grads[j][b]
            out[i, j] = np.mean(s)
    return out


def homogenized(inst, tol: float | None = None, precond: str = "jacobi", maxit: int = 10000, method=None):
    """Solve the d corrector problems with C-PCG and return (A* real d x d, [U_j], [info_j], Astar_complex)."""
    op = Operator(inst, method)
    if tol is None:
        tol = inst.tol
    if precond == "jacobi":
        M = jacobi_inverse(op.P, op.N, op.Ahat)
    elif precond == "frobenius":
        M = frobenius_diag(op.P, op.N, op.Ahat, op.modes if op.method == "conv" else None)
    else:
        raise ValueError(precond)
    Us, infos = [], []
    for j in range(inst.d):
        F = corrector_rhs(op.P, op.N, op.Ahat, j)
        U, info = pcg(op, F, M, tol, maxit)
        Us.append(U)
        infos.append(info)
    Ac = homogenized_from_correctors(op.P, op.N, op.Ahat, Us)
    return Ac.real.copy(), Us, infos, Ac


# ------------------------------------------------------------------------------------ Nyquist-free variant

def nyquist_free_mask(N) -> np.ndarray:
    """True on the modes of K_N^n with no Nyquist component (k_j = -N_j/2 for an even N_j), shape (*N).

    The remaining set K'_N = {k : |k_j| < N_j/2} is closed under k -> -k, which K_N^n is not for even N_j
    (Sec. 2.3 gives K_N^n = {-N/2 <= k_j < N/2}). On K'_N the stiffness matrix of a real coefficient satisfies
    Q(-k, -k') = conj(Q(k, k')) (lambda(-k) = -lambda(k), A~_{-m} = conj(A~_m)), so a real right-hand side has a
    solution with U(-k) = conj(U(k)): the property a half-spectrum (real-arithmetic) storage relies on."""
    N = tuple(int(x) for x in N)
    kg = k_grids(N)
    keep = np.ones(N, dtype=bool)
    for j, Nj in enumerate(N):
        if Nj % 2 == 0:
            keep &= kg[j] != -(Nj // 2)
    return keep


def homogenized_nyquist_free(inst, tol: float | None = None, precond: str = "jacobi", maxit: int = 10000):
    """The homogenization of `homogenized` on the Nyquist-free trial and test space: the Galerkin restriction
    of the discrete scheme (Sec. 3.1.1, eq. n-discrete_equation; App. D) to the modes K'_N of nyquist_free_mask,
    i.e. Q' = Q restricted to K'_N x K'_N (the same lambda = P k, the same coefficient modes, the convolution still
    wrapping modulo N), F' = F on K'_N, then Algorithm 2 and eq. homcoefficient summed over K'_N. For odd N_j it is
    `homogenized` itself. Returns (A* real d x d, [U_j], [info_j], Astar_complex)."""
    op = Operator(inst)
    if tol is None:
        tol = inst.tol
    keep = nyquist_free_mask(op.N)
    if precond == "jacobi":
        M = jacobi_inverse(op.P, op.N, op.Ahat) * keep
    else:
        raise ValueError(precond)

    def restricted(h):
        return keep * op(keep * h)

    Us, infos = [], []
    for j in range(inst.d):
        F = keep * corrector_rhs(op.P, op.N, op.Ahat, j)
        U, info = pcg(restricted, F, M, tol, maxit)
        Us.append(U)
        infos.append(info)
    Ac = homogenized_from_correctors(op.P, op.N, op.Ahat, Us)
    return Ac.real.copy(), Us, infos, Ac


# ------------------------------------------------------------------------------------ manufactured RHS

def manufactured_rhs(P, taps_k, taps_val, kind, d, modes, amps, N) -> np.ndarray:
    """Exact Fourier coefficients of f = -div(A grad u) for u = sum_k U^_k e^{i k.theta} (finitely many modes)
    and tapped A, by the non-wrapped product of the two mode lists (plain double loop), placed on K_N^n.
    F(k) = sum over (m, k') with k = m + k' of sum_ab (P k)_a A~^{ab}_m (P k')_b U^_{k'}.
    Raises if a product mode leaves K_N^n (that case would need folding, which is not wanted here)."""
    P = np.asarray(P, dtype=np.float64)
    pairs = _pairs(kind, d)
    N = tuple(int(x) for x in N)
    out = np.zeros(N, dtype=np.complex128)
    for m, val in zip(taps_k, taps_val):
        Am = np.zeros((d, d), dtype=np.complex128)
        for comp, entries in enumerate(pairs):
            for (a, b) in entries:
                Am[a, b] += val[comp]
        for kp, u in zip(modes, amps):
            k = np.asarray(m, dtype=np.int64) + np.asarray(kp, dtype=np.int64)
            if any(not (-Nj / 2.0 <= kj < Nj / 2.0) for kj, Nj in zip(k, N)):
                raise ValueError("product mode %s outside K_N^n" % (tuple(k),))
            lk = P @ k.astype(np.float64)
            lkp = P @ np.asarray(kp, dtype=np.float64)
            out[tuple(int(kj) % Nj for kj, Nj in zip(k, N))] += (lk @ Am @ lkp) * u
    return out


def modes_to_array(modes, amps, N) -> np.ndarray:
    """Place a mode list on the storage grid (index k mod N)."""
    N = tuple(int(x) for x in N)
    out = np.zeros(N, dtype=np.complex128)
    for k, u in zip(modes, amps):
        out[tuple(int(kj) % Nj for kj, Nj in zip(k, N))] += u
    return out


# ------------------------------------------------------------------------------------ timing helper

def timed_pcg_sample(inst, max_seconds: float = 15.0, precond: str = "jacobi"):
    """Run the oracle's Algorithm 2 on corrector 1 of ``inst`` for as many iterations as fit in about
    ``max_seconds`` of CPU time; return (DOF-iterations done, seconds). Used as the CPU baseline."""
    op = Operator(inst)
    M = jacobi_inverse(op.P, op.N, op.Ahat) if precond == "jacobi" else frobenius_diag(op.P, op.N, op.Ahat)
    F = corrector_rhs(op.P, op.N, op.Ahat, 0)
    op(F)                                   # warm-up (first-call costs), then one timed apply sizes the sample
    t0 = time.perf_counter()
    op(F)
    t1 = time.perf_counter()
    per_it = max(t1 - t0, 1e-6)
    iters = int(max(1, min(10000, max_seconds / per_it - 2)))
    t0 = time.perf_counter()
    _, info = pcg(op, F, M, tol=0.0, maxit=iters)
    t1 = time.perf_counter()
    done = info["iterations"] + 2      # + the initial and the final true-residual applies
    return inst.D * done, t1 - t0, done


__all__ = [n for n in dir() if not n.startswith("_") and n not in ("annotations", "itertools", "time", "np")]
