"""Parity of the CUDA taps backend (through the C ABI) with the FP64 oracle."""
import numpy as np
import pytest

import qp_workloads as W
from oracle import qp_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qp():
    import paper_2404_06841_gb300 as qp
    assert torch.cuda.is_available()
    return qp


def _rand_vecs(nrhs, N, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nrhs,) + tuple(N)) + 1j * rng.standard_normal((nrhs,) + tuple(N))


APPLY_CASES = [
    (1, 2, (8, 8), "scalar", 1, None), (1, 2, (6, 10), "scalar", 2, None), (2, 2, (8, 6), "sym", 3, None),
    (2, 3, (6, 4, 10), "diag", 1, None), (2, 4, (6, 6, 6, 6), "sym", 2, None), (3, 3, (6, 8, 4), "sym", 3, None),
    (3, 6, (4, 4, 4, 4, 4, 4), "diag", 4, 40), (1, 1, (16,), "scalar", 1, None), (2, 2, (30, 34), "scalar", 2, None),
    (1, 3, (12, 18, 10), "scalar", 4, None), (3, 5, (6, 4, 6, 4, 6), "sym", 2, 20),
]


@pytest.mark.parametrize("d,n,N,kind,nrhs,nmodes", APPLY_CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_matches_oracle_convolution(qp, d, n, N, kind, nrhs, nmodes, prec):
    inst = W.random_instance(d, n, N, kind, "taps", seed=d * 100 + n * 10 + len(N), radius=1, nmodes=nmodes)
    plan = qp.plan_from_instance(inst, max_rhs=4)
    h = _rand_vecs(nrhs, N, 7)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    ht = torch.from_numpy(h).to("cuda", dt)
    wt = torch.empty_like(ht)
    qp.qp_apply_stiffness(plan, ht, wt, qp.QP_FP64 if prec == "fp64" else qp.QP_FP32)
    op = O.Operator(inst)
    ref = np.stack([op(h[r]) for r in range(nrhs)])
    got = wt.cpu().numpy().astype(np.complex128)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= (1e-13 if prec == "fp64" else 2e-6), err


def test_apply_full_size_sampled_cfg4(qp):
    """cfg4 (d=3, n=6, N=16, 16.8M modes, 3 right-hand sides) in FP32 as the refinement uses it: sampled
    outputs against the oracle's pointwise formula."""
    inst = W.cfg4()
    plan = qp.plan_from_instance(inst)
    g = torch.Generator(device="cuda").manual_seed(4)
    D = inst.D
    h = torch.randn((3, D), dtype=torch.complex64, device="cuda", generator=g)
    w = torch.empty_like(h)
    qp.qp_apply_stiffness(plan, h, w, qp.QP_FP32)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    flat = [0, 1, D - 1, D // 2] + [int(x) for x in rng.integers(0, D, 60)]
    pts = [np.unravel_index(i, inst.N) for i in flat]
    for r in range(3):
        hr = h[r].cpu().numpy().astype(np.complex128).reshape(inst.N)
        ref = O.apply_taps_at(inst.P, inst.N, inst.coeff.taps_k, inst.coeff.taps_val, "diag", hr, pts)
        got = w[r].cpu().numpy().astype(np.complex128)[flat]
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 2e-6 * scale
    # two right-hand sides take the run-time-geometry kernel (its grid of resident blocks walks 54 segments per
    # block here): bit for bit the compiled-in geometry's values
    w2 = torch.empty((2, D), dtype=torch.complex64, device="cuda")
    qp.qp_apply_stiffness(plan, h[:2].contiguous(), w2, qp.QP_FP32, nrhs=2)
    assert torch.equal(w2, w[:2])


def test_refinement_solve_of_a_unit_in_two_waves(qp):
    """cfg4's geometry at N = 12 (2,985,984 modes: 1,167 chunks of 2,560, more than one wave of 608 resident
    blocks, so the batch kernels walk their chunks in two waves over halves of the vector), refinement solve of
    the three corrector right-hand sides built by the oracle. The residual is recomputed over the whole vector by
    the plain FP64 apply (one run per thread, no chunks), and at sampled modes by the oracle's own sum."""
    inst = W.cfg4(N=12)
    Ahat = O.coefficient_modes(inst)
    F = np.stack([O.corrector_rhs(inst.P, inst.N, Ahat, j).reshape(-1) for j in range(3)])
    del Ahat
    plan = qp.plan_from_instance(inst)
    Ft = torch.from_numpy(F).cuda()
    Ut = torch.zeros_like(Ft)
    infos = qp.qp_pcg_solve(plan, Ft, Ut, tol=1e-10, maxit=2000, mode=qp.QP_MODE_FP32_REFINE)
    assert all(i["status"] == "QP_OK" for i in infos), infos
    QU = torch.empty_like(Ut)
    qp.qp_apply_stiffness(plan, Ut, QU, qp.QP_FP64)
    for r in range(3):
        rel = float(torch.linalg.vector_norm(Ft[r] - QU[r]) / torch.linalg.vector_norm(Ft[r]))
        assert rel <= 1.2e-10, (r, rel)
    U = Ut.cpu().numpy()
    D = inst.D
    rng = np.random.default_rng(1)
    flat = [1, D - 1, D // 2] + [int(x) for x in rng.integers(0, D, 40)]
    pts = [np.unravel_index(i, inst.N) for i in flat]
    for r in range(3):
        qu = O.apply_taps_at(inst.P, inst.N, inst.coeff.taps_k, inst.coeff.taps_val, "diag",
                             U[r].reshape(inst.N), pts)
        assert np.abs(F[r][flat] - qu).max() <= 1.2e-10 * np.linalg.norm(F[r])


@pytest.mark.parametrize("d,n,N,kind", [(2, 3, (6, 8, 4), "sym"), (3, 3, (4, 6, 8), "diag"), (1, 2, (10, 12), "scalar")])
def test_corrector_rhs_and_astar_reduce(qp, d, n, N, kind):
    inst = W.random_instance(d, n, N, kind, "taps", seed=3)
    plan = qp.plan_from_instance(inst)
    Ahat = O.coefficient_modes(inst)
    F = torch.zeros((d,) + N, dtype=torch.complex128, device="cuda")
    qp.qp_corrector_rhs(plan, 0, d, F)
    for j in range(d):
        ref = O.corrector_rhs(inst.P, N, Ahat, j)
        assert np.abs(F[j].cpu().numpy() - ref).max() <= 1e-14 * np.abs(ref).max()
    U = _rand_vecs(d, N, 5)
    U.reshape(d, -1)[:, 0] = 0
    A = qp.qp_homogenized_reduce(plan, torch.from_numpy(U).cuda())
    ref = O.homogenized_from_correctors(inst.P, N, Ahat, [U[j] for j in range(d)])
    assert np.abs(A - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("mode", ["fp64", "refine"])
@pytest.mark.parametrize("precond", ["jacobi", "frobenius"])
def test_pcg_solve_residual_under_oracle_operator(qp, mode, precond):
    inst = W.random_instance(2, 3, (10, 8, 6), "sym", "taps", seed=12)
    plan = qp.plan_from_instance(inst)
    F = _rand_vecs(2, inst.N, 9)
    F.reshape(2, -1)[:, 0] = 0
    Ft = torch.from_numpy(F).cuda()
    Ut = torch.zeros_like(Ft)
    infos = qp.qp_pcg_solve(plan, Ft, Ut, tol=1e-10, maxit=500,
                            precond=qp.QP_PRECOND_JACOBI if precond == "jacobi" else qp.QP_PRECOND_FROBENIUS,
                            mode=qp.QP_MODE_FP64 if mode == "fp64" else qp.QP_MODE_FP32_REFINE)
    op = O.Operator(inst)
    U = Ut.cpu().numpy()
    for r in range(2):
        assert infos[r]["status"] == "QP_OK"
        assert infos[r]["rel_residual"] <= 1e-10
        res = np.linalg.norm(F[r] - op(U[r])) / np.linalg.norm(F[r])
        assert res <= 1.2e-10, res
        assert U[r].reshape(-1)[0] == 0
        if mode == "refine":
            assert infos[r]["outer_iterations"] >= 2


def test_homogenized_cfg0_closed_form_and_oracle(qp):
    inst = W.cfg0()
    plan = qp.plan_from_instance(inst)
    A, infos = qp.qp_homogenized(plan, tol=1e-12)
    A_ref, *_ = O.homogenized(inst)
    a = O.coefficient_grid(inst)[0, 0]
    harmonic = 1.0 / np.mean(1.0 / a)                         # P1: exact discrete identity
    assert abs(A[0, 0].real - A_ref[0, 0]) <= 1e-10 * A_ref[0, 0]
    assert abs(A[0, 0].real - harmonic) <= 1e-12 * harmonic
    assert infos[0]["rel_residual"] <= 1e-12


@pytest.mark.parametrize("mode", ["fp64", "refine"])
def test_homogenized_cfg1_full_size(qp, mode):
    inst = W.cfg1()
    plan = qp.plan_from_instance(inst)
    A, infos = qp.qp_homogenized(plan, tol=1e-10, mode=qp.QP_MODE_FP64 if mode == "fp64" else qp.QP_MODE_FP32_REFINE)
    A_ref, *_ = O.homogenized(inst)
    assert np.abs(A.real - A_ref).max() <= 1e-10 * np.abs(A_ref).max()
    for info in infos:
        assert info["status"] == "QP_OK" and info["rel_residual"] <= 1e-10
    # Voigt-Reuss (P8)
    assert 1 / np.mean(1 / O.coefficient_grid(inst)[0, 0]) <= A[0, 0].real <= 5.0


@pytest.mark.parametrize("which,tol", [("cfg0", 1e-12), ("cfg1", 1e-10)])
def test_manufactured_solution(qp, which, tol):
    inst = getattr(W, which)()
    modes, amps = W.manufactured_modes(inst.n, inst.meta["manufactured_kmax"], inst.meta["manufactured_seed"])
    F = O.manufactured_rhs(inst.P, inst.coeff.taps_k, inst.coeff.taps_val, "scalar", inst.d, modes, amps, inst.N)
    Uex = O.modes_to_array(modes, amps, inst.N)
    plan = qp.plan_from_instance(inst, max_rhs=1)
    Ft = torch.from_numpy(F[None]).cuda()
    Ut = torch.zeros_like(Ft)
    infos = qp.qp_pcg_solve(plan, Ft, Ut, tol=tol)
    err = np.linalg.norm(Ut[0].cpu().numpy() - Uex) / np.linalg.norm(Uex)
    assert err <= 100 * tol, err


def test_edge_cases_zero_rhs_constant_coefficient_warm_start(qp):
    # constant coefficient: Q = c diag(|lambda|^2), one iteration (P5)
    k = np.zeros((1, 3), np.int32)
    inst = W.Instance("c", W.random_P(2, 3, 1), (6, 4, 8), W.Coefficient("scalar", k, np.array([[2.5]], complex)))
    plan = qp.plan_from_instance(inst)
    F = _rand_vecs(2, inst.N, 1)
    Ft = torch.from_numpy(F).cuda()
    Ut = torch.zeros_like(Ft)
    infos = qp.qp_pcg_solve(plan, Ft, Ut, tol=1e-12)
    assert all(i["iterations"] == 1 for i in infos)
    A, _ = qp.qp_homogenized(plan)
    assert np.abs(A - 2.5 * np.eye(2)).max() <= 1e-14
    # zero right-hand side: U = 0, no iterations
    inst = W.random_instance(2, 3, (6, 4, 8), "diag", "taps", seed=2)
    plan = qp.plan_from_instance(inst)
    Ft = torch.zeros((2,) + inst.N, dtype=torch.complex128, device="cuda")
    Ut = torch.ones_like(Ft)
    infos = qp.qp_pcg_solve(plan, Ft, Ut)
    assert all(i["iterations"] == 0 and i["status"] == "QP_OK" for i in infos)
    assert float(Ut.abs().max()) == 0.0
    # warm start from a converged solution: no further iterations
    F = _rand_vecs(2, inst.N, 4)
    Ft = torch.from_numpy(F).cuda()
    Ut = torch.zeros_like(Ft)
    qp.qp_pcg_solve(plan, Ft, Ut, tol=1e-11)
    infos = qp.qp_pcg_solve(plan, Ft, Ut, tol=1e-10)
    assert all(i["iterations"] == 0 for i in infos)


def test_errors_are_reported(qp):
    # P = (1, 2) is not a projection: k = (2, -1) has P k = 0
    k, v = W.cos_sum_taps(2, 3.0, 1.0)
    with pytest.raises(qp.QPError) as ei:
        qp.qp_plan_create(1, 2, [[1.0, 2.0]], [8, 8], W.Coefficient("scalar", k, v))
    assert ei.value.status == qp.QP_ERR_SINGULAR_P
    # a negative mean is not elliptic
    k, v = W.cos_sum_taps(2, -3.0, 1.0)
    with pytest.raises(qp.QPError) as ei:
        qp.qp_plan_create(1, 2, [[1.0, W.SQRT2]], [8, 8], W.Coefficient("scalar", k, v))
    assert ei.value.status == qp.QP_ERR_NOT_ELLIPTIC
    # taps without their Hermitian partner
    with pytest.raises(qp.QPError) as ei:
        qp.qp_plan_create(1, 2, [[1.0, W.SQRT2]], [8, 8],
                          W.Coefficient("scalar", np.array([[0, 0], [1, 0]], np.int32), np.array([[3.0], [0.5]], complex)))
    assert ei.value.status == qp.QP_ERR_INVALID_ARG
    # a tap beyond N/2
    k, v = W.cos_sum_taps(2, 3.0, 1.0)
    with pytest.raises(qp.QPError) as ei:
        qp.qp_plan_create(1, 2, [[1.0, W.SQRT2]], [2, 2], W.Coefficient("scalar", k, v))
    assert ei.value.status == qp.QP_ERR_INVALID_ARG
    # iteration cap
    inst = W.cfg0()
    plan = qp.plan_from_instance(inst)
    A, infos = qp.qp_homogenized(plan, tol=1e-12, maxit=2, raise_on_error=False)
    assert infos[0]["status"] == "QP_ERR_NO_CONVERGENCE" and infos[0]["iterations"] == 2
    with pytest.raises(qp.QPError):
        qp.qp_homogenized(plan, tol=1e-12, maxit=2)
    # the plan stays usable after an error
    A, infos = qp.qp_homogenized(plan, tol=1e-12)
    assert infos[0]["status"] == "QP_OK"
