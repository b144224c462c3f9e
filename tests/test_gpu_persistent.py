"""The persistent (one cooperative launch) form of the solve against the CUDA-graph and host-driven forms and the
oracle.

The three execution forms run the same per-element arithmetic and the same fixed-order reductions, so their
solutions, iteration counts and residuals must be bitwise equal; a* must match the FP64 oracle."""
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


# (d, n, N, kind, nrhs, nmodes): scalar/diagonal/matrix coefficients, 1..4 right-hand sides, a single chunk
# (D = 64) up to many chunks per block
# (the persistent form needs a last axis of even length; (8, 9) checks that it then falls back to the graph)
CASES = [
    (1, 2, (8, 8), "scalar", 1, None),
    (2, 3, (10, 6, 8), "sym", 2, None),
    (2, 4, (6, 6, 6, 4), "diag", 3, None),
    (3, 3, (12, 10, 8), "sym", 4, None),
    (1, 3, (64, 48, 40), "scalar", 2, None),
    (3, 6, (6, 6, 6, 6, 6, 4), "diag", 3, 24),
    (1, 2, (8, 9), "scalar", 2, None),
]


def _solve(qp, inst, exec_mode, F, mode, precond, warm_from=None):
    plan = qp.plan_from_instance(inst, max_rhs=F.shape[0], exec_mode=exec_mode)
    Ft = torch.from_numpy(F).cuda()
    Ut = torch.zeros_like(Ft) if warm_from is None else torch.from_numpy(warm_from).cuda()
    infos = qp.qp_pcg_solve(plan, Ft, Ut, tol=1e-10, maxit=2000, precond=precond, mode=mode)
    return Ut.cpu().numpy(), infos


@pytest.mark.parametrize("d,n,N,kind,nrhs,nmodes", CASES)
@pytest.mark.parametrize("mode", ["fp64", "refine"])
def test_persistent_equals_graph_and_direct_bitwise(qp, d, n, N, kind, nrhs, nmodes, mode):
    inst = W.random_instance(d, n, N, kind, "taps", seed=100 + d * 10 + n, nmodes=nmodes)
    m = qp.QP_MODE_FP64 if mode == "fp64" else qp.QP_MODE_FP32_REFINE
    F = _rand_vecs(nrhs, N, 5)
    F.reshape(nrhs, -1)[:, 0] = 0
    precond = qp.QP_PRECOND_FROBENIUS if kind == "sym" else qp.QP_PRECOND_JACOBI
    Up, ip = _solve(qp, inst, qp.QP_EXEC_PERSISTENT, F, m, precond)
    Ug, ig = _solve(qp, inst, qp.QP_EXEC_GRAPH, F, m, precond)
    Ud, idr = _solve(qp, inst, qp.QP_EXEC_DIRECT, F, m, precond)
    assert np.array_equal(Up, Ug) and np.array_equal(Up, Ud)
    assert ip == ig == idr
    op = O.Operator(inst)
    for r in range(nrhs):
        assert ip[r]["status"] == "QP_OK" and ip[r]["rel_residual"] <= 1e-10
        assert Up[r].reshape(-1)[0] == 0
        res = np.linalg.norm(F[r] - op(Up[r])) / np.linalg.norm(F[r])
        assert res <= 1.2e-10, res


@pytest.mark.parametrize("mode", ["fp64", "refine"])
def test_persistent_warm_start_and_zero_rhs(qp, mode):
    inst = W.random_instance(2, 3, (10, 6, 8), "diag", "taps", seed=7)
    m = qp.QP_MODE_FP64 if mode == "fp64" else qp.QP_MODE_FP32_REFINE
    F = _rand_vecs(3, inst.N, 11)
    F[1] = 0                                   # a zero right-hand side among others: U = 0, no iterations
    U0 = 1e-3 * _rand_vecs(3, inst.N, 12)      # warm start away from the solution
    Up, ip = _solve(qp, inst, qp.QP_EXEC_PERSISTENT, F, m, qp.QP_PRECOND_JACOBI, warm_from=U0)
    Ug, ig = _solve(qp, inst, qp.QP_EXEC_GRAPH, F, m, qp.QP_PRECOND_JACOBI, warm_from=U0)
    assert np.array_equal(Up, Ug) and ip == ig
    assert float(np.abs(Up[1]).max()) == 0.0 and ip[1]["iterations"] == 0
    assert ip[0]["status"] == "QP_OK" and ip[2]["status"] == "QP_OK"


def test_persistent_more_chunks_than_resident_blocks(qp):
    """D = 12^6 modes in 1,167 chunks of 2,560 modes (each five interleaved 512-mode segments): more chunks than
    co-resident blocks, so every block walks several."""
    inst = W.random_instance(2, 6, (12,) * 6, "diag", "taps", seed=31, nmodes=12)
    F = _rand_vecs(2, inst.N, 3)
    for m in (qp.QP_MODE_FP32_REFINE, qp.QP_MODE_FP64):
        Up, ip = _solve(qp, inst, qp.QP_EXEC_PERSISTENT, F, m, qp.QP_PRECOND_JACOBI)
        Ug, ig = _solve(qp, inst, qp.QP_EXEC_GRAPH, F, m, qp.QP_PRECOND_JACOBI)
        assert np.array_equal(Up, Ug) and ip == ig
        assert all(i["status"] == "QP_OK" and i["rel_residual"] <= 1e-10 for i in ip)


def test_persistent_homogenized_matches_oracle(qp):
    for inst in (W.cfg0(), W.random_instance(3, 4, (8, 6, 6, 4), "sym", "taps", seed=17)):
        plan = qp.plan_from_instance(inst, exec_mode=qp.QP_EXEC_PERSISTENT)
        A, infos = qp.qp_homogenized(plan, tol=1e-11)
        A_ref, *_ = O.homogenized(inst, tol=1e-13)
        assert np.abs(A.real - A_ref).max() <= 1e-10 * np.abs(A_ref).max()
        assert all(i["status"] == "QP_OK" for i in infos)


def test_persistent_barrier_timeout_is_reported_and_device_stays_usable(qp):
    """A barrier limit far below one phase makes the waits run out: the solve returns QP_ERR_TIMEOUT (no fault,
    no hang) and the next solve on the same plan, with the default limit back, is correct."""
    inst = W.random_instance(2, 4, (12, 12, 12, 12), "sym", "taps", seed=9)
    plan = qp.plan_from_instance(inst, exec_mode=qp.QP_EXEC_PERSISTENT)
    F = torch.from_numpy(_rand_vecs(2, inst.N, 1)).cuda()
    U = torch.zeros_like(F)
    qp.qp_set_barrier_timeout(1e-9)
    try:
        with pytest.raises(qp.QPError) as ei:
            qp.qp_pcg_solve(plan, F, U, tol=1e-10)
        assert ei.value.status == qp.QP_ERR_TIMEOUT
    finally:
        qp.qp_set_barrier_timeout(2.0)
    infos = qp.qp_pcg_solve(plan, F, U, tol=1e-10)
    assert all(i["status"] == "QP_OK" and i["rel_residual"] <= 1e-10 for i in infos)
    with pytest.raises(qp.QPError):
        qp.qp_set_barrier_timeout(0.0)
