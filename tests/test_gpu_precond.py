"""The diagonal preconditioners of Sec. 4.3 (eq. preconditioner) read through the C ABI and compared element by
element with the oracle: Jacobi and the Frobenius-optimal diagonal on the taps backend (O(gD) column sums) and on
the FFT backend (FFT cross-correlations), and solves with the Frobenius diagonal on the FFT backend."""
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


def _close(got, ref, rtol):
    return np.abs(got - ref).max() <= rtol * np.abs(ref).max() and np.all(np.abs(got - ref) <= rtol * np.abs(ref) + 1e-14 * np.abs(ref).max())


CASES = [(1, 2, (8, 12), "scalar"), (2, 2, (16, 8), "sym"), (2, 3, (8, 6, 4), "diag"), (3, 3, (4, 6, 8), "sym"),
         (2, 4, (6, 4, 8, 4), "sym"), (1, 1, (32,), "scalar"), (3, 3, (6, 4, 6), "diag")]


@pytest.mark.parametrize("d,n,N,kind", CASES)
def test_fft_backend_diagonals_match_oracle(qp, d, n, N, kind):
    inst = W.random_instance(d, n, N, kind, "grid", seed=11 + d + n, nonlinear=True)
    plan = qp.plan_from_instance(inst)
    assert qp.qp_plan_query(plan)["backend"] == "fft"
    Ahat = O.coefficient_modes(inst)
    jac = qp.qp_plan_diagonal(plan, qp.QP_PRECOND_JACOBI).cpu().numpy()
    assert _close(jac, O.jacobi_inverse(inst.P, inst.N, Ahat), 1e-13)
    fro = qp.qp_plan_diagonal(plan, qp.QP_PRECOND_FROBENIUS).cpu().numpy()
    ref = O.frobenius_diag(inst.P, inst.N, Ahat)
    assert fro.reshape(-1)[0] == 0.0
    assert _close(fro, ref, 1e-10), np.abs(fro - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("d,n,N,kind", [(2, 3, (8, 6, 4), "sym"), (1, 2, (12, 16), "scalar"), (3, 3, (6, 4, 8), "diag")])
def test_taps_and_fft_backends_build_the_same_frobenius_diagonal(qp, d, n, N, kind):
    inst = W.random_instance(d, n, N, kind, "taps", seed=3)
    p_t = qp.plan_from_instance(inst)
    p_f = qp.plan_from_instance(inst, backend=qp.QP_BACKEND_FFT)
    ref = O.frobenius_diag(inst.P, inst.N, O.coefficient_modes(inst))
    ft = qp.qp_plan_diagonal(p_t, qp.QP_PRECOND_FROBENIUS).cpu().numpy()
    ff = qp.qp_plan_diagonal(p_f, qp.QP_PRECOND_FROBENIUS).cpu().numpy()
    assert _close(ft, ref, 1e-12)
    assert _close(ff, ref, 1e-10)


@pytest.mark.parametrize("mode", ["fp64", "refine"])
def test_fft_backend_frobenius_solve_matches_oracle(qp, mode):
    inst = W.random_instance(2, 3, (8, 8, 6), "sym", "grid", seed=19, nonlinear=True)
    plan = qp.plan_from_instance(inst)
    m = qp.QP_MODE_FP64 if mode == "fp64" else qp.QP_MODE_FP32_REFINE
    A, infos = qp.qp_homogenized(plan, tol=1e-10, mode=m, precond=qp.QP_PRECOND_FROBENIUS)
    A_ref, *_ = O.homogenized(inst, tol=1e-13)
    assert np.abs(A.real - A_ref).max() <= 1e-10 * np.abs(A_ref).max()
    assert all(i["status"] == "QP_OK" and i["rel_residual"] <= 1e-10 for i in infos)


def test_cfg2_full_size_frobenius(qp):
    """cfg2 (32^4 modes, SPD 2 x 2 grid coefficient): the Frobenius diagonal built by FFT correlations drives the
    refinement solve to the oracle's a*, and at sampled modes equals q / ||Q e_k||^2 summed directly over the
    column (every row k + m of the dense coefficient)."""
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "astar_full_size.json")))["cfg2"]
    inst = W.cfg2()
    plan = qp.plan_from_instance(inst)
    A, infos = qp.qp_homogenized(plan, tol=1e-10, mode=qp.QP_MODE_FP32_REFINE, precond=qp.QP_PRECOND_FROBENIUS)
    ref = np.array(gold["astar_re"])
    assert np.abs(A.real - ref).max() <= 1e-10 * np.abs(ref).max()
    assert all(i["status"] == "QP_OK" for i in infos)
    # sampled modes: column k of Q summed over every row k + m (all D modes of the dense coefficient)
    fro = qp.qp_plan_diagonal(plan, qp.QP_PRECOND_FROBENIUS).cpu().numpy()
    Ahat = O.coefficient_modes(inst)                      # (d, d) + N
    lam = O.lambdas(inst.P, inst.N)                        # (d,) + N
    q = O.jacobi_diag(inst.P, inst.N, Ahat)
    rng = np.random.default_rng(6)
    N = inst.N
    for _ in range(6):
        k = tuple(int(rng.integers(0, Nj)) for Nj in N)
        if k == (0,) * len(N):
            continue
        # rows k + m for every m: roll lambda so that index m holds lambda(k + m)
        lam_row = [np.roll(lam[a], tuple(-x for x in k), axis=tuple(range(len(N)))) for a in range(2)]
        e = sum(lam_row[a] * Ahat[a, b] * lam[(b,) + k] for a in range(2) for b in range(2))
        cn = float(np.sum(np.abs(e) ** 2))
        assert abs(fro[k] - q[k] / cn) <= 1e-10 * abs(q[k] / cn), (k, fro[k], q[k] / cn)
