"""The general quasiperiodic elliptic solve -div(alpha grad u) = f with a user right-hand side, and its error in
the L^2_QP norm (Sec. 5.1), through the C ABI: qp_l2qp_error against numpy, and the paper's first example
(alpha_1, u_1; Sec. 5.1.1, Table 2) reproduced on the GPU."""
import json
import os

import numpy as np
import pytest

import qp_workloads as W
from oracle import qp_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def qp():
    import paper_2404_06841_gb300 as qp
    assert torch.cuda.is_available()
    return qp


@pytest.mark.parametrize("N,nrhs", [((8, 6, 4), 2), ((64, 48), 1), ((16, 12, 10), 4)])
def test_l2qp_error_matches_numpy(qp, N, nrhs):
    inst = W.random_instance(len(N) - 1 if len(N) > 1 else 1, len(N), N, "scalar", "taps", seed=5)
    plan = qp.plan_from_instance(inst, max_rhs=nrhs)
    rng = np.random.default_rng(3)
    U = rng.standard_normal((nrhs,) + N) + 1j * rng.standard_normal((nrhs,) + N)
    V = U + 1e-3 * (rng.standard_normal((nrhs,) + N) + 1j * rng.standard_normal((nrhs,) + N))
    Ut, Vt = torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda()
    e = qp.qp_l2qp_error(plan, Ut, Vt)
    ref = np.array([np.linalg.norm((U - V)[r]) for r in range(nrhs)])
    assert np.abs(e - ref).max() <= 1e-13 * ref.max()
    n = qp.qp_l2qp_error(plan, Ut)
    assert np.abs(n - np.array([np.linalg.norm(U[r]) for r in range(nrhs)])).max() <= 1e-13 * n.max()
    assert qp.qp_l2qp_error(plan, Ut, Ut).max() == 0.0


def test_paper_table2_example_on_gpu(qp):
    """(alpha_1, u_1) with P = 2 pi (1, sqrt2): the right-hand side is the exact f = -div(alpha_1 grad u_1) in
    Fourier space (the oracle's non-aliased convolution), the GPU solve's L^2_QP error e_N sits at rounding
    level as Table 2 prints for N >= 8, and the iteration count does not grow with N (P11)."""
    g = json.load(open(os.path.join(GOLDEN, "table2_pm_efficiency.json")))
    iters = []
    for N, e_paper in zip(g["N"], g["e_N_C_PCG"]):
        inst = W.paper_elliptic_u1(N)
        modes, amps = inst.meta["u_modes"], inst.meta["u_amps"]
        plan = qp.plan_from_instance(inst, max_rhs=1)
        F = O.manufactured_rhs(inst.P, inst.coeff.taps_k, inst.coeff.taps_val, "scalar", 1, modes, amps, inst.N)
        Uex = torch.from_numpy(W.modes_on_grid(inst.N, modes, amps)[None].copy()).cuda()
        # Q applied to the exact coefficients gives the same right-hand side (no aliasing at N >= 8)
        QU = torch.empty_like(Uex)
        qp.qp_apply_stiffness(plan, Uex, QU, qp.QP_FP64)
        assert np.abs(QU[0].cpu().numpy() - F).max() <= 1e-13 * np.abs(F).max()
        Ft = torch.from_numpy(F[None].copy()).cuda()
        U = torch.zeros_like(Ft)
        info = qp.qp_pcg_solve(plan, Ft, U, tol=1e-14, maxit=200)[0]
        assert info["status"] == "QP_OK" and info["rel_residual"] <= 1e-14
        e_N = qp.qp_l2qp_error(plan, U, Uex)[0]
        assert e_N <= 10 * max(e_paper, 1e-16) + 1e-15, (N, e_N, e_paper)
        iters.append(info["iterations"])
        # FP32 inner solves inside FP64 refinement reach the same level
        U2 = torch.zeros_like(Ft)
        info2 = qp.qp_pcg_solve(plan, Ft, U2, tol=1e-13, maxit=400, mode=qp.QP_MODE_FP32_REFINE)[0]
        assert info2["status"] == "QP_OK"
        assert qp.qp_l2qp_error(plan, U2, Uex)[0] <= 1e-12
    assert max(iters[1:]) - min(iters[1:]) <= 3, iters
