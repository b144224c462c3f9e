"""The allocation-free solve (qp_pcg_solve_taps_static) against the plan-based qp_pcg_solve.

qp_pcg_solve_taps_static serves callers that cannot call cudaMalloc (for example when another component owns
the device-memory budget): it works entirely inside one static device array of the library. This file is
named so that pytest collects it last; it passes alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

import qp_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_static_scratch_solve_matches_plan_solve_on_two_calls():
    import paper_2404_06841_gb300 as qp
    inst = W.cfg1()                      # d = 2, n = 4, 16^4 modes, two right-hand sides
    plan = qp.plan_from_instance(inst)
    F = torch.zeros((inst.d, inst.D), dtype=torch.complex128, device="cuda")
    qp.qp_corrector_rhs(plan, 0, inst.d, F)
    U_ref = torch.zeros_like(F)
    ref_infos = qp.qp_pcg_solve(plan, F, U_ref, tol=1e-11)
    for call in range(2):                # the second call reuses the scratch the first one left behind
        U = torch.zeros_like(F)
        infos = qp.qp_pcg_solve_taps_static(inst.d, inst.n, inst.P, inst.N, inst.coeff, F, U, tol=1e-11)
        for a, b in zip(infos, ref_infos):
            assert a["status"] == "QP_OK" and a["rel_residual"] <= 1e-11
            assert a["iterations"] == b["iterations"]
        rel = float((U - U_ref).abs().max() / U_ref.abs().max())
        assert rel <= 1e-10, (call, rel)
    # a problem beyond the scratch is rejected before any device work, with a clear message
    big = W.cfg4()
    Fb = torch.zeros((1, 8), dtype=torch.complex128, device="cuda")
    with pytest.raises(qp.QPError) as ei:
        qp.qp_pcg_solve_taps_static(big.d, big.n, big.P, big.N, big.coeff, Fb, Fb.clone(), nrhs=1)
    assert ei.value.status == qp.QP_ERR_INVALID_ARG and "static scratch" in str(ei.value)
    qp.qp_plan_destroy(plan)
