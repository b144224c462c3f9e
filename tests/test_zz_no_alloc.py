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


def _alloc_state(qp):
    """What would change if a call allocated device memory: the device's free memory, the library pool's
    reserved bytes and allocation count, and torch's allocation count."""
    torch.cuda.synchronize()
    free, _ = torch.cuda.mem_get_info()
    pool = qp.qp_memory_pool_stats()
    return (free, pool["reserved_bytes"], pool["allocations"],
            torch.cuda.memory_stats().get("allocation.all.allocated", 0))


@pytest.mark.parametrize("precond", ["jacobi", "frobenius"])
def test_static_scratch_solve_matches_plan_solve_on_two_calls(precond):
    import paper_2404_06841_gb300 as qp
    pc = qp.QP_PRECOND_JACOBI if precond == "jacobi" else qp.QP_PRECOND_FROBENIUS
    inst = W.cfg1()                      # d = 2, n = 4, 16^4 modes, two right-hand sides
    plan = qp.plan_from_instance(inst)
    F = torch.zeros((inst.d, inst.D), dtype=torch.complex128, device="cuda")
    qp.qp_corrector_rhs(plan, 0, inst.d, F)
    U_ref = torch.zeros_like(F)
    ref_infos = qp.qp_pcg_solve(plan, F, U_ref, tol=1e-11, precond=pc)
    Us = [torch.zeros_like(F) for _ in range(3)]
    qp.qp_pcg_solve_taps_static(inst.d, inst.n, inst.P, inst.N, inst.coeff, F, Us[2], tol=1e-11, precond=pc)
    before = _alloc_state(qp)            # after a first call (module and scratch loaded), all tensors made
    calls = []
    for call in range(2):                # the second call reuses the scratch the first one left behind
        calls.append(qp.qp_pcg_solve_taps_static(inst.d, inst.n, inst.P, inst.N, inst.coeff, F, Us[call],
                                                 tol=1e-11, precond=pc))
    assert _alloc_state(qp) == before    # no device allocation by either call
    for call, infos in enumerate(calls):
        for a, b in zip(infos, ref_infos):
            assert a["status"] == "QP_OK" and a["rel_residual"] <= 1e-11
            assert a["iterations"] == b["iterations"]
        rel = float((Us[call] - U_ref).abs().max() / U_ref.abs().max())
        assert rel <= 1e-10, (call, rel)
    # a problem beyond the scratch is rejected before any device work, with a clear message
    big = W.cfg4()
    Fb = torch.zeros((1, 8), dtype=torch.complex128, device="cuda")
    with pytest.raises(qp.QPError) as ei:
        qp.qp_pcg_solve_taps_static(big.d, big.n, big.P, big.N, big.coeff, Fb, Fb.clone(), nrhs=1)
    assert ei.value.status == qp.QP_ERR_INVALID_ARG and "static scratch" in str(ei.value)
    qp.qp_plan_destroy(plan)


def test_static_scratch_solve_at_a_tight_tolerance():
    """d = 1, n = 2, 32^2 modes to 1e-12: where the recursive residual can meet the tolerance before the true one
    does, both entry points solve again from the current U and report the same iterations and solution."""
    import paper_2404_06841_gb300 as qp
    inst = W.cfg0()
    plan = qp.plan_from_instance(inst)
    F = torch.zeros((1, inst.D), dtype=torch.complex128, device="cuda")
    qp.qp_corrector_rhs(plan, 0, 1, F)
    for tol in (1e-12, 1e-13):
        U_ref = torch.zeros_like(F)
        ref = qp.qp_pcg_solve(plan, F, U_ref, tol=tol, raise_on_error=False)
        U = torch.zeros_like(F)
        got = qp.qp_pcg_solve_taps_static(inst.d, inst.n, inst.P, inst.N, inst.coeff, F, U, tol=tol,
                                          raise_on_error=False)
        assert got[0]["status"] == ref[0]["status"] == "QP_OK", (tol, got, ref)
        assert got[0]["rel_residual"] <= tol and got[0]["iterations"] == ref[0]["iterations"]
        assert float((U - U_ref).abs().max() / U_ref.abs().max()) <= 1e-10
    qp.qp_plan_destroy(plan)
