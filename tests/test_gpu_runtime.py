"""Runtime controls of the library on the GPU: the device-memory pool (statistics and the cache size kept after a
destroy) and the per-phase event timing of solves."""
import pytest

import qp_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qp():
    import paper_2404_06841_gb300 as qp
    assert torch.cuda.is_available()
    return qp


def test_memory_cache_zero_returns_freed_blocks(qp):
    """With a cache of 0 bytes a destroyed plan's memory goes back to the device at once; the default (-1) is
    restored afterwards. Used bytes return to their level before the plan."""
    try:
        qp.qp_set_memory_cache(0)
        before = qp.qp_memory_pool_stats()
        plan = qp.plan_from_instance(W.cfg1())
        during = qp.qp_memory_pool_stats()
        assert during["used_bytes"] > before["used_bytes"]
        assert during["allocations"] > before["allocations"]
        qp.qp_plan_destroy(plan)
        after = qp.qp_memory_pool_stats()
        assert after["used_bytes"] == before["used_bytes"]
        assert after["reserved_bytes"] <= before["reserved_bytes"]
    finally:
        qp.qp_set_memory_cache(-1)
    # with the default cache the freed blocks stay reserved for the next plan
    plan = qp.plan_from_instance(W.cfg1())
    qp.qp_plan_destroy(plan)
    kept = qp.qp_memory_pool_stats()
    plan = qp.plan_from_instance(W.cfg1())
    again = qp.qp_memory_pool_stats()
    assert again["reserved_bytes"] == kept["reserved_bytes"]   # served from the cache
    qp.qp_plan_destroy(plan)


def test_phase_timing_counts_the_solve(qp):
    """Phase timing runs the solve host-driven and counts one FP32 apply, update and h-update launch per inner
    iteration of the batch (at least the most iterations of one corrector, at most their sum); the result equals
    the untimed (persistent) solve bit for bit."""
    inst = W.cfg1()
    plan = qp.plan_from_instance(inst)
    A0, infos0 = qp.qp_homogenized(plan, tol=1e-10, mode=qp.QP_MODE_FP32_REFINE)
    qp.qp_set_phase_timing(True)
    try:
        A1, infos1 = qp.qp_homogenized(plan, tol=1e-10, mode=qp.QP_MODE_FP32_REFINE)
        ph = qp.qp_phase_times()
    finally:
        qp.qp_set_phase_timing(False)
    assert (A0 == A1).all() and [i["iterations"] for i in infos0] == [i["iterations"] for i in infos1]
    its = [i["iterations"] for i in infos1]
    for name in ("apply32", "update32", "hupdate32"):
        ms, n = ph[name]
        assert max(its) <= n <= sum(its) and ms > 0.0, (name, ph[name], its)
    assert ph["residual64"][1] >= 2 and ph["apply64"][1] == 0
    qp.qp_plan_destroy(plan)
