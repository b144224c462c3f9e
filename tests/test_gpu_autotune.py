"""The FFT-backend apply autotuner: every candidate schedule (axis groups x tile budgets, and the per-axis path)
computes the same stiffness apply as the oracle's DFT form, the timed choice is one of them, and the choice is
cached per geometry."""
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


# a 4-axis grid (one group, two and three groups all feasible), a 6-axis grid, a 2-axis grid with an axis above
# 32 (per-axis path only), and cfg2's geometry at a reduced size
CASES = [(2, 4, (6, 4, 8, 4), "sym"), (3, 6, (4, 4, 6, 4, 4, 4), "diag"), (1, 2, (64, 12), "scalar"),
         (2, 4, (16, 16, 16, 16), "sym")]


@pytest.mark.parametrize("d,n,N,kind", CASES)
def test_every_candidate_schedule_matches_oracle(qp, d, n, N, kind):
    inst = W.random_instance(d, n, N, kind, "grid", seed=30 + n, nonlinear=True)
    plan = qp.plan_from_instance(inst, max_rhs=2)
    rng = np.random.default_rng(4)
    h = rng.standard_normal((2,) + N) + 1j * rng.standard_normal((2,) + N)
    Ag = O.coefficient_grid(inst)
    ref = np.stack([O.apply_fft(inst.P, N, Ag, h[r]) for r in range(2)])
    for prec, dt, tol in ((qp.QP_FP64, torch.complex128, 1e-12), (qp.QP_FP32, torch.complex64, 3e-6)):
        info = qp.qp_fft_schedule(plan, prec)
        assert 0 <= info["index"] < info["count"] and info["ms"] > 0, info
        if max(N) > 32:
            assert info["count"] == 1 and info["text"] == "per-axis passes"
        else:
            assert info["count"] >= 2
        for idx in range(info["count"]):
            qp.qp_fft_set_schedule(plan, prec, idx)
            ht = torch.from_numpy(h).to("cuda", dt)
            wt = torch.empty_like(ht)
            qp.qp_apply_stiffness(plan, ht, wt, prec)
            err = np.abs(wt.cpu().numpy().astype(np.complex128) - ref).max() / np.abs(ref).max()
            assert err <= tol, (idx, qp.qp_fft_schedule(plan, prec)["text"], err)
        with pytest.raises(qp.QPError):
            qp.qp_fft_set_schedule(plan, prec, info["count"])


def test_choice_is_cached_per_geometry_and_autotune_can_be_switched_off(qp):
    inst = W.random_instance(2, 4, (8, 6, 4, 6), "sym", "grid", seed=61, nonlinear=True)
    p1 = qp.plan_from_instance(inst, max_rhs=2)
    s1 = qp.qp_fft_schedule(p1, qp.QP_FP32)
    p2 = qp.plan_from_instance(inst, max_rhs=2)        # same geometry: the cached choice, not re-timed
    s2 = qp.qp_fft_schedule(p2, qp.QP_FP32)
    assert s2["index"] == s1["index"] and s2["ms"] == -1.0
    qp.qp_set_fft_autotune(False)
    try:
        other = W.random_instance(2, 4, (8, 6, 4, 4), "sym", "grid", seed=62, nonlinear=True)
        p3 = qp.plan_from_instance(other, max_rhs=2)   # new geometry, tuner off: the heuristic's schedule
        s3 = qp.qp_fft_schedule(p3, qp.QP_FP32)
        assert s3["index"] == -1 and s3["ms"] == -1.0 and s3["count"] >= 2
    finally:
        qp.qp_set_fft_autotune(True)


def test_taps_plan_has_no_fft_schedule(qp):
    plan = qp.plan_from_instance(W.cfg1(4))
    with pytest.raises(qp.QPError) as ei:
        qp.qp_fft_schedule(plan, qp.QP_FP32)
    assert ei.value.status == qp.QP_ERR_UNSUPPORTED
