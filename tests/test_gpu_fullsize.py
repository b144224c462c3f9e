"""Full-size homogenization parity against the oracle's a* (written by tests/golden/make_golden.py, which calls
only oracle/qp_oracle.py): the large workload (d = 3 lifted to n = 6, 16^6 modes, three correctors) in both
solve modes, each element of a* within the stated 1e-10 relative bound (eq. homcoefficient, Sec. 5.2; App. D).
The 64 instances of the batched workload are checked the same way in test_gpu_batch.py."""
import json
import os

import numpy as np
import pytest

import qp_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "astar_full_size.json")


@pytest.fixture(scope="module")
def qp():
    import paper_2404_06841_gb300 as qp
    assert torch.cuda.is_available()
    return qp


@pytest.mark.parametrize("mode", ["refine", "fp64"])
def test_large_form_16_6_against_golden(qp, mode):
    """d = 3, n = 6, 16^6 = 16,777,216 modes, diagonal coefficient with 13 taps per component: FP32 inner solves
    in FP64 refinement, and the plain FP64 solve, both to a true relative residual of 1e-10; Re a* and Im a*
    within 1e-10 of the oracle's (relative to max |a*|)."""
    gold = json.load(open(GOLDEN))["cfg4"]
    inst = W.cfg4()
    plan = qp.plan_from_instance(inst)
    m = qp.QP_MODE_FP32_REFINE if mode == "refine" else qp.QP_MODE_FP64
    A, infos = qp.qp_homogenized(plan, tol=1e-10, mode=m, maxit=2000)
    qp.qp_plan_destroy(plan)
    assert all(i["status"] == "QP_OK" and i["rel_residual"] <= 1e-10 for i in infos), infos
    ref_re = np.array(gold["astar_re"])
    ref_im = np.array(gold["astar_im"])
    scale = np.abs(ref_re).max()
    assert np.abs(A.real - ref_re).max() <= 1e-10 * scale, A.real - ref_re
    assert np.abs(A.imag - ref_im).max() <= 1e-10 * scale, A.imag - ref_im
