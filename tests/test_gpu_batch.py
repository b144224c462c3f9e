"""Batched execution (many plans with different d, n, N in the same launches) against single solves and the
FP64 oracle."""
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


def _mixed_instances():
    c3 = W.cfg3()
    picks = [c3[0], c3[9], c3[33], c3[45]]          # d=1 N=64, d=1 N=128, d=2 N=8, d=2 N=16
    picks.append(W.random_instance(2, 3, (8, 6, 10), "sym", "taps", seed=41))
    picks.append(W.random_instance(3, 4, (6, 4, 6, 4), "diag", "taps", seed=42))
    picks.append(W.random_instance(1, 3, (8, 6, 9), "scalar", "taps", seed=43))   # odd last axis: runs of 1
    return picks


@pytest.mark.parametrize("mode", ["fp64", "refine"])
def test_batch_equals_single_solves_and_oracle(qp, mode):
    insts = _mixed_instances()
    m = qp.QP_MODE_FP64 if mode == "fp64" else qp.QP_MODE_FP32_REFINE
    plans = [qp.plan_from_instance(i) for i in insts]
    batch = qp.qp_batch_create(plans)
    As, infos = qp.qp_batch_homogenized(batch, tol=1e-10, mode=m)
    slot = 0
    for inst, plan, A in zip(insts, plans, As):
        A1, inf1 = qp.qp_homogenized(plan, tol=1e-10, mode=m)
        # same per-unit chunking and reduction order: batched iterates are bitwise those of the single solve
        assert np.array_equal(A, A1.real), (inst.name, A - A1.real)
        for j in range(inst.d):
            assert infos[slot + j]["iterations"] == inf1[j]["iterations"]
            assert infos[slot + j]["status"] == "QP_OK" and infos[slot + j]["rel_residual"] <= 1e-10
        slot += inst.d
        A_ref, *_ = O.homogenized(inst, tol=1e-13)
        assert np.abs(A - A_ref).max() <= 1e-10 * np.abs(A_ref).max(), inst.name


def test_cfg3_full_batch(qp):
    """All 64 instances of the batched workload in one solve (FP32 + FP64 refinement to 1e-10): every entry of
    every a* against the oracle's (tests/golden/astar_full_size.json, written by the oracle only), plus the exact
    1D identity (P1) for the d = 1 instances and symmetry with the Voigt-Reuss bounds (P8) for the d = 2 ones."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                       "astar_full_size.json")))["cfg3"]["instances"]
    insts = W.cfg3()
    plans = [qp.plan_from_instance(i) for i in insts]
    batch = qp.qp_batch_create(plans)
    As, infos = qp.qp_batch_homogenized(batch, tol=1e-10, mode=qp.QP_MODE_FP32_REFINE)
    assert len(infos) == sum(i.d for i in insts)
    assert all(x["status"] == "QP_OK" and x["rel_residual"] <= 1e-10 for x in infos)
    for inst, A, g in zip(insts, As, gold):
        assert g["name"] == inst.name
        ref = np.array(g["astar_re"])
        assert np.abs(A - ref).max() <= 1e-10 * np.abs(ref).max(), (inst.name, A - ref)
        a = W.sample_on_grid(inst.N, inst.coeff.taps_k, inst.coeff.taps_val)[0]
        if inst.d == 1:
            p1 = 1.0 / np.mean(1.0 / a)                        # P1: exact discrete identity in 1D
            assert abs(A[0, 0] - p1) <= 1e-10 * p1, inst.name
        else:
            assert abs(A[0, 1] - A[1, 0]) <= 1e-10 * np.abs(A).max()
            ev = np.linalg.eigvalsh(0.5 * (A + A.T))
            assert 1.0 / np.mean(1.0 / a) - 1e-10 <= ev.min() and ev.max() <= np.mean(a) + 1e-10   # P8
