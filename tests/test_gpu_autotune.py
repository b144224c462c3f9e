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
    assert s2["index"] == s1["index"] and s2["ms"] == s1["ms"]   # the first plan's timing, carried by the cache
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


def test_auto_backend_takes_the_fft_for_a_dense_tap_list(qp):
    """255 taps (|m| <= 2 in 4-D) with a full 2x2 coefficient on 24^4 modes: the stencil's work per mode is
    proportional to the tap count, so the timed choice of QP_BACKEND_AUTO is the FFT backend; its apply and a*
    match the forced stencil's (and the apply the oracle's pointwise sum at sampled modes)."""
    N = (24, 24, 24, 24)
    inst = W.random_instance(2, 4, N, "sym", "taps", seed=71, radius=2, nmodes=127)
    assert len(inst.coeff.taps_k) == 255
    p_auto = qp.plan_from_instance(inst)
    p_taps = qp.plan_from_instance(inst, backend=qp.QP_BACKEND_TAPS)
    assert qp.qp_plan_query(p_auto)["backend"] == "fft" and qp.qp_plan_query(p_taps)["backend"] == "taps"
    rng = np.random.default_rng(6)
    h = torch.complex(torch.randn((2,) + N, dtype=torch.float64), torch.randn((2,) + N, dtype=torch.float64)).cuda()
    wa, wt = torch.empty_like(h), torch.empty_like(h)
    qp.qp_apply_stiffness(p_auto, h, wa, qp.QP_FP64)
    qp.qp_apply_stiffness(p_taps, h, wt, qp.QP_FP64)
    scale = float(wt.abs().max())
    assert float((wa - wt).abs().max()) <= 1e-12 * scale
    pts = [tuple(int(x) for x in (rng.integers(0, Nj) for Nj in N)) for _ in range(16)]
    ref = O.apply_taps_at(inst.P, N, inst.coeff.taps_k, inst.coeff.taps_val, "sym", h[0].cpu().numpy(), pts)
    got = np.array([complex(wa[(0,) + p].item()) for p in pts])
    assert np.abs(got - ref).max() <= 1e-12 * scale
    A1, i1 = qp.qp_homogenized(p_auto, tol=1e-10)
    A2, i2 = qp.qp_homogenized(p_taps, tol=1e-10)
    assert all(i["status"] == "QP_OK" for i in i1 + i2)
    assert np.abs(A1 - A2).max() <= 1e-9 * np.abs(A2).max()


def test_auto_backend_keeps_the_stencil_for_few_taps(qp):
    for inst in (W.cfg1(), W.random_instance(2, 4, (16, 16, 16, 16), "sym", "taps", seed=72, nmodes=20)):
        assert qp.qp_plan_query(qp.plan_from_instance(inst))["backend"] == "taps"


def test_tuning_cache_file_round_trip(qp, tmp_path):
    """The schedule cache saved to a file and loaded by a later plan's process state: with the autotuner off and
    the in-memory cache cleared, a plan takes the heuristic (index -1); after loading the file it takes the timed
    choice with its timing. A malformed file is rejected and merges nothing."""
    inst = W.random_instance(2, 4, (6, 8, 4, 6), "diag", "grid", seed=62, nonlinear=True)
    p1 = qp.plan_from_instance(inst, max_rhs=2)
    s1 = qp.qp_fft_schedule(p1, qp.QP_FP32)
    path = tmp_path / "fft_tune.txt"
    assert qp.qp_fft_tune_cache_save(str(path)) >= 1
    assert path.read_text().startswith("qp-fft-tune-cache 1 ")
    bad = tmp_path / "bad.txt"
    bad.write_text("not a cache\n")
    try:
        qp.qp_fft_tune_cache_clear()
        qp.qp_set_fft_autotune(False)
        p2 = qp.plan_from_instance(inst, max_rhs=2)
        assert qp.qp_fft_schedule(p2, qp.QP_FP32)["index"] == -1
        with pytest.raises(qp.QPError) as ei:
            qp.qp_fft_tune_cache_load(str(bad))
        assert ei.value.status == qp.QP_ERR_INVALID_ARG
        assert qp.qp_fft_tune_cache_load(str(path)) >= 1
        p3 = qp.plan_from_instance(inst, max_rhs=2)
        s3 = qp.qp_fft_schedule(p3, qp.QP_FP32)
        assert s3["index"] == s1["index"] and s3["ms"] == pytest.approx(s1["ms"], rel=1e-6)
        for p in (p2, p3):
            qp.qp_plan_destroy(p)
    finally:
        qp.qp_set_fft_autotune(True)
    qp.qp_plan_destroy(p1)
