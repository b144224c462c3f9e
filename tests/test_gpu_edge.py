"""Edge cases at the limits of the C ABI: the maximum tap count, a 1024-long axis on both backends, the smallest
grids, one torus axis (the periodic case), and sizes beyond the limits rejected with QP_ERR_INVALID_ARG."""
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


def test_maximum_tap_count(qp):
    """255 taps (127 Hermitian pairs within |m| <= 2 and the mean) with a full symmetric 2 x 2 coefficient."""
    inst = W.random_instance(2, 4, (6, 6, 6, 6), "sym", "taps", seed=21, radius=2, nmodes=127)
    assert len(inst.coeff.taps_k) == 255
    plan = qp.plan_from_instance(inst)
    assert qp.qp_plan_query(plan)["ntaps"] == 255
    rng = np.random.default_rng(2)
    h = rng.standard_normal((2,) + inst.N) + 1j * rng.standard_normal((2,) + inst.N)
    ref = np.stack([O.apply_convolution(inst.P, inst.N, O.coefficient_modes(inst), h[r]) for r in range(2)])
    for prec, dt, tol in ((qp.QP_FP64, torch.complex128, 1e-13), (qp.QP_FP32, torch.complex64, 2e-6)):
        ht = torch.from_numpy(h).to("cuda", dt)
        wt = torch.empty_like(ht)
        qp.qp_apply_stiffness(plan, ht, wt, prec)
        err = np.abs(wt.cpu().numpy().astype(np.complex128) - ref).max() / np.abs(ref).max()
        assert err <= tol, err
    A, infos = qp.qp_homogenized(plan, tol=1e-11)
    A_ref, *_ = O.homogenized(inst, tol=1e-13)
    assert np.abs(A.real - A_ref).max() <= 1e-10 * np.abs(A_ref).max()


def test_more_taps_than_the_maximum_are_rejected(qp):
    inst = W.random_instance(1, 4, (8, 8, 8, 8), "scalar", "taps", seed=22, radius=2, nmodes=140)
    assert len(inst.coeff.taps_k) > 256
    with pytest.raises(qp.QPError) as ei:
        qp.plan_from_instance(inst)
    assert ei.value.status == qp.QP_ERR_INVALID_ARG


@pytest.mark.parametrize("backend", ["taps", "fft"])
def test_axis_of_1024_modes_harmonic_mean(qp, backend):
    """d = 1 (a laminate-type quasiperiodic coefficient along one direction): the discrete a* is the harmonic mean
    of the grid samples exactly (pin P1), here with 1024 modes on the first axis."""
    k, v = W.cos_sum_taps(2, 3.0, 1.0)
    inst = W.Instance("long_axis", np.array([[1.0, W.SQRT2]]), (1024, 4), W.Coefficient("scalar", k, v))
    plan = qp.plan_from_instance(inst, backend=qp.QP_BACKEND_TAPS if backend == "taps" else qp.QP_BACKEND_FFT)
    A, infos = qp.qp_homogenized(plan, tol=1e-12)
    a = W.sample_on_grid(inst.N, k, v)[0]
    harmonic = 1.0 / np.mean(1.0 / a)
    assert abs(A[0, 0].real - harmonic) <= 1e-11 * harmonic


def test_smallest_grids_and_one_axis(qp):
    # N = (2, 2): only the mean fits |m| < N/2, so A is constant and Jacobi-PCG converges in one iteration (pin P5)
    k = np.zeros((1, 2), np.int32)
    inst = W.Instance("n2", np.array([[1.0, W.SQRT2]]), (2, 2), W.Coefficient("scalar", k, np.array([[4.0]], complex)))
    A, infos = qp.qp_homogenized(qp.plan_from_instance(inst), tol=1e-12)
    assert abs(A[0, 0].real - 4.0) <= 1e-14 and infos[0]["iterations"] <= 1
    # one torus axis, P = (1): the periodic spectral method; a = 2 + cos theta on 3, 9 and 27 modes (odd lengths)
    k, v = W.cos_sum_taps(1, 2.0, 1.0)
    for N in (3, 9, 27):
        inst = W.Instance("p%d" % N, np.array([[1.0]]), (N,), W.Coefficient("scalar", k, v))
        A, _ = qp.qp_homogenized(qp.plan_from_instance(inst), tol=1e-13)
        a = W.sample_on_grid((N,), k, v)[0]
        assert abs(A[0, 0].real - 1.0 / np.mean(1.0 / a)) <= 1e-12


def test_sizes_beyond_the_limits_are_rejected(qp):
    k, v = W.cos_sum_taps(2, 3.0, 1.0)
    c = W.Coefficient("scalar", k, v)
    for N in ((2048, 4), (4, 1)):
        with pytest.raises(qp.QPError) as ei:
            qp.qp_plan_create(1, 2, [[1.0, W.SQRT2]], list(N), c)
        assert ei.value.status == qp.QP_ERR_INVALID_ARG
    with pytest.raises(qp.QPError) as ei:   # more right-hand sides than QP_MAX_RHS
        qp.qp_plan_create(1, 2, [[1.0, W.SQRT2]], [8, 8], c, max_rhs=5)
    assert ei.value.status == qp.QP_ERR_INVALID_ARG


def test_tap_modes_beyond_127_rejected_by_both_entry_points(qp):
    """Tap modes are held in 8 bits on the device: |m_j| = 130 on an axis of 512 modes (within |m_j| < N_j / 2)
    is rejected with QP_ERR_INVALID_ARG by the plan and by the allocation-free solve, before any device work."""
    k = np.array([[0, 0], [130, 0], [-130, 0]], np.int32)
    v = np.array([[3.0], [0.25], [0.25]], complex)
    c = W.Coefficient("scalar", k, v)
    with pytest.raises(qp.QPError) as ei:
        qp.qp_plan_create(1, 2, [[1.0, W.SQRT2]], [512, 4], c)
    assert ei.value.status == qp.QP_ERR_INVALID_ARG and "127" in str(ei.value)
    F = torch.zeros((1, 512 * 4), dtype=torch.complex128, device="cuda")
    with pytest.raises(qp.QPError) as ei:
        qp.qp_pcg_solve_taps_static(1, 2, [[1.0, W.SQRT2]], [512, 4], c, F, F.clone())
    assert ei.value.status == qp.QP_ERR_INVALID_ARG and "127" in str(ei.value)


def test_indefinite_mean_tap_rejected_by_both_entry_points(qp):
    """A diagonal 2 x 2 coefficient whose mean tap has a negative entry (not elliptic): QP_ERR_NOT_ELLIPTIC from the
    plan and from the allocation-free solve alike."""
    k = np.array([[0, 0, 0, 0], [1, 0, 0, 0], [-1, 0, 0, 0]], np.int32)
    v = np.array([[3.0, -1.0], [0.25, 0.25], [0.25, 0.25]], complex)
    c = W.Coefficient("diag", k, v)
    P = [[1.0, W.SQRT2, 0, 0], [0, 0, 1.0, W.SQRT3]]
    with pytest.raises(qp.QPError) as ei:
        qp.qp_plan_create(2, 4, P, [4, 4, 4, 4], c)
    assert ei.value.status == qp.QP_ERR_NOT_ELLIPTIC
    F = torch.zeros((2, 256), dtype=torch.complex128, device="cuda")
    with pytest.raises(qp.QPError) as ei:
        qp.qp_pcg_solve_taps_static(2, 4, P, [4, 4, 4, 4], c, F, F.clone())
    assert ei.value.status == qp.QP_ERR_NOT_ELLIPTIC
