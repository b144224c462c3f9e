"""The hand-written n-dim DFT (qp_fft) and the FFT backend of the stiffness apply against numpy and the oracle."""
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


FFT_SHAPES = [(2,), (3,), (4,), (6,), (9,), (12,), (18,), (27,), (32,), (48,), (64,), (96,), (128,), (256,),
              (512,), (1024,), (8, 12, 6), (32, 32), (16, 16, 16, 16), (4, 4, 4, 4, 4, 4), (3, 64), (27, 2, 24),
              (1024, 4), (6, 96)]


@pytest.mark.parametrize("shape", FFT_SHAPES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fft_matches_numpy(qp, shape, prec):
    rng = np.random.default_rng(len(shape) * 100 + shape[0])
    count = 3
    x = rng.standard_normal((count,) + shape) + 1j * rng.standard_normal((count,) + shape)
    axes = tuple(range(1, len(shape) + 1))
    fwd = np.fft.fftn(x, axes=axes)
    inv = np.fft.ifftn(x, axes=axes) * np.prod(shape)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    tol = (1e-13 if prec == "fp64" else 2e-6) * np.log2(max(np.prod(shape), 2))
    for sign, ref in ((-1, fwd), (+1, inv)):
        t = torch.from_numpy(x).to("cuda", dt).contiguous()
        qp.qp_fft(t, shape, sign=sign)
        got = t.cpu().numpy().astype(np.complex128)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= tol, (shape, sign, err)


# Grids with every axis <= 32 run group passes (the schedule the autotuner timed fastest; test_gpu_autotune checks
# every candidate); (64, 48) has axes above 32 and takes the per-axis passes.
GRID_CASES = [(1, 2, (8, 12), "scalar"), (2, 2, (16, 8), "sym"), (2, 3, (8, 6, 4), "diag"), (3, 3, (4, 6, 8), "sym"),
              (2, 4, (6, 4, 8, 4), "sym"), (1, 1, (32,), "scalar"), (2, 4, (16, 12, 16, 24), "sym"),
              (3, 6, (6, 6, 6, 6, 6, 6), "diag"), (1, 2, (64, 48), "scalar")]


@pytest.mark.parametrize("d,n,N,kind", GRID_CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fft_apply_matches_oracle_on_full_support_grids(qp, d, n, N, kind, prec):
    inst = W.random_instance(d, n, N, kind, "grid", seed=7 + d + n, nonlinear=True)
    plan = qp.plan_from_instance(inst, max_rhs=2)
    assert qp.qp_plan_query(plan)["backend"] == "fft"
    rng = np.random.default_rng(1)
    h = rng.standard_normal((2,) + N) + 1j * rng.standard_normal((2,) + N)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    ht = torch.from_numpy(h).to("cuda", dt)
    wt = torch.empty_like(ht)
    qp.qp_apply_stiffness(plan, ht, wt, qp.QP_FP64 if prec == "fp64" else qp.QP_FP32)
    Ag = O.coefficient_grid(inst)
    ref = np.stack([O.apply_fft(inst.P, N, Ag, h[r]) for r in range(2)])
    err = np.abs(wt.cpu().numpy().astype(np.complex128) - ref).max() / np.abs(ref).max()
    assert err <= (1e-12 if prec == "fp64" else 1e-5), err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fft_apply_three_group_schedule_sampled(qp, prec):
    """16^5 x 8 modes: the autotuner's schedule, and forced a five-pass schedule (three groups of axes: gradient
    + inverse over the first group, plain passes over the middle one), compared with the taps backend on the
    whole vector and with the oracle's pointwise sum at sampled modes."""
    N = (16, 16, 16, 16, 16, 8)
    inst = W.random_instance(1, 6, N, "scalar", "taps", seed=23, nmodes=6)
    p_f = qp.plan_from_instance(inst, backend=qp.QP_BACKEND_FFT, max_rhs=1)
    p_t = qp.plan_from_instance(inst, max_rhs=1)
    rng = np.random.default_rng(4)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    pr = qp.QP_FP64 if prec == "fp64" else qp.QP_FP32
    h = torch.complex(torch.randn((1,) + N, dtype=torch.float64), torch.randn((1,) + N, dtype=torch.float64))
    h = h.to("cuda", dt)
    w_t = torch.empty_like(h)
    qp.qp_apply_stiffness(p_t, h, w_t, pr)
    tol = 1e-12 if prec == "fp64" else 2e-5
    scale = float(w_t.abs().max())
    pts = [tuple(int(x) for x in (rng.integers(0, Nj) for Nj in N)) for _ in range(64)]
    pts += [(0,) * 6, tuple(Nj // 2 for Nj in N), tuple(Nj - 1 for Nj in N)]
    hc = h[0].cpu().numpy().astype(np.complex128)
    ref = O.apply_taps_at(inst.P, N, inst.coeff.taps_k, inst.coeff.taps_val, "scalar", hc, pts)
    chosen = qp.qp_fft_schedule(p_f, pr)
    five = [i for i in range(chosen["count"]) if (qp.qp_fft_set_schedule(p_f, pr, i) or True)
            and "5 passes" in qp.qp_fft_schedule(p_f, pr)["text"]]
    assert five, "no three-group schedule among the candidates"
    for idx in (chosen["index"], five[0]):
        qp.qp_fft_set_schedule(p_f, pr, idx)
        w_f = torch.empty_like(h)
        qp.qp_apply_stiffness(p_f, h, w_f, pr)
        assert float((w_f - w_t).abs().max()) <= tol * scale
        got = np.array([complex(w_f[(0,) + p].item()) for p in pts])
        assert np.abs(got - ref).max() <= tol * scale


@pytest.mark.parametrize("d,n,N,kind", [(2, 3, (8, 6, 4), "sym"), (1, 2, (12, 16), "scalar"), (3, 3, (6, 4, 8), "diag")])
def test_taps_backend_equals_fft_backend(qp, d, n, N, kind):
    """The same tap coefficient through the stencil and through the DFT gives the same operator."""
    inst = W.random_instance(d, n, N, kind, "taps", seed=3)
    p_t = qp.plan_from_instance(inst)
    p_f = qp.plan_from_instance(inst, backend=qp.QP_BACKEND_FFT)
    rng = np.random.default_rng(2)
    h = torch.from_numpy(rng.standard_normal((d,) + N) + 1j * rng.standard_normal((d,) + N)).cuda()
    w1, w2 = torch.empty_like(h), torch.empty_like(h)
    qp.qp_apply_stiffness(p_t, h, w1, qp.QP_FP64)
    qp.qp_apply_stiffness(p_f, h, w2, qp.QP_FP64)
    assert float((w1 - w2).abs().max() / w1.abs().max()) <= 1e-12
    A1, _ = qp.qp_homogenized(p_t, tol=1e-11)
    A2, _ = qp.qp_homogenized(p_f, tol=1e-11)
    assert np.abs(A1 - A2).max() <= 1e-10 * np.abs(A1).max()


@pytest.mark.parametrize("mode", ["fp64", "refine"])
def test_fft_backend_homogenized_matches_oracle(qp, mode):
    inst = W.random_instance(2, 3, (8, 8, 6), "sym", "grid", seed=19, nonlinear=True)
    plan = qp.plan_from_instance(inst)
    A, infos = qp.qp_homogenized(plan, tol=1e-10, mode=qp.QP_MODE_FP64 if mode == "fp64" else qp.QP_MODE_FP32_REFINE)
    A_ref, Us, _, Ac = O.homogenized(inst, tol=1e-13)
    assert np.abs(A.real - A_ref).max() <= 1e-10 * np.abs(A_ref).max()
    assert all(i["status"] == "QP_OK" and i["rel_residual"] <= 1e-10 for i in infos)
    # RHS and a* reduction on this backend
    Ahat = O.coefficient_modes(inst)
    F = torch.zeros((2,) + inst.N, dtype=torch.complex128, device="cuda")
    qp.qp_corrector_rhs(plan, 0, 2, F)
    for j in range(2):
        ref = O.corrector_rhs(inst.P, inst.N, Ahat, j)
        assert np.abs(F[j].cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
    U = torch.from_numpy(np.stack(Us)).cuda()
    Ared = qp.qp_homogenized_reduce(plan, U)
    assert np.abs(Ared - Ac).max() <= 1e-13 * np.abs(Ac).max()


def test_keller_dykhne_and_one_dimensional_identity_on_the_fft_backend(qp):
    N = 16
    y = 2 * np.pi * np.arange(N) / N
    Y1, Y2 = np.meshgrid(y, y, indexing="ij")
    a = np.exp(0.5 * (np.cos(Y1) - np.cos(Y2)))
    inst = W.Instance("kd", np.eye(2), (N, N), W.Coefficient("scalar", grid=a[None].copy()))
    A, _ = qp.qp_homogenized(qp.plan_from_instance(inst), tol=1e-12)
    assert np.abs(A.real - np.eye(2)).max() <= 1e-10                      # P3: A* = I
    inst1 = W.random_instance(1, 2, (24, 16), "scalar", "grid", seed=8, nonlinear=True)
    A1, _ = qp.qp_homogenized(qp.plan_from_instance(inst1), tol=1e-12)
    g = inst1.coeff.grid[0]
    assert abs(A1[0, 0].real - 1.0 / np.mean(1.0 / g)) <= 1e-11 * A1[0, 0].real   # P1


def test_cfg2_full_size_refinement_against_golden(qp):
    """cfg2 (d=2, n=4, 32^4 modes, SPD 2x2 grid coefficient): FP32 inner solves inside FP64 refinement reach the
    oracle's a* (computed by tests/golden/make_golden.py) to 1e-10 relative, as does the plain FP64 solve."""
    gold = json.load(open(os.path.join(GOLDEN, "astar_full_size.json")))["cfg2"]
    inst = W.cfg2()
    plan = qp.plan_from_instance(inst)
    ref = np.array(gold["astar_re"])
    ref_im = np.array(gold["astar_im"])   # Im A*_12 ~ -5.6e-8: the Nyquist content of the clamped coefficient
    for mode in (qp.QP_MODE_FP32_REFINE, qp.QP_MODE_FP64):
        A, infos = qp.qp_homogenized(plan, tol=1e-10, mode=mode)
        assert all(i["status"] == "QP_OK" and i["rel_residual"] <= 1e-10 for i in infos)
        assert np.abs(A.real - ref).max() <= 1e-10 * np.abs(ref).max(), (mode, A.real - ref)
        assert np.abs(A.imag - ref_im).max() <= 1e-10 * np.abs(ref).max(), (mode, A.imag - ref_im)
