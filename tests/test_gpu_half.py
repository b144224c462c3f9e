"""Half-spectrum plans (QP_SPECTRUM_HALF): the scheme on the Nyquist-free modes K'_N (the oracle's
homogenized_nyquist_free and its restricted operator), vectors holding only the modes with k_{n-1} >= 0.

Parity: the apply against the oracle's restricted operator on conjugate-symmetric vectors (FP64 1e-13, FP32 2e-6
relative to max |Q h|), the corrector right-hand sides and a* against the oracle's, full solves in both modes
against homogenized_nyquist_free (1e-10 relative), and on odd grids (no Nyquist modes) the half plan against the
full plan."""
import json
import os

import numpy as np
import pytest

import qp_workloads as W
from oracle import qp_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "astar_full_size.json")


@pytest.fixture(scope="module")
def qp():
    import paper_2404_06841_gb300 as qp
    assert torch.cuda.is_available()
    return qp


def _half(x, N):
    """The stored half of full-storage arrays x[..., N]: the modes with k_{n-1} = 0 .. ceil(N_{n-1}/2) - 1."""
    return np.ascontiguousarray(x[..., : (N[-1] + 1) // 2])


def _symmetric(N, seed):
    """A random vector on K'_N with h(-k) = conj(h(k)) (a real function), zero at the dropped modes."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    axes = tuple(range(len(N)))
    zm = np.roll(np.flip(z, axis=axes), 1, axis=axes)        # z(-k)
    return 0.5 * (z + np.conj(zm)) * O.nyquist_free_mask(N)


APPLY = [
    (3, 6, (4, 4, 4, 4, 4, 4), "diag", "star"),     # the large form's structure (star-1 taps, diagonal)
    (2, 4, (6, 4, 6, 8), "scalar", "star"),
    (1, 2, (10, 7), "scalar", "star"),              # odd last axis: ceil(7/2) = 4 stored, the wrap mirrored
    (2, 3, (6, 4, 10), "sym", "general"),
    (2, 3, (5, 6, 6), "diag", "general"),           # last axis stores 3 (odd): one mode per step
    (1, 3, (4, 5, 9), "scalar", "general"),
]


def _instance(d, n, N, kind, shape, seed):
    if shape == "star":
        return W.random_star_instance(d, n, N, kind, seed=seed)
    return W.random_instance(d, n, N, kind, "taps", seed=seed, radius=1)


@pytest.mark.parametrize("d,n,N,kind,shape", APPLY)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_half_apply_matches_restricted_oracle_operator(qp, d, n, N, kind, shape, prec):
    inst = _instance(d, n, N, kind, shape, seed=7 * n + d)
    plan = qp.plan_from_instance(inst, max_rhs=2, spectrum=qp.QP_SPECTRUM_HALF)
    info = qp.qp_plan_query(plan)
    assert info["spectrum"] == qp.QP_SPECTRUM_HALF and info["stored"] == plan.D
    keep = O.nyquist_free_mask(N)
    op = O.Operator(inst)
    hs = [_symmetric(N, 3), _symmetric(N, 4)]
    ref = np.stack([_half(keep * op(keep * h), N) for h in hs])
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    ht = torch.from_numpy(np.stack([_half(h, N) for h in hs])).to("cuda", dt)
    wt = torch.empty_like(ht)
    qp.qp_apply_stiffness(plan, ht, wt, qp.QP_FP64 if prec == "fp64" else qp.QP_FP32)
    got = wt.cpu().numpy().astype(np.complex128)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= (1e-13 if prec == "fp64" else 2e-6), err
    qp.qp_plan_destroy(plan)


@pytest.mark.parametrize("d,n,N,kind,shape", APPLY[:4])
def test_half_rhs_and_astar_reduce_match_oracle(qp, d, n, N, kind, shape):
    inst = _instance(d, n, N, kind, shape, seed=11 * n + d)
    plan = qp.plan_from_instance(inst, spectrum=qp.QP_SPECTRUM_HALF)
    Ahat = O.coefficient_modes(inst)
    keep = O.nyquist_free_mask(N)
    F = torch.zeros((d,) + plan.shape, dtype=torch.complex128, device="cuda")
    qp.qp_corrector_rhs(plan, 0, d, F)
    Us = []
    for j in range(d):
        ref = keep * O.corrector_rhs(inst.P, N, Ahat, j)
        assert np.abs(F[j].cpu().numpy() - _half(ref, N)).max() <= 1e-14 * np.abs(ref).max()
        Us.append(_symmetric(N, 20 + j))
    A = qp.qp_homogenized_reduce(plan, torch.from_numpy(np.stack([_half(u, N) for u in Us])).cuda())
    ref = O.homogenized_from_correctors(inst.P, N, Ahat, Us)
    assert np.abs(A - ref).max() <= 1e-13 * np.abs(ref).max()
    qp.qp_plan_destroy(plan)


SOLVE = [
    (3, 6, (4, 4, 4, 4, 4, 4), "diag", "star"), (2, 4, (8, 6, 8, 8), "scalar", "star"),
    (1, 2, (32, 32), "scalar", "star"), (1, 2, (17, 15), "scalar", "star"), (2, 3, (6, 4, 10), "sym", "general"),
    (2, 3, (5, 6, 6), "diag", "general"),
]


@pytest.mark.parametrize("d,n,N,kind,shape", SOLVE)
@pytest.mark.parametrize("mode", ["fp64", "refine"])
def test_half_homogenization_matches_nyquist_free_oracle(qp, d, n, N, kind, shape, mode):
    inst = _instance(d, n, N, kind, shape, seed=13 * n + d)
    plan = qp.plan_from_instance(inst, spectrum=qp.QP_SPECTRUM_HALF)
    m = qp.QP_MODE_FP64 if mode == "fp64" else qp.QP_MODE_FP32_REFINE
    A, infos = qp.qp_homogenized(plan, tol=1e-11, mode=m, maxit=2000)
    assert all(i["status"] == "QP_OK" and i["rel_residual"] <= 1e-11 for i in infos), infos
    A_ref, _, _, Ac_ref = O.homogenized_nyquist_free(inst, tol=1e-13)
    scale = np.abs(A_ref).max()
    assert np.abs(A.real - A_ref).max() <= 1e-10 * scale
    assert np.abs(A.imag).max() <= 1e-12 * scale           # real by construction on K'_N
    qp.qp_plan_destroy(plan)


def test_half_equals_full_on_odd_grids(qp):
    """All N_j odd: K'_N = K_N^n, so the half-spectrum plan solves the full scheme (a* within 1e-10, its solution's
    stored half equal to the full solution's)."""
    inst = W.random_star_instance(2, 4, (7, 5, 9, 7), "diag", seed=3)
    full = qp.plan_from_instance(inst)
    half = qp.plan_from_instance(inst, spectrum=qp.QP_SPECTRUM_HALF)
    A1, _ = qp.qp_homogenized(full, tol=1e-12)
    A2, _ = qp.qp_homogenized(half, tol=1e-12)
    assert np.abs(A1 - A2).max() <= 1e-10 * np.abs(A1).max()
    F = torch.zeros((2,) + inst.N, dtype=torch.complex128, device="cuda")
    qp.qp_corrector_rhs(full, 0, 2, F)
    U1 = torch.zeros_like(F)
    qp.qp_pcg_solve(full, F, U1, tol=1e-12)
    Fh = torch.from_numpy(_half(F.cpu().numpy(), inst.N)).cuda()
    U2 = torch.zeros_like(Fh)
    qp.qp_pcg_solve(half, Fh, U2, tol=1e-12)
    u1 = _half(U1.cpu().numpy(), inst.N)
    assert np.abs(U2.cpu().numpy() - u1).max() <= 1e-9 * np.abs(u1).max()


def test_half_rejects_what_it_does_not_build(qp):
    inst = W.random_instance(2, 3, (6, 6, 4), "sym", "grid", seed=2)
    with pytest.raises(qp.QPError) as ei:
        qp.plan_from_instance(inst, spectrum=qp.QP_SPECTRUM_HALF)
    assert ei.value.status == qp.QP_ERR_UNSUPPORTED
    plan = qp.plan_from_instance(W.cfg1(), spectrum=qp.QP_SPECTRUM_HALF)
    with pytest.raises(qp.QPError) as ei:
        qp.qp_homogenized(plan, precond=qp.QP_PRECOND_FROBENIUS)
    assert ei.value.status == qp.QP_ERR_UNSUPPORTED


def test_large_form_half_spectrum_against_golden(qp):
    """d = 3, n = 6, 16^6 grid on the Nyquist-free modes (15^6 unknowns, 16^5 x 8 stored): FP32 + FP64 refinement
    to 1e-10; a* within 1e-10 of the oracle's homogenized_nyquist_free (tests/golden, written by the oracle)."""
    gold = json.load(open(GOLDEN)).get("cfg4_half")
    if gold is None:
        pytest.skip("no oracle value for the 16^6 Nyquist-free scheme in tests/golden")
    inst = W.cfg4()
    plan = qp.plan_from_instance(inst, spectrum=qp.QP_SPECTRUM_HALF)
    A, infos = qp.qp_homogenized(plan, tol=1e-10, mode=qp.QP_MODE_FP32_REFINE, maxit=2000)
    assert all(i["status"] == "QP_OK" and i["rel_residual"] <= 1e-10 for i in infos), infos
    ref = np.array(gold["astar_re"])
    assert np.abs(A.real - ref).max() <= 1e-10 * np.abs(ref).max(), A.real - ref
    qp.qp_plan_destroy(plan)


@pytest.mark.parametrize("mode", ["fp64", "refine"])
def test_half_plans_in_a_batch(qp, mode):
    """A batch mixing half-spectrum plans (star-1 and general taps) with a full one: every plan's a* equals its
    own solve bit for bit (a unit reduces in the same order alone or batched; the vector passes weigh the half
    units' modes and not the full unit's) and the oracle's value for its scheme."""
    insts = [W.random_star_instance(2, 4, (6, 4, 6, 8), "diag", seed=71),
             W.random_instance(2, 3, (6, 4, 10), "sym", "taps", seed=72, radius=1),
             W.random_star_instance(1, 2, (16, 12), "scalar", seed=73)]
    spectra = [qp.QP_SPECTRUM_HALF, qp.QP_SPECTRUM_HALF, qp.QP_SPECTRUM_FULL]
    m = qp.QP_MODE_FP64 if mode == "fp64" else qp.QP_MODE_FP32_REFINE
    plans = [qp.plan_from_instance(i, spectrum=sp) for i, sp in zip(insts, spectra)]
    batch = qp.qp_batch_create(plans)
    As, infos = qp.qp_batch_homogenized(batch, tol=1e-11, mode=m, maxit=2000)
    assert all(i["status"] == "QP_OK" and i["rel_residual"] <= 1e-11 for i in infos), infos
    for inst, sp, plan, A in zip(insts, spectra, plans, As):
        A1, _ = qp.qp_homogenized(plan, tol=1e-11, mode=m, maxit=2000)
        assert np.array_equal(A, A1.real), inst.name
        if sp == qp.QP_SPECTRUM_HALF:
            A_ref, *_ = O.homogenized_nyquist_free(inst, tol=1e-13)
        else:
            A_ref, *_ = O.homogenized(inst, tol=1e-13)
        assert np.abs(A - A_ref).max() <= 1e-10 * np.abs(A_ref).max(), inst.name
    qp.qp_batch_destroy(batch)
    for p in plans:
        qp.qp_plan_destroy(p)
