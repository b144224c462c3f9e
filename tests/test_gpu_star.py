"""Star-1 plans (scalar or diagonal coefficient, taps only at m = 0 and m = +-e_j) take the specialised stencil
of the compressed mat-vec (Sec. 4.2): the weight lambda(k)^T C_t lambda(k -+ e_j) is formed from |lambda|^2 and
lambda . P_j, and each axis wraps with one compare and one select. Checked against the oracle's wraparound
convolution across the frequency wrap (k = ceil(N/2) - 1 <-> ceil(N/2) - N) and the storage wrap (axes of length
2 and 3, odd lengths, axes without taps), in every execution form, batched beside other plans, and with its kernel
parameter and shared-memory data sources, and its stored FP64 entries Q_ij and the ones it forms, giving bitwise
the same iterates."""
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


# (d, n, N, kind, real tap values, axes with taps); a tap needs |m_j| < N_j / 2, so axes of length 2 carry none
CASES = [
    (1, 2, (3, 4), "scalar", False, None),
    (2, 3, (5, 3, 4), "diag", False, None),
    (2, 4, (6, 7, 2, 8), "scalar", True, (0, 1, 3)),
    (3, 6, (4, 3, 2, 5, 3, 6), "diag", False, (0, 1, 3, 4, 5)),
    (3, 5, (9, 4, 6, 2, 10), "diag", True, (1, 2, 4)),
    (2, 4, (6, 4, 6, 5), "diag", False, None),          # odd last axis: the general stencil, runs of one
]


def _inst(case, seed):
    d, n, N, kind, real, axes = case
    return W.random_star_instance(d, n, N, kind, seed=seed, axes=axes, real=real)


def _rand(nrhs, N, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nrhs,) + tuple(N)) + 1j * rng.standard_normal((nrhs,) + tuple(N))


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("nrhs", [1, 3])
def test_star_apply_matches_oracle(qp, case, nrhs):
    inst = _inst(case, 11)
    plan = qp.plan_from_instance(inst, max_rhs=4)
    info = qp.qp_plan_query(plan)
    # FP64 entries Q_ij are stored for star-1 plans with runs of two modes (even last axis)
    assert info["star"] and info["stored_weights"] == (inst.N[-1] % 2 == 0)
    h = _rand(nrhs, inst.N, 3)
    op = O.Operator(inst)
    ref = np.stack([op(h[r]) for r in range(nrhs)])
    for prec, dt, tol in ((qp.QP_FP64, torch.complex128, 1e-13), (qp.QP_FP32, torch.complex64, 2e-6)):
        ht = torch.from_numpy(h).to("cuda", dt)
        wt = torch.empty_like(ht)
        qp.qp_apply_stiffness(plan, ht, wt, prec)
        err = np.abs(wt.cpu().numpy().astype(np.complex128) - ref).max() / np.abs(ref).max()
        assert err <= tol, (prec, err)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("mode", ["fp64", "refine"])
def test_star_solve_forms_bitwise_and_oracle(qp, case, mode):
    inst = _inst(case, 12)
    m = qp.QP_MODE_FP64 if mode == "fp64" else qp.QP_MODE_FP32_REFINE
    nrhs = 2
    F = _rand(nrhs, inst.N, 5)
    F.reshape(nrhs, -1)[:, 0] = 0
    out = {}
    for ex in (qp.QP_EXEC_PERSISTENT, qp.QP_EXEC_GRAPH, qp.QP_EXEC_DIRECT):
        plan = qp.plan_from_instance(inst, max_rhs=nrhs, exec_mode=ex)
        Ft = torch.from_numpy(F).cuda()
        Ut = torch.zeros_like(Ft)
        infos = qp.qp_pcg_solve(plan, Ft, Ut, tol=1e-10, maxit=2000, mode=m)
        out[ex] = (Ut.cpu().numpy(), infos)
    Up, ip = out[qp.QP_EXEC_PERSISTENT]
    for ex in (qp.QP_EXEC_GRAPH, qp.QP_EXEC_DIRECT):
        assert np.array_equal(Up, out[ex][0]) and ip == out[ex][1]
    op = O.Operator(inst)
    for r in range(nrhs):
        assert ip[r]["status"] == "QP_OK"
        res = np.linalg.norm(F[r] - op(Up[r])) / np.linalg.norm(F[r])
        assert res <= 1.2e-10, res


def test_star_plans_batched_beside_others_bitwise(qp):
    """Batched, a star-1 plan's stencil data comes from shared memory; alone, from the kernel parameter: the
    iterates must not differ by a bit."""
    insts = [_inst(CASES[1], 21), _inst(CASES[3], 22), W.cfg1(6), W.cfg4(4),
             W.random_instance(2, 3, (6, 4, 8), "sym", "taps", seed=23)]
    for mode in (qp.QP_MODE_FP64, qp.QP_MODE_FP32_REFINE):
        plans = [qp.plan_from_instance(i) for i in insts]
        batch = qp.qp_batch_create(plans)
        As, infos = qp.qp_batch_homogenized(batch, tol=1e-10, mode=mode)
        for inst, plan, A in zip(insts, plans, As):
            A1, _ = qp.qp_homogenized(plan, tol=1e-10, mode=mode)
            assert np.array_equal(A, A1.real), inst.name
            A_ref, *_ = O.homogenized(inst, tol=1e-13)
            assert np.abs(A - A_ref).max() <= 1e-10 * np.abs(A_ref).max(), inst.name


@pytest.mark.parametrize("d,n,N,kind,real", [(1, 2, (5, 8), "scalar", False), (2, 4, (6, 5, 4, 8), "diag", True),
                                             (3, 6, (4, 3, 4, 5, 4, 6), "diag", False),
                                             (2, 4, (4, 6, 5, 4), "scalar", False)])
def test_fixed_geometry_plain_apply_is_the_general_one(qp, d, n, N, kind, real):
    """Every axis with taps and d right-hand sides: the plain FP32 apply takes the kernel with the geometry compiled
    in; its first right-hand side must equal, bit for bit, the general kernel's (another right-hand-side count),
    and match the oracle."""
    inst = W.random_star_instance(d, n, N, kind, seed=40 + n, real=real)
    plan = qp.plan_from_instance(inst, max_rhs=4)
    h = _rand(4, inst.N, 9)
    ht = torch.from_numpy(h).to("cuda", torch.complex64)
    w_fixed = torch.empty((d,) + tuple(N), dtype=torch.complex64, device="cuda")
    qp.qp_apply_stiffness(plan, ht[:d].contiguous(), w_fixed, qp.QP_FP32, nrhs=d)
    other = d + 1
    w_gen = torch.empty((other,) + tuple(N), dtype=torch.complex64, device="cuda")
    qp.qp_apply_stiffness(plan, ht[:other].contiguous(), w_gen, qp.QP_FP32, nrhs=other)
    assert torch.equal(w_fixed, w_gen[:d])
    op = O.Operator(inst)
    ref = np.stack([op(h[r]) for r in range(d)])
    err = np.abs(w_fixed.cpu().numpy().astype(np.complex128) - ref).max() / np.abs(ref).max()
    assert err <= 2e-6, err


@pytest.mark.parametrize("d,n,N,kind,real", [(1, 2, (5, 8), "scalar", False), (2, 4, (6, 5, 4, 8), "diag", True),
                                             (3, 6, (4, 3, 4, 5, 4, 6), "diag", False),
                                             (2, 4, (4, 6, 5, 4), "scalar", False),
                                             # 32^4: 1,024 chunks, so the FP32 batch kernel with the geometry
                                             # compiled in walks several chunks per block (grid of resident blocks)
                                             (2, 4, (32, 32, 32, 32), "diag", False),
                                             # six axes and more chunks than resident blocks: the FP32 batch kernel
                                             # with the geometry compiled in walks chunks of contiguous runs (1,024
                                             # chunks of 1,024 modes) and sweep waves (1,152 chunks of 2,048 modes)
                                             (3, 6, (8, 8, 8, 8, 8, 32), "diag", False),
                                             (3, 6, (8, 8, 8, 8, 8, 72), "diag", True)])
def test_fixed_geometry_solves_are_the_general_ones(qp, d, n, N, kind, real):
    """Every axis with taps and d right-hand sides: the persistent solve and the graph form's FP32 batch apply take
    the kernels with the geometry compiled in; with d + 1 right-hand sides the general ones run. Each right-hand
    side's iterates do not depend on the others, so the first d solutions must agree bit for bit across the four
    runs, in FP64 and in refinement mode, and reach the tolerance against the oracle."""
    inst = W.random_star_instance(d, n, N, kind, seed=50 + n, real=real)
    F = _rand(d + 1, inst.N, 6)
    F.reshape(d + 1, -1)[:, 0] = 0
    op = O.Operator(inst)
    for m in (qp.QP_MODE_FP64, qp.QP_MODE_FP32_REFINE):
        runs = []
        for ex in (qp.QP_EXEC_PERSISTENT, qp.QP_EXEC_GRAPH):
            plan = qp.plan_from_instance(inst, max_rhs=d + 1, exec_mode=ex)
            for nr in (d, d + 1):
                Ft = torch.from_numpy(F[:nr].copy()).cuda()
                Ut = torch.zeros_like(Ft)
                infos = qp.qp_pcg_solve(plan, Ft, Ut, tol=1e-10, maxit=2000, mode=m)
                runs.append((Ut.cpu().numpy()[:d], infos[:d]))
        U0, i0 = runs[0]
        for U1, i1 in runs[1:]:
            assert np.array_equal(U0, U1) and i0 == i1
        for r in range(d):
            assert i0[r]["status"] == "QP_OK"
            res = np.linalg.norm(F[r] - op(U0[r])) / np.linalg.norm(F[r])
            assert res <= 1.2e-10, res


def test_general_taps_are_not_star(qp):
    """General taps take the general stencil; with FP64 vectors the plan stores their FP64 entries per (tap, mode)
    (read by its FP64 applies), without them it stores none."""
    inst = W.random_instance(2, 3, (6, 4, 8), "sym", "taps", seed=23)
    info = qp.qp_plan_query(qp.plan_from_instance(inst))
    assert not info["star"] and info["stored_weights"]
    info = qp.qp_plan_query(qp.plan_from_instance(inst, precisions=2))
    assert not info["star"] and not info["stored_weights"]
    inst = W.random_instance(2, 3, (6, 4, 8), "scalar", "taps", seed=24)   # taps off the axes (|m|_inf <= 1)
    assert not qp.qp_plan_query(qp.plan_from_instance(inst))["star"]


@pytest.mark.parametrize("kind,seed", [("sym", 31), ("scalar", 32), ("diag", 33)])
def test_general_taps_stored_fp64_entries_equal_formed(qp, kind, seed):
    """The FP64 apply of a general-taps plan reads its stored entries; a plan without FP64 solve workspace forms
    them (precisions = FP32 solve only still allows FP64 applies): bit for bit the same Q h, and the oracle's."""
    inst = W.random_instance(2, 4, (6, 4, 6, 8), kind, "taps", seed=seed, radius=1)
    p_stored = qp.plan_from_instance(inst)
    p_formed = qp.plan_from_instance(inst, precisions=2)
    assert qp.qp_plan_query(p_stored)["stored_weights"] and not qp.qp_plan_query(p_formed)["stored_weights"]
    rng = np.random.default_rng(seed)
    h = rng.standard_normal((2,) + inst.N) + 1j * rng.standard_normal((2,) + inst.N)
    ht = torch.from_numpy(h).cuda()
    w1, w2 = torch.empty_like(ht), torch.empty_like(ht)
    qp.qp_apply_stiffness(p_stored, ht, w1, qp.QP_FP64)
    qp.qp_apply_stiffness(p_formed, ht, w2, qp.QP_FP64)
    assert torch.equal(w1, w2)
    op = O.Operator(inst)
    ref = np.stack([op(h[r]) for r in range(2)])
    assert np.abs(w1.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()


def test_misaligned_vectors_are_rejected_before_any_launch(qp):
    inst = W.cfg1(4)
    plan = qp.plan_from_instance(inst)
    buf = torch.zeros(inst.D + 1, dtype=torch.complex64, device="cuda")
    good = torch.zeros(inst.D, dtype=torch.complex64, device="cuda")
    with pytest.raises(qp.QPError) as ei:
        qp.qp_apply_stiffness(plan, buf[1:], good, qp.QP_FP32, nrhs=1)   # 8-byte offset
    assert ei.value.status == qp.QP_ERR_INVALID_ARG and "aligned" in str(ei.value)


def test_misaligned_rhs_reduce_and_fft_pointers_are_rejected(qp):
    """qp_corrector_rhs, qp_homogenized_reduce and qp_fft check their device pointers' alignment (16 bytes for
    complex128 vectors) before any launch; the plan and the stream stay usable afterwards."""
    inst = W.cfg1(4)
    plan = qp.plan_from_instance(inst)
    d, D = inst.d, inst.D
    buf = torch.zeros(d * D + 1, dtype=torch.complex128, device="cuda")
    raw = buf.view(torch.float64)[1:1 + 2 * d * D]          # 8 bytes past a 16-byte boundary
    assert raw.data_ptr() % 16 == 8
    for call in (lambda: qp.qp_corrector_rhs(plan, 0, d, raw),
                 lambda: qp.qp_homogenized_reduce(plan, raw),
                 lambda: qp.qp_fft(raw, inst.N, sign=-1, precision=qp.QP_FP64, count=d)):
        with pytest.raises(qp.QPError) as ei:
            call()
        assert ei.value.status == qp.QP_ERR_INVALID_ARG and "aligned" in str(ei.value)
    F = torch.zeros(d, D, dtype=torch.complex128, device="cuda")
    qp.qp_corrector_rhs(plan, 0, d, F)
    torch.cuda.synchronize()
    assert torch.isfinite(torch.view_as_real(F)).all() and F.abs().max().item() > 0.0
