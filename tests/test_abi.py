"""The C ABI library: builds, loads, exports every declared symbol, validates arguments on the host (no GPU)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "qp.h")).read()
    return sorted(set(re.findall(r"^\s*(?:qp_status|const char\*|uint64_t)\s+(qp_\w+)\s*\(", src, re.M)))


def test_library_loads_and_exports_every_declared_symbol():
    import ctypes
    import paper_2404_06841_gb300 as qp
    lib = ctypes.CDLL(qp.LIB_PATH)
    decl = _declared()
    assert len(decl) >= 13
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(qp.EXPORTS) == decl


def test_header_enums_match_binding():
    import paper_2404_06841_gb300 as qp
    src = open(os.path.join(ROOT, "include", "qp.h")).read()
    pairs = re.findall(r"\b(QP_[A-Z0-9_]+)\s*=\s*(\d+)", src)
    names = {n for n, _ in pairs}
    assert {"QP_OK", "QP_ERR_CUDA", "QP_EXEC_AUTO", "QP_EXEC_PERSISTENT", "QP_MODE_FP32_REFINE"} <= names
    for name, val in pairs:
        if name.startswith("QP_MAX_"):
            continue
        assert getattr(qp, name) == int(val), name


@pytest.mark.parametrize("d,n,N,msg", [
    (0, 2, [4, 4], "d must be"), (4, 4, [4] * 4, "d must be"), (2, 1, [4], "n must"), (1, 7, [4] * 7, "n must"),
    (1, 2, [1, 4], "N_j"), (1, 2, [4, 2048], "N_j"),
])
def test_host_validation_rejects_bad_geometry(d, n, N, msg):
    import paper_2404_06841_gb300 as qp
    import qp_workloads as W
    P = np.ones((max(d, 1), max(n, 1)))
    coeff = W.cfg0().coeff
    with pytest.raises(qp.QPError) as ei:
        qp.qp_plan_create(d, n, P.reshape(-1)[: max(d, 0) * max(n, 0)] if d >= 1 and n >= 1 else P, N, coeff,
                          stream=0)
    assert ei.value.status == qp.QP_ERR_INVALID_ARG
    assert msg in str(ei.value)
    assert msg in qp.qp_last_error()


def test_null_arguments_are_rejected_without_touching_the_gpu():
    import ctypes as C
    import paper_2404_06841_gb300 as qp
    lib = qp._lib
    assert lib.qp_plan_create(1, 2, None, None, None, None, None, None) == qp.QP_ERR_INVALID_ARG
    assert lib.qp_apply_stiffness(None, 1, None, None, 0, None) == qp.QP_ERR_INVALID_ARG
    assert lib.qp_pcg_solve(None, 1, None, None, None, None, None) == qp.QP_ERR_INVALID_ARG
    assert lib.qp_homogenized(None, None, None, None, None, None) == qp.QP_ERR_INVALID_ARG
    assert lib.qp_fft(0, None, 1, None, -1, 0, None) == qp.QP_ERR_INVALID_ARG
    n3 = (C.c_int * 1)(5)
    assert lib.qp_fft(1, n3, 1, C.c_void_p(16), -1, 0, None) == qp.QP_ERR_INVALID_ARG   # 5 is not 2^a 3^b
    assert lib.qp_plan_destroy(None) == qp.QP_OK
