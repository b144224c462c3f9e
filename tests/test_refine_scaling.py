"""The property the refinement's power-of-two scale rests on: a preconditioned CG with FP32 vectors and FP64 inner
products (the inner solve's arithmetic: vectors, operator and diagonal in FP32, (r, M r) and (h, Q h) and the
alpha / beta scalars in FP64) gives, for the right-hand side 2^k b, exactly 2^k times the iterates it gives for b.
Every rounding commutes with a power-of-two scaling inside the normal range, the inner products scale by 2^(2k) and
their quotients not at all, so the inner solve is the same whichever power of two scales its right-hand side, while
the conversions into and out of it stay exact exponent shifts."""
import numpy as np
import pytest


def _pcg_fp32(A32, M32, b32, iters):
    x = np.zeros_like(b32)
    r = b32.copy()
    z = M32 * r
    h = z.copy()
    rz = float(np.dot(r.astype(np.float64), z.astype(np.float64)))
    out = []
    for _ in range(iters):
        w = A32 @ h
        alpha = rz / float(np.dot(h.astype(np.float64), w.astype(np.float64)))
        x = x + np.float32(alpha) * h
        r = r - np.float32(alpha) * w
        z = M32 * r
        rz_new = float(np.dot(r.astype(np.float64), z.astype(np.float64)))
        h = z + np.float32(rz_new / rz) * h
        rz = rz_new
        out.append((x.copy(), r.copy(), alpha))
    return out


@pytest.mark.parametrize("k", [-40, -7, 1, 5, 30])
def test_fp32_pcg_iterates_scale_exactly_with_the_right_hand_side(k):
    rng = np.random.default_rng(11)
    n = 96
    G = rng.standard_normal((n, n))
    A = G @ G.T + n * np.eye(n)                      # SPD, moderately conditioned
    A32 = A.astype(np.float32)
    M32 = (1.0 / np.diag(A)).astype(np.float32)      # Jacobi
    b = rng.standard_normal(n).astype(np.float32)
    base = _pcg_fp32(A32, M32, b, 25)
    s = np.float32(2.0 ** k)
    scaled = _pcg_fp32(A32, M32, b * s, 25)
    for (x0, r0, a0), (x1, r1, a1) in zip(base, scaled):
        assert a0 == a1
        assert np.array_equal(x0 * s, x1)
        assert np.array_equal(r0 * s, r1)


def test_a_non_power_of_two_scale_changes_the_iterates():
    """Control: scaling by 1 / ||b|| (not a power of two) does not commute with the FP32 roundings."""
    rng = np.random.default_rng(12)
    n = 96
    G = rng.standard_normal((n, n))
    A32 = (G @ G.T + n * np.eye(n)).astype(np.float32)
    M32 = (1.0 / np.diag(A32.astype(np.float64))).astype(np.float32)
    b = rng.standard_normal(n).astype(np.float32)
    sc = np.float32(1.0 / np.linalg.norm(b.astype(np.float64)))
    base = _pcg_fp32(A32, M32, b, 25)
    scaled = _pcg_fp32(A32, M32, b * sc, 25)
    assert any(not np.array_equal((x0 * sc).astype(np.float32), x1) for (x0, _, _), (x1, _, _) in zip(base, scaled))
