"""Pins of the oracle's adjoint of the least-squares map against central finite
differences of the FP64 map, the normal-equation invariants, and Kaczmarz's
minimum-norm limit on an underdetermined system (Section 2.1) against a
library minimum-norm solve."""
import numpy as np
import pytest

import oracle
import rk_inputs


@pytest.fixture(scope="module")
def small():
    s = rk_inputs.gaussian_system(60, 8, seed=81, noise=0.3)
    xt = rk_inputs.target_vector(8, seed=81).astype(np.float64)
    return s.A.astype(np.float64), s.b.astype(np.float64), xt


def test_adjoint_matches_central_differences(small):
    A, b, xt = small
    x = oracle.lstsq_qr(A, b)
    gA, gb, _ = oracle.lstsq_adjoint(A, b, x, xt)
    rng = np.random.default_rng(0)
    h = 1e-6
    for _ in range(32):
        dA = rng.standard_normal(A.shape)
        db = rng.standard_normal(b.shape)
        fd = (oracle.lstsq_loss(A + h * dA, b + h * db, xt)
              - oracle.lstsq_loss(A - h * dA, b - h * db, xt)) / (2 * h)
        an = np.sum(gA * dA) + np.sum(gb * db)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1.0), (fd, an)


def test_adjoint_invariants(small):
    """At x_LS (A^T r = 0): A^T grad_b = x - x_t and A^T grad_A = -(x - x_t) x^T."""
    A, b, xt = small
    x = oracle.lstsq_qr(A, b)
    gA, gb, _ = oracle.lstsq_adjoint(A, b, x, xt)
    np.testing.assert_allclose(A.T @ gb, x - xt, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(A.T @ gA, -np.outer(x - xt, x), rtol=1e-9, atol=1e-9)


def test_kaczmarz_on_transpose_reaches_min_norm_solution(small):
    A, b, xt = small
    x = oracle.lstsq_qr(A, b)
    gx = x - xt
    At = np.ascontiguousarray(A.T).astype(np.float32)
    tab = oracle.table(At)
    y = oracle.rkab(At, gx, np.zeros(60), q=4, alpha=8, rounds=3000, seed=2, tab=tab, stream=1)
    A32 = At.T.astype(np.float64)                      # the float32 values of A
    y_min, *_ = np.linalg.lstsq(A32.T, gx, rcond=None)  # library minimum-norm solution
    np.testing.assert_allclose(y, y_min, rtol=1e-9, atol=1e-9)
    # and it is A g with g = (A^T A)^{-1} gx
    _, y_ref, _ = oracle.lstsq_adjoint(A32, b, x, xt)
    np.testing.assert_allclose(y, y_ref, rtol=1e-8, atol=1e-8)
