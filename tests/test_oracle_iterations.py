"""Pins of the oracle's RK / RKA / RKAB iterations against the geometry and
convergence theory the paper states (Section 2.1 Eq. (alg), Section 2.2,
Section 2.3.1 Eq. (rka_uni_weights), Section 3.4.1 RKAB), special cases that
reduce one method to another, and library least-squares solves."""
import numpy as np
import pytest

import oracle
import rk_inputs


@pytest.fixture(scope="module")
def small():
    s = rk_inputs.gaussian_system(200, 12, seed=4)
    b64 = s.A.astype(np.float64) @ s.x_star.astype(np.float64)   # exactly consistent in FP64
    return s, b64, oracle.table(s.A)


def test_projection_zeroes_row_residual(small):
    """omega = 1: x_{k+1} lies on the hyperplane H_i of the sampled row (Section 2.1)."""
    s, b64, tab = small
    rng = np.random.default_rng(0)
    x0 = rng.standard_normal(12)
    for t0 in range(10):
        i = int(oracle.sample_rows(tab, 77, 0, t0, 1)[0])
        x1 = oracle.rk(s.A, b64, x0, 1, 77, tab, t0=t0)
        a = s.A[i].astype(np.float64)
        res = b64[i] - a @ x1
        assert abs(res) <= 64 * np.finfo(float).eps * np.linalg.norm(a) * max(np.linalg.norm(x1), 1)


def test_pythagorean_identity(small):
    """Consistent system, omega = 1: ||x_{k+1}-x*||^2 = ||x_k-x*||^2 - ((b_i-<a_i,x_k>)/||a_i||)^2."""
    s, b64, tab = small
    xs = s.x_star.astype(np.float64)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(12)
    for t in range(50):
        i = int(oracle.sample_rows(tab, 5, 0, t, 1)[0])
        a = s.A[i].astype(np.float64)
        drop = ((b64[i] - a @ x) / np.linalg.norm(a)) ** 2
        xn = oracle.rk(s.A, b64, x, 1, 5, tab, t0=t)
        lhs = np.sum((xn - xs) ** 2)
        rhs = np.sum((x - xs) ** 2) - drop
        assert abs(lhs - rhs) <= 1e-10 * np.sum((x - xs) ** 2)
        x = xn


def test_relaxed_projection_moves_fraction_of_the_way(small):
    """omega in (0,2): the row residual becomes (1 - omega) times the old one."""
    s, b64, tab = small
    x0 = np.zeros(12)
    i = int(oracle.sample_rows(tab, 3, 0, 0, 1)[0])
    a = s.A[i].astype(np.float64)
    for om in (0.5, 1.5):
        x1 = oracle.rk(s.A, b64, x0, 1, 3, tab, omega=om)
        assert np.isclose(b64[i] - a @ x1, (1 - om) * (b64[i] - a @ x0), rtol=1e-12, atol=1e-12)


def test_rkab_q1_is_rk(small):
    """q = 1 RKAB is RK (Section 2.3.1: q = 1 recovers RK)."""
    s, b64, tab = small
    x0 = np.zeros(12)
    x_rk = oracle.rk(s.A, b64, x0, 60, 8, tab)
    x_ab = oracle.rkab(s.A, b64, x0, q=1, alpha=20, rounds=3, seed=8, tab=tab)
    assert np.array_equal(x_rk, x_ab)


def test_rkab_identical_streams_is_rk(small):
    """Workers given one stream average identical iterates (Section 3.3.1)."""
    s, b64, tab = small
    x0 = np.zeros(12)
    x_rk = oracle.rk(s.A, b64, x0, 40, 8, tab)
    x_ab = oracle.rkab(s.A, b64, x0, q=4, alpha=10, rounds=4, seed=8, tab=tab, same_stream=True)
    np.testing.assert_allclose(x_ab, x_rk, rtol=1e-13, atol=1e-13)


def test_rkab_alpha1_is_rka_formula(small):
    """alpha = 1 RKAB is the RKA update of Eq. (rka_uni_weights)."""
    s, b64, tab = small
    x0 = np.zeros(12)
    for om in (1.0, 1.7):
        x_f = oracle.rka_formula(s.A, b64, x0, q=5, iters=30, seed=2, tab=tab, omega=om)
        x_ab = oracle.rkab(s.A, b64, x0, q=5, alpha=1, rounds=30, seed=2, tab=tab, omega=om)
        np.testing.assert_allclose(x_ab, x_f, rtol=1e-12, atol=1e-12)


def test_average_obeys_jensen(small):
    """||mean(v) - x*||^2 <= mean(||v - x*||^2) for the averaging step."""
    s, b64, tab = small
    xs = s.x_star.astype(np.float64)
    x = np.zeros(12)
    V = oracle.rkab_round_workers(s.A, b64, x, q=6, alpha=7, rnd=0, seed=1, tab=tab)
    xbar = oracle.rkab(s.A, b64, x, q=6, alpha=7, rounds=1, seed=1, tab=tab)
    np.testing.assert_allclose(xbar, V.mean(axis=0), rtol=1e-14, atol=1e-14)
    assert np.sum((xbar - xs) ** 2) <= np.mean(np.sum((V - xs) ** 2, axis=1)) + 1e-15


def test_resume_matches_uninterrupted(small):
    s, b64, tab = small
    x0 = np.zeros(12)
    full = oracle.rkab(s.A, b64, x0, q=3, alpha=5, rounds=9, seed=4, tab=tab)
    part = oracle.rkab(s.A, b64, x0, q=3, alpha=5, rounds=4, seed=4, tab=tab)
    rest = oracle.rkab(s.A, b64, part, q=3, alpha=5, rounds=5, seed=4, tab=tab, round0=4)
    assert np.array_equal(full, rest)


def test_thread_count_does_not_change_result(small):
    s, b64, tab = small
    x0 = np.zeros(12)
    a = oracle.rkab(s.A, b64, x0, q=7, alpha=11, rounds=5, seed=6, tab=tab, threads=1)
    b = oracle.rkab(s.A, b64, x0, q=7, alpha=11, rounds=5, seed=6, tab=tab, threads=4)
    assert np.array_equal(a, b)


def test_converges_to_qr_solution_consistent():
    """Consistent full-rank system: RK and RKAB reach the unique x* (Section 2.2),
    which a library QR least-squares solve also returns."""
    s = rk_inputs.gaussian_system(50, 10, seed=9)
    b64 = s.A.astype(np.float64) @ s.x_star.astype(np.float64)
    tab = oracle.table(s.A)
    x_qr = oracle.lstsq_qr(s.A, b64)
    np.testing.assert_allclose(x_qr, s.x_star, rtol=1e-10, atol=1e-10)
    x_rk = oracle.rk(s.A, b64, np.zeros(10), 6000, 1, tab)
    np.testing.assert_allclose(x_rk, x_qr, rtol=1e-9, atol=1e-9)
    x_ab = oracle.rkab(s.A, b64, np.zeros(10), q=4, alpha=10, rounds=400, seed=1, tab=tab)
    np.testing.assert_allclose(x_ab, x_qr, rtol=1e-9, atol=1e-9)
    # tiny case 8 x 3
    s8 = rk_inputs.gaussian_system(8, 3, seed=10)
    b8 = s8.A.astype(np.float64) @ s8.x_star.astype(np.float64)
    x8 = oracle.rk(s8.A, b8, np.zeros(3), 3000, 2, oracle.table(s8.A))
    np.testing.assert_allclose(x8, oracle.lstsq_qr(s8.A, b8), rtol=1e-9, atol=1e-9)


def test_expected_error_bound():
    """E||x_k - x*||^2 <= (1 - sigma_min^2/||A||_F^2)^k ||x_0 - x*||^2 (Strohmer and
    Vershynin, as cited in Section 2.2), mean over 10 seeds, 2000 x 100 system."""
    s = rk_inputs.gaussian_system(2000, 100, seed=0)
    A64 = s.A.astype(np.float64)
    b64 = A64 @ s.x_star.astype(np.float64)
    xs = s.x_star.astype(np.float64)
    tab = oracle.table(s.A)
    sv = np.linalg.svd(A64, compute_uv=False)
    rate = 1.0 - sv[-1] ** 2 / np.sum(sv ** 2)
    e0 = np.sum(xs ** 2)
    for k in (100, 400, 1200):
        errs = [np.sum((oracle.rk(s.A, b64, np.zeros(100), k, seed, tab) - xs) ** 2)
                for seed in range(10)]
        assert np.mean(errs) <= rate ** k * e0, (k, np.mean(errs), rate ** k * e0)


def test_inconsistent_horizon_and_cgls():
    """Inconsistent system: CGLS and QR agree on x_LS; RK stalls at a horizon
    away from x_LS, and averaging over more workers shrinks it (Sections 2.2,
    2.3.1, 3.5)."""
    s = rk_inputs.gaussian_system(400, 20, seed=12, noise=0.5)
    b64 = s.b.astype(np.float64)
    x_qr = oracle.lstsq_qr(s.A, b64)
    x_cg = oracle.cgls(s.A, b64)
    np.testing.assert_allclose(x_cg, x_qr, rtol=1e-10, atol=1e-10)
    tab = oracle.table(s.A)
    errs = {}
    for q in (1, 16):
        e = []
        for seed in range(6):
            x = oracle.rkab(s.A, b64, np.zeros(20), q=q, alpha=1, rounds=3000, seed=seed, tab=tab)
            e.append(np.linalg.norm(x - x_qr))
        errs[q] = np.mean(e)
    assert errs[1] > 1e-3 * np.linalg.norm(x_qr)     # no convergence to x_LS
    assert errs[16] < 0.5 * errs[1]                  # horizon shrinks with q


def test_residual_matches_library_matvec():
    s = rk_inputs.gaussian_system(300, 17, seed=13, noise=0.1)
    x = np.random.default_rng(0).standard_normal(17)
    r, rn, an = oracle.residual(s.A, s.b, x)
    A64 = s.A.astype(np.float64)
    r_ref = s.b.astype(np.float64) - A64 @ x
    np.testing.assert_allclose(r, r_ref, rtol=1e-12, atol=1e-12)
    assert np.isclose(rn, np.linalg.norm(r_ref), rtol=1e-12)
    assert np.isclose(an, np.linalg.norm(A64.T @ r_ref), rtol=1e-12)


def test_stop_rule_and_trace():
    s = rk_inputs.gaussian_system(300, 10, seed=14)
    b64 = s.A.astype(np.float64) @ s.x_star.astype(np.float64)
    tab = oracle.table(s.A)
    xs = s.x_star.astype(np.float64)
    x, done, trace = oracle.rkab(s.A, b64, np.zeros(10), q=4, alpha=10, rounds=500, seed=0,
                                 tab=tab, x_ref=xs, tol=1e-6, want_trace=True)
    assert 0 < done < 500
    assert trace[-1] < 1e-6 and (done == 1 or trace[-2] >= 1e-6)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-6
