"""Pins of the oracle's optimal RKA weight (Eq. (best_alpha), Section 2.3.1) and of
the spectrum it is computed from.  CPU only."""
import os

import numpy as np
import pytest

import oracle
import rk_inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "alpha_star_paper.txt")


def test_single_chain_weight_is_one():
    """q = 1 is RK, whose best uniform relaxation in expectation is 1 for any spectrum."""
    for s_min, s_max in [(0.0, 1.0), (1e-5, 2e-4), (0.3, 0.3)]:
        assert oracle.alpha_star(1, s_min, s_max) == 1.0


def test_branches_meet_at_the_switch():
    """Both branches of Eq. (best_alpha) give q / (1 + (q-1) s_min) where
    s_max - s_min = 1 / (q - 1): the weight is continuous in the spectrum."""
    for q in (2, 3, 8, 132):
        s_min = 1e-3
        s_max = s_min + 1.0 / (q - 1)
        a1 = q / (1.0 + (q - 1) * s_min)
        eps = 1e-12
        lo = oracle.alpha_star(q, s_min, s_max - eps)
        hi = oracle.alpha_star(q, s_min, s_max + eps)
        assert lo == pytest.approx(a1, rel=1e-9)
        assert hi == pytest.approx(a1, rel=1e-9)


def test_paper_values_share_one_spectrum():
    """The paper prints alpha* = 1.999 (q = 2) and 3.992 (q = 4) for one matrix.  The
    interval of s_min that rounds to the q = 2 value must map, through the formula's q
    dependence, to an interval containing the q = 4 value (a wrong q-dependence, e.g.
    q / (1 + q s_min), fails)."""
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    (q1, v1, d1), (q2, v2, d2) = [(int(a), float(b), int(c)) for a, b, c in rows]
    half1 = 0.5 * 10.0 ** (-d1)
    # first branch (the spread of a tall matrix is far below 1 / (q - 1) for q <= 4):
    # alpha = q / (1 + (q - 1) s)  <=>  s = (q / alpha - 1) / (q - 1)
    s_hi = (q1 / (v1 - half1) - 1.0) / (q1 - 1)
    s_lo = (q1 / (v1 + half1) - 1.0) / (q1 - 1)
    a_hi = oracle.alpha_star(q2, s_lo, s_lo)
    a_lo = oracle.alpha_star(q2, s_hi, s_hi)
    half2 = 0.5 * 10.0 ** (-d2)
    assert a_lo - half2 <= v2 <= a_hi + half2


def test_spectrum_against_gaussian_edges():
    """For a tall iid N(0,1) matrix the squared singular values sit near the
    Marchenko-Pastur edges (sqrt(m) -/+ sqrt(n))^2 and ||A||_F^2 near m n."""
    m, n = 4000, 100
    s = rk_inputs.gaussian_system(m, n, seed=3)
    lmin, lmax, fro2 = oracle.spectrum(s.A)
    assert lmin == pytest.approx((np.sqrt(m) - np.sqrt(n)) ** 2, rel=0.06)
    assert lmax == pytest.approx((np.sqrt(m) + np.sqrt(n)) ** 2, rel=0.06)
    assert fro2 == pytest.approx(m * n, rel=0.01)
    # the extreme eigenvalues of A^T A bound every Rayleigh quotient
    rng = np.random.default_rng(0)
    A64 = s.A.astype(np.float64)
    for _ in range(20):
        v = rng.standard_normal(n)
        rq = float(np.sum((A64 @ v) ** 2) / (v @ v))
        assert lmin * (1 - 1e-12) <= rq <= lmax * (1 + 1e-12)


def test_optimal_weight_speeds_up_rka():
    """Section 3.3.1 / Table 1: with alpha* the rounds of RKA to a fixed error fall
    roughly as 1/q; with alpha = 1 they stay near those of RK."""
    m, n, q = 2000, 50, 8
    s = rk_inputs.gaussian_system(m, n, seed=5)
    tab = oracle.table(s.A)
    lmin, lmax, fro2 = oracle.spectrum(s.A)
    a = oracle.alpha_star(q, lmin / fro2, lmax / fro2)
    assert 1.0 < a < q
    b64 = s.b.astype(np.float64)
    xs = s.x_star.astype(np.float64)

    def rounds_to(omega, tol=1e-6, cap=20000):
        x = np.zeros(n)
        for k in range(1, cap + 1):
            x = oracle.rkab(s.A, b64, x, q=q, alpha=1, rounds=1, seed=11, tab=tab,
                            round0=k - 1, omega=omega)
            if np.linalg.norm(x - xs) / np.linalg.norm(xs) < tol:
                return k
        return cap

    r1 = rounds_to(1.0)
    ra = rounds_to(a)
    assert ra < r1 / (0.5 * q)
