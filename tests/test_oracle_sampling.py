"""Pins of the oracle's sampler against facts fixed outside the oracle:
published Philox known answers, exact rational row norms, the alias-table
mass identity, and the law of Eq. (prob_line) itself (P{i=l} = ||A_l||^2 /
||A||_F^2, Section 2.2)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import rk_inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,want", _kat())
def test_philox_known_answers(ctr, key, want):
    assert list(oracle.philox4x32_10(ctr, key)) == want


def _exact_norms(A):
    return [math.fsum(float(v) * float(v) for v in row) for row in A.astype(np.float64)]


def test_row_weights_follow_exact_norms():
    """K_i / T matches ||A_i||^2 / ||A||_F^2 (exact sums) to ~2^-40 of the top row."""
    rng = np.random.default_rng(11)
    A = rng.standard_normal((300, 37)).astype(np.float32)
    A[5] *= 1e-3
    A[7] *= 1e3
    A[9] = 0.0
    K, T, L = oracle.row_weights(A)
    assert T == int(K.astype(object).sum()) and T < 2**62
    assert K[9] == 0
    # the top row keeps the precision the 2^62 budget allows: 2^(60-c) <= K_max < 2^(62-c)
    c = int(np.ceil(np.log2(A.shape[0])))
    assert 2 ** (60 - c) <= int(K.max()) < 2 ** (62 - c)
    w = [Fraction(x) for x in _exact_norms(A)]
    W = sum(w)
    wmax = max(w)
    for i in range(A.shape[0]):
        p_exact = w[i] / W
        p_enc = Fraction(int(K[i]), T)
        assert abs(p_enc - p_exact) <= Fraction(1, 2**38) * (wmax / W) + Fraction(1, T), i
    # the encoded weights are floors of w_i / 2^L up to the per-row truncation
    for i in range(A.shape[0]):
        lo = w[i] / Fraction(2) ** L - A.shape[1]   # each term loses < 1 unit before the shift
        assert Fraction(int(K[i])) <= w[i] / Fraction(2) ** L
        assert Fraction(int(K[i])) >= lo - 1


def test_row_weights_invariances():
    """Power-of-two scaling of A changes nothing; permuting rows permutes K."""
    rng = np.random.default_rng(3)
    A = (rng.standard_normal((64, 19)) * rng.uniform(0.01, 100, (64, 1))).astype(np.float32)
    K, T, _ = oracle.row_weights(A)
    for s in (2.0 ** -30, 0.5, 8.0, 2.0 ** 40):
        K2, T2, _ = oracle.row_weights((A * np.float32(s)).astype(np.float32))
        assert T2 == T and np.array_equal(K2, K)
    perm = rng.permutation(64)
    K3, T3, _ = oracle.row_weights(np.ascontiguousarray(A[perm]))
    assert T3 == T and np.array_equal(K3, K[perm])


def test_row_weights_rejects_bad_input():
    with pytest.raises(ValueError):
        oracle.row_weights(np.zeros((4, 3), np.float32))
    A = np.ones((4, 3), np.float32)
    A[2, 1] = np.inf
    with pytest.raises(ValueError):
        oracle.row_weights(A)


def _law_from_table(thr64, alias):
    """Exact probability of each row under the draw rule of the alias table."""
    m = len(thr64)
    p = [Fraction(0)] * m
    two64 = 2**64
    for c in range(m):
        keep = Fraction(int(thr64[c]), two64)
        p[c] += keep / m
        p[int(alias[c])] += (1 - keep) / m
    return p


@pytest.mark.parametrize("case", ["gauss", "skewed", "ties", "single", "zeros"])
def test_alias_table_reproduces_law(case):
    rng = np.random.default_rng(7)
    if case == "gauss":
        A = rng.standard_normal((97, 13)).astype(np.float32)
    elif case == "skewed":
        A = (rng.standard_normal((120, 9)) * 10.0 ** rng.uniform(-2, 2, (120, 1))).astype(np.float32)
    elif case == "ties":
        A = np.ones((64, 4), np.float32)
    elif case == "single":
        A = np.full((1, 5), 3.0, np.float32)
    else:
        A = rng.standard_normal((50, 6)).astype(np.float32)
        A[::3] = 0.0
    tab = oracle.table(A)
    m, T = tab.m, tab.T
    # integer thresholds: thr64 = floor(thr 2^64 / T) with T < 2^64 determines thr
    thr = [T if int(t) == 2**64 - 1 else -(-(int(t) * T) // 2**64) for t in tab.thr64]
    assert all(int(t) == (2**64 - 1 if h == T else (h << 64) // T) for t, h in zip(tab.thr64, thr))
    # mass identity: bucket c holds thr_c of c and T - thr_c of alias_c, exactly
    mass = [0] * m
    for c in range(m):
        mass[c] += thr[c]
        mass[int(tab.alias[c])] += T - thr[c]
    assert mass == [m * int(k) for k in tab.K]
    p = _law_from_table(tab.thr64, tab.alias)
    for i in range(m):
        want = Fraction(int(tab.K[i]), T)
        assert abs(p[i] - want) <= Fraction(2 * m, 2**64), (i, float(p[i]), float(want))
    assert all(int(tab.alias[i]) < m for i in range(m))
    # zero rows are never reachable
    for i in range(m):
        if tab.K[i] == 0:
            assert tab.thr64[i] == 0 and p[i] == 0


def test_sampler_frequencies_match_norms():
    """Chi-square of 400k draws against the law computed from exact norms."""
    scipy_stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(5)
    A = (rng.standard_normal((200, 8)) * 10.0 ** rng.uniform(-1, 1, (200, 1))).astype(np.float32)
    tab = oracle.table(A)
    draws = np.concatenate([oracle.sample_rows(tab, seed=123, worker=g, t0=0, count=100_000)
                            for g in range(4)])
    counts = np.bincount(draws, minlength=200)
    w = np.array(_exact_norms(A))
    expect = w / w.sum() * draws.size
    chi2, pval = scipy_stats.chisquare(counts, expect)
    assert pval > 1e-4, (chi2, pval)


def test_sampler_streams_are_distinct_and_reproducible():
    A = rk_inputs.gaussian_system(500, 20, seed=2).A
    tab = oracle.table(A)
    s0 = oracle.sample_rows(tab, 9, worker=0, t0=0, count=2000)
    s0b = oracle.sample_rows(tab, 9, worker=0, t0=0, count=2000)
    s1 = oracle.sample_rows(tab, 9, worker=1, t0=0, count=2000)
    s2 = oracle.sample_rows(tab, 9, worker=0, t0=0, count=2000, stream=1)
    s3 = oracle.sample_rows(tab, 10, worker=0, t0=0, count=2000)
    assert np.array_equal(s0, s0b)
    for other in (s1, s2, s3):
        assert np.mean(s0 == other) < 0.05
    # a window of the stream equals the same window drawn from its own start
    assert np.array_equal(oracle.sample_rows(tab, 9, 0, 700, 300), s0[700:1000])
    assert s0.min() >= 0 and s0.max() < 500


# --------------------------------------------------------------------------
# Row selections other than the whole law: the Distributed Approach's row blocks
# (Section 3.3.1) and the cyclic sweep (Section 2.1)
# --------------------------------------------------------------------------
def _blocks(m, q):
    return [((g * m) // q, ((g + 1) * m) // q) for g in range(q)]


def test_block_draws_follow_the_block_law():
    """Worker g of q draws only inside rows [g m/q, (g+1) m/q), with probability
    ||a_i||^2 / (block sum): chi-square of 2e5 draws against exact rational norms."""
    rng = np.random.default_rng(4)
    m, n, q = 37, 6, 4                         # blocks of unequal size
    A = (rng.standard_normal((m, n)) * rng.uniform(0.1, 3.0, size=(m, 1))).astype(np.float32)
    A[5] = 0.0                                  # a zero row is never drawn
    tab = oracle.table(A)
    w = np.array([float(sum(Fraction(float(v)) ** 2 for v in row)) for row in A])
    for g, (s0, s1) in enumerate(_blocks(m, q)):
        d = oracle.sample_rows(tab, 11, g, 0, 200_000, sampling="blocks", q=q)
        assert d.min() >= s0 and d.max() < s1
        assert 5 not in set(d.tolist())
        p = w[s0:s1] / w[s0:s1].sum()
        cnt = np.bincount(d - s0, minlength=s1 - s0)
        keep = p > 0
        chi2 = float((((cnt - 200_000 * p) ** 2)[keep] / (200_000 * p[keep])).sum())
        dof = int(keep.sum()) - 1
        assert chi2 < dof + 6 * np.sqrt(2 * dof), (g, chi2, dof)


def test_one_block_is_the_whole_law():
    """q = 1: the single block is the whole matrix, so the block draw follows Eq.
    (prob_line) (same law as the alias draw, from other arithmetic)."""
    s = rk_inputs.gaussian_system(50, 5, seed=8, row_scale_decades=1.0)
    tab = oracle.table(s.A)
    d = oracle.sample_rows(tab, 2, 0, 0, 300_000, sampling="blocks", q=1)
    e = oracle.sample_rows(tab, 2, 0, 300_000, 300_000)
    p = tab.K.astype(np.float64) / float(tab.T)
    for draws in (d, e):
        cnt = np.bincount(draws, minlength=50)
        chi2 = float(((cnt - 300_000 * p) ** 2 / (300_000 * p)).sum())
        assert chi2 < 49 + 6 * np.sqrt(98)


def test_cyclic_sweep_order():
    """Cyclic selection: worker g of q takes rows g m/q, g m/q + 1, ... modulo m."""
    s = rk_inputs.gaussian_system(23, 4, seed=1)
    tab = oracle.table(s.A)
    for g, q in ((0, 1), (1, 3), (2, 3)):
        start = (g * 23) // q
        got = oracle.sample_rows(tab, 0, g, 5, 40, sampling="cyclic", q=q)
        assert np.array_equal(got, (start + 5 + np.arange(40)) % 23)


def test_row_weights_equal_uniform_relaxation():
    """Eq. (rka_eq) with w_i = c for every row is the uniform relaxation c; w_i = 1 is
    the unweighted method (both bit for bit: the product omega w_i is exact)."""
    s = rk_inputs.gaussian_system(200, 10, seed=2)
    tab = oracle.table(s.A)
    b = s.b.astype(np.float64)
    x1 = oracle.rkab(s.A, b, np.zeros(10), q=3, alpha=20, rounds=5, seed=4, tab=tab,
                     row_weight=np.ones(200))
    x2 = oracle.rkab(s.A, b, np.zeros(10), q=3, alpha=20, rounds=5, seed=4, tab=tab)
    assert np.array_equal(x1, x2)
    x3 = oracle.rkab(s.A, b, np.zeros(10), q=3, alpha=20, rounds=5, seed=4, tab=tab,
                     row_weight=np.full(200, 0.5))
    x4 = oracle.rkab(s.A, b, np.zeros(10), q=3, alpha=20, rounds=5, seed=4, tab=tab, omega=0.5)
    assert np.array_equal(x3, x4)


@pytest.mark.parametrize("sampling", ["blocks", "cyclic"])
def test_other_selections_converge(sampling):
    """Consistent 400 x 20 system: RKAB with row blocks (each block of 100 rows keeps
    full column rank) and cyclic Kaczmarz (q = 1) converge to x*."""
    s = rk_inputs.gaussian_system(400, 20, seed=6)
    tab = oracle.table(s.A)
    q = 4 if sampling == "blocks" else 1
    x = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(20), q=q, alpha=100, rounds=60,
                    seed=1, tab=tab, sampling=sampling)
    assert np.linalg.norm(x - s.x_star) / np.linalg.norm(s.x_star) < 1e-5
