"""Pins of the oracle's per-worker weights and Partial Matrix alpha (Section 3.3.1,
Table 1) against facts that hold independently of the oracle's code: a constant
per-worker weight is the uniform relaxation, per-worker weights under the
Distributed Approach are per-row weights of the workers' blocks, a matrix of q
identical blocks has the full matrix's normalised spectrum in every block, and the
paper's finding that the per-thread alpha needs about as many iterations as the
full-matrix alpha."""
import numpy as np
import pytest

import oracle
import rk_inputs


@pytest.fixture(scope="module")
def small():
    s = rk_inputs.gaussian_system(1200, 40, seed=31)
    return s, oracle.table(s.A)


def test_constant_worker_weight_is_the_uniform_relaxation(small):
    s, tab = small
    q = 6
    b = s.b.astype(np.float64)
    x_u = oracle.rkab(s.A, b, np.zeros(40), q=q, alpha=3, rounds=25, seed=4, tab=tab,
                      worker_weight=np.full(q, 1.7))
    x_o = oracle.rkab(s.A, b, np.zeros(40), q=q, alpha=3, rounds=25, seed=4, tab=tab, omega=1.7)
    np.testing.assert_allclose(x_u, x_o, rtol=1e-13, atol=1e-13)


def test_block_worker_weights_are_row_weights_of_the_blocks(small):
    """With the Distributed Approach worker g only draws rows of its block, so a weight
    per worker equals a weight per row constant on each block (bit for bit)."""
    s, tab = small
    m, q = 1200, 7
    u = np.linspace(0.5, 2.5, q)
    w = np.empty(m)
    for g in range(q):
        lo, hi = oracle.block_bounds(m, q, g)
        w[lo:hi] = u[g]
    b = s.b.astype(np.float64)
    x_u = oracle.rkab(s.A, b, np.zeros(40), q=q, alpha=4, rounds=15, seed=9, tab=tab,
                      sampling="blocks", worker_weight=u)
    x_w = oracle.rkab(s.A, b, np.zeros(40), q=q, alpha=4, rounds=15, seed=9, tab=tab,
                      sampling="blocks", row_weight=w)
    assert np.array_equal(x_u, x_w)


def test_worker_weights_differ_per_worker(small):
    """Scaling one worker's weight changes the result (the weight reaches that worker)."""
    s, tab = small
    q = 4
    b = s.b.astype(np.float64)
    base = oracle.rkab(s.A, b, np.zeros(40), q=q, alpha=2, rounds=3, seed=2, tab=tab,
                       worker_weight=np.ones(q))
    for g in range(q):
        u = np.ones(q)
        u[g] = 1.5
        x = oracle.rkab(s.A, b, np.zeros(40), q=q, alpha=2, rounds=3, seed=2, tab=tab,
                        worker_weight=u)
        assert not np.allclose(x, base, rtol=1e-12, atol=0)


def test_stacked_identical_blocks_give_the_full_alpha():
    """A = [B; B; ...; B] (q copies): A^T A = q B^T B and ||A||_F^2 = q ||B||_F^2, so every
    block's s_min, s_max equal those of A and the per-worker alpha equals alpha*."""
    rng = np.random.default_rng(3)
    B = rng.standard_normal((150, 30)).astype(np.float32)
    for q in (2, 3, 5):
        A = np.vstack([B] * q)
        al, sp = oracle.partial_alpha_star(A, q)
        smin, smax, fro = oracle.spectrum(A)
        full = oracle.alpha_star(q, smin / fro, smax / fro)
        np.testing.assert_allclose(al, full, rtol=1e-10)
        np.testing.assert_allclose(sp[:, 2] * q, fro, rtol=1e-12)


def test_wide_blocks_use_their_nonzero_singular_values():
    """A block with fewer rows than columns has min(m_g, n) = m_g singular values; its
    s_min is the smallest of them (not the zero eigenvalues of A_g^T A_g)."""
    rng = np.random.default_rng(8)
    A = rng.standard_normal((90, 40)).astype(np.float32)
    al, sp = oracle.partial_alpha_star(A, 3)            # blocks of 30 x 40
    for g in range(3):
        lo, hi = oracle.block_bounds(90, 3, g)
        sv = np.linalg.svd(A[lo:hi].astype(np.float64), compute_uv=False)
        assert sv.shape == (30,)
        np.testing.assert_allclose(sp[g, 0], sv[-1] ** 2, rtol=1e-12)
        assert sp[g, 0] > 1e-3 * sp[g, 1]


def test_partial_alpha_needs_about_the_full_alpha_iterations():
    """Table 1: the per-thread alpha from the thread's own rows needs about as many
    iterations as alpha* of the whole matrix (differences of a fraction of a percent at
    2 .. 16 threads).  Here: rounds of RKA to 1e-6 within 10% of each other, under both
    row selections."""
    s = rk_inputs.gaussian_system(3000, 60, seed=12)
    tab = oracle.table(s.A)
    xs = s.x_star.astype(np.float64)
    b = s.b.astype(np.float64)
    smin, smax, fro = oracle.spectrum(s.A)
    for q in (2, 4):
        full = oracle.alpha_star(q, smin / fro, smax / fro)
        part, _ = oracle.partial_alpha_star(s.A, q)
        for mode in ("full", "blocks"):
            _, r_full = oracle.rkab(s.A, b, np.zeros(60), q=q, alpha=1, rounds=200000, seed=1,
                                    tab=tab, omega=full, x_ref=xs, tol=1e-6, sampling=mode)
            _, r_part = oracle.rkab(s.A, b, np.zeros(60), q=q, alpha=1, rounds=200000, seed=1,
                                    tab=tab, worker_weight=part, x_ref=xs, tol=1e-6,
                                    sampling=mode)
            assert r_full < 200000 and r_part < 200000
            assert abs(r_part - r_full) <= 0.1 * r_full, (q, mode, r_full, r_part)
