"""Spectrum estimate (rk_spectrum: Lanczos on A^T A) against the oracle's FP64 SVD, RKA
with the optimal uniform weight of Eq. (best_alpha), and the Partial Matrix alpha of
Section 3.3.1 (per-worker weights from each worker's row block) against the oracle."""
import numpy as np
import pytest

import oracle
import rk_inputs
from _parity import assert_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rk():
    import paper_2401_17474_gb300 as rk_
    from paper_2401_17474_gb300 import build
    build.build()
    return rk_


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_spectrum_spanning_space(rk):
    """k = n steps span R^n: the Ritz values at the ends are the extreme eigenvalues of
    A^T A, up to the float32 application of A^T A (one pass of the solve kernel: dots and
    sums in float32, about 1e-6 relative)."""
    s = rk_inputs.gaussian_system(2000, 100, seed=1)
    lmin, lmax, fro2 = oracle.spectrum(s.A)
    sp = rk.spectrum(_dev(s.A), k=100, seed=3)
    assert sp.steps == 100
    assert sp.lambda_min == pytest.approx(lmin, rel=1e-5)
    assert sp.lambda_max == pytest.approx(lmax, rel=1e-5)
    assert sp.fro2 == pytest.approx(fro2, rel=1e-12)


def test_spectrum_partial_inside_and_close(rk):
    """k < n: Ritz values lie inside [lambda_min, lambda_max]; the top converges first."""
    s = rk_inputs.gaussian_system(20000, 500, seed=1)
    lmin, lmax, fro2 = oracle.spectrum(s.A)
    sp = rk.spectrum(_dev(s.A), k=32, seed=0)
    assert sp.steps == 32
    assert lmin * (1 - 1e-5) <= sp.lambda_min <= lmin * (1 + 5e-3)
    assert lmax * (1 - 1e-4) <= sp.lambda_max <= lmax * (1 + 1e-5)
    # the weight of Eq. (best_alpha) from the estimate is within 1e-4 of the exact one
    for q in (8, 132):
        a_est = rk.alpha_star(q, sp.s_min, sp.s_max)
        a_ref = oracle.alpha_star(q, lmin / fro2, lmax / fro2)
        assert a_est == pytest.approx(a_ref, rel=1e-4)
        assert a_est <= a_ref * (1 + 1e-5)   # s_min from above: the weight errs small


def test_spectrum_is_reproducible(rk):
    s = rk_inputs.gaussian_system(3000, 200, seed=2)
    A = _dev(s.A)
    a = rk.spectrum(A, k=20, seed=9)
    b = rk.spectrum(A, k=20, seed=9)
    assert (a.lambda_min, a.lambda_max, a.fro2) == (b.lambda_min, b.lambda_max, b.fro2)


@pytest.mark.parametrize("q,rounds", [(8, 1), (8, 10), (8, 100), (32, 40)])
def test_rka_optimal_weight_matches_oracle(rk, q, rounds):
    """RKA (alpha = 1) with omega = alpha* of Eq. (best_alpha): x within 1e-4 of the
    oracle on the same index stream."""
    s = rk_inputs.gaussian_system(2000, 100, seed=0)
    tab = oracle.table(s.A)
    lmin, lmax, fro2 = oracle.spectrum(s.A)
    a = oracle.alpha_star(q, lmin / fro2, lmax / fro2)
    A = rk.aligned_rows(_dev(s.A))
    plan = rk.rk_setup(A)
    x, info = rk.rka_solve(plan, _dev(s.b), q=q, rounds=rounds, seed=5, omega=a, check_every=0)
    assert info.status == 0
    x_o = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(100), q=q, alpha=1, rounds=rounds,
                      seed=5, tab=tab, omega=float(np.float32(a)))
    assert_close(x.cpu().numpy(), x_o, 1e-4)


def test_rka_optimal_weight_reaches_tolerance_faster(rk):
    """Rounds to 1e-6 with alpha* fall by about the worker count against alpha = 1."""
    s = rk_inputs.gaussian_system(2000, 100, seed=0)
    lmin, lmax, fro2 = oracle.spectrum(s.A)
    q = 16
    a = oracle.alpha_star(q, lmin / fro2, lmax / fro2)
    A = rk.aligned_rows(_dev(s.A))
    plan = rk.rk_setup(A)
    xs = _dev(s.x_star)
    _, i1 = rk.rka_solve(plan, _dev(s.b), q=q, rounds=20000, seed=1, omega=1.0, tol=1e-6, x_ref=xs)
    _, ia = rk.rka_solve(plan, _dev(s.b), q=q, rounds=20000, seed=1, omega=a, tol=1e-6, x_ref=xs)
    assert i1.status == 0 and ia.status == 0
    assert ia.last_metric < 1e-6
    assert ia.rounds_done < i1.rounds_done / (0.4 * q)


def test_spectrum_long_rows_two_pass(rk):
    """A wide matrix with rows longer than the solve kernel holds (30000 columns): the
    process runs on A A^T (two passes a step); the top of the spectrum converges."""
    s = rk_inputs.gaussian_system(800, 30000, seed=4)
    A = _dev(s.A)
    sp = rk.spectrum(A, k=40, seed=1)
    # A A^T (800 x 800) has the same nonzero eigenvalues as A^T A
    ev = np.linalg.eigvalsh(s.A.astype(np.float64) @ s.A.T.astype(np.float64))
    assert sp.lambda_max == pytest.approx(ev[-1], rel=2e-3)
    assert sp.lambda_max <= ev[-1] * (1 + 1e-9)   # a Ritz value, from below
    # the process runs on A A^T: the smallest Ritz value bounds the smallest nonzero
    # eigenvalue from above, far from the 29200 zero eigenvalues of A^T A
    assert sp.lambda_min >= ev[0] * (1 - 1e-6)
    assert sp.fro2 == pytest.approx(float(np.sum(s.A.astype(np.float64) ** 2)), rel=1e-12)


def test_spectrum_wide_spanning_row_space(rk):
    """m < n with k = m steps (Lanczos on A A^T spans R^m): the end Ritz values are the
    extreme squared singular values (the oracle's SVD of a 60 x 400 A)."""
    rng = np.random.default_rng(6)
    A_np = rng.standard_normal((60, 400)).astype(np.float32)
    lmin, lmax, fro2 = oracle.spectrum(A_np)
    sp = rk.spectrum(_dev(A_np), k=200, seed=2)
    assert sp.steps == 60
    assert sp.lambda_min == pytest.approx(lmin, rel=1e-5)
    assert sp.lambda_max == pytest.approx(lmax, rel=1e-5)


@pytest.mark.parametrize("m,n,q", [(1200, 40, 4), (1200, 40, 40), (999, 64, 7)])
def test_partial_alpha_matches_oracle(rk, m, n, q):
    """Per-worker alpha of Section 3.3.1 from each block (tall blocks, wide blocks of 30 x
    40, ragged blocks of 142 or 143 rows) with enough Lanczos steps to span each block's
    row space, against the oracle's (LAPACK SVD of every block).  The float32 application
    of A^T A errs by about 1e-7 lambda_max, so lambda_min of an ill-conditioned block is
    held to 1e-3 and the weights (which depend on it through (q - 1) s_min) to 1e-4."""
    s = rk_inputs.gaussian_system(m, n, seed=m + q)
    w, sps = rk.partial_alpha_star(rk.aligned_rows(_dev(s.A)), q, k=min(n, 512))
    w_o, sp_o = oracle.partial_alpha_star(s.A, q)
    np.testing.assert_allclose(w.cpu().numpy(), w_o, rtol=1e-4)
    for g in range(q):
        assert sps[g].lambda_min == pytest.approx(sp_o[g, 0], rel=1e-3)
        assert sps[g].lambda_max == pytest.approx(sp_o[g, 1], rel=1e-5)
        assert sps[g].fro2 == pytest.approx(sp_o[g, 2], rel=1e-12)


def test_partial_alpha_refuses_empty_blocks(rk):
    A = torch.randn((10, 8), device="cuda")
    with pytest.raises(rk.RkError):
        rk.partial_alpha_star(A, 11)


@pytest.mark.parametrize("q,alpha,rounds,sampling,cluster", [
    (8, 20, 6, "full", 0),        # one CTA a worker
    (8, 20, 6, "blocks", 0),      # the Distributed Approach
    (456, 1, 12, "full", 0),      # RKA with more workers than SMs (workers spread over CTAs)
    (456, 1, 12, "blocks", 0),
    (4, 20, 5, "full", 4),        # 4-CTA cluster workers
])
def test_worker_weights_match_oracle(rk, q, alpha, rounds, sampling, cluster):
    """Per-worker weights (here the Partial Matrix alpha, scaled into (0.5, 1.5) of a
    uniform relaxation so that every worker's weight differs): x within 1e-4 of the oracle
    given the same weights."""
    s = rk_inputs.gaussian_system(2000, 100, seed=0)
    tab = oracle.table(s.A)
    u = np.float32(0.5) + np.random.default_rng(q).random(q).astype(np.float32)
    plan = rk.rk_setup(rk.aligned_rows(_dev(s.A)))
    x, info = rk.rkab_solve(plan, _dev(s.b), q=q, alpha=alpha, rounds=rounds, seed=3,
                            check_every=0, sampling=sampling, cluster_size=cluster,
                            worker_weight=_dev(u))
    assert info.status == 0
    x_o = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(100), q=q, alpha=alpha,
                      rounds=rounds, seed=3, tab=tab, sampling=sampling,
                      worker_weight=u.astype(np.float64))
    assert_close(x.cpu().numpy(), x_o, 1e-4)


@pytest.mark.parametrize("q,sampling", [(4, "full"), (16, "blocks")])
def test_partial_alpha_rka_matches_oracle(rk, q, sampling):
    """RKA with the Partial Matrix alpha end to end: the GPU's weights (rk_partial_alpha_star,
    k spanning each block) and the oracle's own weights (SVD) drive the two solves; x
    within 1e-4, and the run reaches 1e-6 in about the rounds of the full-matrix alpha*
    (Table 1)."""
    s = rk_inputs.gaussian_system(4000, 60, seed=21)
    tab = oracle.table(s.A)
    A = rk.aligned_rows(_dev(s.A))
    w, _ = rk.partial_alpha_star(A, q, k=60)
    w_o, _ = oracle.partial_alpha_star(s.A, q)
    plan = rk.rk_setup(A)
    x, info = rk.rka_solve(plan, _dev(s.b), q=q, rounds=50, seed=7, check_every=0,
                           sampling=sampling, worker_weight=w)
    assert info.status == 0
    x_o = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(60), q=q, alpha=1, rounds=50,
                      seed=7, tab=tab, sampling=sampling, worker_weight=w_o)
    assert_close(x.cpu().numpy(), x_o, 1e-4)
    xs = _dev(s.x_star)
    lmin, lmax, fro2 = oracle.spectrum(s.A)
    a = oracle.alpha_star(q, lmin / fro2, lmax / fro2)
    _, i_full = rk.rka_solve(plan, _dev(s.b), q=q, rounds=100000, seed=1, omega=a, tol=1e-6,
                             x_ref=xs, sampling=sampling)
    _, i_part = rk.rka_solve(plan, _dev(s.b), q=q, rounds=100000, seed=1, tol=1e-6, x_ref=xs,
                             sampling=sampling, worker_weight=w)
    assert i_full.last_metric < 1e-6 and i_part.last_metric < 1e-6
    assert abs(i_part.rounds_done - i_full.rounds_done) <= 0.1 * i_full.rounds_done


def test_spectrum_with_known_frobenius_norm(rk):
    """rk_spectrum_ex skips the Frobenius pass: the same Lanczos extremes as rk_spectrum,
    ||A||_F^2 as given; the plan's law gives ||A||_F^2 = T 2^L within 1e-7 of the oracle's."""
    s = rk_inputs.gaussian_system(3000, 200, seed=2)
    A = _dev(s.A)
    plan = rk.rk_setup(A)
    fro2_o = oracle.spectrum(s.A)[2]
    assert plan.frobenius2() == pytest.approx(fro2_o, rel=1e-7)
    a = rk.spectrum(A, k=12, seed=5)
    b = rk.spectrum(A, k=12, seed=5, fro2=plan.frobenius2())
    assert (b.lambda_min, b.lambda_max) == (a.lambda_min, a.lambda_max)
    assert b.fro2 == plan.frobenius2()
    w_plan, _ = rk.optimal_weight(A, 64, k=12, seed=5, plan=plan)
    w_pass, _ = rk.optimal_weight(A, 64, k=12, seed=5)
    assert w_plan == pytest.approx(w_pass, rel=1e-6)


def test_new_entry_points_refuse_bad_arguments(rk):
    """A non-finite ||A||_F^2 is refused by rk_spectrum_ex; per-worker weights must hold
    exactly q floats."""
    s = rk_inputs.gaussian_system(500, 40, seed=2)
    A = _dev(s.A)
    with pytest.raises(rk.RkError):
        rk.spectrum(A, k=4, fro2=float("nan"))
    plan = rk.rk_setup(A)
    with pytest.raises(ValueError):
        rk.rkab_solve(plan, _dev(s.b), q=4, alpha=2, rounds=1, worker_weight=_dev(np.ones(3, np.float32)))
