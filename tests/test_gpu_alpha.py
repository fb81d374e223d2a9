"""Spectrum estimate (rk_spectrum: Lanczos on A^T A) against the oracle's FP64 SVD, and
RKA with the optimal uniform weight of Eq. (best_alpha) against the oracle."""
import numpy as np
import pytest

import oracle
import rk_inputs

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
    err = np.linalg.norm(x.cpu().numpy() - x_o) / np.linalg.norm(x_o)
    assert err < 1e-4


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
    """Rows longer than the solve kernel holds (30000 columns) take the two residual
    passes for A^T A v; the top of the spectrum still converges."""
    s = rk_inputs.gaussian_system(800, 30000, seed=4)
    A = _dev(s.A)
    sp = rk.spectrum(A, k=40, seed=1)
    # A A^T (800 x 800) has the same nonzero eigenvalues as A^T A
    ev = np.linalg.eigvalsh(s.A.astype(np.float64) @ s.A.T.astype(np.float64))
    assert sp.lambda_max == pytest.approx(ev[-1], rel=2e-3)
    assert sp.lambda_max <= ev[-1] * (1 + 1e-9)   # a Ritz value, from below
    assert sp.fro2 == pytest.approx(float(np.sum(s.A.astype(np.float64) ** 2)), rel=1e-12)
