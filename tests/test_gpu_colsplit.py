"""RKA (alpha = 1) on rows too long for one CTA's shared memory: x split by columns over
the grid (every CTA streams its chunk of each sampled row, the partial dots are summed
across the grid in a fixed order).  Against the FP64 oracle on the same draws: x within
1e-4, every element; FP32, BF16 and FP8 rows; ragged widths; row and worker weights;
the Distributed Approach's row blocks; the stopping rule; resume; argument limits."""
import numpy as np
import pytest

import oracle
import rk_inputs
from _parity import assert_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def rk():
    import paper_2401_17474_gb300 as rk_
    from paper_2401_17474_gb300 import build
    build.build()
    return rk_


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def wide(rk):
    # 300 x 50000: rows of 200 KB, an underdetermined consistent system (the shape of A^T
    # in the adjoint of a 50000 x 300 least-squares problem)
    s = rk_inputs.gaussian_system(300, 50000, seed=41)
    A = _dev(s.A)
    return s, A, rk.rk_setup(A), oracle.table(s.A)


@pytest.mark.parametrize("q,rounds,omega", [(1, 40, 1.0), (8, 30, 1.0), (13, 20, 6.0), (64, 10, 40.0)])
def test_colsplit_matches_oracle(rk, wide, q, rounds, omega):
    s, A, plan, tab = wide
    x0 = np.random.default_rng(q).standard_normal(50000).astype(np.float32)
    x, info = rk.rka_solve(plan, _dev(s.b), _dev(x0), q=q, rounds=rounds, seed=7, omega=omega,
                           check_every=0)
    assert info.status == 0 and info.rounds_done == rounds
    xo = oracle.rkab(s.A, s.b.astype(np.float64), x0.astype(np.float64), q=q, alpha=1, rounds=rounds,
                     seed=7, tab=tab, omega=float(np.float32(omega)))
    assert_close(x.cpu().numpy(), xo, TOL, what=f"q={q}")


@pytest.mark.parametrize("m,n", [(200, 50003), (64, 120001), (120, 200000)])
def test_colsplit_ragged_and_long_rows(rk, m, n):
    """A ragged tail (n % 4 != 0, the last slice masked), an uneven last chunk, and
    rows of 800 KB (each CTA's chunk of 1316 columns)."""
    s = rk_inputs.gaussian_system(m, n, seed=n % 997)
    A = rk.aligned_rows(_dev(s.A))
    plan = rk.rk_setup(A)
    x, info = rk.rka_solve(plan, _dev(s.b), q=16, rounds=6, seed=3, omega=8.0, check_every=0)
    assert info.status == 0
    xo = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(n), q=16, alpha=1, rounds=6, seed=3,
                     tab=oracle.table(s.A), omega=8.0)
    assert_close(x.cpu().numpy(), xo, TOL, what=f"{m}x{n}")


def test_colsplit_very_long_rows(rk):
    """Rows of 700001 columns (2.8 MB): chunks of 1152 slices a CTA, wider than the update's
    rows-outer layout holds, so each thread sums its slices over all rows in turn."""
    s = rk_inputs.gaussian_system(16, 700001, seed=11)
    A = rk.aligned_rows(_dev(s.A))
    plan = rk.rk_setup(A)
    x, info = rk.rka_solve(plan, _dev(s.b), q=4, rounds=6, seed=5, omega=2.0, check_every=0)
    assert info.status == 0
    xo = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(700001), q=4, alpha=1, rounds=6, seed=5,
                     tab=oracle.table(s.A), omega=2.0)
    assert_close(x.cpu().numpy(), xo, TOL, what="700001 columns")


@pytest.mark.parametrize("kind", ["bf16", "fp8"])
def test_colsplit_stored_rows(rk, wide, kind):
    s, A, _, _ = wide
    Aq, sc = rk.quantize(A, kind)
    plan = rk.rk_setup(Aq, kind, sc)
    low = oracle.quantize_bf16(s.A)[1] if kind == "bf16" else oracle.quantize_fp8(s.A)[2]
    x, info = rk.rka_solve(plan, _dev(s.b), q=12, rounds=15, seed=9, omega=6.0, check_every=0)
    assert info.status == 0
    xo = oracle.rkab(low, s.b.astype(np.float64), np.zeros(50000), q=12, alpha=1, rounds=15, seed=9,
                     tab=oracle.table(low), omega=6.0)
    assert_close(x.cpu().numpy(), xo, TOL, what=kind)


def test_colsplit_weights_and_blocks(rk, wide):
    """Per-row weights w_i and per-worker weights (Eq. (rka_eq), the Partial Matrix alpha),
    and the Distributed Approach's row blocks."""
    s, A, plan, tab = wide
    rng = np.random.default_rng(5)
    w = rng.uniform(0.5, 1.5, 300).astype(np.float32)
    u = rng.uniform(0.5, 1.5, 10).astype(np.float32)
    x, info = rk.rka_solve(plan, _dev(s.b), q=10, rounds=12, seed=2, check_every=0, row_weight=_dev(w),
                           worker_weight=_dev(u))
    assert info.status == 0
    xo = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(50000), q=10, alpha=1, rounds=12, seed=2,
                     tab=tab, row_weight=w.astype(np.float64), worker_weight=u.astype(np.float64))
    assert_close(x.cpu().numpy(), xo, TOL, what="weights")
    x, info = rk.rka_solve(plan, _dev(s.b), q=6, rounds=12, seed=4, check_every=0, sampling="blocks")
    assert info.status == 0
    xo = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(50000), q=6, alpha=1, rounds=12, seed=4,
                     tab=tab, sampling="blocks")
    assert_close(x.cpu().numpy(), xo, TOL, what="blocks")


def test_colsplit_stop_rule_and_resume(rk, wide):
    """The criterion ||x - x*|| / ||x*|| checked every 5 rounds stops at the oracle's round
    (to within the check interval); a run resumed at round 7 equals the uninterrupted one
    bit for bit."""
    s, A, plan, tab = wide
    b = _dev(s.b)
    # the minimum-norm solution of the consistent underdetermined system, reached from 0
    x_mn = np.linalg.lstsq(s.A.astype(np.float64), s.b.astype(np.float64), rcond=None)[0]
    xr = _dev(x_mn.astype(np.float32))
    q = 32
    lmin, lmax, fro2 = oracle.spectrum(s.A)
    om = float(np.float32(oracle.alpha_star(q, lmin / fro2, lmax / fro2)))
    x, info = rk.rka_solve(plan, b, q=q, rounds=5000, seed=1, omega=om, x_ref=xr, tol=1e-5,
                           check_every=5)
    assert info.status == 0 and 0 <= info.last_metric < 1e-5 and info.rounds_done % 5 == 0
    _, done_o = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(50000), q=q, alpha=1, rounds=5000,
                            seed=1, tab=tab, omega=om, x_ref=x_mn, tol=1e-5)
    assert abs(info.rounds_done - done_o) <= 5, (info.rounds_done, done_o)
    full, _ = rk.rka_solve(plan, b, q=8, rounds=15, seed=3, check_every=0)
    part, _ = rk.rka_solve(plan, b, q=8, rounds=7, seed=3, check_every=0)
    rest, _ = rk.rka_solve(plan, b, part.clone(), q=8, rounds=8, seed=3, round0=7, check_every=0)
    assert torch.equal(full, rest)


def test_colsplit_limits(rk, wide):
    s, A, plan, tab = wide
    with pytest.raises(rk.RkError) as e:
        rk.rka_solve(plan, _dev(s.b), q=65, rounds=1)   # more than 64 workers a round
    assert e.value.code == -1
    with pytest.raises(rk.RkError):
        rk.rkab_solve(plan, _dev(s.b), q=4, alpha=3, rounds=1)   # RKAB on rows this long: clusters only


def test_colsplit_wait_limit_ends_the_solve_with_a_status(rk, wide):
    """The column-split kernel's device waits are bounded too: with a 1 us limit the first
    wait for a row (a cold copy takes longer) runs out, every CTA winds down (the other CTAs
    leave the grid barrier on the status word, the producers stop at what was consumed and
    drain their copies) and the solve reports RK_ETIMEOUT; the same plan solves normally
    afterwards."""
    s, A, plan, tab = wide
    x, info = rk.rka_solve(plan, _dev(s.b), q=16, rounds=5, seed=1, check_every=0, timeout_s=1e-6,
                           raise_on_error=False)
    torch.cuda.synchronize()
    assert info.status == -4, info   # RK_ETIMEOUT
    x, info = rk.rka_solve(plan, _dev(s.b), q=16, rounds=5, seed=1, check_every=0)
    assert info.status == 0
    assert torch.isfinite(x).all()
