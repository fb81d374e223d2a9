"""Cluster workers (one worker = a thread-block cluster splitting the row's
columns, rows resolved in look-ahead groups through DSMEM) against the FP64
oracle: the same draws, x within 1e-4 relative."""
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


def _rel(xg, xo):
    return np.linalg.norm(np.asarray(xg, np.float64) - xo) / np.linalg.norm(xo)


@pytest.mark.parametrize("C,lookahead", [(2, 4), (4, 6), (8, 4), (8, 6), (16, 6)])
@pytest.mark.parametrize("m,n,q,alpha,rounds", [(3000, 1000, 3, 37, 4), (5000, 4003, 2, 50, 3),
                                                (6000, 10000, 4, 23, 2)])
def test_cluster_workers_match_oracle(rk, C, lookahead, m, n, q, alpha, rounds):
    chunk = -(-(-(-n // 4) // C) // 4) * 4          # slices per CTA
    if 4 * C > (n + 3) // 4 or chunk > 256 * 13:
        pytest.skip("no cluster shape for this row length")
    s = rk_inputs.gaussian_system(m, n, seed=m + n + C)
    plan = rk.rk_setup(rk.aligned_rows(_dev(s.A)))
    tab = oracle.table(s.A)
    x0 = np.random.default_rng(3).standard_normal(n).astype(np.float32)
    x, info = rk.rkab_solve(plan, _dev(s.b), _dev(x0), q=q, alpha=alpha, rounds=rounds, seed=17,
                            cluster_size=C, lookahead=lookahead)
    assert info.status == 0 and info.rounds_done == rounds
    xo = oracle.rkab(s.A, s.b.astype(np.float64), x0.astype(np.float64), q=q, alpha=alpha,
                     rounds=rounds, seed=17, tab=tab)
    assert_close(x.cpu().numpy(), xo, TOL)


@pytest.mark.parametrize("kind", ["bf16", "fp8"])
def test_cluster_workers_on_stored_rows(rk, kind):
    s = rk_inputs.gaussian_system(4000, 2000, seed=71)
    A = _dev(s.A)
    Aq, sc = rk.quantize(A, kind)
    plan = rk.rk_setup(Aq, kind, sc)
    low = oracle.quantize_bf16(s.A)[1] if kind == "bf16" else oracle.quantize_fp8(s.A)[2]
    tab = oracle.table(low)
    x, info = rk.rkab_solve(plan, _dev(s.b), q=3, alpha=40, rounds=3, seed=4, cluster_size=4)
    assert info.status == 0
    xo = oracle.rkab(low, s.b.astype(np.float64), np.zeros(2000), q=3, alpha=40, rounds=3, seed=4,
                     tab=tab)
    assert_close(x.cpu().numpy(), xo, TOL)


def test_cluster_rk_converges_with_stop_rule(rk):
    """q = 1 (RK) on an 8-CTA cluster reaches 1e-6 on a consistent system."""
    s = rk_inputs.gaussian_system(20000, 2000, seed=73)
    plan = rk.rk_setup(_dev(s.A))
    xs = _dev(s.x_star)
    x, info = rk.rkab_solve(plan, _dev(s.b), q=1, alpha=2000, rounds=400, seed=1, x_ref=xs,
                            tol=1e-6, cluster_size=8)
    assert info.status == 0 and info.last_metric < 1e-6, info
    assert _rel(x.cpu().numpy(), s.x_star.astype(np.float64)) < 1e-6


@pytest.mark.parametrize("C", [8, 16])
def test_long_row_cluster_workers_match_oracle(rk, C):
    """Rows of 70000 columns (chunks of more than 1024 slices per CTA: the 256-thread
    cluster variants with look-ahead pairs), an underdetermined consistent system."""
    m, n, q = 300, 70000, 2
    s = rk_inputs.gaussian_system(m, n, seed=C)
    plan = rk.rk_setup(rk.aligned_rows(_dev(s.A)))
    tab = oracle.table(s.A)
    x, info = rk.rkab_solve(plan, _dev(s.b), q=q, alpha=40, rounds=3, seed=5, cluster_size=C)
    assert info.status == 0 and info.rounds_done == 3
    xo = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(n), q=q, alpha=40, rounds=3, seed=5,
                     tab=tab)
    assert_close(x.cpu().numpy(), xo, TOL)


@pytest.mark.parametrize("kind", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("m,n,alpha,shape", [
    (300, 50000, 40, "128 threads x 8 slices"),     # 784 slices a CTA (A^T rows of 50000)
    (120, 200000, 30, "256 threads x 13 slices"),   # 3128 slices a CTA (A^T rows of 200000)
])
def test_adjoint_length_rows_match_oracle(rk, kind, m, n, alpha, shape):
    """The cluster instantiations the adjoint's minimum-norm solve runs on (rows of A^T
    as long as the 50000 x 5000 and 200000 x 20000 differentiation workloads give: six
    workers of 16-CTA clusters, as the benchmark launches them), on float32, BF16 and FP8
    rows: the same draws as the oracle and x within 1e-4, every element."""
    s = rk_inputs.gaussian_system(m, n, seed=n + 3)
    A = _dev(s.A)
    if kind == "f32":
        plan, low = rk.rk_setup(A), s.A
    else:
        Aq, sc = rk.quantize(A, kind)
        plan = rk.rk_setup(Aq, kind, sc)
        low = oracle.quantize_bf16(s.A)[1] if kind == "bf16" else oracle.quantize_fp8(s.A)[2]
    q = 6
    x, info = rk.rkab_solve(plan, _dev(s.b), q=q, alpha=alpha, rounds=3, seed=11, cluster_size=16,
                            check_every=0)
    assert info.status == 0 and info.rounds_done == 3
    xo = oracle.rkab(low, s.b.astype(np.float64), np.zeros(n), q=q, alpha=alpha, rounds=3, seed=11,
                     tab=oracle.table(low))
    assert_close(x.cpu().numpy(), xo, TOL, what=f"{kind} {shape}")


@pytest.mark.parametrize("C", [4, 16])
def test_cluster_wait_limit_ends_the_solve_with_a_status(rk, C):
    """The cluster kernel's device waits are bounded: with a 1 us limit the first wait for
    a row runs out, the CTAs of every cluster wind down (a receive buffer armed for a group
    whose totals never came is waited for again, bounded, before the cluster's CTAs leave)
    and the solve reports RK_ETIMEOUT; the same plan solves normally afterwards."""
    A_t, b_t, _ = rk_inputs.gaussian_system_torch(6000, 10000, seed=9, device="cuda")
    plan = rk.rk_setup(A_t)
    x, info = rk.rkab_solve(plan, b_t, q=3, alpha=40, rounds=3, seed=2, check_every=0, cluster_size=C,
                            timeout_s=1e-6, raise_on_error=False)
    torch.cuda.synchronize()
    assert info.status == -4, info   # RK_ETIMEOUT
    x, info = rk.rkab_solve(plan, b_t, q=3, alpha=40, rounds=3, seed=2, check_every=0, cluster_size=C)
    assert info.status == 0
    assert torch.isfinite(x).all()
