"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs.  Integer work (sampling tables, row draws) must be bit-exact; x must
be within 1e-4 relative (FP32 kernel vs FP64 oracle).

Tolerance: each projection and the average are non-expansive maps
(Section 2.1), so FP32 rounding differences do not grow along the
trajectory; the FP32 unit roundoff (6e-8) times the contraction horizon of
the 2000 x 100 system (1/s_min ~ 170 projections) bounds the drift near 1e-5,
inside the 1e-4 bar."""
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


def _padded(A_np, rk):
    return rk.aligned_rows(_dev(A_np))


def _check_tables(rk, A_np, plan=None):
    tab = oracle.table(A_np)
    if plan is None:
        plan = rk.rk_setup(_padded(A_np, rk))
    T, L = plan.status()
    assert (T, L) == (tab.T, tab.L)
    t = plan.tables()
    K = t["K"].cpu().numpy().view(np.uint64)
    P = t["P"].cpu().numpy().view(np.uint64)
    thr = t["thr64"].cpu().numpy().view(np.uint64)
    al = t["alias"].cpu().numpy().view(np.uint32)
    assert np.array_equal(K, tab.K)
    P_ref = np.concatenate([np.zeros(1, np.uint64), np.cumsum(tab.K[:-1], dtype=np.uint64)])
    assert np.array_equal(P, P_ref)
    assert np.array_equal(thr, tab.thr64)
    assert np.array_equal(al, tab.alias)
    inv = t["inv"].cpu().numpy()
    assert np.all(np.isfinite(inv))
    w = oracle.row_norms(A_np)
    # rows whose ||A_i||^2 has a float32 reciprocal get it; zero rows and rows outside
    # [2^-126, 2^126) (never drawn when the plan succeeds) get 0
    ok = (w >= 2.0 ** -126) & (w < 2.0 ** 126)
    rel = np.abs(inv[ok].astype(np.float64) * w[ok] - 1.0)
    assert np.all(rel <= 2.0 ** -24 * 1.01), rel.max()
    assert np.all(inv[~ok] == 0)
    return plan, tab


@pytest.mark.parametrize("case", ["c1", "skewed", "ragged", "zerorows", "onerow", "onecol", "tiny_values"])
def test_tables_bit_exact(rk, case):
    rng = np.random.default_rng(21)
    if case == "c1":
        A = rk_inputs.gaussian_system(2000, 100, seed=0).A
    elif case == "skewed":
        A = rk_inputs.gaussian_system(5000, 64, seed=1, row_scale_decades=2.0).A
    elif case == "ragged":
        A = rng.standard_normal((3001, 37)).astype(np.float32)
    elif case == "zerorows":
        A = rng.standard_normal((777, 20)).astype(np.float32)
        A[::5] = 0
    elif case == "onerow":
        A = rng.standard_normal((1, 9)).astype(np.float32)
    elif case == "onecol":
        A = rng.standard_normal((513, 1)).astype(np.float32)
    else:
        A = (rng.standard_normal((300, 12)) * 1e-41).astype(np.float32)  # subnormals
        A[3] *= np.float32(1e30)
    _check_tables(rk, A)


@pytest.mark.parametrize("m,n,special", [
    (600, 1025, "ragged"),        # 4 KB rows, a 1-element tail chunk (a warp a row)
    (500, 2500, "ragged"),        # 10 KB rows (a CTA a row, 8 rows in flight)
    (300, 4096, "zerorows"),      # 16 KB rows (a CTA a row, 4 in flight)
    (300, 4097, "skewed"),        # a 1-element tail chunk
    (200, 10000, "tiny_values"),  # 40 KB rows (2 in flight); rows whose largest entry is subnormal
    (120, 16384, "plain"),        # 64 KB rows, the longest staged in shared memory
    (90, 16387, "ragged"),        # past 64 KB rows: a warp a row again
])
def test_tables_bit_exact_long_rows(rk, m, n, special):
    """Sampling tables of rows long enough for the CTA-per-row setup kernel (rows
    staged in shared memory), bit-exact against the oracle."""
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n)).astype(np.float32)
    if special == "zerorows":
        A[::7] = 0
    elif special == "skewed":
        A *= (10.0 ** rng.uniform(-2, 2, size=(m, 1))).astype(np.float32)
    elif special == "tiny_values":
        A[::3] = (A[::3] * 1e-41).astype(np.float32)   # subnormal rows
        A[1::3, :5] *= np.float32(2.0 ** 59)              # the rest of the row floors to 0
        # (||A_i||^2 stays below 2^126, the float32 range of the projection)
        A[2::3, :3] *= np.float32(2.0 ** 20)              # entries below 2^-5 floor to nonzero terms
    _check_tables(rk, A)


def _tiny_system(m, n, seed):
    """A system whose every row lies below the float32 range of the projection
    (entries about 1e-41, subnormal; ||A_i||^2 about 1e-81), b = fl32(A x*)."""
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((m, n)) * 1e-41).astype(np.float32)
    x_star = rng.standard_normal(n)
    b = (A.astype(np.float64) @ x_star).astype(np.float32)
    return A, b


def test_rows_below_float32_range_are_refused(rk):
    """Rows the law draws whose ||A_i||^2 < 2^-126: no float32 reciprocal exists and the
    products <A_i, x> underflow, so the plan fails (RK_ESETUP) and a solve on it reports
    RK_ESETUP instead of projecting with an infinite scale."""
    A, b = _tiny_system(300, 12, seed=5)
    plan = rk.rk_setup(_padded(A, rk))
    with pytest.raises(rk.RkError) as e:
        plan.status()
    assert e.value.code == -8
    x, info = rk.rkab_solve(plan, _dev(b), q=2, alpha=10, rounds=2, seed=1, raise_on_error=False)
    assert info.status == -8


def test_subnormal_system_scaled_into_range_matches_oracle(rk):
    """The same all-subnormal system scaled by 2^120 (exact in float32; Eq. (alg) is
    invariant under scaling a row and its b_i) solves on the GPU and equals the FP64
    oracle run on the unscaled system: same law (the integer weights are invariant
    under power-of-two scaling), same draws, x within 1e-4."""
    A, b = _tiny_system(300, 12, seed=5)
    s2 = np.float32(2.0 ** 120)
    A2, b2 = A * s2, b * s2
    assert np.array_equal(A2 / s2, A) and np.array_equal(b2 / s2, b)
    tab = oracle.table(A)
    plan = rk.rk_setup(_padded(A2, rk))
    assert plan.status() == (tab.T, tab.L + 240)
    x, info = rk.rkab_solve(plan, _dev(b2), q=3, alpha=20, rounds=6, seed=4, check_every=0)
    assert info.status == 0
    xo = oracle.rkab(A, b.astype(np.float64), np.zeros(12), q=3, alpha=20, rounds=6, seed=4, tab=tab)
    assert_close(x.cpu().numpy(), xo, TOL)


def test_out_of_range_rows_never_drawn(rk):
    """Rows below the float32 range in a matrix whose law never draws them (K_i = 0):
    the plan works and the solve matches the oracle; the cyclic sweep, which would visit
    them, is refused with RK_EINVAL."""
    s = rk_inputs.gaussian_system(2000, 100, seed=2)
    A = s.A.copy()
    A[::50] *= np.float32(1e-41)
    b = (A.astype(np.float64) @ s.x_star.astype(np.float64)).astype(np.float32)
    plan, tab = _check_tables(rk, A)
    assert np.all(tab.K[::50] == 0)
    x, info = rk.rkab_solve(plan, _dev(b), q=4, alpha=30, rounds=5, seed=6, check_every=0)
    assert info.status == 0
    xo = oracle.rkab(A, b.astype(np.float64), np.zeros(100), q=4, alpha=30, rounds=5, seed=6, tab=tab)
    assert_close(x.cpu().numpy(), xo, TOL)
    x, info = rk.rkab_solve(plan, _dev(b), q=4, alpha=30, rounds=2, seed=6, sampling="cyclic",
                            raise_on_error=False)
    assert info.status == -1


@pytest.mark.parametrize("n", [9, 3000])
def test_setup_rejects_nonfinite_entries(rk, n):
    for bad in (float("nan"), float("inf")):
        B = torch.randn((64, n), device="cuda")
        B[37, n // 2] = bad
        with pytest.raises(rk.RkError):
            rk.rk_setup(rk.aligned_rows(B)).status()


def test_setup_rejects_zero_and_nonfinite(rk):
    A = torch.zeros((64, 8), device="cuda")
    plan = rk.rk_setup(A)
    with pytest.raises(rk.RkError):
        plan.status()
    B = torch.randn((64, 8), device="cuda")
    B[7, 3] = float("nan")
    plan = rk.rk_setup(B)
    with pytest.raises(rk.RkError):
        plan.status()


def test_row_draws_bit_exact(rk):
    s = rk_inputs.gaussian_system(2000, 100, seed=0)
    plan, tab = _check_tables(rk, s.A)
    for worker, t0, count, stream in [(0, 0, 20000, 0), (3, 12345, 5000, 0), (131, 0, 4000, 1),
                                      (7, (1 << 32) - 100, 300, 2), (1, 1 << 40, 100, 3 | (5 << 8))]:
        got = rk.rk_sample_indices(plan, 0xDEADBEEF12345, worker, t0, count, stream).cpu().numpy()
        want = oracle.sample_rows(tab, 0xDEADBEEF12345, worker, t0, count, stream)
        assert np.array_equal(got.astype(np.int64), want), (worker, t0)


def _rel(xg, xo):
    return np.linalg.norm(xg.astype(np.float64) - xo) / max(np.linalg.norm(xo), 1e-300)


@pytest.fixture(scope="module")
def c1(rk):
    s = rk_inputs.gaussian_system(2000, 100, seed=0)
    plan = rk.rk_setup(_dev(s.A))
    return s, plan, oracle.table(s.A), _dev(s.b)


@pytest.mark.parametrize("q", [1, 4])
@pytest.mark.parametrize("k", [1, 10, 100, 1000, 20000])
def test_c1_rk_and_rka_match_oracle(rk, c1, q, k):
    """2000 x 100, x0 = 0, seed 0: RK (q=1) and RKA (q=4, alpha=1) after k rounds."""
    s, plan, tab, b = c1
    x, info = rk.rkab_solve(plan, b, q=q, alpha=1, rounds=k, seed=0, check_every=0)
    assert info.status == 0
    xo = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(100), q=q, alpha=1, rounds=k, seed=0,
                     tab=tab)
    assert_close(x.cpu().numpy(), xo, TOL)


@pytest.mark.parametrize("m,n,q,alpha,rounds,omega", [
    (3001, 37, 3, 7, 20, 1.0),       # ragged n (tail of a float4), several stages
    (5000, 300, 8, 50, 6, 1.5),      # relaxation
    (4000, 1000, 16, 40, 4, 1.0),    # 128-thread CTAs, wider rows
    (6000, 2600, 5, 30, 3, 0.8),     # 256-thread CTAs, 3 slices a thread
    (3000, 12000, 3, 20, 2, 1.0),    # 256-thread CTAs, 12 slices a thread, row re-read from shared memory
    (2000, 15003, 2, 15, 2, 1.2),    # 16 slices a thread, ragged tail
    (800, 5, 2, 3, 50, 1.0),         # n < 8
])
def test_rkab_matches_oracle(rk, m, n, q, alpha, rounds, omega):
    s = rk_inputs.gaussian_system(m, n, seed=m + n)
    A = _padded(s.A, rk)
    plan = rk.rk_setup(A)
    tab = oracle.table(s.A)
    x0 = np.random.default_rng(1).standard_normal(n).astype(np.float32)
    x, info = rk.rkab_solve(plan, _dev(s.b), _dev(x0), q=q, alpha=alpha, rounds=rounds, seed=77,
                            omega=omega)
    assert info.status == 0 and info.rounds_done == rounds
    xo = oracle.rkab(s.A, s.b.astype(np.float64), x0.astype(np.float64), q=q, alpha=alpha,
                     rounds=rounds, seed=77, tab=tab, omega=omega)
    assert_close(x.cpu().numpy(), xo, TOL)


@pytest.mark.parametrize("lookahead", [1, 2, 4])
@pytest.mark.parametrize("m,n,q,alpha,rounds", [(3000, 600, 4, 37, 5), (6000, 2600, 5, 30, 3),
                                                (8000, 9000, 3, 21, 2)])
def test_lookahead_groups_match_oracle(rk, lookahead, m, n, q, alpha, rounds):
    """Rows resolved in groups (one CTA reduction per group, scalar recurrence)
    follow the same trajectory as one row at a time (alpha not a multiple of
    the group size: the last group of each round is short)."""
    s = rk_inputs.gaussian_system(m, n, seed=m + n + 1)
    plan = rk.rk_setup(_padded(s.A, rk))
    tab = oracle.table(s.A)
    x, info = rk.rkab_solve(plan, _dev(s.b), q=q, alpha=alpha, rounds=rounds, seed=13,
                            lookahead=lookahead)
    assert info.status == 0
    xo = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(n), q=q, alpha=alpha, rounds=rounds,
                     seed=13, tab=tab)
    assert_close(x.cpu().numpy(), xo, TOL)


def test_special_cases_on_gpu(rk, c1):
    s, plan, tab, b = c1
    # q = 1 RKAB with alpha = 30 is RK over 30 * rounds projections
    x1, _ = rk.rkab_solve(plan, b, q=1, alpha=30, rounds=5, seed=3)
    xo = oracle.rk(s.A, s.b.astype(np.float64), np.zeros(100), 150, 3, tab)
    assert_close(x1.cpu().numpy(), xo, TOL)
    # all workers on one stream average identical iterates: equals RK
    x2, _ = rk.rkab_solve(plan, b, q=6, alpha=30, rounds=5, seed=3, same_stream=True)
    assert_close(x2.cpu().numpy(), xo, TOL)
    # rounds = 0 returns x0
    x0 = torch.randn(100, device="cuda")
    x3, _ = rk.rkab_solve(plan, b, x0, q=2, alpha=4, rounds=0, seed=1)
    assert torch.equal(x3, x0)


def test_resume_is_bit_identical(rk, c1):
    s, plan, tab, b = c1
    full, _ = rk.rkab_solve(plan, b, q=4, alpha=9, rounds=12, seed=5)
    part, _ = rk.rkab_solve(plan, b, q=4, alpha=9, rounds=5, seed=5)
    rest, _ = rk.rkab_solve(plan, b, part.clone(), q=4, alpha=9, rounds=7, seed=5, round0=5)
    assert torch.equal(full, rest)
    again, _ = rk.rkab_solve(plan, b, q=4, alpha=9, rounds=12, seed=5)
    assert torch.equal(full, again)   # deterministic run to run


def test_x_may_alias_x0(rk, c1):
    s, plan, tab, b = c1
    x0 = torch.randn(100, device="cuda")
    ref, _ = rk.rkab_solve(plan, b, x0.clone(), q=3, alpha=5, rounds=4, seed=2)
    buf = x0.clone()
    rk.rkab_solve(plan, b, buf, q=3, alpha=5, rounds=4, seed=2, out=buf)
    assert torch.equal(buf, ref)


def test_stop_rule_matches_oracle(rk, c1):
    s, plan, tab, b = c1
    xs = _dev(s.x_star)
    x, info = rk.rkab_solve(plan, b, q=4, alpha=20, rounds=5000, seed=0, x_ref=xs, tol=1e-5)
    _, done_o = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(100), q=4, alpha=20,
                            rounds=5000, seed=0, tab=tab, x_ref=s.x_star.astype(np.float64),
                            tol=1e-5)
    assert abs(info.rounds_done - done_o) <= 1
    assert info.last_metric < 1e-5
    assert _rel(x.cpu().numpy(), s.x_star.astype(np.float64)) < 1.2e-5


def test_argument_errors(rk, c1):
    s, plan, tab, b = c1
    with pytest.raises(rk.RkError):
        rk.rkab_solve(plan, b, q=0, alpha=1, rounds=1)
    with pytest.raises(rk.RkError):
        rk.rkab_solve(plan, b, q=2, alpha=1, rounds=1, omega=4.0)   # omega < 2q
    with pytest.raises(rk.RkError) as e:
        rk.rkab_solve(plan, b, q=100000, alpha=2, rounds=1)
    assert e.value.code == -3   # not co-resident: refused before launch


def test_residual_matches_oracle(rk):
    s = rk_inputs.gaussian_system(3000, 37, seed=3, noise=0.1)
    A = _padded(s.A, rk)
    x = np.random.default_rng(2).standard_normal(37).astype(np.float32)
    r, norms = rk.rk_residual(A, _dev(s.b), _dev(x))
    ro, rn, an = oracle.residual(s.A, s.b, x.astype(np.float64))
    scale = np.abs(s.b).max() + np.abs(s.A).sum(axis=1).max() * np.abs(x).max()
    np.testing.assert_allclose(r.cpu().numpy(), ro, rtol=0, atol=1e-13 * scale)
    nn = norms.cpu().numpy()
    assert abs(nn[0] - rn) <= 1e-12 * rn and abs(nn[1] - an) <= 1e-10 * (an + 1e-300)


@pytest.mark.slow
def test_full_size_sampled_parity(rk):
    """80000 x 10000 (3.2 GB), the launch configuration of the benchmark
    (q = 132, alpha = n): bit-exact tables and draws, one short round of every
    worker against the oracle, and convergence of the full solve to 1e-6."""
    m, n, q = 80000, 10000, 132
    s = rk_inputs.gaussian_system(m, n, seed=0)
    A = _dev(s.A)
    plan, tab = _check_tables(rk, s.A, rk.rk_setup(A))
    for g in (0, 1, 65, 131):
        got = rk.rk_sample_indices(plan, 0, g, 10_000 * 7, 10_000).cpu().numpy()
        assert np.array_equal(got.astype(np.int64), oracle.sample_rows(tab, 0, g, 70_000, 10_000))
    b = _dev(s.b)
    x, info = rk.rkab_solve(plan, b, q=q, alpha=10, rounds=1, seed=0)
    xo = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(n), q=q, alpha=10, rounds=1, seed=0,
                     tab=tab, threads=8)
    assert_close(x.cpu().numpy(), xo, TOL)
    xs = _dev(s.x_star)
    x, info = rk.rkab_solve(plan, b, q=q, alpha=n, rounds=400, seed=0, x_ref=xs, tol=1e-6)
    assert info.status == 0 and info.last_metric < 1e-6, info
    assert _rel(x.cpu().numpy(), s.x_star.astype(np.float64)) < 1e-6
    # the fastest configuration at full size: RKA with 4864 workers spread over the CTAs and
    # the weight alpha* (from 2 Lanczos steps, ||A||_F^2 from the plan): two rounds against
    # the oracle, then convergence to 1e-6
    qa = 4864
    w, _ = rk.optimal_weight(A, qa, k=2, plan=plan)
    x, info = rk.rka_solve(plan, b, q=qa, rounds=2, seed=0, omega=w, check_every=0)
    xo = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(n), q=qa, alpha=1, rounds=2, seed=0,
                     tab=tab, omega=float(np.float32(w)), threads=8)
    assert_close(x.cpu().numpy(), xo, TOL)
    x, info = rk.rka_solve(plan, b, q=qa, rounds=400, seed=0, omega=w, x_ref=xs, tol=1e-6)
    assert info.status == 0 and info.last_metric < 1e-6 and info.rounds_done < 120, info


@pytest.mark.slow
def test_lsq_size_sampled_parity(rk):
    """200000 x 20000 (16 GB) with rows scaled by 10^U(-2,2) and b = A x* + N(0, 1e-3^2),
    the least-squares workload in the benchmark's launch configuration (q = 132, rows of
    80 KB): bit-exact tables, one short round of every worker against the oracle, and the
    residual norms at that x against the oracle's FP64 residual."""
    m, n, q = 200000, 20000, 132
    A, b, _ = rk_inputs.gaussian_system_torch(m, n, seed=0, noise=1e-3, row_scale_decades=2.0,
                                              device="cuda")
    A_np = A.cpu().numpy()
    b_np = b.cpu().numpy()
    plan, tab = _check_tables(rk, A_np, rk.rk_setup(A))
    x, info = rk.rkab_solve(plan, b, q=q, alpha=3, rounds=1, seed=0, check_every=0)
    assert info.status == 0
    xo = oracle.rkab(A_np, b_np.astype(np.float64), np.zeros(n), q=q, alpha=3, rounds=1, seed=0,
                     tab=tab, threads=8)
    assert_close(x.cpu().numpy(), xo, TOL)
    _, norms = rk.rk_residual(A, b, x)
    _, rn, an = oracle.residual(A_np, b_np, x.cpu().numpy().astype(np.float64))
    nn = norms.cpu().numpy()
    assert abs(nn[0] - rn) <= 1e-12 * rn and abs(nn[1] - an) <= 1e-10 * an


def test_wait_limit_ends_the_solve_with_a_status(rk):
    """Every device-side wait is bounded: with a 1 us limit the first wait for a row
    (a cold HBM copy takes longer) runs out, the kernel winds down (copies in flight
    drained, no stage refilled) and reports RK_ETIMEOUT; the context stays usable."""
    A_t, b_t, xs_t = rk_inputs.gaussian_system_torch(20000, 2000, seed=4, device="cuda")
    plan = rk.rk_setup(A_t)
    x, info = rk.rkab_solve(plan, b_t, q=4, alpha=500, rounds=3, seed=1, check_every=0,
                            timeout_s=1e-6, raise_on_error=False)
    torch.cuda.synchronize()
    assert info.status == -4, info   # RK_ETIMEOUT
    # the same plan solves normally afterwards
    x, info = rk.rkab_solve(plan, b_t, q=4, alpha=500, rounds=3, seed=1, check_every=0)
    assert info.status == 0
    assert torch.isfinite(x).all()


@pytest.mark.parametrize("alpha,rounds", [(1, 20), (25, 4)])
def test_more_workers_than_sms_matches_oracle(rk, alpha, rounds):
    """q above the SM count: RKA (alpha = 1) spreads the workers over one CTA per SM,
    RKAB runs two workers per SM (the two-per-SM variants); same draws, x within 1e-4
    of the oracle; RKAB beyond two workers per SM is refused."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    q = sms + 8
    s = rk_inputs.gaussian_system(2000, 100, seed=0)
    tab = oracle.table(s.A)
    plan = rk.rk_setup(_padded(s.A, rk))
    x, info = rk.rkab_solve(plan, _dev(s.b), q=q, alpha=alpha, rounds=rounds, seed=3,
                            check_every=0)
    assert info.status == 0 and info.rounds_done == rounds
    x_o = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(100), q=q, alpha=alpha,
                      rounds=rounds, seed=3, tab=tab)
    assert_close(x.cpu().numpy(), x_o, TOL)
    with pytest.raises(rk.RkError) as e:
        rk.rkab_solve(plan, _dev(s.b), q=2 * sms + 1, alpha=2, rounds=1)
    assert e.value.code == -3


@pytest.mark.parametrize("mult,extra,omega", [(4, 3, 1.0), (16, 0, None), (7, 11, None)])
def test_rka_many_workers_matches_oracle(rk, mult, extra, omega):
    """RKA with q = mult * SMs + extra workers (uneven shares per CTA), unit weight or the
    optimal weight of Eq. (best_alpha): x within 1e-4 of the oracle after 15 rounds."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    q = mult * sms + extra
    s = rk_inputs.gaussian_system(4000, 200, seed=1)
    tab = oracle.table(s.A)
    if omega is None:
        lmin, lmax, fro2 = oracle.spectrum(s.A)
        omega = float(np.float32(oracle.alpha_star(q, lmin / fro2, lmax / fro2)))
    plan = rk.rk_setup(_padded(s.A, rk))
    x, info = rk.rka_solve(plan, _dev(s.b), q=q, rounds=15, seed=9, omega=omega, check_every=0)
    assert info.status == 0 and info.rounds_done == 15
    x_o = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(200), q=q, alpha=1, rounds=15,
                      seed=9, tab=tab, omega=omega)
    assert_close(x.cpu().numpy(), x_o, TOL)


@pytest.mark.parametrize("sampling", ["blocks", "cyclic"])
def test_selection_draws_bit_exact(rk, sampling):
    """Row blocks (Section 3.3.1) and cyclic sweep: the device row choices equal the
    oracle's for workers of uneven blocks, including a zero row."""
    s = rk_inputs.gaussian_system(1003, 16, seed=5, row_scale_decades=2.0)
    A_np = s.A.copy()
    A_np[17] = 0.0
    tab = oracle.table(A_np)
    plan = rk.rk_setup(_padded(A_np, rk))
    for q, g in ((1, 0), (7, 0), (7, 3), (7, 6), (64, 63)):
        got = rk.rk_sample_indices(plan, 21, g, 1000, 3000, sampling=sampling, q=q).cpu().numpy()
        ref = oracle.sample_rows(tab, 21, g, 1000, 3000, sampling=sampling, q=q)
        assert np.array_equal(got.astype(np.int64) & 0xFFFFFFFF, ref), (q, g)


@pytest.mark.parametrize("sampling,q,alpha,rounds", [("blocks", 4, 50, 6), ("cyclic", 3, 40, 5),
                                                     ("blocks", 1, 30, 4)])
def test_selection_solve_matches_oracle(rk, sampling, q, alpha, rounds):
    s = rk_inputs.gaussian_system(2000, 100, seed=0)
    tab = oracle.table(s.A)
    plan = rk.rk_setup(_padded(s.A, rk))
    x, info = rk.rkab_solve(plan, _dev(s.b), q=q, alpha=alpha, rounds=rounds, seed=7,
                            check_every=0, sampling=sampling)
    assert info.status == 0
    x_o = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(100), q=q, alpha=alpha, rounds=rounds,
                      seed=7, tab=tab, sampling=sampling)
    assert_close(x.cpu().numpy(), x_o, TOL)


def test_row_weights_and_many_worker_blocks_match_oracle(rk):
    """Per-row weights w_i of Eq. (rka_eq), and RKA with row blocks for more workers than
    SMs (the workers spread over the CTAs)."""
    s = rk_inputs.gaussian_system(4000, 100, seed=3)
    tab = oracle.table(s.A)
    plan = rk.rk_setup(_padded(s.A, rk))
    w = np.random.default_rng(1).uniform(0.5, 1.5, 4000).astype(np.float32)
    x, info = rk.rkab_solve(plan, _dev(s.b), q=5, alpha=40, rounds=5, seed=2, check_every=0,
                            row_weight=_dev(w))
    x_o = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(100), q=5, alpha=40, rounds=5, seed=2,
                      tab=tab, row_weight=w.astype(np.float64))
    assert info.status == 0
    assert_close(x.cpu().numpy(), x_o, TOL)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    q = 2 * sms + 5
    x, info = rk.rka_solve(plan, _dev(s.b), q=q, rounds=10, seed=4, check_every=0, sampling="blocks")
    x_o = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(100), q=q, alpha=1, rounds=10, seed=4,
                      tab=tab, sampling="blocks")
    assert info.status == 0
    assert_close(x.cpu().numpy(), x_o, TOL)


def test_zero_weight_block_is_refused(rk):
    """A worker whose row block has no weight cannot draw: the solve ends with RK_EINVAL."""
    s = rk_inputs.gaussian_system(400, 20, seed=1)
    A_np = s.A.copy()
    A_np[100:200] = 0.0                      # block 1 of 4
    plan = rk.rk_setup(_padded(A_np, rk))
    with pytest.raises(rk.RkError) as e:
        rk.rkab_solve(plan, _dev(s.b), q=4, alpha=10, rounds=3, seed=0, sampling="blocks")
    assert e.value.code == -1
    with pytest.raises(rk.RkError):
        rk.rkab_solve(plan, _dev(s.b), q=4, alpha=10, rounds=1, sampling="blocks", same_stream=True)


def test_residual_stopping_rules(rk):
    """Stopping rules on the residual (no reference solution): the stretches of rounds
    continue one stream of draws (x equals the oracle's uninterrupted run), and the
    reported criterion equals the FP64 value at the returned x."""
    s = rk_inputs.gaussian_system(2000, 100, seed=0)
    tab = oracle.table(s.A)
    plan = rk.rk_setup(_padded(s.A, rk))
    b64 = s.b.astype(np.float64)
    x, rounds, metric = rk.rkab_solve_residual(plan, _dev(s.b), q=4, alpha=100, max_rounds=400,
                                               check_every=3, tol=1e-6, criterion="residual",
                                               seed=2)
    assert 0 < rounds < 400 and rounds % 3 == 0 and 0 <= metric < 1e-6
    x_o = oracle.rkab(s.A, b64, np.zeros(100), q=4, alpha=100, rounds=rounds, seed=2, tab=tab)
    assert_close(x.cpu().numpy(), x_o, TOL)
    _, rn, _ = oracle.residual(s.A, b64, x.cpu().numpy().astype(np.float64))
    assert metric == pytest.approx(rn / np.linalg.norm(b64), rel=1e-6)
    # least squares: ||A^T r|| / (||A||_F ||r||) on an inconsistent system, uneven stretches
    si = rk_inputs.gaussian_system(2000, 100, seed=1, noise=0.1)
    tabi = oracle.table(si.A)
    plani = rk.rk_setup(_padded(si.A, rk))
    bi = si.b.astype(np.float64)
    x, rounds, metric = rk.rkab_solve_residual(plani, _dev(si.b), q=3, alpha=50, max_rounds=30,
                                               check_every=7, tol=0.0, criterion="normal", seed=4)
    assert rounds == 30
    x_o = oracle.rkab(si.A, bi, np.zeros(100), q=3, alpha=50, rounds=30, seed=4, tab=tabi)
    assert_close(x.cpu().numpy(), x_o, TOL)
    _, rn, an = oracle.residual(si.A, bi, x.cpu().numpy().astype(np.float64))
    fro = np.sqrt(np.sum(si.A.astype(np.float64) ** 2))
    assert metric == pytest.approx(an / (fro * rn), rel=1e-5)


@pytest.mark.parametrize("m,n", [(1, 1), (3, 1), (5, 2), (7, 5), (2, 9)])
@pytest.mark.parametrize("q,alpha", [(1, 1), (3, 7)])
def test_degenerate_shapes_match_oracle(rk, m, n, q, alpha):
    """Single rows and columns, fewer rows than workers, wide systems: the same draws and
    x within 1e-4 of the oracle (the row padding and the tail masking at their limits)."""
    rng = np.random.default_rng(m * 31 + n)
    A = rng.standard_normal((m, n)).astype(np.float32)
    b = rng.standard_normal(m).astype(np.float32)
    tab = oracle.table(A)
    plan = rk.rk_setup(_padded(A, rk))
    x, info = rk.rkab_solve(plan, _dev(b), q=q, alpha=alpha, rounds=5, seed=8, check_every=0)
    assert info.status == 0
    x_o = oracle.rkab(A, b.astype(np.float64), np.zeros(n), q=q, alpha=alpha, rounds=5, seed=8,
                      tab=tab)
    assert_close(x.cpu().numpy(), x_o, TOL)


def test_empty_system_is_refused(rk):
    with pytest.raises((rk.RkError, ValueError)):
        rk.rk_setup(torch.zeros((0, 4), dtype=torch.float32, device="cuda"))
    with pytest.raises((rk.RkError, ValueError)):
        rk.rk_setup(torch.zeros((4, 0), dtype=torch.float32, device="cuda"))


@pytest.mark.parametrize("q,alpha,omega_per_q", [(4, 100, 1.9), (8, 10, 1.9), (200, 1, 1.95)])
def test_divergence_is_reported(rk, c1, q, alpha, omega_per_q):
    """A relaxation beyond the stable range (Section 3.4.2: RKAB can diverge for weights
    above 1) drives the float32 iterate to overflow: the solve stops at the next check
    with RK_EDIVERGED, a host-visible status (no device fault), and the next solve on the
    same plan and context runs normally and matches the oracle."""
    s, plan, tab, b = c1
    x, info = rk.rkab_solve(plan, b, q=q, alpha=alpha, rounds=400, seed=2,
                            omega=omega_per_q * q, raise_on_error=False)
    assert info.status == -5, info
    assert info.rounds_done < 400
    # the check's float32 ||x||^2 overflowed: x itself may still be finite
    assert not torch.isfinite(x).all() or float((x.double() ** 2).sum()) > 3.4e38
    x, info = rk.rkab_solve(plan, b, q=4, alpha=20, rounds=5, seed=3, check_every=1)
    assert info.status == 0 and info.rounds_done == 5
    xo = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(100), q=4, alpha=20, rounds=5,
                     seed=3, tab=tab)
    assert_close(x.cpu().numpy(), xo, TOL)
