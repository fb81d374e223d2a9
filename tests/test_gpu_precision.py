"""Precision form on the GPU against the oracle: stored-row quantisers (bit
exact), sampling tables of the stored rows (bit exact), RKAB on BF16 / FP8 rows
(x within 1e-4 of the oracle run on the stored values), and iterative
refinement (each outer iterate within 1e-4 of the oracle's; convergence to a
relative error of 1e-6 against x*)."""
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


@pytest.fixture(scope="module")
def sysm():
    return rk_inputs.gaussian_system(3001, 37, seed=51)


def test_quantizers_bit_exact(rk, sysm):
    A = rk.aligned_rows(_dev(sysm.A))
    qb, _ = rk.quantize(A, "bf16")
    codes_b, _ = oracle.quantize_bf16(sysm.A)
    assert np.array_equal(qb.cpu().view(torch.int16).numpy().view(np.uint16), codes_b)
    qf, sc = rk.quantize(A, "fp8")
    codes_f, sc_o, _ = oracle.quantize_fp8(sysm.A)
    assert np.array_equal(sc.cpu().numpy(), sc_o)
    assert np.array_equal(qf.cpu().numpy(), codes_f)


@pytest.mark.parametrize("kind", ["bf16", "fp8"])
@pytest.mark.parametrize("shape", [None, (400, 2600), (300, 4100), (250, 9000), (120, 30000),
                                   (100, 60000)])
def test_stored_row_tables_bit_exact(rk, sysm, kind, shape):
    """Short rows (a warp a row) and rows of 8 KB to 64 KB in the stored type (a CTA a
    row, staged in shared memory), bit-exact against the oracle."""
    if shape is not None:
        m, n = shape
        sysm = rk_inputs.gaussian_system(m, n, seed=m + n)
    A = rk.aligned_rows(_dev(sysm.A))
    Aq, sc = rk.quantize(A, kind)
    plan = rk.rk_setup(Aq, kind, sc)
    low = oracle.quantize_bf16(sysm.A)[1] if kind == "bf16" else oracle.quantize_fp8(sysm.A)[2]
    tab = oracle.table(low)
    T, L = plan.status()
    assert (T, L) == (tab.T, tab.L)
    t = plan.tables()
    assert np.array_equal(t["thr64"].cpu().numpy().view(np.uint64), tab.thr64)
    assert np.array_equal(t["alias"].cpu().numpy().view(np.uint32), tab.alias)
    w = oracle.row_norms(low)
    np.testing.assert_allclose(t["inv"].cpu().numpy(), (1.0 / w).astype(np.float32), rtol=2e-7)


@pytest.mark.parametrize("kind", ["bf16", "fp8"])
@pytest.mark.parametrize("m,n,q,alpha,rounds", [(3001, 37, 3, 7, 10), (6000, 2600, 5, 30, 3),
                                                (2500, 300, 8, 40, 6), (2000, 15000, 2, 15, 2),
                                                # x in shared memory: 16 slices a thread with a ragged
                                                # tail, and 12 slices a thread
                                                (1500, 15003, 3, 20, 2), (2500, 11001, 4, 25, 3)])
def test_rkab_on_stored_rows_matches_oracle(rk, kind, m, n, q, alpha, rounds):
    s = rk_inputs.gaussian_system(m, n, seed=m + 2 * n)
    A = rk.aligned_rows(_dev(s.A))
    Aq, sc = rk.quantize(A, kind)
    plan = rk.rk_setup(Aq, kind, sc)
    low = oracle.quantize_bf16(s.A)[1] if kind == "bf16" else oracle.quantize_fp8(s.A)[2]
    tab = oracle.table(low)
    x, info = rk.rkab_solve(plan, _dev(s.b), q=q, alpha=alpha, rounds=rounds, seed=5)
    assert info.status == 0
    xo = oracle.rkab(low, s.b.astype(np.float64), np.zeros(n), q=q, alpha=alpha, rounds=rounds,
                     seed=5, tab=tab)
    assert_close(x.cpu().numpy(), xo, TOL)


@pytest.mark.parametrize("kind", ["bf16", "fp8", "f32"])
def test_refinement_steps_match_oracle(rk, kind):
    s = rk_inputs.gaussian_system(4000, 200, seed=57)
    A = rk.aligned_rows(_dev(s.A))
    if kind == "f32":
        plan, low = rk.rk_setup(A), s.A
    else:
        Aq, sc = rk.quantize(A, kind)
        plan = rk.rk_setup(Aq, kind, sc)
        low = oracle.quantize_bf16(s.A)[1] if kind == "bf16" else oracle.quantize_fp8(s.A)[2]
    tab = oracle.table(low)
    b = _dev(s.b)
    xs_o = oracle.refine(s.A, low, s.b.astype(np.float64), np.zeros(200), q=6, alpha=100,
                         inner_rounds=4, outer=3, seed=2, tab_low=tab)
    for k in range(3):
        x, info = rk.rkab_refine(plan, A, b, q=6, alpha=100, inner_rounds=4, max_outer=k + 1, seed=2)
        assert info.outer_done == k + 1
        assert_close(x.cpu().numpy(), xs_o[k], TOL, what=str((kind, k)))


@pytest.mark.parametrize("kind", ["bf16", "fp8"])
def test_refinement_reaches_1e6(rk, kind):
    s = rk_inputs.gaussian_system(20000, 500, seed=61)
    A = _dev(s.A)
    Aq, sc = rk.quantize(A, kind)
    plan = rk.rk_setup(Aq, kind, sc)
    xs = _dev(s.x_star)
    x, info = rk.rkab_refine(plan, A, _dev(s.b), q=16, alpha=500, inner_rounds=6, max_outer=20,
                             seed=3, x_ref=xs, tol=1e-6)
    assert 0 < info.outer_done < 20 and info.last_metric < 1e-6, info
    assert _rel(x.cpu().numpy(), s.x_star.astype(np.float64)) < 1e-6
