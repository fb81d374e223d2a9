"""Differentiation form on the GPU: transpose, rank-2 gradient, the
minimum-norm solve on A^T against the oracle (same draws; one-CTA workers, and x split by
columns over the grid for rows of A^T too long for one CTA), the whole adjoint at the
GPU's forward point against the FP64 QR adjoint at that point (both solve layouts), and
the autograd gradient against central finite differences of the FP64 map."""
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


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_transpose_and_rank2(rk):
    A = torch.randn(1003, 517, device="cuda")
    At = rk.transpose(A)
    assert torch.equal(At, A.t())
    r, y = torch.randn(1003, device="cuda"), torch.randn(1003, device="cuda")
    g, x = torch.randn(517, device="cuda"), torch.randn(517, device="cuda")
    G = rk.rank2(r, g, y, x).double().cpu().numpy()
    ref = (np.outer(r.double().cpu(), g.double().cpu()) - np.outer(y.double().cpu(), x.double().cpu()))
    scale = np.abs(np.outer(r.double().cpu(), g.double().cpu())) + np.abs(np.outer(y.double().cpu(), x.double().cpu()))
    assert np.all(np.abs(G - ref) <= 2 * 2.0 ** -24 * scale + 1e-30)


@pytest.fixture(scope="module")
def inc(rk):
    s = rk_inputs.gaussian_system(3000, 200, seed=83, noise=1e-3)
    xt = rk_inputs.target_vector(200, seed=83)
    A = _dev(s.A)
    return s, xt, A, rk.rk_setup(A)


def test_min_norm_solve_matches_oracle(rk, inc):
    """The y-solve: RKAB on A^T from y = 0 with the draws of stream 1."""
    s, xt, A, plan = inc
    cfg = rk.AdjointConfig(q=4, alpha_t=50, rounds_t=6, alpha=50, rounds=2, seed=7)
    adj = rk.Adjoint(plan, cfg)
    x = torch.zeros(200, device="cuda")
    gx = _dev(xt) * -1.0
    _, gb, _ = adj.backward(_dev(s.b), x, gx)
    At = np.ascontiguousarray(s.A.T)
    yo = oracle.rkab(At, -xt.astype(np.float64), np.zeros(3000), q=4, alpha=50, rounds=6, seed=7,
                     tab=oracle.table(At), stream=1)
    assert_close(gb.cpu().numpy(), yo, TOL)


def test_adjoint_at_forward_point_matches_qr(rk, inc):
    """Converged y- and g-solves reproduce the FP64 adjoint evaluated at the GPU's x."""
    s, xt, A, plan = inc
    x, _ = rk.rkab_solve(plan, _dev(s.b), q=8, alpha=200, rounds=60, seed=3, check_every=0)
    cfg = rk.AdjointConfig(q=8, alpha_t=200, rounds_t=80, alpha=200, rounds=80, seed=5)
    gx = x - _dev(xt)
    gA, gb, g = rk.Adjoint(plan, cfg).backward(_dev(s.b), x, gx)
    rA, rb, rg = oracle.lstsq_adjoint(s.A, s.b, x.cpu().numpy(), xt)
    assert_close(gb.cpu().numpy(), rb, TOL)
    assert_close(g.cpu().numpy(), rg, TOL)
    assert_close(gA.cpu().numpy(), rA, TOL)


def test_min_norm_solve_column_split_matches_oracle(rk):
    """The y-solve on rows of A^T too long for one CTA (100 x 50000: 200 KB rows) runs RKA
    with x split by columns over the grid (the kernel of the timed adjoints): the same
    draws of stream 1 as the oracle, relaxation omega_t, every element within 1e-4."""
    s = rk_inputs.gaussian_system(50000, 100, seed=87, noise=1e-3)
    xt = rk_inputs.target_vector(100, seed=87)
    plan = rk.rk_setup(_dev(s.A))
    cfg = rk.AdjointConfig(q=4, alpha_t=1, q_t=32, rounds_t=12, omega_t=20.0, alpha=100, rounds=1, seed=7)
    adj = rk.Adjoint(plan, cfg)
    x = torch.zeros(100, device="cuda")
    _, gb, _ = adj.backward(_dev(s.b), x, _dev(xt) * -1.0)
    At = np.ascontiguousarray(s.A.T)
    yo = oracle.rkab(At, -xt.astype(np.float64), np.zeros(50000), q=32, alpha=1, rounds=12, seed=7,
                     tab=oracle.table(At), stream=1, omega=20.0)
    assert_close(gb.cpu().numpy(), yo, TOL)


def test_adjoint_column_split_at_forward_point_matches_qr(rk):
    """40000 x 48 (A^T rows of 160 KB: the column-split minimum-norm solve with alpha* of
    Eq. (best_alpha) from A's spectrum): the whole adjoint at the GPU's forward point against
    the FP64 QR adjoint evaluated there."""
    s = rk_inputs.gaussian_system(40000, 48, seed=89, noise=1e-3)
    xt = rk_inputs.target_vector(48, seed=89)
    plan = rk.rk_setup(_dev(s.A))
    x, _ = rk.rkab_solve(plan, _dev(s.b), q=8, alpha=48, rounds=80, seed=3, check_every=0)
    lmin, lmax, fro2 = oracle.spectrum(s.A)
    om = float(oracle.alpha_star(48, lmin / fro2, lmax / fro2))
    cfg = rk.AdjointConfig(q=8, alpha=48, rounds=80, alpha_t=1, q_t=48, rounds_t=150, omega_t=om, seed=5)
    gx = x - _dev(xt)
    gA, gb, g = rk.Adjoint(plan, cfg).backward(_dev(s.b), x, gx)
    rA, rb, rg = oracle.lstsq_adjoint(s.A, s.b, x.cpu().numpy(), xt)
    assert_close(gb.cpu().numpy(), rb, TOL)
    assert_close(g.cpu().numpy(), rg, TOL)
    assert_close(gA.cpu().numpy(), rA, TOL)


def test_autograd_matches_finite_differences(rk):
    """torch.autograd through the RKAB least-squares solve against central finite
    differences (step 1e-6, 32 random directions) of the FP64 map L(x_LS(A, b))."""
    s = rk_inputs.gaussian_system(4000, 100, seed=85, noise=1e-3)
    xt = rk_inputs.target_vector(100, seed=85)
    A = _dev(s.A).requires_grad_(True)
    b = _dev(s.b).requires_grad_(True)
    cfg = rk.AdjointConfig(q=16, alpha_t=100, rounds_t=200, alpha=100, rounds=200, seed=9)
    # decreasing relaxation brings the forward point inside the horizon of omega = 1
    x = rk.rkab_lstsq(A, b, q=16, alpha=100, seed=1, adjoint=cfg,
                      schedule=[(1.0, 100), (0.1, 100), (0.01, 300), (0.002, 800)])
    loss = 0.5 * ((x - _dev(xt)) ** 2).sum()
    gA, gb = torch.autograd.grad(loss, (A, b))
    x_ls = oracle.lstsq_qr(s.A, s.b)
    err_x = _rel(x.detach().cpu().numpy(), x_ls)
    A64, b64 = s.A.astype(np.float64), s.b.astype(np.float64)
    rng = np.random.default_rng(1)
    gA, gb = gA.cpu().numpy().astype(np.float64), gb.cpu().numpy().astype(np.float64)
    h = 1e-6
    worst = 0.0
    for _ in range(32):
        dA = rng.standard_normal(A64.shape)
        db = rng.standard_normal(b64.shape)
        fd = (oracle.lstsq_loss(A64 + h * dA, b64 + h * db, xt)
              - oracle.lstsq_loss(A64 - h * dA, b64 - h * db, xt)) / (2 * h)
        an = np.sum(gA * dA) + np.sum(gb * db)
        worst = max(worst, abs(fd - an) / abs(fd))
    assert err_x < 2e-6, err_x
    assert worst < TOL, (worst, err_x)
