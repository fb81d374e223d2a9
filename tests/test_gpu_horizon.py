"""The convergence horizon of RKA on an inconsistent system (Section 3.5): the error
to the least-squares solution and the residual logged every K rounds along GPU runs
(stretches of one draw stream, round0 advancing), each logged x against the FP64
oracle's x at the same round, and the plateau error falling with the worker count
q in {1, 2, 20, 50} as the paper's figures show (about as 1/sqrt(q))."""
import numpy as np
import pytest

import oracle
import rk_inputs
from _parity import assert_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4
K = 100          # rounds between logged points
STRETCHES = 30   # 3000 rounds in all


@pytest.fixture(scope="module")
def rk():
    import paper_2401_17474_gb300 as rk_
    from paper_2401_17474_gb300 import build
    build.build()
    return rk_


@pytest.fixture(scope="module")
def system(rk):
    # 4000 x 100, A and x* N(0,1), b = A x* + N(0, 1) (the paper's noisy systems)
    s = rk_inputs.gaussian_system(4000, 100, seed=91, noise=1.0)
    A = torch.from_numpy(s.A).cuda()
    return s, A, torch.from_numpy(s.b).cuda(), rk.rk_setup(A), oracle.table(s.A), \
        oracle.lstsq_qr(s.A, s.b)


def _trace(rk, system, q):
    s, A, b, plan, tab, x_ls = system
    b64 = s.b.astype(np.float64)
    x = torch.zeros(100, device="cuda")
    xo = np.zeros(100)
    err, res, res_o = [], [], []
    for k in range(STRETCHES):
        x, info = rk.rka_solve(plan, b, x.clone(), q=q, rounds=K, seed=3, round0=k * K,
                               check_every=0)
        assert info.status == 0 and info.rounds_done == K
        xo = oracle.rkab(s.A, b64, xo, q=q, alpha=1, rounds=K, seed=3, tab=tab, round0=k * K)
        xg = x.cpu().numpy().astype(np.float64)
        assert_close(xg, xo, TOL, what=f"q={q} round {(k + 1) * K}")
        _, norms = rk.rk_residual(A, b, x, want_atr=False)
        res.append(float(norms[0]))
        res_o.append(oracle.residual(s.A, s.b, xo)[1])
        err.append(np.linalg.norm(xg - x_ls))
    return np.array(err), np.array(res), np.array(res_o)


def test_horizon_shrinks_with_workers(rk, system):
    s, A, b, plan, tab, x_ls = system
    r_ls = oracle.residual(s.A, s.b, x_ls)[1]
    plateau, plateau_res = {}, {}
    for q in (1, 2, 20, 50):
        err, res, res_o = _trace(rk, system, q)
        np.testing.assert_allclose(res, res_o, rtol=TOL)
        assert np.all(res >= r_ls * (1 - 1e-12))      # x_LS minimises the residual
        plateau[q] = err[STRETCHES // 2:].mean()        # after the curves flatten
        plateau_res[q] = res[STRETCHES // 2:].mean() / r_ls
    assert plateau[1] > plateau[2] > plateau[20] > plateau[50], plateau
    assert plateau[50] < 0.2 * plateau[1], plateau       # about 1/sqrt(q)
    assert plateau_res[1] > plateau_res[20] > plateau_res[50] > 1.0, plateau_res
