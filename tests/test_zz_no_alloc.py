"""rkab_solve_noalloc: the solve for callers that cannot allocate device
memory (a plugin hosted by a runtime that owns all device allocations, a
real-time loop that forbids allocation after start-up).  Its scratch is one
fixed device array inside the library; the call must give the same x as
rkab_solve with a caller workspace, on consecutive calls that reuse the
array, and must refuse a q x n that does not fit before doing any work.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

import rk_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4   # the parity tolerance of the other GPU tests (FP32 kernel)


class Result(ctypes.Structure):
    """Mirror of rk_solve_result."""
    _fields_ = [("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("rounds_done", ctypes.c_int64), ("last_metric", ctypes.c_double)]


@pytest.fixture(scope="module")
def env():
    import paper_2401_17474_gb300 as rk
    from paper_2401_17474_gb300 import _lib, build
    build.build()
    L = _lib.load()
    s = rk_inputs.gaussian_system(6000, 300, seed=31)
    A = torch.from_numpy(s.A).cuda()
    b = torch.from_numpy(s.b).cuda()
    xs = torch.from_numpy(s.x_star).cuda()
    plan = rk.rk_setup(A)
    plan.status()
    return rk, _lib, L, plan, b, xs


def _noalloc(L, plan, b, x0, x, q, alpha, rounds, seed, opts, res):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.rkab_solve_noalloc(plan.handle, ctypes.c_void_p(b.data_ptr()),
                                ctypes.c_void_p(x0.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                q, alpha, rounds, seed, ctypes.byref(opts),
                                ctypes.c_void_p(res.data_ptr()), stream)


def _result(res):
    return Result.from_buffer_copy(res.cpu().numpy().tobytes())


def test_noalloc_matches_workspace_solve_twice(env):
    rk, _lib, L, plan, b, xs = env
    x0 = torch.zeros(300, device="cuda")
    for call, (q, alpha, rounds, seed) in enumerate([(8, 50, 6, 11), (5, 30, 9, 12)]):
        ref, info = rk.rkab_solve(plan, b, x0, q=q, alpha=alpha, rounds=rounds, seed=seed)
        x = torch.full((300,), float("nan"), device="cuda")
        res = torch.zeros(24, dtype=torch.uint8, device="cuda")
        rc = _noalloc(L, plan, b, x0, x, q, alpha, rounds, seed, rk.make_opts(), res)
        assert rc == _lib.RK_OK, f"call {call}: {L.rk_strerror(rc).decode()}"
        torch.cuda.synchronize()
        r = _result(res)
        assert r.status == _lib.RK_OK and r.rounds_done == rounds == info.rounds_done
        xr = ref.cpu().numpy().astype(np.float64)
        rel = np.linalg.norm(x.cpu().numpy() - xr) / np.linalg.norm(xr)
        assert rel < TOL, (call, rel)


def test_noalloc_stop_rule_reports_through_result(env):
    rk, _lib, L, plan, b, xs = env
    x0 = torch.zeros(300, device="cuda")
    ref, info = rk.rkab_solve(plan, b, x0, q=8, alpha=300, rounds=500, seed=3, x_ref=xs, tol=1e-5)
    for _ in range(2):
        x = torch.empty(300, device="cuda")
        res = torch.zeros(24, dtype=torch.uint8, device="cuda")
        rc = _noalloc(L, plan, b, x0, x, 8, 300, 500, 3, rk.make_opts(x_ref=xs, tol=1e-5), res)
        assert rc == _lib.RK_OK
        torch.cuda.synchronize()
        r = _result(res)
        assert r.status == 0 and r.rounds_done == info.rounds_done and r.last_metric < 1e-5
        xr = ref.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(x.cpu().numpy() - xr) / np.linalg.norm(xr) < TOL


def test_noalloc_refuses_what_does_not_fit(env):
    rk, _lib, L, _, _, _ = env
    import rk_inputs
    A_t, b_t, _ = rk_inputs.gaussian_system_torch(600, 8000, seed=2, device="cuda")
    big = rk.rk_setup(A_t)
    x0 = torch.zeros(8000, device="cuda")
    x = torch.zeros(8000, device="cuda")
    res = torch.zeros(24, dtype=torch.uint8, device="cuda")
    # 300 workers of 8000 columns: (300 + 1) * 8000 floats exceed 8 MiB: refused before
    # any device work
    rc = _noalloc(L, big, b_t, x0, x, 300, 2, 1, 0, rk.make_opts(), res)
    assert rc == _lib.RK_ETOOLARGE
    assert "fixed scratch" in L.rk_strerror(rc).decode()
    assert torch.count_nonzero(x) == 0 and torch.count_nonzero(res) == 0
