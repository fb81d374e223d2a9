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

import oracle
import rk_inputs
from _parity import assert_close

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


def test_noalloc_matches_oracle(env):
    """Independent of the path it mirrors: the allocation-free solve against the FP64
    oracle on the same draws (x within the parity tolerance, every element)."""
    rk, _lib, L, plan, b, xs = env
    s = rk_inputs.gaussian_system(6000, 300, seed=31)
    x0 = torch.zeros(300, device="cuda")
    for call in range(2):
        x = torch.full((300,), float("nan"), device="cuda")
        res = torch.zeros(24, dtype=torch.uint8, device="cuda")
        assert _noalloc(L, plan, b, x0, x, 6, 40, 5, 21, rk.make_opts(check_every=0), res) == 0
        torch.cuda.synchronize()
        assert _result(res).status == 0
        xo = oracle.rkab(s.A, s.b.astype(np.float64), np.zeros(300), q=6, alpha=40, rounds=5,
                         seed=21, tab=oracle.table(s.A))
        assert_close(x.cpu().numpy(), xo, TOL, what=f"call {call}")


@pytest.mark.parametrize("case", ["cluster2", "rka_spread", "rounds0"])
def test_noalloc_paths_match_workspace_solve(env, case):
    """The launch shapes rkab_solve offers, through the fixed array: 2-CTA cluster
    workers, RKA with the workers spread over one CTA per SM, and rounds = 0 (x = x0)."""
    rk, _lib, L, plan, b, xs = env
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    q, alpha, rounds, kw = {"cluster2": (3, 25, 4, {"cluster_size": 2}),
                            "rka_spread": (4 * sms + 3, 1, 6, {}),
                            "rounds0": (2, 5, 0, {})}[case]
    x0 = torch.randn(300, device="cuda")
    ref, info = rk.rkab_solve(plan, b, x0, q=q, alpha=alpha, rounds=rounds, seed=9,
                              check_every=0, **kw)
    for _ in range(2):
        x = torch.full((300,), float("nan"), device="cuda")
        res = torch.zeros(24, dtype=torch.uint8, device="cuda")
        rc = _noalloc(L, plan, b, x0, x, q, alpha, rounds, 9, rk.make_opts(check_every=0, **kw), res)
        assert rc == _lib.RK_OK, L.rk_strerror(rc).decode()
        torch.cuda.synchronize()
        r = _result(res)
        assert r.status == 0 and r.rounds_done == rounds
        if rounds == 0:
            assert torch.equal(x, x0)
        else:
            assert_close(x.cpu().numpy(), ref.cpu().numpy(), TOL, what=case)


def test_noalloc_result_in_pinned_host_memory(env):
    rk, _lib, L, plan, b, xs = env
    x0 = torch.zeros(300, device="cuda")
    ref, info = rk.rkab_solve(plan, b, x0, q=4, alpha=30, rounds=500, seed=5, x_ref=xs, tol=1e-5)
    res = torch.zeros(24, dtype=torch.uint8).pin_memory()
    x = torch.empty(300, device="cuda")
    assert _noalloc(L, plan, b, x0, x, 4, 30, 500, 5, rk.make_opts(x_ref=xs, tol=1e-5), res) == 0
    torch.cuda.synchronize()
    r = Result.from_buffer_copy(res.numpy().tobytes())
    assert r.status == 0 and r.rounds_done == info.rounds_done and 0 <= r.last_metric < 1e-5
    assert torch.equal(x, ref)


def test_noalloc_checks_options_like_rkab_solve(env):
    rk, _lib, L, plan, b, xs = env
    x0 = torch.zeros(300, device="cuda")
    x = torch.zeros(300, device="cuda")
    res = torch.zeros(24, dtype=torch.uint8, device="cuda")
    for kw in ({"cluster_size": 3}, {"cluster_size": 32}, {"lookahead": 3}, {"omega": 9.0}):
        assert _noalloc(L, plan, b, x0, x, 4, 10, 1, 0, rk.make_opts(**kw), res) == _lib.RK_EINVAL, kw
    torch.cuda.synchronize()
    assert torch.count_nonzero(x) == 0 and torch.count_nonzero(res) == 0


def test_noalloc_sizes_rka_by_the_rows_it_uses(env):
    """RKA with more workers than SMs keeps one row of displacements per SM, so it fits
    the array at sizes where RKAB with as many workers does not (10000 columns: 608 RKA
    workers fit, RKAB with 608 workers of alpha = 2 is refused)."""
    rk, _lib, L, _, _, _ = env
    A_t, b_t, _ = rk_inputs.gaussian_system_torch(3000, 10000, seed=6, device="cuda")
    big = rk.rk_setup(A_t)
    q = 4 * torch.cuda.get_device_properties(0).multi_processor_count
    x0 = torch.zeros(10000, device="cuda")
    ref, _ = rk.rka_solve(big, b_t, x0, q=q, rounds=3, seed=2, check_every=0)
    x = torch.full((10000,), float("nan"), device="cuda")
    res = torch.zeros(24, dtype=torch.uint8, device="cuda")
    assert _noalloc(L, big, b_t, x0, x, q, 1, 3, 2, rk.make_opts(check_every=0), res) == 0
    torch.cuda.synchronize()
    assert _result(res).status == 0
    assert_close(x.cpu().numpy(), ref.cpu().numpy(), TOL)
    assert _noalloc(L, big, b_t, x0, x, q, 2, 1, 2, rk.make_opts(), res) == _lib.RK_ETOOLARGE
