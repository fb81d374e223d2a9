"""Python binding of the RK / RKA / RKAB C ABI (``include/rkab.h``).

Argument marshalling only: torch tensors provide device memory and the
current CUDA stream; every step of the method runs in the library's kernels.
Workspaces are allocated here with torch (the library never allocates).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import RkError, RkOpts, check

_DT = {"f32": _lib.RK_F32, "bf16": _lib.RK_BF16, "fp8": _lib.RK_FP8E4M3}
_ELEM = {"f32": 4, "bf16": 2, "fp8": 1}
_TORCH_DT = {"f32": torch.float32, "bf16": torch.bfloat16, "fp8": torch.uint8}


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def aligned_rows(A: torch.Tensor, elem: int = 4) -> torch.Tensor:
    """Copy of the (m, n) matrix A with rows padded to a multiple of 16 bytes
    (layout only; the padding columns are zero).  Returns A itself when its
    row stride already qualifies."""
    if A.stride(1) == 1 and (A.stride(0) * elem) % 16 == 0 and A.data_ptr() % 16 == 0:
        return A
    m, n = A.shape
    per = 16 // elem
    lda = (n + per - 1) // per * per
    out = torch.zeros((m, lda), dtype=A.dtype, device=A.device)
    out[:, :n] = A
    return out[:, :n]


class Plan:
    """Sampling tables of one matrix (``rk_setup``).  Keeps A, the row scales
    and the workspace alive as long as the plan lives."""

    def __init__(self, A: torch.Tensor, dtype: str = "f32", row_scale: torch.Tensor | None = None,
                 stream=None, workspace: torch.Tensor | None = None):
        L = _lib.load()
        if dtype not in _DT:
            raise ValueError(f"dtype must be one of {list(_DT)}")
        if A.dim() != 2 or not A.is_cuda or A.stride(1) != 1:
            raise ValueError("A must be a 2-D CUDA tensor with unit column stride")
        if A.dtype != _TORCH_DT[dtype]:
            raise ValueError(f"A must have dtype {_TORCH_DT[dtype]} for storage '{dtype}'")
        self.A = A
        self.dtype = dtype
        self.m, self.n = A.shape
        self.lda = A.stride(0)
        self.row_scale = row_scale
        self.device = A.device
        nbytes = L.rk_setup_workspace_bytes(self.m, self.n)
        if workspace is not None and workspace.numel() >= nbytes:
            self.ws = workspace
        else:
            self.ws = _workspace(nbytes, A.device)
        h = ctypes.c_void_p()
        check(L.rk_setup(_ptr(A), _DT[dtype], _ptr(row_scale), self.m, self.n, self.lda,
                         _ptr(self.ws), self.ws.numel(), _stream(stream), ctypes.byref(h)),
              "rk_setup")
        self._h = h

    @property
    def handle(self):
        return self._h

    def status(self, stream=None):
        """(T, L) of the law once the device-side build finished (synchronises)."""
        T = ctypes.c_uint64()
        Lx = ctypes.c_int32()
        check(_lib.load().rk_plan_status(self._h, _stream(stream), ctypes.byref(T),
                                         ctypes.byref(Lx)), "rk_plan_status")
        return int(T.value), int(Lx.value)

    def frobenius2(self, stream=None) -> float:
        """||A||_F^2 of the stored rows from the exact-integer law (rk_plan_frobenius2:
        T 2^L, each row weight truncated to the law's bits; about 1e-8 relative).
        Synchronises."""
        out = ctypes.c_double()
        check(_lib.load().rk_plan_frobenius2(self._h, _stream(stream), ctypes.byref(out)),
              "rk_plan_frobenius2")
        return float(out.value)

    def tables(self):
        """Device tensors K (int64 view of uint64), P, thr64, alias (int32 view), inv."""
        ptrs = [ctypes.c_void_p() for _ in range(5)]
        check(_lib.load().rk_plan_tables(self._h, *[ctypes.byref(p) for p in ptrs]),
              "rk_plan_tables")
        base = self.ws.data_ptr()
        m = self.m

        def view(p, nbytes, dt):
            off = p.value - base
            return self.ws[off: off + nbytes].view(dt)

        return {
            "K": view(ptrs[0], 8 * m, torch.int64),
            "P": view(ptrs[1], 8 * m, torch.int64),
            "thr64": view(ptrs[2], 8 * m, torch.int64),
            "alias": view(ptrs[3], 4 * m, torch.int32),
            "inv": view(ptrs[4], 4 * m, torch.float32),
        }

    def __del__(self):
        try:
            if getattr(self, "_h", None) and self._h.value:
                _lib.load().rk_plan_destroy(self._h)
                self._h = ctypes.c_void_p()
        except Exception:
            pass


def rk_setup(A: torch.Tensor, dtype: str = "f32", row_scale=None, stream=None,
             workspace=None) -> Plan:
    """Build the sampling tables of A; `workspace` (uint8 CUDA tensor) is reused when
    large enough, so repeated setups allocate nothing."""
    return Plan(A, dtype, row_scale, stream, workspace)


def rk_sample_indices(plan: Plan, seed: int, worker: int, t0: int, count: int,
                      stream_id: int = 0, stream=None, sampling="full", q: int = 1) -> torch.Tensor:
    """Row draws t0 .. t0+count-1 of one worker (uint32 values in an int32 tensor); with
    sampling 'blocks' or 'cyclic' the worker is one of q (rk_sample_indices_ex)."""
    out = torch.empty(max(count, 1), dtype=torch.int32, device=plan.device)
    mode = SAMPLING[sampling] if isinstance(sampling, str) else int(sampling)
    if mode == 0 and q == 1:
        check(_lib.load().rk_sample_indices(plan.handle, seed, worker, stream_id, t0, count,
                                            _ptr(out), _stream(stream)), "rk_sample_indices")
    else:
        check(_lib.load().rk_sample_indices_ex(plan.handle, seed, worker, q, stream_id, mode, t0,
                                               count, _ptr(out), _stream(stream)),
              "rk_sample_indices_ex")
    return out[:count]


@dataclass
class SolveInfo:
    status: int
    rounds_done: int
    last_metric: float


SAMPLING = {"full": 0, "blocks": 1, "cyclic": 2}


def make_opts(omega=1.0, check_every=1, tol=0.0, x_ref=None, round0=0, stream_id=0,
              same_stream=False, cluster_size=0, timeout_s=10.0, lookahead=0,
              sampling="full", row_weight=None, worker_weight=None) -> RkOpts:
    o = RkOpts()
    _lib.load().rk_opts_default(ctypes.byref(o))
    o.omega = float(omega)
    o.check_every = int(check_every)
    o.tol = float(tol)
    o.criterion = 1 if x_ref is not None else 0
    o.x_ref = None if x_ref is None else x_ref.data_ptr()
    o.round0 = int(round0)
    o.stream_id = int(stream_id)
    o.same_stream = int(bool(same_stream))
    o.cluster_size = int(cluster_size)
    o.timeout_s = float(timeout_s)
    o.lookahead = int(lookahead)
    o.sampling = SAMPLING[sampling] if isinstance(sampling, str) else int(sampling)
    o.row_weight = None if row_weight is None else row_weight.data_ptr()
    o.worker_weight = None if worker_weight is None else worker_weight.data_ptr()
    return o


class Solver:
    """Reusable solve workspace for one plan and worker count."""

    def __init__(self, plan: Plan, q: int):
        self.plan = plan
        self.q = int(q)
        nbytes = _lib.load().rk_solve_workspace_bytes(plan.handle, self.q)
        if nbytes == 0:
            raise RkError(_lib.RK_EINVAL, "rk_solve_workspace_bytes")
        self.ws = _workspace(nbytes, plan.device)

    def launch(self, b, x0, x, alpha, rounds, seed, opts: RkOpts, stream=None):
        """Enqueue one rkab_solve (asynchronous)."""
        check(_lib.load().rkab_solve(self.plan.handle, _ptr(b), _ptr(x0), _ptr(x), self.q,
                                     int(alpha), int(rounds), int(seed), ctypes.byref(opts),
                                     _ptr(self.ws), self.ws.numel(), _stream(stream)),
              "rkab_solve")

    def info(self, stream=None) -> SolveInfo:
        rd = ctypes.c_int64()
        lm = ctypes.c_double()
        st = _lib.load().rk_solve_status(_ptr(self.ws), _stream(stream), ctypes.byref(rd),
                                         ctypes.byref(lm))
        return SolveInfo(int(st), int(rd.value), float(lm.value))


def _vec(t, n, name):
    if t is None or not t.is_cuda or t.dtype != torch.float32 or t.numel() != n or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of {n} elements")
    return t


def rkab_solve(plan: Plan, b, x0=None, q: int = 1, alpha: int = 1, rounds: int = 1,
               seed: int = 0, *, omega=1.0, x_ref=None, tol=0.0, check_every=1, round0=0,
               stream_id=0, same_stream=False, timeout_s=10.0, lookahead=0, cluster_size=0,
               sampling="full", row_weight=None, worker_weight=None, out=None, solver=None,
               stream=None, raise_on_error=True):
    """RKAB solve (alpha projections per worker between averages); returns (x, info).
    sampling: 'full' (Eq. (prob_line)), 'blocks' (per-worker row blocks), 'cyclic';
    row_weight: optional per-row weights w_i (m floats on the device);
    worker_weight: optional per-worker weights (q floats on the device), e.g. the
    Partial Matrix alpha of `partial_alpha_star`."""
    b = _vec(b, plan.m, "b")
    if x0 is None:
        x0 = torch.zeros(plan.n, dtype=torch.float32, device=plan.device)
    x0 = _vec(x0, plan.n, "x0")
    x = out if out is not None else torch.empty(plan.n, dtype=torch.float32, device=plan.device)
    if x_ref is not None:
        x_ref = _vec(x_ref, plan.n, "x_ref")
    s = solver if solver is not None else Solver(plan, q)
    if row_weight is not None:
        row_weight = _vec(row_weight, plan.m, "row_weight")
    if worker_weight is not None:
        worker_weight = _vec(worker_weight, s.q, "worker_weight")
    opts = make_opts(omega, check_every, tol, x_ref, round0, stream_id, same_stream, cluster_size,
                     timeout_s, lookahead, sampling, row_weight, worker_weight)
    s.launch(b, x0, x, alpha, rounds, seed, opts, stream)
    info = s.info(stream)
    if raise_on_error and info.status != _lib.RK_OK:
        raise RkError(info.status, "rkab_solve (device)")
    return x, info


CRITERIA = {"residual": 2, "normal": 3}


def rkab_solve_residual(plan: Plan, b, x0=None, q: int = 1, alpha: int = 1, max_rounds: int = 100,
                        check_every: int = 1, tol: float = 1e-6, criterion="normal", seed: int = 0,
                        A32=None, stream=None, **opt_kw):
    """RKAB stopped by a residual criterion ('residual': ||r||/||b||; 'normal':
    ||A^T r||/(||A||_F ||r||)) checked every check_every rounds; returns (x, rounds, metric).
    A32: float32 rows of the system when the plan stores BF16/FP8 rows."""
    b = _vec(b, plan.m, "b")
    if x0 is None:
        x0 = torch.zeros(plan.n, dtype=torch.float32, device=plan.device)
    x0 = _vec(x0, plan.n, "x0")
    x = torch.empty(plan.n, dtype=torch.float32, device=plan.device)
    lib = _lib.load()
    ws = _workspace(lib.rk_solve_residual_workspace_bytes(plan.handle, q), plan.device)
    opts = make_opts(**opt_kw)
    done = ctypes.c_int64(0)
    metric = ctypes.c_double(-1.0)
    crit = CRITERIA[criterion] if isinstance(criterion, str) else int(criterion)
    check(lib.rkab_solve_residual(plan.handle, _ptr(A32), 0 if A32 is None else A32.stride(0),
                                  _ptr(b), _ptr(x0), _ptr(x), q, alpha, max_rounds, check_every,
                                  seed, ctypes.byref(opts), crit, float(tol), _ptr(ws), ws.numel(),
                                  _stream(stream), ctypes.byref(done), ctypes.byref(metric)),
          "rkab_solve_residual")
    return x, int(done.value), float(metric.value)


def rka_solve(plan: Plan, b, x0=None, q: int = 1, rounds: int = 1, seed: int = 0, **kw):
    """RKA (alpha = 1): Eq. (rka_uni_weights)."""
    return rkab_solve(plan, b, x0, q=q, alpha=1, rounds=rounds, seed=seed, **kw)


def quantize(A: torch.Tensor, dtype: str, stream=None):
    """Stored copy of the float32 rows of A: 'bf16' -> (bf16 tensor, None);
    'fp8' -> (uint8 e4m3 codes, float32 row scales).  Rows padded to 16 bytes."""
    if dtype not in ("bf16", "fp8"):
        raise ValueError("dtype must be 'bf16' or 'fp8'")
    if A.dtype != torch.float32 or A.stride(1) != 1 or not A.is_cuda:
        raise ValueError("A must be a float32 CUDA matrix with unit column stride")
    m, n = A.shape
    per = 16 // _ELEM[dtype]
    ldo = (n + per - 1) // per * per
    out = torch.empty((m, ldo), dtype=_TORCH_DT[dtype], device=A.device)
    scale = torch.empty(m, dtype=torch.float32, device=A.device) if dtype == "fp8" else None
    check(_lib.load().rk_quantize(_ptr(A), m, n, A.stride(0), _DT[dtype], _ptr(out), ldo,
                                  _ptr(scale), _stream(stream)), "rk_quantize")
    return out[:, :n], scale


@dataclass
class RefineInfo:
    outer_done: int
    last_metric: float


class Refiner:
    """Reusable workspace for rkab_refine on one stored-row plan and worker count."""

    def __init__(self, lowp: Plan, q: int):
        self.plan = lowp
        self.q = int(q)
        nbytes = _lib.load().rk_refine_workspace_bytes(lowp.handle, self.q)
        if nbytes == 0:
            raise RkError(_lib.RK_EINVAL, "rk_refine_workspace_bytes")
        self.ws = _workspace(nbytes, lowp.device)

    def run(self, A32, b, x0, x, alpha, inner_rounds, max_outer, seed, opts: RkOpts, stream=None):
        od = ctypes.c_int64()
        lm = ctypes.c_double()
        check(_lib.load().rkab_refine(self.plan.handle, _ptr(A32), A32.stride(0), _ptr(b), _ptr(x0),
                                      _ptr(x), self.q, int(alpha), int(inner_rounds),
                                      int(max_outer), int(seed), ctypes.byref(opts), _ptr(self.ws),
                                      self.ws.numel(), _stream(stream), ctypes.byref(od),
                                      ctypes.byref(lm)), "rkab_refine")
        return RefineInfo(int(od.value), float(lm.value))


def rkab_refine(lowp: Plan, A32: torch.Tensor, b, x0=None, q: int = 1, alpha: int = 1,
                inner_rounds: int = 1, max_outer: int = 1, seed: int = 0, *, omega=1.0,
                x_ref=None, tol=0.0, timeout_s=10.0, out=None, refiner=None, stream=None):
    """Iterative refinement: FP64-accumulated residual on the float32 master A32,
    RKAB correction on the stored rows of `lowp`; returns (x, RefineInfo)."""
    b = _vec(b, lowp.m, "b")
    if x0 is None:
        x0 = torch.zeros(lowp.n, dtype=torch.float32, device=lowp.device)
    x0 = _vec(x0, lowp.n, "x0")
    x = out if out is not None else torch.empty(lowp.n, dtype=torch.float32, device=lowp.device)
    if x_ref is not None:
        x_ref = _vec(x_ref, lowp.n, "x_ref")
    r = refiner if refiner is not None else Refiner(lowp, q)
    opts = make_opts(omega, 0, tol, x_ref, 0, 0, False, 0, timeout_s)
    info = r.run(A32, b, x0, x, alpha, inner_rounds, max_outer, seed, opts, stream)
    return x, info


class Residual:
    def __init__(self, m: int, n: int, device):
        nbytes = _lib.load().rk_residual_workspace_bytes(m, n)
        self.ws = _workspace(nbytes, device)
        self.m, self.n = m, n

    def launch(self, A, b, x, r=None, norms=None, want_atr=True, stream=None):
        check(_lib.load().rk_residual(_ptr(A), self.m, self.n, A.stride(0), _ptr(b), _ptr(x),
                                      _ptr(r), _ptr(norms), int(bool(want_atr)), _ptr(self.ws),
                                      self.ws.numel(), _stream(stream)), "rk_residual")


def rk_residual(A: torch.Tensor, b, x, want_atr=True, stream=None):
    """r = b - A x (float64), and [||r||, ||A^T r||] (float64, device)."""
    m, n = A.shape
    if A.dtype != torch.float32 or A.stride(1) != 1:
        raise ValueError("A must be float32 with unit column stride")
    b = _vec(b, m, "b")
    x = _vec(x, n, "x")
    r = torch.empty(m, dtype=torch.float64, device=A.device)
    norms = torch.zeros(2, dtype=torch.float64, device=A.device)
    Residual(m, n, A.device).launch(A, b, x, r, norms, want_atr, stream)
    return r, norms


# --------------------------------------------------------------------------
# Optimal uniform weight of RKA (Eq. (best_alpha))
# --------------------------------------------------------------------------
def alpha_star(q: int, s_min: float, s_max: float) -> float:
    """Eq. (best_alpha): optimal uniform weight of RKA with q workers."""
    a = float(_lib.load().rk_alpha_star(int(q), float(s_min), float(s_max)))
    if a <= 0.0:
        raise RkError(_lib.RK_EINVAL, "rk_alpha_star")
    return a


@dataclass
class Spectrum:
    lambda_min: float    # estimate of sigma_min(A)^2 (from above)
    lambda_max: float    # estimate of sigma_max(A)^2 (from below)
    fro2: float          # ||A||_F^2
    steps: int           # Lanczos steps taken
    s_min: float = 0.0   # sigma_min^2 / ||A||_F^2 of Eq. (best_alpha) (rk_spectrum_ratios)
    s_max: float = 0.0   # sigma_max^2 / ||A||_F^2


def _spectrum(out3, steps) -> Spectrum:
    """Spectrum of rk_spectrum's three doubles, the ratios of Eq. (best_alpha) from C."""
    arr = (ctypes.c_double * 3)(out3[0], out3[1], out3[2])
    lo, hi = ctypes.c_double(0.0), ctypes.c_double(0.0)
    check(_lib.load().rk_spectrum_ratios(arr, ctypes.byref(lo), ctypes.byref(hi)), "rk_spectrum_ratios")
    return Spectrum(out3[0], out3[1], out3[2], steps, lo.value, hi.value)


def spectrum(A: torch.Tensor, k: int = 32, seed: int = 0, stream=None, fro2=None) -> Spectrum:
    """Extreme squared singular values of A by k Lanczos steps, and ||A||_F^2 (rk_spectrum;
    rk_spectrum_ex with a known ||A||_F^2, e.g. `Plan.frobenius2()`, skips that pass)."""
    if A.dtype != torch.float32 or A.stride(1) != 1 or not A.is_cuda:
        raise ValueError("A must be a float32 CUDA matrix with unit column stride")
    m, n = A.shape
    lib = _lib.load()
    nbytes = lib.rk_spectrum_workspace_bytes(m, n, int(k))
    if nbytes == 0:
        raise RkError(_lib.RK_EINVAL, "rk_spectrum_workspace_bytes")
    ws = _workspace(nbytes, A.device)
    out = (ctypes.c_double * 3)()
    steps = ctypes.c_int(0)
    if fro2 is None:
        check(lib.rk_spectrum(_ptr(A), m, n, A.stride(0), int(k), int(seed), _ptr(ws), ws.numel(),
                              _stream(stream), out, ctypes.byref(steps)), "rk_spectrum")
    else:
        check(lib.rk_spectrum_ex(_ptr(A), m, n, A.stride(0), int(k), int(seed), float(fro2), _ptr(ws),
                                 ws.numel(), _stream(stream), out, ctypes.byref(steps)), "rk_spectrum_ex")
    return _spectrum(out, steps.value)


def optimal_weight(A: torch.Tensor, q: int, k: int = 32, seed: int = 0, stream=None, plan=None):
    """(alpha*, Spectrum): the weight of Eq. (best_alpha) for RKA with q workers on A
    (rk_optimal_weight); with the plan of A, ||A||_F^2 comes from its sampling law
    (rk_plan_frobenius2) instead of a pass over A."""
    if A.dtype != torch.float32 or A.stride(1) != 1 or not A.is_cuda:
        raise ValueError("A must be a float32 CUDA matrix with unit column stride")
    m, n = A.shape
    lib = _lib.load()
    nbytes = lib.rk_spectrum_workspace_bytes(m, n, int(k))
    if nbytes == 0:
        raise RkError(_lib.RK_EINVAL, "rk_spectrum_workspace_bytes")
    ws = _workspace(nbytes, A.device)
    fro2 = 0.0 if plan is None else plan.frobenius2(stream)
    a = ctypes.c_double(0.0)
    out = (ctypes.c_double * 5)()
    steps = ctypes.c_int(0)
    check(lib.rk_optimal_weight(_ptr(A), m, n, A.stride(0), int(q), int(k), int(seed), float(fro2),
                                _ptr(ws), ws.numel(), _stream(stream), ctypes.byref(a), out,
                                ctypes.byref(steps)), "rk_optimal_weight")
    return a.value, Spectrum(out[0], out[1], out[2], steps.value, out[3], out[4])


def partial_alpha_star(A: torch.Tensor, q: int, k: int = 8, seed: int = 0, stream=None):
    """The Partial Matrix alpha of Section 3.3.1 (rk_partial_alpha_star): for each worker g
    of q, alpha* of Eq. (best_alpha) from the spectrum of its own row block (the
    Distributed Approach's rows), each estimated by k Lanczos steps.  Returns
    (weights: q float32 on A's device, for `worker_weight`; list of Spectrum)."""
    if A.dtype != torch.float32 or A.stride(1) != 1 or not A.is_cuda:
        raise ValueError("A must be a float32 CUDA matrix with unit column stride")
    m, n = A.shape
    lib = _lib.load()
    nbytes = lib.rk_partial_alpha_workspace_bytes(m, n, int(q), int(k))
    if nbytes == 0:
        raise RkError(_lib.RK_EINVAL, "rk_partial_alpha_workspace_bytes")
    ws = _workspace(nbytes, A.device)
    w = (ctypes.c_float * int(q))()
    sp = (ctypes.c_double * (3 * int(q)))()
    check(lib.rk_partial_alpha_star(_ptr(A), m, n, A.stride(0), int(q), int(k), int(seed), _ptr(ws),
                                    ws.numel(), _stream(stream), w, sp), "rk_partial_alpha_star")
    weights = torch.tensor(list(w), dtype=torch.float32, device=A.device)
    return weights, [_spectrum(sp[3 * g: 3 * g + 3], 0) for g in range(int(q))]


def launch_count() -> int:
    """Kernel launches this process has enqueued through the library."""
    return int(_lib.load().rk_launch_count())


# --------------------------------------------------------------------------
# Differentiation form
# --------------------------------------------------------------------------
def transpose(A: torch.Tensor, stream=None) -> torch.Tensor:
    """A^T of a float32 CUDA matrix, rows padded to 16 bytes (returns an (n, m) view)."""
    if A.dtype != torch.float32 or A.stride(1) != 1 or not A.is_cuda:
        raise ValueError("A must be a float32 CUDA matrix with unit column stride")
    m, n = A.shape
    ldt = (m + 3) // 4 * 4
    At = torch.empty((n, ldt), dtype=torch.float32, device=A.device)
    if ldt > m:
        At[:, m:].zero_()
    check(_lib.load().rk_transpose(_ptr(A), m, n, A.stride(0), _ptr(At), ldt, _stream(stream)),
          "rk_transpose")
    return At[:, :m]


def rank2(r, g, y, x, out=None, stream=None) -> torch.Tensor:
    """G = r g^T - y x^T (float32, m x n)."""
    m, n = r.numel(), g.numel()
    ldg = (n + 3) // 4 * 4
    G = out if out is not None else torch.empty((m, ldg), dtype=torch.float32, device=r.device)[:, :n]
    check(_lib.load().rk_rank2(_ptr(r), _ptr(g), _ptr(y), _ptr(x), m, n, _ptr(G), G.stride(0),
                               _stream(stream)), "rk_rank2")
    return G


@dataclass
class AdjointConfig:
    """Parameters of the two solves of the backward pass."""
    q: int = 8                # workers of the solve of A g = y
    alpha_t: int = 0          # projections per worker per round on A^T (0: its row count n)
    rounds_t: int = 40
    alpha: int = 0            # projections per worker per round on A g = y (0: n)
    rounds: int = 40
    seed: int = 1
    cluster_size_t: int = 0   # CTAs per worker on A^T (long rows of length m)
    cluster_size: int = 0
    lookahead: int = 0
    q_t: int = 0              # workers of the solve on A^T (0: q)
    omega_t: float = 1.0      # relaxation of the solve on A^T
    omega: float = 1.0        # relaxation of the solve of A g = y
    check_every: int = 1      # rounds between the divergence checks of both solves


class Adjoint:
    """Plans of A and A^T and the workspace of rkab_adjoint."""

    def __init__(self, plan_A: Plan, cfg: AdjointConfig, stream=None):
        self.plan_A = plan_A
        self.cfg = cfg
        self.At = transpose(plan_A.A, stream)
        self.plan_At = Plan(self.At, "f32", None, stream)
        nbytes = _lib.load().rk_adjoint_workspace_bytes(plan_A.handle, self.plan_At.handle,
                                                        cfg.q_t or cfg.q, cfg.q)
        if nbytes == 0:
            raise RkError(_lib.RK_EINVAL, "rk_adjoint_workspace_bytes")
        self.ws = _workspace(nbytes, plan_A.device)

    def backward(self, b, x, gx, stream=None):
        """(grad_A, grad_b, g) at the point x for dL/dx = gx."""
        m, n = self.plan_A.m, self.plan_A.n
        c = self.cfg
        dev = self.plan_A.device
        grad_b = torch.empty(m, dtype=torch.float32, device=dev)
        g = torch.empty(n, dtype=torch.float32, device=dev)
        ldg = (n + 3) // 4 * 4
        grad_A = torch.empty((m, ldg), dtype=torch.float32, device=dev)[:, :n]
        # no criterion, but a diverging solve ends with RK_EDIVERGED at its next check
        ot = make_opts(omega=c.omega_t, check_every=c.check_every, cluster_size=c.cluster_size_t,
                       lookahead=c.lookahead)
        oa = make_opts(omega=c.omega, check_every=c.check_every, cluster_size=c.cluster_size,
                       lookahead=c.lookahead)
        check(_lib.load().rkab_adjoint(self.plan_A.handle, self.plan_At.handle, _ptr(b), _ptr(x),
                                       _ptr(gx), c.q_t or c.q, c.q, c.alpha_t or n, c.rounds_t,
                                       c.alpha or n,
                                       c.rounds, c.seed, ctypes.byref(ot), ctypes.byref(oa),
                                       _ptr(grad_b), _ptr(g), _ptr(grad_A), grad_A.stride(0),
                                       _ptr(self.ws), self.ws.numel(), _stream(stream)),
              "rkab_adjoint")
        return grad_A, grad_b, g


class RKABLstsq(torch.autograd.Function):
    """x = RKAB least-squares solve of A x ~ b (forward); backward by the adjoint:
    grad_b = y (minimum-norm Kaczmarz solution of A^T y = dL/dx from y = 0),
    grad_A = r g^T - y x^T with A g = y and r = b - A x."""

    @staticmethod
    def forward(ctx, A, b, q, alpha, schedule, seed, cluster_size, adj_cfg):
        plan = Plan(A.detach())
        bb = b.detach().contiguous()
        x = torch.zeros(plan.n, dtype=torch.float32, device=plan.device)
        round0 = 0
        # phases of decreasing relaxation continue one stream of draws; with
        # draws proportional to ||A_i||^2 the expected update is
        # omega/||A||_F^2 A^T (b - A x), zero at x_LS, and the spread around it
        # (the convergence horizon) shrinks with omega
        for omega, rounds in schedule:
            x, _ = rkab_solve(plan, bb, x, q=q, alpha=alpha, rounds=rounds, seed=seed,
                              omega=omega, round0=round0, check_every=0,
                              cluster_size=cluster_size)
            round0 += rounds
        ctx.plan = plan
        ctx.adj_cfg = adj_cfg
        ctx.save_for_backward(b, x)
        return x

    @staticmethod
    def backward(ctx, grad_x):
        b, x = ctx.saved_tensors
        adj = Adjoint(ctx.plan, ctx.adj_cfg)
        grad_A, grad_b, _ = adj.backward(b.detach().contiguous(), x.detach(),
                                         grad_x.detach().contiguous().to(torch.float32))
        return grad_A, grad_b, None, None, None, None, None, None


def rkab_lstsq(A, b, q=8, alpha=0, rounds=40, seed=0, cluster_size=0, adjoint=None,
               schedule=None):
    """Differentiable RKAB least-squares solve (see RKABLstsq).  `schedule` is a list of
    (omega, rounds) phases (default: [(1.0, rounds)])."""
    cfg = adjoint if adjoint is not None else AdjointConfig()
    sched = tuple(schedule) if schedule is not None else ((1.0, rounds),)
    return RKABLstsq.apply(A, b, q, alpha or A.shape[1], sched, seed, cluster_size, cfg)
