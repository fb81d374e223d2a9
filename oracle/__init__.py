"""FP64 CPU oracle for RK / RKA / RKAB (arXiv 2401.17474).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``, never by the product package.  It
shares no code with the CUDA library; the plain C in ``rk_oracle.c`` restates
the paper's definitions (each function there cites its passage) and this module
only marshals numpy arrays into it.  The least-squares references at the end
(QR via LAPACK, CGLS) are library routines or textbook iterations used as
independent checks.

Parity-pinning status of each function is recorded in the tests under
``tests/test_oracle_*.py``; every function here is pinned by at least one
check that does not re-use the oracle's own code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rk_oracle.c")
_LIB = os.path.join(_HERE, "librk_oracle.so")

_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile rk_oracle.c into librk_oracle.so with gcc (no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.orc_philox4x32_10.restype = None
        L.orc_row_weights.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                      _u64p, _u64p, _i32p]
        L.orc_alias_build.argtypes = [_u64p, ctypes.c_int64, ctypes.c_uint64, _u64p, _u32p]
        L.orc_sample_row.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                     ctypes.c_uint32, ctypes.c_int64, _u64p, _u32p]
        L.orc_sample_row.restype = ctypes.c_int64
        L.orc_sample_rows.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                      _u64p, _u32p, _i64p]
        L.orc_sample_rows.restype = None
        L.orc_row_norms.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _f64p]
        L.orc_row_norms.restype = None
        L.orc_rk.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _f64p,
                             _f64p, _f64p, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                             ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, _u64p, _u32p]
        L.orc_rka_formula.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                      _f64p, _f64p, _f64p, ctypes.c_int, ctypes.c_int64,
                                      ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                                      _u64p, _u32p]
        L.orc_rkab.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _f64p,
                               _f64p, _f64p, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                               ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                               _u64p, _u32p, ctypes.c_int, ctypes.c_int, _f64p, ctypes.c_double,
                               _i64p, _f64p]
        L.orc_rkab_ext.argtypes = L.orc_rkab.argtypes + [ctypes.c_int, _u64p, _f64p, _f64p]
        L.orc_select_row.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                     ctypes.c_int, ctypes.c_uint32, ctypes.c_int64, _u64p, _u32p,
                                     _u64p]
        L.orc_select_row.restype = ctypes.c_int64
        L.orc_select_rows.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                      ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64,
                                      ctypes.c_int64, _u64p, _u32p, _u64p, _i64p]
        L.orc_select_rows.restype = None
        L.orc_rkab_round_workers.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int64, _f64p, _f64p, _f64p, ctypes.c_int,
                                             ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                                             ctypes.c_uint32, ctypes.c_double, _u64p, _u32p]
        L.orc_residual.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _f64p,
                                   _f64p, _f64p, _f64p, _f64p]
        L.orc_bf16_rne.argtypes = [ctypes.c_float]
        L.orc_bf16_rne.restype = ctypes.c_uint16
        L.orc_fp8e4m3_rne.argtypes = [ctypes.c_float]
        L.orc_fp8e4m3_rne.restype = ctypes.c_uint8
        L.orc_fp8e4m3_value.argtypes = [ctypes.c_uint8]
        L.orc_fp8e4m3_value.restype = ctypes.c_double
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def _mat(A):
    A = np.asarray(A)
    if A.dtype != np.float32 or A.ndim != 2:
        raise TypeError("A must be a 2-D float32 array")
    if A.strides[1] != 4:
        A = np.ascontiguousarray(A)
    m, n = A.shape
    lda = A.strides[0] // 4
    return A, m, n, lda


# --------------------------------------------------------------------------
# Philox4x32-10 and the sampling law
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c, _u32p), _p(k, _u32p), _p(out, _u32p))
    return out


@dataclass
class Table:
    """Integer sampling law (K, T, L) and its alias table (thr64, alias)."""
    K: np.ndarray
    T: int
    L: int
    thr64: np.ndarray
    alias: np.ndarray

    @property
    def m(self):
        return int(self.K.shape[0])


def row_weights(A):
    A, m, n, lda = _mat(A)
    K = np.zeros(m, np.uint64)
    T = ctypes.c_uint64(0)
    L = ctypes.c_int32(0)
    _check(lib().orc_row_weights(_p(A, _f32p), m, n, lda, _p(K, _u64p), ctypes.byref(T),
                                 ctypes.byref(L)), "row_weights")
    return K, int(T.value), int(L.value)


def alias_build(K, T):
    K = np.ascontiguousarray(K, dtype=np.uint64)
    m = K.shape[0]
    thr = np.zeros(m, np.uint64)
    al = np.zeros(m, np.uint32)
    _check(lib().orc_alias_build(_p(K, _u64p), m, int(T), _p(thr, _u64p), _p(al, _u32p)),
           "alias_build")
    return thr, al


def table(A) -> Table:
    K, T, L = row_weights(A)
    thr, al = alias_build(K, T)
    return Table(K, T, L, thr, al)


SAMPLING = {"full": 0, "blocks": 1, "cyclic": 2}


def sample_rows(tab: Table, seed: int, worker: int, t0: int, count: int, stream: int = 0,
                sampling="full", q: int = 1):
    """Row choices t0 .. t0+count-1 of worker `worker` of q under a row selection
    ('full': the law of Eq. (prob_line); 'blocks': the worker's row block; 'cyclic')."""
    out = np.zeros(count, np.int64)
    mode = SAMPLING[sampling] if isinstance(sampling, str) else int(sampling)
    if mode == 0 and q == 1:
        lib().orc_sample_rows(seed, worker, stream, t0, count, tab.m, _p(tab.thr64, _u64p),
                              _p(tab.alias, _u32p), _p(out, _i64p))
    else:
        K = np.ascontiguousarray(tab.K, np.uint64)
        lib().orc_select_rows(mode, seed, worker, q, stream, t0, count, tab.m,
                              _p(tab.thr64, _u64p), _p(tab.alias, _u32p), _p(K, _u64p),
                              _p(out, _i64p))
    return out


# --------------------------------------------------------------------------
# Iterations
# --------------------------------------------------------------------------
def _vec64(v, n):
    v = np.ascontiguousarray(v, dtype=np.float64)
    if v.shape != (n,):
        raise ValueError("bad vector shape")
    return v


def row_norms(A):
    A, m, n, lda = _mat(A)
    w = np.zeros(m, np.float64)
    lib().orc_row_norms(_p(A, _f32p), m, n, lda, _p(w, _f64p))
    return w


def rk(A, b, x0, iters, seed, tab: Table, worker=0, t0=0, stream=0, omega=1.0):
    A, m, n, lda = _mat(A)
    b = _vec64(b, m)
    x0 = _vec64(x0, n)
    x = np.zeros(n, np.float64)
    _check(lib().orc_rk(_p(A, _f32p), m, n, lda, _p(b, _f64p), _p(x0, _f64p), _p(x, _f64p),
                        iters, t0, seed, worker, stream, omega, _p(tab.thr64, _u64p),
                        _p(tab.alias, _u32p)), "rk")
    return x


def rka_formula(A, b, x0, q, iters, seed, tab: Table, stream=0, omega=1.0):
    A, m, n, lda = _mat(A)
    b = _vec64(b, m)
    x0 = _vec64(x0, n)
    x = np.zeros(n, np.float64)
    _check(lib().orc_rka_formula(_p(A, _f32p), m, n, lda, _p(b, _f64p), _p(x0, _f64p),
                                 _p(x, _f64p), q, iters, seed, stream, omega,
                                 _p(tab.thr64, _u64p), _p(tab.alias, _u32p)), "rka_formula")
    return x


def rkab(A, b, x0, q, alpha, rounds, seed, tab: Table, round0=0, stream=0, omega=1.0,
         same_stream=False, threads=1, x_ref=None, tol=0.0, want_trace=False, sampling="full",
         row_weight=None, worker_weight=None):
    """RKAB rounds; returns x (and rounds done, trace of rel. errors if x_ref given).
    sampling: row selection ('full', 'blocks', 'cyclic'); row_weight: w_i of Eq. (rka_eq);
    worker_weight: q per-worker weights (the Partial Matrix alpha of Section 3.3.1)."""
    A, m, n, lda = _mat(A)
    b = _vec64(b, m)
    x0 = _vec64(x0, n)
    x = np.zeros(n, np.float64)
    done = ctypes.c_int64(0)
    xr = None if x_ref is None else _vec64(x_ref, n)
    trace = np.full(max(rounds, 1), np.nan) if (want_trace and xr is not None) else None
    mode = SAMPLING[sampling] if isinstance(sampling, str) else int(sampling)
    K = np.ascontiguousarray(tab.K, np.uint64)
    wv = None if row_weight is None else _vec64(row_weight, m)
    uv = None if worker_weight is None else _vec64(worker_weight, q)
    _check(lib().orc_rkab_ext(_p(A, _f32p), m, n, lda, _p(b, _f64p), _p(x0, _f64p), _p(x, _f64p),
                              q, alpha, rounds, round0, seed, stream, omega, _p(tab.thr64, _u64p),
                              _p(tab.alias, _u32p), int(bool(same_stream)), threads,
                              None if xr is None else _p(xr, _f64p), tol, ctypes.byref(done),
                              None if trace is None else _p(trace, _f64p), mode, _p(K, _u64p),
                              None if wv is None else _p(wv, _f64p),
                              None if uv is None else _p(uv, _f64p)), "rkab")
    if want_trace:
        return x, int(done.value), trace[: int(done.value)]
    if xr is not None:
        return x, int(done.value)
    return x


def rkab_round_workers(A, b, x, q, alpha, rnd, seed, tab: Table, stream=0, omega=1.0):
    A, m, n, lda = _mat(A)
    b = _vec64(b, m)
    x = _vec64(x, n)
    V = np.zeros((q, n), np.float64)
    _check(lib().orc_rkab_round_workers(_p(A, _f32p), m, n, lda, _p(b, _f64p), _p(x, _f64p),
                                        _p(V, _f64p), q, alpha, rnd, seed, stream, omega,
                                        _p(tab.thr64, _u64p), _p(tab.alias, _u32p)),
           "rkab_round_workers")
    return V


def residual(A, b, x):
    A, m, n, lda = _mat(A)
    b = _vec64(b, m)
    x = _vec64(x, n)
    r = np.zeros(m, np.float64)
    rn = ctypes.c_double(0)
    an = ctypes.c_double(0)
    _check(lib().orc_residual(_p(A, _f32p), m, n, lda, _p(b, _f64p), _p(x, _f64p),
                              _p(r, _f64p), ctypes.byref(rn), ctypes.byref(an)), "residual")
    return r, float(rn.value), float(an.value)


# --------------------------------------------------------------------------
# Stored-row precisions
# --------------------------------------------------------------------------
def bf16_rne(a):
    a = np.ascontiguousarray(a, dtype=np.float32).ravel()
    f = lib().orc_bf16_rne
    return np.array([f(float(v)) for v in a], dtype=np.uint16)


def bf16_values(codes):
    return (np.asarray(codes, np.uint32) << 16).astype(np.uint32).view(np.float32)


def fp8e4m3_rne(a):
    a = np.ascontiguousarray(a, dtype=np.float32).ravel()
    f = lib().orc_fp8e4m3_rne
    return np.array([f(float(v)) for v in a], dtype=np.uint8)


def fp8e4m3_values(codes):
    f = lib().orc_fp8e4m3_value
    table_ = np.array([f(c) for c in range(256)], dtype=np.float64)
    return table_[np.asarray(codes, np.uint8)]


def fp8_row_scales(A):
    """Per-row scale s_i = amax_i / 448 in FP32 (1 for an all-zero row)."""
    A = np.asarray(A, np.float32)
    amax = np.max(np.abs(A), axis=1).astype(np.float32)
    s = (amax / np.float32(448.0)).astype(np.float32)
    s[amax == 0] = np.float32(1.0)
    return s


def quantize_bf16(A):
    """(uint16 codes, float32 values) of the BF16 copy of A (round-to-nearest-even)."""
    A = np.ascontiguousarray(A, np.float32)
    codes = bf16_rne(A).reshape(A.shape)
    return codes, bf16_values(codes).reshape(A.shape)


def quantize_fp8(A):
    """(uint8 e4m3 codes, float32 row scales, float32 stored values fl32(s_i q_ij)):
    s_i = amax_i / 448 in float32, q_ij = e4m3 round-to-nearest-even of a_ij / s_i
    (float32 division), saturating."""
    A = np.ascontiguousarray(A, np.float32)
    s = fp8_row_scales(A)
    ratio = (A / s[:, None]).astype(np.float32)
    codes = fp8e4m3_rne(ratio).reshape(A.shape)
    vals = fp8e4m3_values(codes).astype(np.float32)
    stored = (vals * s[:, None]).astype(np.float32)
    return codes, s, stored


def refine(A32, A_low, b, x0, q, alpha, inner_rounds, outer, seed, tab_low, omega=1.0):
    """Iterative refinement of A32 x = b: for each outer step o, r = b - A32 x (FP64),
    d = RKAB on the stored rows A_low for A_low d = r from d = 0 (Philox stream id
    3 + (o << 8)), x = x + d.  Returns the iterates after each step."""
    x = np.array(x0, np.float64)
    xs = []
    for o in range(outer):
        r, _, _ = residual(A32, b, x)
        d = rkab(A_low, r, np.zeros(x.shape[0]), q=q, alpha=alpha, rounds=inner_rounds, seed=seed,
                 tab=tab_low, stream=3 + (o << 8), omega=omega)
        x = x + d
        xs.append(x.copy())
    return xs


# --------------------------------------------------------------------------
# Least-squares references (library QR, textbook CGLS)
# --------------------------------------------------------------------------
def lstsq_qr(A, b):
    """x_LS of Eq. (ls_system) by Householder QR in FP64 (LAPACK via numpy)."""
    A64 = np.asarray(A, np.float64)
    Q, R = np.linalg.qr(A64, mode="reduced")
    return np.linalg.solve(R, Q.T @ np.asarray(b, np.float64))


def lstsq_adjoint(A, b, x, x_t):
    """FP64 adjoint of x_LS(A, b) for L = 0.5 ||x - x_t||^2, evaluated at the point x:
    g = (A^T A)^{-1} (x - x_t) through the QR factor (R^T R = A^T A), y = A g,
    r = b - A x; returns (grad_A = r g^T - y x^T, grad_b = y, g)."""
    A64 = np.asarray(A, np.float64)
    x = np.asarray(x, np.float64)
    gx = x - np.asarray(x_t, np.float64)
    _, R = np.linalg.qr(A64, mode="reduced")
    g = np.linalg.solve(R, np.linalg.solve(R.T, gx))
    y = A64 @ g
    r = np.asarray(b, np.float64) - A64 @ x
    return np.outer(r, g) - np.outer(y, x), y, g


def lstsq_loss(A, b, x_t):
    """L(A, b) = 0.5 ||x_LS(A, b) - x_t||^2 in FP64 (QR)."""
    x = lstsq_qr(A, b)
    return 0.5 * float(np.sum((x - np.asarray(x_t, np.float64)) ** 2))


def cgls(A, b, x0=None, tol=1e-14, maxiter=10000):
    """Conjugate gradients on the normal equations (CGLS), FP64; the solver the
    paper names for x_LS of its inconsistent data set (Section 3.1)."""
    A64 = np.asarray(A, np.float64)
    b64 = np.asarray(b, np.float64)
    n = A64.shape[1]
    x = np.zeros(n) if x0 is None else np.array(x0, np.float64)
    r = b64 - A64 @ x
    s = A64.T @ r
    p = s.copy()
    gamma = s @ s
    g0 = gamma
    for _ in range(maxiter):
        if gamma <= (tol ** 2) * g0 or gamma == 0.0:
            break
        qv = A64 @ p
        a = gamma / (qv @ qv)
        x += a * p
        r -= a * qv
        s = A64.T @ r
        gnew = s @ s
        p = s + (gnew / gamma) * p
        gamma = gnew
    return x


# --------------------------------------------------------------------------
# Optimal uniform weight of RKA (Eq. (best_alpha)) and the spectrum it needs
# --------------------------------------------------------------------------
def spectrum(A):
    """(sigma_min^2, sigma_max^2, ||A||_F^2) of A in FP64: singular values by LAPACK's
    SVD (numpy), the Frobenius norm as the plain sum of squares."""
    A64 = np.asarray(A, np.float64)
    sv = np.linalg.svd(A64, compute_uv=False)
    return float(sv[-1] ** 2), float(sv[0] ** 2), float(np.sum(A64 * A64))


def block_bounds(m, q, g):
    """Rows [lo, hi) of worker g's block in the Distributed Approach (Section 3.3.1):
    lo = floor(g m / q), hi = floor((g + 1) m / q)."""
    return (g * m) // q, ((g + 1) * m) // q


def partial_alpha_star(A, q):
    """The Partial Matrix alpha of Section 3.3.1 (Table 1): for each worker g, Eq.
    (best_alpha) with q workers and s_min, s_max of its own block A_g (the Distributed
    Approach's rows), s = sigma^2(A_g) / ||A_g||_F^2 over the min(m_g, n) singular values
    of A_g (LAPACK SVD through `spectrum`).  Returns (alphas (q,), spectra (q, 3))."""
    A = np.asarray(A)
    m = A.shape[0]
    if not 1 <= q <= m:
        raise ValueError("1 <= q <= m")
    al = np.zeros(q)
    sp = np.zeros((q, 3))
    for g in range(q):
        lo, hi = block_bounds(m, q, g)
        sp[g] = spectrum(A[lo:hi])
        al[g] = alpha_star(q, sp[g, 0] / sp[g, 2], sp[g, 1] / sp[g, 2])
    return al, sp


def alpha_star(q, s_min, s_max):
    """Eq. (best_alpha): the optimal uniform row weight alpha of RKA (Eq. (rka_eq) with
    w_i = alpha) for a consistent system, from s_min = sigma_min^2 / ||A||_F^2 and
    s_max = sigma_max^2 / ||A||_F^2.  The first branch holds when the spread
    s_max - s_min is at most 1 / (q - 1) (always for q = 1, where it gives 1)."""
    q = int(q)
    if q < 1:
        raise ValueError("q >= 1")
    if q == 1 or s_max - s_min <= 1.0 / (q - 1):
        return q / (1.0 + (q - 1) * s_min)
    return 2.0 * q / (1.0 + (q - 1) * (s_min + s_max))
