"""The C-ABI library builds, loads, and exports every function the public
header declares; the Python binding declares exactly those.  No device work."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rkab.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b([a-z_][a-z0-9_]*)\s*\([^;{]*\)\s*;", text)
    return sorted(set(n for n in names if n.startswith(("rk", "rka", "rkab"))))


@pytest.fixture(scope="module")
def lib():
    from paper_2401_17474_gb300 import build
    path = build.build()
    return ctypes.CDLL(path), path


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("rk_setup", "rka_solve", "rkab_solve", "rk_residual", "rk_sample_indices",
                 "rk_setup_workspace_bytes", "rk_solve_workspace_bytes", "rk_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    L, path = lib
    for name in _declared():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True)
    exported = set(re.findall(r"\s[TW]\s+(\S+)$", out.stdout, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_declares_exactly_the_header(lib):
    from paper_2401_17474_gb300 import _lib
    assert sorted(_lib.declared_functions()) == _declared()


def test_host_side_queries_need_no_device(lib):
    from paper_2401_17474_gb300 import _lib
    L = _lib.load()
    assert L.rk_setup_workspace_bytes(1000, 10) > 1000 * 32
    assert L.rk_setup_workspace_bytes(0, 10) == 0
    assert L.rk_strerror(-4) == b"device-side wait exceeded its time limit"
    o = _lib.RkOpts()
    L.rk_opts_default(ctypes.byref(o))
    assert o.omega == 1.0 and o.check_every == 1 and o.timeout_s == 10.0
    # argument checks fail before any device work
    h = ctypes.c_void_p()
    assert L.rk_setup(None, 0, None, 10, 10, 10, None, 0, None, ctypes.byref(h)) == _lib.RK_EINVAL
    assert L.rk_setup(ctypes.c_void_p(16), 0, None, 10, 10, 12, ctypes.c_void_p(256), 0, None,
                      ctypes.byref(h)) == _lib.RK_EWORKSPACE
    assert L.rk_setup(ctypes.c_void_p(16), 0, None, 10, 10, 10, ctypes.c_void_p(256), 1 << 30, None,
                      ctypes.byref(h)) == _lib.RK_EALIGN      # lda*4 = 40 not a multiple of 16
    assert L.rkab_solve(None, None, None, None, 1, 1, 1, 0, None, None, 0, None) == _lib.RK_EINVAL


def test_alpha_star_is_the_oracle_formula(lib):
    """rk_alpha_star (host arithmetic in the library) reproduces Eq. (best_alpha) as the
    oracle writes it, on both branches, bit for bit."""
    import oracle
    from paper_2401_17474_gb300 import _lib
    L = _lib.load()
    cases = [(1, 0.2, 0.4), (2, 5e-4, 5e-4), (4, 6.7e-4, 2e-3), (132, 4.19e-5, 1.83e-4),
             (8, 0.01, 0.5), (64, 0.001, 0.9), (3, 0.0, 1.0)]
    for q, s0, s1 in cases:
        assert L.rk_alpha_star(q, s0, s1) == oracle.alpha_star(q, s0, s1), (q, s0, s1)
    # invalid arguments give 0
    assert L.rk_alpha_star(0, 0.1, 0.2) == 0.0
    assert L.rk_alpha_star(4, -0.1, 0.2) == 0.0
    assert L.rk_alpha_star(4, 0.1, 1.5) == 0.0
    # spectrum workspace query: host only
    assert L.rk_spectrum_workspace_bytes(1000, 100, 32) > 33 * 100 * 8
    assert L.rk_spectrum_workspace_bytes(1000, 100, 0) == 0
    assert L.rk_spectrum_workspace_bytes(1000, 100, 513) == 0


def test_header_is_plain_c(tmp_path):
    """The boundary header compiles as C99 and C++ (no torch or CUDA types), and a C
    caller links against the library's exported symbols."""
    src = tmp_path / "caller.c"
    src.write_text('#include "rkab.h"\n'
                   'int main(void) {\n'
                   '    rk_opts o; rk_opts_default(&o);\n'
                   '    return (int)(rk_setup_workspace_bytes(10, 4) == 0) + (o.omega != 1.0f)\n'
                   '           + (rk_alpha_star(1, 0.1, 0.2) != 1.0);\n'
                   '}\n')
    inc = os.path.join(ROOT, "include")
    for cc, std in (("gcc", "-std=c99"), ("g++", "-std=c++17")):
        r = subprocess.run([cc, std, "-Wall", "-Wextra", "-Werror", "-I", inc, "-fsyntax-only",
                            "-x", "c" if cc == "gcc" else "c++", str(src)],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
    from paper_2401_17474_gb300 import build
    lib = build.build()
    exe = tmp_path / "caller"
    r = subprocess.run(["gcc", "-std=c99", "-I", inc, str(src), lib, "-o", str(exe),
                        "-Wl,-rpath," + os.path.dirname(lib)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stderr)
