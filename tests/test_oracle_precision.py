"""Pins of the oracle's stored-row quantisers against library conversions
(torch's BF16 and FP8 e4m3fn casts, run at test time)."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")


def _values():
    rng = np.random.default_rng(0)
    v = np.concatenate([
        rng.standard_normal(3000).astype(np.float32),
        (rng.standard_normal(1000) * 1e-30).astype(np.float32),
        (rng.standard_normal(1000) * 1e30).astype(np.float32),
        np.array([0.0, -0.0, 1.0, -1.0, 1.00390625, 1.01171875, 3.4e38, 1e-45, -1e-45],
                 np.float32),
    ])
    # exact ties between two bf16 neighbours
    ties = (np.arange(1, 200, dtype=np.uint32) << 16 | 0x8000).view(np.float32)
    return np.concatenate([v, ties])


def test_bf16_matches_torch():
    v = _values()
    ours = oracle.bf16_rne(v)
    ref = torch.from_numpy(v).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, ref)


def test_fp8_matches_torch_in_range():
    rng = np.random.default_rng(1)
    v = np.concatenate([
        rng.uniform(-448, 448, 4000).astype(np.float32),
        (rng.standard_normal(2000) * 0.01).astype(np.float32),
        np.array([0.0, -0.0, 448.0, -448.0, 2.0 ** -9, 2.0 ** -10, 3 * 2.0 ** -11, 0.5],
                 np.float32),
    ])
    # ties between neighbouring e4m3 values
    codes = np.arange(0, 0x7E, dtype=np.uint8)
    vals = oracle.fp8e4m3_values(codes)
    mids = ((vals[:-1] + vals[1:]) / 2).astype(np.float32)
    v = np.concatenate([v, mids, -mids])
    ours = oracle.fp8e4m3_rne(v)
    ref = torch.from_numpy(v).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(ours, ref)


def test_fp8_saturates():
    assert oracle.fp8e4m3_rne(np.array([1e6, -1e6, 460.0], np.float32)).tolist() == [0x7E, 0xFE, 0x7E]
    assert oracle.fp8e4m3_values(np.array([0x7E]))[0] == 448.0


def test_fp8_row_scales():
    A = np.array([[1.0, -896.0, 3.0], [0.0, 0.0, 0.0]], np.float32)
    s = oracle.fp8_row_scales(A)
    assert s[0] == np.float32(896.0) / np.float32(448.0) and s[1] == 1.0


# --------------------------------------------------------------------------
# Refinement (oracle composition of residual + RKAB)
# --------------------------------------------------------------------------
import rk_inputs  # noqa: E402


def test_refine_step_with_exact_copy_is_the_plain_solve():
    """Kaczmarz projections commute with translation: one refinement step whose
    inner solve uses the exact rows equals the plain solve started at x0 with the
    same draws (Eq. (alg): (x0 + d) - P(x0 + d) = d - P_r(d) for r = b - A x0)."""
    s = rk_inputs.gaussian_system(300, 12, seed=41)
    b64 = s.A.astype(np.float64) @ s.x_star.astype(np.float64)
    tab = oracle.table(s.A)
    x0 = np.random.default_rng(0).standard_normal(12)
    xs = oracle.refine(s.A, s.A, b64, x0, q=3, alpha=7, inner_rounds=5, outer=1, seed=9, tab_low=tab)
    plain = oracle.rkab(s.A, b64, x0, q=3, alpha=7, rounds=5, seed=9, tab=tab, stream=3)
    np.testing.assert_allclose(xs[0], plain, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("kind,factor", [("bf16", 0.05), ("fp8", 0.5)])
def test_refine_with_stored_rows_converges_to_fp64_solution(kind, factor):
    """Refinement with a perturbed copy contracts the error each outer step and
    reaches the solution of the float32 master system to FP64 accuracy."""
    s = rk_inputs.gaussian_system(2000, 40, seed=43)
    b64 = s.A.astype(np.float64) @ s.x_star.astype(np.float64)
    if kind == "bf16":
        _, low = oracle.quantize_bf16(s.A)
    else:
        _, _, low = oracle.quantize_fp8(s.A)
    tab = oracle.table(low)
    xs = oracle.refine(s.A, low, b64, np.zeros(40), q=4, alpha=200, inner_rounds=20, outer=8,
                       seed=1, tab_low=tab)
    xr = s.x_star.astype(np.float64)
    errs = [np.linalg.norm(x - xr) / np.linalg.norm(xr) for x in xs]
    for e0, e1 in zip(errs[:3], errs[1:4]):
        assert e1 < factor * e0, errs
    assert errs[-1] < 1e-10, errs


def test_quantized_copies_are_close():
    rng = np.random.default_rng(2)
    A = (rng.standard_normal((50, 33)) * 10.0 ** rng.uniform(-3, 3, (50, 1))).astype(np.float32)
    _, vb = oracle.quantize_bf16(A)
    assert np.all(np.abs(vb - A) <= 2.0 ** -8 * np.abs(A))   # 8 significant bits
    _, sc, vf = oracle.quantize_fp8(A)
    amax = np.abs(A).max(axis=1, keepdims=True)
    # normal range: relative half-spacing 2^-4; subnormal range: half of the spacing 2^-9
    # of one scaled unit s_i = amax_i / 448
    bound = 2.0 ** -4 * np.abs(A) + 2.0 ** -10 * sc[:, None] + 1e-6 * np.abs(A)
    assert np.all(np.abs(vf - A) <= bound)
    assert np.all(np.abs(vf) <= amax * (1 + 1e-6))
