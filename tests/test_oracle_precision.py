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
