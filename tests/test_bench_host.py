"""Host logic of bench.py that needs no GPU: the size of the oracle's timed sample, the
roofline's algorithmic bytes, and the recorded DRAM traffic that is used only for the kernel
source it was measured on.

The sample must stay bounded and close to its time target whatever the probes
measure (a slow first call that pages A in, a noisy difference between probes)."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


class _Fake:
    """oracle_sample stand-in: fixed cost + per-projection cost, the first call slower."""

    def __init__(self, fixed, per, first_extra=0.0, jitter=None):
        self.fixed, self.per, self.first_extra = fixed, per, first_extra
        self.jitter = list(jitter or [])
        self.calls = 0

    def __call__(self, A_np, b_np, tab, q, alpha_sample, seed, threads):
        t = self.fixed + self.per * alpha_sample
        if self.calls == 0:
            t += self.first_extra
        if self.jitter:
            t += self.jitter.pop(0)
        self.calls += 1
        return q * alpha_sample, t


class _A:
    shape = (80000, 10000)


@pytest.mark.parametrize("fixed,per,first_extra,jitter", [
    (0.35, 0.002, 0.0, None),        # plain
    (0.35, 0.002, 5.0, None),        # a slow first call (pages of A, thread start)
    (0.35, 0.002, 0.0, [0.0, 0.3, 0.0]),    # the smaller warm probe slower than usual
    (0.35, 0.002, 0.0, [0.0, 0.0, -0.3]),   # the larger warm probe faster than usual
])
def test_sample_alpha_stays_near_target(monkeypatch, fixed, per, first_extra, jitter):
    fake = _Fake(fixed, per, first_extra, jitter)
    monkeypatch.setattr(bench, "oracle_sample", fake)
    target = 20.0
    alpha = bench.sample_alpha(_A(), None, None, 132, 0, 8, target)
    t = fixed + per * alpha   # the time the sampled round would take
    assert 10 <= alpha
    assert t <= 3 * target, (alpha, t)
    assert t >= target / 10, (alpha, t)


def test_sample_alpha_tiny_target_keeps_a_minimum(monkeypatch):
    monkeypatch.setattr(bench, "oracle_sample", _Fake(0.35, 0.002))
    assert bench.sample_alpha(_A(), None, None, 132, 0, 8, 0.01) == 10


def test_algorithmic_bytes_of_the_roofline():
    """The roofline's numerator: per projection the row, b_i, 1/||A_i||^2 and the alias
    entry; per round the averaging traffic of the partial iterates written (q of them, or
    one per CTA for RKA spread over the CTAs)."""
    n = 10000
    per_proj = n * 4 + 4 + 4 + 12
    # the benchmark configuration: 132 workers, alpha = n, 28 rounds (1.4796e12 B)
    assert bench.algorithmic_bytes(n, 132, n, 28) == 28 * (132 * n * per_proj + 3 * 132 * n * 4)
    assert bench.algorithmic_bytes(n, 132, n, 28) == 1479582720000
    # RKA with 4864 workers on 152 SMs: 152 partial iterates a round
    assert bench.algorithmic_bytes(n, 4864, 1, 85, 4, 152) == 85 * (4864 * per_proj + 3 * 152 * n * 4)
    # BF16 rows: 2 bytes an element
    assert bench.algorithmic_bytes(n, 132, 1, 1, 2) == 132 * (n * 2 + 20) + 3 * 132 * n * 4


def test_recorded_traffic_only_for_the_kernel_it_was_taken_on(tmp_path, monkeypatch):
    """The roofline's DRAM traffic comes from an ncu record tied to a hash of the solve
    kernel's source: the record is used while the hash matches the source as it is, and
    ignored (traffic null) once the source has changed or when no record exists."""
    monkeypatch.setattr(bench, "PROFILE_DIR", str(tmp_path))
    assert bench.recorded_traffic("c2") is None                     # no record
    h = bench.kernel_hash()
    (tmp_path / "rkab_kernel_c2.txt").write_text(
        "DRAM bytes of one launch\n"
        f"traffic_bytes_per_proj 38995.2 src {h}\n")
    assert bench.recorded_traffic("c2") == pytest.approx(38995.2)
    (tmp_path / "rkab_kernel_c2.txt").write_text(
        f"traffic_bytes_per_proj 38995.2 src {'0' * len(h)}\n")    # taken on other source
    assert bench.recorded_traffic("c2") is None
    assert len(h) == 12 and h == bench.kernel_hash()               # stable for unchanged source
