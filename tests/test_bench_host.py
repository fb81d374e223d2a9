"""Host logic of bench.py that needs no GPU: the size of the oracle's timed sample.

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
