"""Host logic of the run harness (paper_2508_06273_gb300/runlog.py) with a
stand-in solver on the CPU: the time-step rule, the log's records and
cadence, the drift, the stop on a bad wave speed, and the checkpoint round
trip."""
import io
import json

import numpy as np
import pytest

from paper_2508_06273_gb300 import runlog


class FakeSolver:
    """Duck-typed stand-in: a 'state' that drifts by a known amount per step."""

    def __init__(self, speeds, torch):
        self.torch = torch
        self.device = "cpu"
        self.speeds = list(speeds)
        self.k = 0
        self.bits = 0
        self.steps = []
        self.state = [torch.full(s, float(i + 1), dtype=torch.float64) for i, s in enumerate(((4, 3, 5), (4, 4, 6), (4, 3, 6), (4, 4, 5)))]
        self.lo = torch.zeros((4, 3, 5), dtype=torch.float64)

    def max_speed(self):
        return self.speeds[min(self.k, len(self.speeds) - 1)]

    def step(self, dt):
        self.steps.append(dt)
        self.k += 1
        self.state[0][0] += 1e-3
        if self.k == 3:
            self.bits |= 64  # a device status bit, kept until read

    def totals(self):
        return np.array([float(self.state[0][v].sum()) for v in range(4)])

    def state_min(self):
        return float(self.state[0][0].min()), float(self.state[0][3].min())

    def counters(self):
        return [self.k, 0, 0, 0]

    def status(self):
        b, self.bits = self.bits, 0
        return b

    def surrogate_stats(self, reset=False):
        return 30, 10

    def get_state(self):
        return tuple(a.clone() for a in self.state)

    def set_state(self, *a):
        self.state = [x.clone() for x in a]

    def get_avg_lo(self):
        return self.lo.clone()

    def set_avg_lo(self, t):
        self.lo = t.clone()


def test_time_step_rule_log_and_drift():
    torch = pytest.importorskip("torch")
    s = FakeSolver([2.0, 4.0, 1.0], torch)
    buf = io.StringIO()
    t, step, hist = runlog.run(s, 1.0, 0.3, 0.1, log=buf, every=2, surrogate=True)
    assert t == pytest.approx(1.0, rel=1e-14) and step == len(hist) == len(s.steps)
    assert hist[0] == pytest.approx(0.3 * 0.1 / 2.0) and hist[1] == pytest.approx(0.3 * 0.1 / 4.0)
    assert all(d == pytest.approx(0.03) for d in hist[2:-1]) and hist[-1] <= 0.03 + 1e-15
    recs = [json.loads(x) for x in buf.getvalue().splitlines()]
    assert [r["step"] for r in recs] == [k for k in range(2, step + 1, 2)] + ([step] if step % 2 else [])
    r = recs[-1]
    assert r["t"] == pytest.approx(1.0) and r["counters"]["eg1"] == step
    # mass drift: 1e-3 per step on 15 cells, relative to the L1 size of the starting averages (15 * (1+1+1+1))
    assert r["drift"][0] == pytest.approx(step * 15e-3 / 60.0) and r["drift"][1] == 0.0
    assert r["surrogate"]["fallback_fraction"] == pytest.approx(0.25)
    assert [x["status"] for x in recs[:3]] == [0, 64, 0]


def test_stop_on_bad_speed_and_max_steps():
    torch = pytest.importorskip("torch")
    s = FakeSolver([1.0, 1.0, float("nan")], torch)
    buf = io.StringIO()
    t, step, _ = runlog.run(s, 10.0, 0.5, 1.0, log=buf)
    assert step == 2 and t == pytest.approx(1.0)
    assert "stopped" in json.loads(buf.getvalue().splitlines()[-1])
    s = FakeSolver([1.0], torch)
    t, step, _ = runlog.run(s, 10.0, 0.5, 1.0, max_steps=3)
    assert step == 3 and t == pytest.approx(1.5)


def test_checkpoint_round_trip(tmp_path):
    torch = pytest.importorskip("torch")
    s = FakeSolver([1.0], torch)
    path = str(tmp_path / "ck.npz")
    t, step, hist = runlog.run(s, 10.0, 0.5, 1.0, max_steps=4, checkpoint=path, checkpoint_every=2)
    s2 = FakeSolver([1.0], torch)
    s2.lo += 7.0
    t2, step2, hist2 = runlog.load_checkpoint(path, s2)
    assert (t2, step2, hist2) == (t, step, hist)
    for a, b in zip(s.get_state(), s2.get_state()):
        assert torch.equal(a, b)
    assert torch.equal(s.get_avg_lo(), s2.get_avg_lo())
