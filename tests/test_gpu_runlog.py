"""Diagnostics of a run on the GPU: af_state_min against the state read
back, the run harness's JSON-lines log on a four-quadrant problem, and a run
resumed from the harness's checkpoint repeating the uninterrupted run bit for
bit."""
import json

import numpy as np
import pytest

from paper_2508_06273_gb300 import runlog
from paper_2508_06273_gb300 import workloads as W
from test_gpu_parity import env, solver  # noqa: F401

pytestmark = pytest.mark.gpu


def _prim_min(state, g=1.4):
    avg = state[0].astype(np.float64)
    r = avg[0]
    p = (g - 1) * (avg[3] - 0.5 * (avg[1] ** 2 + avg[2] ** 2) / r)
    rmin = min([r.min()] + [a[0].min() for a in state[1:]])
    pmin = min([p.min()] + [a[3].min() for a in state[1:]])
    return rmin, pmin


def test_state_min_matches_the_state(env):
    torch, af, _ = env
    prob = W.four_quadrant(61, seed=3)
    s = solver(env, prob)
    for _ in range(5):
        s.step(0.3 * prob.dx / s.max_speed())
    rmin, pmin = s.state_min()
    want = _prim_min([t.cpu().numpy() for t in s.get_state()])
    assert rmin == pytest.approx(want[0], rel=1e-6) and pmin == pytest.approx(want[1], rel=1e-5)
    s.close()


def test_log_and_checkpoint_resume(env, tmp_path):
    torch, af, _ = env
    prob = W.four_quadrant(48, seed=1)
    h = min(prob.dx, prob.dy)
    log = tmp_path / "run.jsonl"
    ck = tmp_path / "ck.npz"
    a = solver(env, prob)
    t, step, hist = runlog.run(a, 0.05, 0.3, h, log=str(log), every=5, max_steps=12, checkpoint=str(ck),
                               checkpoint_every=6)
    recs = [json.loads(x) for x in log.read_text().splitlines()]
    assert [r["step"] for r in recs] == [5, 10, 12]
    for r in recs:
        assert r["min_rho"] > 0 and r["min_p"] > 0
        assert not r["status"] & (af.ST_AVG_NONPOS | af.ST_NONFINITE | af.ST_TIMEOUT)
        # transmissive box: the totals change by what the boundary fluxes carry
        assert all(np.isfinite(r["drift"])) and r["t"] <= 0.05
    t2, step2, hist2 = runlog.run(a, 0.05, 0.3, h, t=t, step=step, dt_hist=hist, max_steps=8)
    # resume from the checkpoint of step 12 in a fresh solver
    b = solver(env, prob)
    tb, stepb, histb = runlog.load_checkpoint(str(ck), b)
    assert (tb, stepb, histb) == (t, step, hist)
    tb, stepb, histb = runlog.run(b, 0.05, 0.3, h, t=tb, step=stepb, dt_hist=histb, max_steps=8)
    assert (tb, stepb) == (t2, step2) and histb == hist2
    for x, y in zip(a.get_state(), b.get_state()):
        assert torch.equal(x, y)
    assert torch.equal(a.get_avg_lo(), b.get_avg_lo())
    a.close()
    b.close()
