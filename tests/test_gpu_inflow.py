"""Inflow boundaries (Sec. 4.3) on the GPU, through the C ABI: a constant
inflow state is preserved, the shock-reflection problem follows the FP64
oracle step by step, and at t = 6 its wall plateau takes the state of the
oblique-shock relations."""
import numpy as np
import pytest

from helpers import make_oracle
from paper_2508_06273_gb300 import workloads as W
from test_gpu_parity import assert_parity, env, host, solver  # noqa: F401
from test_oracle_pins import _regular_reflection

pytestmark = pytest.mark.gpu


def test_constant_inflow_state_is_preserved(env):
    U = (1.3, 0.7, -0.4, 0.9)
    prob = W.Problem("inflow_const", 40, 24, 0.0, 0.0, 1.0, 0.6, (3, 3, 3, 3), lambda x, y: U, 1.0,
                     inflow={k: U for k in range(4)})
    s = solver(env, prob)
    s0 = host(s.get_state())
    for _ in range(5):
        s.step(0.3 * prob.dx / s.max_speed())
    assert_parity(host(s.get_state()), s0, 1e-6, what="constant inflow")
    assert s.status() == 0


def test_shock_reflection_follows_the_oracle(env):
    torch, af, oracle = env
    prob = W.shock_reflection()
    st = W.to_f32(W.discretise(prob))
    o = make_oracle(oracle, prob, state=st)
    s = solver(env, prob, state=st)
    for _ in range(8):
        dt = 0.3 * prob.dx / o.max_speed()
        o.step(dt)
        s.step(dt)
    assert_parity(host(s.get_state()), o.get_state(), 8e-5, what="shock reflection")
    assert s.status() == 0


def test_shock_reflection_reaches_the_regular_reflection_state(env):
    torch, af, _ = env
    prob = W.shock_reflection()
    s = solver(env, prob)
    t = 0.0
    while t < prob.t_end - 1e-12:
        dt = min(0.3 * prob.dx / s.max_speed(), prob.t_end - t)
        s.step(dt)
        t += dt
    assert s.status() == 0
    avg = host(s.get_state())[0]
    x = (np.arange(prob.nx) + 0.5) * prob.dx
    y = (np.arange(prob.ny) + 0.5) * prob.dy
    sel = (x[None, :] > 3.2) & (x[None, :] < 3.8) & (y[:, None] < 0.15)
    rho3, p3 = _regular_reflection(prob.inflow[3])
    p = 0.4 * (avg[3] - 0.5 * (avg[1] ** 2 + avg[2] ** 2) / avg[0])
    assert abs(avg[0][sel].mean() / rho3 - 1) < 5e-3
    assert abs(p[sel].mean() / p3 - 1) < 5e-3
