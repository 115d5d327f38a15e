"""Failure detection without a GPU fault: the bounded waits of the
point-value kernel (for its TMA-staged tile) and of the surrogate (for its
tensor-core MMAs) are made to run out by a test hook that arms the barrier
and issues no copy or MMA, so nothing is in flight when a block gives up.
The step returns normally with AF_ST_TIMEOUT set, the status is sticky, the
handle (or batch) refuses further steps, and the CUDA context stays usable."""
import numpy as np
import pytest

from paper_2508_06273_gb300 import workloads as W
from test_gpu_parity import env, solver  # noqa: F401

pytestmark = pytest.mark.gpu


def _fresh_step_is_clean(env, prob, dt):
    s = solver(env, prob)
    s.step(dt)
    assert s.status() == 0
    s.close()


def test_tile_wait_times_out_and_the_handle_refuses_steps(env):
    torch, af, _ = env
    prob = W.shu_vortex(32)
    s = solver(env, prob, {"test_timeout": 1})
    dt = 0.3 * prob.dx / s.max_speed()
    s.step(dt)  # returns normally: only the status word reports the time-out
    assert s.status() & af.ST_TIMEOUT
    assert s.status() & af.ST_TIMEOUT  # sticky
    with pytest.raises(af.AFError, match="timed out"):
        s.step(dt)
    with pytest.raises(af.AFError, match="timed out"):
        s.run(6, dt)
    s.get_state()  # the state can still be read (its values are invalid)
    s.close()
    _fresh_step_is_clean(env, prob, dt)


def test_surrogate_mma_wait_times_out(env):
    torch, af, _ = env
    prob = W.shu_vortex(64)
    nets = [af.Mlp(seed=k) for k in (3, 4)]
    s = solver(env, prob)
    s.set_surrogate(*nets)
    s.set_option("surrogate", 1)
    s.set_option("test_timeout", 1)
    dt = 0.3 * prob.dx / s.max_speed()
    s.step(dt)
    assert s.status() & af.ST_TIMEOUT
    with pytest.raises(af.AFError, match="timed out"):
        s.step(dt)
    s.close()
    for n in nets:
        n.close()
    _fresh_step_is_clean(env, prob, dt)


def test_batch_instance_timeout_stops_the_batch(env):
    torch, af, _ = env
    probs = [W.shu_vortex_seeded(40, seed=3), W.shu_vortex_seeded(48, seed=4)]
    b = af.Batch([(p.nx, p.ny) for p in probs], [(p.dx, p.dy) for p in probs], bcs=[p.bc for p in probs])
    for k, p in enumerate(probs):
        b.set_state(k, *[torch.from_numpy(np.asarray(a, dtype=np.float32)).cuda()
                         for a in W.to_f32(W.discretise(p))])
    b.set_option("test_timeout", 1, 1)
    b.run(1)
    _, _, _, status = b.query()
    assert not status[0] & af.ST_TIMEOUT and status[1] & af.ST_TIMEOUT, status
    with pytest.raises(af.AFError, match="timed out"):
        b.run(1)
    b.close()
    _fresh_step_is_clean(env, probs[0], 1e-3)
