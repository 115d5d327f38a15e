"""Batched ensembles through the C ABI (af_batch_*): every instance of a
batch must evolve exactly as the same grid stepped alone with the same dt
sequence, and as the FP64 oracle within the per-step tolerance; dt is
chosen on the device per instance from its own wave speed (CFL condition,
Sec. 2) and the last step is clipped to the instance's end time."""
import numpy as np
import pytest

from helpers import make_oracle
from paper_2508_06273_gb300 import workloads as W
from test_gpu_parity import MILD, assert_parity, env, host, solver, state_err, to_dev  # noqa: F401

pytestmark = pytest.mark.gpu


def _mixed():
    """Small instances of uneven sizes, all boundary kinds and option sets."""
    return [
        W.shu_vortex_seeded(48, seed=11),
        W.fourier_smooth(40, 24, seed=4, lx=1.0, ly=0.6),
        W.four_quadrant(33, states=MILD),
        W.double_rarefaction(36),
        W.gaussian_pulse(50, 20),
    ]


def _batch(env, probs, tile_h=None):
    torch, af, _ = env
    b = af.Batch([(p.nx, p.ny) for p in probs], [(p.dx, p.dy) for p in probs],
                 bcs=[p.bc for p in probs])
    for k, p in enumerate(probs):
        for key, v in p.options.items():
            b.set_option(key, v, k)
        b.set_state(k, *to_dev(torch, W.to_f32(W.discretise(p))))
    if tile_h:
        b.set_tile(tile_h)
    return b


def _run_with_hist(env, b, nsteps):
    torch = env[0]
    hist = torch.zeros((nsteps + 1, b.n), dtype=torch.float64, device="cuda")
    b.run(nsteps, hist)
    return hist.cpu().numpy()


def test_batch_matches_each_grid_stepped_alone(env):
    torch, af, _ = env
    probs = _mixed()
    b = _batch(env, probs)
    hist = _run_with_hist(env, b, 6)
    t, steps, active, status = b.query()
    assert np.all(steps == 6) and np.all(active == 1)
    for k, p in enumerate(probs):
        assert np.isclose(t[k], hist[:6, k].sum(), rtol=0, atol=1e-15), k
        s = solver(env, p)
        # the first dt is cfl * h / (max speed of the initial state)
        assert hist[0, k] == pytest.approx(0.3 * min(p.dx, p.dy) / s.max_speed(), rel=1e-6)
        for n in range(6):
            s.step(hist[n, k])
        want = host(s.get_state())
        got = host(b.get_state(k))
        assert_parity(got, want, 1e-6, what=f"instance {k} ({p.name})")
        assert s.status() & ~8 == 0 and status[k] & ~8 == 0, (k, status[k])
        s.close()
    b.close()


def test_batch_instances_match_the_oracle(env, oracle_mod):
    torch, af, _ = env
    probs = _mixed()[:3]
    b = _batch(env, probs)
    hist = _run_with_hist(env, b, 3)
    for k, p in enumerate(probs):
        o = make_oracle(oracle_mod, p, state=W.to_f32(W.discretise(p)))
        for n in range(3):
            o.step(hist[n, k])
        assert_parity(host(b.get_state(k)), o.get_state(), 3e-5, what=f"instance {k} ({p.name})")
    b.close()


@pytest.mark.parametrize("tile_h", [4, 16])
def test_tile_heights_give_the_same_state(env, tile_h):
    probs = _mixed()
    ref = _batch(env, probs, 8)
    other = _batch(env, probs, tile_h)
    ref.run(4)
    other.run(4)
    for k in range(len(probs)):
        for a, c in zip(ref.get_state(k), other.get_state(k)):
            assert env[0].equal(a, c), (k, tile_h)
    ref.close()
    other.close()


def test_one_graph_run_equals_single_steps(env):
    probs = _mixed()
    a = _batch(env, probs)
    c = _batch(env, probs)
    a.run(9)
    for _ in range(9):
        c.run(1)
    for k in range(len(probs)):
        for x, y in zip(a.get_state(k), c.get_state(k)):
            assert env[0].equal(x, y), k
    assert np.array_equal(a.query()[0], c.query()[0])
    a.close()
    c.close()


def test_end_times_are_met_exactly_and_instances_stop(env):
    probs = _mixed()[:3]
    b = _batch(env, probs)
    ends = np.array([0.05, 0.013, 0.0])  # the last one never starts
    b.set_end(ends)
    hist = _run_with_hist(env, b, 40)
    t, steps, active, _ = b.query()
    assert np.all(active == 0)
    assert steps[2] == 0 and t[2] == 0.0
    for k in range(2):
        assert t[k] == pytest.approx(ends[k], rel=1e-14)
        assert np.isclose(hist[: steps[k], k].sum(), t[k], rtol=1e-14)
    before = [host(b.get_state(k)) for k in range(3)]
    b.run(5)  # nothing active: the state does not move
    for k in range(3):
        for x, y in zip(before[k], host(b.get_state(k))):
            assert np.array_equal(x, y)
    # a later end time re-activates the instances that have state
    b.set_end(np.array([0.06, 0.013, 0.01]))
    b.run(40)
    t, steps, active, _ = b.query()
    assert t[0] == pytest.approx(0.06, rel=1e-14) and t[2] == pytest.approx(0.01, rel=1e-14)
    b.close()


def test_a_failing_instance_stops_alone(env):
    """Four-quadrant data whose averages lose positivity at once (seed 0 at
    64^2 with neither the flux limiter nor the Sec. 3.4 blend): that
    instance is flagged and stopped, the others run on unchanged."""
    probs = [W.shu_vortex_seeded(40, seed=3), W.four_quadrant(64, seed=0)]
    probs[1].options = dict(probs[1].options, flux_limiter=0, shock_blend=0)
    b = _batch(env, probs)
    hist = _run_with_hist(env, b, 12)
    t, steps, active, status = b.query()
    assert active[1] == 0 and (status[1] & (2 | 32)) == (2 | 32), status
    assert active[0] == 1 and steps[0] == 12 and status[0] == 0
    s = solver(env, probs[0])
    for n in range(12):
        s.step(hist[n, 0])
    assert_parity(host(b.get_state(0)), host(s.get_state()), 1e-6, what="running instance")
    s.close()
    b.close()


def test_autotune_keeps_the_state(env):
    probs = _mixed()
    b = _batch(env, probs)
    b.run(2)
    t0 = b.query()[0]
    before = [host(b.get_state(k)) for k in range(len(probs))]
    th, ms = b.autotune()
    assert th in (4, 8, 16) and all(v > 0 for v in ms.values()) and ms[th] == min(ms.values())
    assert np.array_equal(b.query()[0], t0)
    for k in range(len(probs)):
        for x, y in zip(before[k], host(b.get_state(k))):
            assert np.array_equal(x, y)
    # and stepping after tuning still matches an untuned batch
    ref = _batch(env, probs)
    ref.run(2)
    ref.run(3)
    b.run(3)
    for k in range(len(probs)):
        for x, y in zip(ref.get_state(k), b.get_state(k)):
            assert env[0].equal(x, y)
    ref.close()
    b.close()
