"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: relative L1 <= 1e-5 after one step and <= 1e-4 at the final
time on smooth data; the metric is per array and per variable, with
velocities (and momenta) measured against the local speed scale
|u| + |v| + c so that a vanishing velocity field has a defined error.
Positivity of the point values is checked exactly.
"""
import numpy as np
import pytest

from helpers import make_oracle
from paper_2508_06273_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-5
FINAL_TOL = 1e-4


@pytest.fixture(scope="module")
def env(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2508_06273_gb300 import af

    return torch, af, oracle_mod


def to_dev(torch, state):
    return [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda() for a in state]


def solver(env, prob, opts=None, state=None):
    torch, af, _ = env
    o = dict(prob.options)
    o.update(opts or {})
    s = af.Solver(prob.nx, prob.ny, prob.dx, prob.dy, prob.gamma, prob.bc, options=o, inflow=prob.inflow)
    s.set_state(*to_dev(torch, state if state is not None else W.to_f32(W.discretise(prob))))
    return s


def host(ts):
    return [t.cpu().double().numpy() for t in ts]


def _scales(want, conservative):
    """Per-element scale of each variable: |q| for rho, p and E; the local
    speed scale |u| + |v| + c for the velocities (rho (|u| + |v| + c) for the
    momenta)."""
    g = 1.4
    want = np.asarray(want, dtype=np.float64)
    if conservative:
        r = want[0]
        u, v = want[1] / r, want[2] / r
        p = (g - 1) * (want[3] - 0.5 * r * (u * u + v * v))
        vel = np.abs(r) * (np.abs(u) + np.abs(v) + np.sqrt(np.abs(g * p / r)))
    else:
        vel = np.abs(want[1]) + np.abs(want[2]) + np.sqrt(np.abs(g * want[3] / want[0]))
    return [np.abs(want[0]), vel, vel, np.abs(want[3])]


def rel_l1(got, want, conservative):
    """max over variables of the relative L1 distance of one array."""
    sc = _scales(want, conservative)
    out = 0.0
    for v in range(4):
        out = max(out, np.abs(got[v] - want[v]).sum() / sc[v].sum())
    return out


def state_err(got, want):
    return max(rel_l1(a, b, k == 0) for k, (a, b) in enumerate(zip(got, want)))


def state_max_err(got, want, first_conservative=True):
    """Largest per-element error relative to the element's own scale, with its
    place: (error, array, variable, index, got, want)."""
    best = (0.0, None, None, None, None, None)
    for k, (a, b) in enumerate(zip(got, want)):
        a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
        sc = _scales(b, first_conservative and k == 0)
        for v in range(4):
            e = np.abs(a[v] - b[v]) / np.maximum(sc[v], 1e-300)
            at = np.unravel_index(int(np.argmax(e)), e.shape)
            if e[at] > best[0] or best[1] is None:
                best = (float(e[at]), k, v, tuple(int(x) for x in at), float(a[v][at]), float(b[v][at]))
    return best


# per-element bound: a factor ELEM_FACTOR above the L1 gates (one node wrong by
# 1% passes a whole-array L1 gate of 1e-5 on a small grid, not this one)
ELEM_FACTOR = 10.0


def assert_parity(got, want, l1_tol, elem_tol=None, first_conservative=True, what=""):
    """Both gates: relative L1 per array and variable, and every element
    within elem_tol (default ELEM_FACTOR x l1_tol) of its own scale."""
    elem_tol = ELEM_FACTOR * l1_tol if elem_tol is None else elem_tol
    l1 = max(rel_l1(a, b, first_conservative and k == 0) for k, (a, b) in enumerate(zip(got, want)))
    e, k, v, idx, a, b = state_max_err(got, want, first_conservative)
    assert l1 < l1_tol, f"{what}: relative L1 {l1:.3e} >= {l1_tol:.1e}"
    assert e < elem_tol, (f"{what}: element error {e:.3e} >= {elem_tol:.1e} at array {k} variable {v} "
                          f"index {idx}: got {a!r}, want {b!r}")
    return l1, e


def _flow(base, n=37, m=29, amp=0.05, seed=3):
    """Smooth periodic field about a uniform state ``base`` (rho, u, v, p):
    sets how the Mach-cone bases cross the grid lines (supersonic: no
    crossing of a line; sonic: tangent; at rest: P' on the lines)."""
    rng = np.random.default_rng(seed)
    c = rng.normal(size=(4, 3, 3, 2)) * amp / 3

    def f(x, y):
        out = []
        for k in range(4):
            s = base[k] + 0 * x
            for a in range(3):
                for b in range(3):
                    ph = 2 * np.pi * (a * x + b * y)
                    s = s + c[k, a, b, 0] * np.cos(ph) + c[k, a, b, 1] * np.sin(ph)
            out.append(s)
        return tuple(out)

    return W.Problem("flow", n, m, 0.0, 0.0, 1.0, m / n, (0, 0, 0, 0), f, 1.0)


SMOOTH = {
    "vortex32": lambda: W.shu_vortex(32),
    "fourier_ragged": lambda: W.fourier_smooth(50, 37, seed=5, lx=1.0, ly=0.81),
    "vortex_seeded128": lambda: W.shu_vortex_seeded(128),
    "supersonic_x": lambda: _flow((1.0, 1.9, 0.2, 1.0)),
    "supersonic_xy": lambda: _flow((1.0, -1.5, 1.6, 1.0)),
    "sonic_x": lambda: _flow((1.0, 1.4 ** 0.5, 0.0, 1.0)),
    "at_rest": lambda: _flow((1.0, 0.0, 0.0, 1.0)),
    # c = 1.18: both lines crossed, node outside the circle, u, v < 0
    "outside_neg": lambda: _flow((1.0, -0.95, -0.9, 1.0)),
    # only the vertical line crossed, u, v < 0
    "supersonic_y": lambda: _flow((1.0, -0.3, -1.7, 1.0)),
    # node inside the circle (quarter arc present), u < 0
    "inside_neg": lambda: _flow((1.0, -0.5, 0.4, 1.0)),
}
MODES = {"avg": {}, "point": {"lin_mode": 1}, "alg1": {"lin_mode": 2}, "nocorr": {"correction": 0},
         "tsw": {"tsw": 1}, "ubar_c2p": {"ubar": 1}}


@pytest.mark.parametrize("case", list(SMOOTH))
@pytest.mark.parametrize("mode", list(MODES))
def test_one_step_parity(env, case, mode):
    if mode not in ("avg", "ubar_c2p") and case not in ("vortex32", "fourier_ragged", "vortex_seeded128"):
        pytest.skip("linearisation modes are covered on the first three cases")
    torch, af, oracle = env
    prob = SMOOTH[case]()
    st = W.to_f32(W.discretise(prob))
    o = make_oracle(oracle, prob, MODES[mode], state=st)
    dt = prob.cfl * min(prob.dx, prob.dy) / o.max_speed()
    o.step(dt)
    s = solver(env, prob, dict(MODES[mode], keep_half=1), st)
    s.step(dt)
    assert s.status() == 0
    assert_parity(host(s.get_state()), o.get_state(), STEP_TOL, what="t^n+1")
    assert_parity(host(s.get_half()), o.get_half(), STEP_TOL, first_conservative=False, what="t^n+1/2")


def test_final_time_vortex32(env):
    """32x32 isentropic vortex, CFL 0.3, to t = 10 (one period)."""
    torch, af, oracle = env
    prob = W.shu_vortex(32)
    st = W.to_f32(W.discretise(prob))
    o = make_oracle(oracle, prob, state=st)
    s = solver(env, prob, state=st)
    t, n = 0.0, 0
    while t < prob.t_end * (1 - 1e-12):
        dt = min(prob.cfl * prob.dx / o.max_speed(), prob.t_end - t)
        o.step(dt)
        s.step(dt)
        t += dt
        n += 1
    assert s.status() == 0
    assert_parity(host(s.get_state()), o.get_state(), FINAL_TOL, what=f"after {n} steps")


def test_conservation_periodic(env):
    torch, af, _ = env
    prob = W.fourier_smooth(64, 48, seed=8, lx=1.0, ly=0.75)
    s = solver(env, prob)
    t0 = s.totals()
    absq = np.abs(W.discretise(prob)[0]).sum(axis=(1, 2)) * prob.dx * prob.dy
    for _ in range(50):
        s.step(0.3 * prob.dx / 2.0)
    drift = np.abs(s.totals() - t0) / absq
    assert s.status() == 0
    assert np.all(drift < 1e-13), drift


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1), (2, 2, 2, 2), (1, 2, 0, 0)])
def test_constant_state_preserved(env, bc):
    """Constant data.  The FP32 centre value from inverse Simpson cannot be
    exactly consistent with FP32 averages, so point values settle within a
    few ulp of the constant (a bounded offset, not a drift).  Without walls
    every node sees the same arithmetic, every face flux is the same and the
    averages stay bitwise unchanged; wall nodes are linearised about their own
    value, so next to a wall the averages move by FP32 round-off only."""
    torch, af, _ = env
    U = (0.8, 0.0 if 2 in bc else 0.3, 0.0 if 2 in bc else -0.6, 1.7)
    prob = W.Problem("const", 33, 20, 0.0, 0.0, 3.3, 2.0, bc, lambda x, y: U, 1.0)
    st = W.to_f32(W.discretise(prob))
    s = solver(env, prob, state=st)
    dt = 0.3 * min(prob.dx, prob.dy) / s.max_speed()
    dev = []
    for k in range(40):
        s.step(dt)
        if k in (19, 39):
            got = host(s.get_state())
            if 2 in bc:
                np.testing.assert_allclose(got[0], st[0], rtol=2e-6, atol=2e-6)
            else:
                assert np.array_equal(got[0], st[0])
            dev.append(max(np.max(np.abs(a - b) / (np.abs(b) + 1.0)) for a, b in zip(got[1:], st[1:])))
    assert s.status() == 0
    assert dev[1] < 2e-6 and dev[1] <= 1.5 * dev[0] + 1e-7, dev


def _wall_problem(n=40):
    rng = np.random.default_rng(4)
    c = rng.normal(size=(4, 3, 3)) * 0.05

    def f(x, y):
        out = []
        for k in range(4):
            s = [1.0, 0.2, 0.0, 1.0][k] + 0.0 * x
            for a in range(3):
                for b in range(3):
                    if k == 2:
                        s = s + c[k, a, b] * np.cos(2 * np.pi * a * x) * np.sin(np.pi * (b + 1) * y)
                    else:
                        s = s + c[k, a, b] * np.cos(2 * np.pi * a * x) * np.cos(np.pi * b * y)
            out.append(s)
        return tuple(out)

    return W.Problem("wall", n, n - 7, 0.0, 0.0, 1.0, 1.0, (1, 1, 2, 2), f, 0.05)


def test_walls_and_outflow_parity(env):
    torch, af, oracle = env
    prob = _wall_problem()
    st = W.to_f32(W.discretise(prob))
    o = make_oracle(oracle, prob, state=st)
    s = solver(env, prob, state=st)
    for _ in range(5):
        dt = 0.3 * prob.dy / o.max_speed()
        o.step(dt)
        s.step(dt)
        assert_parity(host(s.get_state()), o.get_state(), STEP_TOL, what="walls")
    _, vtx, xe, ye = host(s.get_state())
    assert np.max(np.abs(vtx[2, [0, -1], :])) < 1e-6
    assert np.max(np.abs(ye[2, [0, -1], :])) < 1e-6


MILD = [(1.0, 0.1, -0.1, 1.0), (0.9, -0.15, 0.05, 1.1), (1.1, 0.05, 0.15, 0.95), (0.95, -0.1, -0.05, 1.05)]


@pytest.mark.parametrize("force", [1, 2])
@pytest.mark.parametrize("data", ["mild_quadrants", "fourier", "supersonic_xy", "supersonic_y", "outside_neg",
                                  "inside_neg"])
def test_low_order_paths_parity(env, force, data):
    """Alg. 3's EG1-on-pc and Lax-Friedrichs updates, forced at every node,
    on data where every EG1 value is clearly admissible (so FP32 and FP64
    take the same branches); the flows cover every way the Mach circle can
    meet the grid lines (no line, one line, both with the node outside or
    inside the circle) and both signs of the velocity."""
    torch, af, oracle = env
    if data == "fourier":
        prob = W.fourier_smooth(30, 26, seed=7)
    elif data == "mild_quadrants":
        prob = W.four_quadrant(24, states=MILD)
    else:
        prob = SMOOTH[data]()
    st = W.to_f32(W.discretise(prob))
    opts = {"force_lo": force, "tsw": 0, "shock_blend": 0, "flux_limiter": 0}
    o = make_oracle(oracle, prob, opts, state=st)
    dt = 0.3 * min(prob.dx, prob.dy) / o.max_speed()
    o.step(dt)
    s = solver(env, prob, dict(opts, keep_half=1), st)
    s.step(dt)
    assert_parity(host(s.get_half()), o.get_half(), STEP_TOL, first_conservative=False, what="t^n+1/2")
    assert_parity(host(s.get_state())[1:], o.get_state()[1:], STEP_TOL, first_conservative=False, what="t^n+1")
    assert s.counters()[:2] == o.counters()[:2]


def test_riemann_limiter_positivity(env):
    """Four-quadrant data with Alg. 2 and Alg. 3: every point value stays
    admissible; the distance to the oracle is reported loosely (branch
    decisions near rho, p = 0 may differ between FP32 and FP64)."""
    torch, af, oracle = env
    prob = W.four_quadrant(64, seed=5)
    st = W.to_f32(W.discretise(prob))
    o = make_oracle(oracle, prob, state=st)
    s = solver(env, prob, state=st)
    for _ in range(30):
        dt = 0.3 * prob.dx / o.max_speed()
        o.step(dt)
        s.step(dt)
        for a in host(s.get_state())[1:]:
            assert np.all(a[0] > 0) and np.all(a[3] > 0)
    st_bits = s.status()
    assert not (st_bits & af.ST_NONFINITE)
    err = np.abs(host(s.get_state())[0][0] - o.get_state()[0][0]).sum() / np.abs(o.get_state()[0][0]).sum()
    assert err < 1e-2, err


def test_double_rarefaction_positivity(env):
    torch, af, _ = env
    prob = W.double_rarefaction(128)
    s = solver(env, prob)
    for _ in range(40):
        s.step(0.3 * prob.dx / s.max_speed())
        assert all(np.all(a[0] > 0) and np.all(a[3] > 0) for a in host(s.get_state())[1:])
    assert sum(s.counters()[:2]) >= 0


def test_status_flags_and_errors(env):
    torch, af, _ = env
    prob = W.shu_vortex(16)
    s = solver(env, prob)
    s.step(3.0 * prob.dx / s.max_speed())  # CFL 3: the cone base leaves the stencil
    assert s.status() & af.ST_CFL
    st = W.to_f32(W.discretise(prob))
    with pytest.raises(af.AFError):  # host memory passed as device memory
        af._check(s.L.af_set_state(s.h, *[np.asarray(a, dtype=np.float32).ctypes.data for a in st], None))
    bad = [a.copy() for a in st]
    bad[1][0, 3, -1] += 1.0  # periodic duplicate line differs from the first
    with pytest.raises(af.AFError):
        s.set_state(*to_dev(torch, bad))
    fresh = af.Solver(8, 8, 0.1, 0.1)
    with pytest.raises(af.AFError):
        fresh.step(0.01)
    with pytest.raises(af.AFError):
        fresh.set_option("lin_mode", 7)


def test_host_transfer_roundtrip(env):
    torch, af, _ = env
    prob = W.fourier_smooth(30, 20, seed=2)
    st = [np.asarray(a, dtype=np.float32) for a in W.discretise(prob)]
    s = af.Solver(prob.nx, prob.ny, prob.dx, prob.dy, bc=prob.bc)
    s.set_state(*st)
    for a, b in zip(s.get_state_host(), st):
        assert np.array_equal(a, b)
    for a, b in zip(host(s.get_state()), st):
        assert np.array_equal(a, b)


def _pinned(torch, shapes, fill=None):
    out = []
    for k, sh in enumerate(shapes):
        a = torch.empty(sh, dtype=torch.float32, pin_memory=True).numpy()
        a[...] = 0.0 if fill is None else fill[k]
        out.append(a)
    return out


def test_async_host_pipeline_matches_synchronous_transfers(env):
    """Uploads, steps and downloads pipelined through the asynchronous host
    calls (the download of one step overlapping the upload of the next) give
    bitwise the states of the synchronous calls; the inputs change every
    step, so a stale staging area would show."""
    torch, af, _ = env
    prob = W.shu_vortex(64)
    base = [np.asarray(a, dtype=np.float32) for a in W.discretise(prob)]
    ins = [[(a * (1.0 + 1e-3 * k)).astype(np.float32) for a in base] for k in range(3)]
    dt = 0.3 * prob.dx / 2.5
    sync = af.Solver(prob.nx, prob.ny, prob.dx, prob.dy, bc=prob.bc)
    want = []
    for st in ins:
        sync.set_state(*st)
        sync.step(dt)
        want.append(sync.get_state_host())
    a = af.Solver(prob.nx, prob.ny, prob.dx, prob.dy, bc=prob.bc)
    shapes = a.shapes()
    pin_in = [_pinned(torch, shapes, st) for st in ins]
    pin_out = [_pinned(torch, shapes) for _ in ins]
    for k in range(3):
        a.set_state_host_async(*pin_in[k])
        a.step(dt)
        a.get_state_host_async(pin_out[k])
    a.host_sync()
    for k in range(3):
        for x, y in zip(pin_out[k], want[k]):
            assert np.array_equal(x, y), k
    # a periodic duplicate line that differs is reported by host_sync
    bad = [x.copy() for x in pin_in[0]]
    bad[1][0, -1, 3] += 1.0
    bad = _pinned(torch, shapes, bad)
    a.set_state_host_async(*bad)
    with pytest.raises(af.AFError):
        a.host_sync()
    sync.close()
    a.close()


def test_full_size_sampled_windows(env):
    """The 8192^2 seeded vortex in the benchmark's launch configuration: one
    step on the GPU; windows of 16x16 cells are recomputed by the oracle
    (outflow ghosts at the window edge) and their central cells and nodes
    compared; conservation and status at full size."""
    torch, af, oracle = env
    n = 8192
    prob = W.shu_vortex_seeded(n)
    dev = W.discretise_torch(prob, "cuda")
    s = af.Solver(n, n, prob.dx, prob.dy, prob.gamma, prob.bc)
    s.set_state(*dev)
    t0 = s.totals()
    dt = prob.cfl * prob.dx / s.max_speed()
    s.step(dt)
    assert s.status() == 0
    t1 = s.totals()
    mass = float(dev[0][0].double().sum()) * prob.dx * prob.dy
    assert abs(t1[0] - t0[0]) < 1e-12 * mass
    out = s.get_state()
    rng = np.random.default_rng(0)
    w, m = 16, 4
    for _ in range(4):
        i0, j0 = (int(x) for x in rng.integers(0, n - w, size=2))
        win = [dev[0][:, j0:j0 + w, i0:i0 + w], dev[1][:, j0:j0 + w + 1, i0:i0 + w + 1],
               dev[2][:, j0:j0 + w, i0:i0 + w + 1], dev[3][:, j0:j0 + w + 1, i0:i0 + w]]
        sub = W.subproblem(prob, i0, j0, w, w)
        o = make_oracle(oracle, sub, state=[a.cpu().double().numpy() for a in win])
        o.step(dt)
        ref = o.get_state()
        got = [out[0][:, j0:j0 + w, i0:i0 + w], out[1][:, j0:j0 + w + 1, i0:i0 + w + 1],
               out[2][:, j0:j0 + w, i0:i0 + w + 1], out[3][:, j0:j0 + w + 1, i0:i0 + w]]
        got = [a.cpu().double().numpy()[:, m:-m, m:-m] for a in got]
        ref = [a[:, m:-m, m:-m] for a in ref]
        assert_parity(got, ref, STEP_TOL, what=f"window at {(i0, j0)}")
    s.close()


@pytest.mark.parametrize("nsteps", [7, 10])
def test_graph_replay_is_bitwise_equal_to_steps(env, nsteps):
    """af_run replays two captured steps as a CUDA graph; the kernels are
    deterministic, so the result equals nsteps calls of af_step bit for bit."""
    torch, af, _ = env
    prob = W.fourier_smooth(40, 33, seed=21)
    st = W.to_f32(W.discretise(prob))
    a, b = solver(env, prob, state=st), solver(env, prob, state=st)
    dt = 0.3 * prob.dx / a.max_speed()
    for _ in range(nsteps):
        a.step(dt)
    b.run(nsteps, dt)
    b.run(nsteps, dt)  # second call replays the cached graph
    for _ in range(nsteps):
        a.step(dt)
    assert a.status() == 0 and b.status() == 0
    for x, y in zip(host(a.get_state()), host(b.get_state())):
        assert np.array_equal(x, y)
    assert np.array_equal(host([a.get_avg_lo()])[0], host([b.get_avg_lo()])[0])


def test_fused_max_speed_matches_reduction(env):
    """The flux kernel's wave-speed maximum of the new state equals the
    standalone reduction over the same state."""
    torch, af, _ = env
    prob = W.shu_vortex_seeded(96)
    s = solver(env, prob)
    s.step(0.3 * prob.dx / s.max_speed())
    fused = s.max_speed()
    s.set_state(*s.get_state())  # invalidates the cached value: reduction kernel
    again = s.max_speed()
    assert abs(fused - again) <= 1e-6 * again


@pytest.mark.parametrize("tile_h", [4, 16])
def test_tile_height_does_not_change_the_result(env, tile_h):
    torch, af, _ = env
    prob = W.double_rarefaction(40, p=0.1)
    a, b = solver(env, prob), solver(env, prob, {"tile_h": tile_h})
    for _ in range(3):
        dt = 0.3 * prob.dx / a.max_speed()
        a.step(dt)
        b.step(dt)
    for x, y in zip(a.get_state(), b.get_state()):
        assert torch.equal(x, y)


@pytest.mark.parametrize("prob_name", ["vortex", "four_quadrant"])
def test_checkpoint_resume_is_bitwise(env, prob_name):
    """Checkpoint and restart: the state (af_get_state) and the averages' low
    words (af_get_avg_lo) of a run, loaded into a fresh handle (af_set_state,
    af_set_avg_lo), continue bit for bit as the original run does; without the
    low words the restarted run differs."""
    torch, af, _ = env
    prob = W.shu_vortex_seeded(96) if prob_name == "vortex" else W.four_quadrant(64, seed=2)
    a = solver(env, prob)
    dts = []
    for _ in range(5):
        dts.append(prob.cfl * min(prob.dx, prob.dy) / a.max_speed())
        a.step(dts[-1])
    ck = [t.clone() for t in a.get_state()]
    ck_lo = a.get_avg_lo().clone()
    a.status()  # clear the status bits of the steps before the checkpoint
    b = solver(env, prob, state=[t.cpu().numpy() for t in ck])
    b.set_avg_lo(ck_lo)
    c = solver(env, prob, state=[t.cpu().numpy() for t in ck])  # low words dropped
    for _ in range(5):
        dt = prob.cfl * min(prob.dx, prob.dy) / a.max_speed()
        for s in (a, b, c):
            s.step(dt)
    for x, y in zip(a.get_state(), b.get_state()):
        assert torch.equal(x, y)
    assert torch.equal(a.get_avg_lo(), b.get_avg_lo())
    assert not torch.equal(a.get_state()[0], c.get_state()[0]) or not torch.equal(a.get_avg_lo(), c.get_avg_lo())
    assert a.status() == b.status()
    for s in (a, b, c):
        s.close()


def test_node_flux_path_matches_the_three_level_flux_kernel(env):
    """With AF_OPT_NODE_FLUX the single-grid step writes each node's Simpson-in-
    time flux from the point-value kernel and the flux kernel reads those; a batch instance takes
    the other design (t^{n+1/2} written, fluxes formed from three levels in
    the flux kernel).  Both form every node flux with the same sequence of
    operations, so the states agree to FP32 round-off (the compilers may
    contract differently in the two kernels); the half level is refused unless
    it was kept."""
    torch, af, _ = env
    prob = W.fourier_smooth(45, 38, seed=31, lx=1.0, ly=0.84)
    st = W.to_f32(W.discretise(prob))
    s = solver(env, prob, {"node_flux": 1}, state=st)
    b = af.Batch([(prob.nx, prob.ny)], [(prob.dx, prob.dy)], bcs=[prob.bc])
    b.set_state(0, *to_dev(torch, st))
    hist = torch.zeros((4, 1), dtype=torch.float64, device="cuda")
    b.run(3, hist)
    for dt in hist[:3, 0].cpu().numpy():
        s.step(float(dt))
    assert s.status() == 0
    assert_parity(host(s.get_state()), host(b.get_state(0)), 1e-6, what="node fluxes vs three levels")
    with pytest.raises(af.AFError, match="KEEP_HALF"):
        s.get_half()
    b.close()
    s.close()
