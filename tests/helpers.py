"""Shared test helpers: run the FP64 oracle on a workload, norms, restriction."""
import numpy as np

from paper_2508_06273_gb300 import workloads as W

OPTS = {"lin_mode": 0, "tsw": 1, "limiter": 2, "correction": 3, "force_lo": 4, "flux_limiter": 9,
        "shock_blend": 10, "node_bounds": 12, "ubar": 13}


def make_oracle(oracle, prob, opts=None, state=None):
    o = oracle.Oracle(prob.nx, prob.ny, prob.dx, prob.dy, prob.gamma, prob.bc)
    merged = dict(prob.options)
    merged.update(opts or {})
    for k, v in merged.items():
        o.set_option(OPTS[k] if isinstance(k, str) else k, v)
    for side, U in getattr(prob, "inflow", {}).items():
        o.set_inflow(side, U)
    o.set_state(*(state if state is not None else W.discretise(prob)))
    return o


def run_oracle(oracle, prob, opts=None, t_end=None, state=None, max_steps=10 ** 9):
    o = make_oracle(oracle, prob, opts, state)
    t, n, t_end = 0.0, 0, prob.t_end if t_end is None else t_end
    while t < t_end * (1 - 1e-12) and n < max_steps:
        dt = min(prob.cfl * min(prob.dx, prob.dy) / o.max_speed(), t_end - t)
        o.step(dt)
        t += dt
        n += 1
    return o, n


def restrict2(a):
    """2x2 averaging of cell arrays (..., 2ny, 2nx) -> (..., ny, nx)."""
    return 0.25 * (a[..., 0::2, 0::2] + a[..., 1::2, 0::2] + a[..., 0::2, 1::2] + a[..., 1::2, 1::2])


def rel_l1(a, b):
    """max over variables of sum|a-b| / sum|b| (over the given arrays)."""
    out = 0.0
    for v in range(4):
        num = sum(np.abs(x[v] - y[v]).sum() for x, y in zip(a, b))
        den = sum(np.abs(y[v]).sum() for y in b)
        out = max(out, num / den)
    return out


def read_table(path):
    rows = []
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([float(x) for x in line.split()])
    return np.array(rows)
