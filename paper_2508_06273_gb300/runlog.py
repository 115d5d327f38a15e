"""Run a Solver to a final time with a JSON-lines log and checkpoints.

The step itself runs in the library; this module only chooses dt from the
state's maximum wave speed (dt = cfl * min(dx, dy) / max speed, cut to land
on the final time), reads the library's diagnostics and writes them out.

Per logged step one JSON object: the step number, t and dt; the FP64
conserved totals and their drift from the totals at the start of the run
(relative to the L1 size of the starting averages, so that a vanishing total
has a defined drift); the minimum density and pressure of the state (cell
averages and all point values); the step's counters (EG1 and Lax-Friedrichs
fall-backs of Alg. 3, values kept at t^n, vertices flagged by Alg. 2); the
status bits seen since the previous log line; and, with the surrogate on,
how many node values came from the network and how many from the exact
fallback.

A checkpoint (numpy .npz) holds the state, the low words of the compensated
averages and (t, step, dt history), so that a run resumed from it repeats
the uninterrupted run bit for bit.
"""
from __future__ import annotations

import json

import numpy as np

_ARRAYS = ("avg", "vtx", "xe", "ye")


def save_checkpoint(path, solver, t, step, dt_hist):
    """Write the solver's state, the averages' low words and the run's clock."""
    state = [a.cpu().numpy() for a in solver.get_state()]
    lo = solver.get_avg_lo().cpu().numpy()
    np.savez(path, **dict(zip(_ARRAYS, state)), avg_lo=lo, t=np.float64(t), step=np.int64(step),
             dt=np.asarray(dt_hist, dtype=np.float64))


def load_checkpoint(path, solver):
    """Put a checkpoint's state into the solver; returns (t, step, dt history)."""
    import torch

    z = np.load(path)
    dev = solver.device
    solver.set_state(*[torch.from_numpy(np.ascontiguousarray(z[k])).to(dev) for k in _ARRAYS])
    solver.set_avg_lo(torch.from_numpy(np.ascontiguousarray(z["avg_lo"])).to(dev))
    return float(z["t"]), int(z["step"]), list(z["dt"])


def run(solver, t_end, cfl, h, log=None, every=1, t=0.0, step=0, dt_hist=None, max_steps=None,
        checkpoint=None, checkpoint_every=0, surrogate=False):
    """Advance solver from time t to t_end; returns (t, step, dt history).

    h: the cell size the CFL number refers to (min(dx, dy)); log: a path or an
    open text file for the JSON lines (None: no log); every: log every
    every-th step (and the last one); max_steps: stop after that many steps of
    this call; checkpoint: a path written every checkpoint_every steps and at
    the end."""
    out = open(log, "a") if isinstance(log, str) else log
    dt_hist = list(dt_hist or [])
    totals0 = solver.totals()
    scale = np.abs(totals0).sum() or 1.0
    n = 0
    try:
        while t < t_end * (1 - 1e-12) and (max_steps is None or n < max_steps):
            speed = solver.max_speed()
            if not np.isfinite(speed) or speed <= 0:
                if out:
                    out.write(json.dumps({"step": step, "t": t, "stopped": "wave speed not finite and positive",
                                          "speed": float(speed)}) + "\n")
                break
            dt = min(cfl * h / speed, t_end - t)
            solver.step(dt)
            t += dt
            step += 1
            n += 1
            dt_hist.append(dt)
            last = t >= t_end * (1 - 1e-12) or (max_steps is not None and n >= max_steps)
            if out and (step % every == 0 or last):
                status = solver.status()  # the bits of every step since the last read
                tot = solver.totals()
                rmin, pmin = solver.state_min()
                rec = {"step": step, "t": t, "dt": dt, "totals": tot.tolist(),
                       "drift": ((tot - totals0) / scale).tolist(), "min_rho": rmin, "min_p": pmin,
                       "counters": dict(zip(("eg1", "lf", "kept", "tsw"), solver.counters())),
                       "status": status}
                if surrogate:
                    net, exact = solver.surrogate_stats(reset=True)
                    rec["surrogate"] = {"network": int(net), "fallback": int(exact),
                                        "fallback_fraction": exact / max(net + exact, 1)}
                out.write(json.dumps(rec) + "\n")
            if checkpoint and checkpoint_every and step % checkpoint_every == 0:
                save_checkpoint(checkpoint, solver, t, step, dt_hist)
        if checkpoint:
            save_checkpoint(checkpoint, solver, t, step, dt_hist)
    finally:
        if out is not None and isinstance(log, str):
            out.close()
    return t, step, dt_hist
