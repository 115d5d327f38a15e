"""Cases run by tests/test_gpu_bounds.py in a process of their own, once with
the normal library and once with the checking build (AF_LIBRARY names it):
every kernel family of the step on small grids with all boundary kinds.
Writes the final states to an .npz file and, for the checking build, the
library's index-check report.

    python tests/bounds_cases.py OUT.npz
"""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

from paper_2508_06273_gb300 import af  # noqa: E402
from paper_2508_06273_gb300 import workloads as W  # noqa: E402


def dev(state):
    return [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda() for a in W.to_f32(state)]


def run_single(prob, steps, opts=None, cfl=0.3):
    o = dict(prob.options)
    o.update(opts or {})
    s = af.Solver(prob.nx, prob.ny, prob.dx, prob.dy, prob.gamma, prob.bc, options=o, inflow=prob.inflow)
    s.set_state(*dev(W.discretise(prob)))
    for _ in range(steps):
        s.step(cfl * min(prob.dx, prob.dy) / s.max_speed())
    out = [t.cpu().numpy() for t in s.get_state()] + [t.cpu().numpy() for t in s.get_half()]
    st = s.status()
    s.close()
    return out, st


def main(path):
    res, status = {}, {}
    cases = {
        "vortex_37x29_periodic": (W.fourier_smooth(37, 29, seed=3, lx=1.0, ly=0.78), 3, {}),
        "vortex_seeded_64": (W.shu_vortex_seeded(64), 3, {}),
        "alg1_tsw_ubar": (W.fourier_smooth(33, 41, seed=4, lx=0.8, ly=1.0), 2, {"lin_mode": 2, "tsw": 1, "ubar": 1}),
        "four_quadrant_47": (W.four_quadrant(47, seed=2), 4, {}),
        "double_rarefaction_40": (W.double_rarefaction(40), 4, {}),
        "shock_reflection_40x12": (W.shock_reflection(40, 12), 4, {}),
        "tile_16": (W.fourier_smooth(45, 35, seed=6, lx=1.0, ly=0.78), 2, {"tile_h": 16}),
        "tile_4": (W.fourier_smooth(45, 35, seed=6, lx=1.0, ly=0.78), 2, {"tile_h": 4}),
        "node_flux": (W.fourier_smooth(45, 35, seed=6, lx=1.0, ly=0.78), 2, {"node_flux": 1, "keep_half": 1}),
    }
    for name, (prob, steps, opts) in cases.items():
        arrs, st = run_single(prob, steps, opts)
        for k, a in enumerate(arrs):
            res[f"{name}_{k}"] = a
        status[name] = st
    # FP64 path
    prob = W.fourier_smooth(31, 23, seed=7, lx=1.0, ly=0.74)
    s = af.Solver(prob.nx, prob.ny, prob.dx, prob.dy, prob.gamma, prob.bc, options={"limiter": 0})
    s.set_option("fp64", 1)
    s.set_state_f64(*[torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda() for a in W.discretise(prob)])
    for _ in range(3):
        s.step(0.3 * prob.dx / s.max_speed())
    for k, t in enumerate(s.get_state_f64()):
        res[f"fp64_{k}"] = t.cpu().numpy()
    status["fp64"] = s.status()
    s.close()
    # batch of uneven grids, periodic and transmissive
    probs = [W.shu_vortex(24), W.four_quadrant(30, seed=1), W.fourier_smooth(40, 18, seed=2, lx=1.0, ly=0.45)]
    b = af.Batch([(p.nx, p.ny) for p in probs], [(p.dx, p.dy) for p in probs], bcs=[p.bc for p in probs],
                 options={"tsw": 1, "shock_blend": 1, "flux_limiter": 1, "node_bounds": 1})
    for k, p in enumerate(probs):
        b.set_state(k, *dev(W.discretise(p)))
    b.set_end(np.array([0.05, 0.01, 0.02]))
    b.run(12)
    for k in range(len(probs)):
        for q, t in enumerate(b.get_state(k)):
            res[f"batch{k}_{q}"] = t.cpu().numpy()
    status["batch"] = [int(x) for x in b.query()[3]]
    b.close()
    checking, word = af.debug_bounds()
    np.savez_compressed(path, **res)
    print(json.dumps({"checking": checking, "bounds": word, "status": status}))


if __name__ == "__main__":
    main(sys.argv[1])
