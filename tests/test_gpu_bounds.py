"""The checking build (AF_CHECK_BOUNDS: index checks in the kernels, new
state filled with NaN; build.py check_bounds=True) on every kernel family of
the step: no index check fails, every result is finite (no kernel reads a
point that no call wrote: a NaN would show), and the results agree with the
normal build's to a few units in the last place (the checks change how the
compiler schedules, and so contracts, some of the arithmetic)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _run(out, lib=None):
    env = dict(os.environ, PYTHONPATH=ROOT)
    env.pop("AF_LIBRARY", None)
    if lib:
        env["AF_LIBRARY"] = lib
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_cases.py"), str(out)], env=env,
                       capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1]), np.load(out)


def test_checking_build_finds_no_bad_index_and_changes_nothing(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    from paper_2508_06273_gb300 import build

    __graft_entry__.build()
    checking_lib = build.build(check_bounds=True)
    rep0, plain = _run(tmp_path / "plain.npz")
    rep1, checked = _run(tmp_path / "checked.npz", checking_lib)
    assert rep0["checking"] is False and rep0["bounds"] == 0
    assert rep1["checking"] is True
    assert rep1["bounds"] == 0, f"failed index checks, AF_BD_* bits {rep1['bounds']:#x}"
    assert rep1["status"] == rep0["status"]
    assert sorted(plain.files) == sorted(checked.files)
    for k in plain.files:
        a, b = plain[k], checked[k]
        assert np.all(np.isfinite(b)), k
        scale = max(float(np.max(np.abs(a))), 1.0)
        assert np.max(np.abs(a - b)) <= 1e-5 * scale, (k, float(np.max(np.abs(a - b))))
