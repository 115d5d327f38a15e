"""NVTX ranges of the host API: a small NVTX injection library
(tests/nvtx_record.c, loaded through NVTX_INJECTION64_PATH) records the
ranges that af_step, af_run and af_batch_run open, and the step's stages
inside them, with every push matched by a pop."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_api_calls_and_stages_open_nvtx_ranges(tmp_path):
    so = tmp_path / "libnvtx_record.so"
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    subprocess.run(["gcc", "-shared", "-fPIC", "-I", cuda_inc, "-o", str(so), os.path.join(HERE, "nvtx_record.c")],
                   check=True)
    log = tmp_path / "ranges.txt"
    prog = textwrap.dedent("""
        import numpy as np, torch
        from paper_2508_06273_gb300 import af, workloads as W
        p = W.shu_vortex(32)
        s = af.Solver(p.nx, p.ny, p.dx, p.dy, p.gamma, p.bc)
        s.set_state(*[torch.from_numpy(np.asarray(a, dtype=np.float32)).cuda() for a in W.discretise(p)])
        s.step(0.01)
        s.run(6, 0.01)
        qs = [W.shu_vortex(16), W.shu_vortex(24)]
        b = af.Batch([(q.nx, q.ny) for q in qs], [(q.dx, q.dy) for q in qs], bcs=[q.bc for q in qs])
        for k, q in enumerate(qs):
            b.set_state(k, *[torch.from_numpy(np.asarray(a, dtype=np.float32)).cuda() for a in W.discretise(q)])
        b.set_end(0.05)
        b.run(4)
        torch.cuda.synchronize()
        print("done")
    """)
    env = dict(os.environ, NVTX_INJECTION64_PATH=str(so), AF_NVTX_LOG=str(log), PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", prog], env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0 and "done" in r.stdout, r.stderr[-2000:]
    lines = log.read_text().splitlines()
    pushes = [ln[5:] for ln in lines if ln.startswith("push ")]
    assert len(pushes) == sum(ln == "pop" for ln in lines)
    for name in ("af_step", "ghost fill", "point values", "flux update", "af_run", "af_run/capture", "af_batch_run"):
        assert name in pushes, (name, sorted(set(pushes)))
    # one step: its three stages nest inside af_step
    k = pushes.index("af_step")
    assert pushes[k + 1:k + 4] == ["ghost fill", "point values", "flux update"]
