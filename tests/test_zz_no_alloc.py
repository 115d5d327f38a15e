"""af_conserved_totals_noalloc: conserved totals without any allocation by
the library, for callers that cannot allocate at the point of the call (a
stepping loop that must not take cudaFree's device-wide synchronisation, or
memory owned by another allocator).  Compared through the C ABI with
af_conserved_totals of a handle holding the same state, on two calls in a
row; calls after the first leave the device's free memory unchanged; host
pointers are rejected.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from paper_2508_06273_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-13  # relative to sum |Q|; the two reductions differ only in summation order


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def test_totals_without_allocation_match_the_handle_totals():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2508_06273_gb300 import af

    L = af.lib()
    prob = W.fourier_smooth(96, 70, seed=13, lx=1.0, ly=0.75)
    st = [torch.from_numpy(np.asarray(a, dtype=np.float32)).cuda() for a in W.discretise(prob)]
    s = af.Solver(prob.nx, prob.ny, prob.dx, prob.dy, prob.gamma, prob.bc)
    s.set_state(*st)
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        if call == 1:
            dt = 0.3 * prob.dx / s.max_speed()
            for _ in range(3):
                s.step(dt)
        avg, lo = s.get_state()[0], s.get_avg_lo()
        rc = L.af_conserved_totals_noalloc(_ptr(avg), _ptr(lo), prob.nx, prob.ny, prob.dx, prob.dy,
                                           _ptr(out), stream)
        assert rc == 0, L.af_last_error().decode()
        got = out.cpu().numpy()
        want = s.totals()
        scale = (avg.double().abs().sum(dim=(1, 2)) * prob.dx * prob.dy).cpu().numpy()
        assert np.all(np.abs(got - want) <= TOL * scale), (call, got, want)
    # the same input twice gives the same bits (fixed-order reduction)
    first = out.clone()
    rc = L.af_conserved_totals_noalloc(_ptr(avg), _ptr(lo), prob.nx, prob.ny, prob.dx, prob.dy,
                                       _ptr(out), stream)
    assert rc == 0 and torch.equal(first, out)
    s.close()


def test_calls_after_the_first_allocate_nothing():
    """After the first call on the device (which loads the entry point's
    device code and its static array), further calls leave the device's free
    memory unchanged: nothing is allocated."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2508_06273_gb300 import af

    L = af.lib()
    nx, ny = 300, 211
    avg = torch.rand((4, ny, nx), dtype=torch.float32, device="cuda")
    lo = torch.rand((4, ny, nx), dtype=torch.float32, device="cuda") * 1e-7
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    args = (_ptr(avg), _ptr(lo), nx, ny, 0.01, 0.02, _ptr(out), None)
    assert L.af_conserved_totals_noalloc(*args) == 0  # set-up call
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert L.af_conserved_totals_noalloc(*args) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    want = (avg.double() + lo.double()).sum(dim=(1, 2)) * 0.01 * 0.02
    assert torch.allclose(out, want, rtol=1e-12, atol=0)


def test_host_or_foreign_pointers_are_rejected_before_any_launch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_06273_gb300 import af

    L = af.lib()
    avg = torch.ones((4, 3, 5), dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    host_out = np.full(4, 7.0)
    rc = L.af_conserved_totals_noalloc(_ptr(avg), None, 5, 3, 1.0, 1.0, C.c_void_p(host_out.ctypes.data), None)
    assert rc == -1 and b"out" in L.af_last_error()
    assert np.all(host_out == 7.0)
    host_lo = np.zeros((4, 3, 5), dtype=np.float32)
    rc = L.af_conserved_totals_noalloc(_ptr(avg), C.c_void_p(host_lo.ctypes.data), 5, 3, 1.0, 1.0, _ptr(out),
                                       None)
    assert rc == -1 and b"avg_lo" in L.af_last_error()
    torch.cuda.synchronize()
    assert torch.count_nonzero(out) == 0


def test_rows_beyond_the_static_limit_are_rejected():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_06273_gb300 import af

    L = af.lib()
    avg = torch.zeros((4, 2, 2), dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    too_many = 16384 + 1
    rc = L.af_conserved_totals_noalloc(_ptr(avg), None, 2, too_many, 1.0, 1.0, _ptr(out), None)
    assert rc == -1 and b"16384" in L.af_last_error()
    assert torch.count_nonzero(out) == 0
