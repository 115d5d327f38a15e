"""Thin ctypes binding of the C ABI in include/af.h (argument marshalling only).

Every numerical step runs in the CUDA kernels of libaf.so; this module only
passes pointers, sizes and streams.  PyTorch provides device memory and the
current CUDA stream.  The library must have been built
(``__graft_entry__.build()``); if it is missing, loading raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# AF_LIBRARY may name another build of the same library (the checking build of
# build.py, check_bounds=True); by default the in-tree libaf.so
LIB_PATH = os.environ.get("AF_LIBRARY") or os.path.join(_HERE, "_build", "libaf.so")
_LOCK = threading.Lock()
_LIB = None

BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTING, BC_INFLOW = 0, 1, 2, 3
OPT = {"lin_mode": 0, "tsw": 1, "limiter": 2, "correction": 3, "force_lo": 4, "profile": 5, "surrogate": 6,
       "surr_tol": 7, "surr_abs": 8,
       "flux_limiter": 9, "shock_blend": 10, "tile_h": 11, "node_bounds": 12, "ubar": 13, "test_timeout": 14, "keep_half": 15, "node_flux": 16, "fp64": 17,
       "surr_smooth": 18}
STAGES = ("prep", "pointvalue", "flux", "reduce")
ST_CFL, ST_AVG_NONPOS, ST_NONFINITE, ST_KEPT, ST_TIMEOUT, ST_STOPPED, ST_FLUX_LIMITED = 1, 2, 4, 8, 16, 32, 64
EXPORTS = [
    "af_create", "af_destroy", "af_last_error", "af_set_stream", "af_set_option",
    "af_get_option", "af_set_state", "af_set_state_host", "af_get_state", "af_get_state_host",
    "af_set_state_host_async", "af_get_state_host_async", "af_host_sync", "af_set_state_f64", "af_get_state_f64",
    "af_get_avg_lo", "af_set_avg_lo", "af_get_half", "af_step", "af_run", "af_status", "af_debug_bounds", "af_state_min",
    "af_counters", "af_conserved_totals", "af_max_speed", "af_profile",
    "af_conserved_totals_noalloc",
    "af_batch_create", "af_batch_destroy", "af_batch_set_option", "af_batch_set_state",
    "af_batch_get_state", "af_batch_set_end", "af_batch_run", "af_batch_query", "af_batch_counters",
    "af_batch_set_tile", "af_batch_autotune", "af_batch_active_cells", "af_batch_set_stream",
    "af_gemm_bf16",
    "af_mlp_create", "af_mlp_destroy", "af_mlp_set_params", "af_mlp_get_params", "af_mlp_fit_scales",
    "af_mlp_forward", "af_mlp_loss_grad", "af_mlp_train",
    "af_set_surrogate", "af_surrogate_stats", "af_batch_set_sampler", "af_set_inflow", "af_batch_set_inflow",
]
MLP_NPARAM, MLP_NTRAIN = 43480, 43408


class AFError(RuntimeError):
    pass


def lib():
    """Load libaf.so (raises if it has not been built)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            if not os.path.exists(LIB_PATH):
                raise AFError(f"{LIB_PATH} is missing: build the CUDA library first "
                              "(python -c 'import __graft_entry__ as g; g.build()')")
            L = C.CDLL(LIB_PATH)
            vp, i, d, fp = C.c_void_p, C.c_int, C.c_double, C.c_void_p
            sig = {
                "af_create": (vp, [i, i, d, d, d, C.c_uint32]),
                "af_debug_bounds": (i, [C.POINTER(C.c_uint)]),
                "af_state_min": (i, [vp, fp]),
                "af_destroy": (None, [vp]),
                "af_last_error": (C.c_char_p, []),
                "af_set_stream": (i, [vp, vp]),
                "af_set_option": (i, [vp, i, d]),
                "af_get_option": (i, [vp, i, C.POINTER(C.c_double)]),
                "af_set_state": (i, [vp, fp, fp, fp, fp, vp]),
                "af_set_state_host": (i, [vp, fp, fp, fp, fp]),
                "af_get_state": (i, [vp, fp, fp, fp, fp, vp]),
                "af_get_state_host": (i, [vp, fp, fp, fp, fp]),
                "af_set_state_host_async": (i, [vp, fp, fp, fp, fp]),
                "af_get_state_host_async": (i, [vp, fp, fp, fp, fp]),
                "af_host_sync": (i, [vp]),
                "af_set_state_f64": (i, [vp, fp, fp, fp, fp, vp]),
                "af_get_state_f64": (i, [vp, fp, fp, fp, fp, vp]),
                "af_get_avg_lo": (i, [vp, fp, vp]),
                "af_set_avg_lo": (i, [vp, fp, vp]),
                "af_get_half": (i, [vp, fp, fp, fp, vp]),
                "af_step": (i, [vp, d]),
                "af_run": (i, [vp, i, d]),
                "af_status": (i, [vp]),
                "af_counters": (i, [vp, C.POINTER(C.c_int64)]),
                "af_conserved_totals": (i, [vp, C.POINTER(C.c_double)]),
                "af_max_speed": (i, [vp, C.POINTER(C.c_float)]),
                "af_profile": (i, [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), i]),
                "af_conserved_totals_noalloc": (i, [fp, fp, i, i, d, d, fp, vp]),
                "af_batch_create": (vp, [i, fp, fp, fp, fp, d, fp]),
                "af_batch_destroy": (None, [vp]),
                "af_batch_set_option": (i, [vp, i, i, d]),
                "af_batch_set_state": (i, [vp, i, fp, fp, fp, fp, vp]),
                "af_batch_get_state": (i, [vp, i, fp, fp, fp, fp, vp]),
                "af_batch_set_end": (i, [vp, fp, d]),
                "af_batch_run": (i, [vp, i, fp, i]),
                "af_batch_query": (i, [vp, fp, fp, fp, fp]),
                "af_batch_counters": (i, [vp, fp]),
                "af_batch_set_tile": (i, [vp, i]),
                "af_batch_autotune": (i, [vp, C.POINTER(C.c_int), fp]),
                "af_batch_active_cells": (C.c_longlong, [vp]),
                "af_batch_set_stream": (i, [vp, vp]),
                "af_gemm_bf16": (i, [vp, i, vp, i, fp, i, i, i, i, fp, i, i, fp, vp]),
                "af_mlp_create": (vp, [C.c_uint64]),
                "af_mlp_destroy": (None, [vp]),
                "af_mlp_set_params": (i, [vp, fp]),
                "af_mlp_get_params": (i, [vp, fp]),
                "af_mlp_fit_scales": (i, [vp, fp, fp, C.c_longlong]),
                "af_mlp_forward": (i, [vp, fp, fp, i, vp]),
                "af_mlp_loss_grad": (i, [vp, fp, fp, i, C.POINTER(C.c_double), fp]),
                "af_mlp_train": (i, [vp, fp, fp, C.c_longlong, i, i, d, C.c_uint64, fp]),
                "af_set_surrogate": (i, [vp, vp, vp]),
                "af_surrogate_stats": (i, [vp, C.POINTER(C.c_int64), i]),
                "af_batch_set_sampler": (i, [vp, fp, fp, fp, i, fp, fp, fp, i, fp, C.c_uint64, d]),
                "af_set_inflow": (i, [vp, i, C.POINTER(C.c_double)]),
                "af_batch_set_inflow": (i, [vp, i, i, C.POINTER(C.c_double)]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _LIB = L
    return _LIB


def _check(rc):
    if rc < 0:
        raise AFError(f"af error {rc}: {lib().af_last_error().decode()}")
    return rc


BD_PLANE, BD_BOX, BD_RECORD, BD_RECORD64 = 1, 2, 4, 8


def debug_bounds():
    """(checking build?, AF_BD_* bits of the index checks that failed since
    the last call, on the current device); synchronises the device."""
    out = C.c_uint(0)
    rc = lib().af_debug_bounds(C.byref(out))
    if rc < 0:
        raise AFError(lib().af_last_error().decode())
    return bool(rc), int(out.value)


def bc_code(bc):
    if isinstance(bc, int):
        return bc
    a, b, c, d = bc
    return a | (b << 8) | (c << 16) | (d << 24)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class Solver:
    """One grid on one GPU (an af_ctx).  Work is enqueued on ``stream``
    (default: PyTorch's current stream at construction)."""

    def __init__(self, nx, ny, dx, dy, gamma=1.4, bc=(0, 0, 0, 0), stream=None, options=None, inflow=None):
        import torch

        self.torch = torch
        self.L = lib()
        self.nx, self.ny, self.dx, self.dy, self.gamma = nx, ny, dx, dy, gamma
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.h = self.L.af_create(nx, ny, dx, dy, gamma, bc_code(bc))
        if not self.h:
            raise AFError(self.L.af_last_error().decode())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        _check(self.L.af_set_stream(self.h, C.c_void_p(self.stream.cuda_stream)))
        for k, v in (options or {}).items():
            self.set_option(k, v)
        for side, U in (inflow or {}).items():
            self.set_inflow(side, U)

    def set_inflow(self, side, U):
        """Primitive inflow state of side 0..3 (xlo, xhi, ylo, yhi)."""
        u = (C.c_double * 4)(*[float(x) for x in U])
        _check(self.L.af_set_inflow(self.h, int(side), u))

    def close(self):
        if getattr(self, "h", None):
            self.L.af_destroy(self.h)
            self.h = None

    __del__ = close

    def shapes(self):
        nx, ny = self.nx, self.ny
        return (4, ny, nx), (4, ny + 1, nx + 1), (4, ny, nx + 1), (4, ny + 1, nx)

    def _s(self):
        return C.c_void_p(self.stream.cuda_stream)

    def set_option(self, key, value):
        _check(self.L.af_set_option(self.h, OPT[key] if isinstance(key, str) else key, float(value)))

    def set_state(self, avg, vtx, xe, ye):
        """State from CUDA float32 tensors (device) or numpy arrays (host)."""
        arrs = (avg, vtx, xe, ye)
        if all(isinstance(a, np.ndarray) for a in arrs):
            hs = [np.ascontiguousarray(a, dtype=np.float32) for a in arrs]
            for a, s in zip(hs, self.shapes()):
                if a.shape != s:
                    raise ValueError(f"shape {a.shape} != {s}")
            _check(self.L.af_set_state_host(self.h, *[C.c_void_p(a.ctypes.data) for a in hs]))
            return
        ts = []
        for a, s in zip(arrs, self.shapes()):
            if tuple(a.shape) != s or a.dtype != self.torch.float32 or not a.is_cuda:
                raise ValueError(f"need CUDA float32 tensors of shape {s}")
            ts.append(a.contiguous())
        _check(self.L.af_set_state(self.h, *[_ptr(t) for t in ts], self._s()))

    def set_state_f64(self, avg, vtx, xe, ye):
        """State of a handle in FP64 mode from CUDA float64 tensors."""
        ts = []
        for a, s in zip((avg, vtx, xe, ye), self.shapes()):
            if tuple(a.shape) != s or a.dtype != self.torch.float64 or not a.is_cuda:
                raise ValueError(f"need CUDA float64 tensors of shape {s}")
            ts.append(a.contiguous())
        _check(self.L.af_set_state_f64(self.h, *[_ptr(t) for t in ts], self._s()))

    def get_state_f64(self):
        """Current state of a handle in FP64 mode as CUDA float64 tensors."""
        out = [self.torch.empty(s, dtype=self.torch.float64, device=self.device) for s in self.shapes()]
        _check(self.L.af_get_state_f64(self.h, *[_ptr(t) for t in out], self._s()))
        return tuple(out)

    def get_state(self):
        """Current state as CUDA float32 tensors."""
        out = [self.torch.empty(s, dtype=self.torch.float32, device=self.device) for s in self.shapes()]
        _check(self.L.af_get_state(self.h, *[_ptr(t) for t in out], self._s()))
        return tuple(out)

    def get_state_host(self, out=None):
        """Current state copied into host numpy arrays (optionally pre-allocated)."""
        out = out or [np.empty(s, dtype=np.float32) for s in self.shapes()]
        _check(self.L.af_get_state_host(self.h, *[C.c_void_p(a.ctypes.data) for a in out]))
        return tuple(out)

    def set_state_host_async(self, avg, vtx, xe, ye):
        """Enqueue the upload of a state held in host numpy arrays (pinned
        memory for overlap); the arrays must stay untouched until host_sync()."""
        arrs = (avg, vtx, xe, ye)
        for a, s in zip(arrs, self.shapes()):
            if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.shape == s
                    and a.flags["C_CONTIGUOUS"]):
                raise ValueError(f"need C-contiguous float32 arrays of shape {s}")
        _check(self.L.af_set_state_host_async(self.h, *[C.c_void_p(a.ctypes.data) for a in arrs]))

    def get_state_host_async(self, out):
        """Enqueue the download of the current state into host numpy arrays
        (pinned memory for overlap); their contents are valid after host_sync()."""
        for a, s in zip(out, self.shapes()):
            if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.shape == s
                    and a.flags["C_CONTIGUOUS"] and a.flags["WRITEABLE"]):
                raise ValueError(f"need writeable C-contiguous float32 arrays of shape {s}")
        _check(self.L.af_get_state_host_async(self.h, *[C.c_void_p(a.ctypes.data) for a in out]))

    def host_sync(self):
        """Wait for the asynchronous host transfers."""
        _check(self.L.af_host_sync(self.h))

    def get_avg_lo(self):
        t = self.torch.empty(self.shapes()[0], dtype=self.torch.float32, device=self.device)
        _check(self.L.af_get_avg_lo(self.h, _ptr(t), self._s()))
        return t

    def set_avg_lo(self, t):
        _check(self.L.af_set_avg_lo(self.h, _ptr(t.contiguous()), self._s()))

    def get_half(self):
        out = [self.torch.empty(s, dtype=self.torch.float32, device=self.device) for s in self.shapes()[1:]]
        _check(self.L.af_get_half(self.h, *[_ptr(t) for t in out], self._s()))
        return tuple(out)

    def step(self, dt):
        _check(self.L.af_step(self.h, float(dt)))

    def run(self, nsteps, dt):
        _check(self.L.af_run(self.h, int(nsteps), float(dt)))

    def status(self):
        return _check(self.L.af_status(self.h))

    def counters(self):
        out = (C.c_int64 * 4)()
        _check(self.L.af_counters(self.h, out))
        return list(out)

    def totals(self):
        out = (C.c_double * 4)()
        _check(self.L.af_conserved_totals(self.h, out))
        return np.array(list(out))

    def profile(self, reset=False):
        """(ms per stage, kernel launches per stage) since the last reset."""
        ms, n = (C.c_double * 4)(), (C.c_int64 * 4)()
        _check(self.L.af_profile(self.h, ms, n, 1 if reset else 0))
        return dict(zip(STAGES, list(ms))), dict(zip(STAGES, list(n)))

    def max_speed(self):
        out = C.c_float()
        _check(self.L.af_max_speed(self.h, C.byref(out)))
        return out.value

    def state_min(self):
        """(min rho, min p) over the primitive averages and all point values
        (NaN, NaN if a value is not finite)."""
        out = (C.c_float * 2)()
        _check(self.L.af_state_min(self.h, out))
        return float(out[0]), float(out[1])

    def set_surrogate(self, vertex_net, edge_net, tol=None):
        """Attach networks (Mlp) and switch the surrogate on (None, None: off)."""
        self._nets = (vertex_net, edge_net)  # keep them alive while attached
        _check(self.L.af_set_surrogate(self.h, vertex_net.h if vertex_net else None,
                                       edge_net.h if edge_net else None))
        if vertex_net:
            if tol is not None:
                self.set_option("surr_tol", tol)
            self.set_option("surrogate", 1)

    def surrogate_stats(self, reset=False):
        """(nodes from the network, nodes from the exact fallback)."""
        out = (C.c_int64 * 2)()
        _check(self.L.af_surrogate_stats(self.h, out, 1 if reset else 0))
        return out[0], out[1]


def _shapes(nx, ny):
    return (4, ny, nx), (4, ny + 1, nx + 1), (4, ny, nx + 1), (4, ny + 1, nx)


class Batch:
    """An ensemble of independent grids (an af_batch) advanced together by
    batched kernels, each instance with its own device-side time step."""

    def __init__(self, sizes, spacings, gamma=1.4, bcs=None, stream=None, options=None):
        import torch

        self.torch = torch
        self.L = lib()
        self.n = len(sizes)
        self.sizes = [(int(a), int(b)) for a, b in sizes]
        self.spacings = [(float(a), float(b)) for a, b in spacings]
        bcs = bcs or [(0, 0, 0, 0)] * self.n
        nx = np.array([s[0] for s in self.sizes], dtype=np.int32)
        ny = np.array([s[1] for s in self.sizes], dtype=np.int32)
        dx = np.array([s[0] for s in self.spacings], dtype=np.float64)
        dy = np.array([s[1] for s in self.spacings], dtype=np.float64)
        bc = np.array([bc_code(b) for b in bcs], dtype=np.uint32)
        self._keep = (nx, ny, dx, dy, bc)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.h = self.L.af_batch_create(self.n, *[C.c_void_p(a.ctypes.data) for a in (nx, ny, dx, dy)],
                                        float(gamma), C.c_void_p(bc.ctypes.data))
        if not self.h:
            raise AFError(self.L.af_last_error().decode())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        _check(self.L.af_batch_set_stream(self.h, C.c_void_p(self.stream.cuda_stream)))
        for k, v in (options or {}).items():
            self.set_option(k, v)

    def close(self):
        if getattr(self, "h", None):
            self.L.af_batch_destroy(self.h)
            self.h = None

    __del__ = close

    def _s(self):
        return C.c_void_p(self.stream.cuda_stream)

    def set_option(self, key, value, k=-1):
        """Option of instance k (all instances if k = -1)."""
        _check(self.L.af_batch_set_option(self.h, int(k), OPT[key] if isinstance(key, str) else key,
                                          float(value)))

    def set_inflow(self, k, side, U):
        u = (C.c_double * 4)(*[float(x) for x in U])
        _check(self.L.af_batch_set_inflow(self.h, int(k), int(side), u))

    def set_state(self, k, avg, vtx, xe, ye):
        ts = []
        for a, s in zip((avg, vtx, xe, ye), _shapes(*self.sizes[k])):
            if tuple(a.shape) != s or a.dtype != self.torch.float32 or not a.is_cuda:
                raise ValueError(f"need CUDA float32 tensors of shape {s}")
            ts.append(a.contiguous())
        _check(self.L.af_batch_set_state(self.h, k, *[_ptr(t) for t in ts], self._s()))

    def get_state(self, k):
        out = [self.torch.empty(s, dtype=self.torch.float32, device=self.device)
               for s in _shapes(*self.sizes[k])]
        _check(self.L.af_batch_get_state(self.h, k, *[_ptr(t) for t in out], self._s()))
        return tuple(out)

    def set_end(self, t_end, cfl=0.3):
        te = np.ascontiguousarray(np.broadcast_to(np.asarray(t_end, dtype=np.float64), (self.n,)))
        _check(self.L.af_batch_set_end(self.h, C.c_void_p(te.ctypes.data), float(cfl)))

    def run(self, nsteps, hist=None):
        """Advance up to nsteps steps; hist: optional CUDA float64 tensor
        [steps, n] that receives each instance's dt per step."""
        hp, hs = (None, 0) if hist is None else (_ptr(hist), int(hist.shape[0]))
        _check(self.L.af_batch_run(self.h, int(nsteps), hp, hs))

    def query(self):
        """(t, steps, active, status) per instance; clears the status words."""
        t = np.zeros(self.n, dtype=np.float64)
        st, ac, ss = (np.zeros(self.n, dtype=np.int32) for _ in range(3))
        _check(self.L.af_batch_query(self.h, *[C.c_void_p(a.ctypes.data) for a in (t, st, ac, ss)]))
        return t, st, ac, ss

    def counters(self):
        out = np.zeros((self.n, 4), dtype=np.int64)
        _check(self.L.af_batch_counters(self.h, C.c_void_p(out.ctypes.data)))
        return out

    def set_tile(self, tile_h):
        _check(self.L.af_batch_set_tile(self.h, int(tile_h)))

    def autotune(self):
        """Pick the fastest point-value tile height; returns (height, {height: ms})."""
        th, ms = C.c_int(), np.zeros(3, dtype=np.float64)
        _check(self.L.af_batch_autotune(self.h, C.byref(th), C.c_void_p(ms.ctypes.data)))
        return th.value, dict(zip((4, 8, 16), ms.tolist()))

    def active_cells(self):
        return _check(self.L.af_batch_active_cells(self.h))

    def set_sampler(self, cap_v, cap_e, seed=1, rate=0.01):
        """Collect surrogate training samples (features, targets, ids) into
        device tensors held by this object; returns them as a dict."""
        t = self.torch
        dev = self.device
        self._samples = {
            "Xv": t.zeros((cap_v, 64), dtype=t.float32, device=dev), "Tv": t.zeros((cap_v, 8), dtype=t.float32, device=dev),
            "idv": t.zeros((cap_v, 4), dtype=t.int32, device=dev),
            "Xe": t.zeros((cap_e, 64), dtype=t.float32, device=dev), "Te": t.zeros((cap_e, 8), dtype=t.float32, device=dev),
            "ide": t.zeros((cap_e, 4), dtype=t.int32, device=dev),
            "counts": t.zeros(2, dtype=t.int32, device=dev)}
        S = self._samples
        _check(self.L.af_batch_set_sampler(self.h, _ptr(S["Xv"]), _ptr(S["Tv"]), _ptr(S["idv"]), int(cap_v),
                                           _ptr(S["Xe"]), _ptr(S["Te"]), _ptr(S["ide"]), int(cap_e),
                                           _ptr(S["counts"]), int(seed), float(rate)))
        return S

    def stop_sampler(self):
        _check(self.L.af_batch_set_sampler(self.h, None, None, None, 0, None, None, None, 0, None, 0, 0.0))

    def samples(self):
        """(Xv, Tv, idv, Xe, Te, ide) trimmed to the rows filled so far."""
        S = self._samples
        self.torch.cuda.synchronize()
        nv, ne = (min(int(c), cap) for c, cap in zip(S["counts"].tolist(), (S["Xv"].shape[0], S["Xe"].shape[0])))
        return S["Xv"][:nv], S["Tv"][:nv], S["idv"][:nv], S["Xe"][:ne], S["Te"][:ne], S["ide"][:ne]


class Mlp:
    """The surrogate network (an af_mlp) on the current CUDA device."""

    def __init__(self, seed=1):
        import torch

        self.torch = torch
        self.L = lib()
        self.h = self.L.af_mlp_create(int(seed))
        if not self.h:
            raise AFError(self.L.af_last_error().decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.af_mlp_destroy(self.h)
            self.h = None

    __del__ = close

    def get_params(self):
        out = np.zeros(MLP_NPARAM, dtype=np.float32)
        _check(self.L.af_mlp_get_params(self.h, C.c_void_p(out.ctypes.data)))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.shape != (MLP_NPARAM,):
            raise ValueError(f"need {MLP_NPARAM} floats")
        _check(self.L.af_mlp_set_params(self.h, C.c_void_p(p.ctypes.data)))

    def fit_scales(self, X, T):
        _check(self.L.af_mlp_fit_scales(self.h, _ptr(X.contiguous()), _ptr(T.contiguous()), X.shape[0]))

    def forward(self, X):
        """(n, 8) outputs for CUDA float32 features X (n, 64)."""
        X = X.contiguous()
        Y = self.torch.empty((X.shape[0], 8), dtype=self.torch.float32, device=X.device)
        _check(self.L.af_mlp_forward(self.h, _ptr(X), _ptr(Y), X.shape[0],
                                     C.c_void_p(self.torch.cuda.current_stream().cuda_stream)))
        return Y

    def loss_grad(self, X, T):
        """(loss, gradient of the trained parameters as a float32 array)."""
        loss = C.c_double()
        g = np.zeros(MLP_NTRAIN, dtype=np.float32)
        self.torch.cuda.synchronize()
        _check(self.L.af_mlp_loss_grad(self.h, _ptr(X.contiguous()), _ptr(T.contiguous()), X.shape[0],
                                       C.byref(loss), C.c_void_p(g.ctypes.data)))
        return loss.value, g

    def train(self, X, T, steps, batch=8192, lr=1e-3, seed=1):
        """Adam steps on minibatches of (X, T); returns the loss per step."""
        hist = np.zeros(max(steps, 1), dtype=np.float32)
        self.torch.cuda.synchronize()
        _check(self.L.af_mlp_train(self.h, _ptr(X.contiguous()), _ptr(T.contiguous()), X.shape[0], int(steps),
                                   int(batch), float(lr), int(seed), C.c_void_p(hist.ctypes.data)))
        return hist[:steps]
