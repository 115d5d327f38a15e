"""ctypes binding of the FP64 C oracle (afo.c) -- TEST INFRASTRUCTURE ONLY.

The shared object is compiled with gcc on first use (or by ``build()``) into
``oracle/_build/``; nothing else is needed.  Arrays are numpy float64 in the
layout of afo.h: averages (4, ny, nx), vertices (4, ny+1, nx+1), x-edge
midpoints (4, ny, nx+1), y-edge midpoints (4, ny+1, nx).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "afo.c")
_HDR = os.path.join(_HERE, "afo.h")
_OUT = os.path.join(_HERE, "_build", "libafo.so")
_LOCK = threading.Lock()
_LIB = None

VTX, XE, YE = 0, 1, 2
BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTING, BC_INFLOW = 0, 1, 2, 3
OPT_LIN_MODE, OPT_TSW, OPT_LIMITER, OPT_CORRECTION, OPT_FORCE_LO, OPT_THREADS = 0, 1, 2, 3, 4, 16
OPT_FLUX_LIMITER, OPT_SHOCK_BLEND, OPT_NODE_BOUNDS, OPT_UBAR = 9, 10, 12, 13
ST_FLUX_LIMITED = 64
ST_CFL, ST_AVG_NONPOS, ST_NONFINITE, ST_KEPT = 1, 2, 4, 8


def build(force: bool = False) -> str:
    """Compile afo.c into oracle/_build/libafo.so (gcc, OpenMP, no FP contraction)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < newest:
        tmp = _OUT + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
    return _OUT


_dp = C.POINTER(C.c_double)
FIELD_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_double, C.c_double, _dp)


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = C.CDLL(build())
            vp, i, d = C.c_void_p, C.c_int, C.c_double
            sig = {
                "afo_create": (vp, [i, i, d, d, d, C.c_uint32]),
                "afo_destroy": (None, [vp]),
                "afo_set_option": (i, [vp, i, d]),
                "afo_set_state": (i, [vp, _dp, _dp, _dp, _dp]),
                "afo_get_state": (i, [vp, _dp, _dp, _dp, _dp]),
                "afo_get_half": (i, [vp, _dp, _dp, _dp]),
                "afo_step": (i, [vp, d]),
                "afo_conserved_totals": (i, [vp, _dp]),
                "afo_max_speed": (d, [vp]),
                "afo_status": (i, [vp]),
                "afo_counters": (i, [vp, C.POINTER(C.c_int64)]),
                "afo_prepare": (i, [vp]),
                "afo_cell_prim": (i, [vp, i, i, _dp, _dp]),
                "afo_recon_eval": (i, [vp, i, i, d, d, _dp]),
                "afo_node_eg": (i, [vp, i, i, i, i, _dp, d, _dp]),
                "afo_node_lf": (i, [vp, i, i, i, d, _dp]),
                "afo_node_corr": (i, [vp, i, i, i, _dp]),
                "afo_correction_T": (None, [_dp, _dp, _dp, d, _dp]),
                "afo_eg_field": (i, [FIELD_FN, vp, i, d, d, _dp, d, d, _dp]),
                "afo_set_quadrature": (None, [i, d]),
                "afo_shock_theta": (d, [vp, i, i, i]),
                "afo_set_inflow": (i, [vp, i, _dp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = lib
    return _LIB


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _vec(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(4))


def bc_code(bc) -> int:
    if isinstance(bc, int):
        return bc
    xlo, xhi, ylo, yhi = bc
    return xlo | (xhi << 8) | (ylo << 16) | (yhi << 24)


class Oracle:
    """One FP64 grid; mirrors the library's af_* interface on host arrays."""

    def __init__(self, nx, ny, dx, dy, gamma=1.4, bc=(0, 0, 0, 0)):
        self.lib = _lib()
        self.nx, self.ny, self.dx, self.dy, self.gamma = nx, ny, dx, dy, gamma
        self.h = self.lib.afo_create(nx, ny, dx, dy, gamma, bc_code(bc))
        if not self.h:
            raise ValueError("afo_create rejected the arguments")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.afo_destroy(h)
            self.h = None

    def shapes(self):
        nx, ny = self.nx, self.ny
        return (4, ny, nx), (4, ny + 1, nx + 1), (4, ny, nx + 1), (4, ny + 1, nx)

    def set_option(self, key, val):
        if self.lib.afo_set_option(self.h, key, float(val)) != 0:
            raise ValueError(f"bad option {key}={val}")

    def set_state(self, avg, vtx, xe, ye):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (avg, vtx, xe, ye)]
        for a, s in zip(arrs, self.shapes()):
            if a.shape != s:
                raise ValueError(f"shape {a.shape} != {s}")
        if self.lib.afo_set_state(self.h, *[_p(a) for a in arrs]) != 0:
            raise ValueError("afo_set_state rejected the state (periodic duplicate lines?)")

    def get_state(self):
        arrs = [np.empty(s) for s in self.shapes()]
        self.lib.afo_get_state(self.h, *[_p(a) for a in arrs])
        return tuple(arrs)

    def get_half(self):
        arrs = [np.empty(s) for s in self.shapes()[1:]]
        self.lib.afo_get_half(self.h, *[_p(a) for a in arrs])
        return tuple(arrs)

    def step(self, dt):
        if self.lib.afo_step(self.h, float(dt)) != 0:
            raise ValueError("afo_step rejected dt")

    def totals(self):
        out = np.empty(4)
        self.lib.afo_conserved_totals(self.h, _p(out))
        return out

    def max_speed(self):
        return self.lib.afo_max_speed(self.h)

    def status(self):
        return self.lib.afo_status(self.h)

    def set_inflow(self, side, U):
        """Primitive inflow state of side 0..3 (xlo, xhi, ylo, yhi)."""
        u = np.ascontiguousarray(U, dtype=np.float64)
        if self.lib.afo_set_inflow(self.h, int(side), _p(u)) != 0:
            raise ValueError("afo_set_inflow rejected the state")

    def shock_theta(self, kind, i, j):
        """Sec. 3.4 blend weight of a node from the current Ubar (after prepare())."""
        return self.lib.afo_shock_theta(self.h, kind, i, j)

    def counters(self):
        out = (C.c_int64 * 4)()
        self.lib.afo_counters(self.h, out)
        return list(out)

    # --- unit-level hooks for the pin tests
    def prepare(self):
        self.lib.afo_prepare(self.h)

    def cell_prim(self, i, j):
        uc, ub = np.empty(4), np.empty(4)
        if self.lib.afo_cell_prim(self.h, i, j, _p(uc), _p(ub)) != 0:
            raise IndexError((i, j))
        return uc, ub

    def recon(self, i, j, xi, eta):
        out = np.empty(4)
        if self.lib.afo_recon_eval(self.h, i, j, float(xi), float(eta), _p(out)) != 0:
            raise IndexError((i, j))
        return out

    def node_eg(self, kind, i, j, op, ulin, tau):
        out = np.empty(4)
        u = _vec(ulin)
        self.lib.afo_node_eg(self.h, kind, i, j, op, _p(u), float(tau), _p(out))
        return out

    def node_lf(self, kind, i, j, tau):
        out = np.empty(4)
        self.lib.afo_node_lf(self.h, kind, i, j, float(tau), _p(out))
        return out

    def node_corr(self, kind, i, j):
        out = np.empty(4)
        self.lib.afo_node_corr(self.h, kind, i, j, _p(out))
        return out


def correction_T(U, Ux, Uy, gamma=1.4):
    out = np.empty(4)
    a, b, c = _vec(U), _vec(Ux), _vec(Uy)
    _lib().afo_correction_T(_p(a), _p(b), _p(c), float(gamma), _p(out))
    return out


def eg_field(fn, op, xbar, ybar, ulin, tau, gamma=1.4):
    """EG2 (op=0) or EG1 (op=1) of a smooth field fn(x, y) -> 4 primitive values."""

    def cb(_user, x, y, out):
        v = fn(x, y)
        for k in range(4):
            out[k] = float(v[k])

    cfn = FIELD_FN(cb)
    out = np.empty(4)
    u = _vec(ulin)
    _lib().afo_eg_field(cfn, None, op, float(xbar), float(ybar), _p(u), float(tau),
                        float(gamma), _p(out))
    return out


def set_quadrature(npts=12, max_piece=np.pi / 2):
    _lib().afo_set_quadrature(int(npts), float(max_piece))
