"""Seeded, synthetic initial data for the Active Flux solver and its oracle.

This module only defines initial conditions and turns them into the
method's degrees of freedom (cell averages of the conserved variables by a
5x5 Gauss-Legendre rule per cell, and point values at vertices and edge
midpoints).  It holds none of the method's own arithmetic, so both the CUDA
path and the FP64 oracle can take their inputs from it.

Problems (paper sections in brackets):
  * ``gaussian_pulse``  -- Example 1, 1D density/pressure pulse [Sec. 2]
  * ``compact_vortex``  -- Example 2, compactly supported travelling vortex
    [Sec. 2]; the velocity profile is read as 1024 (1-r)^6 r^6, the only
    profile whose pressure balance gives the printed p(r)
  * ``shu_vortex``      -- isentropic vortex on a periodic box; strength,
    centre and box are parameters (not from the paper; a standard smooth test)
  * ``four_quadrant``   -- four constant states meeting at (0.5, 0.5), as in
    the 2D Riemann problems of Sec. 4.1; states drawn from a seed
  * ``double_rarefaction`` -- two states moving apart at x = 0.5, cf.
    Example 4 (double rarefaction), with the stated near-vacuum data
  * ``kelvin_helmholtz`` -- the shear-layer data of Sec. 4.2
  * ``fourier_smooth``  -- seeded smooth periodic field used for parity tests
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional

import numpy as np

GAMMA = 1.4
PERIODIC, TRANSMISSIVE, REFLECTING = 0, 1, 2

# 5-point Gauss-Legendre on [0, 1]
_GLX, _GLW = np.polynomial.legendre.leggauss(5)
_GLX = 0.5 * (_GLX + 1.0)
_GLW = 0.5 * _GLW

Field = Callable[[np.ndarray, np.ndarray], tuple]


@dataclasses.dataclass
class Problem:
    name: str
    nx: int
    ny: int
    x0: float
    y0: float
    lx: float
    ly: float
    bc: tuple  # (xlo, xhi, ylo, yhi)
    field: Field  # (x, y) -> (rho, u, v, p), vectorised
    t_end: float
    cfl: float = 0.3
    gamma: float = GAMMA
    options: dict = dataclasses.field(default_factory=dict)
    exact: Optional[Callable[[float], Field]] = None
    inflow: dict = dataclasses.field(default_factory=dict)  # side (0..3) -> primitive state, for BC 3
    centre: Optional[tuple] = None  # vortex centre at t = 0 (moving with velocity (1, 1))

    def vortex_centre(self, t):
        """Centre of the translating vortex at time t, wrapped into the box."""
        cx, cy = self.centre
        u0, v0 = getattr(self, "velocity", (1.0, 1.0))
        return self.x0 + (cx + u0 * t - self.x0) % self.lx, self.y0 + (cy + v0 * t - self.y0) % self.ly

    @property
    def dx(self):
        return self.lx / self.nx

    @property
    def dy(self):
        return self.ly / self.ny

    @property
    def bc_code(self):
        a, b, c, d = self.bc
        return a | (b << 8) | (c << 16) | (d << 24)


def conserved(U, gamma=GAMMA):
    """Conserved variables (rho, rho u, rho v, E) of primitive (rho, u, v, p)."""
    r, u, v, p = U
    return np.stack([r, r * u, r * v, p / (gamma - 1.0) + 0.5 * r * (u * u + v * v)])


def _eval(field, x, y):
    return np.stack([np.broadcast_to(np.asarray(c, dtype=np.float64), np.broadcast(x, y).shape)
                     for c in field(x, y)])


def discretise(prob: Problem, field: Optional[Field] = None):
    """Degrees of freedom of ``field`` (default: the problem's initial data).

    Returns float64 arrays avg (4,ny,nx) conservative, vtx (4,ny+1,nx+1),
    xe (4,ny,nx+1), ye (4,ny+1,nx) primitive.  On periodic axes the last node
    line is an exact copy of the first one.
    """
    f = field or prob.field
    nx, ny, dx, dy = prob.nx, prob.ny, prob.dx, prob.dy
    xn = prob.x0 + dx * np.arange(nx + 1)
    yn = prob.y0 + dy * np.arange(ny + 1)
    xc = prob.x0 + dx * (np.arange(nx) + 0.5)
    yc = prob.y0 + dy * (np.arange(ny) + 0.5)
    vtx = _eval(f, xn[None, :], yn[:, None])
    xe = _eval(f, xn[None, :], yc[:, None])
    ye = _eval(f, xc[None, :], yn[:, None])
    avg = np.zeros((4, ny, nx))
    for a, wa in zip(_GLX, _GLW):
        for b, wb in zip(_GLX, _GLW):
            X = prob.x0 + dx * (np.arange(nx)[None, :] + a)
            Y = prob.y0 + dy * (np.arange(ny)[:, None] + b)
            avg += wa * wb * conserved(_eval(f, X, Y), prob.gamma)
    if prob.bc[0] == PERIODIC:
        vtx[:, :, nx] = vtx[:, :, 0]
        xe[:, :, nx] = xe[:, :, 0]
    if prob.bc[2] == PERIODIC:
        vtx[:, ny, :] = vtx[:, 0, :]
        ye[:, ny, :] = ye[:, 0, :]
    return avg, vtx, xe, ye


def discretise_torch(prob: Problem, device, field: Optional[Field] = None, dtype=None):
    """Same as ``discretise`` but evaluated with torch in float64 on ``device``
    (for large grids); returns float32 tensors unless ``dtype`` is given.
    Only for fields written against numpy/torch alike (``shu_vortex``,
    the four-quadrant data)."""
    import torch

    f = field or prob.field
    f64 = torch.float64
    nx, ny, dx, dy = prob.nx, prob.ny, prob.dx, prob.dy
    xn = prob.x0 + dx * torch.arange(nx + 1, device=device, dtype=f64)
    yn = prob.y0 + dy * torch.arange(ny + 1, device=device, dtype=f64)
    xc = prob.x0 + dx * (torch.arange(nx, device=device, dtype=f64) + 0.5)
    yc = prob.y0 + dy * (torch.arange(ny, device=device, dtype=f64) + 0.5)
    out_t = dtype or torch.float32

    def ev(x, y):
        vals = f(x, y)
        shape = torch.broadcast_shapes(x.shape, y.shape)
        return torch.stack([torch.as_tensor(v, dtype=f64, device=device).expand(shape) for v in vals])

    vtx = ev(xn[None, :], yn[:, None]).to(out_t)
    xe = ev(xn[None, :], yc[:, None]).to(out_t)
    ye = ev(xc[None, :], yn[:, None]).to(out_t)
    avg = torch.zeros((4, ny, nx), dtype=f64, device=device)
    ia = torch.arange(nx, device=device, dtype=f64)[None, :]
    ja = torch.arange(ny, device=device, dtype=f64)[:, None]
    for a, wa in zip(_GLX, _GLW):
        X = prob.x0 + dx * (ia + a)
        for b, wb in zip(_GLX, _GLW):
            Y = prob.y0 + dy * (ja + b)
            r, u, v, p = f(X, Y)
            avg[0] += wa * wb * r
            avg[1] += wa * wb * r * u
            avg[2] += wa * wb * r * v
            avg[3] += wa * wb * (p / (prob.gamma - 1.0) + 0.5 * r * (u * u + v * v))
    avg = avg.to(out_t)
    if prob.bc[0] == PERIODIC:
        vtx[:, :, nx] = vtx[:, :, 0]
        xe[:, :, nx] = xe[:, :, 0]
    if prob.bc[2] == PERIODIC:
        vtx[:, ny, :] = vtx[:, 0, :]
        ye[:, ny, :] = ye[:, 0, :]
    return avg, vtx, xe, ye


def subproblem(prob: Problem, i0: int, j0: int, ni: int, nj: int, bc=(1, 1, 1, 1)):
    """The cells [i0, i0+ni) x [j0, j0+nj) of ``prob`` as a problem of its
    own (for checking sampled windows of a large grid)."""
    return Problem(prob.name + "_window", ni, nj, prob.x0 + i0 * prob.dx, prob.y0 + j0 * prob.dy,
                   ni * prob.dx, nj * prob.dy, bc, prob.field, prob.t_end, prob.cfl, prob.gamma,
                   dict(prob.options), prob.exact)


def to_f32(state):
    """Round a state to FP32 (the GPU's storage) and back to float64."""
    return tuple(np.asarray(a, dtype=np.float32).astype(np.float64) for a in state)


def _wrap(d, period):
    return d - period * _mod(d).floor(d / period + 0.5)


# ----------------------------------------------------------------- problems
def _mod(x):
    """numpy, or torch when the coordinates are torch tensors."""
    if type(x).__module__.startswith("torch"):
        import torch

        return torch
    return np


def shu_vortex(n=32, eps=5.0, xc=5.0, yc=5.0, L=10.0, t_end=10.0, ny=None, cfl=0.3, vel=(1.0, 1.0)):
    """Isentropic vortex of strength eps on the periodic box [0,L]^2 moving
    with the background velocity ``vel`` (default (1,1)) through rho = p = 1
    (minimum-image distance to the centre, so the data are single valued on
    the torus)."""
    g = GAMMA
    u0, v0 = vel

    def at(t):
        cx, cy = xc + u0 * t, yc + v0 * t

        def f(x, y):
            m = _mod(x)
            X = x - cx
            X = X - L * m.floor(X / L + 0.5)
            Y = y - cy
            Y = Y - L * m.floor(Y / L + 0.5)
            r2 = X * X + Y * Y
            e = m.exp(0.5 * (1.0 - r2))
            T = 1.0 - (g - 1.0) * eps * eps / (8.0 * g * np.pi ** 2) * e * e
            rho = T ** (1.0 / (g - 1.0))
            return rho, u0 - eps / (2 * np.pi) * e * Y, v0 + eps / (2 * np.pi) * e * X, rho ** g

        return f

    p = Problem("shu_vortex", n, ny or n, 0.0, 0.0, L, L, (0, 0, 0, 0), at(0.0), t_end,
                cfl=cfl, exact=at, centre=(xc, yc))
    p.velocity = (u0, v0)
    return p


# Background velocity of the long vortex runs (the convergence sweep and the
# surrogate evaluation): the standing vortex.  The scheme amplifies
# perturbations of states whose Mach circle crosses both grid lines through a
# vertex without holding it (oblique flow near Mach 1.2); a moving vortex
# carries such states in the quadrant where its swirl adds to the background
# (with the default (1, 1) runs of about 900 FP32 steps blow up, with (0.5,
# 0.5) about 1600 at 1024^2, with (0.25, 0.25) the error grows), the standing
# one (swirl at most 0.95, c >= 0.95) does not.
STABLE_VELOCITY = (0.0, 0.0)


def shu_vortex_seeded(n, seed=2508, t_end=2.0, vel=(1.0, 1.0)):
    """Vortex with centre in [3,6]^2 and strength in [3,6] drawn from ``seed``."""
    rng = np.random.default_rng(seed)
    xc, yc = rng.uniform(3.0, 6.0, size=2)
    eps = rng.uniform(3.0, 6.0)
    p = shu_vortex(n, eps=eps, xc=xc, yc=yc, t_end=t_end, vel=vel)
    p.name = f"shu_vortex_seed{seed}"
    return p


_EX2_P = np.array([1 / 72, -6 / 35, 15 / 17, -74 / 33, 57 / 32, 174 / 31, -269 / 15, 450 / 29,
                   153 / 8, -1564 / 27, 510 / 13, 204 / 5, -1473 / 16, 1014 / 23, 1053 / 22,
                   -558 / 7, 783 / 20, 54 / 19, -38 / 9, -222 / 17, 609 / 32, -184 / 15, 9 / 2,
                   -12 / 13, 1 / 12])  # coefficients of r^36 ... r^12, Example 2


def ex2_pressure(r):
    """p(r) of Example 2 (coefficients of r^36 down to r^12, times 1024^2)."""
    if _mod(r) is np:
        r = np.asarray(r, dtype=np.float64)
    s = 0.0 * r
    for k, c in enumerate(_EX2_P):
        s = s * r + c
    return 1024.0 ** 2 * s * r ** 12


def compact_vortex(n=32, t_end=1.0, cfl=0.3):
    """Example 2 on [0,1]^2, periodic, translating with (1,1); the exact
    solution at integer times equals the initial data."""
    rc, uc, vc, pc, R = 0.5, 1.0, 1.0, 0.1, 0.4
    p1 = float(ex2_pressure(1.0))

    def at(t):
        def f(x, y):
            m = _mod(x)
            X = _wrap(x - 0.5 - uc * t, 1.0)
            Y = _wrap(y - 0.5 - vc * t, 1.0)
            d = m.sqrt(X * X + Y * Y)
            r = d / R
            inside = (r < 1.0) * 1.0
            safe = d + (d == 0) * 1.0
            rr = m.minimum(r, 0.0 * r + 1.0)
            prof = 1024.0 * (1.0 - rr) ** 6 * rr ** 6
            rho = rc + inside * 0.5 * (1.0 - rr * rr) ** 6
            u = uc - inside * prof * Y / safe
            v = vc + inside * prof * X / safe
            p = pc + inside * (ex2_pressure(rr) - p1)
            return rho, u, v, p

        return f

    return Problem("compact_vortex", n, n, 0.0, 0.0, 1.0, 1.0, (0, 0, 0, 0), at(0.0), t_end,
                   cfl=cfl, exact=at)


def gaussian_pulse(nx=32, ny=8, t_end=0.25, cfl=0.3):
    """Example 1: rho = p = 1 + exp(-80 (x-1/2)^2)/2, u = v = 0 on x in
    [0,1]; ``ny`` square cells in y, periodic both ways."""

    def f(x, y):
        g = 1.0 + 0.5 * _mod(x).exp(-80.0 * (x - 0.5) ** 2) + 0.0 * y
        return g, 0.0 * g, 0.0 * g, g

    dx = 1.0 / nx
    return Problem("gaussian_pulse", nx, ny, 0.0, 0.0, 1.0, ny * dx, (0, 0, 0, 0), f, t_end,
                   cfl=cfl)


def _piecewise(states, xs, ys):
    """Four quadrant states (ll, lr, ul, ur) meeting at (xs, ys); points on a
    dividing line take the mean of the adjacent states (the corner the mean of
    all four)."""
    S = np.asarray(states, dtype=np.float64)  # (4 quadrants, 4 vars)

    def f(x, y):
        m = _mod(x)
        if m is np:
            x, y = np.broadcast_arrays(np.asarray(x, dtype=np.float64), np.asarray(y, dtype=np.float64))
        else:
            x, y = m.broadcast_tensors(x, y)
        one = (lambda c: c.astype(np.float64)) if m is np else (lambda c: c.to(x.dtype))
        wx_r = one(x > xs) + 0.5 * one(x == xs)
        wy_u = one(y > ys) + 0.5 * one(y == ys)
        w = [(1 - wx_r) * (1 - wy_u), wx_r * (1 - wy_u), (1 - wx_r) * wy_u, wx_r * wy_u]
        return tuple(sum(w[q] * float(S[q, k]) for q in range(4)) for k in range(4))

    return f


def four_quadrant(n=64, seed=0, t_end=0.25, cfl=0.3, states=None):
    """Four-quadrant Riemann data on [0,1]^2 split at (0.5,0.5), outflow
    boundaries; rho in [0.1,1.5], p in [0.01,1.5], u, v in [-1.2,1.2] drawn
    from ``seed``, unless ``states`` (lower-left, lower-right, upper-left,
    upper-right; each rho, u, v, p) is given.  Run with Alg. 2, Alg. 3 (with
    the node bounds), the Sec. 3.4 blend and the cell-average flux limiter."""
    if states is None:
        rng = np.random.default_rng(seed)
        st = np.stack([rng.uniform(0.1, 1.5, 4), rng.uniform(-1.2, 1.2, 4),
                       rng.uniform(-1.2, 1.2, 4), rng.uniform(0.01, 1.5, 4)], axis=1)
    else:
        st = np.asarray(states, dtype=np.float64)
    p = Problem(f"four_quadrant_seed{seed}", n, n, 0.0, 0.0, 1.0, 1.0, (1, 1, 1, 1),
                _piecewise(st, 0.5, 0.5), t_end, cfl=cfl,
                options={"tsw": 1, "limiter": 1, "flux_limiter": 1, "shock_blend": 1, "node_bounds": 1,
                         "ubar": 1})
    p.states = st
    return p


def double_rarefaction(n=64, t_end=0.25, cfl=0.3, rho=1.0, p=0.4, speed=2.0):
    """rho = 1, p = 0.4, u = -2 for x < 0.5 and +2 for x > 0.5 (u = 0 on the
    line), v = 0; outflow at x = 0, 1 and solid walls at y = 0, 1."""
    st = [(rho, -speed, 0.0, p), (rho, speed, 0.0, p), (rho, -speed, 0.0, p), (rho, speed, 0.0, p)]
    return Problem("double_rarefaction", n, n, 0.0, 0.0, 1.0, 1.0, (1, 1, 2, 2),
                   _piecewise(st, 0.5, -1.0), t_end, cfl=cfl,
                   options={"limiter": 1, "flux_limiter": 1, "node_bounds": 1, "ubar": 1})


def kelvin_helmholtz(n=64, t_end=1.0, cfl=0.3):
    """Sec. 4.2: shear layer on [-1/2,1/2]^2, periodic; nodes on |y| = 1/4
    take the mean of the two layers."""

    def f(x, y):
        x, y = np.broadcast_arrays(np.asarray(x, dtype=np.float64), np.asarray(y, dtype=np.float64))
        inner = np.where(np.abs(y) < 0.25, 1.0, np.where(np.abs(y) == 0.25, 0.5, 0.0))
        rho = 1.0 + inner
        u = 0.5 - inner
        v = 1e-2 * np.sin(2 * np.pi * x)
        return rho, u, v, 2.5 + 0.0 * x

    return Problem("kelvin_helmholtz", n, n, -0.5, -0.5, 1.0, 1.0, (0, 0, 0, 0), f, t_end,
                   cfl=cfl, options={"limiter": 1, "ubar": 1})


def shock_reflection(nx=120, ny=30, t_end=6.0, cfl=0.3):
    """Shock reflection on [0,4] x [0,1] (Sec. 4.3's final example, data as
    printed): (1, 2.9, 0, 1/1.4) everywhere except on y = 1, which carries
    (1.69997, 2.61934, -0.50632, 1.52819); the same states flow in at the
    left and top boundaries; solid wall at the bottom, outflow on the right.
    The paper runs it without any limiter."""
    A = (1.0, 2.9, 0.0, 1.0 / 1.4)
    B = (1.69997, 2.61934, -0.50632, 1.52819)

    def f(x, y):
        m = _mod(y)
        top = (y >= 1.0) * 1.0 if m is np else (y >= 1.0).to(y.dtype)
        return tuple(a + (b - a) * top for a, b in zip(A, B))

    p = Problem("shock_reflection", nx, ny, 0.0, 0.0, 4.0, 1.0, (3, 1, 2, 3), f, t_end, cfl=cfl,
                options={"limiter": 0, "ubar": 1}, inflow={0: A, 3: B})
    return p


def ensemble(n=256, seed=4096, lo=64, ratio=8.0, steps=200):
    """Ensemble of ``n`` independent problems of uneven sizes: N x N cells
    with N = round(lo * ratio**U), U ~ U[0,1) drawn from ``seed`` (64^2 to
    512^2 by default, log-uniform); even instances are seeded isentropic
    vortices (centre and strength in [3,6] on periodic [0,10]^2), odd ones
    seeded four-quadrant Riemann problems on [0,1]^2 with outflow boundaries.
    Every instance runs ``steps`` steps (end time +inf)."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(lo * ratio ** rng.uniform(0.0, 1.0, size=n)).astype(int)
    probs = []
    for k, N in enumerate(sizes):
        if k % 2 == 0:
            p = shu_vortex_seeded(int(N), seed=seed + k, t_end=np.inf)
        else:
            p = four_quadrant(int(N), seed=seed + k, t_end=np.inf)
        probs.append(p)
    return probs


def fourier_smooth(nx=32, ny=32, seed=1, amp=0.15, lx=1.0, ly=1.0, modes=3):
    """Smooth periodic field: every primitive variable is a background value
    plus a few seeded Fourier modes (used for parity tests)."""
    rng = np.random.default_rng(seed)
    base = np.array([1.0, 0.3, -0.2, 1.0])
    coef = rng.normal(size=(4, modes, modes, 2)) * amp / modes

    def f(x, y):
        out = []
        for k in range(4):
            s = base[k] + 0.0 * (x + y)
            for a in range(modes):
                for b in range(modes):
                    ph = 2 * np.pi * (a * x / lx + b * y / ly)
                    s = s + coef[k, a, b, 0] * np.cos(ph) + coef[k, a, b, 1] * np.sin(ph)
            out.append(s)
        return tuple(out)

    return Problem(f"fourier_smooth_seed{seed}", nx, ny, 0.0, 0.0, lx, ly, (0, 0, 0, 0), f, 1.0)


def cell_mean_exact(prob: Problem, field: Field):
    """Cell averages of the conserved variables of ``field`` (5x5 Gauss)."""
    return discretise(prob, field)[0]
