"""FP64 reference of the learned point-value surrogate: its input features,
its targets and the MLP (forward, backward, loss), in plain numpy.

TEST INFRASTRUCTURE ONLY: imported by tests/ (and by nothing on the
product path).  It shares no code with the CUDA library.

The surrogate replaces the exact point-value operator of Alg. 1 (EG2 with
the correction of Corollary 1) at one node by a small network.  Its inputs
are taken from the t^n data around the node, relative to the node's
linearisation state u~ (the averaged state of eq. (Un+1/2): the mean of the
primitive cell averages Ubar of the cells that share the node) and scaled by
rho', c' = sqrt(gamma p'/rho') (rho by rho', u and v by c', p by rho' c'^2):

* vertex (i-1/2, j-1/2): Ubar of its 4 cells (LL, LR, UL, UR) and the point
  values of the 3 x 3 vertices around it (row by row from (i-3/2, j-3/2)),
  per variable (rho, u, v, p): 4 + 9 = 13 values x 4 = 52 inputs;
* x-edge (i-1/2, j): Ubar of its 2 cells (left, right), the 6 vertices of
  the two cells (lower row left to right, then upper row) and 7 edge points
  (x-edges at i-3/2, i-1/2, i+1/2 on row j, then the y-edges (i-1, j-1/2),
  (i, j-1/2), (i-1, j+1/2), (i, j+1/2)): 15 values x 4 = 60 inputs;
* y-edge (i, j-1/2): the x-edge stencil of the frame with x and y (and u
  and v) exchanged, so that one network serves both edge kinds;

then the geometry of the Mach-cone base over one step in cell units,
c' dt / h, u' dt / h and v' dt / h (square cells, h = dx = dy; u and v
exchanged for y-edges), zero-padded to 64: 55 vertex and 63 edge inputs.
Outputs: (U^{n+1/2} - U^n) and (U^{n+1} - U^n) at the node in the same
scaling (8 values, rotated for y-edges).

Network: 64 -> 128 -> 128 -> 128 -> 16 (the first 8 outputs used), GELU
on the hidden layers in the tanh form of Hendrycks & Gimpel (2016),
gelu(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))); loss: mean
squared error over the 8 outputs.
"""
from __future__ import annotations

import numpy as np

GAMMA = 1.4
NIN, NH, NOUT, NOUT_PAD = 64, 128, 8, 16
G = 2  # ghost layers
VERTEX, XEDGE, YEDGE = 0, 1, 2


# ----------------------------------------------------------------- ghosts
def _map(idx, n, node, periodic, lo_refl, hi_refl):
    """Ghost index map along one axis (Sec. 4.3): periodic wrap, or the mirror
    copy (node arrays mirror about the boundary node, cell arrays about the
    face); returns (source index, flip of the normal velocity)."""
    idx = np.asarray(idx)
    if periodic:
        return np.mod(idx, n), np.zeros(idx.shape, bool)
    own = n + 1 if node else n
    src = idx.copy()
    flip = np.zeros(idx.shape, bool)
    lo, hi = idx < 0, idx >= own
    src[lo] = -idx[lo] if node else -1 - idx[lo]
    src[hi] = 2 * n - idx[hi] if node else 2 * n - 1 - idx[hi]
    flip[lo] = lo_refl
    flip[hi] = hi_refl
    return src, flip


def extend(state, bc):
    """Ghost-extended copies (G layers each side) of the four DoF arrays:
    avg (conservative), vtx, xe, ye (primitive); index [v, j + G, i + G]."""
    avg, vtx, xe, ye = (np.asarray(a, dtype=np.float64) for a in state)
    ny, nx = avg.shape[1:]
    per_x, per_y = bc[0] == 0, bc[2] == 0
    rx = (bc[0] == 2, bc[1] == 2)
    ry = (bc[2] == 2, bc[3] == 2)

    def ext(a, nodex, nodey):
        ni = nx + 1 if nodex else nx
        nj = ny + 1 if nodey else ny
        I = np.arange(-G, ni + G)
        J = np.arange(-G, nj + G)
        si, fx = _map(I, nx, nodex, per_x, *rx)
        sj, fy = _map(J, ny, nodey, per_y, *ry)
        out = a[:, sj[:, None], si[None, :]].copy()
        out[1] *= np.where(fx[None, :], -1.0, 1.0)
        out[2] *= np.where(fy[:, None], -1.0, 1.0)
        return out

    return (ext(avg, False, False), ext(vtx, True, True), ext(xe, True, False),
            ext(ye, False, True))


# ------------------------------------------------------------- cell prep
def c2p(Q, gamma=GAMMA):
    r = Q[0]
    u, v = Q[1] / r, Q[2] / r
    return np.stack([r, u, v, (gamma - 1) * (Q[3] - 0.5 * r * (u * u + v * v))])


def p2c(U, gamma=GAMMA):
    r, u, v, p = U
    return np.stack([r, r * u, r * v, p / (gamma - 1) + 0.5 * r * (u * u + v * v)])


def ubar(ext, gamma=GAMMA, c2p_mode=0):
    """Primitive cell averages Ubar of the cells -1 .. n, returned at
    [v, j + 1, i + 1].  Default (Sec. 2): invert Simpson's rule for the
    conserved centre value Q_c, U_c = C2P(Q_c), then Simpson's rule over the
    primitive point values and U_c.  c2p_mode = 1: the primitive state of the
    conservative cell average (the reading after Sec. 3.5)."""
    avg, vtx, xe, ye = ext
    ny, nx = avg.shape[1] - 2 * G, avg.shape[2] - 2 * G
    o = G - 1  # extended index of cell -1
    cy, cx = slice(o, o + ny + 2), slice(o, o + nx + 2)
    cy1, cx1 = slice(o + 1, o + ny + 3), slice(o + 1, o + nx + 3)
    Qa = avg[:, cy, cx]
    if c2p_mode:
        return c2p(Qa, gamma)
    corners = [vtx[:, cy, cx], vtx[:, cy, cx1], vtx[:, cy1, cx], vtx[:, cy1, cx1]]
    edges = [xe[:, cy, cx], xe[:, cy, cx1], ye[:, cy, cx], ye[:, cy1, cx]]
    Qs = sum(p2c(U, gamma) for U in corners) + 4 * sum(p2c(U, gamma) for U in edges)
    Uc = c2p((36 * Qa - Qs) / 16, gamma)
    return (sum(corners) + 4 * sum(edges) + 16 * Uc) / 36


# --------------------------------------------------------------- features
def _scale(ut, gamma):
    rho, p = ut[0], ut[3]
    c = np.sqrt(gamma * p / rho)
    return np.stack([rho, c, c, rho * c * c]), c


def features(state, bc, kind, I, J, dt, h, gamma=GAMMA, ubar_c2p=0):
    """Features (n, 64), linearisation states (n, 4) and scales (n, 4) of the
    nodes (kind, I[k], J[k]) (array indices of that kind); ubar_c2p selects
    the definition of Ubar (see ubar)."""
    ext = extend(state, bc)
    avg, vtx, xe, ye = ext
    ub = ubar(ext, gamma, ubar_c2p)  # cells -1..n at [j + 1, i + 1]
    I = np.asarray(I)
    J = np.asarray(J)
    cb = lambda i, j: ub[:, j + 1, i + 1]  # noqa: E731
    pv = lambda a, i, j: a[:, j + G, i + G]  # noqa: E731
    if kind == VERTEX:
        cells = [cb(I - 1, J - 1), cb(I, J - 1), cb(I - 1, J), cb(I, J)]
        pts = [pv(vtx, I + a, J + b) for b in (-1, 0, 1) for a in (-1, 0, 1)]
        swap = False
    elif kind == XEDGE:
        cells = [cb(I - 1, J), cb(I, J)]
        pts = ([pv(vtx, I + a, J) for a in (-1, 0, 1)] + [pv(vtx, I + a, J + 1) for a in (-1, 0, 1)]
               + [pv(xe, I + a, J) for a in (-1, 0, 1)]
               + [pv(ye, I - 1, J), pv(ye, I, J), pv(ye, I - 1, J + 1), pv(ye, I, J + 1)])
        swap = False
    else:  # y-edge (i, j-1/2) in the exchanged frame
        cells = [cb(I, J - 1), cb(I, J)]
        pts = ([pv(vtx, I, J + a) for a in (-1, 0, 1)] + [pv(vtx, I + 1, J + a) for a in (-1, 0, 1)]
               + [pv(ye, I, J + a) for a in (-1, 0, 1)]
               + [pv(xe, I, J - 1), pv(xe, I, J), pv(xe, I + 1, J - 1), pv(xe, I + 1, J)])
        swap = True
    ut = sum(cells) / len(cells)
    s, c = _scale(ut, gamma)
    vals = cells + pts
    n = len(I)
    X = np.zeros((n, NIN))
    order = [0, 2, 1, 3] if swap else [0, 1, 2, 3]
    per = len(vals)
    for q, v in enumerate(order):
        for m, w in enumerate(vals):
            X[:, q * per + m] = (w[v] - ut[v]) / s[v]
    X[:, 4 * per] = c * dt / h
    X[:, 4 * per + 1] = ut[order[1]] * dt / h
    X[:, 4 * per + 2] = ut[order[2]] * dt / h
    return X, ut.T, s.T


def targets(U0, U1, U2, ut, s, kind):
    """(n, 8): (U^{n+1/2} - U^n) / s, (U^{n+1} - U^n) / s, per node (rows),
    in the exchanged frame for y-edges."""
    order = [0, 2, 1, 3] if kind == YEDGE else [0, 1, 2, 3]
    T = np.zeros((len(U0), NOUT))
    for q, v in enumerate(order):
        T[:, q] = (U1[:, v] - U0[:, v]) / s[:, v]
        T[:, 4 + q] = (U2[:, v] - U0[:, v]) / s[:, v]
    return T


def node_values(state, kind, I, J):
    """Point values (n, 4) of the nodes (kind, I, J) from the DoF arrays."""
    a = state[1 + kind]
    return np.asarray(a, dtype=np.float64)[:, J, I].T


# -------------------------------------------------------------------- MLP
K_GELU = np.sqrt(2.0 / np.pi)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(K_GELU * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    t = np.tanh(K_GELU * (z + 0.044715 * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * K_GELU * (1.0 + 3 * 0.044715 * z * z)


LAYERS = (("W1", "b1", NH, NIN), ("W2", "b2", NH, NH), ("W3", "b3", NH, NH), ("W4", "b4", NOUT_PAD, NH))


def init_params(seed=0):
    """He-style initial weights (rows 8..15 of the last layer zero)."""
    rng = np.random.default_rng(seed)
    P = {}
    for w, b, o, i in LAYERS:
        P[w] = rng.normal(0.0, np.sqrt(2.0 / i), size=(o, i))
        P[b] = np.zeros(o)
    P["W4"][NOUT:] = 0.0
    P["W4"] *= 0.1
    return P


def bf16_round(a):
    """Nearest BF16 value (ties to even) of each element, via its FP32 value:
    the upper 16 bits of the FP32 word after adding half a BF16 unit (0x7FFF)
    plus the lowest kept bit, the usual round-to-nearest-even on the bits.
    Returned in FP64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _keep(a):
    return a


def forward(P, X, rnd=None):
    """Outputs (n, 16) and the cache of pre-activations and activations.
    rnd (optional) rounds each hidden activation where a reduced-precision
    implementation stores it (e.g. bf16_round); the products stay exact."""
    r = rnd or _keep
    H = [np.asarray(X, dtype=np.float64)]
    Z = []
    for k, (w, b, _, _) in enumerate(LAYERS):
        z = H[-1] @ P[w].T + P[b]
        Z.append(z)
        H.append(r(gelu(z)) if k < 3 else z)
    return H[-1], (H, Z)


def loss_and_grads(P, X, T, rnd=None):
    """Mean squared error over the first 8 outputs and every row, and its
    gradient with respect to every parameter (reverse-mode, layer by layer).
    rnd (optional) rounds the hidden activations (as in forward) and the
    operands of the backward products, dY and each dZ, where a
    reduced-precision implementation stores them; the bias gradients are
    the sums of the unrounded values."""
    r = rnd or _keep
    Y, (H, Z) = forward(P, X, rnd)
    n = X.shape[0]
    R = Y[:, :NOUT] - T
    loss = float(np.mean(R * R))
    dY = np.zeros_like(Y)
    dY[:, :NOUT] = 2.0 * R / (n * NOUT)
    grads = {}
    d = dY
    for k in range(3, -1, -1):
        w, b, _, _ = LAYERS[k]
        grads[b] = d.sum(axis=0)
        d = r(d)
        grads[w] = d.T @ H[k]
        if k > 0:
            d = (d @ P[w]) * gelu_grad(Z[k - 1])
    grads["W4"][NOUT:] = 0.0
    grads["b4"][NOUT:] = 0.0
    return loss, grads
