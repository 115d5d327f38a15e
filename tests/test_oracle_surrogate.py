"""Pins of the FP64 surrogate reference (oracle/surrogate.py): its cell prep
against the C oracle's, symmetry (to rounding) of the edge features under
the exchange of x and y, constant states, the GELU identities, and the MLP's
gradient against central finite differences."""
import numpy as np
import pytest

from oracle import surrogate as S
from paper_2508_06273_gb300 import workloads as W


@pytest.mark.parametrize("mode", [0, 1])
def test_ubar_matches_the_c_oracle(oracle_mod, mode):
    prob = W.four_quadrant(12, states=[(1.0, 0.1, -0.2, 1.0), (0.8, 0.3, 0.1, 0.7),
                                       (1.2, -0.1, 0.2, 1.1), (0.9, 0.0, 0.3, 0.9)])
    prob.bc = (1, 2, 2, 1)  # outflow and walls: ghost cells of both kinds
    st = W.discretise(prob)
    o = oracle_mod.Oracle(prob.nx, prob.ny, prob.dx, prob.dy, prob.gamma, prob.bc)
    o.set_option(oracle_mod.OPT_UBAR, mode)
    o.set_state(*st)
    o.prepare()
    ub = S.ubar(S.extend(st, prob.bc), c2p_mode=mode)
    for j in range(-1, prob.ny + 1):
        for i in range(-1, prob.nx + 1):
            _, want = o.cell_prim(i, j)
            assert np.allclose(ub[:, j + 1, i + 1], want, rtol=1e-13, atol=1e-13), (i, j)


def test_constant_state_has_only_the_cone_features():
    prob = W.fourier_smooth(8, 6, amp=0.0, lx=1.0, ly=0.75)
    st = W.discretise(prob)
    r, u, v, p = st[1][:, 0, 0]
    c = np.sqrt(1.4 * p / r)
    dt, h = 0.01, prob.dx
    for kind, n in ((S.VERTEX, 52), (S.XEDGE, 60), (S.YEDGE, 60)):
        X, ut, s = S.features(st, prob.bc, kind, np.array([0, 3, 7]), np.array([0, 2, 5]), dt, h)
        assert np.abs(X[:, :n]).max() < 1e-14 and np.all(X[:, n + 3:] == 0)
        a, b = (v, u) if kind == S.YEDGE else (u, v)
        assert np.allclose(X[:, n:n + 3], np.array([c, a, b]) * dt / h, rtol=1e-14)


def _transpose(state):
    """The state of the grid with x and y (and u and v) exchanged."""
    avg, vtx, xe, ye = state
    sw = lambda a: a[[0, 2, 1, 3]].transpose(0, 2, 1)  # noqa: E731
    return sw(avg), sw(vtx), sw(ye), sw(xe)


def test_y_edge_features_are_x_edge_features_of_the_exchanged_grid():
    prob = W.fourier_smooth(10, 7, seed=9, amp=0.2, lx=1.0, ly=0.7)
    prob.bc = (1, 2, 0, 0)
    st = W.discretise(prob)
    stT = _transpose(st)
    bcT = (prob.bc[2], prob.bc[3], prob.bc[0], prob.bc[1])
    I, J = np.array([0, 4, 9, 3]), np.array([0, 2, 6, 7])
    Xy, uty, sy = S.features(st, prob.bc, S.YEDGE, I, J, 0.02, prob.dx)
    Xx, utx, sx = S.features(stT, bcT, S.XEDGE, J, I, 0.02, prob.dx)
    # equal up to the summation order of the cell prep (the corners and edges
    # of a cell are visited in another order in the exchanged frame)
    assert np.allclose(Xy, Xx, rtol=0, atol=1e-14)
    # and the targets rotate the same way
    rng = np.random.default_rng(1)
    U0, U1, U2 = (rng.normal(size=(4, 4)) for _ in range(3))
    sw = [0, 2, 1, 3]
    Ty = S.targets(U0, U1, U2, uty, sy, S.YEDGE)
    Tx = S.targets(U0[:, sw], U1[:, sw], U2[:, sw], utx[:, sw], sx[:, sw], S.XEDGE)
    assert np.allclose(Ty, Tx, rtol=1e-15)


def test_gelu_identities():
    x = np.linspace(-6, 6, 101)
    assert S.gelu(np.array(0.0)) == 0.0
    assert np.allclose(S.gelu(x) - S.gelu(-x), x, rtol=0, atol=1e-15)  # tanh is odd
    assert np.allclose(S.gelu(np.array([20.0])), 20.0) and abs(S.gelu(np.array([-20.0]))[0]) < 1e-12
    h = 1e-6
    assert np.allclose(S.gelu_grad(x), (S.gelu(x + h) - S.gelu(x - h)) / (2 * h), rtol=1e-7, atol=1e-8)


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(7)
    P = S.init_params(3)
    for k in P:
        P[k] = P[k] + 0.05 * rng.normal(size=P[k].shape)
    P["W4"][S.NOUT:] = 0.0
    P["b4"][S.NOUT:] = 0.0
    X = rng.normal(size=(5, S.NIN))
    T = rng.normal(size=(5, S.NOUT))
    loss, g = S.loss_and_grads(P, X, T)
    h = 1e-6
    for name, idx in (("W1", (3, 7)), ("b1", (100,)), ("W2", (64, 5)), ("W3", (1, 127)), ("b3", (17,)),
                      ("W4", (2, 40)), ("b4", (7,))):
        Pp = {k: v.copy() for k, v in P.items()}
        Pm = {k: v.copy() for k, v in P.items()}
        Pp[name][idx] += h
        Pm[name][idx] -= h
        fd = (S.loss_and_grads(Pp, X, T)[0] - S.loss_and_grads(Pm, X, T)[0]) / (2 * h)
        assert g[name][idx] == pytest.approx(fd, rel=1e-6, abs=1e-10), name


def test_zero_change_has_zero_targets():
    rng = np.random.default_rng(2)
    U0 = rng.uniform(0.5, 1.5, size=(6, 4))
    ut = rng.uniform(0.5, 1.5, size=(6, 4))
    s = rng.uniform(0.5, 1.5, size=(6, 4))
    assert np.all(S.targets(U0, U0, U0, ut, s, S.VERTEX) == 0)


def test_bf16_rounding_of_the_reference():
    """bf16_round: ties go to the even BF16 value, other values to the
    nearest; the result agrees with torch's BF16 conversion element by element
    and leaves values already in BF16 alone."""
    one = np.float32(1.0)
    ulp = np.float32(2.0 ** -7)  # BF16 unit at 1
    cases = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -20, -1.0 - 2.0 ** -8,
                      3.0, 0.0], dtype=np.float32)
    want = np.array([1.0, 1.0, 1.0 + 2 * ulp, 1.0 + ulp, -1.0, 3.0, 0.0])
    assert np.array_equal(S.bf16_round(cases), want)
    assert one + ulp == np.float32(1.0078125)
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(3).normal(scale=10.0, size=4096).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).double().numpy()
    assert np.array_equal(S.bf16_round(x), ref)
    assert np.array_equal(S.bf16_round(ref), ref)


def test_rounded_gradients_reduce_to_the_exact_ones():
    """With rounding switched on but an identity in its place the gradients
    are the exact ones; with BF16 rounding they stay within a few BF16 units."""
    rng = np.random.default_rng(9)
    P = S.init_params(4)
    X = rng.normal(size=(16, S.NIN))
    T = rng.normal(size=(16, S.NOUT))
    l0, g0 = S.loss_and_grads(P, X, T)
    l1, g1 = S.loss_and_grads(P, X, T, rnd=lambda a: a)
    assert l0 == l1 and all(np.array_equal(g0[k], g1[k]) for k in g0)
    _, g2 = S.loss_and_grads(P, X, T, rnd=S.bf16_round)
    for k in g0:
        n = np.linalg.norm(g0[k])
        if n > 0:
            assert np.linalg.norm(g2[k] - g0[k]) / n < 3e-2, k
