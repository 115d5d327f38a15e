"""The learned surrogate on the GPU, through the C ABI: the batched sampler's
features and targets against the FP64 reference (oracle/surrogate.py with
the C oracle's step), the exact fallback (a network that never passes the
check must reproduce the plain method bit for bit), and a trained network
against the method without it."""
import numpy as np
import pytest

from helpers import make_oracle
from oracle import surrogate as S
from paper_2508_06273_gb300 import workloads as W
from test_gpu_parity import MILD, env, host, solver, state_err, to_dev  # noqa: F401

pytestmark = pytest.mark.gpu


def _batch(env, probs):
    torch, af, _ = env
    b = af.Batch([(p.nx, p.ny) for p in probs], [(p.dx, p.dy) for p in probs], bcs=[p.bc for p in probs])
    for k, p in enumerate(probs):
        for key, v in p.options.items():
            b.set_option(key, v, k)
        b.set_state(k, *to_dev(torch, W.to_f32(W.discretise(p))))
    return b


def test_sampled_features_and_targets_match_the_oracle(env, oracle_mod):
    torch, af, _ = env
    probs = [W.shu_vortex_seeded(24, seed=21), W.four_quadrant(20, states=MILD)]
    b = _batch(env, probs)
    b.set_sampler(4000, 8000, seed=77, rate=0.3)
    hist = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
    b.run(1, hist)
    Xv, Tv, idv, Xe, Te, ide = (t.cpu().numpy() for t in b.samples())
    assert len(Xv) > 100 and len(Xe) > 200
    dts = hist[0].cpu().numpy()
    checked = 0
    for k, p in enumerate(probs):
        st = W.to_f32(W.discretise(p))
        o = make_oracle(oracle_mod, p, state=st)
        o.step(dts[k])
        half, new = o.get_half(), o.get_state()
        for X, T, ids in ((Xv, Tv, idv), (Xe, Te, ide)):
            sel = ids[:, 0] == k
            assert np.all(ids[sel, 1] == 1)
            for kind in (0, 1, 2):
                m = sel & (ids[:, 2] == kind)
                if not m.any():
                    continue
                I, J = ids[m, 3] & 0xFFFF, ids[m, 3] >> 16
                Xo, ut, sc = S.features(st, p.bc, kind, I, J, dts[k], p.dx,
                                        ubar_c2p=p.options.get("ubar", 0))
                U0 = S.node_values(st, kind, I, J)
                U1 = np.asarray(half[kind])[:, J, I].T
                U2 = np.asarray(new[1 + kind])[:, J, I].T
                To = S.targets(U0, U1, U2, ut, sc, kind)
                assert np.abs(X[m] - Xo).max() < 2e-4, (k, kind, np.abs(X[m] - Xo).max())
                assert np.abs(T[m] - To).max() < 2e-4 * max(1.0, np.abs(To).max()), (k, kind)
                checked += int(m.sum())
    assert checked == len(Xv) + len(Xe)
    b.close()


def test_a_network_that_never_passes_falls_back_to_the_exact_operator(env):
    torch, af, _ = env
    prob = W.shu_vortex_seeded(40, seed=8)
    nets = [af.Mlp(seed=s) for s in (1, 2)]
    for n in nets:
        p = n.get_params()
        p[-8:] = np.nan  # output scales: every decoded value is NaN
        n.set_params(p)
    plain, surr = solver(env, prob), solver(env, prob)
    surr.set_surrogate(*nets)
    dt = 0.3 * prob.dx / plain.max_speed()
    for _ in range(3):
        plain.step(dt)
        surr.step(dt)
    for a, c in zip(plain.get_state(), surr.get_state()):
        assert torch.equal(a, c)
    n_net, n_fall = surr.surrogate_stats()
    assert n_net == 0 and n_fall == 3 * 3 * 40 * 40
    assert surr.status() == 0
    for s in (plain, surr):
        s.close()


def test_fallback_on_a_transmissive_grid_with_an_odd_tile_count(env):
    """Non-periodic 64^2 four-quadrant data with its limiters: 65 x 65 nodes
    give 3 x 17 tiles, an odd count (the counters behind the tile flags must
    still be 8-byte aligned).  A network that never passes falls back at
    every node, bit for bit the plain method."""
    torch, af, _ = env
    prob = W.four_quadrant(64, states=MILD)
    nets = [af.Mlp(seed=s) for s in (1, 2)]
    for n in nets:
        p = n.get_params()
        p[-8:] = np.nan
        n.set_params(p)
    plain, surr = solver(env, prob), solver(env, prob)
    surr.set_surrogate(*nets)
    dt = 0.3 * prob.dx / plain.max_speed()
    for _ in range(3):
        plain.step(dt)
        surr.step(dt)
    for a, c in zip(plain.get_state(), surr.get_state()):
        assert torch.equal(a, c)
    n_net, n_fall = surr.surrogate_stats()
    assert n_net == 0 and n_fall > 0
    assert not surr.status() & (af.ST_AVG_NONPOS | af.ST_NONFINITE)
    for s in (plain, surr):
        s.close()


def _training_set(env, seeds, n_lo=48, n_hi=96, steps=12, rate=0.08):
    torch, af, _ = env
    rng = np.random.default_rng(seeds[0])
    probs = [W.shu_vortex_seeded(int(rng.integers(n_lo, n_hi)), seed=s, t_end=np.inf) for s in seeds]
    b = _batch(env, probs)
    b.set_sampler(400000, 800000, seed=seeds[0] + 1, rate=rate)
    b.run(steps)
    out = [t.clone() for t in b.samples()]
    b.close()
    return out


def test_trained_surrogate_beats_the_method_without_it(env):
    """Trained on samples of seeded vortices, evaluated on held-out ones:
    its prediction error is far below that of predicting no change (the
    step without the point-value update) and of the untrained network, and
    a surrogate run stays close to the plain method with few fallbacks."""
    torch, af, _ = env
    Xv, Tv, _, Xe, Te, _ = _training_set(env, list(range(100, 116)))
    Hv, HTv, _, He, HTe, _ = _training_set(env, [300, 301], steps=6)
    nets = []
    for X, T, HX, HT in ((Xv, Tv, Hv, HTv), (Xe, Te, He, HTe)):
        m = af.Mlp(seed=5)
        m.fit_scales(X, T)
        untrained = ((m.forward(HX) - HT) ** 2).mean().item()
        hist = m.train(X, T, steps=1500, batch=4096, lr=2e-3, seed=3)
        trained = ((m.forward(HX) - HT) ** 2).mean().item()
        no_change = (HT ** 2).mean().item()
        assert np.isfinite(hist).all()
        assert trained < 0.01 * no_change and trained < 0.01 * untrained, (trained, no_change, untrained)
        nets.append(m)
    prob = W.shu_vortex_seeded(64, seed=999)
    plain, surr = solver(env, prob), solver(env, prob)
    surr.set_surrogate(*nets, tol=0.5)
    for _ in range(10):
        dt = 0.3 * prob.dx / plain.max_speed()
        plain.step(dt)
        surr.step(dt)
    n_net, n_fall = surr.surrogate_stats()
    assert n_fall < 0.05 * (n_net + n_fall), (n_net, n_fall)
    err = state_err(host(surr.get_state()), host(plain.get_state()))
    assert err < 2e-3, err
    assert surr.status() & ~8 == 0
    for s in (plain, surr):
        s.close()
    for m in nets:
        m.close()


def test_the_stencil_limit_sends_wide_stencils_to_the_exact_operator(env):
    """AF_OPT_SURR_SMOOTH: with a limit of 0 no stencil of smooth nonuniform
    data qualifies and the step is bit for bit the plain method; a limit no
    stencil reaches changes nothing against no limit."""
    torch, af, _ = env
    prob = W.fourier_smooth(40, 40, seed=9)
    nets = [af.Mlp(seed=s) for s in (1, 2)]
    plain, surr = solver(env, prob), solver(env, prob)
    surr.set_surrogate(*nets)
    surr.set_option("surr_smooth", 0.0)
    dt = 0.3 * prob.dx / plain.max_speed()
    for _ in range(3):
        plain.step(dt)
        surr.step(dt)
    for a, c in zip(plain.get_state(), surr.get_state()):
        assert torch.equal(a, c)
    n_net, n_fall = surr.surrogate_stats()
    assert n_net == 0 and n_fall == 3 * 3 * 40 * 40
    a, b = solver(env, prob), solver(env, prob)
    for s in (a, b):
        s.set_surrogate(*nets)
    b.set_option("surr_smooth", 1e30)
    for _ in range(3):
        a.step(dt)
        b.step(dt)
    for x, y in zip(a.get_state(), b.get_state()):
        assert torch.equal(x, y)
    assert a.surrogate_stats() == b.surrogate_stats()
    for s in (plain, surr, a, b):
        s.close()
