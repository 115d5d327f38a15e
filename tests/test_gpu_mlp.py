"""Tensor-core (tcgen05) BF16 GEMM of the surrogate's training, through the
C ABI, against FP64 products of the same BF16-rounded operands."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2508_06273_gb300 import af

    return torch, af.lib()


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _gemm(torch, L, A, B, D, bias=None, splits=1, accumulate=0):
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    M, K = A.shape
    N = B.shape[0]
    rc = L.af_gemm_bf16(_p(A), A.stride(0), _p(B), B.stride(0), _p(D), D.stride(0), M, N, K, _p(bias), splits,
                        accumulate, _p(err), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, L.af_last_error().decode()
    torch.cuda.synchronize()
    assert int(err.item()) == 0


@pytest.mark.parametrize("M,N,K,splits", [(128, 128, 64, 1), (300, 16, 40, 1), (256, 64, 1024, 1),
                                          (128, 96, 4096, 8), (129, 128, 128, 2), (1000, 48, 136, 3)])
def test_gemm_matches_fp64(lib, M, N, K, splits):
    torch, L = lib
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    bias = torch.randn(N, device="cuda", generator=g)
    D = torch.full((M, N), float("nan"), device="cuda")
    _gemm(torch, L, A, B, D, bias, splits)
    a, b = A.double().cpu().numpy(), B.double().cpu().numpy()
    want = a @ b.T + bias.double().cpu().numpy()
    scale = np.abs(a) @ np.abs(b).T + 1.0
    err = np.abs(D.double().cpu().numpy() - want) / scale
    assert err.max() < 1e-6, (err.max(), np.unravel_index(err.argmax(), err.shape))


def test_gemm_accumulates_and_respects_leading_dimensions(lib):
    torch, L = lib
    g = torch.Generator(device="cuda").manual_seed(5)
    Abig = torch.randn(200, 96, device="cuda", generator=g).to(torch.bfloat16)
    Bbig = torch.randn(40, 72, device="cuda", generator=g).to(torch.bfloat16)
    A, B = Abig[:, :64], Bbig[:, :64]  # row strides 96 and 72 elements
    Dbig = torch.randn(200, 50, device="cuda", generator=g)
    D = Dbig[:, :40]
    before = Dbig.clone()
    _gemm(torch, L, A, B, D, accumulate=1)
    want = before[:, :40].double() + A.double() @ B.double().T
    assert torch.allclose(D.double(), want, rtol=1e-5, atol=1e-4)
    assert torch.equal(Dbig[:, 40:], before[:, 40:])  # untouched columns


def test_gemm_rejects_bad_shapes(lib):
    torch, L = lib
    A = torch.zeros(128, 60, dtype=torch.bfloat16, device="cuda")
    D = torch.zeros(128, 200, device="cuda")
    s = C.c_void_p(0)
    assert L.af_gemm_bf16(_p(A), 60, _p(A), 60, _p(D), 200, 128, 129, 60, None, 1, 0, None, s) == -1
    assert L.af_gemm_bf16(_p(A), 60, _p(A), 60, _p(D), 200, 128, 64, 60, None, 1, 0, None, s) == -1  # K % 8


# ------------------------------------------------------------ the network
from oracle import surrogate as S  # noqa: E402

LAYERS = (("W1", 0, (128, 64)), ("b1", 8192, (128,)), ("W2", 8320, (128, 128)), ("b2", 24704, (128,)),
          ("W3", 24832, (128, 128)), ("b3", 41216, (128,)), ("W4", 41344, (16, 128)), ("b4", 43392, (16,)))


def _unpack(p, bf16_weights):
    import torch

    P = {}
    for name, off, shape in LAYERS:
        a = np.asarray(p[off:off + int(np.prod(shape))], dtype=np.float32).reshape(shape)
        if bf16_weights and name.startswith("W"):
            a = torch.from_numpy(a.copy()).to(torch.bfloat16).float().numpy()
        P[name] = a.astype(np.float64)
    return P, p[43408:43472].astype(np.float64), p[43472:43480].astype(np.float64)


def _bf16(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).double().numpy()


@pytest.fixture(scope="module")
def net(lib):
    torch, L = lib
    from paper_2508_06273_gb300 import af

    m = af.Mlp(seed=11)
    p = m.get_params()
    rng = np.random.default_rng(4)
    p[8192:8320] = rng.normal(0, 0.1, 128)     # b1
    p[41216:41344] = rng.normal(0, 0.1, 128)   # b3
    p[43392:43400] = rng.normal(0, 0.1, 8)     # b4 (used rows)
    p[43408:43472] = rng.uniform(0.5, 2.0, 64)  # input scales
    p[43472:43480] = rng.uniform(0.5, 2.0, 8)   # output scales
    m.set_params(p)
    yield m, p
    m.close()


def _data(torch, n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 64)).astype(np.float32)
    T = rng.normal(size=(n, 8)).astype(np.float32)
    return X, T, torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()


def test_mlp_forward_matches_the_oracle(lib, net):
    torch, _ = lib
    m, p = net
    X, _, Xd, _ = _data(torch, 333, 1)
    P, ins, outs = _unpack(p, True)
    got = m.forward(Xd).double().cpu().numpy()
    # FP64 products with the hidden activations rounded to BF16 where the GPU
    # stores them: only the FP32 accumulation differs
    want = S.forward(P, _bf16(X * ins), rnd=S.bf16_round)[0][:, :8] * outs
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert rel < 1e-3, rel
    # without the rounding the difference is that of BF16 activations
    plain = S.forward(P, _bf16(X * ins))[0][:, :8] * outs
    assert np.linalg.norm(got - plain) / np.linalg.norm(plain) < 1e-2


def test_mlp_gradient_matches_the_oracle(lib, net):
    torch, _ = lib
    m, p = net
    X, T, Xd, Td = _data(torch, 1000, 2)
    P, ins, outs = _unpack(p, True)
    lg, gg = m.loss_grad(Xd, Td)
    # FP64 reference rounding the activations, dY and each dZ to BF16 where
    # the GPU stores them (the bias gradients sum the unrounded values)
    lo, go = S.loss_and_grads(P, _bf16(X * ins), T / outs, rnd=S.bf16_round)
    assert lg == pytest.approx(lo, rel=1e-3)
    for name, off, shape in LAYERS:
        a = gg[off:off + int(np.prod(shape))].reshape(shape).astype(np.float64)
        b = go[name]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert rel < 2e-3, (name, rel)
    # against exact FP64 the BF16 storage costs a few per cent at most
    _, g64 = S.loss_and_grads(P, _bf16(X * ins), T / outs)
    for name, off, shape in LAYERS:
        a = gg[off:off + int(np.prod(shape))].reshape(shape).astype(np.float64)
        assert np.linalg.norm(a - g64[name]) / max(np.linalg.norm(g64[name]), 1e-30) < 3e-2, name


def test_mlp_training_reduces_the_loss(lib):
    torch, _ = lib
    from paper_2508_06273_gb300 import af

    rng = np.random.default_rng(5)
    n = 20000
    X = rng.normal(size=(n, 64)).astype(np.float32)
    A = rng.normal(size=(64, 8)) / 8
    T = (X @ A + 0.3 * np.tanh(X[:, :8])).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    m = af.Mlp(seed=2)
    m.fit_scales(Xd, Td)
    hist = m.train(Xd, Td, steps=400, batch=1024, lr=2e-3, seed=9)
    assert np.all(np.isfinite(hist))
    assert hist[-20:].mean() < 0.05 * hist[:5].mean(), (hist[:5], hist[-20:])
    m.close()
