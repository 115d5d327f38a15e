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
