"""GPU: the tcgen05 BF16 GEMM (FP32 accumulation in tensor memory) against FP32 products of the
same bf16 values. Exact bf16 x bf16 products accumulated in FP32 differ from an FP64 sum by
about K * 2^-24 relative; the bar is 1e-5 relative to the largest output."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _lib():
    import paper_2406_06640_gb300 as pg

    lib = pg.load()
    lib.ptycho_gemm_bf16.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    lib.ptycho_gemm_bf16.restype = ctypes.c_int
    return lib


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (256, 32, 128), (128, 48, 64), (384, 64, 192),
                                   (128, 128, 64), (256, 256, 576), (512, 96, 320)])
def test_gemm_matches_reference(M, N, K):
    dev = torch.device("cuda:0")
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    ref = A.double() @ B.double().T
    Ad, Bd = A.to(dev), B.to(dev)
    D = torch.zeros(M, N, dtype=torch.float32, device=dev)
    st = _lib().ptycho_gemm_bf16(Ad.data_ptr(), Bd.data_ptr(), D.data_ptr(), M, N, K, 0, None)
    assert st == 0
    err = (D.cpu().double() - ref).abs().max().item() / ref.abs().max().item()
    assert err < 1e-5, err
    # accumulate mode: D += A B^T
    st = _lib().ptycho_gemm_bf16(Ad.data_ptr(), Bd.data_ptr(), D.data_ptr(), M, N, K, 1, None)
    assert st == 0
    err2 = (D.cpu().double() - 2 * ref).abs().max().item() / ref.abs().max().item()
    assert err2 < 2e-5, err2


def test_gemm_rejects_bad_shapes():
    lib = _lib()
    assert lib.ptycho_gemm_bf16(1, 1, 1, 100, 16, 64, 0, None) == 1
    assert lib.ptycho_gemm_bf16(1, 1, 1, 128, 20, 64, 0, None) == 1
    assert lib.ptycho_gemm_bf16(1, 1, 1, 128, 16, 60, 0, None) == 1
