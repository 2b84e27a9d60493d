"""Tensor-core BF16 GEMM (tcgen05) through the C ABI: D = alpha A B^T + beta Cin.

* small-integer operands: every product and partial sum is an integer below
  2^24, exact in FP32, so D must equal the int64 product bit for bit;
* Gaussian operands rounded to BF16: products are exact in FP32 and the
  accumulation errs by at most gamma_K (u = 2^-24) times |A||B^T|; the test
  allows 2 gamma_K;
* ragged m, n, K (not multiples of the 128 x 128 x 64 tiles) and an
  in-place Schur-style update D <- D - A B^T.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
U32 = 2.0 ** -24


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def tc(lib, A, Bt, alpha=1.0, beta=0.0, Cin=None, D=None):
    m, K = A.shape
    n = Bt.shape[0]
    if D is None:
        D = torch.empty((m, n), dtype=torch.float32, device=DEV)
    st = lib.genp_gemm_bf16(m, n, K, alpha, _p(A), A.stride(0), _p(Bt), Bt.stride(0), beta, _p(Cin),
                            Cin.stride(0) if Cin is not None else 0, _p(D), D.stride(0),
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, st
    torch.cuda.synchronize()
    assert lib.genp_device_check(1) == 0
    return D


@pytest.mark.parametrize("m,n,K", [(128, 128, 64), (1, 1, 8), (200, 130, 72), (256, 384, 512), (515, 260, 1000)])
def test_tc_gemm_integer_exact(genp_lib, m, n, K):
    rng = np.random.default_rng(m + n + K)
    A = rng.integers(-8, 9, (m, K))
    B = rng.integers(-8, 9, (n, K))
    Ad = torch.tensor(A, dtype=torch.bfloat16, device=DEV)
    Bd = torch.tensor(B, dtype=torch.bfloat16, device=DEV)
    D = tc(genp_lib, Ad, Bd)
    assert np.array_equal(D.cpu().numpy().astype(np.int64), A @ B.T)


@pytest.mark.parametrize("m,n,K", [(128, 128, 128), (300, 200, 136), (1024, 768, 2048)])
def test_tc_gemm_accumulation_bound(genp_lib, m, n, K):
    g = torch.Generator().manual_seed(m * 7 + K)
    A = torch.randn(m, K, generator=g).to(torch.bfloat16)
    B = torch.randn(n, K, generator=g).to(torch.bfloat16)
    D = tc(genp_lib, A.to(DEV), B.to(DEV), alpha=-2.0)
    a, b = A.double().numpy(), B.double().numpy()
    ref = -2.0 * a @ b.T
    bound = 2 * (K * U32 / (1 - K * U32)) * 2.0 * (np.abs(a) @ np.abs(b).T)
    assert np.all(np.abs(D.cpu().double().numpy() - ref) <= bound)


def test_tc_gemm_inplace_update(genp_lib):
    m, n, K = 260, 390, 128
    rng = np.random.default_rng(5)
    A = rng.integers(-4, 5, (m, K))
    B = rng.integers(-4, 5, (n, K))
    C0 = rng.integers(-1000, 1000, (m, n))
    Ad = torch.tensor(A, dtype=torch.bfloat16, device=DEV)
    Bd = torch.tensor(B, dtype=torch.bfloat16, device=DEV)
    # padded leading dimension on the output
    Cbuf = torch.zeros((m, n + 6), dtype=torch.float32, device=DEV)
    Cbuf[:, :n] = torch.tensor(C0, dtype=torch.float32)
    C = Cbuf[:, :n]
    tc(genp_lib, Ad, Bd, alpha=-1.0, beta=1.0, Cin=C, D=C)
    out = Cbuf.cpu().numpy()
    assert np.array_equal(out[:, :n].astype(np.int64), C0 - A @ B.T)
    assert np.all(out[:, n:] == 0)


def test_tc_gemm_rejects_misaligned(genp_lib):
    A = torch.zeros((16, 12), dtype=torch.bfloat16, device=DEV)   # ld 12: not a multiple of 8
    D = torch.empty((16, 16), dtype=torch.float32, device=DEV)
    st = genp_lib.genp_gemm_bf16(16, 16, 12, 1.0, _p(A), 12, _p(A), 12, 0.0, None, 0, _p(D), 16, None)
    assert st == -1
