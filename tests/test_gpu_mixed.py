"""Mixed precision on the tensor cores (GENP_BF16, GENP_BF16X3) vs the oracle.

Error bounds (u32 = 2^-24):
* C = A G with G on the BF16 grid: BF16 rounds A once (relative 2^-9), so
  |dC| <= (2^-8 + 2 n u32) |A||G|; BF16X3 splits A into three BF16 terms
  (remainder below 2^-27 |a|) and accumulates three products in FP32:
  |dC| <= (2^-26 + 4 n u32) |A||G|.
* GENP with the Schur updates on the tensor cores: every update's operands
  carry 2^-9 relative error (BF16) or about 2^-24 (BF16X3), the accumulation
  and the FP32 trailing matrix add gamma_n(u32), so
  |L U - C| <= c |L||U| with c = 2^-7 + 4 n u32 (BF16), 8 n u32 + 2^-20 (BF16X3).
* BF16X3 factors + FP64 refinement reach backward error <= 1e-14 on the
  n = 256 workload with every multiplier.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def g(genp_lib):
    import paper_1212_4560_gb300 as genp
    assert genp_lib.genp_device_check(1) == 0
    return genp


def cu(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dtype)


@pytest.mark.parametrize("prec_name", ["BF16", "BF16X3"])
@pytest.mark.parametrize("n", [128, 200, 256, 520])
def test_precondition_tensor_cores(g, prec_name, n):
    prec = getattr(g, prec_name)
    A, _, _ = W.lead_deficient(n, 16, 8, 1, seed=n)
    A = A.numpy()
    G = g.make_multiplier(g.GAUSSIAN, n, seed=2, value_grid=g.BF16)
    Gd = torch.empty((n, n), dtype=torch.float64, device=DEV)
    g.multiplier_export(G, dense=Gd)
    Gm = Gd.cpu().numpy()
    C = torch.empty((n, n), dtype=torch.float32, device=DEV)
    g.precondition(G, cu(A), C, c_prec=prec)
    torch.cuda.synchronize()
    assert g._lib.load().genp_device_check(1) == 0
    ref = oracle.matmul(A, Gm)
    absprod = np.abs(A) @ np.abs(Gm)
    c = (2.0**-8 + 2 * n * U32) if prec_name == "BF16" else (2.0**-26 + 4 * n * U32)
    assert np.all(np.abs(C.cpu().double().numpy() - ref) <= c * absprod)


@pytest.mark.parametrize("prec_name", ["BF16", "BF16X3"])
@pytest.mark.parametrize("n,nb", [(128, 0), (256, 0), (300, 0), (384, 64), (520, 128)])
def test_factor_tensor_cores_backward_error(g, prec_name, n, nb):
    prec = getattr(g, prec_name)
    A, _, _ = W.lead_deficient(n, 16, 8, 1, seed=n + 1)
    C0 = oracle.precondition(A.numpy(), oracle.multiplier(0, n, seed=5)).astype(np.float32)
    C = cu(C0, torch.float32)
    F = g.factor(C, prec=prec, nb=nb)
    info = g.info_fetch(F)
    assert info.breakdown_step == -1
    assert g._lib.load().genp_device_check(1) == 0
    LU = C.cpu().double().numpy()
    L, U = oracle.split_lu(LU)
    c = (2.0**-7 + 4 * n * U32) if prec_name == "BF16" else (8 * n * U32 + 2.0**-20)
    assert np.all(np.abs(L @ U - C0.astype(np.float64)) <= c * (np.abs(L) @ np.abs(U)))


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_bf16x3_with_fp64_refinement(g, kind):
    A, _, B = (t.numpy() for t in W.lead_deficient(256, 32, 16, 1, seed=0))
    X, info, G, F = g.solve_system(cu(A), cu(B), kind=kind, seed=5, prec=g.BF16X3, refine_steps=20, tol=1e-16)
    eta = oracle.backward_error(A, X.cpu().numpy(), B)
    assert eta <= 1e-14
    assert info.bwd_err[0] > 1e-12            # the unrefined solution is at FP32-level accuracy
    assert g._lib.load().genp_device_check(1) == 0


def test_bf16_refinement_improves(g):
    n = 256
    A, _, B = (t.numpy() for t in W.shifted(1, n, 2, seed=3))
    A, B = A[0], B[0]
    X, info, G, F = g.solve_system(cu(A), cu(B), kind=g.SPARSE_PM1, seed=2, prec=g.BF16, refine_steps=20, tol=1e-16)
    assert info.breakdown_step == -1
    assert info.bwd_err[0] < 0.5                 # BF16 factors alone: a coarse solution
    assert info.bwd_err[-1] < info.bwd_err[0]
    eta = oracle.backward_error(A, X.cpu().numpy(), B)
    assert eta == pytest.approx(info.bwd_err[-1], rel=1e-6, abs=1e-15)


def test_bf16x3_adjoint(g):
    n, nrhs = 128, 3
    A, _, B = (t.numpy() for t in W.shifted(1, n, nrhs, seed=9))
    A, B = A[0], B[0]
    X, info, G, F = g.solve_system(cu(A), cu(B), kind=g.CIRCULANT, seed=1, prec=g.BF16X3, refine_steps=10, tol=1e-16)
    dA = torch.empty((n, n), dtype=torch.float32, device=DEV)
    dB = torch.empty((n, nrhs), dtype=torch.float64, device=DEV)
    g.adjoint(F, G, X, X, dA, dB)
    x = X.cpu().numpy()
    dA_ref, dB_ref = oracle.adjoint(A, x, x)
    assert np.linalg.norm(dA.cpu().double().numpy() - dA_ref) <= 1e-3 * np.linalg.norm(dA_ref)
    assert np.linalg.norm(dB.cpu().numpy() - dB_ref) <= 1e-3 * np.linalg.norm(dB_ref)
