"""Batched solves (one persistent launch) and the autograd binding vs the oracle.

* multipliers: system i's G_i (dense or circulant) equals the oracle's
  single-precision draw with stream id i, bit for bit;
* uneven sizes 2..512 (ragged against every tile) with a_11 = 0 (plain GENP
  breaks down): FP32 factors + GMRES-IR reach backward error <= 1e-14 and
  forward error <= 1e-14 kappa(A) against the FP64 oracle, with no system
  escalated; an unreachable target sends every system through the
  double-float escalation launch, which still ends at FP64 accuracy;
* the adjoint through the factors against the oracle gradient
  (lambda = A^{-T} gX by GEPP on A^T): FP32 factors 1e-3 relative, the FP64
  path 1e-10 and central finite differences (h = 1e-6) 1e-6;
* a CUDA-graph replay of the run reproduces the eager results bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def B(genp_lib):
    import paper_1212_4560_gb300.batched as batched
    return batched


def systems(sizes, nrhs, seed, zero_a11=True, shift=0.0):
    g = torch.Generator().manual_seed(seed)
    mats, xs, bs = [], [], []
    for n in sizes:
        A = torch.randn(n, n, generator=g, dtype=torch.float64) + shift * n * torch.eye(n, dtype=torch.float64)
        if zero_a11 and n >= 2:
            A[0, 0] = 0.0
        X = torch.randn(n, nrhs, generator=g, dtype=torch.float64)
        mats.append(A)
        xs.append(X)
        bs.append(A @ X)
    return mats, xs, bs


@pytest.mark.parametrize("kind", [0, 1])
def test_batched_multipliers_bit_exact(B, kind):
    sizes = [1, 5, 17, 64, 130]
    plan = B.BatchedPlan(sizes, 2, kind=kind, max_iter=0)
    mats, _, bs = systems(sizes, 2, 1, zero_a11=False, shift=1.0)
    Ap, Bp = plan.pack(mats, bs)
    Xp = torch.empty_like(Bp)
    plan.run(77, Ap, Bp, Xp)
    if kind == 0:
        Gp = torch.empty(plan.mat_size, dtype=torch.float32, device=DEV)
        plan.multipliers(G_pool=Gp)
        Gp = Gp.cpu().double().numpy()
        for i, n in enumerate(sizes):
            ref = oracle.multiplier(0, n, seed=77, stream=i, grid="fp32")["G"]
            assert np.array_equal(Gp[plan.mat_off[i]:plan.mat_off[i + 1]].reshape(n, n), ref)
    else:
        gp = torch.empty(sum(sizes), dtype=torch.float32, device=DEV)
        plan.multipliers(g_pool=gp)
        gp = gp.cpu().double().numpy()
        off = 0
        for i, n in enumerate(sizes):
            ref = oracle.multiplier(1, n, seed=77, stream=i, grid="fp32")["g"]
            assert np.array_equal(gp[off:off + n], ref)
            off += n


@pytest.mark.parametrize("a_dtype", [torch.float64, torch.float32])
def test_batched_uneven_refined(B, a_dtype):
    sizes = [2, 3, 16, 17, 31, 33, 64, 65, 100, 129, 200, 257, 300, 512]
    nrhs = 4
    plan = B.BatchedPlan(sizes, nrhs, kind=0, a_dtype=a_dtype, max_iter=12, tol=1e-15)
    mats, _, bs = systems(sizes, nrhs, 3)
    if a_dtype == torch.float32:     # the system solved is the FP32 one, exactly in FP64
        mats = [m.float().double() for m in mats]
        bs = [m @ x for m, x in zip(mats, systems(sizes, nrhs, 3)[1])]
    Ap, Bp = plan.pack(mats, bs)
    Xp = torch.zeros_like(Bp)
    plan.run(5, Ap, Bp, Xp)
    st = plan.status()
    torch.cuda.synchronize()
    for i, n in enumerate(sizes):
        A, b = mats[i].numpy(), bs[i].numpy()
        x = plan.unpack_vec(Xp, i).cpu().numpy()
        eta = oracle.backward_error(A, x, b)
        assert eta <= 1e-14, (n, eta, st["eta"][i], st["iters"][i])
        assert st["status"][i] == 0, (n, st["status"][i])
        assert abs(st["eta"][i] - eta) <= 4 * (n + 1) * 2.0**-53
        xd = oracle.gepp_solve(A, b)
        assert np.abs(x - xd).max() / np.abs(xd).max() <= 1e-14 * np.linalg.cond(A, np.inf)
    assert np.all(st["eta0"] > 1e-12)          # FP32 factors before refinement
    assert np.all(st["escalated"] < 2)        # no double-float refactorization
    assert np.all(st["krylov"][np.array(sizes) >= 100] > 0)


def test_batched_gaussian_512_all_converge(B):
    """The benchmark's systems at their largest order: FP32 GENP of A G loses
    u32 times an element growth of 1e3 .. 1e4, classic refinement would
    diverge on most of them; GMRES-IR brings every one to 1e-14."""
    sizes = [512] * 6 + [384] * 6
    plan = B.BatchedPlan(sizes, 4, kind=0, max_iter=10, tol=1e-14)
    mats, _, bs = systems(sizes, 4, 31)
    Ap, Bp = plan.pack(mats, bs)
    Xp = torch.empty_like(Bp)
    plan.run(3, Ap, Bp, Xp)
    st = plan.status()
    assert np.all(st["status"] == 0), st
    assert np.median(st["eta0"]) > 1e-6       # the FP32 factors alone are poor
    for i in range(len(sizes)):
        x = plan.unpack_vec(Xp, i).cpu().numpy()
        assert oracle.backward_error(mats[i].numpy(), x, bs[i].numpy()) <= 1e-14


def test_batched_escalation_launch(B):
    """tol = 0 cannot be met: every system stalls in GMRES-IR and goes through
    the double-float escalation launch, which refines it to FP64 accuracy."""
    sizes = [40, 130, 257]
    plan = B.BatchedPlan(sizes, 2, kind=0, max_iter=10, tol=0.0, escalate=True)
    mats, _, bs = systems(sizes, 2, 17)
    Ap, Bp = plan.pack(mats, bs)
    Xp = torch.empty_like(Bp)
    plan.run(4, Ap, Bp, Xp)
    st = plan.status()
    assert np.all(st["escalated"] == 2)
    for i in range(len(sizes)):
        x = plan.unpack_vec(Xp, i).cpu().numpy()
        assert oracle.backward_error(mats[i].numpy(), x, bs[i].numpy()) <= 1e-14


def test_batched_fp32_circulant_unrefined_and_refined(B):
    n, batch, nrhs = 128, 3, 8
    A, X, Bm = W.shifted(batch, n, nrhs, seed=2, dtype=torch.float32)
    for refine in (0, 10):
        plan = B.BatchedPlan([n] * batch, nrhs, kind=1, a_dtype=torch.float32, max_iter=refine, tol=1e-15)
        Ap = A.reshape(-1).to(DEV)
        Bp = Bm.double().reshape(-1).to(DEV)
        Xp = torch.empty_like(Bp)
        plan.run(9, Ap, Bp, Xp)
        st = plan.status()
        for i in range(batch):
            Ai = A[i].double().numpy()
            bi = Bm[i].double().numpy()
            x = plan.unpack_vec(Xp, i).cpu().numpy()
            eta = oracle.backward_error(Ai, x, bi)
            if refine:
                assert eta <= 1e-14
            else:   # FP32 factors alone: u32 times the element growth (about 1e2 here)
                assert eta <= 1e-4 and st["iters"][i] == 0


def test_batched_adjoint_vs_oracle(B):
    n, batch, nrhs = 64, 2, 3
    A, _, Bm = W.shifted(batch, n, nrhs, seed=5, dtype=torch.float32)
    plan = B.BatchedPlan([n] * batch, nrhs, kind=1, a_dtype=torch.float32, max_iter=10, tol=1e-16)
    Ap, Bp = A.reshape(-1).to(DEV), Bm.double().reshape(-1).to(DEV)
    Xp = torch.empty_like(Bp)
    plan.run(3, Ap, Bp, Xp)
    dA = torch.empty(plan.mat_size, dtype=torch.float32, device=DEV)
    dB = torch.empty_like(Bp)
    plan.adjoint(Ap, Xp, Xp, dA, dB)      # loss 0.5 ||X||^2: gX = X
    for i in range(batch):
        Ai, x = A[i].double().numpy(), plan.unpack_vec(Xp, i).cpu().numpy()
        dA_ref, dB_ref = oracle.adjoint(Ai, x, x)
        got_A = dA[plan.mat_off[i]:plan.mat_off[i + 1]].view(n, n).cpu().double().numpy()
        got_B = plan.unpack_vec(dB, i).cpu().numpy()
        # Lambda is refined in FP64 (1e-10); dA is then rounded to float
        assert np.linalg.norm(got_B - dB_ref) <= 1e-10 * np.linalg.norm(dB_ref)
        assert np.linalg.norm(got_A - dA_ref) <= 1e-6 * np.linalg.norm(dA_ref)
    # unrefined adjoint (max_iter = 0): FP32-factor accuracy only
    plan0 = B.BatchedPlan([n] * batch, nrhs, kind=1, a_dtype=torch.float32, max_iter=0)
    plan0.run(3, Ap, Bp, Xp)
    plan0.adjoint(Ap, Xp, Xp, None, dB)
    x = plan.unpack_vec(Xp, 0).cpu().numpy()
    assert np.linalg.norm(plan0.unpack_vec(dB, 0).cpu().numpy() - oracle.adjoint(A[0].double().numpy(), x, x)[1]) \
        <= 1e-3 * np.linalg.norm(x)


def test_autograd_fp64_vs_finite_differences_and_oracle(B):
    """Loss = sum(x^2) at n = 64 in FP64: gradient vs central differences
    (h = 1e-6, 1e-6 normwise over sampled entries) and vs the oracle gradient
    (1e-10)."""
    n, batch, nrhs = 64, 2, 2
    A, _, Bm = W.shifted(batch, n, nrhs, seed=11)
    Ad = A.to(DEV).requires_grad_(True)
    Bd = Bm.to(DEV).requires_grad_(True)
    X = B.genp_solve(Ad, Bd, kind=1, seed=4)
    loss = (X ** 2).sum()
    loss.backward()
    for b in range(batch):
        Ab, Bb = A[b].numpy(), Bm[b].numpy()
        x = oracle.gepp_solve(Ab, Bb)
        dA_ref, dB_ref = oracle.adjoint(Ab, x, 2 * x)
        assert np.linalg.norm(Ad.grad[b].cpu().numpy() - dA_ref) <= 1e-10 * np.linalg.norm(dA_ref)
        assert np.linalg.norm(Bd.grad[b].cpu().numpy() - dB_ref) <= 1e-10 * np.linalg.norm(dB_ref)
    rng = np.random.default_rng(0)
    h = 1e-6
    fd, an = [], []

    def lossf(Am, Bm_):
        with torch.no_grad():
            return float((B.genp_solve(Am, Bm_, kind=1, seed=4) ** 2).sum())

    for _ in range(10):
        b, i, j = rng.integers(0, batch), rng.integers(0, n), rng.integers(0, n)
        E = torch.zeros_like(Ad)
        E[b, i, j] = h
        fd.append((lossf(Ad.detach() + E, Bd.detach()) - lossf(Ad.detach() - E, Bd.detach())) / (2 * h))
        an.append(float(Ad.grad[b, i, j]))
    fd, an = np.array(fd), np.array(an)
    assert np.linalg.norm(fd - an) <= 1e-6 * np.linalg.norm(an)


def test_autograd_fp32_close_to_fp64(B):
    n, batch, nrhs = 128, 2, 8
    A, _, Bm = W.shifted(batch, n, nrhs, seed=12, dtype=torch.float32)
    A32 = A.to(DEV).requires_grad_(True)
    B32 = Bm.to(DEV).requires_grad_(True)
    (B.genp_solve(A32, B32, kind=1) ** 2).sum().backward()
    A64 = A.double().to(DEV).requires_grad_(True)
    B64 = Bm.double().to(DEV).requires_grad_(True)
    (B.genp_solve(A64, B64, kind=1) ** 2).sum().backward()
    # FP32 factors, forward and adjoint refined in FP64: only the float32
    # outputs (X, dA) are rounded
    assert torch.linalg.norm(A32.grad.double() - A64.grad) <= 1e-6 * torch.linalg.norm(A64.grad)
    assert torch.linalg.norm(B32.grad.double() - B64.grad) <= 1e-6 * torch.linalg.norm(B64.grad)


def test_batched_graph_replay_matches_eager(B):
    sizes = [16, 40, 100, 33, 250, 64]
    plan = B.BatchedPlan(sizes, 4, kind=0, max_iter=8, tol=1e-15)
    mats, _, bs = systems(sizes, 4, 21)
    Ap, Bp = plan.pack(mats, bs)
    X_eager = torch.empty_like(Bp)
    plan.run(1, Ap, Bp, X_eager)
    torch.cuda.synchronize()
    X_graph = torch.empty_like(Bp)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.run(1, Ap, Bp, X_graph)          # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    X_graph.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.run(1, Ap, Bp, X_graph)
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(X_graph, X_eager)


def test_batched_autotune(B):
    sizes = [20, 50, 120, 300, 600]
    plan = B.BatchedPlan(sizes, 4, kind=0, max_iter=8, tol=1e-15, autotune=True, escalate=True)
    for n in sizes:
        assert plan.block_size(n) in (64, 128)
    mats, _, bs = systems(sizes, 4, 8)
    Ap, Bp = plan.pack(mats, bs)
    Xp = torch.empty_like(Bp)
    plan.run(2, Ap, Bp, Xp)
    st = plan.status()
    assert np.all(st["eta"] <= 1e-14)
