"""genp_make_sparse_noalloc: the allocation-free entry point for callers that
cannot call cudaMalloc (their device memory belongs to another allocator, or
they must not pay the synchronization an allocation can cause).

It must produce exactly the multiplier the allocating path produces
(genp_make_multiplier + genp_multiplier_export); the data is integer, so the
comparison is bit for bit, as in the other multiplier tests.  Two calls in a
row check that the shared device scratch carries nothing over between calls.
This file is collected last so that a failing run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
ARG = -1


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(lib, n, nnz, seed, sid, stream):
    rows = torch.full((nnz, n), -7, dtype=torch.int32, device=DEV)
    signs = torch.zeros((nnz, n), dtype=torch.int8, device=DEV)
    inv_rows = torch.full((nnz, n), -7, dtype=torch.int32, device=DEV)
    inv_signs = torch.zeros((nnz, n), dtype=torch.int8, device=DEV)
    st = lib.genp_make_sparse_noalloc(n, nnz, seed, sid, _p(rows), _p(signs), _p(inv_rows), _p(inv_signs),
                                      ctypes.c_void_p(stream.cuda_stream))
    assert st == 0
    return rows, signs, inv_rows, inv_signs


def _allocating(n, nnz, seed, sid):
    import paper_1212_4560_gb300 as genp
    G = genp.make_multiplier(genp.SPARSE_PM1, n, seed=seed, stream_id=sid, nnz_per_col=nnz)
    rows = torch.empty((nnz, n), dtype=torch.int32, device=DEV)
    signs = torch.empty((nnz, n), dtype=torch.int8, device=DEV)
    genp.multiplier_export(G, rows=rows, signs=signs)
    torch.cuda.synchronize()
    return rows.cpu().numpy(), signs.cpu().numpy()


def test_noalloc_matches_allocating_path_twice(genp_lib):
    lib = genp_lib
    stream = torch.cuda.current_stream()
    # two calls in a row: a larger draw, then a smaller one with another seed,
    # so stale scratch from the first call would show up in the second
    for n, nnz, seed, sid in ((50_000, 4, 11, 0), (7_001, 4, 12, 3)):
        rows, signs, inv_rows, inv_signs = _noalloc(lib, n, nnz, seed, sid, stream)
        torch.cuda.synchronize()
        ref_rows, ref_signs = _allocating(n, nnz, seed, sid)
        r, s = rows.cpu().numpy(), signs.cpu().numpy()
        assert np.array_equal(r, ref_rows)
        assert np.array_equal(s, ref_signs)
        ir, isg = inv_rows.cpu().numpy(), inv_signs.cpu().numpy()
        for t in range(nnz):
            assert np.array_equal(ir[t][r[t]], np.arange(n))       # inverse permutation
            assert np.array_equal(isg[t][r[t]], s[t])


def test_noalloc_accepts_exactly_its_scratch(genp_lib):
    """n * nnz_per_col equal to GENP_NOALLOC_MAX_ENTRIES (2^20) fills the
    scratch array to its last entry and must still match the allocating path."""
    n, nnz = 1 << 18, 4
    rows, signs, _, _ = _noalloc(genp_lib, n, nnz, 5, 1, torch.cuda.current_stream())
    torch.cuda.synchronize()
    ref_rows, ref_signs = _allocating(n, nnz, 5, 1)
    assert np.array_equal(rows.cpu().numpy(), ref_rows)
    assert np.array_equal(signs.cpu().numpy(), ref_signs)


def test_noalloc_rejects_sizes_beyond_its_scratch(genp_lib):
    lib = genp_lib
    limit = 1 << 20
    dummy = torch.zeros(8, dtype=torch.int32, device=DEV)
    p = _p(dummy)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.genp_make_sparse_noalloc(limit // 4 + 1, 4, 1, 0, p, p, p, p, s) == ARG
    assert lib.genp_make_sparse_noalloc(limit + 1, 1, 1, 0, p, p, p, p, s) == ARG
    assert lib.genp_make_sparse_noalloc(16, 4, 1, 0, None, p, p, p, s) == ARG
    torch.cuda.synchronize()
    assert torch.all(dummy == 0)
