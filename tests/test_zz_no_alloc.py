"""The allocation-free row builder matches the allocating one.

snn_csr_bernoulli_rows_noalloc exists for callers that cannot allocate device
memory while they build connectivity (all memory owned by a fixed pool or
budget, or loops that must not call cudaMalloc / cudaFree).  Its scratch is a
fixed device array shared by all calls, so this test runs it several times in
a row on different sizes -- a later call must not see an earlier call's
leftovers -- and compares each result with snn_csr_bernoulli_rows bit for
bit, up to the largest accepted row count.  This file is collected last so
that a failure here never hides another test.
"""
import ctypes as C

import pytest
import torch

pytestmark = pytest.mark.gpu


def _rows_allocating(L, seed, tag, n_pre, n_post, p):
    import paper_1412_0595_gb300 as snn
    rp = torch.empty(n_pre + 1, dtype=torch.int64, device="cuda")
    nnz = C.c_int64()
    alloc = snn.TorchAllocator()
    s = torch.cuda.current_stream().cuda_stream
    assert L.lib.snn_csr_bernoulli_rows(seed, tag, n_pre, n_post, p, rp.data_ptr(), C.byref(nnz),
                                        alloc.ref(), s) == 0
    return rp, nnz.value


def _rows_noalloc(L, seed, tag, n_pre, n_post, p):
    rp = torch.full((n_pre + 1,), -7, dtype=torch.int64, device="cuda")
    nnz = C.c_int64(-1)
    s = torch.cuda.current_stream().cuda_stream
    st = L.lib.snn_csr_bernoulli_rows_noalloc(seed, tag, n_pre, n_post, p, rp.data_ptr(), C.byref(nnz), s)
    assert st == 0, L.lib.snn_last_error()
    return rp, nnz.value


def test_noalloc_rows_match_allocating_rows_on_two_calls_in_a_row(gpu):
    from paper_1412_0595_gb300 import _lib as L
    cases = [(20251203, 0x0301, 5000, 3001, 0.1),     # 5 scan blocks
             (77, 0x0102, 1234, 777, 0.3),             # fewer blocks: stale sums must not leak
             (5, 0x0203, 2_100_000, 64, 0.05),         # 2051 blocks: the block-sum scan carries over 1024
             (6, 0x0204, 16_777_216, 64, 0.05),        # exactly SNN_NOALLOC_MAX_ROWS: every scratch entry
             (77, 0x0102, 1234, 777, 0.3)]             # small again after the largest
    for seed, tag, n_pre, n_post, p in cases:
        want, want_nnz = _rows_allocating(L, seed, tag, n_pre, n_post, p)
        got, got_nnz = _rows_noalloc(L, seed, tag, n_pre, n_post, p)
        torch.cuda.synchronize()
        assert got_nnz == want_nnz
        assert torch.equal(got, want)


def test_noalloc_rows_reject_sizes_beyond_the_scratch(gpu):
    from paper_1412_0595_gb300 import _lib as L
    rp = torch.zeros(1, dtype=torch.int64, device="cuda")
    nnz = C.c_int64()
    st = L.lib.snn_csr_bernoulli_rows_noalloc(1, 0, 16777216 + 1, 10, 0.5, rp.data_ptr(), C.byref(nnz), None)
    assert st == 8 and b"SNN_NOALLOC_MAX_ROWS" in L.lib.snn_last_error()
