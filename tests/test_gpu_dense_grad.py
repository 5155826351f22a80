"""Rank-K update D += R^T N (the dense weight gradient over a checkpoint
segment) on the tensor cores and on the CUDA cores, through the C-ABI,
against the FP64 definition (needs a GPU)."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


def _case(K, m, n, seed=0, pad=(0, 0, 0)):
    rng = np.random.default_rng(seed)
    R = rng.uniform(0.0, 1.0, (K, m + pad[0])).astype(np.float32)       # releases in (0, 1)
    N = rng.normal(0.0, 1.0, (n, K + pad[1])).astype(np.float32)        # dL/dG of either sign
    D0 = rng.normal(0.0, 1.0, (m, n + pad[2])).astype(np.float32)
    return R, N, D0


def _bound(R, N, K):
    # FP32 sum of K products: |error| <= c K 2^-24 sum_t |r n|; the three-part
    # BF16 split drops terms below 2^-24 of each product (c = 2, K + 8)
    return 2.0 * (K + 8) * 2.0 ** -24 * (np.abs(R.astype(np.float64)).T @ np.abs(N.astype(np.float64)).T)


def _run(gpu, R, N, D0, m, n, K, engine):
    h = gpu.DenseGrad()
    Rt = torch.from_numpy(R).cuda()[:, :m]
    Nt = torch.from_numpy(N).cuda()[:, :K]
    Dt = torch.from_numpy(D0).cuda()
    h.run(Rt, Nt, Dt[:, :n], engine=engine)
    h.check()
    out = Dt.cpu().numpy()
    h.close()
    return out


@pytest.mark.parametrize("engine", ["cuda", "tensor"])
@pytest.mark.parametrize("K,m,n", [(1, 5, 7), (16, 128, 128), (37, 300, 250), (100, 129, 513), (512, 200, 140)])
def test_rank_update_matches_definition(gpu, engine, K, m, n):
    # one tile, exact tiles, ragged tiles in every dimension, the longest
    # segment (16 K tiles through the four-stage pipeline); strided R, N, D
    R, N, D0 = _case(K, m, n, seed=K + m, pad=(3, 5, 2))
    got = _run(gpu, R, N, D0, m, n, K, engine)
    want = oracle.dense_grad_update(R[:, :m], N[:, :K], D0[:, :n])
    err = np.abs(got[:, :n] - want)
    assert np.all(err <= _bound(R[:, :m], N[:, :K], K) + 2.0 ** -24 * np.abs(want)), err.max()
    assert np.array_equal(got[:, n:], D0[:, n:])         # the stride padding stays untouched


def test_tensor_split_carries_fp32_operands(gpu):
    # K = 1 with operands whose low bits matter: D = r n exactly representable
    # only with all three parts of both operands (one BF16 part would be off
    # by ~2^-9 relative)
    rng = np.random.default_rng(4)
    m, n = 64, 96
    R = (1.0 + rng.integers(0, 2 ** 23, (1, m)) * 2.0 ** -23).astype(np.float32)
    N = (1.0 + rng.integers(0, 2 ** 11, (n, 1)) * 2.0 ** -11).astype(np.float32)
    D0 = np.zeros((m, n), np.float32)
    got = _run(gpu, R, N, D0, m, n, 1, "tensor")
    want = R[0].astype(np.float64)[:, None] * N[:, 0].astype(np.float64)[None, :]
    assert np.abs(got - want).max() <= 4 * 2.0 ** -24 * np.abs(want).max()


def test_full_size_rank_update_sampled(gpu):
    # the dense recurrent projection of the 4096-neuron workload over one
    # 100-step segment, checked on sampled rows against the definition
    K, m, n = 100, 4096, 4096
    R, N, D0 = _case(K, m, n, seed=11)
    got = _run(gpu, R, N, D0, m, n, K, "tensor")
    rows = np.random.default_rng(1).choice(m, 64, replace=False)
    want = oracle.dense_grad_update(R[:, rows], N, D0[rows])
    assert np.all(np.abs(got[rows] - want) <= _bound(R[:, rows], N, K) + 2.0 ** -24 * np.abs(want))


def test_bad_arguments_are_rejected(gpu):
    import paper_1412_0595_gb300 as snn
    from paper_1412_0595_gb300 import _lib as L
    h = gpu.DenseGrad()
    D = torch.zeros(4, 4, device="cuda")
    R = torch.zeros(600, 4, device="cuda")
    N = torch.zeros(4, 600, device="cuda")
    with pytest.raises(snn.SNNError):                       # K above 512
        h.run(R, N, D)
    with pytest.raises(snn.SNNError):                       # ldr < m
        L.check(L.lib.snn_dense_grad_run(h.h, R.data_ptr(), 2, N.data_ptr(), 600, 4, 4, 8, D.data_ptr(), 4, 1, None))
    h.close()
