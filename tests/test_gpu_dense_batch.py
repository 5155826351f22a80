"""Dense delivery for batched instances sharing one projection, on the CUDA
cores and on the tensor cores (tcgen05, three BF16 parts of W, FP32
accumulation), against the FP64 definition (needs a GPU)."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


def _case(B, n_pre, n_post, frac, seed=0, empty_rows=()):
    rng = np.random.default_rng(seed)
    W = rng.lognormal(-3.0, 0.5, (n_pre, n_post)).astype(np.float32)
    spikes = []
    for b in range(B):
        k = 0 if b in empty_rows else max(1, int(rng.binomial(n_pre, frac)))
        spikes.append(np.sort(rng.choice(n_pre, min(k, n_pre), replace=False)))
    scale = rng.uniform(0.1, 10.0, B).astype(np.float32)
    G0 = rng.uniform(0.0, 1.0, (B, n_post)).astype(np.float32)
    return W, spikes, scale, G0


def _run(gpu, engine, W, spikes, scale, G0, ld_pad=0):
    h = gpu.DenseBatch(W)
    G = torch.zeros((len(spikes), W.shape[1] + ld_pad), dtype=torch.float32, device="cuda")
    G[:, : W.shape[1]] = torch.from_numpy(G0).cuda()
    h.deliver(spikes, scale, G, engine=engine)
    h.check()
    out = G[:, : W.shape[1]].cpu().numpy().astype(np.float64)
    tail = G[:, W.shape[1]:].cpu().numpy()
    h.close()
    return out, tail


def _close(got, want):
    # FP32 accumulation: 1e-5 of each row's largest delivered magnitude
    scale = np.maximum(np.abs(want).max(axis=1, keepdims=True), 1e-30)
    return np.abs(got - want) <= 1e-5 * scale


@pytest.mark.parametrize("engine", ["cuda", "tensor"])
def test_single_ragged_tile(gpu, engine):
    # sizes that fill no tile: 5 instances, 70 pre, 200 post; one instance
    # without spikes; rows padded in G (ldg > n_post) stay untouched
    W, spikes, scale, G0 = _case(5, 70, 200, 0.3, empty_rows=(2,))
    got, tail = _run(gpu, engine, W, spikes, scale, G0, ld_pad=3)
    want = oracle.dense_batch_deliver(W.astype(np.float64), spikes, scale, G0)
    assert np.all(_close(got, want))
    assert np.array_equal(got[2], G0[2].astype(np.float64))
    assert np.all(tail == 0.0)


@pytest.mark.parametrize("engine", ["cuda", "tensor"])
@pytest.mark.parametrize("frac", [0.01, 0.3, 1.0])
def test_many_tiles(gpu, engine, frac):
    # 300 instances (3 row tiles, the last ragged), 1000 pre (16 K tiles),
    # 1000 post (8 column tiles)
    W, spikes, scale, G0 = _case(300, 1000, 1000, frac, seed=1)
    got, _ = _run(gpu, engine, W, spikes, scale, G0)
    want = oracle.dense_batch_deliver(W.astype(np.float64), spikes, scale, G0)
    assert np.all(_close(got, want))


def test_tensor_split_carries_all_of_the_weights(gpu):
    # one spike per instance: the result is scale * one row of W, which the
    # three BF16 parts must reproduce to FP32 rounding (a single part would
    # be off by ~2^-9)
    rng = np.random.default_rng(3)
    W = rng.uniform(0.5, 1.0, (64, 128)).astype(np.float32)
    spikes = [np.array([b]) for b in range(64)]
    scale = np.ones(64, np.float32)
    G0 = np.zeros((64, 128), np.float32)
    got, _ = _run(gpu, "tensor", W, spikes, scale, G0)
    assert np.abs(got - W.astype(np.float64)).max() <= 2.0 ** -23


def test_bad_spike_index_is_reported(gpu):
    import paper_1412_0595_gb300 as snn
    W, spikes, scale, G0 = _case(3, 40, 50, 0.2)
    spikes[1] = np.array([3, 40])                  # 40 is outside [0, 40)
    h = gpu.DenseBatch(W)
    G = torch.zeros((3, 50), dtype=torch.float32, device="cuda")
    h.deliver(spikes, scale, G, engine="tensor")
    with pytest.raises(snn.SNNError):
        h.check()
    h.close()
