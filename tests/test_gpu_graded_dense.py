"""Differentiable form with dense (Eq. 2) storage on the GPU against the FP64
oracle: the dense forward product, the dense rows of the adjoint gather, and
the weight gradient as a rank-K product per checkpoint segment on the tensor
cores (three BF16 parts per operand, six products) and on the CUDA cores."""
import numpy as np
import pytest
import torch

import snn_inputs as I
from oracle.graded import GradedOracle

pytestmark = pytest.mark.gpu


def _rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _cos(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


def _mse(net, target, K, backward=True):
    """Recorded forward, squared-error loss of y (torch) and, optionally, the
    adjoint seeded by its dL/dy."""
    from paper_1412_0595_gb300.network import squared_error
    tgt = target if isinstance(target, torch.Tensor) else torch.from_numpy(target)
    y = net.forward_record(tgt.shape[0], checkpoint_every=K)
    loss, dl = squared_error(y, tgt)
    if not backward:
        return loss, y
    gs, gw = net.backward(dl)
    return loss, y, gs, gw


def _smooth_dense_spec(n_pre=12, n_mid=18, n_out=6):
    # no spikes: clamped pre cells near the release threshold drive passive
    # cells whose releases are centred at rest, so every weight matters
    import test_oracle_graded as TG
    pops = [I.hh_pop(n_pre, v0_range=(-26.0, -14.0)), TG._passive(n_mid), TG._passive(n_out)]
    pops[0]["hh"]["C"] = 1e300
    for d in pops[1:]:
        d["v0_range"] = (-64.0, -60.0)
    projs = [TG._graded_proj(0, 1, 0.0), TG._graded_proj(1, 1, 0.0), TG._graded_proj(1, 2, 0.0)]
    for d, wmax in zip(projs, (5.0, 1.0, 5.0)):
        d["layout"] = "dense"
        d["weight"] = ("uniform", 0.0, wmax)
    projs[1]["v_thr"] = projs[2]["v_thr"] = -62.0
    return I.net(pops, projs, dt=0.05, steps=1)


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("sizes", [(12, 18, 6), (40, 150, 20), (64, 300, 130)])
def test_dense_gradients_match_oracle_smooth_network(gpu, engine, sizes):
    # ragged sizes: 150 and 130 posts are not multiples of 4 (scalar paths of
    # the forward product and the gather); 300 rows span three 128-row tiles
    spec = _smooth_dense_spec(*sizes)
    T = 400
    net = gpu.GradedNetwork.from_spec(spec)
    net.set_option("dense_grad", engine)
    ref = GradedOracle(spec)
    target = I.target_trace(spec, T, ref.n_out)
    loss, _, gs, gw = _mse(net, target, 100)
    rloss, _ = ref.forward(target.astype(np.float64))
    rgs, rgw = ref.backward()
    assert loss == pytest.approx(rloss, rel=1e-5)
    assert _rel_l2(gs.cpu().numpy(), rgs) < 1e-4
    for q in range(3):
        assert gw[q].numel() == ref.nnz[q]
        assert _rel_l2(gw[q].cpu().numpy(), rgw[q]) < 1e-4, q


def test_dense_forward_matches_oracle_200_neuron_copy(gpu):
    T = 2000
    spec = I.config_graded_dense_small(steps=T)
    net = gpu.GradedNetwork.from_spec(spec)
    ref = GradedOracle(spec)
    target = I.target_trace(spec, T, ref.n_out)
    loss, y = _mse(net, target, 100, backward=False)
    rloss, ry = ref.forward(target.astype(np.float64))
    assert loss == pytest.approx(rloss, rel=1e-3)
    assert np.abs(y.cpu().numpy() - ry).max() < 0.05


@pytest.mark.parametrize("engine", [0, 1])
def test_dense_gradients_match_oracle_before_divergence(gpu, engine):
    # 200 steps of the spiking 200-neuron copy: the FP32 trajectory still
    # follows the FP64 one
    T = 200
    spec = I.config_graded_dense_small(steps=T)
    net = gpu.GradedNetwork.from_spec(spec)
    net.set_option("dense_grad", engine)
    ref = GradedOracle(spec)
    target = I.target_trace(spec, T, ref.n_out)
    _, _, gs, gw = _mse(net, target, 64)
    ref.forward(target.astype(np.float64))
    rgs, rgw = ref.backward()
    assert _rel_l2(gs.cpu().numpy(), rgs) < 1e-3
    for q in range(3):
        assert _rel_l2(gw[q].cpu().numpy(), rgw[q]) < 2e-3, q
        assert _cos(gw[q].cpu().numpy(), rgw[q]) > 0.99999, q


def test_tensor_and_cuda_core_gradients_agree_for_every_segment_length(gpu):
    # segment lengths 1 (one K tile of padding), 37 (ragged K tile), 100 and
    # 512 (16 K tiles through the four-stage pipeline); 300 posts and rows
    # (three ragged tiles each way).  Both engines carry FP32 accuracy, so
    # they agree to FP32 rounding; the forward is bit-identical throughout.
    T = 600
    spec = I.config_graded_dense_small(steps=T, n_mid=300)
    net = gpu.GradedNetwork.from_spec(spec)
    target = torch.from_numpy(I.target_trace(spec, T, spec["pops"][2]["n"]))
    losses = []
    for K in (1, 37, 100, 512):
        got = []
        for engine in (0, 1):
            net.set_option("dense_grad", engine)
            loss, _, gs, gw = _mse(net, target, K)
            losses.append(loss)
            got.append((gs.cpu().numpy(), [g.cpu().numpy() for g in gw]))
        (gs0, gw0), (gs1, gw1) = got
        assert np.allclose(gs0, gs1, rtol=1e-12, atol=0), K   # dL/ds does not depend on the engine
        for q in (1, 2):
            assert _rel_l2(gw1[q], gw0[q]) < 1e-5, (K, q)
        assert np.array_equal(gw1[0], gw0[0]), K           # compressed rows: same kernel
    assert all(l == losses[0] for l in losses)


def test_dense_weights_can_be_set_and_change_the_loss(gpu):
    # new Mid -> Out weights (ten times stronger) on both sides; 1000 steps so
    # the middle population has spiked and the projection moves the loss.
    # The stronger drive makes the output population spike, after which FP32
    # and FP64 part (the R17 reading): 1e-2.  Writing the creation weights
    # back restores the first loss bit for bit (the forward is deterministic).
    T = 1000
    spec = I.config_graded_dense_small(steps=T)
    net = gpu.GradedNetwork.from_spec(spec)
    ref = GradedOracle(spec)
    target = torch.from_numpy(I.target_trace(spec, T, ref.n_out))
    l0 = _mse(net, target, 100, backward=False)[0]
    rl0, _ = ref.forward(target.numpy().astype(np.float64))
    w = np.random.default_rng(3).uniform(0.0, 600.0, ref.nnz[2]).astype(np.float32)
    net.set_weights(2, torch.from_numpy(w).cuda())
    l1 = _mse(net, target, 100, backward=False)[0]
    for k in range(ref.nnz[2]):
        ref.set_weight(2, k, float(w[k]))
    rl1, _ = ref.forward(target.numpy().astype(np.float64))
    assert abs(rl1 - rl0) > 1e-1 * rl0                 # the change matters
    assert l0 == pytest.approx(rl0, rel=1e-3)
    assert l1 == pytest.approx(rl1, rel=1e-2)
    w0 = I.weights(spec, 2, ref.nnz[2]).astype(np.float32)
    net.set_weights(2, torch.from_numpy(w0).cuda())
    assert _mse(net, target, 100, backward=False)[0] == l0
