"""Differentiable form on the GPU against the FP64 oracle: recorded forward
(the output filter y) and the discrete adjoint (dL/ds, dL/dw) seeded by a
caller's dL/dy, for the squared-error loss and for another loss of y."""
import numpy as np
import pytest
import torch

import snn_inputs as I  # noqa: E402
from oracle.graded import GradedOracle

pytestmark = pytest.mark.gpu


def _rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _cos(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


def _pair(gpu, spec, T):
    net = gpu.GradedNetwork.from_spec(spec)
    ref = GradedOracle(spec)
    target = I.target_trace(spec, T, ref.n_out)
    return net, ref, target


def _mse(gpu, net, target, K, backward=True):
    """Recorded forward, squared-error loss on top of y (torch), and the
    adjoint seeded by its dL/dy: (loss, y, dL/ds, dL/dw)."""
    from paper_1412_0595_gb300.network import squared_error
    T = target.shape[0]
    y = net.forward_record(T, checkpoint_every=K)
    loss, dl = squared_error(y, torch.from_numpy(target))
    if not backward:
        return loss, y, None, None
    gs, gw = net.backward(dl)
    return loss, y, gs, gw


def test_graded_forward_matches_oracle_200_neuron_copy(gpu):
    T = 2000
    spec = I.config_graded_small(steps=T)
    net, ref, target = _pair(gpu, spec, T)
    loss, y, _, _ = _mse(gpu, net, target, 100, backward=False)
    rloss, ry = ref.forward(target.astype(np.float64))
    assert loss == pytest.approx(rloss, rel=1e-3)
    assert np.abs(y.cpu().numpy() - ry).max() < 0.05
    assert net.t == T


def test_graded_gradients_match_oracle_adjoint_before_divergence(gpu):
    # 200 steps (10 ms): the FP32 trajectory still follows the FP64 one
    T = 200
    spec = I.config_graded_small(steps=T)
    net, ref, target = _pair(gpu, spec, T)
    _, _, gs, gw = _mse(gpu, net, target, 64)
    ref.forward(target.astype(np.float64))
    rgs, rgw = ref.backward()                       # the oracle's own squared-error adjoint
    assert _rel_l2(gs.cpu().numpy(), rgs) < 1e-3
    for q in range(3):
        assert _rel_l2(gw[q].cpu().numpy(), rgw[q]) < 2e-3, q
        assert _cos(gw[q].cpu().numpy(), rgw[q]) > 0.99999, q


def test_gradients_of_another_loss_match_the_oracle_adjoint_with_the_same_dl_dy(gpu):
    # a loss of y other than the squared error, mean |y - target|^3: both
    # adjoints are seeded with the same dL/dy (taken from the GPU's y)
    T = 200
    spec = I.config_graded_small(steps=T)
    net, ref, target = _pair(gpu, spec, T)
    y = net.forward_record(T, checkpoint_every=64)
    d = y - torch.from_numpy(target).cuda()
    dl = 3.0 * d.abs() * d / d.numel()
    gs, gw = net.backward(dl)
    ref.forward(target.astype(np.float64))
    rgs, rgw = ref.backward(dL_dy=dl.double().cpu().numpy())
    assert np.all(np.abs(rgs) > 0)
    assert _rel_l2(gs.cpu().numpy(), rgs) < 1e-3
    for q in range(3):
        assert _rel_l2(gw[q].cpu().numpy(), rgw[q]) < 2e-3, q
        assert _cos(gw[q].cpu().numpy(), rgw[q]) > 0.99999, q
    # dL/dy is linear in the seed: twice the seed, twice the gradients
    gs2, _ = net.backward(2.0 * dl)
    assert torch.allclose(gs2, 2.0 * gs, rtol=1e-6, atol=0)


def test_graded_gradients_match_oracle_adjoint_smooth_network(gpu):
    # no spikes: clamped pre cells near threshold drive passive cells
    import test_oracle_graded as TG
    pops = [I.hh_pop(20, v0_range=(-26.0, -14.0)), TG._passive(30), TG._passive(10)]
    pops[0]["hh"]["C"] = 1e300
    for d in pops[1:]:
        d["v0_range"] = (-64.0, -60.0)
    projs = [TG._graded_proj(0, 1, 0.0, p=0.5), TG._graded_proj(1, 1, 0.0, p=0.3), TG._graded_proj(1, 2, 0.0, p=0.5)]
    for d, wmax in zip(projs, (5.0, 1.0, 5.0)):
        d["weight"] = ("uniform", 0.0, wmax)
    projs[1]["v_thr"] = projs[2]["v_thr"] = -62.0
    spec = I.net(pops, projs, dt=0.05, steps=1)
    T = 600
    net, ref, target = _pair(gpu, spec, T)
    loss, _, gs, gw = _mse(gpu, net, target, 100)
    rloss, _ = ref.forward(target.astype(np.float64))
    rgs, rgw = ref.backward()
    assert loss == pytest.approx(rloss, rel=1e-5)
    assert _rel_l2(gs.cpu().numpy(), rgs) < 1e-4
    for q in range(3):
        assert _rel_l2(gw[q].cpu().numpy(), rgw[q]) < 1e-4, q


def test_graded_gradients_2000_steps_output_projection(gpu):
    # over the full 2000 steps the spiking middle population amplifies FP32
    # rounding; the output projection's gradient stays well conditioned
    T = 2000
    spec = I.config_graded_small(steps=T)
    net, ref, target = _pair(gpu, spec, T)
    _, _, gs, gw = _mse(gpu, net, target, 100)
    ref.forward(target.astype(np.float64))
    rgs, rgw = ref.backward()
    assert gs[2].item() == pytest.approx(rgs[2], rel=1e-2)
    assert _rel_l2(gw[2].cpu().numpy(), rgw[2]) < 2e-2
    assert _cos(gw[2].cpu().numpy(), rgw[2]) > 0.999
    assert torch.isfinite(gs).all() and all(torch.isfinite(g).all() for g in gw)


def test_checkpoint_interval_does_not_change_the_gradient(gpu):
    T = 600
    spec = I.config_graded_small(steps=T)
    net, ref, target = _pair(gpu, spec, T)
    out = []
    for K in (100, 37, 512):
        l, _, gs, gw = _mse(gpu, net, target, K)
        out.append((l, gs.cpu().numpy(), [g.cpu().numpy() for g in gw]))
    for l, gs, gw in out[1:]:
        assert l == out[0][0]                                   # the forward is deterministic
        assert np.allclose(gs, out[0][1], rtol=1e-5, atol=0)
        for q in range(3):
            assert _rel_l2(gw[q], out[0][2][q]) < 1e-5


@pytest.mark.parametrize("spec_fn", [I.config_graded_small, I.config_graded_dense_small])
def test_stored_trajectory_gives_the_recomputed_gradients(gpu, spec_fn):
    # the recorded forward keeps every step (SNN_OPT_GRADED_STORE 1) or only
    # checkpoints whose segments the backward recomputes (0): the recompute is
    # bit-identical, so are the states the adjoint reads
    T = 300
    spec = spec_fn(steps=T)
    net, ref, target = _pair(gpu, spec, T)
    out = []
    for store in (0, 1):
        net.set_option("graded_store", store)
        l, y, gs, gw = _mse(gpu, net, target, 64)
        out.append((l, y.cpu().numpy(), gs.cpu().numpy(), [g.cpu().numpy() for g in gw]))
    (l0, y0, s0, w0), (l1, y1, s1, w1) = out
    assert l0 == l1 and np.array_equal(y0, y1)
    assert np.allclose(s0, s1, rtol=1e-6, atol=0)             # FP64 sums of FP32 terms in atomic order
    for a, b in zip(w0, w1):
        assert np.array_equal(a, b)


def test_autograd_function_and_a_descent_step(gpu):
    # y from the autograd node, any torch loss on top; autograd's dL/dy
    # reaches the network's adjoint
    from paper_1412_0595_gb300.network import squared_error
    T = 400
    spec = I.config_graded_small(steps=T)
    net, ref, target = _pair(gpu, spec, T)
    tgt = torch.from_numpy(target).cuda()
    scales = torch.tensor([ref.scale(q) for q in range(3)], dtype=torch.float64, device="cuda", requires_grad=True)
    ws = [torch.from_numpy(ref.rows[q][2].astype(np.float32)).cuda().requires_grad_(True) for q in range(3)]
    y = gpu.SNNFunction.apply(net, T, 2, 5.0, 100, scales, *ws)
    assert tuple(y.shape) == (T, ref.n_out)
    loss = ((y - tgt) ** 2).mean() + 0.1 * (y - tgt).abs().mean()
    loss.backward()
    d = (y - tgt).detach()
    gs, gw = net.backward(2.0 * d / d.numel() + 0.1 * torch.sign(d) / d.numel())
    assert torch.allclose(scales.grad.float(), gs, rtol=1e-6, atol=0)
    assert torch.allclose(ws[0].grad, gw[0], rtol=1e-6, atol=1e-12 * gw[0].abs().max().item())
    with torch.no_grad():                                      # a small step downhill on the scales
        new_scales = scales * (1.0 - 1e-5 * torch.sign(scales.grad))
    y2 = gpu.SNNFunction.apply(net, T, 2, 5.0, 100, new_scales, *[w.detach() for w in ws])
    loss2 = ((y2 - tgt) ** 2).mean() + 0.1 * (y2 - tgt).abs().mean()
    assert loss2.item() < loss.item()
    mse, _ = squared_error(y2, tgt)
    assert mse == pytest.approx(((y2.double() - tgt.double()) ** 2).mean().item(), rel=1e-12)


def test_full_size_differentiable_workload_first_100_steps(gpu):
    # 20,000 middle neurons, three projections at p = 0.05 (2e7 recurrent synapses)
    T = 100
    spec = I.config_graded(steps=T)
    net, ref, target = _pair(gpu, spec, T)
    loss, _, gs, gw = _mse(gpu, net, target, 50)
    rloss, _ = ref.forward(target.astype(np.float64))
    assert loss == pytest.approx(rloss, rel=1e-4)
    rgs, rgw = ref.backward()
    assert _rel_l2(gs.cpu().numpy(), rgs) < 1e-3
    for q in range(3):
        assert _cos(gw[q].cpu().numpy(), rgw[q]) > 0.9999, q
    assert all(torch.isfinite(g).all() for g in gw)


def test_backward_without_forward_is_rejected(gpu):
    import paper_1412_0595_gb300 as snn
    net = gpu.GradedNetwork.from_spec(I.config_graded_small(steps=10))
    with pytest.raises(snn.SNNError) as e:
        net.backward(torch.zeros((10, 20), device="cuda"))
    assert e.value.name == "SNN_ERR_STATE"



def _fan_in_spec(n_in, n_out, p, T):
    """In (driven, started between -30 and -10 mV so that it releases from
    the first step) -> Out through one graded projection: the forward
    product's paths by the pre population's size (16- or 32-bit transposed
    indices) and by the posts' row lengths (stages of whole posts with a warp
    or a lane per post, or a warp per post from HBM when a post is longer than
    a stage)."""
    pops = [I.hh_pop(n_in, v0_range=(-30.0, -10.0), drive=dict(I.INPUT_DRIVE)), I.hh_pop(n_out)]
    pr = I.proj(0, 1, "csr", p, ("uniform", 0.0, I.GRADED_WEIGHTS[0]))
    pr.update(synapse="graded", v_thr=I.GRADED["v_thr"], v_slope=I.GRADED["v_slope"])
    return I.net(pops, [pr], dt=0.05, steps=T)


@pytest.mark.parametrize("n_in,n_out,p", [
    (70000, 40, 0.02),      # 32-bit pre indices, 1,400 synapses per post
    (6000, 24, 0.8),        # 4,800 synapses per post: longer than a stage
    (3000, 600, 0.002),     # 6 synapses per post: a lane per post
])
def test_forward_product_paths_match_oracle(gpu, n_in, n_out, p):
    # the scale gradient sums G over every post and step, so an error in the
    # product shows in it directly
    T = 20
    spec = _fan_in_spec(n_in, n_out, p, T)
    net, ref, target = _pair(gpu, spec, T)
    loss, y, gs, gw = _mse(gpu, net, target, 10)
    rloss, ry = ref.forward(target.astype(np.float64))
    assert loss == pytest.approx(rloss, rel=1e-4)
    assert np.abs(y.cpu().numpy() - ry).max() < 1e-3
    rgs, rgw = ref.backward()
    assert _rel_l2(gs.cpu().numpy(), rgs) < 1e-3
    assert _cos(gw[0].cpu().numpy(), rgw[0]) > 0.9999


def test_product_launch_leaves_the_state_and_rejects_spiking_networks(gpu):
    # snn_graded_launch_product (the timing entry point of the forward
    # product) advances nothing; a spiking network has no graded product
    import paper_1412_0595_gb300 as snn
    from paper_1412_0595_gb300 import _lib as L
    from paper_1412_0595_gb300.network import _stream
    spec = I.config_graded_small(steps=20)
    net = gpu.GradedNetwork.from_spec(spec)
    net.step(5)
    before = [net.read_host(p, f).copy() for p in range(3) for f in ("V", "m", "h", "n")]
    for _ in range(3):
        net.launch_product()
    net.sync()
    after = [net.read_host(p, f) for p in range(3) for f in ("V", "m", "h", "n")]
    assert all(np.array_equal(x, y) for x, y in zip(before, after))
    assert net.t == 5
    spiking = gpu.Network.from_spec(I.config_small(steps=10, n_hh=300))
    with pytest.raises(snn.SNNError) as e:
        L.check(L.lib.snn_graded_launch_product(spiking.h, _stream(None)))
    assert e.value.name == "SNN_ERR_STATE"
