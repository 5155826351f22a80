"""A dense projection shared by every instance of a batch, delivered on the
time-step path (snn_add_shared_dense): each instance against its own FP64
oracle network holding the same W with the instance's scale, on the CUDA
cores, on the tensor cores (W in three BF16 parts, FP32 accumulation) and
with the per-step choice by spike density."""
import numpy as np
import pytest
import torch

import oracle
import snn_inputs as I

pytestmark = pytest.mark.gpu

N_PRE, N_POST = 200, 300


def _rel_ok(got, want, rel=1e-5):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    floor = 1e-5 * np.abs(want).max() if want.size else 0.0
    return np.all(np.abs(got - want) <= rel * np.maximum(np.abs(want), floor) + 1e-30)


def _batch(gpu, n_inst, rate_hz, seed=7):
    specs = [I.net([I.source_pop(N_PRE, rate_hz), I.hh_pop(N_POST)], [], dt=0.1, steps=1, instance=b)
             for b in range(n_inst)]
    rng = np.random.default_rng(seed)
    W = rng.uniform(0.0, 0.03, (N_PRE, N_POST)).astype(np.float32)   # subthreshold drive: V compares tightly
    scales = np.exp(rng.uniform(np.log(0.1), np.log(10.0), n_inst))
    net = gpu.Network.from_specs(specs)
    net.add_shared_dense(0, 1, torch.from_numpy(W), scales)
    refs = []
    for b, sp in enumerate(specs):
        pops = [dict(sp["pops"][0], v0=None), dict(sp["pops"][1], v0=I.v0(sp, 1).astype(np.float64))]
        proj = dict(pre=0, post=1, layout="dense", channel=0, w=W.astype(np.float64).ravel(), k1=1.0, k2=0.0, k3=0.0,
                    n_conn=float(N_PRE), user_scale=float(scales[b]))
        refs.append(oracle.OracleNet(pops, [proj], sp["dt"], sp["n_sub"], sp["seed"], b))
    return net, refs


@pytest.mark.parametrize("engine,rate_hz", [(0, 2000.0), (1, 2000.0), (2, 2000.0), (2, 20.0), (1, 20.0)])
def test_shared_dense_batch_matches_each_instance_oracle(gpu, engine, rate_hz):
    # 2000 Hz sources: 20 % of the pre neurons spike per step (the density
    # choice takes the tensor cores); 20 Hz: 0.2 % (the CUDA cores)
    n_inst = 40
    net, refs = _batch(gpu, n_inst, rate_hz)
    net.set_option("shared_dense", engine)
    assert net.engine == "plain"
    for t in range(60):
        net.step()
        for r in refs:
            r.step()
        if t % 10 == 9 or t == 0:
            for b, r in enumerate(refs):
                o = net.pop_offsets[b]
                assert np.array_equal(net.read_host(o, "spikes"), r.spikes(0)), (t, b)
                assert _rel_ok(net.read_host(o + 1, "g0"), r.get(1, "g0")), (t, b)
                vo = r.get(1, "V")
                assert vo.max() < -57.5253
                assert np.abs(net.read_host(o + 1, "V") - vo).max() <= 1e-3, (t, b)
    # synaptic events: every spike of a pre population times n_post
    spikes = sum(net.counters(net.pop_offsets[b])[0] for b in range(n_inst))
    assert net.synaptic_events() == spikes * N_POST


def test_shared_dense_engines_agree_over_many_steps(gpu):
    a, _ = _batch(gpu, 24, 2000.0)
    b, _ = _batch(gpu, 24, 2000.0)
    a.set_option("shared_dense", 0)
    b.set_option("shared_dense", 1)
    a.step(300)
    b.step(300)
    for k in range(24):
        o = a.pop_offsets[k] + 1
        ga, gb = a.read_host(o, "g0"), b.read_host(o, "g0")
        assert np.abs(ga - gb).max() <= 1e-5 * np.abs(ga).max()
        assert np.abs(a.read_host(o, "V") - b.read_host(o, "V")).max() < 1e-4


def test_shared_dense_rejects_instances_of_other_shapes(gpu):
    import paper_1412_0595_gb300 as snn
    specs = [I.net([I.source_pop(N_PRE, 20.0), I.hh_pop(N_POST + b)], [], dt=0.1, steps=1, instance=b)
             for b in range(3)]
    net = gpu.Network.from_specs(specs)
    with pytest.raises(snn.SNNError) as e:
        net.add_shared_dense(0, 1, torch.zeros((N_PRE, N_POST)), [1.0, 1.0, 1.0])
    assert e.value.name == "SNN_ERR_INVALID_ARG"
