"""Batched form (many independent instances in one network object),
checkpoint/resume and the autotuner (needs a GPU)."""
import numpy as np
import pytest
import torch

import oracle
import snn_inputs as I

pytestmark = pytest.mark.gpu


def _instances(weight_hi=0.05, sizes=(1000, 2500, 777, 5000, 1234, 3000), steps=400):
    rng = np.random.default_rng(9)
    scales = np.exp(rng.uniform(np.log(0.1), np.log(10.0), len(sizes)))
    return [I.config_small(steps=steps, n_hh=n, user_scale=float(c), instance=b, weight_hi=weight_hi)
            for b, (n, c) in enumerate(zip(sizes, scales))]


def test_batch_equals_standalone_runs_subthreshold(gpu):
    specs = _instances()
    batch = gpu.Network.from_specs(specs)
    batch.step(400)
    for b, spec in enumerate(specs):
        solo = gpu.Network.from_spec(spec)
        solo.step(400)
        o = batch.pop_offsets[b]
        for k in range(2):
            assert batch.counters(o + k) == solo.counters(k)
        assert np.abs(batch.read_host(o + 1, "V") - solo.read_host(1, "V")).max() < 1e-5
        assert np.array_equal(batch.read_host(o, "spikes"), solo.read_host(0, "spikes"))


def test_batch_equals_standalone_runs_spiking(gpu):
    specs = _instances(weight_hi=60.0, steps=1500)
    for eng in (0, 1):
        batch = gpu.Network.from_specs(specs)
        batch.set_option("engine", eng)
        batch.step(1500)
        for b, spec in enumerate(specs):
            solo = gpu.Network.from_spec(spec)
            solo.step(1500)
            o = batch.pop_offsets[b]
            cb, cs = batch.counters(o + 1)[0], solo.counters(1)[0]
            assert abs(cb - cs) <= 0.02 * cs + 1, (eng, b, cb, cs)
            assert batch.counters(o + 1)[1] == solo.counters(1)[1] == 0


def test_batch_instances_match_oracle(gpu):
    specs = _instances(sizes=(300, 520), steps=120)
    batch = gpu.Network.from_specs(specs)
    refs = [oracle.from_spec(s) for s in specs]
    for t in range(120):
        batch.step()
        for b, ref in enumerate(refs):
            ref.step()
            o = batch.pop_offsets[b]
            assert np.array_equal(batch.read_host(o, "spikes"), ref.spikes(0))
            assert np.abs(batch.read_host(o + 1, "V") - ref.get(1, "V")).max() <= 1e-3


def test_snapshot_resume_reproduces_the_run(gpu):
    spec = I.config_four_pop(steps=300, n_mid=2000)
    net = gpu.Network.from_spec(spec)
    net.step(100)
    snap = net.save_state()
    host_snap = snap.cpu()
    net.step(150)
    want_v = [net.read_host(p, "V") for p in range(4)]
    want_c = [net.counters(p) for p in range(4)]
    want_s = net.read_host(0, "spikes")
    for buf in (snap, host_snap):
        net.load_state(buf)
        assert net.t == 100
        net.step(150)
        assert net.t == 250
        for p in range(4):
            assert np.abs(net.read_host(p, "V") - want_v[p]).max() < 1e-5
            assert net.counters(p) == want_c[p]
        assert np.array_equal(net.read_host(0, "spikes"), want_s)
    # into a fresh network built from the same description
    other = gpu.Network.from_spec(spec)
    other.load_state(host_snap)
    other.step(150)
    assert np.abs(other.read_host(1, "V") - want_v[1]).max() < 1e-5


def test_snapshot_of_another_shape_is_rejected(gpu):
    import paper_1412_0595_gb300 as snn
    a = gpu.Network.from_spec(I.config_small(steps=1, n_hh=300))
    b = gpu.Network.from_spec(I.config_small(steps=1, n_hh=400))
    with pytest.raises(snn.SNNError) as e:
        b.load_state(a.save_state())
    assert e.value.name == "SNN_ERR_STATE"


def test_autotune_picks_a_configuration_and_keeps_the_trajectory(gpu):
    spec = I.config_four_pop(steps=300, n_mid=3000)
    a = gpu.Network.from_spec(spec)
    b = gpu.Network.from_spec(spec)
    a.step(50)
    b.step(50)
    r = a.autotune(trial_steps=100)
    assert r["engine"] in ("plain", "persistent", "cluster") and r["us_per_step"] > 0 and not r["cached"]
    assert a.t == 50
    a.step(200)
    b.step(200)
    for p in range(4):
        assert np.abs(a.read_host(p, "V") - b.read_host(p, "V")).max() < 1e-4
        assert a.counters(p) == b.counters(p)
    c = gpu.Network.from_spec(spec)
    assert c.autotune(trial_steps=100)["cached"]


def test_occupancy_configuration_is_the_plain_step_and_keeps_the_trajectory(gpu):
    # the paper's occupancy rule (Sec. 3) as a baseline beside the autotuner
    spec = I.config_four_pop(steps=300, n_mid=3000)
    a = gpu.Network.from_spec(spec)
    b = gpu.Network.from_spec(spec)
    a.step(50)
    b.step(50)
    r = a.occupancy_config(trial_steps=100)
    assert r["engine"] == "plain" and r["tiled"] == 0 and r["chunk"] == 1024 and not r["cached"]
    assert r["prop_blocks"] % 152 == 0 and r["us_per_step"] > 0
    assert a.engine == "plain" and a.t == 50
    a.step(200)
    b.step(200)
    for p in range(4):
        assert np.abs(a.read_host(p, "V") - b.read_host(p, "V")).max() < 1e-4
        assert a.counters(p) == b.counters(p)
    with pytest.raises(Exception):
        gpu.GradedNetwork.from_spec(I.config_graded_small(steps=10)).occupancy_config()
