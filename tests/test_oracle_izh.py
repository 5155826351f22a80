"""Pins of the oracle's Izhikevich population (the cortical network of Sec.
5.1, neuron model of the paper's ref. [9]) against closed forms and
invariants of that model: the rest point on the v- and u-nullclines, the
onset of firing (the rest point's loss of stability at I_H and its
disappearance at the saddle-node current I* = (5 - b)^2 / 0.16 - 140), the
reset rule, and the moments and lattice of the counter-based draws."""
import math

import numpy as np
import pytest

import oracle
import snn_inputs as I


def _one(bias, v0, izh=None, steps=1, dt=1.0, n_sub=2):
    izh = dict(izh or I.IZH_EXC)
    izh.update(noise=0.0, bias=float(bias))
    pop = dict(kind="izh", n=1, izh=izh, v0_range=(v0, v0), E_syn=(0.0, 0.0), tau_syn=(0.0, 0.0),
               v_thresh=30.0)
    return oracle.from_spec(I.net([pop], [], dt=dt, n_sub=n_sub, steps=steps))


def _rest(b, bias):
    # rest point: 0.04 v^2 + (5 - b) v + 140 + I = 0 (u = b v), the lower root
    disc = (5.0 - b) ** 2 - 0.16 * (140.0 + bias)
    return (-(5.0 - b) - math.sqrt(disc)) / 0.08


@pytest.mark.parametrize("bias", [0.0, 2.0, 3.5])
def test_rest_point_is_a_fixed_point(bias):
    v = _rest(0.2, bias)
    if bias == 0.0:
        assert v == pytest.approx(-70.0, abs=1e-12)
    net = _one(bias, v)
    net.set(0, "m", np.array([0.2 * v]))          # u on its nullcline
    net.step(2000)
    assert net.get(0, "V")[0] == pytest.approx(v, abs=1e-9)
    assert net.get(0, "m")[0] == pytest.approx(0.2 * v, abs=1e-9)
    assert net.counters(0) == (0, 0)


def test_onset_of_firing():
    # The rest point exists for I <= I* = (5 - b)^2 / 0.16 - 140 = 4 (saddle-node)
    # and is stable while the trace of the Jacobian, 0.08 v* + 5 - a, is
    # negative: v* < v_H = (a - 5) / 0.08 = -62.25, i.e. I < I_H = 3.7975.
    a, b = 0.02, 0.2
    i_star = (5.0 - b) ** 2 / 0.16 - 140.0
    assert i_star == pytest.approx(4.0, abs=1e-12)
    v_h = (a - 5.0) / 0.08
    i_h = -(0.04 * v_h * v_h + (5.0 - b) * v_h + 140.0)
    assert i_h == pytest.approx(3.7975, abs=1e-12)
    # below I_H: a 1 mV kick off the rest point decays without a spike
    v_rest = _rest(b, 3.5)
    below = _one(3.5, v_rest + 1.0)
    below.set(0, "m", np.array([b * v_rest]))
    below.step(5000)
    assert below.counters(0)[0] == 0
    assert below.get(0, "V")[0] == pytest.approx(v_rest, abs=1e-3)
    # between I_H and I*: the rest point is unstable, the same kick ends in spikes
    v_rest = _rest(b, 3.9)
    mid = _one(3.9, v_rest + 1.0)
    mid.set(0, "m", np.array([b * v_rest]))
    mid.step(5000)
    assert mid.counters(0)[0] > 0
    # above I*: no rest point, a neuron started at the I = 0 rest fires
    above = _one(i_star + 0.2, -70.0)
    above.step(5000)
    assert above.counters(0)[0] > 0


def test_reset_sets_c_and_spike_list():
    # a strongly driven population: every listed neuron sits exactly at its c
    spec = I.net([I.izh_pop(64, excitatory=True, bias=20.0, noise=0.0)], [], dt=1.0, n_sub=2, steps=50)
    net = oracle.from_spec(spec)
    seen = 0
    for _ in range(50):
        net.step()
        spk = net.spikes(0)
        v = net.get(0, "V")
        for i in spk:
            r = oracle.izh_r(spec["seed"], 0, int(i))
            assert v[i] == -65.0 + 15.0 * r * r
        seen += len(spk)
    assert seen > 0


def test_parameter_draw_lattice_and_moments():
    r = np.array([oracle.izh_r(12345, 7, i) for i in range(20000)])
    assert np.all((r >= 0.0) & (r < 1.0))
    assert np.all(r * 2.0 ** 24 == np.floor(r * 2.0 ** 24))
    assert abs(r.mean() - 0.5) < 5 * math.sqrt(1 / 12 / len(r))


def test_irwin_hall_noise_moments_and_lattice():
    z = np.array([oracle.izh_noise(12345, 3, t, i) for t in range(40) for i in range(1000)])
    n = len(z)
    assert np.all((z >= -6.0) & (z < 6.0))
    assert np.all(z * 2.0 ** 20 == np.floor(z * 2.0 ** 20))
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / n) + 1e-3
    # Irwin-Hall(12) - 6 has kurtosis 3 - 1.2 / 12 = 2.9 (a normal has 3)
    kurt = ((z - z.mean()) ** 4).mean() / z.var() ** 2
    assert abs(kurt - 2.9) < 0.05
    # distinct neurons and steps draw distinct values
    assert len(np.unique(z)) > 0.9 * n


def test_noise_enters_as_a_current():
    # with u at rest and no synapses, one substep of v moves by hs * sigma * z
    spec = I.net([I.izh_pop(3, excitatory=True, noise=5.0)], [], dt=1.0, n_sub=1, steps=1)
    net = oracle.from_spec(spec)
    v0 = net.get(0, "V").copy()
    u0 = net.get(0, "m").copy()
    net.step()
    z = np.array([oracle.izh_noise(spec["seed"], 0, 0, i) for i in range(3)])
    dv = 0.04 * v0 * v0 + 5.0 * v0 + 140.0 - u0
    assert np.allclose(net.get(0, "V"), v0 + 1.0 * (dv + 5.0 * z), rtol=0, atol=1e-12)


def test_excitatory_inhibitory_parameters():
    # inhibitory neurons: a = 0.02 + 0.08 r, b = 0.25 - 0.05 r, so u0 = b v0
    spec = I.net([I.izh_pop(50, excitatory=False)], [], dt=1.0, n_sub=2, steps=1)
    net = oracle.from_spec(spec)
    r = np.array([oracle.izh_r(spec["seed"], 0, i) for i in range(50)])
    assert np.allclose(net.get(0, "m"), (0.25 - 0.05 * r) * -65.0, rtol=0, atol=1e-12)
    assert np.allclose(net.get(0, "h"), r, rtol=0, atol=0)


def test_threaded_step_matches_sequential():
    # the multi-threaded step (used for the all-core timing) gives the same
    # spikes; neuron states are bit-identical, conductances equal to rounding
    import snn_inputs as I2
    spec = I2.config_four_pop(steps=200, n_mid=2000)
    a = oracle.from_spec(spec)
    oracle.set_threads(4)
    try:
        b = oracle.from_spec(spec)
        for t in range(200):
            oracle.set_threads(1)
            a.step()
            oracle.set_threads(4)
            b.step()
            for p in range(4):
                assert np.array_equal(a.spikes(p), b.spikes(p)), (t, p)
        for p in range(4):
            assert np.allclose(a.get(p, "V"), b.get(p, "V"), rtol=0, atol=1e-9)
            assert np.allclose(a.get(p, "g0"), b.get(p, "g0"), rtol=1e-12, atol=1e-15)
            assert a.counters(p) == b.counters(p)
        assert a.events == b.events
    finally:
        oracle.set_threads(1)
