"""Pins of the oracle's HH neuron, synapse and step order against closed
forms, special cases and invariants (the paper prints no HH example)."""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
import snn_inputs as I

TR = I.TRAUB


def test_rate_special_values():
    a_m, b_m, a_h, b_h, a_n, b_n = range(6)
    # removable singularities: the linoid limit k * A
    assert oracle.hh_rates(-52.0)[a_m] == pytest.approx(1.28, rel=1e-14)
    assert oracle.hh_rates(-25.0)[b_m] == pytest.approx(1.4, rel=1e-14)
    assert oracle.hh_rates(-50.0)[a_n] == pytest.approx(0.16, rel=1e-14)
    # exponential rates at their reference voltage
    assert oracle.hh_rates(-48.0)[a_h] == pytest.approx(0.128, rel=1e-14)
    assert oracle.hh_rates(-25.0)[b_h] == pytest.approx(2.0, rel=1e-14)
    assert oracle.hh_rates(-55.0)[b_n] == pytest.approx(0.5, rel=1e-14)
    # the exponential scales: halving / tripling points
    assert oracle.hh_rates(-48.0 + 18.0 * math.log(2.0))[a_h] == pytest.approx(0.064, rel=1e-13)
    assert oracle.hh_rates(-25.0 + 5.0 * math.log(3.0))[b_h] == pytest.approx(3.0, rel=1e-13)
    assert oracle.hh_rates(-55.0 - 40.0 * math.log(2.0))[b_n] == pytest.approx(1.0, rel=1e-13)
    # linear asymptotes of the linoid rates far from their singularity
    assert oracle.hh_rates(100.0)[a_m] == pytest.approx(0.32 * 152.0, rel=1e-12)
    assert oracle.hh_rates(-200.0)[b_m] == pytest.approx(0.28 * 175.0, rel=1e-12)
    assert oracle.hh_rates(100.0)[a_n] == pytest.approx(0.032 * 150.0, rel=1e-12)


@pytest.mark.parametrize("v0", [-52.0, -25.0, -50.0])
def test_rates_continuous_across_singularities(v0):
    for eps in (1e-9, 1e-7, 1e-5, 1e-3):
        lo, hi = oracle.hh_rates(v0 - eps), oracle.hh_rates(v0 + eps)
        mid = oracle.hh_rates(v0)
        assert np.allclose(lo, mid, rtol=5 * eps + 1e-13) and np.allclose(hi, mid, rtol=5 * eps + 1e-13)


def test_current_special_cases():
    V = -20.0
    I1 = oracle.hh_currents(TR, V, 1.0, 1.0, 1.0)
    assert I1[0] == pytest.approx(TR["gNa"] * (V - TR["ENa"]), rel=1e-15)
    assert I1[1] == pytest.approx(TR["gK"] * (V - TR["EK"]), rel=1e-15)
    assert I1[2] == pytest.approx(TR["gL"] * (V - TR["EL"]), rel=1e-15)
    Ih = oracle.hh_currents(TR, V, 0.5, 1.0, 0.5)
    assert Ih[0] == pytest.approx(TR["gNa"] / 8 * (V - TR["ENa"]), rel=1e-15)   # m^3
    assert Ih[1] == pytest.approx(TR["gK"] / 16 * (V - TR["EK"]), rel=1e-15)    # n^4
    Ihh = oracle.hh_currents(TR, V, 1.0, 0.25, 0.0)
    assert Ihh[0] == pytest.approx(TR["gNa"] / 4 * (V - TR["ENa"]), rel=1e-15)  # linear in h
    assert Ihh[1] == 0.0
    assert np.all(oracle.hh_currents(TR, TR["ENa"], 1, 1, 0)[0] == 0.0)


def _one(hh=None, v0=-60.0, **kw):
    pop = I.hh_pop(1, v0_range=(v0, v0), **kw)
    if hh:
        pop["hh"].update(hh)
    return pop


def test_passive_membrane_closed_form():
    # gNa = gK = 0: V_k = EL + (V0 - EL)(1 - hs gL / C)^k for k Euler substeps
    spec = I.net([_one(dict(gNa=0.0, gK=0.0), v0=-40.0)], [], dt=0.1, n_sub=4, steps=1)
    net = oracle.from_spec(spec)
    v0 = float(np.float32(-40.0))
    hs = 0.1 / 4
    for steps in (1, 10, 250):
        net2 = oracle.from_spec(spec)
        net2.step(steps)
        want = TR["EL"] + (v0 - TR["EL"]) * (1 - hs * TR["gL"] / TR["C"]) ** (4 * steps)
        assert net2.get(0, "V")[0] == pytest.approx(want, rel=1e-13)
    del net


def test_voltage_clamp_gating_closed_form():
    # huge C freezes V; each gate is then a linear ODE whose Euler iterate is
    # x_k = x_inf + (x_0 - x_inf)(1 - hs (alpha + beta))^k
    V = -45.0
    spec = I.net([_one(dict(C=1e300), v0=V)], [], dt=0.1, n_sub=4, steps=1)
    net = oracle.from_spec(spec)
    Vf = float(np.float32(V))
    x0 = {"m": 0.9, "h": 0.1, "n": 0.7}
    for f, v in x0.items():
        net.set(0, f, [v])
    steps, hs = 30, 0.025
    net.step(steps)
    a = oracle.hh_rates(Vf)
    for f, (al, be) in {"m": (a[0], a[1]), "h": (a[2], a[3]), "n": (a[4], a[5])}.items():
        xinf = al / (al + be)
        want = xinf + (x0[f] - xinf) * (1 - hs * (al + be)) ** (4 * steps)
        assert net.get(0, f)[0] == pytest.approx(want, rel=1e-12), f
    assert net.get(0, "V")[0] == Vf


def _steady_current(V):
    a = oracle.hh_rates(V)
    m, h, n = a[0] / (a[0] + a[1]), a[2] / (a[2] + a[3]), a[4] / (a[4] + a[5])
    return oracle.hh_currents(TR, V, m, h, n).sum()


def test_resting_fixed_point_and_saddle():
    v_rest = brentq(_steady_current, -70.0, -60.0, xtol=1e-13)
    v_saddle = brentq(_steady_current, -60.0, -55.0, xtol=1e-13)
    assert v_rest == pytest.approx(-63.3021, abs=1e-4)
    assert v_saddle == pytest.approx(-57.5253, abs=1e-4)
    # the integrated, undriven neuron relaxes onto the static root from both sides
    for v0 in (-62.0, -58.0, -66.0):
        net = oracle.from_spec(I.net([_one(v0=v0)], [], dt=0.1, steps=1))
        net.step(20000)
        assert net.get(0, "V")[0] == pytest.approx(v_rest, abs=1e-6)
        assert 0.0 <= net.get(0, "m")[0] <= 1.0


def test_synaptic_reversal_fixed_point():
    # passive cell with a constant conductance g on channel 0 (no decay):
    # V* = (gL EL + g E) / (gL + g)
    g, E = 10.0, 0.0
    spec = I.net([_one(dict(gNa=0.0, gK=0.0), tau_syn=(1e300, 1.0), E_syn=(E, -92.0))], [],
                 dt=0.1, steps=1)
    net = oracle.from_spec(spec)
    net.set(0, "g0", [g])
    net.step(5000)
    want = (TR["gL"] * TR["EL"] + g * E) / (TR["gL"] + g)
    assert net.get(0, "V")[0] == pytest.approx(want, abs=1e-9)
    assert net.get(0, "isyn")[0] == pytest.approx(g * (E - want), rel=1e-9)


def test_spike_rule_is_upward_crossing_of_threshold():
    spec = I.net([_one(v0=-63.3, drive=dict(rate_hz=0.0, amp=0.0, tau=1e300))], [], dt=0.1, steps=1)
    net = oracle.from_spec(spec)
    net.set(0, "iext", [300.0])
    prev = net.get(0, "V")[0]
    crossings, listed = [], []
    for t in range(3000):
        net.step()
        v = net.get(0, "V")[0]
        if prev < 0.0 <= v:
            crossings.append(t)
        if len(net.spikes(0)):
            listed.append(t)
        prev = v
    assert len(crossings) > 5 and crossings == listed
    assert net.counters(0)[0] == len(crossings)


def test_synapse_jump_decay_and_one_step_delay():
    # a source that spikes every step (p = 1) onto one HH cell through w:
    # after step t the conductance is s w (1 - d^(t+1)) / (1 - d), d = exp(-dt/tau)
    w, tau, dt, c = 0.75, 2.0, 0.1, 2.5
    pops = [I.source_pop(1, 1.0 / (dt * 1e-3)), _one(tau_syn=(tau, 1.0))]
    spec = I.net(pops, [I.proj(0, 1, "csr", 1.0, ("const", w, 0.0), user_scale=c)], dt=dt, steps=1)
    net = oracle.from_spec(spec)
    s = oracle.gscale(1.0, 0.0, 0.0, 1.0) * c
    assert net.scale(0) == pytest.approx(s, rel=1e-15)
    d = math.exp(-dt / tau)
    w32 = float(np.float32(w))
    g_prev = 0.0
    for t in range(40):
        v_start = net.get(1, "V")[0]
        net.step()
        assert net.get(1, "isyn")[0] == pytest.approx(g_prev * (0.0 - v_start), rel=1e-13, abs=1e-300)
        g = net.get(1, "g0")[0]
        assert g == pytest.approx(s * w32 * (1 - d ** (t + 1)) / (1 - d), rel=1e-13)
        g_prev = g


def test_nan_states_are_counted_every_step():
    spec = I.net([I.hh_pop(10)], [], dt=0.1, steps=1)
    net = oracle.from_spec(spec)
    v = net.get(0, "V")
    v[[2, 5, 7]] = np.nan
    net.set(0, "V", v)
    net.step(4)
    assert net.counters(0)[1] == 3 * 4
    assert np.isnan(net.get(0, "V")).sum() == 3


def test_dense_and_csr_propagation_equal_matvec():
    rng = np.random.default_rng(5)
    n_pre, n_post = 24, 37
    spec = I.net([I.source_pop(n_pre, 0.0), I.hh_pop(n_post), I.hh_pop(n_post)],
                 [I.proj(0, 1, "csr", 0.3, ("uniform", 0.0, 1.0)),
                  I.proj(0, 2, "dense", 0.3, ("uniform", 0.0, 1.0))], dt=0.1, steps=1)
    spec["projs"][1]["weight"] = spec["projs"][0]["weight"]
    net = oracle.from_spec(spec)
    rp, col = oracle.csr_bernoulli(spec["seed"], I.rng_tag(0, 0), n_pre, n_post, 0.3)
    w = I.weights(spec, 0, len(col)).astype(np.float64)
    W = np.zeros((n_pre, n_post))
    W[np.repeat(np.arange(n_pre), np.diff(rp)), col] = w
    spk = np.sort(rng.choice(n_pre, 9, replace=False)).astype(np.int32)
    net.deliver(0, spk)
    x = np.zeros(n_pre)
    x[spk] = 1.0
    want = net.scale(0) * (W.T @ x)
    assert np.allclose(net.get(1, "g0"), want, rtol=1e-14, atol=0)
    # projection 1 has its own draws (different tag) but the same law: check vs its own matvec
    rp1, col1 = oracle.csr_bernoulli(spec["seed"], I.rng_tag(0, 1), n_pre, n_post, 0.3)
    w1 = I.weights(spec, 1, len(col1)).astype(np.float64)
    W1 = np.zeros((n_pre, n_post))
    W1[np.repeat(np.arange(n_pre), np.diff(rp1)), col1] = w1
    net.deliver(1, spk)
    assert np.allclose(net.get(2, "g0"), net.scale(1) * (W1.T @ x), rtol=1e-14, atol=0)


def test_gating_stays_in_unit_interval_under_drive():
    spec = I.net([I.hh_pop(50, drive=dict(I.INPUT_DRIVE))], [], dt=0.1, steps=1)
    net = oracle.from_spec(spec)
    for _ in range(50):
        net.step(40)
        for f in ("m", "h", "n"):
            x = net.get(0, f)
            assert np.all(x >= 0.0) and np.all(x <= 1.0)
    assert net.counters(0)[0] > 0
