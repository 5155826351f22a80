"""Pins of the FP64 graded-synapse oracle and of its discrete adjoint:
rate derivatives against finite differences of the rates, closed-form
steady states of the graded conductance path, the output filter recursion,
and central finite differences of the loss against the adjoint."""
import math

import numpy as np
import pytest

import oracle
import snn_inputs as I
from oracle.graded import GradedOracle, hh_rate_derivs


@pytest.mark.parametrize("V", [-90.0, -70.0, -52.0, -50.0, -48.0, -25.0, -10.0, 10.0, 40.0])
def test_rate_derivatives_match_finite_differences(V):
    h = 1e-5
    fd = (oracle.hh_rates(V + h) - oracle.hh_rates(V - h)) / (2 * h)
    # central differences of rates O(1) with h = 1e-5 carry ~1e-10 rounding noise
    assert np.allclose(hh_rate_derivs(V), fd, rtol=1e-7, atol=1e-9)


def _clamped(n, v):
    p = I.hh_pop(n, v0_range=(v, v))
    p["hh"]["C"] = 1e300          # V never moves
    return p


def _passive(n, v0=-63.563):
    p = I.hh_pop(n, v0_range=(v0, v0))
    p["hh"].update(gNa=0.0, gK=0.0)
    return p


def _graded_proj(pre, post, w, p=1.0):
    d = I.proj(pre, post, "csr", p, ("const", w, 0.0))
    d.update(synapse="graded", v_thr=-20.0, v_slope=2.0)
    return d


def test_graded_conductance_steady_state_closed_form():
    # three clamped pre neurons at -24, -20, -16 mV drive one passive cell
    # through weights w: G = w sum_i r_i, r_i = 1 / (1 + exp((-20 - V_i)/2));
    # steady state V* = (gL EL + s G E) / (gL + s G), s = gScale(1/(p N_pre)) = 1/3
    pops = [_clamped(1, -24.0), _clamped(1, -20.0), _clamped(1, -16.0), _passive(1)]
    w = 4.0
    projs = [_graded_proj(k, 3, w) for k in range(3)]
    spec = I.net(pops, projs, dt=0.05, steps=1)
    g = GradedOracle(spec, out_pop=3)
    T = 6000
    loss, y = g.forward(np.zeros((T, 1)))
    tr = I.TRAUB
    G = sum(w / (1.0 + math.exp((-20.0 - v) / 2.0)) for v in (-24.0, -20.0, -16.0))
    s = 1.0                       # each projection has p = 1, N_pre = 1
    v_star = (tr["gL"] * tr["EL"] + s * G * 0.0) / (tr["gL"] + s * G)
    assert y[-1, 0] == pytest.approx(v_star, abs=1e-6)
    assert g.scale(0) == pytest.approx(1.0)


def test_output_filter_recursion_and_loss():
    # a passive output cell relaxing from -40 mV: V_t = EL + (V0 - EL)(1 - hs gL/C)^(4t);
    # y_{t+1} = y_t + (dt/tau)(V_{t+1} - y_t), y_0 = V_0; loss = mean (y - target)^2
    tr = I.TRAUB
    spec = I.net([_passive(1, -40.0)], [], dt=0.05, steps=1)
    tau = 5.0
    g = GradedOracle(spec, out_pop=0, tau_f=tau)
    T = 300
    target = np.linspace(-50.0, -60.0, T)[:, None]
    loss, y = g.forward(target)
    hs, a = 0.05 / 4, 0.05 / tau
    v0 = float(np.float32(-40.0))
    yy, want = v0, []
    for t in range(T):
        v = tr["EL"] + (v0 - tr["EL"]) * (1 - hs * tr["gL"] / tr["C"]) ** (4 * (t + 1))
        yy = yy + a * (v - yy)
        want.append(yy)
    want = np.array(want)
    assert np.allclose(y[:, 0], want, rtol=0, atol=1e-10)
    assert loss == pytest.approx(np.mean((want - target[:, 0]) ** 2), rel=1e-12)


def _fd_check(g, target, scale_step=1e-8, weight_step=1e-7, n_weights=3, seed=0):
    """Worst relative error of central differences against the adjoint over
    all scales and, per projection, the largest-gradient and some random
    weights; gradients below 1e-3 of their projection's largest are judged
    against that floor (finite differences cannot resolve them)."""
    g.forward(target)
    gs, gw = g.backward()
    worst = 0.0
    for q in range(len(gs)):
        s0 = g.scale(q)
        h = scale_step * abs(s0)
        g.set_scale(q, s0 + h)
        lp, _ = g.forward(target)
        g.set_scale(q, s0 - h)
        lm, _ = g.forward(target)
        g.set_scale(q, s0)
        fd = (lp - lm) / (2 * h)
        worst = max(worst, abs(fd - gs[q]) / max(abs(gs[q]), 1e-300))
    rng = np.random.default_rng(seed)
    for q in range(len(gw)):
        idx = list(np.argsort(-np.abs(gw[q]))[:n_weights]) + list(rng.choice(len(gw[q]), n_weights, replace=False))
        floor = 1e-3 * np.abs(gw[q]).max()
        for k in idx:
            w0 = g.weight(q, k)
            h = weight_step * max(abs(w0), 1e-3)
            g.set_weight(q, k, w0 + h)
            lp, _ = g.forward(target)
            g.set_weight(q, k, w0 - h)
            lm, _ = g.forward(target)
            g.set_weight(q, k, w0)
            fd = (lp - lm) / (2 * h)
            worst = max(worst, abs(fd - gw[q][k]) / max(abs(gw[q][k]), floor, 1e-300))
    return worst, gs


def test_adjoint_matches_central_differences_smooth_network():
    # no spikes anywhere: clamped pre cells near the release threshold drive
    # passive middle and output cells; releases of the passive cells are
    # centred at rest (v_thr = -62 mV) so every parameter matters
    pops = [I.hh_pop(20, v0_range=(-26.0, -14.0)), _passive(30), _passive(10)]
    pops[0]["hh"]["C"] = 1e300
    for d in pops[1:]:
        d["v0_range"] = (-64.0, -60.0)
    projs = [_graded_proj(0, 1, 0.0, p=0.5), _graded_proj(1, 1, 0.0, p=0.3), _graded_proj(1, 2, 0.0, p=0.5)]
    for d, wmax in zip(projs, (5.0, 1.0, 5.0)):
        d["weight"] = ("uniform", 0.0, wmax)
    projs[1]["v_thr"] = projs[2]["v_thr"] = -62.0
    spec = I.net(pops, projs, dt=0.05, steps=1)
    g = GradedOracle(spec)
    target = I.target_trace(spec, 600, g.n_out).astype(np.float64)
    worst, gs = _fd_check(g, target, scale_step=1e-3, weight_step=1e-3)
    assert np.all(np.abs(gs) > 1e-3)
    assert worst < 1e-5


def test_adjoint_matches_central_differences_200_neuron_copy():
    # the 200-neuron copy of the differentiable workload, 2000 steps of 0.05 ms;
    # spikes make the loss sharply curved, so central differences need small
    # steps and then carry rounding noise: agreement to 5e-4 relative
    spec = I.config_graded_small(steps=2000)
    g = GradedOracle(spec)
    target = I.target_trace(spec, 2000, g.n_out).astype(np.float64)
    worst, gs = _fd_check(g, target)
    assert np.all(np.abs(gs) > 1e-3)
    assert worst < 5e-4


def test_finite_difference_error_shrinks_with_the_step():
    # spike-timing curvature makes h = 1e-6 too coarse on the 2000-step loss;
    # the central-difference error falls as the step shrinks
    spec = I.config_graded_small(steps=2000)
    g = GradedOracle(spec)
    target = I.target_trace(spec, 2000, g.n_out).astype(np.float64)
    g.forward(target)
    gs, _ = g.backward()
    s0 = g.scale(0)
    errs = []
    for rel in (1e-5, 1e-6, 1e-7, 1e-8):
        h = rel * abs(s0)
        g.set_scale(0, s0 + h)
        lp, _ = g.forward(target)
        g.set_scale(0, s0 - h)
        lm, _ = g.forward(target)
        g.set_scale(0, s0)
        errs.append(abs((lp - lm) / (2 * h) - gs[0]) / abs(gs[0]))
    assert errs[0] > errs[1] > errs[2] and errs[3] < 1e-4


def test_dense_storage_adjoint_matches_central_differences():
    # the smooth network with dense (Eq. 2) storage of all three projections:
    # every (pre, post) pair is a parameter, gradients in row-major order
    pops = [I.hh_pop(12, v0_range=(-26.0, -14.0)), _passive(18), _passive(6)]
    pops[0]["hh"]["C"] = 1e300
    for d in pops[1:]:
        d["v0_range"] = (-64.0, -60.0)
    projs = [_graded_proj(0, 1, 0.0), _graded_proj(1, 1, 0.0), _graded_proj(1, 2, 0.0)]
    for d, wmax in zip(projs, (5.0, 1.0, 5.0)):
        d["layout"] = "dense"
        d["weight"] = ("uniform", 0.0, wmax)
    projs[1]["v_thr"] = projs[2]["v_thr"] = -62.0
    spec = I.net(pops, projs, dt=0.05, steps=1)
    g = GradedOracle(spec)
    assert g.nnz == [12 * 18, 18 * 18, 18 * 6]
    target = I.target_trace(spec, 400, g.n_out).astype(np.float64)
    worst, gs = _fd_check(g, target, scale_step=1e-3, weight_step=1e-3)
    assert np.all(np.abs(gs) > 1e-3)
    assert worst < 1e-5


def test_dense_storage_equals_compressed_rows_of_the_same_matrix():
    # a thinned dense projection (p < 1) is the compressed-row projection with
    # zeros filled in: same loss, and the dense gradient restricted to the
    # stored synapses is the compressed-row gradient
    spec_c = I.config_graded_small(steps=300)
    spec_d = I.config_graded_small(steps=300)
    spec_d["projs"][2]["layout"] = "dense"
    gc, gd = GradedOracle(spec_c), GradedOracle(spec_d)
    target = I.target_trace(spec_c, 300, gc.n_out).astype(np.float64)
    lc, _ = gc.forward(target)
    ld, _ = gd.forward(target)
    assert ld == pytest.approx(lc, rel=1e-12)
    gsc, gwc = gc.backward()
    gsd, gwd = gd.backward()
    assert np.allclose(gsd, gsc, rtol=1e-10, atol=0)
    rp, col, _ = gc.rows[2]
    n_post = spec_c["pops"][2]["n"]
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    assert np.allclose(gwd[2][rows * n_post + col], gwc[2], rtol=1e-10, atol=1e-300)


def _cubic(y, target):
    """A loss other than the squared error: mean |y - target|^3, and its dL/dy."""
    d = y - target
    n = d.size
    return float(np.sum(np.abs(d) ** 3) / n), 3.0 * np.abs(d) * d / n


def _fd_check_loss(g, target, loss_fn, scale_step, weight_step, n_weights=3, seed=0):
    """Like _fd_check, for the loss loss_fn(y, target) of the forward pass's
    filter values y, with the adjoint seeded by its dL/dy."""
    _, y = g.forward(target)
    _, dl = loss_fn(y, target)
    gs, gw = g.backward(dL_dy=dl)

    def L():
        return loss_fn(g.forward(target)[1], target)[0]

    worst = 0.0
    for q in range(len(gs)):
        s0 = g.scale(q)
        h = scale_step * abs(s0)
        g.set_scale(q, s0 + h)
        lp = L()
        g.set_scale(q, s0 - h)
        lm = L()
        g.set_scale(q, s0)
        worst = max(worst, abs((lp - lm) / (2 * h) - gs[q]) / max(abs(gs[q]), 1e-300))
    rng = np.random.default_rng(seed)
    for q in range(len(gw)):
        idx = list(np.argsort(-np.abs(gw[q]))[:n_weights]) + list(rng.choice(len(gw[q]), n_weights, replace=False))
        floor = 1e-3 * np.abs(gw[q]).max()
        for k in idx:
            w0 = g.weight(q, k)
            h = weight_step * max(abs(w0), 1e-3)
            g.set_weight(q, k, w0 + h)
            lp = L()
            g.set_weight(q, k, w0 - h)
            lm = L()
            g.set_weight(q, k, w0)
            worst = max(worst, abs((lp - lm) / (2 * h) - gw[q][k]) / max(abs(gw[q][k]), floor, 1e-300))
    return worst, gs


def test_adjoint_seeded_by_dl_dy_equals_the_squared_error_adjoint():
    # dL/dy = 2 (y - target) / (T n_out) is the squared-error loss's own seed
    spec = I.config_graded_small(steps=400)
    g = GradedOracle(spec)
    target = I.target_trace(spec, 400, g.n_out).astype(np.float64)
    _, y = g.forward(target)
    gs0, gw0 = g.backward()
    gs1, gw1 = g.backward(dL_dy=2.0 * (y - target) / y.size)
    assert np.allclose(gs1, gs0, rtol=1e-12, atol=0)
    for a, b in zip(gw1, gw0):
        assert np.allclose(a, b, rtol=1e-11, atol=1e-14 * np.abs(b).max())


def test_adjoint_of_another_loss_matches_central_differences():
    # a loss of y other than the squared error (mean |y - target|^3): the
    # adjoint seeded by its dL/dy against central differences of that loss,
    # on the smooth network (no spikes) and on the 200-neuron copy
    pops = [I.hh_pop(20, v0_range=(-26.0, -14.0)), _passive(30), _passive(10)]
    pops[0]["hh"]["C"] = 1e300
    for d in pops[1:]:
        d["v0_range"] = (-64.0, -60.0)
    projs = [_graded_proj(0, 1, 0.0, p=0.5), _graded_proj(1, 1, 0.0, p=0.3), _graded_proj(1, 2, 0.0, p=0.5)]
    for d, wmax in zip(projs, (5.0, 1.0, 5.0)):
        d["weight"] = ("uniform", 0.0, wmax)
    projs[1]["v_thr"] = projs[2]["v_thr"] = -62.0
    spec = I.net(pops, projs, dt=0.05, steps=1)
    g = GradedOracle(spec)
    target = I.target_trace(spec, 600, g.n_out).astype(np.float64)
    worst, gs = _fd_check_loss(g, target, _cubic, scale_step=1e-3, weight_step=1e-3)
    assert np.all(np.abs(gs) > 1e-4)
    assert worst < 1e-5
    spec = I.config_graded_small(steps=2000)
    g = GradedOracle(spec)
    target = I.target_trace(spec, 2000, g.n_out).astype(np.float64)
    worst, gs = _fd_check_loss(g, target, _cubic, scale_step=1e-8, weight_step=1e-7)
    assert worst < 5e-4
