"""The paper's conductance-scale procedure (Sec. 5.1) on the batched GPU form,
for the HH network and for the Izhikevich cortical network (Table 1, Fig. 2).

1. Sweep: one network instance per (nConn, gScale) pair, all run in one
   batched network object (every simulation step runs in the CUDA library).
2. Select: for every nConn, among the runs without NaN states (sumNANs ==
   0, the reading taken of the paper's rejection rule), the gScale whose
   average spike count per neuron (avgSpike) is closest to that of the
   reference run (ref_nConn, ref_gScale).
3. Fit gScale = k1 / (k2 + nConn) + k3 by non-linear least squares (the
   rewritten form (gScale - k3)(nConn + k2) = k1 of Sec. 5.1) and report the
   mean absolute percentage error of the fit, as the paper does.

The fit and the selection are host-side analysis (the paper ran them in
Matlab); they read only the per-run counters the GPU produced.
"""
from __future__ import annotations

import math

import numpy as np


def sweep_specs(n_conn_values, gscale_values, n_src=1000, n_hh=1000, rate_hz=20.0, weight_max=0.25, steps=5000,
                seed=None):
    """Instances of the sweep: n_src Poisson sources at rate_hz -> n_hh HH
    neurons, each post neuron drawing nConn inputs on average (p = nConn /
    n_src), weights U(0, weight_max) nS, conductance scale = gScale exactly
    (k1 = 0, k3 = 1 in the law, times the user factor gScale)."""
    import snn_inputs as I
    seed = I.SEED if seed is None else seed
    specs, keys = [], []
    b = 0
    for nc in n_conn_values:
        for gs in gscale_values:
            sp = I.net([I.source_pop(n_src, rate_hz), I.hh_pop(n_hh)],
                       [I.proj(0, 1, "csr", nc / n_src, ("uniform", 0.0, weight_max), k=(0.0, 0.0, 1.0),
                               user_scale=float(gs))],
                       dt=0.1, steps=steps, seed=seed, instance=b, name=f"gscale_{nc}_{gs:.4g}")
            specs.append(sp)
            keys.append((float(nc), float(gs)))
            b += 1
    return specs, keys


def izhikevich_sweep_specs(n_conn_values, gscale_values, steps=1000, n=1000, seed=None):
    """Instances of the sweep on the paper's cortical network (Sec. 5.1,
    Table 1 / Fig. 2): n Izhikevich neurons, 4 : 1 excitatory : inhibitory,
    nConn inputs per neuron, all weights times gScale."""
    import snn_inputs as I
    seed = I.SEED if seed is None else seed
    specs, keys = [], []
    b = 0
    for nc in n_conn_values:
        for gs in gscale_values:
            specs.append(I.config_izhikevich(n_conn=nc, gscale=float(gs), steps=steps, n=n, seed=seed, instance=b))
            keys.append((float(nc), float(gs)))
            b += 1
    return specs, keys


def run_sweep(specs, keys, device=None, engine=None):
    """Runs every instance in one batched network; returns one record per run
    with avgSpike (spikes per neuron of the instance's spiking model
    populations, sources excluded, over the run) and sumNANs (NaN
    neuron-steps of those populations)."""
    from .network import Network
    net = Network.from_specs(specs, device=device)
    if engine is not None:
        net.set_option("engine", {"plain": 0, "persistent": 1}[engine])
    steps = specs[0]["steps"]
    net.step(steps)
    out = []
    for b, ((nc, gs), sp) in enumerate(zip(keys, specs)):
        o = net.pop_offsets[b]
        count = nans = n = 0
        for k, pop in enumerate(sp["pops"]):
            if pop["kind"] == "source":
                continue
            c, z = net.counters(o + k)
            count, nans, n = count + c, nans + z, n + pop["n"]
        out.append({"n_conn": nc, "gscale": gs, "avg_spike": count / n, "sum_nans": nans})
    net.close()
    return out


def select(records, ref_n_conn, ref_gscale):
    """The conductance scale that keeps a network's activity at the
    reference's (Sec. 5.1): for each nConn, the gScale whose avgSpike lies
    closest to the reference run's avgSpike, counting only runs that ended
    without NaN states.  All runs are ranked at once by (nConn, distance to
    the reference rate, gScale); the first NaN-free run of each nConn wins."""
    n_conn = np.array([r["n_conn"] for r in records], np.float64)
    gs = np.array([r["gscale"] for r in records], np.float64)
    avg = np.array([r["avg_spike"] for r in records], np.float64)
    clean = np.array([r["sum_nans"] == 0 for r in records])
    is_ref = (n_conn == ref_n_conn) & (gs == ref_gscale)
    if not is_ref.any():
        raise ValueError("reference run not in the sweep")
    target = float(avg[np.argmax(is_ref)])
    order = np.lexsort((gs[clean], np.abs(avg[clean] - target), n_conn[clean]))
    nc_sorted, gs_sorted = n_conn[clean][order], gs[clean][order]
    first = np.ones(len(order), bool)
    first[1:] = nc_sorted[1:] != nc_sorted[:-1]
    return nc_sorted[first], gs_sorted[first], target


def law(x, k1, k2, k3):
    return k1 / (k2 + x) + k3


def fit_linear(x, y):
    """The rewritten law (gScale - k3)(nConn + k2) = k1 is linear in
    (k1 + k2 k3, k2, k3) once expanded: y x = (k1 + k2 k3) - k2 y + k3 x.
    Ordinary least squares of y x on [1, y, x] gives the paper's "linear
    regression" estimate."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    A = np.stack([np.ones_like(x), y, x], axis=1)
    (a, b, c), *_ = np.linalg.lstsq(A, y * x, rcond=None)
    k2, k3 = -b, c
    return (a - k2 * k3, k2, k3)


def fit(x, y):
    """Non-linear least squares of y = k1 / (k2 + x) + k3 in relative
    residuals, started from the linear estimate; returns (k1, k2, k3) and the
    mean absolute percentage error of the fitted curve."""
    from scipy.optimize import curve_fit
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    p0 = fit_linear(x, y)
    lo = -float(x.min()) + 1e-9 * max(1.0, float(x.min()))   # keep k2 + nConn > 0 over the data
    p0 = (p0[0], max(p0[1], lo + 1e-6 * abs(lo) + 1e-12), p0[2])
    p, _ = curve_fit(law, x, y, p0=p0, sigma=np.abs(y) + 1e-300, bounds=([-np.inf, lo, -np.inf], [np.inf, np.inf, np.inf]),
                     maxfev=20000, xtol=1e-15, ftol=1e-15, gtol=1e-15)
    mape = float(np.mean(np.abs((law(x, *p) - y) / y)) * 100.0)
    return tuple(float(v) for v in p), mape


def log_grid(lo, hi, n):
    return list(np.exp(np.linspace(math.log(lo), math.log(hi), n)))
