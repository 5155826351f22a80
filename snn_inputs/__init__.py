"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds no arithmetic of the simulated method: it only states
network shapes and parameters and draws the seeded input arrays (initial
potentials, synaptic weights) with numpy.  Everything the method derives
from them -- connectivity from the seed, gScale, Poisson thresholds, decay
factors, initial gating -- each side computes itself.

Units throughout: mV, ms, nS, pF, pA, Hz.

Workload shapes follow the paper's populations (Sec. 5.1: a 1000-neuron
network with a density sweep; the insect-olfaction model with input,
Kenyon-cell-like, output and lateral-inhibition populations) at the sizes of
the five benchmark configurations listed in ``CONFIGS``.  The paper's own
simulation outputs are not available; these synthetic networks stand in for
them.
"""
from __future__ import annotations

import math

import numpy as np

SEED = 12345

# Traub-Miles HH cell of the insect-olfaction model family (C in pF, g in nS).
TRAUB = dict(C=143.0, gNa=7150.0, ENa=50.0, gK=1430.0, EK=-95.0, gL=26.72, EL=-63.563)

E_EXC = 0.0
E_INH = -92.0

# Purposes folded into numpy seed sequences.
_V0, _W, _TARGET, _BATCH = 1, 2, 3, 4

# Poisson current drive of input HH neurons: an event adds `amp` pA with
# probability rate*dt per step; the drive current decays with `tau` ms.
# Calibrated once on the FP64 oracle: 100 driven neurons fire at ~19.5 Hz
# over 1 s (amp 50 gives ~11 Hz, 80 gives ~30 Hz).
INPUT_DRIVE = dict(rate_hz=1000.0, amp=60.0, tau=1.0)


def hh_pop(n, *, v0_range=(-62.0, -58.0), drive=None, E_syn=(E_EXC, E_INH), tau_syn=(1.0, 1.0),
           v_thresh=0.0):
    return dict(kind="hh", n=int(n), hh=dict(TRAUB), v0_range=v0_range, drive=drive,
                E_syn=tuple(E_syn), tau_syn=tuple(tau_syn), v_thresh=v_thresh)


# Cortical neurons of the paper's first network (Sec. 5.1, ref. [9]): with one
# uniform r per neuron, excitatory a = 0.02, b = 0.2, c = -65 + 15 r^2,
# d = 8 - 6 r^2; inhibitory a = 0.02 + 0.08 r, b = 0.25 - 0.05 r, c = -65,
# d = 2; thalamic input noise of standard deviation 5 (excitatory) / 2
# (inhibitory) per 1 ms step; peak 30 mV.
IZH_EXC = dict(a0=0.02, a1=0.0, b0=0.2, b1=0.0, c0=-65.0, c2=15.0, d0=8.0, d2=-6.0, noise=5.0, bias=0.0)
IZH_INH = dict(a0=0.02, a1=0.08, b0=0.25, b1=-0.05, c0=-65.0, c2=0.0, d0=2.0, d2=0.0, noise=2.0, bias=0.0)


def izh_pop(n, *, excitatory=True, v0=-65.0, **overrides):
    """An Izhikevich population; synaptic input is a current pulse (the
    channels clear every step), v starts at v0 and u at b v."""
    izh = dict(IZH_EXC if excitatory else IZH_INH)
    izh.update(overrides)
    return dict(kind="izh", n=int(n), izh=izh, v0_range=(float(v0), float(v0)), E_syn=(0.0, 0.0),
                tau_syn=(0.0, 0.0), v_thresh=30.0)


def source_pop(n, rate_hz):
    return dict(kind="source", n=int(n), rate_hz=float(rate_hz))


def proj(pre, post, layout, p, weight, *, channel=0, k=(1.0, 0.0, 0.0), user_scale=1.0):
    """A projection.  ``weight`` = ('uniform', lo, hi) or ('lognormal', mu, sigma),
    in nS.  ``k`` = (k1, k2, k3) of the gScale law; nConn is p * N_pre."""
    return dict(pre=pre, post=post, layout=layout, p=float(p), weight=tuple(weight),
                channel=channel, k1=float(k[0]), k2=float(k[1]), k3=float(k[2]),
                user_scale=float(user_scale))


def net(pops, projs, *, dt, n_sub=4, steps, seed=SEED, instance=0, name=""):
    return dict(pops=pops, projs=projs, dt=float(dt), n_sub=int(n_sub), steps=int(steps),
                seed=int(seed), instance=int(instance), name=name)


# --------------------------------------------------------------------------
# The five workloads
# --------------------------------------------------------------------------
def config_small(steps=1000, n_hh=1000, n_src=100, p=0.1, user_scale=1.0, seed=SEED, instance=0,
                 weight_hi=0.05):
    """100 Poisson sources (20 Hz) -> 1,000 HH neurons, compressed rows p=0.1,
    weights U[0, 0.05] nS x 1/(p N_pre), tau = 1 ms, dt = 0.1 ms, 4 substeps."""
    return net([source_pop(n_src, 20.0), hh_pop(n_hh)],
               [proj(0, 1, "csr", p, ("uniform", 0.0, weight_hi), user_scale=user_scale)],
               dt=0.1, steps=steps, seed=seed, instance=instance,
               name=f"small_src{n_src}_hh{n_hh}_p{p}")


def config_four_pop(steps=10000, n_in=100, n_mid=10000, n_out=100, n_inh=20, p_mid=0.5,
                    mid_layout="csr", weight=("lognormal", -3.0, 0.5), seed=SEED):
    """Four-population feed-forward HH network: In (100, Poisson-current drive)
    -> Mid (10,000, rows p=0.5) -> Out (100, dense); Inh (20) dense from In,
    inhibitory (-92 mV) onto Out.  Weights lognormal(-3, 0.5) nS x 1/(p N_pre)."""
    pops = [hh_pop(n_in, drive=dict(INPUT_DRIVE)), hh_pop(n_mid), hh_pop(n_out), hh_pop(n_inh)]
    projs = [proj(0, 1, mid_layout, p_mid, weight),
             proj(1, 2, "dense", 1.0, weight),
             proj(0, 3, "dense", 1.0, weight),
             proj(3, 2, "dense", 1.0, weight, channel=1)]
    return net(pops, projs, dt=0.1, steps=steps, seed=seed,
               name=f"four_pop_in{n_in}_mid{n_mid}_out{n_out}_inh{n_inh}_p{p_mid}_{mid_layout}")


def config_izhikevich(n_conn=1000, gscale=1.0, steps=1000, n=1000, layout=None, seed=SEED, instance=0):
    """The paper's first network (Sec. 5.1): n cortical neurons, excitatory to
    inhibitory 4 : 1, every neuron receiving nConn inputs on average (one
    Bernoulli(nConn / n) draw per ordered pair, self-pairs included), weights
    U(0, 0.5) from excitatory and U(-1, 0) from inhibitory neurons (the
    synaptic input is a current), all scaled by gScale; dt = 1 ms, v in two
    substeps of 0.5 ms, 1000 steps = 1 s."""
    ne = n * 4 // 5
    ni = n - ne
    p = min(1.0, n_conn / n)
    layout = layout or ("dense" if p >= 0.5 else "csr")
    pops = [izh_pop(ne, excitatory=True), izh_pop(ni, excitatory=False)]
    k = (0.0, 0.0, 1.0)
    w_e, w_i = ("uniform", 0.0, 0.5), ("uniform", -1.0, 0.0)
    projs = [proj(0, 0, layout, p, w_e, k=k, user_scale=gscale), proj(0, 1, layout, p, w_e, k=k, user_scale=gscale),
             proj(1, 0, layout, p, w_i, k=k, user_scale=gscale), proj(1, 1, layout, p, w_i, k=k, user_scale=gscale)]
    return net(pops, projs, dt=1.0, n_sub=2, steps=steps, seed=seed, instance=instance,
               name=f"izhikevich_n{n}_nconn{n_conn}_gscale{gscale:.4g}")


SWEEP_N_MID = (1_000, 10_000, 100_000, 1_000_000)
SWEEP_P = (0.01, 0.05, 0.2, 0.5)


def config_sweep(n_mid, p, layout="csr", steps=1000):
    """Scaling sweep point: the four-population shape without Inh, middle
    population n_mid at density p."""
    pops = [hh_pop(100, drive=dict(INPUT_DRIVE)), hh_pop(n_mid), hh_pop(100)]
    w = ("lognormal", -3.0, 0.5)
    projs = [proj(0, 1, layout, p, w), proj(1, 2, "dense", 1.0, w)]
    return net(pops, projs, dt=0.1, steps=steps, name=f"sweep_mid{n_mid}_p{p}_{layout}")


def config_batched(n_instances=512, steps=5000, seed=SEED, n_lo=1_000, n_hi=50_000,
                   c_lo=0.1, c_hi=10.0, weight_hi=0.05):
    """n_instances copies of the small workload with middle sizes and
    conductance factors drawn log-uniform (the paper's sweep over scaling
    factors, Sec. 2 / Fig. 1).  weight_hi is the upper end of the uniform
    weights (nS): 0.05 as in the small workload (subthreshold with the
    1/(p N_pre) scaling), or larger for a forced-activity variant."""
    rng = np.random.default_rng([seed, _BATCH])
    sizes = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), n_instances)).astype(np.int64)
    scales = np.exp(rng.uniform(math.log(c_lo), math.log(c_hi), n_instances))
    return [config_small(steps=steps, n_hh=int(sizes[b]), user_scale=float(scales[b]), seed=seed,
                         instance=b, weight_hi=weight_hi) for b in range(n_instances)]


# Graded-synapse (differentiable) workload
GRADED = dict(v_thr=-20.0, v_slope=2.0, tau_filter=5.0, target_jitter=0.1)


# Graded weights (nS, uniform [0, max]) per projection In -> Mid, recurrent,
# Mid -> Out; calibrated once on the FP64 oracle (200-neuron copy, 2000 steps)
# so that the middle and output populations respond to the input spikes
# (filtered output range about -63 to -58 mV) while central finite
# differences still agree with the adjoint.
GRADED_WEIGHTS = (60.0, 5.0, 60.0)


def config_graded(n_in=100, n_mid=20000, n_out=100, p=0.05, p_in=None, steps=2000, dt=0.05,
                  recurrent=True, weights=GRADED_WEIGHTS, seed=SEED):
    """Graded sigmoidal synapses, release 1/(1 + exp((V_thr - V_pre)/2 mV)),
    V_thr = -20 mV.  In (Poisson-current drive) -> Mid, Mid -> Mid, Mid -> Out,
    all compressed rows at density p, excitatory; weights uniform in nS."""
    pops = [hh_pop(n_in, drive=dict(INPUT_DRIVE)), hh_pop(n_mid), hh_pop(n_out)]
    w = [("uniform", 0.0, float(x)) for x in weights]
    projs = [proj(0, 1, "csr", p if p_in is None else p_in, w[0]),
             proj(1, 1, "csr", p, w[1]) if recurrent else proj(2, 2, "csr", p, w[1]),
             proj(1, 2, "csr", p, w[2])]
    for d in projs:
        d.update(synapse="graded", v_thr=GRADED["v_thr"], v_slope=GRADED["v_slope"])
    return net(pops, projs, dt=dt, steps=steps, seed=seed,
               name=f"graded_in{n_in}_mid{n_mid}_out{n_out}_p{p}")


def config_graded_small(steps=2000, recurrent=True, seed=SEED):
    """200-neuron copy used for finite-difference checks: In 20 / Mid 160 /
    Out 20, In -> Mid at p = 0.25 so no row is empty."""
    return config_graded(n_in=20, n_mid=160, n_out=20, p=0.05, p_in=0.25, steps=steps,
                         recurrent=recurrent, seed=seed)


def config_graded_dense(n_in=100, n_mid=4096, n_out=100, p_in=0.05, steps=2000, dt=0.05,
                        weights=GRADED_WEIGHTS, seed=SEED):
    """The graded workload with dense storage (Eq. 2) for the middle
    population's projections: In -> Mid compressed rows at p_in; Mid -> Mid
    and Mid -> Out dense (every pair a weight, p = 1, nConn = N_mid, so the
    mean drive per post matches the sparse form's)."""
    pops = [hh_pop(n_in, drive=dict(INPUT_DRIVE)), hh_pop(n_mid), hh_pop(n_out)]
    w = [("uniform", 0.0, float(x)) for x in weights]
    projs = [proj(0, 1, "csr", p_in, w[0]), proj(1, 1, "dense", 1.0, w[1]), proj(1, 2, "dense", 1.0, w[2])]
    for d in projs:
        d.update(synapse="graded", v_thr=GRADED["v_thr"], v_slope=GRADED["v_slope"])
    return net(pops, projs, dt=dt, steps=steps, seed=seed,
               name=f"graded_dense_in{n_in}_mid{n_mid}_out{n_out}")


def config_graded_dense_small(steps=2000, n_mid=160, seed=SEED):
    """200-neuron copy of the dense form: In 20 / Mid 160 / Out 20, In -> Mid
    at p = 0.25."""
    return config_graded_dense(n_in=20, n_mid=n_mid, n_out=20, p_in=0.25, steps=steps, seed=seed)


CONFIGS = {
    "small": config_small,
    "four_pop": config_four_pop,
    "sweep": config_sweep,
    "batched": config_batched,
    "graded": config_graded,
    "graded_dense": config_graded_dense,
}


# --------------------------------------------------------------------------
# Seeded arrays
# --------------------------------------------------------------------------
def v0(spec, pop):
    """Initial membrane potentials of population `pop`: uniform in its
    v0_range, drawn in FP64 and rounded to FP32 (both sides read these bits)."""
    d = spec["pops"][pop]
    if d["kind"] not in ("hh", "izh"):
        return None
    lo, hi = d["v0_range"]
    if lo == hi:
        return np.full(d["n"], lo, np.float32)
    rng = np.random.default_rng([spec["seed"], _V0, spec["instance"], pop])
    return rng.uniform(lo, hi, d["n"]).astype(np.float32)


def weights(spec, q, nnz):
    """`nnz` synaptic weights (nS) of projection q in storage order, FP64
    draws rounded to FP32."""
    kind, a, b = spec["projs"][q]["weight"]
    rng = np.random.default_rng([spec["seed"], _W, spec["instance"], q])
    if kind == "uniform":
        w = rng.uniform(a, b, nnz)
    elif kind == "lognormal":
        w = rng.lognormal(a, b, nnz)
    elif kind == "const":
        w = np.full(nnz, a)
    else:
        raise ValueError(kind)
    return w.astype(np.float32)


def target_trace(spec, n_steps, n_out):
    """Seeded target for the graded workload's output filter (mV), used only
    when a reachable target is not generated by a perturbed forward run."""
    rng = np.random.default_rng([spec["seed"], _TARGET])
    return (-60.0 + rng.standard_normal((n_steps, n_out))).astype(np.float32)


def rng_tag(instance, index):
    """Philox counter word 2 for population / projection `index` of `instance`."""
    return (int(instance) << 8) | int(index)


def n_pre_post(spec, q):
    d = spec["projs"][q]
    return spec["pops"][d["pre"]]["n"], spec["pops"][d["post"]]["n"]
