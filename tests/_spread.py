"""The oracle's own spread under rounding-level perturbation (test helper).

A neuron whose potential passes the saddle of the resting state (about
-57.5 mV for the Traub-Miles cell) but does not reach threshold amplifies any
small change of its state for a while: an FP32 trajectory and the FP64 one
part there by more than 1e-3 mV although both are correct to their precision.
For such neurons the parity bound is the spread that the FP64 oracle itself
shows when its state is rounded at FP32 level: after every time step each of
V, m, h, n is multiplied by (1 + e) with e uniform in [-eps, eps].  With eps =
2^-22 the perturbation covers what one FP32 step adds (four substep roundings
of the stored state, 2^-24 each, and the relative error of about 2^-22 of the
hardware exponentials entering the rates).  The bound of neuron i is the
largest |V_perturbed - V_oracle| over `runs` seeded runs and the window.

Only the oracle runs here; the GPU path is never consulted.
"""
import numpy as np

import oracle

EPS_FP32_STEP = 2.0 ** -22


def perturbed_spread(spec, pop, steps, runs=60, eps=EPS_FP32_STEP, seed=0x5EED):
    """(V of the unperturbed oracle [steps, n], max deviation per neuron [n])
    for population `pop` of `spec`; the other populations run unperturbed."""
    base = oracle.from_spec(spec)
    v_base = []
    for _ in range(steps):
        base.step()
        v_base.append(base.get(pop, "V"))
    v_base = np.array(v_base)
    n = v_base.shape[1]
    worst = np.zeros(n)
    for r in range(runs):
        rng = np.random.default_rng([seed, r])
        ref = oracle.from_spec(spec)
        for t in range(steps):
            ref.step()
            if eps > 0:
                for f in ("V", "m", "h", "n"):
                    x = ref.get(pop, f)
                    ref.set(pop, f, x * (1.0 + rng.uniform(-eps, eps, n)))
            worst = np.maximum(worst, np.abs(ref.get(pop, "V") - v_base[t]))
    return v_base, worst
