"""The rounding-spread helper used as a parity bound (CPU, oracle only)."""
import numpy as np

import snn_inputs as I
from _spread import perturbed_spread

SADDLE_MV = -57.5253


def _input_only(steps):
    spec = I.config_four_pop(steps=steps)
    spec["pops"], spec["projs"] = [spec["pops"][0]], []
    return spec


def test_no_perturbation_gives_no_spread():
    v, spread = perturbed_spread(_input_only(50), 0, 50, runs=2, eps=0.0)
    assert v.shape == (50, 100)
    assert np.all(spread == 0.0)


def test_spread_is_small_below_the_saddle_and_grows_past_it():
    v, spread = perturbed_spread(_input_only(200), 0, 200, runs=8)
    below = v.max(axis=0) < SADDLE_MV - 1.0
    crossed = v.max(axis=0) > -30.0
    assert below.sum() > 10 and crossed.sum() > 10
    # a resting neuron forgets perturbations (the rest state is stable)
    assert spread[below].max() < 1e-2
    # an upstroke amplifies them by orders of magnitude
    assert np.median(spread[crossed]) > 100 * np.median(spread[below])


def test_spread_scales_with_the_perturbation():
    _, s1 = perturbed_spread(_input_only(100), 0, 100, runs=6, eps=2.0 ** -24)
    _, s2 = perturbed_spread(_input_only(100), 0, 100, runs=6, eps=2.0 ** -20)
    assert np.median(s2) > 4 * np.median(s1)
