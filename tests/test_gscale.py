"""The paper's gScale selection and fit (Sec. 5.1, Fig. 1): host-side logic on
known data (no GPU), and the batched sweep on the GPU against stand-alone runs
and the oracle."""
import math

import numpy as np
import pytest

import snn_inputs as I


def _gs():
    import importlib.util
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1412_0595_gb300",
                        "gscale.py")
    spec = importlib.util.spec_from_file_location("_gscale_logic", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_fit_recovers_the_table_constants():
    G = _gs()
    x = np.arange(100, 1001, 50, dtype=np.float64)             # nConn 100..1000 step 50 (Sec. 5.1)
    for k in [(1.318e3, 1.099e2, -2.800e-1), (1.118e-1, 9.810, 4.972e-5), (1.354e3, -6.338, 1.672e-3)]:
        y = G.law(x, *k)
        p, mape = G.fit(x, y)
        assert np.allclose(p, k, rtol=1e-6, atol=1e-9)
        assert mape < 1e-6


def test_selection_follows_fig1():
    G = _gs()
    recs = []
    for nc in (100.0, 200.0, 400.0):
        for gs in (0.5, 1.0, 2.0, 4.0):
            recs.append({"n_conn": nc, "gscale": gs, "avg_spike": nc * gs / 100.0, "sum_nans": 0})
    recs.append({"n_conn": 100.0, "gscale": 8.0, "avg_spike": 2.0, "sum_nans": 5})    # NaN run: rejected
    x, y, target = G.select(recs, 200.0, 1.0)                   # reference avgSpike = 2
    assert target == 2.0
    assert list(x) == [100.0, 200.0, 400.0] and list(y) == [2.0, 1.0, 0.5]


def test_sweep_specs_shape():
    G = _gs()
    specs, keys = G.sweep_specs([100, 500], [0.5, 1.0, 2.0], n_src=200, n_hh=50, steps=10)
    assert len(specs) == 6 and keys[0] == (100.0, 0.5)
    assert specs[1]["projs"][0]["p"] == pytest.approx(0.5) and specs[1]["instance"] == 1
    assert specs[4]["projs"][0]["user_scale"] == 1.0


@pytest.mark.gpu
def test_batched_sweep_matches_standalone_runs_and_oracle(gpu):
    import oracle
    from paper_1412_0595_gb300 import gscale as G
    specs, keys = G.sweep_specs([100, 300], [0.5, 2.0], n_src=300, n_hh=200, weight_max=1.0, steps=800)
    recs = G.run_sweep(specs, keys)
    for r, sp in zip(recs, specs):
        solo = gpu.Network.from_spec(sp)
        solo.step(sp["steps"])
        assert solo.counters(1)[0] / 200 == pytest.approx(r["avg_spike"], abs=0.02 * r["avg_spike"] + 1 / 200)
        ref = oracle.from_spec(sp)
        ref.step(sp["steps"])
        assert ref.counters(1)[0] / 200 == pytest.approx(r["avg_spike"], abs=0.02 * r["avg_spike"] + 1 / 200)
        assert r["sum_nans"] == 0
    # more conductance, more spikes
    a = {k: r["avg_spike"] for k, r in zip(keys, recs)}
    assert a[(100.0, 2.0)] >= a[(100.0, 0.5)] and a[(300.0, 2.0)] >= a[(300.0, 0.5)]


def test_izhikevich_sweep_specs_shape():
    G = _gs()
    specs, keys = G.izhikevich_sweep_specs([100, 1000], [0.5, 1.0], steps=10, n=200)
    assert len(specs) == 4 and keys[3] == (1000.0, 1.0)
    assert [p["kind"] for p in specs[0]["pops"]] == ["izh", "izh"]
    assert [p["n"] for p in specs[0]["pops"]] == [160, 40]
    assert specs[0]["projs"][0]["p"] == pytest.approx(0.5) and specs[0]["projs"][0]["layout"] == "dense"
    assert specs[3]["projs"][2]["user_scale"] == 1.0 and specs[3]["instance"] == 3


@pytest.mark.gpu
def test_izhikevich_sweep_matches_oracle(gpu):
    # batched Izhikevich runs: avgSpike over the whole network within the
    # rounding sensitivity of the network (2 % of the count plus one spike)
    import oracle
    from paper_1412_0595_gb300 import gscale as G
    specs, keys = G.izhikevich_sweep_specs([100, 400], [0.5, 2.0], steps=600, n=300)
    recs = G.run_sweep(specs, keys)
    for r, sp in zip(recs, specs):
        ref = oracle.from_spec(sp)
        ref.step(sp["steps"])
        count = sum(ref.counters(p)[0] for p in (0, 1))
        assert count / 300 == pytest.approx(r["avg_spike"], abs=0.03 * r["avg_spike"] + 1 / 300), (r, count)
        assert r["sum_nans"] == 0
    a = {k: r["avg_spike"] for k, r in zip(keys, recs)}
    assert a[(100.0, 2.0)] >= a[(100.0, 0.5)] and a[(400.0, 2.0)] >= a[(400.0, 0.5)]
