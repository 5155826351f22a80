"""The persistent engine (one cooperative launch for many steps, one grid
barrier per step) against the oracle and against the plain two-kernel engine."""
import numpy as np
import pytest

import oracle
import snn_inputs as I

pytestmark = pytest.mark.gpu


def _rel_ok(got, want, rel=1e-5):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    floor = 1e-5 * np.abs(want).max() if want.size else 0.0
    return np.all(np.abs(got - want) <= rel * np.maximum(np.abs(want), floor) + 1e-30)


def test_engine_choice(gpu):
    net = gpu.Network.from_spec(I.config_four_pop(steps=1))
    assert net.engine == "cluster"                 # 10,220 neurons fit one 16-CTA cluster
    net.set_option("engine", 1)
    assert net.engine == "persistent"
    net.set_option("engine", 0)
    assert net.engine == "plain"
    big = gpu.Network.from_spec(I.config_small(steps=1, n_hh=200_000))
    assert big.engine == "persistent"              # too big for a cluster, one resident CTA per tile
    assert big.cluster_size == 0


def test_options_read_back(gpu):
    net = gpu.Network.from_spec(I.config_four_pop(steps=1))
    # 43 tiles of 256 neurons (344 warps) over 16 CTAs: 22 warps (704 neurons) per CTA
    assert net.cluster_size == 16
    for name, value in (("persist_steps", 250), ("chunk", 512), ("graph_steps", 7), ("engine", 1), ("tiled", 0)):
        net.set_option(name, value)
        assert net.get_option(name) == value
    with pytest.raises(Exception):
        net.set_option("cluster_ctas", 8)          # read only


@pytest.mark.parametrize("engine", [1, 3])
def test_persistent_engine_matches_oracle_step_by_step(gpu, engine):
    pops = [I.source_pop(257, 500.0), I.hh_pop(1), I.hh_pop(255), I.hh_pop(513)]
    projs = [I.proj(0, 1, "csr", 0.5, ("uniform", 0, 3.0)), I.proj(0, 2, "dense", 1.0, ("uniform", 0, 0.3)),
             I.proj(0, 3, "csr", 0.1, ("uniform", 0, 3.0), channel=1)]
    spec = I.net(pops, projs, dt=0.1, steps=1)
    net = gpu.Network.from_spec(spec)
    net.set_option("engine", engine)
    net.set_option("record_isyn", 1)
    ref = oracle.from_spec(spec)
    for t in range(60):
        net.step()
        ref.step()
        assert np.array_equal(net.read_host(0, "spikes"), ref.spikes(0)), t
        for p in (1, 2, 3):
            assert np.abs(net.read_host(p, "V") - ref.get(p, "V")).max() <= 1e-3, (t, p)
            assert _rel_ok(net.read_host(p, "isyn"), ref.get(p, "isyn")), (t, p)
            assert _rel_ok(net.read_host(p, "g0"), ref.get(p, "g0")), (t, p)
            assert _rel_ok(net.read_host(p, "g1"), ref.get(p, "g1")), (t, p)
    for p in range(4):
        assert net.counters(p) == ref.counters(p)


@pytest.mark.parametrize("engine", [1, 3])
def test_persistent_engine_long_launch_matches_oracle(gpu, engine):
    # forced activity: the HH population spikes, rows are pushed by their owners
    spec = I.config_small(steps=3000, n_hh=400, n_src=100, p=0.2, weight_hi=60.0)
    net = gpu.Network.from_spec(spec)
    net.set_option("engine", engine)
    net.set_option("persist_steps", 700)        # several launches, ragged last one
    ref = oracle.from_spec(spec)
    net.step(spec["steps"])
    ref.step(spec["steps"])
    cg, co = net.counters(1)[0], ref.counters(1)[0]
    assert co > 200 and abs(cg - co) <= 0.02 * co + 1
    assert net.counters(0) == ref.counters(0)
    assert net.t == spec["steps"]
    assert net.synaptic_events() == ref.events or abs(net.synaptic_events() - ref.events) <= 0.02 * ref.events


def test_engines_alternate_on_one_trajectory(gpu):
    spec = I.config_four_pop(steps=300, n_mid=3000)
    a = gpu.Network.from_spec(spec)
    b = gpu.Network.from_spec(spec)
    a.set_option("engine", 0)
    a.step(300)
    for eng in (1, 0, 3):
        b.set_option("engine", eng)
        b.step(100)
    for p in range(4):
        assert np.abs(a.read_host(p, "V") - b.read_host(p, "V")).max() < 1e-4
        assert np.abs(a.read_host(p, "g0") - b.read_host(p, "g0")).max() <= 1e-6 * (1 + np.abs(a.read_host(p, "g0")).max())
        assert a.counters(p) == b.counters(p)
    assert a.t == b.t == 300
    assert np.array_equal(a.read_host(0, "spikes"), b.read_host(0, "spikes"))


def test_persistent_engine_with_more_tiles_than_resident_ctas(gpu):
    # 400,000 HH neurons = 1563 tiles: CTAs loop over tiles, state goes through HBM
    spec = I.config_small(steps=40, n_hh=400_000, n_src=100, p=0.001)
    net = gpu.Network.from_spec(spec)
    net.set_option("engine", 1)
    ref = oracle.from_spec(spec)
    net.step(40)
    ref.step(40)
    assert np.abs(net.read_host(1, "V") - ref.get(1, "V")).max() <= 1e-3
    assert _rel_ok(net.read_host(1, "g0"), ref.get(1, "g0"))
    assert net.counters(0) == ref.counters(0)


@pytest.mark.parametrize("n_pre,n_post,p,ks", [
    (64, 20001, 0.4, (1, 5, 64)),
    (64, 8192, 0.4, (1, 5, 64)),
    (64, 3, 0.4, (1, 5, 64)),
    (64, 20001, 0.9, (1, 64)),            # segments of ~3,700 synapses per row and tile
    (40000, 20001, 0.01, (40000,)),       # ~1,300 pieces per CTA: several descriptor batches
    (300, 70001, 0.05, (1, 33, 65, 300)), # segment form: row groups of up to 64 rows, ragged last span
    (200, 50001, 0.0005, (1, 7, 200)),    # most row segments of a tile empty, odd last tile width
])
@pytest.mark.parametrize("mode", [1, 3])              # bulk-copy pieces, warp-streamed segments
def test_post_tiled_propagation_matches_oracle(gpu, n_pre, n_post, p, ks, mode):
    spec = I.net([I.source_pop(n_pre, 0.0), I.hh_pop(n_post)],
                 [I.proj(0, 1, "csr", p, ("uniform", 0.0, 1.0))], dt=0.1, steps=1)
    net = gpu.Network.from_spec(spec)
    net.set_option("engine", 0)
    net.set_option("tiled", mode)
    assert net.proj_mode(0) == {1: 1, 3: 2}[mode]
    ref = oracle.from_spec(spec)
    rng = np.random.default_rng(2)
    for k in ks:
        spk = np.sort(rng.choice(n_pre, k, replace=False)).astype(np.int32)
        net.debug_propagate(0, spk)
        ref.deliver(0, spk)
        assert _rel_ok(net.read_host(1, "g0"), ref.get(1, "g0"))


@pytest.mark.parametrize("mode", [1, 3])
def test_post_tiled_steps_match_row_kernel(gpu, mode):
    # rows of ~6,000 synapses over 30,000 posts; sources fire often, the HH
    # population stays subthreshold so V compares tightly
    spec = I.net([I.source_pop(100, 2000.0), I.hh_pop(30000, v0_range=(-64.0, -62.0))],
                 [I.proj(0, 1, "csr", 0.2, ("uniform", 0.0, 0.5))], dt=0.1, steps=1)
    a = gpu.Network.from_spec(spec)
    b = gpu.Network.from_spec(spec)
    for net, tiled in ((a, 0), (b, mode)):
        net.set_option("engine", 0)
        net.set_option("tiled", tiled)
        net.step(150)
    assert np.abs(a.read_host(1, "g0") - b.read_host(1, "g0")).max() <= 1e-5 * (1 + np.abs(a.read_host(1, "g0")).max())
    assert np.abs(a.read_host(1, "V") - b.read_host(1, "V")).max() < 1e-4
    ref = oracle.from_spec(spec)
    ref.step(150)
    assert np.abs(b.read_host(1, "V") - ref.get(1, "V")).max() <= 1e-3
    assert a.synaptic_events() == b.synaptic_events() == ref.events


def test_barrier_wait_times_out_and_reset_recovers(gpu):
    # the barrier waits for one arrival nobody makes: every CTA gives up after
    # the spin limit, the host reads SNN_ERR_TIMEOUT, nothing hangs
    import paper_1412_0595_gb300 as snn
    spec = I.config_small(steps=50, n_hh=600)
    net = gpu.Network.from_spec(spec)
    net.set_option("engine", 1)
    net.set_option("spin_limit", 2000)
    net.set_option("test_barrier_extra", 1)
    net.step(20)
    with pytest.raises(snn.SNNError) as e:
        net.sync()
    assert e.value.name == "SNN_ERR_TIMEOUT"
    net.set_option("test_barrier_extra", 0)
    net.set_option("spin_limit", 1 << 22)
    net.reset()
    net.step(50)
    net.sync()
    ref = gpu.Network.from_spec(spec)
    ref.set_option("engine", 1)
    ref.step(50)
    assert np.abs(net.read_host(1, "V") - ref.read_host(1, "V")).max() < 1e-5
    assert net.counters(0) == ref.counters(0)


def test_cluster_engine_spiking_four_population_network(gpu):
    # the cluster engine on the four-population shape with forced activity in
    # every population (dense and compressed rows, both channels)
    spec = I.config_four_pop(steps=600, n_mid=3000, weight=("lognormal", 5.0, 0.5))
    a = gpu.Network.from_spec(spec)
    b = gpu.Network.from_spec(spec)
    a.set_option("engine", 3)
    b.set_option("engine", 0)
    a.step(600)
    b.step(600)
    ref = oracle.from_spec(spec)
    ref.step(600)
    for p in range(4):
        ca, cb, co = a.counters(p)[0], b.counters(p)[0], ref.counters(p)[0]
        assert abs(ca - co) <= 0.02 * co + 1 and abs(cb - co) <= 0.02 * co + 1, (p, ca, cb, co)
    assert a.counters(1)[0] > 1000 and a.counters(2)[0] > 100 and a.counters(3)[0] > 10


@pytest.mark.parametrize("n_hh", [1000, 30_500, 60_000])
def test_cluster_engine_over_the_shared_memory_range(gpu, n_hh):
    # slices from 96 to 3776 neurons per CTA: dynamic shared memory from 2 KB to
    # past 48 KB, and sizes whose dynamic part stays below 48 KB while static
    # plus dynamic exceed it (the launch must opt in either way); the cluster
    # engine's spike counts follow the plain engine's
    spec = I.config_small(steps=200, n_hh=n_hh, n_src=100, p=0.1, weight_hi=60.0)
    a = gpu.Network.from_spec(spec)
    b = gpu.Network.from_spec(spec)
    assert a.cluster_size == 16
    a.set_option("engine", 3)
    b.set_option("engine", 0)
    a.step(200)
    b.step(200)
    assert a.counters(0) == b.counters(0)                 # sources: identical draws
    ca, cb = a.counters(1), b.counters(1)
    assert cb[0] > 0 and abs(ca[0] - cb[0]) <= 0.02 * cb[0] + 1   # delivery order differs (FP atomics)
    assert ca[1] == cb[1] == 0
