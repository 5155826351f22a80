"""Benchmark of the HH spiking-network time-step loop on one GB300 (or N replicas).

One bench step = one full simulation of the four-population feed-forward HH
network (In 100 with Poisson current drive -> Mid 10,000 over compressed rows
at p = 0.5 -> Out 100 dense; Inh 20 dense from In, inhibitory onto Out;
lognormal(-3, 0.5) nS weights scaled by gScale = 1/(p N_pre)) for 10,000 time
steps of 0.1 ms with 4 Euler substeps: every time step runs the neuron update
with spike compaction and the propagation of that step's spikes.

Metric: synaptic events/s (events = stored synapses of the spiking rows,
counted exactly from per-neuron spike counts), with HH neuron-steps/s beside
it.  Inputs are resident in HBM when the timed region starts; L2 is flushed
(256 MiB written, then another 256 MiB read) between timed steps.  `e2e`
repeats the measurement through the public API from pinned host buffers
(weights and initial potentials copied in, connectivity drawn on the device,
counters copied out).

--impl reference times the FP64 CPU oracle (the only reference this method
has) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import snn_inputs as I  # noqa: E402

# Algorithmic work per unit (see the roofline notes of the design document).
FLOPS_PER_SUBSTEP = 64          # rates 28, currents 16, gating 12, updates 8
FLOPS_PER_STEP_EXTRA = 9        # I_syn 5, decays 3, threshold test 1
BYTES_PER_EVENT = 8             # 4 B post index + 4 B weight streamed from HBM
BYTES_PER_ROW = 12              # 8 B row start + 4 B spike id per spiking row
L2_BYTES = 129e6                # GB300 L2
SM_COUNT = 152
FP32_LANES = 128


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sim-steps", type=int, default=10_000)
    ap.add_argument("--cpu-steps", type=int, default=4_000,
                    help="time steps of the bounded oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--steady-steps", type=int, default=2000,
                    help="time steps run before the per-kernel timing")
    ap.add_argument("--phase-reps", type=int, default=200,
                    help="back-to-back launches per kernel in the per-kernel timing")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-sequential comparison")
    ap.add_argument("--batch-instances", type=int, default=512)
    ap.add_argument("--batch-steps", type=int, default=5000)
    ap.add_argument("--no-graded", action="store_true", help="skip the differentiable-form measurement")
    ap.add_argument("--no-graded-dense", action="store_true",
                    help="skip the differentiable form with dense storage and the rank-K weight-gradient update")
    ap.add_argument("--no-gscale", action="store_true", help="skip the gScale sweep and fit")
    ap.add_argument("--no-dense-batch", action="store_true",
                    help="skip the tensor-core dense delivery for batched instances")
    ap.add_argument("--no-occupancy", action="store_true",
                    help="skip the occupancy-rule baseline (the paper's block sizing) beside the autotuned run")
    ap.add_argument("--no-scale-point", action="store_true",
                    help="skip the forced-activity propagation measurement at 100 x 1,000,000, p = 0.5")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    return rank, world, local


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        rows = []
        for ln in (self.out or "").strip().splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) >= 9:
                rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": reasons, "samples": len(rows)}


def _forced_propagation(snn, torch, dev, n_mid, p, layout, reps=7, flush=None, tiled=None):
    """Forced activity: all 100 input rows spike; times the production
    propagation kernel alone (L2 flushed before each launch) and returns
    algorithmic bytes / time.  tiled: SNN_OPT_TILED (None: the library's choice)."""
    spec = I.net([I.source_pop(100, 0.0), I.hh_pop(n_mid)],
                 [I.proj(0, 1, layout, p, ("lognormal", -3.0, 0.5))], dt=0.1, steps=1)
    net = snn.Network.from_spec(spec, device=dev)
    if tiled is not None:
        net.set_option("tiled", tiled)
    rows = 100
    net.debug_propagate(0, np.arange(rows, dtype=np.int32))
    nnz = net.nnz(0)
    if layout == "dense":
        events, nbytes = rows * n_mid, rows * n_mid * 4 + rows * 4
    else:
        events, nbytes = nnz, nnz * BYTES_PER_EVENT + rows * BYTES_PER_ROW
    s = torch.cuda.current_stream()
    times = []
    for _ in range(reps):
        if flush is not None:
            _flush_l2(flush)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        net.launch_phase(3)
        e1.record(s)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    mode = net.proj_mode(0)
    net.sync()
    net.close()
    t = statistics.median(times) * 1e-3
    return {"n_mid": n_mid, "p": p, "layout": layout, "events": events, "bytes": nbytes,
            "us": t * 1e6, "gbs": nbytes / t / 1e9, "events_per_s": events / t,
            "kernel": "k_propagate" if layout == "dense" else PROPAGATION_KERNELS[mode]}


PROPAGATION_KERNELS = {0: "k_propagate", 1: "k_propagate_tiled", 2: "k_propagate_seg"}


def _forced_propagation_cycled(snn, torch, dev, n_mid, p, layout, rounds=6, tiled=None):
    """The forced-activity propagation of _forced_propagation with inputs
    larger than L2 instead of a flush: copies of the network (different
    connectivity seeds) whose synapses total at least three times L2 are
    launched in turn, back to back (a device-side sleep holds the stream while
    the host enqueues every launch), so each launch streams its rows from HBM
    while code, page-table entries and the launch's small state stay warm, as
    in a run of many steps.  Returns the mean time per launch."""
    rows = 100
    one = None
    nets = []
    while True:
        spec = I.net([I.source_pop(100, 0.0), I.hh_pop(n_mid)],
                     [I.proj(0, 1, layout, p, ("lognormal", -3.0, 0.5))], dt=0.1, steps=1, seed=101 + len(nets))
        net = snn.Network.from_spec(spec, device=dev)
        if tiled is not None:
            net.set_option("tiled", tiled)
        net.debug_propagate(0, np.arange(rows, dtype=np.int32))
        nets.append(net)
        if one is None:
            nnz = net.nnz(0)
            one = rows * n_mid * 4 if layout == "dense" else nnz * BYTES_PER_EVENT
            want = max(1, min(16, int(np.ceil(3 * L2_BYTES / one))))
        if len(nets) >= want:
            break
    s = torch.cuda.current_stream()
    for net in nets:                                       # warm-up
        net.launch_phase(3)
    torch.cuda.synchronize()
    torch.cuda._sleep(int(2e6))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(rounds):
        for net in nets:
            net.launch_phase(3)
    e1.record(s)
    e1.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / (rounds * len(nets))
    mode = nets[0].proj_mode(0)
    for net in nets:
        net.sync()
        net.close()
    return {"us_cycled": us, "copies": want, "synapse_bytes_per_copy": one,
            "kernel": "k_propagate" if layout == "dense" else PROPAGATION_KERNELS[mode]}


def _neuron_rate(snn, torch, dev, n, reps=50):
    spec = I.net([I.hh_pop(n)], [], dt=0.1, steps=1)
    net = snn.Network.from_spec(spec, device=dev)
    net.set_option("engine", 0)
    t = _phase_time_ms(net, 0, reps, torch)
    net.close()
    flops = n * (FLOPS_PER_SUBSTEP * 4 + FLOPS_PER_STEP_EXTRA)
    return {"n": n, "us": t * 1e3, "neuron_steps_per_s": n / (t * 1e-3), "tflops": flops / (t * 1e-3) / 1e12}


def _batched(snn, torch, dev, n_inst, steps, weight_hi=0.05):
    """The batched form (n_inst instances of the small workload, middle sizes
    and conductance factors log-uniform, one network object) against the same
    instances run one after another as stand-alone networks.  weight_hi = 60
    nS is the forced-activity variant (the 0.05 nS of the small workload
    leaves every middle population silent under the 1/(p N_pre) scaling)."""
    specs = I.config_batched(n_inst, steps=steps, weight_hi=weight_hi)
    batch = snn.Network.from_specs(specs, device=dev)
    tune = batch.autotune(trial_steps=100)
    batch.reset()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    batch.step(steps)
    e1.record()
    e1.synchronize()
    t_batch = e0.elapsed_time(e1) * 1e-3
    n_hh = [s["pops"][1]["n"] for s in specs]
    rate_b = np.array([batch.counters(batch.pop_offsets[b] + 1)[0] / n_hh[b] / (steps * specs[0]["dt"] * 1e-3)
                       for b in range(n_inst)])
    nan_b = np.array([batch.counters(batch.pop_offsets[b] + 1)[1] for b in range(n_inst)])
    ev_b = batch.synaptic_events()
    batch.close()
    solos = [snn.Network.from_spec(s, device=dev) for s in specs]
    for net in solos:
        net.step(1)
        net.reset()
    torch.cuda.synchronize()
    e0.record()
    for net in solos:
        net.step(steps)
    e1.record()
    e1.synchronize()
    t_seq = e0.elapsed_time(e1) * 1e-3
    rate_s = np.array([solos[b].counters(1)[0] / n_hh[b] / (steps * specs[0]["dt"] * 1e-3) for b in range(n_inst)])
    nan_s = np.array([solos[b].counters(1)[1] for b in range(n_inst)])
    for net in solos:
        net.close()
    neuron_steps = (sum(n_hh) + 100 * n_inst) * steps
    # per-instance agreement of the rates in the sense of the 2 % rule
    # (|r_b - r_s| <= 0.02 r_s + one spike over the run), NaN-free instances only
    spikes_b = rate_b * np.array(n_hh) * steps * specs[0]["dt"] * 1e-3
    spikes_s = rate_s * np.array(n_hh) * steps * specs[0]["dt"] * 1e-3
    clean = (nan_b == 0) & (nan_s == 0)
    within = np.abs(spikes_b - spikes_s) <= 0.02 * spikes_s + 1.0
    return {"workload": f"{n_inst} instances of 100 Poisson sources -> N HH (p = 0.1), N log-uniform 1k-50k, "
                        f"conductance factor log-uniform 0.1-10, weights U(0, {weight_hi}) nS, {steps} steps",
            "instances_spiking": int((spikes_s > 0).sum()),
            "rates_within_2pct_plus_one_spike": int((within & clean).sum()), "nan_free_instances": int(clean.sum()),
            "neurons": sum(n_hh) + 100 * n_inst, "autotune": tune,
            "batched_s": t_batch, "sequential_s": t_seq, "speedup": t_seq / t_batch,
            "batched_neuron_steps_per_s": neuron_steps / t_batch,
            "sequential_neuron_steps_per_s": neuron_steps / t_seq,
            "batched_events": ev_b,
            "mean_rate_hz": float(rate_b.mean()), "max_rate_diff_hz": float(np.abs(rate_b - rate_s).max()),
            "instances_with_nan": int((nan_b > 0).sum()), "nan_counts_equal": bool(np.array_equal(nan_b, nan_s))}


def _timed(torch, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    r = fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1), r


def _plain_forward_runs(net, steps, n=6):
    """The n plain forward runs a central difference over the 3 scales needs:
    snn_step from the creation state, recording nothing (no checkpoints, no
    filter: a lower bound on what each difference quotient costs)."""
    for _ in range(n):
        net.reset()
        net.step(steps)


def _shared_dense_batch(snn, torch, dev, n_inst=512, n=1024, rate_hz=500.0, steps=1000):
    """Batched instances sharing one dense projection on the time-step path
    (snn_add_shared_dense): n_inst instances of n Poisson sources (rate_hz,
    5 % spiking per 0.1 ms step at 500 Hz) -> n HH neurons through one shared
    n x n weight matrix with per-instance scales; steps/s with the delivery on
    the CUDA cores, on the tensor cores and chosen by spike density."""
    specs = [I.net([I.source_pop(n, rate_hz), I.hh_pop(n)], [], dt=0.1, steps=1, instance=b) for b in range(n_inst)]
    rng = np.random.default_rng([I.SEED, 11])
    W = torch.from_numpy(rng.uniform(0.0, 0.03, (n, n)).astype(np.float32))
    scales = np.exp(rng.uniform(np.log(0.1), np.log(10.0), n_inst))
    net = snn.Network.from_specs(specs, device=dev)
    net.add_shared_dense(0, 1, W, scales)
    s = torch.cuda.current_stream()
    out = {"workload": f"{n_inst} instances of {n} Poisson sources ({rate_hz:g} Hz) -> {n} HH, one shared {n} x {n} "
                       f"dense projection, {steps} steps", "neurons": 2 * n * n_inst}
    for name, engine in (("cuda_cores", 0), ("tensor_cores", 1), ("by_density", 2)):
        net.set_option("shared_dense", engine)
        net.reset()
        net.step(100)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        net.step(steps)
        e1.record(s)
        e1.synchronize()
        t = e0.elapsed_time(e1) * 1e-3
        out[name + "_steps_per_s"] = steps / t
        out[name + "_us_per_step"] = t / steps * 1e6
    out["tensor_over_cuda_cores"] = out["tensor_cores_steps_per_s"] / out["cuda_cores_steps_per_s"]
    out["spike_density"] = sum(net.counters(net.pop_offsets[b])[0] for b in range(n_inst)) / (n_inst * n * (steps + 100))
    net.close()
    return out


def _largest_sweep_network(snn, torch, dev, flush, steps=1000):
    """The whole time step at the scaling sweep's largest point: In 100
    (driven) -> Mid 1,000,000 (compressed rows, p = 0.5: 5e7 synapses) -> Out
    100 (dense, 1e8 weights), 1000 steps through snn_step with the autotuned
    launch configuration, L2 flushed before each timed run.  Reports synaptic
    events/s, HH neuron-steps/s and the per-phase kernel times."""
    spec = I.config_sweep(1_000_000, 0.5, "csr", steps=steps)
    net = snn.Network.from_spec(spec, device=dev)
    tune = net.autotune(trial_steps=200)
    s = torch.cuda.current_stream()
    ms, evs = [], []
    for k in range(4):
        net.reset()
        _flush_l2(flush)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        net.step(steps)
        e1.record(s)
        e1.synchronize()
        if k:                                   # the first run warms up
            ms.append(e0.elapsed_time(e1))
            evs.append(net.synaptic_events())
    t = statistics.median(ms) * 1e-3
    n_neurons = sum(p["n"] for p in spec["pops"])
    spikes = [net.counters(p)[0] for p in range(len(spec["pops"]))]
    out = {"workload": spec["name"] + f", {steps} steps", "neurons": n_neurons, "synapses": net.nnz(0),
           "dense_weights": net.nnz(1), "engine": net.engine, "autotune": tune, "ms": t * 1e3,
           "synaptic_events_per_s": statistics.median(evs) / t, "neuron_steps_per_s": n_neurons * steps / t,
           "spikes_per_population": spikes}
    if net.engine == "plain":
        t_n = _phase_time_ms(net, 0, 50, torch)
        t_p = _phase_time_ms(net, 1, 50, torch)
        out.update({"k_neuron_step_us": t_n * 1e3, "k_propagate_us": t_p * 1e3,
                    "neuron_kernel_steps_per_s": n_neurons / (t_n * 1e-3)})
    net.close()
    return out


def _differentiable(snn, torch, dev, steps=2000, K=100):
    """Differentiable form (graded synapses, 20,000 middle neurons, p = 0.05):
    recorded forward (y) + squared-error loss on top (torch) + adjoint
    backward (dL/dy seed) against the 6 plain forward runs a central finite
    difference over the 3 projection scales needs."""
    from paper_1412_0595_gb300.network import squared_error
    spec = I.config_graded(steps=steps)
    net = snn.GradedNetwork.from_spec(spec, device=dev)
    n_out = spec["pops"][-1]["n"]
    target = torch.from_numpy(I.target_trace(spec, steps, n_out)).to(dev)
    nnz = sum(net.nnz(q) for q in range(net.n_projs))
    y = net.forward_record(steps, checkpoint_every=K)
    net.backward(squared_error(y, target)[1])
    torch.cuda.synchronize()
    t_f, y = _timed(torch, lambda: net.forward_record(steps, checkpoint_every=K))
    loss, dl = squared_error(y, target)
    t_b, (gs, gw) = _timed(torch, lambda: net.backward(dl))
    t_fd, _ = _timed(torch, lambda: [net.forward_record(steps, checkpoint_every=K) for _ in range(6)])
    t_plain, _ = _timed(torch, lambda: _plain_forward_runs(net, steps))
    peaks, src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    # the transposed pre indices are 16-bit when every pre population has at most 65,536 neurons
    per_syn = 6 if max(spec["pops"][d["pre"]]["n"] for d in spec["projs"]) <= 65536 else 8
    fwd_gbs = nnz * per_syn * steps / (t_f * 1e-3) / 1e9
    # the forward product alone (k_graded_spmv), L2 flushed before each launch
    flush = _flush_buffers(torch, dev)
    s = torch.cuda.current_stream()
    times = []
    for _ in range(12):
        _flush_l2(flush)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        net.launch_product()
        e1.record(s)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    del flush
    prod_us = statistics.median(times[2:]) * 1e3
    prod_gbs = nnz * per_syn / (prod_us * 1e-6) / 1e9
    out = {"workload": f"graded HH: In 100 -> Mid 20,000 (+ recurrent) -> Out 100, p = 0.05, {steps} steps of 0.05 ms",
           "synapses": nnz, "checkpoint_every": K, "loss": loss,
           "forward_ms": t_f, "backward_ms": t_b, "adjoint_total_ms": t_f + t_b,
           "six_plain_forward_runs_ms": t_plain, "adjoint_vs_plain_fd": t_plain / (t_f + t_b),
           "six_recorded_forward_runs_ms": t_fd, "adjoint_vs_fd_speedup": t_fd / (t_f + t_b),
           "gradients": 3 + nnz, "grad_scale": gs.cpu().tolist(),
           "forward_bytes_per_synapse": per_syn,
           "forward_synapse_stream_gbs": fwd_gbs, "forward_frac_hbm": fwd_gbs / hbm,
           "product_kernel": {"kernel": "k_graded_spmv", "us": prod_us, "gbs": prod_gbs, "frac_hbm": prod_gbs / hbm,
                              "bytes": nnz * per_syn, "l2": "flushed before each launch"},
           "finite": bool(torch.isfinite(gs).all() and all(torch.isfinite(g).all() for g in gw))}
    net.close()
    return out


def _differentiable_dense(snn, torch, dev, steps=2000, K=100):
    """Differentiable form with dense storage (Eq. 2) of the middle
    population's projections: In 100 -> Mid 4096 (compressed rows, p = 0.05),
    Mid -> Mid and Mid -> Out dense.  Recorded forward, adjoint with the
    weight gradient on the tensor cores and on the CUDA cores, and the 6
    forward runs of a central difference over the 3 scales."""
    from paper_1412_0595_gb300.network import squared_error
    spec = I.config_graded_dense(steps=steps)
    net = snn.GradedNetwork.from_spec(spec, device=dev)
    n_out = spec["pops"][-1]["n"]
    target = torch.from_numpy(I.target_trace(spec, steps, n_out)).to(dev)
    y = net.forward_record(steps, checkpoint_every=K)
    net.backward(squared_error(y, target)[1])
    torch.cuda.synchronize()
    t_f, y = _timed(torch, lambda: net.forward_record(steps, checkpoint_every=K))
    loss, dl = squared_error(y, target)
    net.set_option("dense_grad", 1)
    t_bt, (gs, gw) = _timed(torch, lambda: net.backward(dl))
    net.set_option("dense_grad", 0)
    t_bc, (gs_c, gw_c) = _timed(torch, lambda: net.backward(dl))
    net.set_option("dense_grad", 1)
    t_fd, _ = _timed(torch, lambda: [net.forward_record(steps, checkpoint_every=K) for _ in range(6)])
    t_plain, _ = _timed(torch, lambda: _plain_forward_runs(net, steps))
    n_mid = spec["pops"][1]["n"]
    dense_w = n_mid * n_mid + n_mid * n_out
    peaks, _ = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    fwd_gbs = 4.0 * dense_w * steps / (t_f * 1e-3) / 1e9
    rel = [float(torch.linalg.norm(a - b) / torch.linalg.norm(b).clamp_min(1e-30)) for a, b in zip(gw, gw_c)]
    out = {"workload": f"graded HH, dense storage: In 100 -> Mid {n_mid} (p = 0.05), Mid -> Mid and Mid -> Out dense, "
                       f"{steps} steps of 0.05 ms",
           "dense_weights": dense_w, "checkpoint_every": K, "loss": loss,
           "forward_ms": t_f, "backward_tensor_ms": t_bt, "backward_cuda_core_ms": t_bc,
           "six_plain_forward_runs_ms": t_plain, "adjoint_vs_plain_fd": t_plain / (t_f + t_bt),
           "six_recorded_forward_runs_ms": t_fd, "adjoint_vs_fd_speedup": t_fd / (t_f + t_bt),
           "forward_dense_weight_stream_gbs": fwd_gbs, "forward_frac_hbm": fwd_gbs / hbm,
           "weight_grad_rel_diff_tensor_vs_cuda_core": rel,
           "finite": bool(torch.isfinite(gs).all() and all(torch.isfinite(g).all() for g in gw))}
    net.close()
    return out


def _dense_grad(snn, torch, dev, reps=20):
    """Rank-K weight-gradient update D += R^T N (one checkpoint segment of a
    dense projection) on the tensor cores (three BF16 parts per operand, six
    products) and on the CUDA cores.  Useful work 2 m n K FLOP; the tensor
    cores execute 6 x 2 x mp x np x kp (padded to 128 / 128 / 32).  Bytes:
    D read and written (8 m n) plus the operands (4 K (m + n))."""
    peaks, src = _peaks()
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    rng = np.random.default_rng(12)
    out = []
    for K, m, n in ((100, 4096, 4096), (512, 4096, 4096), (100, 20000, 100)):
        R = torch.from_numpy(rng.uniform(0, 1, (K, m)).astype(np.float32)).to(dev)
        N = torch.from_numpy(rng.normal(0, 1, (n, K)).astype(np.float32)).to(dev)
        D = torch.zeros((m, n), dtype=torch.float32, device=dev)
        h = snn.DenseGrad(device=dev)
        row = {"K": K, "m": m, "n": n}
        for eng in ("cuda", "tensor"):
            h.run(R, N, D, engine=eng)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                h.run(R, N, D, engine=eng)
            e1.record()
            e1.synchronize()
            row[eng + "_us"] = 1e3 * e0.elapsed_time(e1) / reps
        h.check()
        h.close()
        mp, np_, kp = -(-m // 128) * 128, -(-n // 128) * 128, -(-K // 32) * 32
        row["tensor_executed_tflops"] = 6 * 2 * mp * np_ * kp / (row["tensor_us"] * 1e-6) / 1e12
        row["tensor_frac_bf16_peak"] = row["tensor_executed_tflops"] / bf16
        nbytes = 8.0 * m * n + 4.0 * K * (m + n)
        row["tensor_gbs"] = nbytes / (row["tensor_us"] * 1e-6) / 1e9
        row["tensor_frac_hbm"] = row["tensor_gbs"] / hbm
        row["cuda_core_useful_tflops"] = 2.0 * m * n * K / (row["cuda_us"] * 1e-6) / 1e12
        row["speedup_tensor_over_cuda"] = row["cuda_us"] / row["tensor_us"]
        out.append(row)
    return {"rows": out, "peak_bf16_tflops": bf16, "peak_hbm_gbs": hbm, "peak_source": src,
            "traffic_4096x4096_K100": _traffic("k_dense_grad_mma")}


def _dense_batch(snn, torch, dev, reps=20):
    """Dense delivery for B instances sharing one projection: tensor cores
    (tcgen05, three BF16 parts of W, FP32 accumulation) against the CUDA-core
    rows, per step, at several activity levels.  Tensor work counts the
    padded product the MMAs execute: 3 x 2 x Bp x Kp x Np FLOP."""
    peaks, src = _peaks()
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    rng = np.random.default_rng(11)
    out = []
    for B, n_pre, n_post in ((512, 1000, 1000), (1024, 4096, 4096)):
        W = torch.from_numpy(rng.lognormal(-3.0, 0.5, (n_pre, n_post)).astype(np.float32))
        h = snn.DenseBatch(W, device=dev)
        scale = torch.ones(B, dtype=torch.float32, device=dev)
        G = torch.zeros((B, n_post), dtype=torch.float32, device=dev)
        for frac in (0.01, 0.1, 0.5):
            spikes = [np.sort(rng.choice(n_pre, max(1, int(frac * n_pre)), replace=False)) for _ in range(B)]
            lens = [len(x) for x in spikes]
            off = torch.tensor(np.concatenate([[0], np.cumsum(lens)]), dtype=torch.int32, device=dev)
            idx = torch.tensor(np.concatenate(spikes), dtype=torch.int32, device=dev)
            row = {"B": B, "n_pre": n_pre, "n_post": n_post, "activity": frac}
            for eng in ("cuda", "tensor"):
                h.deliver((off, idx), scale, G, engine=eng)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    h.deliver((off, idx), scale, G, engine=eng)
                e1.record()
                e1.synchronize()
                row[eng + "_us"] = 1e3 * e0.elapsed_time(e1) / reps
            h.check()
            bp, kp, np_ = -(-B // 256) * 256, -(-n_pre // 48) * 48, -(-n_post // 128) * 128   # the kernel's padding
            flops = 3 * 2 * bp * kp * np_
            row["tensor_tflops"] = flops / (row["tensor_us"] * 1e-6) / 1e12
            row["tensor_frac_bf16_peak"] = row["tensor_tflops"] / bf16
            row["speedup_tensor_over_cuda"] = row["cuda_us"] / row["tensor_us"]
            out.append(row)
        h.close()
    # DRAM bytes of the 1024 x 4096 x 4096 launch at 50 % activity (the ncu capture of --profile dense_batch)
    return {"rows": out, "peak_bf16_tflops": bf16, "peak_source": f"bf16_tflops ({src})",
            "traffic_1024x4096x4096": _traffic("k_dense_batch_mma")}


def _gscale_procedure(dev, steps=5000):
    """The paper's Fig. 1 procedure on the batched form: nConn 100..1000 step
    50 x gScale 2^(k/4), k = -8..16, reference (1000, 1.0); selection by
    closest avgSpike among NaN-free runs; fit of k1 / (k2 + nConn) + k3."""
    from paper_1412_0595_gb300 import gscale as G
    import torch
    n_conn = list(range(100, 1001, 50))
    grid = [2.0 ** (k / 4.0) for k in range(-8, 17)]
    specs, keys = G.sweep_specs(n_conn, grid, steps=steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    recs = G.run_sweep(specs, keys, device=dev)
    t_run = time.perf_counter() - t0
    x, y, target = G.select(recs, 1000.0, 1.0)
    (k1, k2, k3), mape = G.fit(x, y)
    return {"runs": len(recs), "steps": steps, "seconds_incl_build": t_run, "reference_avg_spike": target,
            "k1": k1, "k2": k2, "k3": k3, "mape_percent": mape,
            "selected": {str(int(a)): float(b) for a, b in zip(x, y)},
            "nan_runs": int(sum(r["sum_nans"] > 0 for r in recs))}


# Table 1 of the paper: the law fitted on its Izhikevich network
TABLE1_IZHIKEVICH = (1.318e3, 1.099e2, -2.800e-1)


def _gscale_procedure_izhikevich(dev, steps=1000):
    """Fig. 1's procedure on the paper's cortical network (Table 1, Fig. 2):
    nConn 100..1000 step 50 x gScale 2^(k/8), k = -8..32, reference (1000,
    1.0), 1 s per run; the fitted law next to Table 1's at nConn 100, 500,
    1000 (the paper's runs and raw numbers are not available; its constants
    are context, not a target)."""
    from paper_1412_0595_gb300 import gscale as G
    import torch
    n_conn = list(range(100, 1001, 50))
    grid = [2.0 ** (k / 8.0) for k in range(-8, 33)]
    specs, keys = G.izhikevich_sweep_specs(n_conn, grid, steps=steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    recs = G.run_sweep(specs, keys, device=dev)
    t_run = time.perf_counter() - t0
    x, y, target = G.select(recs, 1000.0, 1.0)
    (k1, k2, k3), mape = G.fit(x, y)
    at = {str(n): {"fit": G.law(n, k1, k2, k3), "table1": G.law(n, *TABLE1_IZHIKEVICH)} for n in (100, 500, 1000)}
    return {"runs": len(recs), "neurons_per_run": 1000, "steps": steps, "seconds_incl_build": t_run,
            "reference_avg_spike": target, "k1": k1, "k2": k2, "k3": k3, "mape_percent": mape,
            "table1": dict(zip(("k1", "k2", "k3"), TABLE1_IZHIKEVICH)), "gscale_at": at,
            "selected": {str(int(a)): float(b) for a, b in zip(x, y)},
            "nan_runs": int(sum(r["sum_nans"] > 0 for r in recs))}


def _cpu_baseline(sim_steps):
    """The FP64 oracle, as it stands, on a bounded sample: all host cores
    (its threaded step) and one thread."""
    import oracle
    spec = I.config_four_pop(steps=sim_steps)
    n_neurons = sum(p["n"] for p in spec["pops"])
    cores = os.cpu_count() or 1
    out = {}
    for threads in (cores, 1):
        oracle.set_threads(threads)
        ref = oracle.from_spec(spec)
        t0 = time.perf_counter()
        ref.step(sim_steps)
        out[threads] = (ref.events / (time.perf_counter() - t0), time.perf_counter() - t0)
    oracle.set_threads(1)
    return {"value": out[cores][0], "unit": "synaptic events/s", "cores": cores, "kind": "oracle",
            "sample": f"{sim_steps} of the 10,000 time steps of the same network, FP64, {cores} threads "
                      "(neurons and post ranges in parallel)",
            "seconds": out[cores][1], "neuron_steps_per_s": n_neurons * sim_steps / out[cores][1],
            "single_thread": {"value": out[1][0], "seconds": out[1][1]}}


def reduce_over_ranks(total_ms, events, device):
    """Whole-job figures of replicas: the slowest rank's time (every rank ran
    the same work, so the job ends with the slowest) and the sum of the
    ranks' events.  Needs an initialised process group; `device` is where
    the backend reduces (CUDA for NCCL, CPU for gloo)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms)], device=device, dtype=torch.float64)
    e = torch.tensor([float(events)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), float(e.item())


def run_reference(a):
    rank, world, _ = _dist()
    if rank != 0:
        return
    import oracle
    spec = I.config_four_pop(steps=a.cpu_steps)
    n_neurons = sum(p["n"] for p in spec["pops"])
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    times, events = [], 0
    for k in range(a.warmup + a.steps):
        ref = oracle.from_spec(spec)
        t0 = time.perf_counter()
        ref.step(a.cpu_steps)
        dt = time.perf_counter() - t0
        if k >= a.warmup:
            times.append(dt)
            events += ref.events
    total = sum(times)
    value = events / total
    line = {"impl": "reference", "metric": "synaptic events/s", "value": value, "unit": "synaptic events/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * total / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": spec["name"], "sim_steps_per_step": a.cpu_steps, "dt_ms": spec["dt"],
                       "substeps": spec["n_sub"]},
            "neuron_steps_per_s": n_neurons * a.cpu_steps * a.steps / total,
            "cpu_baseline": {"value": value, "unit": "synaptic events/s", "cores": cores, "kind": "oracle",
                             "sample": f"{a.cpu_steps} time steps of the same network per step, {cores} threads"},
            "e2e": {"value": value, "unit": "synaptic events/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _flush_buffers(torch, dev):
    """Two 256 MiB buffers (each larger than the 129 MB L2) for _flush_l2."""
    return (torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device=dev),
            torch.ones(64 * 1024 * 1024, dtype=torch.float32, device=dev))


def _flush_l2(buf):
    """Writes a buffer larger than L2, then reads a second one of the same
    size: the second pass evicts the written lines (their write-back happens
    here, not inside the timed kernel) and leaves L2 holding clean lines of
    unrelated data."""
    buf[0].add_(1.0)
    buf[1].sum()


def _persistent_time_ms(net, reps, torch, phase=2):
    """Average device time of one multi-step launch (SNN_OPT_PERSIST_STEPS
    complete steps; phase 2 the persistent kernel, 4 the cluster kernel),
    timed with events on the launching stream."""
    s = torch.cuda.current_stream()
    net.launch_phase(phase)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        net.launch_phase(phase)
    e1.record(s)
    e1.synchronize()
    net.sync()
    return e0.elapsed_time(e1) / reps


def _phase_time_ms(net, phase, reps, torch):
    """Average device time of one launch of a step phase: `reps` launches
    captured back to back in a CUDA graph and timed with events."""
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            for _ in range(reps):
                net.launch_phase(phase, stream=s)
        g.replay()
        s.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        g.replay()
        e1.record(s)
        s.synchronize()
    return e0.elapsed_time(e1) / reps


def run_ours(a):
    import torch
    import torch.distributed as dist

    import paper_1412_0595_gb300 as snn

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    spec = I.config_four_pop(steps=a.sim_steps)
    n_neurons = sum(p["n"] for p in spec["pops"])
    n_hh = sum(p["n"] for p in spec["pops"] if p["kind"] == "hh")
    net = snn.Network.from_spec(spec, device=dev)
    tune = net.autotune(trial_steps=500)
    stream = torch.cuda.current_stream()
    flush = _flush_buffers(torch, dev)

    def one_run():
        net.reset()
        _flush_l2(flush)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        net.step(a.sim_steps)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), net.synaptic_events()

    for _ in range(a.warmup):
        one_run()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ms, events = [], 0
    wall0 = time.perf_counter()
    with Clocks(local) as clk:
        for _ in range(a.steps):
            t, ev = one_run()
            ms.append(t)
            events += ev
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    total_ms = sum(ms)
    if world > 1:
        total_ms, events = reduce_over_ranks(total_ms, events, dev)
    value = events / (total_ms * 1e-3)
    neuron_steps = world * n_neurons * a.sim_steps * a.steps / (total_ms * 1e-3)

    # ---- per-kernel times for the roofline (same network, steady state) ----
    net.reset()
    net.step(a.steady_steps)
    torch.cuda.synchronize()
    spikes = [net.counters(p)[0] for p in range(len(spec["pops"]))]
    ev_total = net.synaptic_events()
    engine = net.engine
    PERSIST = 1000
    net.set_option("persist_steps", PERSIST)
    t_neuron = _phase_time_ms(net, 0, a.phase_reps, torch)
    t_prop = _phase_time_ms(net, 1, a.phase_reps, torch)
    multi = engine in ("persistent", "cluster")
    t_persist = _persistent_time_ms(net, 3, torch, 4 if engine == "cluster" else 2) if multi else None
    peaks, src = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = SM_COUNT * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12        # TFLOP/s
    flops_per_neuron_step = FLOPS_PER_SUBSTEP * spec["n_sub"] + FLOPS_PER_STEP_EXTRA
    neuron_tflops = n_hh * flops_per_neuron_step / (t_neuron * 1e-3) / 1e12
    # algorithmic bytes of one propagation launch in the steady state above:
    # compressed rows stream 8 B per synapse + 12 B per spiking row, dense
    # rows 4 B per stored weight + 4 B per spiking row
    dense_ev = dense_rows = csr_rows = 0
    for d in spec["projs"]:
        if d["layout"] == "dense":
            dense_ev += spikes[d["pre"]] * spec["pops"][d["post"]]["n"]
            dense_rows += spikes[d["pre"]]
        else:
            csr_rows += spikes[d["pre"]]
    prop_bytes = ((ev_total - dense_ev) * BYTES_PER_EVENT + csr_rows * BYTES_PER_ROW
                  + dense_ev * 4 + dense_rows * 4) / a.steady_steps
    prop_gbs = prop_bytes / (t_prop * 1e-3) / 1e9
    other = {"k_neuron_step_us": 1e3 * t_neuron, "k_propagate_us": 1e3 * t_prop,
             "neuron_tflops": neuron_tflops, "propagate_gbs": prop_gbs}
    if multi:
        kname = "k_step_cluster" if engine == "cluster" else "k_step_persistent"
        flops = PERSIST * n_hh * flops_per_neuron_step
        ach = flops / (t_persist * 1e-3) / 1e12
        roof = {"kernel": kname, "bound": "alu", "achieved": ach, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": ach / fp32_peak, "traffic": _traffic(kname),
                "peak_source": "FP32 FMA peak from 152 SMs x 128 lanes x 2 x max SM clock "
                               f"({sm_mhz:.0f} MHz, {src})",
                "launch_us": 1e3 * t_persist, "steps_per_launch": PERSIST, "flops_per_launch": flops,
                "us_per_step": 1e3 * t_persist / PERSIST}
        if engine == "cluster":
            sms = net.cluster_size
            roof["sms_used"] = sms
            roof["frac_of_used_sms"] = ach / (fp32_peak * sms / SM_COUNT)
            # the special-function (XU) pipe: 16 lanes per clock per SM, i.e.
            # one warp instruction per 2 clocks; executed XU warp instructions
            # per launch from the ncu table (null when the kernel changed since)
            xu = _counter(kname, "xu_warp_inst_per_launch", "xu_sources_sha256")
            xu_peak = SM_COUNT * sm_mhz * 1e6 * 16 / 32                 # warp instructions / s
            if xu is not None:
                xu_rate = xu / (t_persist * 1e-3)
                roof["sfu"] = {"xu_warp_inst_per_launch": xu, "neuron_steps_per_launch": PERSIST * n_hh,
                               "xu_lane_ops_per_neuron_step": 32.0 * xu / (PERSIST * n_hh),
                               "achieved_warp_inst_per_s": xu_rate, "peak_warp_inst_per_s": xu_peak,
                               "frac": xu_rate / xu_peak, "frac_of_used_sms": xu_rate / (xu_peak * sms / SM_COUNT),
                               "peak_source": "152 SMs x 16 XU lanes per clock x max SM clock"}
            else:
                roof["sfu"] = None
        other[kname + "_us_per_step"] = 1e3 * t_persist / PERSIST
    elif t_neuron >= t_prop:
        roof = {"kernel": "k_neuron_step", "bound": "alu", "achieved": neuron_tflops, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": neuron_tflops / fp32_peak, "traffic": None,
                "peak_source": "FP32 FMA peak from 152 SMs x 128 lanes x 2 x max SM clock "
                               f"({sm_mhz:.0f} MHz, {src})",
                "launch_us": 1e3 * t_neuron, "flops_per_launch": n_hh * flops_per_neuron_step}
    else:
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        roof = {"kernel": "k_propagate", "bound": "hbm", "achieved": prop_gbs, "peak": hbm, "unit": "GB/s",
                "frac": prop_gbs / hbm, "traffic": None, "peak_source": f"hbm_gbs ({src})",
                "launch_us": 1e3 * t_prop, "bytes_per_launch": prop_bytes}
    roof["other"] = other

    # ---- forced-activity propagation at the sweep's largest point ----
    scale = None
    if not a.no_scale_point:
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        scale = []
        # 100 spiking rows onto 1,000,000 posts: each launch timed after an L2
        # flush (cold: page-table walks and code fetch included) and, as in a
        # run of many steps, cycled over copies larger than L2 (us_cycled)
        for layout, p in (("csr", 0.05), ("csr", 0.2), ("csr", 0.5), ("dense", 0.5)):
            r = _forced_propagation(snn, torch, dev, 1_000_000, p, layout, flush=flush)
            c = _forced_propagation_cycled(snn, torch, dev, 1_000_000, p, layout)
            r.update(us_cycled=c["us_cycled"], cycled_copies=c["copies"])
            r["frac_hbm"] = r["gbs"] / hbm
            r["frac_hbm_cycled"] = r["bytes"] / (c["us_cycled"] * 1e-6) / 1e9 / hbm
            r["traffic"] = _traffic(f"{r['kernel']} p={p}" if layout == "csr" else r["kernel"])
            scale.append(r)

    # ---- the paper's occupancy rule as a baseline to the autotuner ----
    occupancy = None
    if not a.no_occupancy and rank == 0:
        occupancy = _occupancy_baseline(snn, torch, dev, spec, a.sim_steps, value, flush)

    # ---- end to end through the public API from pinned host buffers ----
    e2e = None
    if not a.no_e2e:
        e2e = _e2e(a, spec, dev, torch, snn)

    batched = batched_forced = None
    if not a.no_batched and rank == 0:
        batched = _batched(snn, torch, dev, a.batch_instances, a.batch_steps)
        batched_forced = _batched(snn, torch, dev, a.batch_instances, a.batch_steps, weight_hi=60.0)
    largest = None
    if not a.no_scale_point and rank == 0:
        largest = _largest_sweep_network(snn, torch, dev, flush)
    shared_dense = None
    if not a.no_dense_batch and rank == 0:
        shared_dense = _shared_dense_batch(snn, torch, dev)
    differentiable = None
    if not a.no_graded and rank == 0:
        differentiable = _differentiable(snn, torch, dev)
    dense_batch = None
    if not a.no_dense_batch and rank == 0:
        dense_batch = _dense_batch(snn, torch, dev)
    graded_dense = dense_grad = None
    if not a.no_graded_dense and rank == 0:
        graded_dense = _differentiable_dense(snn, torch, dev)
        dense_grad = _dense_grad(snn, torch, dev)
    gscale_fit = gscale_izh = None
    if not a.no_gscale and rank == 0:
        gscale_fit = _gscale_procedure(dev)
        gscale_izh = _gscale_procedure_izhikevich(dev)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = _cpu_baseline(a.cpu_steps)

    if rank == 0:
        line = {"metric": "synaptic events/s", "value": value, "unit": "synaptic events/s", "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": total_ms / a.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": spec["name"], "sim_steps_per_step": a.sim_steps, "dt_ms": spec["dt"],
                           "substeps": spec["n_sub"], "neurons": n_neurons,
                           "l2": "flushed between timed steps (256 MiB written, then another 256 MiB read)",
                           "parallelism": "replicas" if world > 1 else "single"},
                "neuron_steps_per_s": neuron_steps,
                "events_per_step": events / (a.steps * world),
                "wall_s": wall,
                "roofline": roof,
                "propagation_at_scale": scale,
                "cpu_baseline": cpu,
                "e2e": e2e,
                "engine": engine,
                "autotune": tune,
                "occupancy_baseline": occupancy,
                "batched": batched,
                "batched_forced_activity": batched_forced,
                "largest_sweep_network": largest,
                "shared_dense_batch": shared_dense,
                "differentiable": differentiable,
                "dense_batch": dense_batch,
                "differentiable_dense": graded_dense,
                "dense_grad": dense_grad,
                "gscale_fit": gscale_fit,
                "gscale_fit_izhikevich": gscale_izh,
                "gpu_launches": a.steps * ((-(-a.sim_steps // 1000)) + 2 if multi
                                           else 2 * a.sim_steps + 2),
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    net.close()
    if world > 1:
        dist.destroy_process_group()


def _occupancy_baseline(snn, torch, dev, spec, sim_steps, tuned_value, flush):
    """The same workload under the configuration the paper's occupancy rule
    gives (Sec. 3: plain two-kernel step, grids filled to the resident-block
    limit), timed like the headline run; the autotuned/occupancy ratio is the
    autotuner's gain."""
    net = snn.Network.from_spec(spec, device=dev)
    cfg = net.occupancy_config(trial_steps=500)
    stream = torch.cuda.current_stream()
    ms = []
    for k in range(4):
        net.reset()
        _flush_l2(flush)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        net.step(sim_steps)
        e1.record(stream)
        e1.synchronize()
        if k:
            ms.append(e0.elapsed_time(e1))
    ev = net.synaptic_events()
    net.close()
    value = ev / (statistics.median(ms) * 1e-3)
    return {"config": cfg, "ms_per_run": statistics.median(ms), "value": value, "unit": "synaptic events/s",
            "autotuned_over_occupancy": tuned_value / value}


def _e2e(a, spec, dev, torch, snn):
    """Same metric through the public API: pinned host inputs copied in,
    network created, run, spike counters copied back, every step."""
    host_v0 = {k: torch.from_numpy(I.v0(spec, k)).pin_memory()
               for k, d in enumerate(spec["pops"]) if d["kind"] == "hh"}
    host_w = {}
    for q, d in enumerate(spec["projs"]):
        n_pre, n_post = I.n_pre_post(spec, q)
        if d["layout"] == "dense":
            host_w[q] = torch.from_numpy(I.weights(spec, q, n_pre * n_post)).pin_memory()
    nnz = {}
    for q, d in enumerate(spec["projs"]):
        if d["layout"] != "dense":
            rp, col = snn.csr_bernoulli(spec["seed"], I.rng_tag(spec["instance"], q), *I.n_pre_post(spec, q), d["p"],
                                        dev)
            nnz[q] = col.numel()
            host_w[q] = torch.from_numpy(I.weights(spec, q, nnz[q])).pin_memory()
    out_host = torch.empty(len(spec["pops"]) * 2, dtype=torch.int64).pin_memory()
    h2d = sum(t.numel() * 4 for t in host_v0.values()) + sum(t.numel() * 4 for t in host_w.values())
    d2h = out_host.numel() * 8

    def run():
        pops = []
        for k, d in enumerate(spec["pops"]):
            e = dict(d)
            if k in host_v0:
                e["v0"] = host_v0[k].to(dev, non_blocking=True)
            pops.append(e)
        projs = []
        for q, d in enumerate(spec["projs"]):
            e = dict(d)
            e["w"] = host_w[q].to(dev, non_blocking=True)
            if d["layout"] != "dense":
                rp, col = snn.csr_bernoulli(spec["seed"], I.rng_tag(spec["instance"], q),
                                            *I.n_pre_post(spec, q), d["p"], dev)
                e["row_ptr"], e["col"] = rp, col
            else:
                e["row_ptr"] = None
            projs.append(e)
        net = snn.Network(pops, projs, spec["dt"], spec["n_sub"], spec["seed"], spec["instance"], device=dev)
        net.autotune(trial_steps=500)          # cached after the first network of this shape
        net.step(a.sim_steps)
        ev = net.synaptic_events()
        cnt = torch.stack([torch.cat([net.read(p, "spike_count"), net.read(p, "nan_count")])
                           for p in range(len(spec["pops"]))]).flatten()
        out_host.copy_(cnt)
        torch.cuda.synchronize()
        net.close()
        return ev

    for _ in range(min(a.warmup, 2)):
        run()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    events = 0
    k = max(1, min(a.steps, 3))
    for _ in range(k):
        events += run()
    dt = time.perf_counter() - t0
    return {"value": events / dt, "unit": "synaptic events/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": k,
            "note": "wall clock per step: pinned H2D of weights and V0, device connectivity draw, "
                    "network creation, 10,000 time steps, D2H of counters"}


_KERNEL_SOURCES = {
    "k_step_cluster": ["cluster.cu", "neuron_update.cuh", "device_math.cuh", "compaction.cuh", "snn_internal.cuh"],
    "k_neuron_step": ["neuron.cu", "neuron_update.cuh", "device_math.cuh", "compaction.cuh", "snn_internal.cuh"],
    "k_propagate_tiled": ["propagate_tiled.cu", "snn_internal.cuh"],
    "k_propagate_seg": ["propagate_tiled.cu", "snn_internal.cuh"],
    "k_propagate": ["propagate.cu", "snn_internal.cuh"],
    "k_dense_batch_mma": ["dense_batch.cu", "tc_common.cuh", "snn_internal.cuh"],
    "k_dense_grad_mma": ["graded_dense.cu", "tc_common.cuh", "snn_internal.cuh"],
}


def _sources_sha256(rels):
    import hashlib
    h = hashlib.sha256()
    for rel in rels:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _counter(kernel, key, hash_key):
    """A per-launch ncu counter of `kernel` from profiles/traffic.json, or
    None when the kernel's sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            table = json.load(f)
    except (OSError, ValueError):
        return None
    row = table.get(kernel)
    if not row or key not in row:
        return None
    return row[key] if _sources_sha256(row["sources"]) == row.get(hash_key) else None


def _traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu table
    (profiles/traffic.json), or None when the kernel's sources changed since
    the counters were taken (the table stores a hash of them)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            table = json.load(f)
    except (OSError, ValueError):
        return None
    row = table.get(kernel)
    if not row:
        return None
    return row["bytes_per_launch"] if _sources_sha256(row["sources"]) == row["sources_sha256"] else None


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
