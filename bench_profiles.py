"""Measurement modes that are not the bench line: the launches the ncu
summaries under profiles/ were captured from, the propagation sweeps, and
the per-kernel counter table that bench.py reads (profiles/traffic.json).

  python bench_profiles.py --profile <target>     a few launches of one kernel (see run_profile)
  python bench_profiles.py --sweep                neuron-update rate and forced-activity propagation
                                                  over the scaling sweep's sizes and densities
  python bench_profiles.py --tiled-crossover      row kernel against post-tiled kernel
  python bench_profiles.py --record-traffic KERNEL BYTES COMMAND
  python bench_profiles.py --record-xu KERNEL WARP_INSTRUCTIONS NEURON_STEPS COMMAND
"""
from __future__ import annotations

import argparse
import json
import os
import statistics

import numpy as np

import snn_inputs as I
from bench import (BYTES_PER_EVENT, ROOT, _KERNEL_SOURCES, _flush_buffers, _flush_l2, _forced_propagation,
                   _neuron_rate, _peaks, _sources_sha256)


def run_tiled_crossover(a):
    """Forced activity (100 spiking rows, caches flushed before each of 7
    launches, median): the row kernel (SNN_OPT_TILED 0) against the
    post-tiled kernels (1 bulk copies, 3 segments) at several post-population
    sizes and densities;
    fraction of the measured copy bandwidth at 8 B per synapse."""
    import torch

    import paper_1412_0595_gb300 as snn
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    peaks, _ = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    flush = _flush_buffers(torch, dev)
    rows = np.arange(100, dtype=np.int32)
    for n_mid in (1_000_000, 300_000, 100_000):
        for p in (0.01, 0.02, 0.05, 0.1, 0.2, 0.5):
            spec = I.net([I.source_pop(100, 0.0), I.hh_pop(n_mid)],
                         [I.proj(0, 1, "csr", p, ("lognormal", -3.0, 0.5))], dt=0.1, steps=1)
            net = snn.Network.from_spec(spec, device=dev)
            net.debug_propagate(0, rows)
            nnz = net.nnz(0)
            line = {"n_mid": n_mid, "p": p, "synapses": nnz}
            for t in (0, 1, 3):
                net.set_option("tiled", t)
                net.debug_propagate(0, rows)
                s = torch.cuda.current_stream()
                times = []
                for _ in range(7):
                    _flush_l2(flush)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(s)
                    net.launch_phase(3)
                    e1.record(s)
                    e1.synchronize()
                    times.append(e0.elapsed_time(e1))
                net.sync()
                us = statistics.median(times) * 1e3
                name = {0: "row", 1: "tiled", 3: "segments"}[t]
                line[name + "_us"] = us
                line[name + "_frac_hbm"] = nnz * BYTES_PER_EVENT / (us * 1e-6) / 1e9 / hbm
            print(json.dumps(line), flush=True)
            net.close()



def run_sweep(a):
    import torch

    import paper_1412_0595_gb300 as snn
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    peaks, src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    flush = _flush_buffers(torch, dev)
    for n in I.SWEEP_N_MID:
        r = _neuron_rate(snn, torch, dev, n)
        r["kind"] = "neuron_update"
        print(json.dumps(r), flush=True)
        for p in I.SWEEP_P:
            for layout in ("csr", "dense"):
                r = _forced_propagation(snn, torch, dev, n, p, layout, flush=flush)
                r.update(kind="propagation", frac_hbm=r["gbs"] / hbm, hbm_peak=hbm, peak_source=src)
                print(json.dumps(r), flush=True)



def run_profile(a):
    """A few launches of one kernel on its workload, nothing timed: the
    command the ncu summaries under profiles/ were captured from.
      cluster: the four-population network, cluster engine, 1000 steps per launch;
      tiled:   forced-activity propagation, 100 rows x 1,000,000 posts, p = 0.5, CSR;
      csr_mid: the same at p = 0.05 (below the post-tiled threshold: the row kernel);
      dense:   the same with dense rows;
      neuron:  8,000,000 HH neurons, one neuron phase per launch;
      graded:  the differentiable workload (20,000 middle neurons), 200 steps
               recorded forward and the adjoint;
      dense_batch: tensor-core delivery for 1024 instances sharing a 4096 x 4096
               dense projection, half of the pre neurons spiking, three launches;
      dense_grad: the tensor-core rank-100 weight-gradient update of a 4096 x 4096
               dense projection, three launches;
      graded_dense: the dense differentiable workload (4096 middle neurons), 200
               steps recorded forward and the adjoint."""
    import torch

    import paper_1412_0595_gb300 as snn
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    if a.profile == "cluster":
        net = snn.Network.from_spec(I.config_four_pop(steps=1), device=dev)
        net.set_option("engine", 3)
        net.set_option("persist_steps", 1000)
        for _ in range(3):
            net.launch_phase(4)
    elif a.profile in ("tiled", "dense", "csr_mid", "seg_mid", "seg_dense"):
        flush = _flush_buffers(torch, dev)
        p = 0.05 if a.profile in ("csr_mid", "seg_mid") else 0.2 if a.profile == "seg_dense" else 0.5
        tiled = 3 if a.profile.startswith("seg") else None
        _forced_propagation(snn, torch, dev, 1_000_000, p, "dense" if a.profile == "dense" else "csr", reps=3,
                            flush=flush, tiled=tiled)
        return
    elif a.profile == "dense_batch":
        rng = np.random.default_rng(11)
        W = torch.from_numpy(rng.lognormal(-3.0, 0.5, (4096, 4096)).astype(np.float32))
        h = snn.DenseBatch(W, device=dev)
        spikes = [np.sort(rng.choice(4096, 2048, replace=False)) for _ in range(1024)]
        G = torch.zeros((1024, 4096), dtype=torch.float32, device=dev)
        scale = torch.ones(1024, dtype=torch.float32, device=dev)
        for _ in range(3):
            h.deliver(spikes, scale, G, engine="tensor")
        h.check()
        h.close()
        return
    elif a.profile == "dense_grad":
        rng = np.random.default_rng(12)
        R = torch.from_numpy(rng.uniform(0, 1, (100, 4096)).astype(np.float32)).to(dev)
        N = torch.from_numpy(rng.normal(0, 1, (4096, 100)).astype(np.float32)).to(dev)
        D = torch.zeros((4096, 4096), dtype=torch.float32, device=dev)
        h = snn.DenseGrad(device=dev)
        for _ in range(3):
            h.run(R, N, D, engine="tensor")
        h.check()
        h.close()
        return
    elif a.profile == "graded_dense":
        from paper_1412_0595_gb300.network import squared_error
        spec = I.config_graded_dense(steps=200)
        net = snn.GradedNetwork.from_spec(spec, device=dev)
        target = torch.from_numpy(I.target_trace(spec, 200, spec["pops"][-1]["n"])).to(dev)
        net.backward(squared_error(net.forward_record(200, checkpoint_every=100), target)[1])
    elif a.profile == "neuron":
        net = snn.Network.from_spec(I.net([I.hh_pop(8_000_000)], [], dt=0.1, steps=1), device=dev)
        net.set_option("engine", 0)
        for _ in range(4):
            net.launch_phase(0)
    else:
        from paper_1412_0595_gb300.network import squared_error
        spec = I.config_graded(steps=200)
        net = snn.GradedNetwork.from_spec(spec, device=dev)
        target = torch.from_numpy(I.target_trace(spec, 200, spec["pops"][-1]["n"])).to(dev)
        net.backward(squared_error(net.forward_record(200, checkpoint_every=100), target)[1])
    torch.cuda.synchronize()
    net.sync()
    net.close()



def record_traffic(kernel, nbytes, command):
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            table = json.load(f)
    except (OSError, ValueError):
        table = {}
    # a key may name the workload after the kernel ("k_propagate_stream p=0.2")
    rels = ["paper_1412_0595_gb300/csrc/" + x for x in _KERNEL_SOURCES[kernel.split(" ")[0]]]
    table[kernel] = {"bytes_per_launch": float(nbytes), "command": command, "sources": rels,
                     "sources_sha256": _sources_sha256(rels)}
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
        f.write("\n")


def record_xu(kernel, xu_inst, neuron_steps, command):
    """Executed XU-pipe (special-function unit) warp instructions of one
    launch of `kernel` from an ncu capture (sm__inst_executed_pipe_xu.sum),
    with the neuron-steps that launch performs, for bench.py's SFU roofline."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            table = json.load(f)
    except (OSError, ValueError):
        table = {}
    rels = ["paper_1412_0595_gb300/csrc/" + x for x in _KERNEL_SOURCES[kernel]]
    row = table.get(kernel, {})
    row.update({"xu_warp_inst_per_launch": float(xu_inst), "neuron_steps_per_launch": float(neuron_steps),
                "xu_command": command, "xu_sources_sha256": _sources_sha256(rels), "sources": rels})
    table[kernel] = row
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
        f.write("\n")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--profile", choices=["cluster", "tiled", "dense", "neuron", "graded", "dense_batch", "dense_grad",
                                          "graded_dense", "csr_mid", "seg_mid", "seg_dense"])
    ap.add_argument("--sweep", action="store_true")
    ap.add_argument("--tiled-crossover", action="store_true")
    ap.add_argument("--record-traffic", nargs=3, metavar=("KERNEL", "BYTES", "COMMAND"))
    ap.add_argument("--record-xu", nargs=4, metavar=("KERNEL", "XU_INST", "NEURON_STEPS", "COMMAND"))
    a = ap.parse_args()
    if a.record_traffic:
        record_traffic(*a.record_traffic)
    elif a.record_xu:
        record_xu(*a.record_xu)
    elif a.profile:
        run_profile(a)
    elif a.sweep:
        run_sweep(a)
    elif a.tiled_crossover:
        run_tiled_crossover(a)
    else:
        ap.print_help()


if __name__ == "__main__":
    main()
