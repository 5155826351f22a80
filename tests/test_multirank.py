"""The N > 1 path of bench.py (replicas, no data-path collective) on CPU
ranks with the gloo backend: whole-job time is the slowest rank's, events
add up, and the reference arm prints from rank 0 only."""
import io
import os
import socket
import sys
import types
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import torch
    total_ms, events = bench.reduce_over_ranks(10.0 + 5.0 * rank, 1000 * (rank + 1), torch.device("cpu"))
    # the reference arm: rank 0 runs the oracle sample and prints one line,
    # the other ranks return without work
    buf = io.StringIO()
    args = types.SimpleNamespace(cpu_steps=20, steps=1, warmup=0)
    with redirect_stdout(buf):
        bench.run_reference(args)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, total_ms, events, buf.getvalue()))


def test_replicas_reduce_and_reference_prints_once():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        rank, t, e, printed = q.get(timeout=300)
        out[rank] = (t, e, printed)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(world):
        t, e, _ = out[rank]
        assert t == 15.0 and e == 3000.0          # max of 10, 15; 1000 + 2000
    assert '"impl": "reference"' in out[0][2] and out[0][2].count("\n") == 1
    assert out[1][2] == ""
    # the line keeps the bench contract
    import json
    line = json.loads(out[0][2])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["metric"] == line["unit"] == "synaptic events/s" and line["higher_is_better"] is True
    # 20 steps are too few for spikes to reach the middle population: events, and value, may be 0
    assert line["n_gpus"] == world and line["value"] >= 0 and line["ms_per_step"] > 0 and line["dtype"] == "f64"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == line["e2e"]["d2h_bytes_per_step"] == 0
