"""ctypes binding of the C-ABI in ``include/snn.h`` (argument marshalling only).

Every computation runs in the CUDA library ``_build/libsnn.so``; if it is
missing, importing this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from pathlib import Path

LIB_PATH = Path(__file__).resolve().parent / "_build" / "libsnn.so"

# status codes (snn_status)
SNN_OK = 0
STATUS = {0: "SNN_OK", 1: "SNN_ERR_INVALID_ARG", 2: "SNN_ERR_CSR", 3: "SNN_ERR_GSCALE", 4: "SNN_ERR_OOM",
          5: "SNN_ERR_CUDA", 6: "SNN_ERR_TIMEOUT", 7: "SNN_ERR_STATE", 8: "SNN_ERR_SIZE"}
POP_HH, POP_SOURCE, POP_IZH = 0, 1, 2
LAYOUT_CSR, LAYOUT_DENSE = 0, 1
SYN_EXP, SYN_GRADED = 0, 1
FIELD = {"V": 0, "m": 1, "h": 2, "n": 3, "g0": 4, "g1": 5, "iext": 6, "isyn": 7, "spikes": 8, "nspk": 9,
         "spike_count": 10, "nan_count": 11, "neuron_spikes": 12}
OPT = {"record_isyn": 0, "graph_steps": 1, "prop_blocks": 2, "chunk": 3, "spin_limit": 4, "engine": 5,
       "persist_steps": 6, "tiled": 7, "test_barrier_extra": 8, "cluster_ctas": 9, "dense_grad": 10,
       "shared_dense": 11, "graded_store": 12}


class PopDesc(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("n", C.c_int32),
        ("C", C.c_double), ("gNa", C.c_double), ("ENa", C.c_double), ("gK", C.c_double),
        ("EK", C.c_double), ("gL", C.c_double), ("EL", C.c_double),
        ("E_syn", C.c_double * 2), ("tau_syn", C.c_double * 2), ("v_thresh", C.c_double),
        ("src_rate_hz", C.c_double), ("drive_rate_hz", C.c_double), ("drive_amp", C.c_double),
        ("drive_tau", C.c_double),
        ("v0", C.c_void_p), ("v0_on_device", C.c_int32), ("reserved", C.c_int32),
        ("izh", C.c_double * 8), ("noise_sigma", C.c_double), ("bias", C.c_double),
    ]


class ProjDesc(C.Structure):
    _fields_ = [
        ("pre", C.c_int32), ("post", C.c_int32), ("layout", C.c_int32), ("channel", C.c_int32),
        ("synapse", C.c_int32), ("on_device", C.c_int32), ("input_dense", C.c_int32),
        ("reserved", C.c_int32), ("nnz", C.c_int64),
        ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("w", C.c_void_p),
        ("k1", C.c_double), ("k2", C.c_double), ("k3", C.c_double), ("density", C.c_double),
        ("n_conn", C.c_double), ("user_scale", C.c_double), ("v_thr", C.c_double), ("v_slope", C.c_double),
    ]


class NetDesc(C.Structure):
    _fields_ = [("pops", C.POINTER(PopDesc)), ("n_pops", C.c_int32), ("projs", C.POINTER(ProjDesc)),
                ("n_projs", C.c_int32), ("rng_instance", C.c_uint32), ("reserved", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("engine", C.c_int32), ("prop_blocks", C.c_int32), ("chunk", C.c_int32), ("tiled", C.c_int32),
                ("us_per_step", C.c_double), ("cached", C.c_int32), ("reserved", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


def _load():
    if not LIB_PATH.exists():
        raise ImportError(
            f"CUDA library {LIB_PATH} is missing: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (there is no CPU fallback)")
    L = C.CDLL(str(LIB_PATH), mode=os.RTLD_NOW | getattr(os, "RTLD_GLOBAL", 0))
    vp, i32, i64, u32, u64, dbl, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double, C.c_size_t
    P = C.POINTER
    sig = {
        "snn_create_network": ([P(PopDesc), i32, P(ProjDesc), i32, dbl, i32, u64, u32, P(Allocator), vp, P(vp)]),
        "snn_create_batch": [P(NetDesc), i32, dbl, i32, u64, P(Allocator), vp, P(vp)],
        "snn_add_shared_dense": [vp, i32, i32, i32, i32, vp, i32, i32, dbl, dbl, dbl, dbl, dbl, P(dbl), vp],
        "snn_destroy": [vp],
        "snn_step": [vp, i64, vp],
        "snn_sync": [vp, vp],
        "snn_read_state": [vp, i32, i32, vp, sz, i32, vp],
        "snn_write_state": [vp, i32, i32, vp, sz, i32, vp],
        "snn_reset": [vp, vp],
        "snn_set_option": [vp, i32, i64],
        "snn_get_option": [vp, i32, C.POINTER(C.c_int64)],
        "snn_get_step": [vp, P(i64), vp],
        "snn_get_engine": [vp, P(i32)],
        "snn_synaptic_events": [vp, P(i64), vp],
        "snn_launch_phase": [vp, i32, vp],
        "snn_proj_scale": [vp, i32, P(C.c_float)],
        "snn_proj_nnz": [vp, i32, P(i64)],
        "snn_proj_mode": [vp, i32, P(i32)],
        "snn_graded_launch_product": [vp, vp],
        "snn_debug_propagate": [vp, i32, vp, i32, i32, vp],
        "snn_event_list": [vp, i32, vp, i32, i32, vp, vp, i64, P(i64), vp],
        "snn_csr_bernoulli_rows": [u64, u32, i64, i64, dbl, vp, P(i64), P(Allocator), vp],
        "snn_csr_bernoulli_fill": [u64, u32, i64, i64, dbl, vp, vp, vp],
        "snn_csr_bernoulli_rows_noalloc": [u64, u32, i64, i64, dbl, vp, P(i64), vp],
        "snn_set_scale": [vp, i32, dbl],
        "snn_set_weights": [vp, i32, vp, i32, vp],
        "snn_forward_record": [vp, i64, i32, i32, dbl, vp, vp],
        "snn_backward": [vp, vp, vp, P(vp), vp],
        "snn_state_size": [vp, P(sz)],
        "snn_save_state": [vp, vp, sz, i32, vp],
        "snn_load_state": [vp, vp, sz, i32, vp],
        "snn_autotune": [vp, i32, P(Tuning), vp],
        "snn_occupancy_config": [vp, i32, P(Tuning), vp],
        "snn_dense_batch_create": [vp, i32, i32, i32, P(Allocator), vp, P(vp)],
        "snn_dense_batch_destroy": [vp],
        "snn_dense_batch_deliver": [vp, i32, vp, vp, vp, vp, i64, i32, vp],
        "snn_dense_batch_check": [vp, vp],
        "snn_dense_grad_create": [P(Allocator), vp, P(vp)],
        "snn_dense_grad_destroy": [vp],
        "snn_dense_grad_run": [vp, vp, i64, vp, i64, i32, i32, i32, vp, i64, i32, vp],
        "snn_dense_grad_check": [vp, vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.snn_last_error.argtypes = []
    L.snn_last_error.restype = C.c_char_p
    return L


lib = _load()


class SNNError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


def check(status):
    if status != SNN_OK:
        raise SNNError(status, lib.snn_last_error().decode(errors="replace"))
    return status
