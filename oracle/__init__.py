"""FP64 CPU oracle of the HH spiking-network time step (ctypes shim over plain C).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the product package may
not.  It shares no code with the CUDA library.

What it follows (paper sections): Sec. 2 (HH neurons at discrete time steps,
scaled synaptic conductance, NaN counting), Sec. 3 (compressed-row synapse
storage, Eq. 1 / Eq. 2), Sec. 5.1 (gScale = k1 / (k2 + nConn) + k3, Tables 1
and 2; Fig. 1 for spike and NaN counts).  The readings taken where the paper
is silent are stated in ``snn_oracle.c`` and ``snn_oracle_graded.c``.

Pins: every function here is checked in ``tests/test_oracle_*.py`` against
closed forms, published known-answer vectors, special cases and brute force.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "libsnn_oracle.so"
_SOURCES = [_HERE / "snn_oracle.c", _HERE / "snn_oracle_graded.c"]

POP_HH = 0
POP_SOURCE = 1
POP_IZH = 2

FIELD = {"V": 0, "m": 1, "h": 2, "n": 3, "g0": 4, "g1": 5, "iext": 6, "isyn": 7}


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree;
    OpenMP for the optional multi-threaded step used only for timing)."""
    _BUILD.mkdir(exist_ok=True)
    srcs = [s for s in _SOURCES if s.exists()]
    newest = max(s.stat().st_mtime for s in srcs)
    if not force and _LIB_PATH.exists() and _LIB_PATH.stat().st_mtime >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH.with_suffix(f".so.tmp{os.getpid()}")
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           f"-I{_HERE}", *map(str, srcs), "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OraclePop(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("n", C.c_int32),
        ("C", C.c_double), ("gNa", C.c_double), ("ENa", C.c_double), ("gK", C.c_double),
        ("EK", C.c_double), ("gL", C.c_double), ("EL", C.c_double),
        ("E_syn", C.c_double * 2), ("tau_syn", C.c_double * 2),
        ("v_thresh", C.c_double), ("src_rate_hz", C.c_double),
        ("drive_rate_hz", C.c_double), ("drive_amp", C.c_double), ("drive_tau", C.c_double),
        ("v0", C.POINTER(C.c_double)),
        ("izh", C.c_double * 8), ("noise_sigma", C.c_double), ("bias", C.c_double),
    ]


class OracleProj(C.Structure):
    _fields_ = [
        ("pre", C.c_int32), ("post", C.c_int32), ("dense", C.c_int32), ("channel", C.c_int32),
        ("nnz", C.c_int64),
        ("row_ptr", C.POINTER(C.c_int64)), ("col", C.POINTER(C.c_int32)),
        ("w", C.POINTER(C.c_double)),
        ("k1", C.c_double), ("k2", C.c_double), ("k3", C.c_double),
        ("n_conn", C.c_double), ("user_scale", C.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(str(build()))
        L = _lib
        u32p, i64p, i32p, f64p = (C.POINTER(C.c_uint32), C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int32), C.POINTER(C.c_double))
        L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.oracle_bernoulli_threshold.argtypes = [C.c_double]
        L.oracle_bernoulli_threshold.restype = C.c_uint64
        L.oracle_gscale.argtypes = [C.c_double] * 4 + [f64p]
        L.oracle_gscale.restype = C.c_int
        L.oracle_memory_words.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_int]
        L.oracle_memory_words.restype = C.c_int64
        L.oracle_hh_rates.argtypes = [C.c_double, f64p]
        L.oracle_hh_currents.argtypes = [f64p, C.c_double, C.c_double, C.c_double, C.c_double, f64p]
        L.oracle_net_create.argtypes = [C.POINTER(OraclePop), C.c_int, C.POINTER(OracleProj), C.c_int,
                                        C.c_double, C.c_int, C.c_uint64, C.c_uint32]
        L.oracle_net_create.restype = C.c_void_p
        L.oracle_net_destroy.argtypes = [C.c_void_p]
        L.oracle_net_step.argtypes = [C.c_void_p]
        L.oracle_net_run.argtypes = [C.c_void_p, C.c_int64]
        L.oracle_net_scale.argtypes = [C.c_void_p, C.c_int]
        L.oracle_net_scale.restype = C.c_double
        L.oracle_net_time.argtypes = [C.c_void_p]
        L.oracle_net_time.restype = C.c_uint32
        L.oracle_net_events.argtypes = [C.c_void_p]
        L.oracle_net_events.restype = C.c_int64
        L.oracle_net_get.argtypes = [C.c_void_p, C.c_int, C.c_int, f64p]
        L.oracle_net_set.argtypes = [C.c_void_p, C.c_int, C.c_int, f64p]
        L.oracle_net_spikes.argtypes = [C.c_void_p, C.c_int, i32p]
        L.oracle_net_spikes.restype = C.c_int32
        L.oracle_net_counters.argtypes = [C.c_void_p, C.c_int, i64p, i64p]
        L.oracle_net_deliver.argtypes = [C.c_void_p, C.c_int, i32p, C.c_int32]
        L.oracle_event_list.argtypes = [i64p, i32p, f64p, i32p, C.c_int32, i32p, f64p]
        L.oracle_event_list.restype = C.c_int64
        L.oracle_csr_rows.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_int64, C.c_double, i64p]
        L.oracle_csr_rows.restype = C.c_int64
        L.oracle_csr_fill.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_int64, C.c_double,
                                      i64p, i32p]
        L.oracle_source_spike.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                          C.c_double, C.c_double]
        L.oracle_source_spike.restype = C.c_int
        L.oracle_set_threads.argtypes = [C.c_int]
        L.oracle_get_threads.restype = C.c_int
        L.oracle_izh_r.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32]
        L.oracle_izh_r.restype = C.c_double
        L.oracle_izh_noise.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32]
        L.oracle_izh_noise.restype = C.c_double
        if hasattr(L, "oracle_graded_create"):
            _bind_graded(L)
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


# --------------------------------------------------------------------------
# Scalar functions
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def bernoulli_threshold(p: float) -> int:
    return int(lib().oracle_bernoulli_threshold(float(p)))


def gscale(k1, k2, k3, n_conn):
    """Sec. 5.1 scaling law; returns None at the pole nConn + k2 <= 0."""
    out = C.c_double()
    rc = lib().oracle_gscale(float(k1), float(k2), float(k3), float(n_conn), C.byref(out))
    return None if rc != 0 else out.value


def memory_words(nnz, n_pre, n_post, dense):
    return int(lib().oracle_memory_words(int(nnz), int(n_pre), int(n_post), int(bool(dense))))


def hh_rates(V: float) -> np.ndarray:
    """(alpha_m, beta_m, alpha_h, beta_h, alpha_n, beta_n) in 1/ms."""
    out = np.zeros(6)
    lib().oracle_hh_rates(float(V), _ptr(out, C.c_double))
    return out


def hh_currents(params, V, m, h, n) -> np.ndarray:
    p = np.array([params[k] for k in ("C", "gNa", "ENa", "gK", "EK", "gL", "EL")], dtype=np.float64)
    out = np.zeros(3)
    lib().oracle_hh_currents(_ptr(p, C.c_double), float(V), float(m), float(h), float(n),
                             _ptr(out, C.c_double))
    return out


def csr_bernoulli(seed: int, tag: int, n_pre: int, n_post: int, p: float):
    """Compressed rows drawn from the seed (row_ptr int64, col int32)."""
    row_ptr = np.zeros(n_pre + 1, dtype=np.int64)
    nnz = lib().oracle_csr_rows(seed, tag, n_pre, n_post, p, _ptr(row_ptr, C.c_int64))
    col = np.zeros(max(nnz, 1), dtype=np.int32)
    lib().oracle_csr_fill(seed, tag, n_pre, n_post, p, _ptr(row_ptr, C.c_int64), _ptr(col, C.c_int32))
    return row_ptr, col[:nnz]


def event_list(row_ptr, col, w, spk):
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    w = np.ascontiguousarray(w, np.float64)
    spk = np.ascontiguousarray(spk, np.int32)
    n = lib().oracle_event_list(_ptr(row_ptr, C.c_int64), _ptr(col, C.c_int32), _ptr(w, C.c_double),
                                _ptr(spk, C.c_int32), len(spk), None, None)
    post = np.zeros(max(n, 1), np.int32)
    wv = np.zeros(max(n, 1), np.float64)
    lib().oracle_event_list(_ptr(row_ptr, C.c_int64), _ptr(col, C.c_int32), _ptr(w, C.c_double),
                            _ptr(spk, C.c_int32), len(spk), _ptr(post, C.c_int32), _ptr(wv, C.c_double))
    return post[:n], wv[:n]


def source_spike(seed, tag, t, i, rate_hz, dt):
    return int(lib().oracle_source_spike(seed, tag, t, i, rate_hz, dt))


def dense_batch_deliver(W, spikes, scale, G0):
    """Dense delivery for B instances sharing W (Sec. 3, Eq. 2 storage), the
    plain definition in FP64: G[b, j] = G0[b, j] + scale[b] * sum over the
    spikes i of instance b of W[i, j], i.e. G0 + diag(scale) S W with S the
    0/1 spike matrix (a library matrix product as one step)."""
    W = np.asarray(W, np.float64)
    S = np.zeros((len(spikes), W.shape[0]))
    for b, spk in enumerate(spikes):
        S[b, np.asarray(spk, np.int64)] = 1.0
    return np.asarray(G0, np.float64) + np.asarray(scale, np.float64)[:, None] * (S @ W)


def dense_grad_update(R, N, D0):
    """Rank-K update of a dense weight gradient over a checkpoint segment, the
    plain definition in FP64: D[i, j] = D0[i, j] + sum_t R[t, i] N[j, t]
    (R: K x m releases, N: n x K dL/dG), i.e. D0 + R^T N^T (a library matrix
    product as one step)."""
    R = np.asarray(R, np.float64)
    N = np.asarray(N, np.float64)
    return np.asarray(D0, np.float64) + R.T @ N.T


def set_threads(n):
    """Threads of the network step (timing only; 1 = the sequential step)."""
    lib().oracle_set_threads(int(n))


def get_threads():
    return int(lib().oracle_get_threads())


def izh_r(seed, tag, i):
    """Per-neuron parameter draw r of an Izhikevich population."""
    return float(lib().oracle_izh_r(seed, tag, i))


def izh_noise(seed, tag, t, i):
    """Irwin-Hall input noise z of neuron i at step t."""
    return float(lib().oracle_izh_noise(seed, tag, t, i))


# --------------------------------------------------------------------------
# Network
# --------------------------------------------------------------------------
class OracleNet:
    """FP64 network built from the description dicts of ``snn_inputs``.

    ``pops``: list of dicts with keys kind ('hh' | 'source'), n, hh (dict of
    C, gNa, ENa, gK, EK, gL, EL), E_syn, tau_syn, v_thresh, rate_hz, drive
    (rate_hz, amp, tau) and v0 (array or None).
    ``projs``: list of dicts with keys pre, post, layout ('csr' | 'dense'),
    channel, row_ptr, col, w, k1, k2, k3, n_conn, user_scale.
    """

    def __init__(self, pops, projs, dt, n_sub, seed, instance=0):
        L = lib()
        self._keep = []
        P = (OraclePop * len(pops))()
        for k, d in enumerate(pops):
            p = P[k]
            p.kind = {"source": POP_SOURCE, "hh": POP_HH, "izh": POP_IZH}[d["kind"]]
            p.n = d["n"]
            hh = d.get("hh") or {}
            for f in ("C", "gNa", "ENa", "gK", "EK", "gL", "EL"):
                setattr(p, f, float(hh.get(f, 0.0)))
            E = d.get("E_syn", (0.0, -92.0))
            tau = d.get("tau_syn", (1.0, 1.0))
            p.E_syn[0], p.E_syn[1] = float(E[0]), float(E[1])
            p.tau_syn[0], p.tau_syn[1] = float(tau[0]), float(tau[1])
            p.v_thresh = float(d.get("v_thresh", 0.0))
            p.src_rate_hz = float(d.get("rate_hz", 0.0))
            drv = d.get("drive") or {}
            p.drive_rate_hz = float(drv.get("rate_hz", 0.0))
            p.drive_amp = float(drv.get("amp", 0.0))
            p.drive_tau = float(drv.get("tau", 0.0))
            izh = d.get("izh")
            if izh is not None:
                for j, f in enumerate(("a0", "a1", "b0", "b1", "c0", "c2", "d0", "d2")):
                    p.izh[j] = float(izh[f])
                p.noise_sigma = float(izh.get("noise", 0.0))
                p.bias = float(izh.get("bias", 0.0))
            v0 = d.get("v0")
            if v0 is not None:
                v0 = np.ascontiguousarray(v0, dtype=np.float64)
                self._keep.append(v0)
                p.v0 = _ptr(v0, C.c_double)
        Q = (OracleProj * max(len(projs), 1))()
        for k, d in enumerate(projs):
            q = Q[k]
            q.pre, q.post = d["pre"], d["post"]
            q.dense = 1 if d["layout"] == "dense" else 0
            q.channel = d.get("channel", 0)
            w = np.ascontiguousarray(d["w"], dtype=np.float64)
            self._keep.append(w)
            q.w = _ptr(w, C.c_double)
            if not q.dense:
                rp = np.ascontiguousarray(d["row_ptr"], dtype=np.int64)
                col = np.ascontiguousarray(d["col"], dtype=np.int32)
                self._keep += [rp, col]
                q.row_ptr, q.col = _ptr(rp, C.c_int64), _ptr(col, C.c_int32)
                q.nnz = len(col)
            else:
                q.nnz = len(w)
            q.k1, q.k2, q.k3 = float(d["k1"]), float(d["k2"]), float(d["k3"])
            q.n_conn = float(d["n_conn"])
            q.user_scale = float(d.get("user_scale", 1.0))
        h = L.oracle_net_create(P, len(pops), Q, len(projs), float(dt), int(n_sub), int(seed),
                                int(instance))
        self._keep = None
        if not h:
            raise ValueError("oracle rejected the network description")
        self.h = h
        self.sizes = [d["n"] for d in pops]
        self.n_pops = len(pops)

    def __del__(self):
        if getattr(self, "h", None):
            lib().oracle_net_destroy(self.h)
            self.h = None

    def step(self, n=1):
        if n == 1:
            lib().oracle_net_step(self.h)
        else:
            lib().oracle_net_run(self.h, int(n))

    @property
    def t(self):
        return int(lib().oracle_net_time(self.h))

    def scale(self, q):
        return float(lib().oracle_net_scale(self.h, q))

    @property
    def events(self):
        """Synaptic events delivered so far (stored synapses of spiking rows)."""
        return int(lib().oracle_net_events(self.h))

    def get(self, pop, field):
        out = np.zeros(self.sizes[pop], dtype=np.float64)
        if lib().oracle_net_get(self.h, pop, FIELD[field], _ptr(out, C.c_double)) != 0:
            raise ValueError(field)
        return out

    def set(self, pop, field, values):
        v = np.ascontiguousarray(values, dtype=np.float64)
        assert v.shape == (self.sizes[pop],)
        if lib().oracle_net_set(self.h, pop, FIELD[field], _ptr(v, C.c_double)) != 0:
            raise ValueError(field)

    def spikes(self, pop):
        out = np.zeros(max(self.sizes[pop], 1), dtype=np.int32)
        n = lib().oracle_net_spikes(self.h, pop, _ptr(out, C.c_int32))
        return out[:n].copy()

    def counters(self, pop):
        a, b = C.c_int64(), C.c_int64()
        lib().oracle_net_counters(self.h, pop, C.byref(a), C.byref(b))
        return a.value, b.value

    def deliver(self, proj, spk):
        s = np.ascontiguousarray(spk, dtype=np.int32)
        lib().oracle_net_deliver(self.h, proj, _ptr(s, C.c_int32), len(s))


def _bind_graded(L):
    from . import graded  # noqa: F401  (binds argtypes of the graded entry points)
    graded._bind(L)


def from_spec(spec, instance=None):
    """Builds an ``OracleNet`` from a ``snn_inputs`` network description: the
    oracle draws each projection's connectivity from the seed itself, uses
    nConn = p * N_pre (the nominal in-degree), and reads the shared seeded
    weights and initial potentials."""
    import snn_inputs as I
    inst = spec["instance"] if instance is None else instance
    pops = []
    for k, d in enumerate(spec["pops"]):
        e = dict(d)
        v0 = I.v0(spec, k)
        e["v0"] = None if v0 is None else v0.astype(np.float64)
        pops.append(e)
    projs = []
    for q, d in enumerate(spec["projs"]):
        n_pre, n_post = I.n_pre_post(spec, q)
        e = dict(d)
        e["n_conn"] = d["p"] * n_pre
        if d["layout"] == "dense" and d["p"] >= 1.0:
            e["w"] = I.weights(spec, q, n_pre * n_post).astype(np.float64)
        else:
            rp, col = csr_bernoulli(spec["seed"], I.rng_tag(inst, q), n_pre, n_post, d["p"])
            w = I.weights(spec, q, len(col)).astype(np.float64)
            if d["layout"] == "dense":
                W = np.zeros((n_pre, n_post))
                rows = np.repeat(np.arange(n_pre), np.diff(rp))
                W[rows, col] = w
                e["w"] = W.ravel()
            else:
                e["row_ptr"], e["col"], e["w"] = rp, col, w
        projs.append(e)
    return OracleNet(pops, projs, spec["dt"], spec["n_sub"], spec["seed"], inst)
