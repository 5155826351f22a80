"""ctypes shim of the FP64 graded-synapse oracle and its discrete adjoint
(test infrastructure only; see snn_oracle_graded.c)."""
from __future__ import annotations

import ctypes as C

import numpy as np


class OracleGPop(C.Structure):
    _fields_ = [("n", C.c_int32), ("C", C.c_double), ("gNa", C.c_double), ("ENa", C.c_double),
                ("gK", C.c_double), ("EK", C.c_double), ("gL", C.c_double), ("EL", C.c_double),
                ("E_syn", C.c_double * 2), ("drive_rate_hz", C.c_double), ("drive_amp", C.c_double),
                ("drive_tau", C.c_double), ("v0", C.POINTER(C.c_double))]


class OracleGProj(C.Structure):
    _fields_ = [("pre", C.c_int32), ("post", C.c_int32), ("channel", C.c_int32), ("nnz", C.c_int64),
                ("row_ptr", C.POINTER(C.c_int64)), ("col", C.POINTER(C.c_int32)), ("w", C.POINTER(C.c_double)),
                ("k1", C.c_double), ("k2", C.c_double), ("k3", C.c_double), ("n_conn", C.c_double),
                ("user_scale", C.c_double), ("v_thr", C.c_double), ("v_slope", C.c_double)]


def _bind(L):
    f64p, i64p = C.POINTER(C.c_double), C.POINTER(C.c_int64)
    L.oracle_graded_create.argtypes = [C.POINTER(OracleGPop), C.c_int, C.POINTER(OracleGProj), C.c_int, C.c_double,
                                       C.c_int, C.c_uint64, C.c_uint32, C.c_int, C.c_double]
    L.oracle_graded_create.restype = C.c_void_p
    L.oracle_graded_destroy.argtypes = [C.c_void_p]
    L.oracle_graded_forward.argtypes = [C.c_void_p, C.c_int, f64p, f64p]
    L.oracle_graded_forward.restype = C.c_double
    L.oracle_graded_backward.argtypes = [C.c_void_p, f64p, C.POINTER(f64p)]
    L.oracle_graded_backward.restype = C.c_int
    L.oracle_graded_backward_dy.argtypes = [C.c_void_p, f64p, f64p, C.POINTER(f64p)]
    L.oracle_graded_backward_dy.restype = C.c_int
    L.oracle_graded_get_scale.argtypes = [C.c_void_p, C.c_int]
    L.oracle_graded_get_scale.restype = C.c_double
    L.oracle_graded_set_scale.argtypes = [C.c_void_p, C.c_int, C.c_double]
    L.oracle_graded_set_weight.argtypes = [C.c_void_p, C.c_int, C.c_int64, C.c_double]
    L.oracle_graded_get_weight.argtypes = [C.c_void_p, C.c_int, C.c_int64]
    L.oracle_graded_get_weight.restype = C.c_double
    L.oracle_hh_rate_derivs.argtypes = [C.c_double, f64p]
    del i64p


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def hh_rate_derivs(V):
    from . import lib
    out = np.zeros(6)
    lib().oracle_hh_rate_derivs(float(V), _p(out, C.c_double))
    return out


class GradedOracle:
    """FP64 graded-synapse network: forward(T, target) -> loss, backward() ->
    (dL/ds per projection, [dL/dw per projection in compressed-row order;
    row-major n_pre x n_post for a dense projection])."""

    def __init__(self, spec, out_pop=None, tau_f=None, instance=None):
        import snn_inputs as I

        from . import csr_bernoulli, lib
        L = lib()
        inst = spec["instance"] if instance is None else instance
        self.spec = spec
        self.out_pop = len(spec["pops"]) - 1 if out_pop is None else out_pop
        tau_f = I.GRADED["tau_filter"] if tau_f is None else tau_f
        keep = []
        P = (OracleGPop * len(spec["pops"]))()
        for k, d in enumerate(spec["pops"]):
            p = P[k]
            p.n = d["n"]
            for f in ("C", "gNa", "ENa", "gK", "EK", "gL", "EL"):
                setattr(p, f, float(d["hh"][f]))
            p.E_syn[0], p.E_syn[1] = d["E_syn"]
            drv = d.get("drive") or {}
            p.drive_rate_hz, p.drive_amp, p.drive_tau = (float(drv.get("rate_hz", 0.0)), float(drv.get("amp", 0.0)),
                                                         float(drv.get("tau", 0.0)))
            v0 = I.v0(spec, k).astype(np.float64)
            keep.append(v0)
            p.v0 = _p(v0, C.c_double)
        Q = (OracleGProj * max(1, len(spec["projs"])))()
        self.rows = []
        for q, d in enumerate(spec["projs"]):
            n_pre, n_post = I.n_pre_post(spec, q)
            if d["layout"] == "dense":
                # Eq. 2 storage: every (pre, post) pair is a weight, in row-major
                # order (absent synapses of a thinned matrix are zeros); written
                # as compressed rows that hold all pairs
                if d["p"] >= 1.0:
                    W = I.weights(spec, q, n_pre * n_post).astype(np.float64)
                else:
                    rp, col = csr_bernoulli(spec["seed"], I.rng_tag(inst, q), n_pre, n_post, d["p"])
                    Wm = np.zeros((n_pre, n_post))
                    Wm[np.repeat(np.arange(n_pre), np.diff(rp)), col] = I.weights(spec, q, len(col))
                    W = Wm.ravel()
                rp = np.arange(n_pre + 1, dtype=np.int64) * n_post
                col = np.tile(np.arange(n_post, dtype=np.int32), n_pre)
                w = np.ascontiguousarray(W, dtype=np.float64)
            else:
                rp, col = csr_bernoulli(spec["seed"], I.rng_tag(inst, q), n_pre, n_post, d["p"])
                w = I.weights(spec, q, len(col)).astype(np.float64)
            keep += [rp, col, w]
            self.rows.append((rp, col, w))
            x = Q[q]
            x.pre, x.post, x.channel, x.nnz = d["pre"], d["post"], d.get("channel", 0), len(col)
            x.row_ptr, x.col, x.w = _p(rp, C.c_int64), _p(col, C.c_int32), _p(w, C.c_double)
            x.k1, x.k2, x.k3 = d["k1"], d["k2"], d["k3"]
            x.n_conn = d["p"] * n_pre
            x.user_scale = d.get("user_scale", 1.0)
            x.v_thr = d.get("v_thr", I.GRADED["v_thr"])
            x.v_slope = d.get("v_slope", I.GRADED["v_slope"])
        h = L.oracle_graded_create(P, len(spec["pops"]), Q, len(spec["projs"]), spec["dt"], spec["n_sub"],
                                   spec["seed"], inst, self.out_pop, float(tau_f))
        if not h:
            raise ValueError("oracle rejected the graded network")
        self.h = h
        self.n_out = spec["pops"][self.out_pop]["n"]
        self.nnz = [len(r[1]) for r in self.rows]

    def __del__(self):
        try:
            from . import lib
            if getattr(self, "h", None):
                lib().oracle_graded_destroy(self.h)
                self.h = None
        except ImportError:        # interpreter shutdown: the process frees everything
            pass

    def forward(self, target):
        from . import lib
        target = np.ascontiguousarray(target, dtype=np.float64)
        T = target.shape[0]
        y = np.zeros((T, self.n_out))
        loss = lib().oracle_graded_forward(self.h, T, _p(target, C.c_double), _p(y, C.c_double))
        return loss, y

    def backward(self, dL_dy=None):
        """Gradients of the forward pass's squared-error loss, or, with
        dL_dy (T x n_out, dL/dy of the filter values the forward returned),
        of any loss of y."""
        from . import lib
        gs = np.zeros(len(self.nnz))
        gw = [np.zeros(max(n, 1)) for n in self.nnz]
        arr = (C.POINTER(C.c_double) * max(1, len(gw)))(*[_p(a, C.c_double) for a in gw])
        if dL_dy is None:
            rc = lib().oracle_graded_backward(self.h, _p(gs, C.c_double), arr)
        else:
            d = np.ascontiguousarray(dL_dy, dtype=np.float64)
            assert d.ndim == 2 and d.shape[1] == self.n_out
            rc = lib().oracle_graded_backward_dy(self.h, _p(d, C.c_double), _p(gs, C.c_double), arr)
        if rc != 0:
            raise RuntimeError("no recorded forward")
        return gs, [a[:n] for a, n in zip(gw, self.nnz)]

    def scale(self, q):
        from . import lib
        return lib().oracle_graded_get_scale(self.h, q)

    def set_scale(self, q, s):
        from . import lib
        lib().oracle_graded_set_scale(self.h, q, float(s))

    def weight(self, q, k):
        from . import lib
        return lib().oracle_graded_get_weight(self.h, q, int(k))

    def set_weight(self, q, k, w):
        from . import lib
        lib().oracle_graded_set_weight(self.h, q, int(k), float(w))
