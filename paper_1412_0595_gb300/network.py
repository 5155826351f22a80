"""Python layer over the C-ABI: device memory and streams come from PyTorch,
every step of the simulation runs in the CUDA library.

``Network``  -- a conductance-based HH network (Sec. 2) with compressed-row or
               dense projections (Sec. 3) scaled by gScale (Sec. 5.1).
``csr_bernoulli`` -- compressed rows drawn on the GPU from a seed.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L
from ._lib import check

_F32 = {"V", "m", "h", "n", "g0", "g1", "iext", "isyn"}


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream if hasattr(s, "cuda_stream") else int(s)


class TorchAllocator:
    """snn_allocator backed by PyTorch's caching allocator."""

    def __init__(self, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device).index

        def _alloc(nbytes, stream, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), self.device, int(stream or 0))
            except Exception:        # out of memory: the library reports SNN_ERR_OOM
                return None

        def _free(ptr, stream, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        self._a = L.ALLOC_FN(_alloc)
        self._f = L.FREE_FN(_free)
        self.struct = L.Allocator(self._a, self._f, None)

    def ref(self):
        return C.byref(self.struct)


def _dev(x, dtype, device):
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=dtype).contiguous()
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=device)


def csr_bernoulli(seed, tag, n_pre, n_post, p, device=None, stream=None):
    """Compressed rows (row_ptr int64[n_pre+1], col int32[nnz]) drawn on the
    GPU: post j is in row i when word j%4 of Philox4x32-10(counter=(j/4, i,
    tag, 3), key=seed) is below round(p * 2^32)."""
    device = torch.device("cuda") if device is None else torch.device(device)
    row_ptr = torch.empty(n_pre + 1, dtype=torch.int64, device=device)
    nnz = C.c_int64()
    alloc = TorchAllocator(device.index)
    s = _stream(stream)
    check(L.lib.snn_csr_bernoulli_rows(int(seed), int(tag), int(n_pre), int(n_post), float(p),
                                       row_ptr.data_ptr(), C.byref(nnz), alloc.ref(), s))
    col = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=device)
    check(L.lib.snn_csr_bernoulli_fill(int(seed), int(tag), int(n_pre), int(n_post), float(p),
                                       row_ptr.data_ptr(), col.data_ptr(), s))
    return row_ptr, col[:nnz.value]


def _descs(pops, projs, device, keep):
    """ctypes descriptor arrays for populations and projections (device copies
    of the arrays are appended to `keep` until the library has copied them)."""
    P = (L.PopDesc * len(pops))()
    for k, d in enumerate(pops):
        p = P[k]
        p.kind = {"source": L.POP_SOURCE, "hh": L.POP_HH, "izh": L.POP_IZH}[d["kind"]]
        p.n = int(d["n"])
        for f, v in (d.get("hh") or {}).items():
            setattr(p, f, float(v))
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
        if v0 is not None and p.kind != L.POP_SOURCE:
            t = _dev(v0, torch.float32, device)
            assert t.numel() == p.n
            keep.append(t)
            p.v0, p.v0_on_device = t.data_ptr(), 1
    Q = (L.ProjDesc * max(len(projs), 1))()
    for k, d in enumerate(projs):
        q = Q[k]
        q.pre, q.post = int(d["pre"]), int(d["post"])
        q.layout = L.LAYOUT_DENSE if d["layout"] == "dense" else L.LAYOUT_CSR
        q.channel = int(d.get("channel", 0))
        q.synapse = L.SYN_GRADED if d.get("synapse") == "graded" else L.SYN_EXP
        q.on_device = 1
        w = _dev(d["w"], torch.float32, device)
        keep.append(w)
        q.w = w.data_ptr()
        if d.get("row_ptr") is None:
            q.input_dense = 1
            q.nnz = w.numel()
        else:
            rp = _dev(d["row_ptr"], torch.int64, device)
            col = _dev(d["col"], torch.int32, device)
            keep += [rp, col]
            q.row_ptr, q.col, q.nnz = rp.data_ptr(), col.data_ptr(), col.numel()
        q.k1, q.k2, q.k3 = float(d.get("k1", 1.0)), float(d.get("k2", 0.0)), float(d.get("k3", 0.0))
        q.density = float(d.get("p", d.get("density", 1.0)))
        q.n_conn = float(d.get("n_conn", 0.0) or 0.0)
        q.user_scale = float(d.get("user_scale", 1.0))
        q.v_thr = float(d.get("v_thr", -20.0))
        q.v_slope = float(d.get("v_slope", 2.0))
    return P, Q


def _spec_arrays(spec, device, stream, inst):
    """Population and projection dicts of a ``snn_inputs`` description with
    device arrays: connectivity drawn on the GPU, seeded weights and V0."""
    import snn_inputs as I
    pops = []
    for k, d in enumerate(spec["pops"]):
        e = dict(d)
        v0 = I.v0(spec, k)
        if v0 is not None:
            e["v0"] = torch.from_numpy(v0).to(device)
        pops.append(e)
    projs = []
    for q, d in enumerate(spec["projs"]):
        n_pre, n_post = I.n_pre_post(spec, q)
        e = dict(d)
        if d["layout"] == "dense" and d["p"] >= 1.0:
            e["w"] = torch.from_numpy(I.weights(spec, q, n_pre * n_post)).to(device)
            e["row_ptr"] = None
        else:
            rp, col = csr_bernoulli(spec["seed"], I.rng_tag(inst, q), n_pre, n_post, d["p"], device, stream)
            e["row_ptr"], e["col"] = rp, col
            e["w"] = torch.from_numpy(I.weights(spec, q, col.numel())).to(device)
        projs.append(e)
    return pops, projs


class Network:
    """An HH spiking network living on one GPU.

    pops:  list of dicts (keys of ``snn_inputs.hh_pop`` / ``source_pop``), with
           optional ``v0`` (array or tensor of n FP32 potentials).
    projs: list of dicts with pre, post, layout ('csr' | 'dense'), channel,
           k1, k2, k3, density (p), optional n_conn, user_scale, and either
           row_ptr/col/w (compressed rows) or w of n_pre*n_post (dense input).
    """

    def __init__(self, pops, projs, dt, n_sub=4, seed=0, instance=0, device=None, stream=None,
                 torch_alloc=True):
        self._setup(device, torch_alloc)
        self.sizes = [int(d["n"]) for d in pops]
        self.n_projs = len(projs)
        keep = []
        P, Q = _descs(pops, projs, self.device, keep)
        h = C.c_void_p()
        torch.cuda.synchronize(self.device)
        check(L.lib.snn_create_network(P, len(pops), Q, len(projs), float(dt), int(n_sub), int(seed),
                                       int(instance), self._alloc.ref() if self._alloc else None,
                                       _stream(stream), C.byref(h)))
        self.h = h.value
        self.dt = float(dt)
        self.pop_offsets = [0]

    def _setup(self, device, torch_alloc):
        self.device = torch.device("cuda") if device is None else torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self._alloc = TorchAllocator(self.device.index) if torch_alloc else None

    @classmethod
    def batch(cls, instances, dt, n_sub=4, seed=0, device=None, stream=None, torch_alloc=True):
        """Many independent networks in one object (snn_create_batch).
        ``instances``: list of (pops, projs, rng_instance).  Population k of
        instance b is population ``pop_offsets[b] + k`` of the batch."""
        self = cls.__new__(cls)
        self._setup(device, torch_alloc)
        keep, descs, self.sizes, self.pop_offsets = [], [], [], []
        D = (L.NetDesc * len(instances))()
        n_projs = 0
        for b, (pops, projs, inst) in enumerate(instances):
            P, Q = _descs(pops, projs, self.device, keep)
            keep += [P, Q]
            self.pop_offsets.append(len(self.sizes))
            self.sizes += [int(d["n"]) for d in pops]
            D[b].pops, D[b].n_pops = C.cast(P, C.POINTER(L.PopDesc)), len(pops)
            D[b].projs, D[b].n_projs = C.cast(Q, C.POINTER(L.ProjDesc)), len(projs)
            D[b].rng_instance = int(inst)
            n_projs += len(projs)
        self.n_projs = n_projs
        h = C.c_void_p()
        torch.cuda.synchronize(self.device)
        check(L.lib.snn_create_batch(D, len(instances), float(dt), int(n_sub), int(seed),
                                     self._alloc.ref() if self._alloc else None, _stream(stream), C.byref(h)))
        self.h = h.value
        self.dt = float(dt)
        return self

    def add_shared_dense(self, pre, post, W, user_scale, *, channel=0, k=(1.0, 0.0, 0.0), density=1.0, n_conn=0.0,
                         pops_per_instance=None, stream=None):
        """A dense projection W (n_pre x n_post) that every instance of this
        batch shares (snn_add_shared_dense): instance b's population `post`
        (index within an instance) receives s_b W[i] for each spike i of its
        population `pre`, s_b = (k1 / (k2 + nConn) + k3) * user_scale[b]."""
        B = len(self.pop_offsets)
        ppi = pops_per_instance if pops_per_instance is not None else len(self.sizes) // B
        w = _dev(W, torch.float32, self.device)
        sc = (C.c_double * B)(*[float(x) for x in user_scale])
        check(L.lib.snn_add_shared_dense(self.h, int(pre), int(post), int(ppi), B, w.data_ptr(), 1, int(channel),
                                         float(k[0]), float(k[1]), float(k[2]), float(density), float(n_conn), sc,
                                         _stream(stream)))

    @classmethod
    def from_specs(cls, specs, device=None, stream=None, **kw):
        """Batch of ``snn_inputs`` descriptions (same dt, substeps and seed),
        each with its own instance number."""
        device = torch.device("cuda") if device is None else torch.device(device)
        s0 = specs[0]
        inst = []
        for spec in specs:
            assert spec["dt"] == s0["dt"] and spec["n_sub"] == s0["n_sub"] and spec["seed"] == s0["seed"]
            pops, projs = _spec_arrays(spec, device, stream, spec["instance"])
            inst.append((pops, projs, spec["instance"]))
        return cls.batch(inst, s0["dt"], s0["n_sub"], s0["seed"], device=device, stream=stream, **kw)

    # ------------------------------------------------------------------ build
    @classmethod
    def from_spec(cls, spec, device=None, stream=None, instance=None, **kw):
        """Builds the network of a ``snn_inputs`` description: connectivity is
        drawn on the GPU from the seed, weights and initial potentials are the
        shared seeded arrays, nConn = p * N_pre inside the library."""
        inst = spec["instance"] if instance is None else instance
        device = torch.device("cuda") if device is None else torch.device(device)
        pops, projs = _spec_arrays(spec, device, stream, inst)
        return cls(pops, projs, spec["dt"], spec["n_sub"], spec["seed"], inst, device=device, stream=stream, **kw)

    # ------------------------------------------------------------------ run
    def close(self):
        if getattr(self, "h", None):
            L.lib.snn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1, stream=None):
        check(L.lib.snn_step(self.h, int(n), _stream(stream)))

    def sync(self, stream=None):
        check(L.lib.snn_sync(self.h, _stream(stream)))

    def reset(self, stream=None):
        check(L.lib.snn_reset(self.h, _stream(stream)))

    def set_option(self, name, value):
        check(L.lib.snn_set_option(self.h, L.OPT[name], int(value)))

    def get_option(self, name):
        v = C.c_int64(0)
        check(L.lib.snn_get_option(self.h, L.OPT[name], C.byref(v)))
        return int(v.value)

    @property
    def cluster_size(self):
        """CTAs (SMs) of the cluster engine's plan; 0 if the network does not fit one cluster."""
        return self.get_option("cluster_ctas")

    @property
    def engine(self):
        """Engine snn_step uses: 'plain', 'persistent' or 'cluster'."""
        v = C.c_int32()
        check(L.lib.snn_get_engine(self.h, C.byref(v)))
        return {0: "plain", 1: "persistent", 3: "cluster"}[v.value]

    @property
    def t(self):
        v = C.c_int64()
        check(L.lib.snn_get_step(self.h, C.byref(v), _stream(None)))
        return v.value

    def scale(self, q):
        v = C.c_float()
        check(L.lib.snn_proj_scale(self.h, int(q), C.byref(v)))
        return v.value

    def nnz(self, q):
        v = C.c_int64()
        check(L.lib.snn_proj_nnz(self.h, int(q), C.byref(v)))
        return v.value

    def proj_mode(self, q):
        """Propagation kernel of projection q: 0 rows (k_propagate), 1 pieces
        (k_propagate_tiled), 2 segments (k_propagate_seg)."""
        v = C.c_int32()
        check(L.lib.snn_proj_mode(self.h, int(q), C.byref(v)))
        return v.value

    # ------------------------------------------------------------------ state
    def read(self, pop, field, stream=None) -> torch.Tensor:
        """A field of population `pop` as a device tensor (copied)."""
        s = _stream(stream)
        fid = L.FIELD[field]
        if field in _F32:
            out = torch.empty(self.sizes[pop], dtype=torch.float32, device=self.device)
            nbytes = 4 * out.numel()
        elif field in ("spikes", "neuron_spikes"):
            out = torch.empty(max(self.sizes[pop], 1), dtype=torch.int32, device=self.device)
            nbytes = 4 * out.numel()
        elif field == "nspk":
            out = torch.empty(1, dtype=torch.int32, device=self.device)
            nbytes = 4
        else:
            out = torch.empty(1, dtype=torch.int64, device=self.device)
            nbytes = 8
        check(L.lib.snn_read_state(self.h, int(pop), fid, out.data_ptr(), nbytes, 1, s))
        if field == "neuron_spikes":
            return out[: self.sizes[pop]]
        if field == "spikes":
            return out[: int(self.read(pop, "nspk", stream).item())]
        return out

    def read_host(self, pop, field):
        """Same as read() but through a host buffer (numpy)."""
        s = _stream(None)
        if field in _F32:
            out = np.empty(self.sizes[pop], dtype=np.float32)
        elif field == "nspk":
            out = np.empty(1, dtype=np.int32)
        elif field in ("spike_count", "nan_count"):
            out = np.empty(1, dtype=np.int64)
        else:
            out = np.empty(max(self.sizes[pop], 1), dtype=np.int32)
        check(L.lib.snn_read_state(self.h, int(pop), L.FIELD[field], out.ctypes.data, out.nbytes, 0, s))
        if field == "spikes":
            return out[: int(self.read_host(pop, "nspk")[0])]
        return out

    def write(self, pop, field, values, stream=None):
        t = _dev(values, torch.float32, self.device)
        assert t.numel() == self.sizes[pop]
        check(L.lib.snn_write_state(self.h, int(pop), L.FIELD[field], t.data_ptr(), 4 * t.numel(), 1,
                                    _stream(stream)))

    def synaptic_events(self, stream=None):
        v = C.c_int64()
        check(L.lib.snn_synaptic_events(self.h, C.byref(v), _stream(stream)))
        return v.value

    def launch_phase(self, phase, stream=None):
        check(L.lib.snn_launch_phase(self.h, int(phase), _stream(stream)))

    def counters(self, pop):
        return int(self.read(pop, "spike_count").item()), int(self.read(pop, "nan_count").item())

    # ------------------------------------------------------------------ checkpoints, tuning
    def save_state(self, stream=None) -> torch.Tensor:
        """Snapshot of the whole dynamic state as a device byte tensor."""
        n = C.c_size_t()
        check(L.lib.snn_state_size(self.h, C.byref(n)))
        buf = torch.empty(n.value, dtype=torch.uint8, device=self.device)
        check(L.lib.snn_save_state(self.h, buf.data_ptr(), n.value, 1, _stream(stream)))
        return buf

    def load_state(self, buf, stream=None):
        if buf.is_cuda:
            check(L.lib.snn_load_state(self.h, buf.data_ptr(), buf.numel(), 1, _stream(stream)))
        else:
            b = buf.contiguous()
            check(L.lib.snn_load_state(self.h, b.data_ptr(), b.numel(), 0, _stream(stream)))

    @staticmethod
    def _tuning(r):
        return {"engine": {0: "plain", 1: "persistent", 3: "cluster"}[r.engine], "prop_blocks": r.prop_blocks,
                "chunk": r.chunk, "tiled": r.tiled, "us_per_step": r.us_per_step, "cached": bool(r.cached)}

    def autotune(self, trial_steps=200, stream=None):
        r = L.Tuning()
        check(L.lib.snn_autotune(self.h, int(trial_steps), C.byref(r), _stream(stream)))
        return self._tuning(r)

    def occupancy_config(self, trial_steps=200, stream=None):
        """The paper's occupancy-based configuration (Sec. 3), applied and timed."""
        r = L.Tuning()
        check(L.lib.snn_occupancy_config(self.h, int(trial_steps), C.byref(r), _stream(stream)))
        return self._tuning(r)

    # ------------------------------------------------------------------ checks
    def debug_propagate(self, q, spk, stream=None):
        t = _dev(spk, torch.int32, self.device)
        check(L.lib.snn_debug_propagate(self.h, int(q), t.data_ptr() if t.numel() else None, t.numel(), 1,
                                        _stream(stream)))

    def event_list(self, q, spk, stream=None):
        t = _dev(spk, torch.int32, self.device)
        n = C.c_int64()
        s = _stream(stream)
        st = L.lib.snn_event_list(self.h, int(q), t.data_ptr() if t.numel() else None, t.numel(), 1, None, None, 0,
                                  C.byref(n), s)
        if st not in (L.SNN_OK, 8):
            check(st)
        post = torch.empty(max(n.value, 1), dtype=torch.int32, device=self.device)
        w = torch.empty(max(n.value, 1), dtype=torch.float32, device=self.device)
        check(L.lib.snn_event_list(self.h, int(q), t.data_ptr() if t.numel() else None, t.numel(), 1,
                                   post.data_ptr(), w.data_ptr(), n.value, C.byref(n), s))
        return post[: n.value], w[: n.value]


class GradedNetwork(Network):
    """A network whose projections are all graded (the differentiable form):
    recorded forward with checkpoints and the discrete adjoint."""

    def set_scale(self, q, scale):
        check(L.lib.snn_set_scale(self.h, int(q), float(scale)))

    def set_weights(self, q, w, stream=None):
        t = _dev(w, torch.float32, self.device)
        assert t.numel() == self.nnz(q)
        check(L.lib.snn_set_weights(self.h, int(q), t.data_ptr(), 1, _stream(stream)))

    def launch_product(self, stream=None):
        """Enqueues the forward product alone (timing; the state does not advance)."""
        check(L.lib.snn_graded_launch_product(self.h, _stream(stream)))

    def forward_record(self, n_steps, out_pop=None, tau_f=5.0, checkpoint_every=100, stream=None):
        """Recorded run of n_steps from the creation state; returns the output
        filter y as a (n_steps, n_out) device tensor (y[t] = y(t + 1))."""
        out_pop = len(self.sizes) - 1 if out_pop is None else int(out_pop)
        y = torch.empty((int(n_steps), self.sizes[out_pop]), dtype=torch.float32, device=self.device)
        check(L.lib.snn_forward_record(self.h, int(n_steps), int(checkpoint_every), out_pop, float(tau_f),
                                       y.data_ptr(), _stream(stream)))
        return y

    def backward(self, dL_dy, stream=None):
        """(dL/ds per projection, [dL/dw per projection, compressed-row order])
        of a loss of the last recorded y, given dL/dy in y's layout."""
        g = _dev(dL_dy, torch.float32, self.device)
        gs = torch.empty(self.n_projs, dtype=torch.float32, device=self.device)
        gw = [torch.empty(max(self.nnz(q), 1), dtype=torch.float32, device=self.device) for q in range(self.n_projs)]
        ptrs = (C.c_void_p * max(1, self.n_projs))(*[t.data_ptr() for t in gw])
        check(L.lib.snn_backward(self.h, g.data_ptr(), gs.data_ptr(), ptrs, _stream(stream)))
        return gs, [x[: self.nnz(q)] for q, x in enumerate(gw)]


def squared_error(y, target):
    """Mean squared error of y against target and its gradient dL/dy (a loss
    on top of the network's output; computed in torch, outside the library)."""
    t = target.to(device=y.device, dtype=y.dtype)
    d = y - t
    return (d.double() ** 2).mean().item(), (2.0 / d.numel()) * d


class SNNFunction(torch.autograd.Function):
    """y(scales, weights) of a graded network as an autograd node.

    forward(net, n_steps, out_pop, tau_f, checkpoint_every, scales, *weights):
    sets every projection's scale s_q and weights, runs the recorded forward
    and returns the output filter y (n_steps x n_out); backward takes dL/dy
    from whatever loss or torch graph sits on top and returns dL/ds and dL/dw
    from the network's discrete adjoint.  The network holds one recorded run:
    call backward before the next forward on the same network."""

    @staticmethod
    def forward(ctx, net, n_steps, out_pop, tau_f, checkpoint_every, scales, *weights):
        for q in range(net.n_projs):
            net.set_scale(q, float(scales[q]))
            net.set_weights(q, weights[q].detach())
        y = net.forward_record(n_steps, out_pop, tau_f, checkpoint_every)
        ctx.net = net
        ctx.scale_dtype = scales.dtype
        return y

    @staticmethod
    def backward(ctx, grad_y):
        gs, gw = ctx.net.backward(grad_y.contiguous())
        return (None, None, None, None, None, gs.to(ctx.scale_dtype), *gw)


class DenseBatch:
    """A dense projection W (n_pre x n_post) shared by many network instances,
    delivered for all of them at once (``snn_dense_batch_*``): engine
    "tensor" multiplies the step's 0/1 spike matrix with W on the tensor cores
    (W split into three BF16 parts, FP32 accumulation), engine "cuda" sums the
    spike rows on the CUDA cores."""

    ENGINES = {"cuda": 0, "tensor": 1}

    def __init__(self, W, device=None, stream=None):
        self.device = torch.device("cuda") if device is None else torch.device(device)
        w = _dev(W, torch.float32, self.device)
        assert w.dim() == 2
        self.n_pre, self.n_post = int(w.shape[0]), int(w.shape[1])
        self._alloc = TorchAllocator(self.device.index)
        h = C.c_void_p()
        check(L.lib.snn_dense_batch_create(w.data_ptr(), self.n_pre, self.n_post, 1, self._alloc.ref(),
                                           _stream(stream), C.byref(h)))
        self.h = h

    def deliver(self, spikes, scale, G, engine="tensor", stream=None):
        """G[b] += scale[b] * W[spikes[b]].sum(0) for every instance b; `spikes`
        is a list of index arrays (or (offsets, indices) tensors), G a CUDA
        tensor of shape (B, >= n_post) whose rows are contiguous."""
        if isinstance(spikes, tuple):
            off, idx = spikes
        else:
            lens = [len(s) for s in spikes]
            off = torch.tensor(np.concatenate([[0], np.cumsum(lens)]), dtype=torch.int32)
            idx = torch.tensor(np.concatenate([np.asarray(s, np.int64) for s in spikes]) if sum(lens) else [0],
                               dtype=torch.int32)
        off = off.to(self.device, torch.int32).contiguous()
        idx = idx.to(self.device, torch.int32).contiguous()
        sc = _dev(scale, torch.float32, self.device)
        assert G.is_cuda and G.dtype == torch.float32 and G.stride(1) == 1
        check(L.lib.snn_dense_batch_deliver(self.h, int(G.shape[0]), off.data_ptr(), idx.data_ptr(), sc.data_ptr(),
                                            G.data_ptr(), int(G.stride(0)), self.ENGINES[engine], _stream(stream)))
        self._keep = (off, idx, sc)

    def check(self, stream=None):
        check(L.lib.snn_dense_batch_check(self.h, _stream(stream)))

    def close(self):
        if getattr(self, "h", None):
            L.lib.snn_dense_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DenseGrad:
    """Rank-K update D += R^T N (``snn_dense_grad_*``): the weight gradient of
    a dense graded projection over a checkpoint segment, R (K x m, step-major)
    the releases and N (n x K, time-contiguous) dL/dG.  Engine "tensor": three
    BF16 parts per operand, six tensor-core products, FP32 accumulation;
    engine "cuda": FP32 products on the CUDA cores."""

    ENGINES = {"cuda": 0, "tensor": 1}

    def __init__(self, device=None, stream=None):
        self.device = torch.device("cuda") if device is None else torch.device(device)
        self._alloc = TorchAllocator(self.device.index)
        h = C.c_void_p()
        check(L.lib.snn_dense_grad_create(self._alloc.ref(), _stream(stream), C.byref(h)))
        self.h = h

    def run(self, R, N, D, engine="tensor", stream=None):
        """D[i, j] += sum_t R[t, i] N[j, t]; CUDA FP32 tensors with unit
        stride in their last dimension."""
        for t in (R, N, D):
            assert t.is_cuda and t.dtype == torch.float32 and t.dim() == 2 and t.stride(1) == 1
        K, m = R.shape
        n = N.shape[0]
        assert N.shape[1] == K and tuple(D.shape) == (m, n)
        check(L.lib.snn_dense_grad_run(self.h, R.data_ptr(), int(R.stride(0)), N.data_ptr(), int(N.stride(0)), m, n, K,
                                       D.data_ptr(), int(D.stride(0)), self.ENGINES[engine], _stream(stream)))

    def check(self, stream=None):
        check(L.lib.snn_dense_grad_check(self.h, _stream(stream)))

    def close(self):
        if getattr(self, "h", None):
            L.lib.snn_dense_grad_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
