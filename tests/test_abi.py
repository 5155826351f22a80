"""The C-ABI library loads on a machine without a GPU, exports every entry
point that include/snn.h declares, and rejects bad descriptions on the host
before touching the device (no compute calls here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(snn_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    import paper_1412_0595_gb300 as snn
    names = _declared()
    assert {"snn_create_network", "snn_step", "snn_read_state", "snn_destroy"} <= names
    missing = [n for n in sorted(names) if not hasattr(snn.lib, n)]
    assert not missing, missing


def _pop(kind=0, n=10):
    from paper_1412_0595_gb300 import _lib as L
    p = L.PopDesc()
    p.kind, p.n = kind, n
    p.C, p.gNa, p.ENa, p.gK, p.EK, p.gL, p.EL = 143.0, 7150.0, 50.0, 1430.0, -95.0, 26.72, -63.563
    p.tau_syn[0] = p.tau_syn[1] = 1.0
    return p


def _create(pops, projs, dt=0.1, n_sub=4):
    from paper_1412_0595_gb300 import _lib as L
    P = (L.PopDesc * len(pops))(*pops)
    Q = (L.ProjDesc * max(1, len(projs)))(*projs) if projs else None
    h = C.c_void_p()
    st = L.lib.snn_create_network(P, len(pops), Q, len(projs), dt, n_sub, 1, 0, None, None, C.byref(h))
    return st, L.lib.snn_last_error().decode()


@pytest.mark.parametrize("dt,n_sub", [(0.0, 4), (-0.1, 4), (float("nan"), 4), (0.1, 0)])
def test_bad_time_step_is_rejected_on_the_host(dt, n_sub):
    st, msg = _create([_pop()], [], dt=dt, n_sub=n_sub)
    assert st == 1 and msg


def test_scaling_law_pole_is_rejected():
    from paper_1412_0595_gb300 import _lib as L
    q = L.ProjDesc()
    q.pre, q.post, q.layout, q.nnz = 0, 1, L.LAYOUT_CSR, 0
    rp = (C.c_int64 * 11)()
    q.row_ptr = C.cast(rp, C.c_void_p)
    # PN-LHI constants of Table 2 at nConn = 6: nConn + k2 = -0.338 <= 0
    q.k1, q.k2, q.k3, q.n_conn, q.user_scale = 1.354e3, -6.338, 1.672e-3, 6.0, 1.0
    st, msg = _create([_pop(1, 10), _pop(0, 10)], [q])
    assert st == 3 and "gScale" in msg


def test_bad_descriptions_are_rejected():
    from paper_1412_0595_gb300 import _lib as L
    assert _create([_pop(kind=7)], [])[0] == 1
    assert _create([_pop(n=-1)], [])[0] == 1
    q = L.ProjDesc()
    q.pre, q.post = 0, 5                      # post out of range
    assert _create([_pop()], [q])[0] == 1
    q = L.ProjDesc()
    q.pre, q.post, q.k1, q.density = 0, 0, 1.0, 1.0
    q.channel = 2                             # no such channel
    assert _create([_pop()], [q])[0] == 1
    q = L.ProjDesc()
    q.pre, q.post, q.k1, q.density = 1, 0, 1.0, 1.0   # post is a source population
    assert _create([_pop(), _pop(kind=1)], [q])[0] == 1
