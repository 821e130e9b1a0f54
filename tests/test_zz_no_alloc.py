"""kpme_spread_noalloc: the allocation-free spreading entry point, for callers that may
not call cudaMalloc (stream capture, foreign pool allocators, latency-critical loops).

Checked through the C ABI against the plan-based kpme_spread (float32 mesh) and against the
oracle's spreading on two calls in a row with different inputs, so that a stale static
scratch array would show up.
Kept in a file collected last: it shares one static device array for the whole process.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import spme
from paper_2601_18838_gb300 import workloads as wl
from tests._gpu_util import cuda_or_skip, dev, host

pytestmark = pytest.mark.gpu

TOL = 2e-6   # same bar as the float32 spreading parity test (relative to max |Q|)


def _params(L, s):
    from paper_2601_18838_gb300._binding import Params
    p = Params()
    L.kpme_default_params(C.byref(p))
    p.center = (C.c_double * 3)(*s.center)
    p.radius = s.radius
    p.order = s.order
    p.K = s.K
    p.precision = 1   # float32 mesh, like the no-alloc path
    p.max_n = s.n
    return p


def _noalloc(torch, L, s, stream):
    p = _params(L, s)
    x, q = dev(torch, s.x), dev(torch, s.q)
    Q = torch.full((s.K,) * 3, float("nan"), dtype=torch.float64, device="cuda:0")
    st = L.kpme_spread_noalloc(C.byref(p), C.c_void_p(stream.cuda_stream), C.c_int64(s.n),
                               C.c_void_p(x.data_ptr()), C.c_void_p(q.data_ptr()), C.c_void_p(Q.data_ptr()))
    assert st == 0, L.kpme_status_string(st)
    torch.cuda.synchronize()
    return host(Q)


def _with_plan(torch, L, s, stream):
    p = _params(L, s)
    h = C.c_void_p()
    assert L.kpme_plan(C.byref(p), C.c_void_p(stream.cuda_stream), C.byref(h)) == 0
    try:
        x, q = dev(torch, s.x), dev(torch, s.q)
        Q = torch.empty((s.K,) * 3, dtype=torch.float64, device="cuda:0")
        assert L.kpme_spread(h, C.c_int64(s.n), C.c_void_p(x.data_ptr()), C.c_void_p(q.data_ptr()),
                             C.c_void_p(Q.data_ptr())) == 0
        torch.cuda.synchronize()
        return host(Q)
    finally:
        L.kpme_destroy(h)


def test_noalloc_spread_matches_plan_spread_twice():
    torch = cuda_or_skip()
    import __graft_entry__ as g
    g.build()
    from paper_2601_18838_gb300._binding import lib
    L = lib()
    stream = torch.cuda.current_stream()
    systems = [wl.random_system(1999, 21.0, 64, 6, seed=101), wl.random_system(777, 13.0, 32, 4, seed=202)]
    for s in systems:   # two calls in a row; the second uses a smaller mesh than the first
        a = _noalloc(torch, L, s, stream)
        b = _with_plan(torch, L, s, stream)
        ref = spme.spread(s.x, s.q, s.box, s.K, s.order)
        assert np.all(np.isfinite(a))
        assert np.abs(a - b).max() <= TOL * np.abs(b).max()
        assert np.abs(a - ref).max() <= TOL * np.abs(ref).max()
        assert abs(a.sum() - s.q.sum()) < 1e-4


def test_noalloc_rejects_mesh_above_limit():
    torch = cuda_or_skip()
    from paper_2601_18838_gb300._binding import lib
    L = lib()
    s = wl.random_system(16, 30.0, 96, 4, seed=3)
    p = _params(L, s)
    x, q = dev(torch, s.x), dev(torch, s.q)
    Q = torch.empty((96,) * 3, dtype=torch.float64, device="cuda:0")
    st = L.kpme_spread_noalloc(C.byref(p), C.c_void_p(torch.cuda.current_stream().cuda_stream), C.c_int64(s.n),
                               C.c_void_p(x.data_ptr()), C.c_void_p(q.data_ptr()), C.c_void_p(Q.data_ptr()))
    assert st == 5   # KPME_ERR_CAPACITY: K above KPME_NOALLOC_MAX_K
