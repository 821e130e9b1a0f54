"""CPU-side checks of the C ABI: the library loads, exports every declared entry point,
validates arguments before touching a GPU, and the host-side math it relies on holds."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "kpme.h")) as fh:
        txt = fh.read()
    return sorted(set(re.findall(r"\b(kpme_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    from paper_2601_18838_gb300 import _binding
    return _binding.lib()


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(L, n), n
    from paper_2601_18838_gb300 import EXPORTS
    assert sorted(EXPORTS) == names


def test_defaults_and_status_strings(L):
    from paper_2601_18838_gb300._binding import Params
    p = Params()
    assert L.kpme_default_params(C.byref(p)) == 0
    assert p.K == 32 and p.order == 4 and abs(p.beta - 0.35) < 1e-15
    assert L.kpme_default_params(None) == 1
    assert L.kpme_status_string(0) == b"ok"
    assert b"capacity" in L.kpme_status_string(5)


@pytest.mark.parametrize("field,value", [("radius", 0.0), ("beta", -1.0), ("order", 5), ("K", 31),
                                         ("K", 6), ("precision", 9), ("max_n", -1), ("skp_tol", -1e-3)])
def test_plan_rejects_invalid_parameters_without_gpu(L, field, value):
    from paper_2601_18838_gb300._binding import Params
    p = Params()
    L.kpme_default_params(C.byref(p))
    p.radius = 10.0
    setattr(p, field, value)
    h = C.c_void_p()
    assert L.kpme_plan(C.byref(p), None, C.byref(h)) == 1   # KPME_ERR_INVALID_ARG
    assert not h.value


@pytest.mark.parametrize("K,order,n", [(15, 6, 1000), (34, 6, 1000), (32, 5, 1000), (32, 6, 0)])
def test_update_rate_rejects_invalid_arguments_without_gpu(L, K, order, n):
    g = C.c_double(-1.0)
    assert L.kpme_measure_update_rate(K, order, n, C.byref(g), None, None) == 1   # KPME_ERR_INVALID_ARG
    assert g.value == -1.0


def test_skp_file_calls_reject_null_arguments_without_gpu(L):
    assert L.kpme_save_skp(None, b"/tmp/x.bin") == 1   # KPME_ERR_INVALID_ARG
    assert L.kpme_load_skp(None, b"/tmp/x.bin") == 1


def test_null_plan_is_rejected(L):
    assert L.kpme_energy_forces(None, 0, None, None, None, None, None, None) == 1
    assert L.kpme_set_profiling(None, 1) == 1
    L.kpme_destroy(None)


def test_weighted_half_range_svd_equals_full_grid():
    # The GPU build decomposes T on [0, K/2]^3 weighted by sqrt(w_m) per axis; its singular
    # values must be those of the full-grid matricisation the paper decomposes.
    from oracle import spme
    K = 12
    T = spme.influence(K, 4, 9.0, 0.4)
    full = np.linalg.svd(T.reshape(K * K, K).T, compute_uv=False)
    Kh = K // 2 + 1
    m = np.arange(Kh)
    sw = np.where((m == 0) | (2 * m == K), 1.0, np.sqrt(2.0))
    Th = T[:Kh, :Kh, :Kh] * sw[:, None, None] * sw[None, :, None] * sw[None, None, :]
    half = np.linalg.svd(Th.reshape(Kh * Kh, Kh).T, compute_uv=False)
    np.testing.assert_allclose(half, full[:Kh], rtol=1e-12, atol=1e-14 * full[0])
    assert np.all(full[Kh:] < 1e-13 * full[0])


@pytest.mark.parametrize("interp", [1, 2])
def test_per_cell_form_parameters_are_validated_without_gpu(L, interp):
    from paper_2601_18838_gb300._binding import Params

    def plan_status(**kw):
        p = Params()
        L.kpme_default_params(C.byref(p))
        p.radius, p.interp, p.order, p.K, p.modes, p.skp_method = 10.0, interp, 8, 64, 4, 1
        for k, v in kw.items():
            setattr(p, k, v)
        h = C.c_void_p()
        st = L.kpme_plan(C.byref(p), None, C.byref(h))
        if h.value:   # a GPU is present and the plan was made
            L.kpme_destroy(h)
            assert st == 0
        return st

    # past validation: KPME_OK with a GPU, else the missing GPU is the first error (KPME_ERR_CUDA)
    assert plan_status() in (0, 3)
    assert plan_status(order=16, K=32, modes=64) in (0, 3)
    for bad in (dict(skp_method=0), dict(order=5), dict(order=10, K=60), dict(K=60), dict(modes=0),
                dict(modes=65), dict(K=1024), dict(interp=3)):
        assert plan_status(**bad) == 1, bad   # KPME_ERR_INVALID_ARG
