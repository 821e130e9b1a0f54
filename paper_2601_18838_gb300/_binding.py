"""ctypes binding of libkpme (include/kpme.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts torch
tensors to device pointers, passes the current CUDA stream, and turns status
codes into exceptions.  If ``libkpme.so`` has not been built the import of
``lib()`` raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
# KPME_LIB=debug loads the checked build (libkpme_debug.so, `build(debug=True)`)
LIB_PATH = os.path.join(PKG, "libkpme_debug.so" if os.environ.get("KPME_LIB") == "debug" else "libkpme.so")

PRECISIONS = {"fp64": 0, "fp32": 1, "tf32": 2, "tf32x3": 3, "bf16": 4, "bf16x3": 5, "bf16x6": 6, "bf16x10": 7}
SKP_METHODS = {"svd": 0, "sinc": 1}
STEP_NAMES = ["spread", "split", "skp_stage1", "skp_stage2", "skp_stage3", "gather", "virial"]

EXPORTS = [
    "kpme_default_params", "kpme_plan", "kpme_destroy", "kpme_set_stream", "kpme_set_precision",
    "kpme_build_skp", "kpme_set_skp", "kpme_get_skp", "kpme_potential", "kpme_virial_tensor", "kpme_energy_forces",
    "kpme_spread", "kpme_apply", "kpme_gather", "kpme_set_profiling", "kpme_get_profile",
    "kpme_get_info", "kpme_status_string", "kpme_last_error", "kpme_spread_noalloc",
    "kpme_batch_create", "kpme_batch_destroy", "kpme_batch_set_stream", "kpme_batch_build_skp",
    "kpme_batch_energy_forces", "kpme_batch_last_error", "kpme_autotune", "kpme_set_tune",
    "kpme_batch_autotune",
    "kpme_measure_update_rate", "kpme_save_skp", "kpme_load_skp",
]


class Params(C.Structure):
    _fields_ = [
        ("center", C.c_double * 3), ("radius", C.c_double), ("beta", C.c_double),
        ("order", C.c_int), ("K", C.c_int), ("skp_tol", C.c_double), ("skp_method", C.c_int),
        ("precision", C.c_int), ("max_n", C.c_int64), ("coulomb_k", C.c_double),
        ("interp", C.c_int), ("modes", C.c_int),
    ]


INTERP = {"bspline": 0, "lagrange": 1, "lagrange_modes": 2}


class Tune(C.Structure):
    _fields_ = [("tile", C.c_int), ("fused", C.c_int), ("split", C.c_int), ("from_cache", C.c_int),
                ("ms_per_eval", C.c_double)]


def _tune_dict(t):
    return {f: getattr(t, f) for f, _ in Tune._fields_}


class Info(C.Structure):
    _fields_ = [
        ("K", C.c_int), ("order", C.c_int), ("precision", C.c_int), ("r0", C.c_int), ("R", C.c_int),
        ("skp_rel_err", C.c_double), ("max_n", C.c_int64), ("scratch_bytes", C.c_int64),
        ("flops_useful", C.c_double), ("flops_executed", C.c_double), ("kernels_per_eval", C.c_int),
    ]


class KpmeError(RuntimeError):
    def __init__(self, func, status, detail=""):
        self.status = status
        msg = f"{func} failed: {_LIB.kpme_status_string(status).decode() if _LIB else status}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


_LIB = None
_vp, _i64, _dp, _ip = C.c_void_p, C.c_int64, C.c_void_p, C.POINTER(C.c_int)


def lib():
    """Load libkpme.so (built by ``__graft_entry__.build()`` / ``python -m paper_2601_18838_gb300.build``)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                           "(python -m paper_2601_18838_gb300.build)")
    L = C.CDLL(LIB_PATH)
    st = C.c_int
    sig = {
        "kpme_default_params": (st, [C.POINTER(Params)]),
        "kpme_plan": (st, [C.POINTER(Params), _vp, C.POINTER(_vp)]),
        "kpme_destroy": (None, [_vp]),
        "kpme_set_stream": (st, [_vp, _vp]),
        "kpme_set_precision": (st, [_vp, C.c_int]),
        "kpme_build_skp": (st, [_vp, _ip, C.POINTER(C.c_double)]),
        "kpme_set_skp": (st, [_vp, C.c_int, _ip, _dp, _dp, _dp, C.c_double]),
        "kpme_get_skp": (st, [_vp, _ip, _ip, _ip, _dp, _dp, _dp, _dp, _dp, C.POINTER(C.c_double)]),
        "kpme_potential": (st, [_vp, _i64, _vp, _vp, _i64, _vp, _vp]),
        "kpme_virial_tensor": (st, [_vp, _i64, _vp, _vp, _vp, _vp]),
        "kpme_energy_forces": (st, [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp]),
        "kpme_spread": (st, [_vp, _i64, _vp, _vp, _vp]),
        "kpme_apply": (st, [_vp, _vp, _vp]),
        "kpme_gather": (st, [_vp, _i64, _vp, _vp, _vp, _vp, _vp]),
        "kpme_set_profiling": (st, [_vp, C.c_int]),
        "kpme_get_profile": (st, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int, _ip, C.c_int]),
        "kpme_get_info": (st, [_vp, C.POINTER(Info)]),
        "kpme_status_string": (C.c_char_p, [C.c_int]),
        "kpme_last_error": (C.c_char_p, [_vp]),
        "kpme_spread_noalloc": (st, [C.POINTER(Params), _vp, _i64, _vp, _vp, _vp]),
        "kpme_batch_create": (st, [C.c_int, C.POINTER(Params), _vp, C.POINTER(_vp)]),
        "kpme_batch_destroy": (None, [_vp]),
        "kpme_batch_set_stream": (st, [_vp, _vp]),
        "kpme_batch_build_skp": (st, [_vp, _ip]),
        "kpme_batch_energy_forces": (st, [_vp, C.POINTER(C.c_int64), _vp, _vp, _vp, _vp, _vp, _vp]),
        "kpme_batch_last_error": (C.c_char_p, [_vp]),
        "kpme_autotune": (st, [_vp, _i64, _vp, _vp, C.c_char_p, C.POINTER(Tune)]),
        "kpme_set_tune": (st, [_vp, C.POINTER(Tune)]),
        "kpme_batch_autotune": (st, [_vp, C.POINTER(C.c_int64), _vp, _vp, C.c_char_p, _ip]),
        "kpme_measure_update_rate": (st, [C.c_int, C.c_int, _i64] + [C.POINTER(C.c_double)] * 3),
        "kpme_save_skp": (st, [_vp, C.c_char_p]),
        "kpme_load_skp": (st, [_vp, C.c_char_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


def measure_update_rate(K: int, order: int, n_particles: int) -> dict:
    """kpme_measure_update_rate: float32 atomic adds per second in the spreading's pattern
    (global mesh and shared-memory tile region) and reads per second in the gathering's."""
    g, s, r = C.c_double(), C.c_double(), C.c_double()
    st = lib().kpme_measure_update_rate(int(K), int(order), int(n_particles), C.byref(g), C.byref(s), C.byref(r))
    if st != 0:
        raise KpmeError("kpme_measure_update_rate", st)
    return {"global_atomic": g.value, "shared_atomic": s.value, "read": r.value}


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _np_ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _check_dev(t, name, dtype, shape=None):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


class Plan:
    """One reciprocal-space problem: box, mesh, B-spline order, Ewald beta, SKP, arithmetic.

    Mirrors ``kpme_plan``.  ``box`` is the side L = 2 r_B; positions live in
    [center - L/2, center + L/2)^3 (wrapped periodically)."""

    def __init__(self, box: float, K: int, order: int, beta: float = 0.35, center=None,
                 precision: str = "bf16x10", skp_tol: float = 1e-8, skp_method: str = "svd",
                 max_n: int = 1 << 20, coulomb_k: float = 1.0, stream=None, interp: str = "bspline",
                 modes: int = 0):
        """interp="lagrange": the per-cell form (K / order cells per axis, `order` Lagrange nodes
        per cell, modes |m|_inf <= `modes`); it needs skp_method="sinc".  interp="lagrange_modes":
        the same form with the node operator applied in mode space (one diagonal)."""
        import torch
        L = lib()
        p = Params()
        L.kpme_default_params(C.byref(p))
        c = (0.5 * box,) * 3 if center is None else tuple(center)
        p.center = (C.c_double * 3)(*c)
        p.radius = 0.5 * box
        p.beta = beta
        p.order = order
        p.K = K
        p.skp_tol = skp_tol
        p.skp_method = SKP_METHODS[skp_method]
        p.precision = PRECISIONS[precision]
        p.max_n = max_n
        p.coulomb_k = coulomb_k
        p.interp = INTERP[interp]
        p.modes = modes
        self.params = p
        self.interp, self.modes = interp, modes
        self.box, self.K, self.order, self.beta = box, K, order, beta
        self.precision = precision
        self._stream = stream
        h = C.c_void_p()
        st = L.kpme_plan(C.byref(p), self._stream_handle(), C.byref(h))
        if st != 0:
            raise KpmeError("kpme_plan", st)
        self._h = h
        self.R = 0

    def _stream_handle(self):
        import torch
        s = self._stream if self._stream is not None else torch.cuda.current_stream()
        return C.c_void_p(s.cuda_stream)

    def _call(self, name, *args):
        L = lib()
        L.kpme_set_stream(self._h, self._stream_handle())
        st = getattr(L, name)(self._h, *args)
        if st != 0:
            raise KpmeError(name, st, L.kpme_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().kpme_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- SKP ----
    def build_skp(self):
        r = C.c_int()
        e = C.c_double()
        self._call("kpme_build_skp", C.byref(r), C.byref(e))
        self.R = r.value
        return r.value, e.value

    def set_skp(self, r1, gen3, gen2, gen1, c: float = 0.0):
        import numpy as np
        r1 = np.ascontiguousarray(r1, dtype=np.int32)
        g3 = np.ascontiguousarray(gen3, dtype=np.float64)
        g2 = np.ascontiguousarray(gen2, dtype=np.float64)
        g1 = np.ascontiguousarray(gen1, dtype=np.float64)
        R = int(r1.sum())
        if g3.shape != (r1.size, self.K) or g2.shape != (R, self.K) or g1.shape != (R, self.K):
            raise ValueError("generator shapes must be (r0, K), (R, K), (R, K)")
        self._call("kpme_set_skp", C.c_int(r1.size), r1.ctypes.data_as(_ip), _np_ptr(g3), _np_ptr(g2),
                   _np_ptr(g1), C.c_double(c))
        self.R = R

    def get_skp(self) -> dict:
        import numpy as np
        r0, R = C.c_int(), C.c_int()
        self._call("kpme_get_skp", C.byref(r0), C.byref(R), None, None, None, None, None, None, None)
        r1 = np.zeros(r0.value, np.int32)
        g3 = np.zeros((r0.value, self.K))
        g2 = np.zeros((R.value, self.K))
        g1 = np.zeros((R.value, self.K))
        so = np.zeros(r0.value)
        si = np.zeros(R.value)
        c = C.c_double()
        self._call("kpme_get_skp", C.byref(r0), C.byref(R), r1.ctypes.data_as(_ip), _np_ptr(g3), _np_ptr(g2),
                   _np_ptr(g1), _np_ptr(so), _np_ptr(si), C.byref(c))
        return dict(r0=r0.value, R=R.value, r1=r1, gen3=g3, gen2=g2, gen1=g1, sigma_outer=so,
                    sigma_inner=si, c=c.value)

    def autotune(self, x, q, cache: str | None = None) -> dict:
        """kpme_autotune on the particles x, q: leaves the plan on the fastest configuration."""
        import torch
        n = x.shape[0]
        _check_dev(x, "x", torch.float64, (n, 3))
        _check_dev(q, "q", torch.float64, (n,))
        t = Tune()
        self._call("kpme_autotune", C.c_int64(n), _ptr(x), _ptr(q), cache.encode() if cache else None, C.byref(t))
        return _tune_dict(t)

    def save_skp(self, path: str):
        """kpme_save_skp: store this plan's SKP in a file (generator form, with K, order, box, beta)."""
        self._call("kpme_save_skp", os.fspath(path).encode())

    def load_skp(self, path: str):
        """kpme_load_skp: install an SKP stored by save_skp on a plan of the same mesh and box."""
        self._call("kpme_load_skp", os.fspath(path).encode())

    def set_tune(self, tile: int, fused: int, split: int):
        t = Tune(tile, fused, split, 0, 0.0)
        self._call("kpme_set_tune", C.byref(t))

    def skp_c(self) -> float:
        """The m = 0 correction constant c of the installed SKP (0 for the SVD form)."""
        if getattr(self, "interp", "bspline") != "bspline":   # dense factors: sizes and c only
            r0, R, c = C.c_int(), C.c_int(), C.c_double()
            self._call("kpme_get_skp", C.byref(r0), C.byref(R), None, None, None, None, None, None, C.byref(c))
            return float(c.value)
        return float(self.get_skp()["c"])

    def set_precision(self, precision: str):
        self._call("kpme_set_precision", C.c_int(PRECISIONS[precision]))
        self.precision = precision

    # ---- evaluation ----
    def energy_forces(self, x, q, forces: bool = True, dEdq: bool = True, virial: bool = False, out=None):
        """Energy (and -dE/dx, dE/dq, virial trace) for positions x (n,3) and charges q (n,), float64 CUDA."""
        import torch
        n = x.shape[0]
        _check_dev(x, "x", torch.float64, (n, 3))
        _check_dev(q, "q", torch.float64, (n,))
        dev = x.device
        o = out or {}
        E = o.get("energy") if o.get("energy") is not None else torch.empty(1, dtype=torch.float64, device=dev)
        F = (o.get("forces") if o.get("forces") is not None else torch.empty((n, 3), dtype=torch.float64, device=dev)) if forces else None
        P = (o.get("dEdq") if o.get("dEdq") is not None else torch.empty(n, dtype=torch.float64, device=dev)) if dEdq else None
        W = (o.get("virial") if o.get("virial") is not None else torch.empty(1, dtype=torch.float64, device=dev)) if virial else None
        self._call("kpme_energy_forces", C.c_int64(n), _ptr(x), _ptr(q), _ptr(E), _ptr(F), _ptr(P), _ptr(W))
        return dict(energy=E, forces=F, dEdq=P, virial=W)

    def potential(self, y, q, x):
        import torch
        _check_dev(y, "y", torch.float64, (y.shape[0], 3))
        _check_dev(q, "q", torch.float64, (y.shape[0],))
        _check_dev(x, "x", torch.float64, (x.shape[0], 3))
        p = torch.empty(x.shape[0], dtype=torch.float64, device=x.device)
        self._call("kpme_potential", C.c_int64(y.shape[0]), _ptr(y), _ptr(q), C.c_int64(x.shape[0]), _ptr(x), _ptr(p))
        return p

    def virial_tensor(self, x, q):
        """kpme_virial_tensor: the full reciprocal virial tensor (3, 3) and the mesh energy."""
        import torch
        n = x.shape[0]
        _check_dev(x, "x", torch.float64, (n, 3))
        _check_dev(q, "q", torch.float64, (n,))
        out = torch.empty(10, dtype=torch.float64, device=x.device)
        self._call("kpme_virial_tensor", C.c_int64(n), _ptr(x), _ptr(q), _ptr(out), C.c_void_p(out.data_ptr() + 72))
        return out[:9].reshape(3, 3), out[9]

    def spread(self, x, q):
        import torch
        n = x.shape[0]
        _check_dev(x, "x", torch.float64, (n, 3))
        _check_dev(q, "q", torch.float64, (n,))
        Q = torch.empty((self.K,) * 3, dtype=torch.float64, device=x.device)
        self._call("kpme_spread", C.c_int64(n), _ptr(x), _ptr(q), _ptr(Q))
        return Q

    def apply(self, Q):
        import torch
        _check_dev(Q, "Q", torch.float64, (self.K,) * 3)
        Phi = torch.empty_like(Q)
        self._call("kpme_apply", _ptr(Q), _ptr(Phi))
        return Phi

    def gather(self, x, q, Phi, forces: bool = True):
        import torch
        n = x.shape[0]
        _check_dev(x, "x", torch.float64, (n, 3))
        _check_dev(q, "q", torch.float64, (n,))
        _check_dev(Phi, "Phi", torch.float64, (self.K,) * 3)
        phi = torch.empty(n, dtype=torch.float64, device=x.device)
        F = torch.empty((n, 3), dtype=torch.float64, device=x.device) if forces else None
        self._call("kpme_gather", C.c_int64(n), _ptr(x), _ptr(q), _ptr(Phi), _ptr(phi), _ptr(F))
        return phi, F

    # ---- introspection ----
    def set_profiling(self, on: bool = True):
        self._call("kpme_set_profiling", C.c_int(1 if on else 0))

    def get_profile(self, reset: bool = True) -> dict:
        ms = (C.c_double * 16)()
        nl = (C.c_int64 * 16)()
        n = C.c_int()
        self._call("kpme_get_profile", ms, nl, C.c_int(16), C.byref(n), C.c_int(1 if reset else 0))
        return {STEP_NAMES[i]: (ms[i], nl[i]) for i in range(min(n.value, len(STEP_NAMES)))}

    def info(self) -> dict:
        i = Info()
        self._call("kpme_get_info", C.byref(i))
        return {f: getattr(i, f) for f, _ in Info._fields_}


class Batch:
    """Independent systems evaluated by one graph launch (``kpme_batch_*``).

    ``systems``: list of dicts with keys box, K, order and optionally beta, center,
    skp_tol, max_n.  ``energy_forces`` takes the concatenated positions / charges and the
    host offsets delimiting each system."""

    def __init__(self, systems, precision: str = "bf16x10", skp_method: str = "svd", coulomb_k: float = 1.0,
                 stream=None):
        L = lib()
        arr = (Params * len(systems))()
        for i, sd in enumerate(systems):
            p = arr[i]
            L.kpme_default_params(C.byref(p))
            box = float(sd["box"])
            c = sd.get("center") or (0.5 * box,) * 3
            p.center = (C.c_double * 3)(*c)
            p.radius = 0.5 * box
            p.beta = sd.get("beta", 0.35)
            p.order = sd["order"]
            p.K = sd["K"]
            p.skp_tol = sd.get("skp_tol", 1e-8)
            p.skp_method = SKP_METHODS[skp_method]
            p.precision = PRECISIONS[precision]
            p.max_n = sd.get("max_n", 1 << 20)
            p.coulomb_k = coulomb_k
        self.n_sys = len(systems)
        self._stream = stream
        h = C.c_void_p()
        st = L.kpme_batch_create(C.c_int(self.n_sys), arr, self._stream_handle(), C.byref(h))
        if st != 0:
            raise KpmeError("kpme_batch_create", st)
        self._h = h

    def _stream_handle(self):
        import torch
        s = self._stream if self._stream is not None else torch.cuda.current_stream()
        return C.c_void_p(s.cuda_stream)

    def _call(self, name, *args):
        L = lib()
        L.kpme_batch_set_stream(self._h, self._stream_handle())
        st = getattr(L, name)(self._h, *args)
        if st != 0:
            raise KpmeError(name, st, L.kpme_batch_last_error(self._h).decode())

    def build_skp(self):
        import numpy as np
        r = np.zeros(self.n_sys, np.int32)
        self._call("kpme_batch_build_skp", r.ctypes.data_as(_ip))
        return r

    def autotune(self, x, q, offsets, cache: str | None = None) -> int:
        """kpme_batch_autotune: returns the number of systems that were timed."""
        import numpy as np
        import torch
        n = x.shape[0]
        _check_dev(x, "x", torch.float64, (n, 3))
        _check_dev(q, "q", torch.float64, (n,))
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        k = C.c_int()
        self._call("kpme_batch_autotune", off.ctypes.data_as(C.POINTER(C.c_int64)), _ptr(x), _ptr(q),
                   cache.encode() if cache else None, C.byref(k))
        return k.value

    def energy_forces(self, x, q, offsets, forces: bool = True, dEdq: bool = True, virial: bool = False):
        import numpy as np
        import torch
        n = x.shape[0]
        _check_dev(x, "x", torch.float64, (n, 3))
        _check_dev(q, "q", torch.float64, (n,))
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        if off.size != self.n_sys + 1 or off[-1] != n:
            raise ValueError("offsets must have n_sys + 1 entries ending at the particle count")
        dev = x.device
        E = torch.empty(self.n_sys, dtype=torch.float64, device=dev)
        F = torch.empty((n, 3), dtype=torch.float64, device=dev) if forces else None
        P = torch.empty(n, dtype=torch.float64, device=dev) if dEdq else None
        W = torch.empty(self.n_sys, dtype=torch.float64, device=dev) if virial else None
        self._call("kpme_batch_energy_forces", off.ctypes.data_as(C.POINTER(C.c_int64)), _ptr(x), _ptr(q), _ptr(E),
                   _ptr(F), _ptr(P), _ptr(W))
        return dict(energy=E, forces=F, dEdq=P, virial=W)

    def close(self):
        if getattr(self, "_h", None):
            lib().kpme_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
