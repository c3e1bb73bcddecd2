"""Python binding of ``libsusp.so``, the GB300 library that advances the
minimal dense-suspension model of Li, Royer & Ness (arXiv 2307.13802).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  The functions keep the names of the C ABI (``include/susp.h``);
``System`` wraps one handle.  Importing this package loads the library and
raises if it is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsusp.so")

SUSP_OK, SUSP_EINVAL, SUSP_ENOMEM, SUSP_ECUDA, SUSP_ESTATE = 0, 1, 2, 3, 4
SUSP_ENEIGH, SUSP_EUNSTABLE, SUSP_ENODEV = 5, 6, 8
SUSP_FP64, SUSP_MIXED = 0, 1
SUSP_STRESS_LEN = 76
SUSP_INFO_LEN = 14
SUSP_PROFILE_LEN = 15
PROFILE_FAMILIES = ("integrate", "rebuild", "pair", "reduce", "finalize")

ERROR_NAMES = {0: "SUSP_OK", 1: "SUSP_EINVAL", 2: "SUSP_ENOMEM", 3: "SUSP_ECUDA",
               4: "SUSP_ESTATE", 5: "SUSP_ENEIGH", 6: "SUSP_EUNSTABLE",
               8: "SUSP_ENODEV"}


class SuspError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class susp_params(C.Structure):
    """Mirror of ``susp_params`` in include/susp.h."""
    _fields_ = [
        ("eta", C.c_double), ("rho", C.c_double), ("kn", C.c_double),
        ("kt", C.c_double), ("mu", C.c_double), ("xi_min", C.c_double),
        ("xi_max", C.c_double), ("skin", C.c_double),
        ("shear_rate", C.c_double), ("kT", C.c_double),
        ("torque_sign", C.c_double), ("dt", C.c_double), ("seed", C.c_uint64),
        ("precision", C.c_int32), ("noise", C.c_int32),
        ("lubrication", C.c_int32), ("onebody", C.c_int32),
        ("contact", C.c_int32), ("sample_every", C.c_int32),
        ("kmax", C.c_int32), ("threads_per_particle", C.c_int32),
        ("use_graphs", C.c_int32), ("structural", C.c_int32),
        ("series_cap", C.c_int32), ("rebuild_every", C.c_int32),
        ("rep_A", C.c_double), ("rep_cut", C.c_double), ("shell", C.c_double),
        ("deterministic", C.c_int32), ("autotune", C.c_int32),
    ]


_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)
_H = C.c_void_p

# name -> (restype, argtypes)
_SIGNATURES = {
    "susp_default_params": (None, [C.POINTER(susp_params)]),
    "susp_create": (C.c_int, [C.POINTER(_H), C.c_int64, _D, _D, C.POINTER(susp_params)]),
    "susp_create_batch": (C.c_int, [C.POINTER(_H), C.c_int32, _I64, _D, _D,
                                    C.POINTER(susp_params)]),
    "susp_destroy": (None, [_H]),
    "susp_last_error": (C.c_char_p, [_H]),
    "susp_create_error": (C.c_char_p, []),
    "susp_set_stream": (C.c_int, [_H, C.c_void_p]),
    "susp_set_allocator": (C.c_int, [_H, C.c_void_p, C.c_void_p, C.c_void_p]),
    "susp_set_state": (C.c_int, [_H, _D, _D, _D]),
    "susp_set_state_device": (C.c_int, [_H, C.c_void_p, C.c_void_p, C.c_void_p]),
    "susp_set_clock": (C.c_int, [_H, C.c_int64, C.c_int32, C.c_double]),
    "susp_get_state": (C.c_int, [_H, _D, _D, _D]),
    "susp_get_forces": (C.c_int, [_H, _D, _D]),
    "susp_build_neighbors": (C.c_int, [_H]),
    "susp_evaluate": (C.c_int, [_H]),
    "susp_step": (C.c_int, [_H, C.c_int64, C.c_double, C.c_double, C.c_double,
                            C.c_uint64]),
    "susp_step_batch": (C.c_int, [_H, C.c_int64, C.c_double]),
    "susp_stress": (C.c_int, [_H, _D, C.c_int32]),
    "susp_profile": (C.c_int, [_H, C.c_int64, C.c_double, _D]),
    "susp_get_pairs": (C.c_int, [_H, _I32, C.c_int64, _I64]),
    "susp_get_history": (C.c_int, [_H, _I32, _D, C.c_int64, _I64]),
    "susp_get_info": (C.c_int, [_H, _D]),
    "susp_pair_stress_noalloc": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.c_int64, C.c_void_p, _D,
                                           C.c_double, C.POINTER(susp_params), C.c_double,
                                           C.c_int64, C.c_void_p, C.c_void_p]),
    "susp_get_series": (C.c_int, [_H, C.c_int32, _D, C.c_int64, _I64, _I64]),
    "susp_measure_peaks": (C.c_int, [_D]),
    "susp_green_kubo": (C.c_int, [_D, C.c_int64, C.c_int64, C.c_double, C.c_double,
                                  C.c_double, _D, _D, _D]),
    "susp_set_skin": (C.c_int, [_H, C.c_double]),
    "susp_autotune": (C.c_int, [_H, C.c_int64, C.c_double, _D, C.c_int32, _D, _D]),
    "susp_save": (C.c_int, [_H, C.c_char_p]),
    "susp_load": (C.c_int, [_H, C.c_char_p]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (nvcc required); "
            "there is no CPU fallback")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in _SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


def _vec(a, N):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != 3 * N:
        raise ValueError(f"expected {N}x3 values, got shape {a.shape}")
    return a


def default_params(**kw) -> susp_params:
    p = susp_params()
    lib.susp_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": SUSP_FP64, "mixed": SUSP_MIXED}[v]
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def green_kubo(x, max_lag: int, dt: float, V: float, kT: float):
    """Autocorrelation C, running Green-Kubo viscosity eta (Eq. 33) and the
    fit (eta_phi, tau_phi) of a stress series, computed by the library."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    Cc, eta, fit = np.zeros(max_lag), np.zeros(max_lag), np.zeros(2)
    check(lib.susp_green_kubo(_dp(x), len(x), int(max_lag), float(dt), float(V), float(kT),
                              _dp(Cc), _dp(eta), _dp(fit)))
    return Cc, eta, (float(fit[0]), float(fit[1]))


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


def torch_allocator(device=None):
    """(alloc, release) callables that take device memory from PyTorch's
    caching allocator on `device` (default: the current device), for
    ``System.set_allocator``."""
    import torch

    dev = torch.cuda.current_device() if device is None else torch.device(device).index

    def alloc(nbytes):
        return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev))

    def release(ptr):
        torch.cuda.caching_allocator_delete(int(ptr))

    return alloc, release


def measure_peaks() -> dict:
    """Peak FP64 and FP32 multiply-add rates of the current device (GFLOP/s)."""
    out = np.zeros(2)
    check(lib.susp_measure_peaks(_dp(out)))
    return {"fp64_gflops": float(out[0]), "fp32_gflops": float(out[1])}


def check(code: int, h=None):
    if code != SUSP_OK:
        msg = lib.susp_last_error(h).decode() if h else lib.susp_create_error().decode()
        raise SuspError(code, msg)


class System:
    """One handle: a single system (``radii``, ``box``) or, with
    ``System.batch``, several replicas stepped together."""

    def __init__(self, radii, box, **params):
        radii = np.ascontiguousarray(radii, dtype=np.float64)
        box = np.ascontiguousarray(box, dtype=np.float64)
        self.N = len(radii)
        self.R = 1
        self.params = default_params(**params)
        h = _H()
        check(lib.susp_create(C.byref(h), self.N, _dp(radii), _dp(box),
                              C.byref(self.params)))
        self._h = h
        self.offsets = np.array([0, self.N])

    @classmethod
    def batch(cls, sizes, radii, boxes, params_list):
        self = cls.__new__(cls)
        sizes = np.ascontiguousarray(sizes, dtype=np.int64)
        radii = np.ascontiguousarray(radii, dtype=np.float64)
        boxes = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 3)
        R = len(sizes)
        arr = (susp_params * R)()
        for r, kw in enumerate(params_list):
            arr[r] = default_params(**kw)
        self.N = int(sizes.sum())
        self.R = R
        self.params = arr[0]
        h = _H()
        check(lib.susp_create_batch(C.byref(h), R, sizes.ctypes.data_as(_I64),
                                    _dp(radii), _dp(boxes), arr))
        self._h = h
        self.offsets = np.concatenate([[0], np.cumsum(sizes)])
        return self

    def close(self):
        if getattr(self, "_h", None):
            lib.susp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, code):
        check(code, self._h)

    # -- plumbing -----------------------------------------------------------
    def set_stream(self, stream_ptr: int):
        self._chk(lib.susp_set_stream(self._h, C.c_void_p(stream_ptr)))

    def set_allocator(self, alloc, release):
        """Device memory of this handle from alloc(nbytes) -> pointer and
        back through release(pointer); before the first set_state."""
        def a(n, _ctx):
            try:
                return alloc(n) or None
            except Exception:
                return None

        def r(ptr, _ctx):
            release(ptr)

        # the C callbacks must outlive the handle
        self._allocator = (_ALLOC_FN(a), _FREE_FN(r))
        self._chk(lib.susp_set_allocator(self._h, C.cast(self._allocator[0], C.c_void_p),
                                         C.cast(self._allocator[1], C.c_void_p), None))

    # -- state --------------------------------------------------------------
    def set_state(self, x, U=None, W=None):
        x, U, W = _vec(x, self.N), _vec(U, self.N), _vec(W, self.N)
        self._chk(lib.susp_set_state(self._h, _dp(x), _dp(U), _dp(W)))

    def set_state_device(self, x_ptr, U_ptr=None, W_ptr=None):
        self._chk(lib.susp_set_state_device(self._h, C.c_void_p(x_ptr),
                                            C.c_void_p(U_ptr) if U_ptr else None,
                                            C.c_void_p(W_ptr) if W_ptr else None))

    def set_clock(self, k: int, strain: float, replica: int = -1):
        self._chk(lib.susp_set_clock(self._h, int(k), int(replica), float(strain)))

    def state(self):
        x, U, W = (np.zeros((self.N, 3)) for _ in range(3))
        self._chk(lib.susp_get_state(self._h, _dp(x), _dp(U), _dp(W)))
        return x, U, W

    def forces(self):
        F, T = np.zeros((self.N, 3)), np.zeros((self.N, 3))
        self._chk(lib.susp_get_forces(self._h, _dp(F), _dp(T)))
        return F, T

    # -- the method -----------------------------------------------------------
    def build_neighbors(self):
        self._chk(lib.susp_build_neighbors(self._h))

    def evaluate(self):
        self._chk(lib.susp_evaluate(self._h))

    def step(self, n: int, shear_rate: float, kT: float, dt: float, seed: int):
        self._chk(lib.susp_step(self._h, int(n), float(shear_rate), float(kT),
                                float(dt), int(seed)))

    def step_batch(self, n: int, dt: float):
        self._chk(lib.susp_step_batch(self._h, int(n), float(dt)))

    def profile(self, n: int, dt: float) -> dict:
        """Per kernel family: total ms, launches, mean ms per launch."""
        out = np.zeros(SUSP_PROFILE_LEN)
        self._chk(lib.susp_profile(self._h, int(n), float(dt), _dp(out)))
        return {f: dict(ms=out[3 * i], launches=int(out[3 * i + 1]), ms_per_launch=out[3 * i + 2])
                for i, f in enumerate(PROFILE_FAMILIES)}

    def stress(self, replica: int = 0) -> dict:
        out = np.zeros(SUSP_STRESS_LEN)
        self._chk(lib.susp_stress(self._h, _dp(out), int(replica)))
        t = out[:54].reshape(6, 3, 3)
        return dict(contact=t[0], lubrication=t[1], brownian=t[2], drag=t[3],
                    kinetic=t[4], kinetic_rot=t[5], eta_r=out[54], N1=out[55],
                    N2=out[56], samples=int(out[57]),
                    repulsion=out[58:67].reshape(3, 3), structural=out[67:76].reshape(3, 3))

    def series(self, replica: int = 0):
        """Sigma^B_xy of each sampled evaluation since the last call (which
        resets the record), and the number of samples dropped beyond the
        capacity."""
        n, dropped = C.c_int64(0), C.c_int64(0)
        self._chk(lib.susp_get_series(self._h, int(replica), None, 0, C.byref(n),
                                      C.byref(dropped)))
        out = np.zeros(max(n.value, 1))
        self._chk(lib.susp_get_series(self._h, int(replica), _dp(out), n.value, C.byref(n),
                                      C.byref(dropped)))
        return out[:n.value], dropped.value

    def pairs(self):
        n = C.c_int64(0)
        self._chk(lib.susp_get_pairs(self._h, None, 0, C.byref(n)))
        ij = np.zeros((max(n.value, 1), 2), dtype=np.int32)
        self._chk(lib.susp_get_pairs(self._h, ij.ctypes.data_as(_I32), n.value,
                                     C.byref(n)))
        return ij[:n.value]

    def history(self):
        n = C.c_int64(0)
        self._chk(lib.susp_get_history(self._h, None, None, 0, C.byref(n)))
        ij = np.zeros((max(n.value, 1), 2), dtype=np.int32)
        xi = np.zeros((max(n.value, 1), 3))
        self._chk(lib.susp_get_history(self._h, ij.ctypes.data_as(_I32), _dp(xi),
                                       n.value, C.byref(n)))
        return ij[:n.value], xi[:n.value]

    def info(self) -> dict:
        out = np.zeros(SUSP_INFO_LEN)
        self._chk(lib.susp_get_info(self._h, _dp(out)))
        keys = ("k", "nbuilds", "max_row", "kmax", "npairs", "strain", "tilt",
                "threads_per_particle", "precision", "replicas", "N",
                "graph_steps", "device_bytes", "launches")
        return dict(zip(keys, out.tolist()))

    def set_skin(self, skin: float):
        self._chk(lib.susp_set_skin(self._h, float(skin)))

    def autotune(self, trial_steps: int, dt: float, skins):
        """Times trial_steps steps at each candidate skin from the current
        state, keeps the fastest and restores the state; returns
        (chosen skin, ms per step of each candidate)."""
        sk = np.ascontiguousarray(skins, dtype=np.float64)
        ms = np.zeros(len(sk))
        chosen = C.c_double(0.0)
        self._chk(lib.susp_autotune(self._h, int(trial_steps), float(dt), _dp(sk), len(sk),
                                    _dp(ms), C.byref(chosen)))
        return chosen.value, ms

    def save(self, path: str):
        self._chk(lib.susp_save(self._h, path.encode()))

    def load(self, path: str):
        self._chk(lib.susp_load(self._h, path.encode()))
