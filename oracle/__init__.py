"""ctypes binding of the plain FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this module.  The product library
(``paper_2307_13802_gb300``) never imports it, and the two share no code.

The oracle follows the equations of Li, Royer & Ness (arXiv 2307.13802),
Sec. II (Eqs. 1-24) and Sec. II.E (tilted box); see the header of
``oracle.c`` for the passage behind each part and the readings taken.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
          "-shared"]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp"
    subprocess.run(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    """Mirror of ``o_params`` in oracle.c."""
    _fields_ = [
        ("eta", C.c_double), ("rho", C.c_double), ("kn", C.c_double),
        ("kt", C.c_double), ("mu", C.c_double), ("xi_min", C.c_double),
        ("xi_max", C.c_double), ("skin", C.c_double),
        ("shear_rate", C.c_double), ("kT", C.c_double), ("dt", C.c_double),
        ("torque_sign", C.c_double),
        ("seed", C.c_int64), ("noise", C.c_int64), ("lubrication", C.c_int64),
        ("onebody", C.c_int64), ("contact", C.c_int64), ("freeze", C.c_int64),
        ("rebuild_every_step", C.c_int64),
        ("rep_A", C.c_double), ("rep_cut", C.c_double), ("shell", C.c_double),
        ("structural", C.c_int64),
    ]


DEFAULTS = dict(eta=1.0, rho=1.0, kn=1e4, kt=0.0, mu=0.0, xi_min=1e-3,
                xi_max=0.05, skin=0.3, shear_rate=1.0, kT=0.0, dt=1e-4,
                torque_sign=-1.0, seed=0, noise=1, lubrication=1, onebody=1,
                contact=1, freeze=0, rebuild_every_step=0, rep_A=0.0, rep_cut=10.0,
                shell=0.05, structural=0)


def make_params(**kw) -> Params:
    d = dict(DEFAULTS)
    unknown = set(kw) - set(d)
    if unknown:
        raise TypeError(f"unknown oracle parameters {sorted(unknown)}")
    d.update(kw)
    return Params(**d)


_lib = None
_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_U32 = C.POINTER(C.c_uint32)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.o_create.restype = C.c_void_p
        L.o_create.argtypes = [C.c_int32, _D, _D, C.POINTER(Params)]
        L.o_destroy.argtypes = [C.c_void_p]
        L.o_set_state.argtypes = [C.c_void_p, _D, _D, _D]
        L.o_set_strain.argtypes = [C.c_void_p, C.c_double]
        L.o_set_velocities.argtypes = [C.c_void_p, _D, _D]
        L.o_set_k.argtypes = [C.c_void_p, C.c_int64]
        L.o_set_tags.argtypes = [C.c_void_p, _U32]
        L.o_set_tags.restype = C.c_int
        L.o_evaluate.argtypes = [C.c_void_p]
        L.o_evaluate.restype = C.c_int
        L.o_build.argtypes = [C.c_void_p]
        L.o_build.restype = C.c_int
        L.o_step.argtypes = [C.c_void_p, C.c_int64]
        L.o_step.restype = C.c_int
        L.o_get_state.argtypes = [C.c_void_p, _D, _D, _D]
        L.o_get_forces.argtypes = [C.c_void_p, _D, _D]
        L.o_get_stress.argtypes = [C.c_void_p, _D]
        L.o_take_stress_sums.argtypes = [C.c_void_p, _D]
        L.o_take_stress_sums.restype = C.c_int64
        L.o_get_info.argtypes = [C.c_void_p, _D]
        L.o_list_size.argtypes = [C.c_void_p]
        L.o_list_size.restype = C.c_int64
        L.o_get_list.argtypes = [C.c_void_p, _I32, _D, _I32]
        L.o_brute_pairs.argtypes = [C.c_void_p, _I32, C.c_int64]
        L.o_brute_pairs.restype = C.c_int64
        L.o_philox4x32_10.argtypes = [_U32, _U32, _U32]
        L.o_gaussians6.argtypes = [C.c_int64, C.c_int64, C.c_uint32,
                                   C.c_uint32, _D]
        L.o_resistances.argtypes = [C.c_double, C.c_double, C.c_double,
                                    C.c_double, _D]
        L.o_lubrication.argtypes = [_D, _D, _D, _D, _D, _D, _D, _D]
        L.o_pair_brownian.argtypes = [_D, _D, _D, _D, C.c_double, C.c_double,
                                      _D, _D, _D]
        L.o_drag_stress_xy.argtypes = [C.c_int32, _D, _D, C.c_double,
                                       C.c_double]
        L.o_drag_stress_xy.restype = C.c_double
        L.o_timescales.argtypes = [C.c_double] * 6 + [_D]
        L.o_autocorr.argtypes = [_D, C.c_int64, C.c_int64, _D]
        L.o_green_kubo.argtypes = [_D, C.c_int64, C.c_int64, C.c_double, C.c_double,
                                   C.c_double, _D, _D]
        L.o_gk_fit.argtypes = [_D, C.c_int64, C.c_double, C.c_int64, _D]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


# ---------------------------------------------------------------------------
# pure functions
# ---------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().o_philox4x32_10(c.ctypes.data_as(_U32), k.ctypes.data_as(_U32),
                          out.ctypes.data_as(_U32))
    return out


def gaussians6(seed: int, k: int, t1: int, t2: int) -> np.ndarray:
    out = np.zeros(6)
    lib().o_gaussians6(int(seed), int(k), int(t1), int(t2), _dp(out))
    return out


def resistances(eta, ai, aj, xi_e) -> np.ndarray:
    """[XA11, YA11, YB11, YB21, YC11, YC12, YC21, YC22], Eqs. 9-12, 15-18."""
    out = np.zeros(8)
    lib().o_resistances(eta, ai, aj, xi_e, _dp(out))
    return out


def lubrication(R, n, dU, Wi, Wj):
    """Force on i and torques on i, j (Eqs. 8, 13, 14)."""
    R, n, dU, Wi, Wj = (_f64(v) for v in (R, n, dU, Wi, Wj))
    Fi, Ti, Tj = np.zeros(3), np.zeros(3), np.zeros(3)
    lib().o_lubrication(_dp(R), _dp(n), _dp(dU), _dp(Wi), _dp(Wj), _dp(Fi),
                        _dp(Ti), _dp(Tj))
    return Fi, Ti, Tj


def pair_brownian(R, n, theta, chi, c, torque_sign=-1.0):
    """Pair Brownian force on i and torques on i, j (Eqs. 22-24)."""
    R, n, theta, chi = (_f64(v) for v in (R, n, theta, chi))
    Fi, Ti, Tj = np.zeros(3), np.zeros(3), np.zeros(3)
    lib().o_pair_brownian(_dp(R), _dp(n), _dp(theta), _dp(chi), c,
                          torque_sign, _dp(Fi), _dp(Ti), _dp(Tj))
    return Fi, Ti, Tj


def drag_stress_xy(radii, box, eta, rate) -> float:
    r = _f64(radii)
    b = _f64(box)
    return lib().o_drag_stress_xy(len(r), _dp(r), _dp(b), eta, rate)


def timescales(a, rho, kn, eta, kT, rate) -> np.ndarray:
    """[tau_C, tau_I, tau_B, tau_S, Pe], Eqs. 27-30 and Sec. II.F."""
    out = np.zeros(5)
    lib().o_timescales(a, rho, kn, eta, kT, rate, _dp(out))
    return out


def green_kubo(series, max_lag: int, dt: float, V: float, kT: float):
    """Autocorrelation C(tau) of a stress series and the running Green-Kubo
    integral eta(t) = V/kT int_0^t C (Eq. 33, trapezoid rule)."""
    x = _f64(series)
    C_, eta = np.zeros(max_lag), np.zeros(max_lag)
    lib().o_green_kubo(_dp(x), len(x), int(max_lag), float(dt), float(V), float(kT),
                       _dp(C_), _dp(eta))
    return C_, eta


def gk_fit(eta, dt: float, grid: int = 400):
    """(eta_phi, tau_phi) of eta(t) ~ eta_phi (1 - exp(-t/tau_phi)) by least
    squares on a log grid of tau (Sec. III.D)."""
    e = _f64(eta)
    out = np.zeros(2)
    lib().o_gk_fit(_dp(e), len(e), float(dt), int(grid), _dp(out))
    return float(out[0]), float(out[1])


# ---------------------------------------------------------------------------
# a simulated system
# ---------------------------------------------------------------------------
class System:
    """One oracle system: tags are the input indices 0..N-1."""

    def __init__(self, radii, box, **params):
        self.radii = _f64(radii)
        self.N = len(self.radii)
        self.box = _f64(box)
        self.params = make_params(**params)
        self._h = lib().o_create(self.N, _dp(self.radii), _dp(self.box),
                                 C.byref(self.params))
        if not self._h:
            raise ValueError("oracle: invalid system")

    def close(self):
        if self._h:
            lib().o_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, x, U=None, W=None):
        x = _f64(x, (self.N, 3))
        U = None if U is None else _f64(U, (self.N, 3))
        W = None if W is None else _f64(W, (self.N, 3))
        lib().o_set_state(self._h, _dp(x), _dp(U) if U is not None else None,
                          _dp(W) if W is not None else None)

    def set_velocities(self, U, W):
        """New velocities; positions, list and tangential history are kept."""
        U, W = _f64(U, (self.N, 3)), _f64(W, (self.N, 3))
        lib().o_set_velocities(self._h, _dp(U), _dp(W))

    def set_strain(self, strain: float):
        lib().o_set_strain(self._h, float(strain))

    def set_k(self, k: int):
        lib().o_set_k(self._h, int(k))

    def set_tags(self, tags):
        """Noise-counter tags (increasing with the index)."""
        t = np.ascontiguousarray(tags, dtype=np.uint32)
        if len(t) != self.N or lib().o_set_tags(self._h, t.ctypes.data_as(_U32)):
            raise ValueError("tags must be N values increasing with the index")

    def evaluate(self):
        if lib().o_evaluate(self._h):
            raise MemoryError("oracle: evaluate failed")

    def build(self):
        if lib().o_build(self._h):
            raise MemoryError("oracle: build failed")

    def step(self, n: int):
        if lib().o_step(self._h, int(n)):
            raise MemoryError("oracle: step failed")

    def state(self):
        x, U, W = (np.zeros((self.N, 3)) for _ in range(3))
        lib().o_get_state(self._h, _dp(x), _dp(U), _dp(W))
        return x, U, W

    def forces(self):
        F, T = np.zeros((self.N, 3)), np.zeros((self.N, 3))
        lib().o_get_forces(self._h, _dp(F), _dp(T))
        return F, T

    _KEYS = ("contact", "lubrication", "brownian", "repulsion", "structural",
             "kinetic", "kinetic_rot")

    def stress(self):
        """Last evaluation: dict of 3x3 tensors (contact, lubrication,
        brownian pair, repulsion, structural Brownian) and the kinetic
        tensors of the last full-step velocities."""
        out = np.zeros(63)
        lib().o_get_stress(self._h, _dp(out))
        return dict(zip(self._KEYS, out.reshape(7, 3, 3)))

    def take_stress_sums(self):
        out = np.zeros(63)
        n = lib().o_take_stress_sums(self._h, _dp(out))
        return n, dict(zip(self._KEYS, out.reshape(7, 3, 3)))

    def info(self):
        out = np.zeros(8)
        lib().o_get_info(self._h, _dp(out))
        keys = ("strain", "tilt", "k", "nlist", "nbuilds", "ncontacts",
                "nlub", "max_overlap")
        return dict(zip(keys, out.tolist()))

    def verlet_list(self):
        n = lib().o_list_size(self._h)
        ij = np.zeros((n, 2), dtype=np.int32)
        hist = np.zeros((n, 3))
        contact = np.zeros(n, dtype=np.int32)
        if n:
            lib().o_get_list(self._h, ij.ctypes.data_as(_I32), _dp(hist),
                             contact.ctypes.data_as(_I32))
        return ij, hist, contact

    def brute_pairs(self):
        n = lib().o_brute_pairs(self._h, None, 0)
        ij = np.zeros((max(n, 1), 2), dtype=np.int32)
        lib().o_brute_pairs(self._h, ij.ctypes.data_as(_I32), n)
        return ij[:n]
