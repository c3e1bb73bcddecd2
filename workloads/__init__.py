"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module holds no arithmetic of the suspension model: it only draws
radii, box sizes, sphere positions (random placement followed by geometric
overlap removal, ``packing.c``) and run parameters.  Both the oracle and
the CUDA library consume what it produces; neither is imported here.

Recipes (a = 1 is the small radius; eta = rate = 1; rho = 1; k_n = 1e4;
k_t = k_n / 2 when mu > 0; dt = 1e-4; skin 0.3; kT = 6 pi eta a^3 rate / Pe,
the Peclet number of Sec. II.F):

* ``bidisperse``: radii 1.0 and 1.4, exactly N/2 each, order shuffled;
* ``polydisperse``: radii uniform in [1.0, 1.4];
* the cubic box edge follows from the volume fraction,
  L = (sum 4/3 pi a^3 / phi)^(1/3);
* positions: uniform random, then overlap removal to a largest overlap
  <= ``tol`` * a_min;
* large systems (``tile`` = k > 1): one seeded packing of N / k^3 spheres in
  a box of edge L / k is replicated k x k x k times, which keeps the volume
  fraction, the size distribution and the absence of overlaps exactly;
* velocities: the imposed shear flow at each centre, U = rate (y - L/2) x,
  Omega = -(rate / 2) z.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "packing.c")
_LIB = os.path.join(_HERE, "libpacking.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp",
                    "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _packlib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        D = C.POINTER(C.c_double)
        L.wl_relax.argtypes = [C.c_int64, D, D, D, C.c_double, C.c_int32,
                               C.c_int32, C.c_double, D]
        L.wl_relax.restype = C.c_int64
        _lib = L
    return _lib


def bidisperse_radii(N: int, seed: int, a_small=1.0, a_large=1.4):
    rng = np.random.Generator(np.random.PCG64(seed))
    r = np.full(N, a_small)
    r[N // 2:] = a_large
    rng.shuffle(r)
    return r


def polydisperse_radii(N: int, seed: int, lo=1.0, hi=1.4):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=N)


def box_for_phi(radii, phi: float) -> float:
    vol = float(np.sum(4.0 / 3.0 * math.pi * np.asarray(radii) ** 3))
    return (vol / phi) ** (1.0 / 3.0)


def packing(radii, L: float, seed: int, tol: float = 1e-4,
            max_sweeps: int = 4000, nstages: int = 0, scale0: float = 0.8):
    """Seeded positions (N, 3) in [0, L)^3 with largest overlap <= tol*a_min
    (or the sweep limit).  Returns (x, stats) with stats = (overlap/a_min,
    sweeps)."""
    radii = np.ascontiguousarray(radii, dtype=np.float64)
    N = len(radii)
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.ascontiguousarray(rng.uniform(0.0, L, size=(N, 3)))
    box = np.array([L, L, L], dtype=np.float64)
    stats = np.zeros(2)
    D = C.POINTER(C.c_double)
    rc = _packlib().wl_relax(N, radii.ctypes.data_as(D), box.ctypes.data_as(D),
                             x.ctypes.data_as(D), scale0, nstages, max_sweeps,
                             tol, stats.ctypes.data_as(D))
    if rc < 0:
        raise MemoryError("packing: allocation failed")
    return x, (float(stats[0]), int(stats[1]))


def shear_velocities(x, L: float, rate: float):
    """Imposed flow at each centre: U = rate (y - L/2) x, Omega = -rate/2 z."""
    N = len(x)
    U = np.zeros((N, 3))
    U[:, 0] = rate * (x[:, 1] - 0.5 * L)
    W = np.zeros((N, 3))
    W[:, 2] = -0.5 * rate
    return U, W


def kT_for_pe(pe: float, eta=1.0, a=1.0, rate=1.0) -> float:
    """Thermal energy giving Peclet number pe = 6 pi eta a^3 rate / kT."""
    return 6.0 * math.pi * eta * a ** 3 * rate / pe


@dataclass
class Workload:
    """One synthetic system ready for the oracle or the CUDA library."""
    name: str
    radii: np.ndarray
    L: float
    x: np.ndarray
    U: np.ndarray
    W: np.ndarray
    params: dict
    steps: int
    pack_stats: tuple = (0.0, 0)
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return len(self.radii)

    @property
    def box(self):
        return np.array([self.L, self.L, self.L])


def base_params(pe: float, mu: float, seed: int, rate: float = 1.0,
                dt: float = 1e-4) -> dict:
    kn = 1e4
    return dict(eta=1.0, rho=1.0, kn=kn, kt=0.5 * kn if mu > 0 else 0.0,
                mu=mu, xi_min=1e-3, xi_max=0.05, skin=0.3, shear_rate=rate,
                kT=kT_for_pe(pe, rate=rate) if pe > 0 else 0.0, dt=dt,
                torque_sign=-1.0, seed=seed)


def tile_packing(radii, x, L: float, k: int):
    """Replicate a periodic packing k x k x k times (box edge k L)."""
    rs, xs, box = tile_packing_box(radii, x, L, (k, k, k))
    return rs, xs, L * k


def tile_packing_box(radii, x, L: float, ks):
    """Replicate a periodic packing of a cubic box of edge L kx x ky x kz
    times; returns radii, positions and the box edges (kx L, ky L, kz L)."""
    kx, ky, kz = ks
    n = len(radii)
    shifts = np.array([(i, j, l) for l in range(kz) for j in range(ky)
                       for i in range(kx)], dtype=np.float64) * L
    xs = (x[None, :, :] + shifts[:, None, :]).reshape(n * kx * ky * kz, 3)
    rs = np.tile(radii, kx * ky * kz)
    return rs, np.ascontiguousarray(xs), np.array([kx * L, ky * L, kz * L])


def make(N: int, phi: float, pe: float, mu: float, *, poly: bool = False,
         pack_seed: int = 1000, dyn_seed: int = 2000, steps: int = 100,
         tol: float = 1e-4, name: str = "custom", rate: float = 1.0,
         max_sweeps: int = 4000, tile: int = 1) -> Workload:
    if N % (tile ** 3):
        raise ValueError("N must be divisible by tile^3")
    n = N // tile ** 3
    radii = polydisperse_radii(n, pack_seed) if poly else bidisperse_radii(n, pack_seed)
    L = box_for_phi(radii, phi)
    x, st = packing(radii, L, pack_seed + 1, tol=tol, max_sweeps=max_sweeps)
    if tile > 1:
        radii, x, L = tile_packing(radii, x, L, tile)
    U, W = shear_velocities(x, L, rate)
    return Workload(name=name, radii=radii, L=L, x=x, U=U, W=W,
                    params=base_params(pe, mu, dyn_seed, rate=rate),
                    steps=steps, pack_stats=st,
                    meta=dict(N=N, phi=phi, pe=pe, mu=mu, poly=poly,
                              tile=tile))


# Named workloads: sizes, volume fractions, Peclet numbers, friction, step
# counts and seeds (packing seed, dynamics seed).
WORKLOADS = {
    "bidisperse-500-phi0.50-pe10-mu0": dict(
        N=500, phi=0.50, pe=10.0, mu=0.0, poly=False, steps=1000, seeds=(1001, 2001)),
    "bidisperse-10k-phi0.56": dict(
        N=10_000, phi=0.56, pe=10.0, mu=1.0, poly=False, steps=20_000, seeds=(1002, 2002)),
    "bidisperse-1M-phi0.58-pe1000-mu1": dict(
        N=1_000_000, phi=0.58, pe=1000.0, mu=1.0, poly=False, steps=10_000,
        tile=4, seeds=(1003, 2003)),
    "polydisperse-8M-phi0.60-pe100-mu1": dict(
        N=8_000_000, phi=0.60, pe=100.0, mu=1.0, poly=True, steps=2000, tile=8,
        seeds=(1005, 2005)),
}


def scaled_tiles(tile_n: int, ks, phi: float, pe: float, mu: float, *, poly: bool,
                 pack_seed: int, dyn_seed: int, name: str = "tiled", rate: float = 1.0):
    """One seeded periodic packing of tile_n spheres replicated kx x ky x kz
    times: systems of different sizes with the same local structure (for
    scaling in N).  Returns (radii, box[3], x, U, W, params)."""
    n = tile_n
    radii = polydisperse_radii(n, pack_seed) if poly else bidisperse_radii(n, pack_seed)
    L = box_for_phi(radii, phi)
    x, _ = packing(radii, L, pack_seed + 1)
    rs, xs, box = tile_packing_box(radii, x, L, ks)
    U = np.zeros_like(xs)
    U[:, 0] = rate * (xs[:, 1] - 0.5 * box[1])
    W = np.zeros_like(xs)
    W[:, 2] = -0.5 * rate
    return rs, box, xs, U, W, base_params(pe, mu, dyn_seed, rate=rate)


def named(name: str, **override) -> Workload:
    c = dict(WORKLOADS[name])
    c.update(override)
    ps, ds = c["seeds"]
    return make(c["N"], c["phi"], c["pe"], c["mu"], poly=c["poly"],
                pack_seed=ps, dyn_seed=ds, steps=c["steps"], name=name,
                tile=c.get("tile", 1))


def replica_table(R: int = 256, seed: int = 4000, n_lo: int = 500,
                  n_hi: int = 20_000):
    """Batched-ensemble recipe: per replica N ~ U_int[n_lo, n_hi],
    phi ~ U[0.45, 0.60], Pe log-uniform in [0.1, 1000], mu in {0, 0.5, 1},
    dynamics seed 3000 + r."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ns = rng.integers(n_lo, n_hi + 1, size=R)
    Ns = Ns - (Ns % 2)
    phis = rng.uniform(0.45, 0.60, size=R)
    pes = 10.0 ** rng.uniform(-1.0, 3.0, size=R)
    mus = rng.choice(np.array([0.0, 0.5, 1.0]), size=R)
    return [dict(N=int(Ns[r]), phi=float(phis[r]), pe=float(pes[r]),
                 mu=float(mus[r]), seed=3000 + r) for r in range(R)]


def _make_replica(job):
    r, row, pack_seed, tol, max_sweeps = job
    return make(row["N"], row["phi"], row["pe"], row["mu"],
                pack_seed=pack_seed + 2 * r, dyn_seed=row["seed"], tol=tol,
                name=f"replica{r}", max_sweeps=max_sweeps)


def make_replicas(table, pack_seed: int = 5000, tol: float = 1e-4,
                  max_sweeps: int = 2000, processes: int = 1):
    """One workload per row of ``replica_table``; with processes > 1 the
    packings are made by a pool of freshly spawned interpreters (safe to
    start after CUDA is initialised), with the same results."""
    jobs = [(r, row, pack_seed, tol, max_sweeps) for r, row in enumerate(table)]
    if processes <= 1:
        return [_make_replica(j) for j in jobs]
    import multiprocessing as mp
    build()
    # one OpenMP thread per worker: the pool supplies the parallelism
    prev = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "1"
    try:
        with mp.get_context("spawn").Pool(processes) as pool:
            return pool.map(_make_replica, jobs, chunksize=1)
    finally:
        if prev is None:
            os.environ.pop("OMP_NUM_THREADS", None)
        else:
            os.environ["OMP_NUM_THREADS"] = prev
