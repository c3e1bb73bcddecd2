"""Flow-curve campaigns in one batch handle (Sec. IV.D, Table 1; Sec. II.E).

The paper measures the relative viscosity eta_r(Pe) of bidisperse
suspensions (radii a and 1.4a, mixed about equally by volume, Sec. II.E)
over Peclet numbers Pe = 6 pi eta a^3 rate / kT (Sec. II.F), with the
friction coefficient as a second axis (Fig. 6(b)), averaging each state point
over 10-800 realisations (Sec. II.E).  Table 1 fixes how Pe is varied: below
Pe = 1 the shear rate changes at a fixed thermal energy, above it the thermal
energy changes at a fixed shear rate.

This module lays such a campaign out as replicas of one batch handle of the
library -- every (Pe, mu, realisation) is one replica with its own packing,
shear rate, kT, friction and noise seed -- steps them together and reduces
the library's own stress averages (susp_stress) into eta_r, N1 and N2 per
state point, with error bars from the spread over realisations and, per
realisation, from block averages over time.  It does no arithmetic of the
model itself.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def table1_point(pe: float, rate0: float = 1.0, eta: float = 1.0, a: float = 1.0):
    """(shear rate, kT) of Peclet number pe under the protocol of Table 1:
    Pe = 1 at the shear rate rate0 and kT0 = 6 pi eta a^3 rate0; below it
    the rate is pe * rate0 at kT0, above it the rate is rate0 at kT0 / pe."""
    kT0 = 6.0 * math.pi * eta * a ** 3 * rate0
    if pe < 1.0:
        return pe * rate0, kT0
    return rate0, kT0 / pe


def equal_volume_counts(N: int, a_small: float = 1.0, a_large: float = 1.4):
    """Numbers of small and large spheres of total N whose volumes are as
    equal as integers allow: (a_large / a_small)^3 small spheres per large
    one (2.744 for radii 1 and 1.4)."""
    ratio = (a_large / a_small) ** 3
    n_large = int(round(N / (1.0 + ratio)))
    return N - n_large, n_large


@dataclass
class Replica:
    """One realisation: a packing (radii [N], cubic box edge L, positions
    [N][3]) at one state point."""
    pe: float
    mu: float
    radii: np.ndarray
    L: float
    x: np.ndarray
    seed: int


def replica_params(rep: Replica, rate0: float = 1.0, eta: float = 1.0, rho: float = 1.0,
                   kn: float = 1e4, kt_ratio: float = 0.5, dt: float = 1e-4,
                   skin: float = 0.3, precision: str = "mixed", **extra) -> dict:
    """susp_params of a replica: Table 1's rate and kT for its Pe, k_t =
    kt_ratio k_n when it has friction."""
    rate, kT = table1_point(rep.pe, rate0, eta)
    return dict(precision=precision, eta=eta, rho=rho, kn=kn,
                kt=kt_ratio * kn if rep.mu > 0 else 0.0, mu=rep.mu, skin=skin,
                shear_rate=rate, kT=kT, seed=rep.seed, dt=dt, **extra)


def run(replicas, steps: int, burn: int, blocks: int = 10, dt: float = 1e-4,
        stream=None, **param_kw):
    """Steps every replica of the campaign in one batch handle: `burn` steps
    whose stresses are dropped, then `steps` steps in `blocks` equal blocks,
    each block's stress average read per replica.  Returns (per-state-point
    results, per-replica block means).  Each state point (Pe, mu) gets the
    mean over its realisations of eta_r, N1 and N2 (each realisation's time
    average), the standard error of that mean from the spread over the
    realisations, and the mean of the realisations' own block-average errors
    (the standard deviation of the block means over sqrt(blocks))."""
    import paper_2307_13802_gb300 as susp

    if steps % blocks:
        raise ValueError("steps must be a multiple of blocks")
    sizes = [len(r.radii) for r in replicas]
    boxes = np.array([[r.L, r.L, r.L] for r in replicas])
    params = [replica_params(r, dt=dt, **param_kw) for r in replicas]
    h = susp.System.batch(sizes, np.concatenate([r.radii for r in replicas]), boxes, params)
    if stream is not None:
        h.set_stream(stream)
    x = np.concatenate([r.x for r in replicas])
    U = np.zeros_like(x)
    W = np.zeros_like(x)
    off = 0
    for r, p in zip(replicas, params):
        n = len(r.radii)
        # start in the imposed flow: U = rate (y - L/2) x, Omega = -rate/2 z
        U[off:off + n, 0] = p["shear_rate"] * (r.x[:, 1] - 0.5 * r.L)
        W[off:off + n, 2] = -0.5 * p["shear_rate"]
        off += n
    h.set_state(x, U, W)
    R = len(replicas)
    if burn > 0:
        h.step_batch(burn, dt)
    for r in range(R):
        h.stress(r)
    per = np.zeros((R, blocks, 3))
    for blk in range(blocks):
        h.step_batch(steps // blocks, dt)
        for r in range(R):
            s = h.stress(r)
            per[r, blk] = (s["eta_r"], s["N1"], s["N2"])
    h.close()
    points = {}
    for r, rep in enumerate(replicas):
        points.setdefault((rep.pe, rep.mu), []).append(r)
    results = []
    for (pe, mu), idx in sorted(points.items()):
        tav = per[idx].mean(axis=1)                       # [realisations][3]
        blk_se = per[idx].std(axis=1, ddof=1) / math.sqrt(blocks) if blocks > 1 else None
        n = len(idx)
        se = tav.std(axis=0, ddof=1) / math.sqrt(n) if n > 1 else np.full(3, np.nan)
        rate, kT = table1_point(pe, param_kw.get("rate0", 1.0), param_kw.get("eta", 1.0))
        res = dict(pe=pe, mu=mu, rate=rate, kT=kT, realisations=n,
                   eta_r=float(tav[:, 0].mean()), eta_r_se=float(se[0]),
                   N1=float(tav[:, 1].mean()), N1_se=float(se[1]),
                   N2=float(tav[:, 2].mean()), N2_se=float(se[2]))
        if blk_se is not None:
            res["eta_r_block_se"] = float(blk_se[:, 0].mean())
        results.append(res)
    return results, per


def make_campaign(pes, mus, realisations: int, N: int, phi: float, seed: int = 9100,
                  a_small: float = 1.0, a_large: float = 1.4):
    """Replicas of a campaign from the repository's seeded packing generator
    (``workloads``): equal-volume bidisperse packings of N spheres at volume
    fraction phi, one packing and one noise seed per realisation, the same
    packings at every state point."""
    import workloads

    ns, nl = equal_volume_counts(N, a_small, a_large)
    packs = []
    for k in range(realisations):
        rng = np.random.Generator(np.random.PCG64(seed + 17 * k))
        radii = np.concatenate([np.full(ns, a_small), np.full(nl, a_large)])
        rng.shuffle(radii)
        L = workloads.box_for_phi(radii, phi)
        x, _ = workloads.packing(radii, L, seed + 17 * k + 1, tol=1e-3)
        packs.append((radii, L, x))
    reps = []
    for pe in pes:
        for mu in mus:
            for k, (radii, L, x) in enumerate(packs):
                reps.append(Replica(pe=float(pe), mu=float(mu), radii=radii, L=L, x=x,
                                    seed=seed + 1000 + len(reps)))
    return reps


def main(argv=None):
    """python -m paper_2307_13802_gb300.flowcurve: a flow curve printed as
    one JSON line per state point."""
    import argparse
    import json

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--pe", type=float, nargs="+", default=[0.1, 1.0, 10.0, 100.0, 1000.0])
    ap.add_argument("--mu", type=float, nargs="+", default=[0.0, 0.5, 1.0])
    ap.add_argument("--realisations", type=int, default=16)
    ap.add_argument("--N", type=int, default=1000)
    ap.add_argument("--phi", type=float, default=0.55)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--burn", type=int, default=10000)
    ap.add_argument("--blocks", type=int, default=10)
    ap.add_argument("--precision", choices=("mixed", "fp64"), default="mixed")
    a = ap.parse_args(argv)
    reps = make_campaign(a.pe, a.mu, a.realisations, a.N, a.phi)
    results, _ = run(reps, a.steps, a.burn, a.blocks, precision=a.precision)
    for r in results:
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
