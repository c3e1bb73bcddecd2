"""A reduced flow-curve campaign (Sec. IV.D, Table 1 protocol; Fig. 6(b)
friction axis) run by the harness as one batch handle, each state point
checked against an oracle ensemble of the same packings with other noise
seeds: 3 Peclet numbers x 2 friction coefficients x 6 realisations of 500
equal-volume bidisperse spheres at phi 0.5, 6,000 steps after 1,000.  The
means must agree within four standard errors of their difference (six state
points with three quantities each)."""
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

PES, MUS, REAL, N, PHI, STEPS, BURN = (0.5, 5.0, 50.0), (0.0, 1.0), 6, 500, 0.5, 6000, 1000


def _oracle_point(job):
    import oracle
    from paper_2307_13802_gb300 import flowcurve
    rep, seed = job
    p = flowcurve.replica_params(rep)
    o = oracle.System(rep.radii, [rep.L] * 3,
                      **{k: p[k] for k in ("eta", "rho", "kn", "kt", "mu", "skin",
                                           "shear_rate", "kT", "dt")}, seed=seed)
    x = rep.x
    U = np.zeros_like(x)
    W = np.zeros_like(x)
    U[:, 0] = p["shear_rate"] * (x[:, 1] - 0.5 * rep.L)
    W[:, 2] = -0.5 * p["shear_rate"]
    o.set_state(x, U, W)
    o.step(BURN)
    o.take_stress_sums()
    o.step(STEPS)
    n, s = o.take_stress_sums()
    sig = (s["contact"] + s["lubrication"]) / n
    rate = p["shear_rate"]
    eta_r = (sig[0, 1] + oracle.drag_stress_xy(rep.radii, [rep.L] * 3, 1.0, rate)) / rate
    return eta_r, sig[0, 0] - sig[1, 1], sig[1, 1] - sig[2, 2]


def test_reduced_flow_curve_matches_the_oracle_ensemble(record):
    import concurrent.futures as cf
    import multiprocessing as mp

    from paper_2307_13802_gb300 import flowcurve

    reps = flowcurve.make_campaign(PES, MUS, REAL, N, PHI)
    assert len(reps) == len(PES) * len(MUS) * REAL
    results, per = flowcurve.run(reps, STEPS, BURN, blocks=6, precision="fp64")
    os.environ["OMP_NUM_THREADS"] = "1"
    with cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1),
                                mp_context=mp.get_context("spawn")) as ex:
        ref = list(ex.map(_oracle_point, [(r, 50_000 + i) for i, r in enumerate(reps)]))
    ref = np.array(ref)
    for res in results:
        idx = [i for i, r in enumerate(reps) if (r.pe, r.mu) == (res["pe"], res["mu"])]
        o = ref[idx]
        assert res["realisations"] == len(idx) == REAL
        for c, name in enumerate(("eta_r", "N1", "N2")):
            mo = o[:, c].mean()
            se = math.sqrt(res[f"{name}_se"] ** 2 + o[:, c].var(ddof=1) / len(idx))
            print(f"Pe {res['pe']} mu {res['mu']} {name}: harness {res[name]:.4f} "
                  f"+- {res[name + '_se']:.4f}, oracle {mo:.4f}")
            record(f"pe{res['pe']}_mu{res['mu']}_{name}_diff_over_se", abs(res[name] - mo) / se, 4.0)
            assert abs(res[name] - mo) <= 4.0 * se, (res, name, mo, se)
    # the realisations' own block-average errors are reported with each point
    assert all(r["eta_r_block_se"] > 0 for r in results)
