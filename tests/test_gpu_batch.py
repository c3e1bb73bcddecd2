"""Batched replicas: one handle stepping several independent systems of
uneven size, volume fraction, Peclet number and friction gives each replica
the run a handle of its own gives it.

The replicas share kernels and launches but no data: each has its own box,
cell grid, strain, noise key and stress sums, and its particles are never
paired with another replica's.  The per-replica results therefore equal
those of separate handles up to the order of the force sums (atomics), the
same bar as two runs of one handle.  Bars are about 10 times the largest
difference measured on a GB300 over 200 steps (seven runs): FP64 x 8e-15,
U 1.4e-13, F 4.4e-13; mixed (single-precision force atomics) x 4.5e-8,
U 1.2e-6, F 4.5e-6 of the largest entry.  The mixed maxima are heavy-tailed
from run to run (1.6e-7 to 4.5e-6 in F): the noisiest replica (Pe 0.5)
amplifies a different order of the float atomics, and a pair that enters
the cutoff or touches one step apart moves the largest force entry."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

ROWS = [dict(N=300, phi=0.45, pe=1000.0, mu=0.0, seed=71),
        dict(N=520, phi=0.55, pe=10.0, mu=1.0, seed=72),
        dict(N=410, phi=0.50, pe=0.5, mu=0.5, seed=73)]
# (x absolute, U relative to its largest entry, F normwise)
TOL = {"fp64": (1e-13, 3e-12, 5e-12), "mixed": (5e-7, 1e-5, 5e-5)}


def _kw(w, precision):
    p = w.params
    return dict(precision=precision, eta=p["eta"], rho=p["rho"], kn=p["kn"], kt=p["kt"],
                mu=p["mu"], xi_min=p["xi_min"], xi_max=p["xi_max"], skin=p["skin"],
                shear_rate=p["shear_rate"], kT=p["kT"], seed=p["seed"],
                torque_sign=p["torque_sign"], dt=p["dt"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_separate_handles(precision, record):
    import paper_2307_13802_gb300 as susp

    ws = [workloads.make(r["N"], r["phi"], r["pe"], r["mu"], pack_seed=700 + i,
                         dyn_seed=r["seed"]) for i, r in enumerate(ROWS)]
    steps, dt = 200, ws[0].params["dt"]
    sizes = [w.N for w in ws]
    bt = susp.System.batch(sizes, np.concatenate([w.radii for w in ws]),
                           np.stack([w.box for w in ws]), [_kw(w, precision) for w in ws])
    bt.set_state(np.concatenate([w.x for w in ws]), np.concatenate([w.U for w in ws]),
                 np.concatenate([w.W for w in ws]))
    bt.step_batch(steps, dt)
    xb, Ub, Wb = bt.state()
    Fb, Tb = bt.forces()
    tx, tu, tf = TOL[precision]
    off = np.concatenate([[0], np.cumsum(sizes)])
    for r, w in enumerate(ws):
        p = w.params
        g = susp.System(w.radii, w.box, **_kw(w, precision))
        g.set_state(w.x, w.U, w.W)
        g.step(steps, p["shear_rate"], p["kT"], dt, p["seed"])
        x, U, W = g.state()
        F, T = g.forces()
        sl = slice(off[r], off[r + 1])
        record(f"r{r}_x", np.abs(xb[sl] - x).max(), tx)
        record(f"r{r}_U", np.abs(Ub[sl] - U).max() / np.abs(U).max(), tu)
        record(f"r{r}_F", np.abs(Fb[sl] - F).max() / np.abs(F).max(), tf)
        record(f"r{r}_T", np.abs(Tb[sl] - T).max() / np.abs(T).max(), tf)
        assert np.abs(xb[sl] - x).max() <= tx, r
        assert np.abs(Ub[sl] - U).max() <= tu * np.abs(U).max(), r
        assert np.abs(Fb[sl] - F).max() <= tf * np.abs(F).max(), r
        assert np.abs(Tb[sl] - T).max() <= tf * np.abs(T).max(), r
        sg, sb = g.stress(), bt.stress(r)
        assert sb["samples"] == sg["samples"]
        for key in ("contact", "lubrication", "brownian", "kinetic"):
            scale = np.abs(sg[key]).max()
            assert np.abs(sb[key] - sg[key]).max() <= 10 * tf * max(scale, 1e-300), (r, key)
        assert sb["eta_r"] == pytest.approx(sg["eta_r"], rel=10 * tf)
