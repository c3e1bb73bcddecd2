"""GPU: the deterministic force sums of the FP64 path (deterministic = 1).

With the parameter set, every listed pair writes its shares to its own slot
and every sphere sums its one-body terms, its own row and the slots where it
is the partner in a fixed order, so two runs from the same state, seed and
parameters give bitwise-equal trajectories, forces, histories and stresses
(the atomics of the default path change the summation order, and with it the
last bits, from run to run).  The order differs from the atomic path's, so
against the oracle the same bars hold as for the default FP64 path.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def susp():
    import paper_2307_13802_gb300 as s
    return s


def _kw(w, **extra):
    p = w.params
    kw = dict(precision="fp64", eta=p["eta"], rho=p["rho"], kn=p["kn"], kt=p["kt"],
              mu=p["mu"], xi_min=p["xi_min"], xi_max=p["xi_max"], skin=p["skin"],
              shear_rate=p["shear_rate"], kT=p["kT"], seed=p["seed"],
              torque_sign=p["torque_sign"], dt=p["dt"])
    kw.update(extra)
    return kw


def _relerr(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / scale if scale > 0 else np.abs(a - b).max()


def _run(susp, w, steps, **extra):
    p = w.params
    g = susp.System(w.radii, w.box, **_kw(w, **extra))
    g.set_state(w.x, w.U, w.W)
    g.set_clock(0, 0.45)   # the strain flips within the run
    g.step(steps, p["shear_rate"], p["kT"], p["dt"], p["seed"])
    x, U, W = g.state()
    F, T = g.forces()
    ij, xi = g.history()
    return g, dict(x=x, U=U, W=W, F=F, T=T, ij=ij, xi=xi, stress=g.stress(), info=g.info())


@pytest.mark.parametrize("graphs", [0, 1])
def test_two_runs_are_bitwise_equal(susp, graphs, record):
    # 1,500 frictional spheres, phi = 0.55, Pe = 10, strain flip and several
    # rebuilds: every reverse list is rebuilt along the way
    w = workloads.make(1500, 0.55, 10.0, 1.0, pack_seed=81, dyn_seed=82)
    _, a = _run(susp, w, 1500, deterministic=1, use_graphs=graphs)
    _, b = _run(susp, w, 1500, deterministic=1, use_graphs=graphs)
    assert a["info"]["nbuilds"] >= 3 and a["info"]["strain"] < 0
    assert len(a["ij"]) > 100
    for key in ("x", "U", "W", "F", "T", "ij", "xi"):
        assert np.array_equal(a[key], b[key]), key
    for key in ("contact", "lubrication", "brownian", "kinetic"):
        assert np.array_equal(a["stress"][key], b["stress"][key]), key
    assert a["stress"]["eta_r"] == b["stress"]["eta_r"]
    # the atomic path reaches the same state up to its rounding
    _, c = _run(susp, w, 1500, deterministic=0, use_graphs=graphs)
    # (measured on a GB300: x 3.3e-13, F 2.6e-12)
    record("vs_atomic_x", np.abs(a["x"] - c["x"]).max(), 5e-12)
    record("vs_atomic_F", _relerr(a["F"], c["F"]), 5e-11)
    assert np.abs(a["x"] - c["x"]).max() <= 5e-12
    assert _relerr(a["F"], c["F"]) <= 5e-11


def test_one_evaluation_matches_oracle(susp, record):
    w = workloads.make(700, 0.56, 1.0, 0.5, poly=True, pack_seed=11, dyn_seed=12)
    w.x, w.L = w.x * 0.985, float(w.box[0] * 0.985)
    g = susp.System(w.radii, w.box, **_kw(w, deterministic=1))
    g.set_state(w.x, w.U, w.W)
    g.set_clock(5, 0.37)
    g.evaluate()
    F, T = g.forces()
    sg = g.stress()
    o = oracle.System(w.radii, w.box, **w.params)
    o.set_state(w.x, w.U, w.W)
    o.set_strain(0.37)
    o.set_k(5)
    o.evaluate()
    Fo, To = o.forces()
    so = o.stress()
    assert o.info()["ncontacts"] > 10
    record("force", _relerr(F, Fo), 1e-13)
    record("torque", _relerr(T, To), 1e-13)
    assert _relerr(F, Fo) <= 1e-13 and _relerr(T, To) <= 1e-13
    for key in ("contact", "lubrication", "brownian"):
        assert _relerr(sg[key], so[key]) <= 1e-13, key


def test_trajectory_matches_oracle(susp, record):
    # the bars of the default FP64 trajectory test: 500 frictional spheres,
    # phi = 0.5, Pe = 10, ten chunks of 100 steps
    w = workloads.make(500, 0.50, 10.0, 1.0, pack_seed=1001, dyn_seed=2001)
    p = w.params
    g = susp.System(w.radii, w.box, **_kw(w, deterministic=1))
    g.set_state(w.x, w.U, w.W)
    o = oracle.System(w.radii, w.box, **p)
    o.set_state(w.x, w.U, w.W)
    errs, serr = [], 0.0
    for _ in range(10):
        g.step(100, p["shear_rate"], p["kT"], p["dt"], p["seed"])
        o.step(100)
        F, T = g.forces()
        Fo, To = o.forces()
        errs.append(max(_relerr(F, Fo), _relerr(T, To)))
        n, so = o.take_stress_sums()
        sg = g.stress()
        assert sg["samples"] == n == 100
        for key in ("contact", "lubrication", "brownian"):
            serr = max(serr, _relerr(sg[key], so[key] / n))
    record("first_chunk_force", errs[0], 5e-12)
    record("max_chunk_force", max(errs), 5e-11)
    record("stress_avg", serr, 2e-11)
    assert errs[0] <= 5e-12 and max(errs) <= 5e-11 and serr <= 2e-11


def test_batch_runs_are_bitwise_equal(susp):
    rows = [dict(N=300, phi=0.45, pe=1000.0, mu=0.0), dict(N=520, phi=0.55, pe=10.0, mu=1.0),
            dict(N=410, phi=0.50, pe=0.5, mu=0.5)]
    ws = [workloads.make(r["N"], r["phi"], r["pe"], r["mu"], pack_seed=900 + i,
                         dyn_seed=910 + i) for i, r in enumerate(rows)]
    out = []
    for _ in range(2):
        bt = susp.System.batch([w.N for w in ws], np.concatenate([w.radii for w in ws]),
                               np.stack([w.box for w in ws]),
                               [_kw(w, deterministic=1) for w in ws])
        bt.set_state(np.concatenate([w.x for w in ws]), np.concatenate([w.U for w in ws]),
                     np.concatenate([w.W for w in ws]))
        bt.step_batch(400, ws[0].params["dt"])
        out.append((bt.state(), bt.forces(), [bt.stress(r)["eta_r"] for r in range(len(ws))]))
    (sa, fa, ea), (sb, fb, eb) = out
    for u, v in zip(sa + fa, sb + fb):
        assert np.array_equal(u, v)
    assert ea == eb


def test_mixed_precision_rejects_it(susp):
    w = workloads.make(300, 0.45, 10.0, 0.0, pack_seed=5)
    with pytest.raises(susp.SuspError) as e:
        susp.System(w.radii, w.box, **_kw(w, precision="mixed", deterministic=1))
    assert e.value.code == susp.SUSP_EINVAL


def test_a_grown_row_capacity_gives_the_same_bits(susp):
    # the capacity grows from 6 at the first build; the rows, and the order
    # of every deterministic sum, are those of a handle created with 48
    w = workloads.make(1500, 0.55, 10.0, 1.0, pack_seed=83, dyn_seed=84)
    out = []
    for kmax in (6, 48):
        _, r = _run(susp, w, 300, deterministic=1, kmax=kmax)
        out.append(r)
    a, b = out
    assert a["info"]["kmax"] > 6 and b["info"]["kmax"] == 48
    for key in ("x", "U", "W", "F", "T", "ij", "xi"):
        assert np.array_equal(a[key], b[key]), key
