"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle
on the same seeded inputs.

Tolerances: the FP64 pair kernel evaluates the oracle's expressions with
multiply-adds contracted (one rounding instead of two) and with reciprocal
products in place of the printed quotients of the resistances and the unit
vector (a few ulps); beyond that they differ only in the last bits of log,
sin, cos (CUDA vs libm) and in the order of the force sums (atomics).  The
required agreement of one evaluation is 1e-11 relative to the largest entry
of the same quantity (normwise); measured, forces, torques and stresses
agree to a few 1e-15, and the bar is set at 1e-13.  Neighbour sets, which are
decided by the same d^2 < r_list^2 expression, agree exactly.

Bars of the longer runs are 10-20 times the largest error measured on a
GB300 (the atomics change the summation order from run to run, and the
trajectories amplify rounding): forces agree to 2.6e-13 after 100 steps
(bar 5e-12) and 3.5e-12 after 1,000 (bar 5e-11), the time-averaged stresses
to 1.0e-12 (bar 2e-11); the tangential history after 300 frictional steps to
3.9e-13 (bar 5e-12)."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

RTOL_FP64 = 1e-13


@pytest.fixture(scope="module")
def susp():
    import paper_2307_13802_gb300 as s
    return s


def _gpu_system(susp, w, **kw):
    p = dict(w.params)
    args = dict(precision=kw.pop("precision", "fp64"), eta=p["eta"], rho=p["rho"],
                kn=p["kn"], kt=p["kt"], mu=p["mu"], xi_min=p["xi_min"],
                xi_max=p["xi_max"], skin=p["skin"], shear_rate=p["shear_rate"],
                kT=p["kT"], seed=p["seed"], torque_sign=p["torque_sign"], dt=p["dt"])
    args.update(kw)
    return susp.System(w.radii, w.box, **args)


def _relerr(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / scale if scale > 0 else np.abs(a - b).max()


CASES = [
    dict(N=500, phi=0.50, pe=10.0, mu=0.0, poly=False),
    dict(N=500, phi=0.50, pe=10.0, mu=1.0, poly=False),
    dict(N=700, phi=0.56, pe=1.0, mu=0.5, poly=True),
    dict(N=300, phi=0.45, pe=1000.0, mu=0.0, poly=False),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"N{c['N']}-phi{c['phi']}-pe{c['pe']}-mu{c['mu']}")
@pytest.mark.parametrize("strain", [0.0, 0.37, -0.49])
def test_one_evaluation_matches_oracle(susp, case, strain, record):
    w = workloads.make(case["N"], case["phi"], case["pe"], case["mu"], poly=case["poly"],
                       pack_seed=11, dyn_seed=12)
    # compress a little so that many pairs overlap
    x = w.x * 0.985
    box = w.box * 0.985
    w.x, w.L = x, float(box[0])
    g = _gpu_system(susp, w)
    g.set_state(w.x, w.U, w.W)
    g.set_clock(5, strain)
    g.evaluate()
    F, T = g.forces()
    sg = g.stress()
    o = oracle.System(w.radii, w.box, **w.params)
    o.set_state(w.x, w.U, w.W)
    o.set_strain(strain)
    o.set_k(5)
    o.evaluate()
    Fo, To = o.forces()
    so = o.stress()
    assert o.info()["ncontacts"] > 10
    record("force", _relerr(F, Fo), RTOL_FP64)
    record("torque", _relerr(T, To), RTOL_FP64)
    for key in ("contact", "lubrication", "brownian"):
        record(key, _relerr(sg[key], so[key]), RTOL_FP64)
    assert _relerr(F, Fo) <= RTOL_FP64
    assert _relerr(T, To) <= RTOL_FP64
    for key in ("contact", "lubrication", "brownian"):
        assert _relerr(sg[key], so[key]) <= RTOL_FP64, key
    assert sg["samples"] == 1


@pytest.mark.parametrize("poly", [False, True])
@pytest.mark.parametrize("strain", [0.0, 0.21, 0.5, -0.33])
def test_neighbour_list_is_brute_force_exactly(susp, poly, strain):
    w = workloads.make(2000, 0.55, 10.0, 0.0, poly=poly, pack_seed=21)
    g = _gpu_system(susp, w)
    g.set_state(w.x, w.U, w.W)
    g.set_clock(0, strain)
    g.build_neighbors()
    ij = g.pairs()
    o = oracle.System(w.radii, w.box, **w.params)
    o.set_state(w.x, w.U, w.W)
    o.set_strain(strain)
    bp = o.brute_pairs()
    assert len(ij) == len(bp)
    assert np.array_equal(ij, bp)


def test_neighbour_list_after_shearing_is_brute_force(susp):
    # positions evolved on the GPU through several rebuilds and a flip
    w = workloads.make(1500, 0.5, 10.0, 0.0, pack_seed=31, dyn_seed=32)
    g = _gpu_system(susp, w)
    g.set_state(w.x, w.U, w.W)
    g.set_clock(0, 0.45)
    g.step(1500, 1.0, w.params["kT"], 1e-4, 5)
    info = g.info()
    assert info["nbuilds"] >= 2
    assert info["strain"] < 0          # flipped
    x, U, W = g.state()
    g.build_neighbors()
    ij = g.pairs()
    o = oracle.System(w.radii, w.box, **w.params)
    o.set_state(x, U, W)
    o.set_strain(info["strain"])
    assert np.array_equal(ij, o.brute_pairs())


@pytest.mark.parametrize("graphs", [0, 1])
@pytest.mark.parametrize("mu", [0.0, 1.0])
def test_trajectory_parity_500_spheres(susp, graphs, mu, record):
    # 500 bidisperse spheres, phi = 0.5, Pe = 10: 1000 steps of 1e-4 on both
    w = workloads.make(500, 0.50, 10.0, mu, pack_seed=1001, dyn_seed=2001)
    p = w.params
    g = _gpu_system(susp, w, use_graphs=graphs)
    g.set_state(w.x, w.U, w.W)
    o = oracle.System(w.radii, w.box, **p)
    o.set_state(w.x, w.U, w.W)
    errs = []
    serr = 0.0
    for chunk in range(10):
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
            assert _relerr(sg[key], so[key] / n) <= 2e-11, (chunk, key)
    print("per-chunk max relative force error:", ["%.1e" % e for e in errs])
    record("first_chunk_force", errs[0], 5e-12)
    record("max_chunk_force", max(errs), 5e-11)
    record("stress_avg", serr, 2e-11)
    assert errs[0] <= 5e-12
    assert max(errs) <= 5e-11
    if graphs:
        assert g.info()["graph_steps"] > 0


def test_friction_history_parity(susp, record):
    w = workloads.make(600, 0.55, 100.0, 1.0, pack_seed=41, dyn_seed=42)
    p = w.params
    g = _gpu_system(susp, w)
    g.set_state(w.x, w.U, w.W)
    o = oracle.System(w.radii, w.box, **p)
    o.set_state(w.x, w.U, w.W)
    g.step(300, p["shear_rate"], p["kT"], p["dt"], p["seed"])
    o.step(300)
    ij, xi = g.history()
    oij, ohist, ocontact = o.verlet_list()
    sel = ocontact.astype(bool)
    assert len(ij) == sel.sum() > 20
    assert np.array_equal(ij, oij[sel])
    F, T = g.forces()
    Fo, To = o.forces()
    record("history", _relerr(xi, ohist[sel]), 5e-12)
    record("force", _relerr(F, Fo), 5e-12)
    record("torque", _relerr(T, To), 5e-12)
    assert _relerr(xi, ohist[sel]) <= 5e-12
    assert _relerr(F, Fo) <= 5e-12 and _relerr(T, To) <= 5e-12


def test_errors_are_reported(susp):
    w = workloads.make(500, 0.5, 10.0, 0.0, pack_seed=61)
    g = _gpu_system(susp, w, kmax=2)
    g.set_state(w.x, w.U, w.W)
    with pytest.raises(susp.SuspError) as e:
        g.build_neighbors()
    assert e.value.code == susp.SUSP_ENEIGH
    g2 = _gpu_system(susp, w)
    x = w.x.copy()
    x[7, 1] = np.nan
    with pytest.raises(susp.SuspError) as e:
        g2.set_state(x, w.U, w.W)
    assert e.value.code == susp.SUSP_EUNSTABLE
    with pytest.raises(susp.SuspError) as e:
        susp.System(w.radii, [5.0, 5.0, 5.0])
    assert e.value.code == susp.SUSP_EINVAL
    g3 = _gpu_system(susp, w)
    with pytest.raises(susp.SuspError) as e:
        g3.step(1, 1.0, 1.0, 1e-4, 0)
    assert e.value.code == susp.SUSP_ESTATE


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_row_capacity_grows_and_the_run_is_unchanged(susp, precision, record):
    # rows of up to ~12 entries at phi = 0.55: a capacity of 6 overflows at
    # the first build, grows before any step, and the run then follows a
    # run created with the default capacity (the rows hold the same pairs in
    # the same order; only the order of the force atomics differs)
    w = workloads.make(1500, 0.55, 10.0, 1.0, pack_seed=81, dyn_seed=82)
    p = w.params
    runs = {}
    for kmax in (6, 48):
        g = _gpu_system(susp, w, precision=precision, kmax=kmax)
        g.set_state(w.x, w.U, w.W)
        g.step(300, p["shear_rate"], p["kT"], p["dt"], p["seed"])
        x, _, _ = g.state()
        F, _ = g.forces()
        runs[kmax] = (x, F, g.info(), g.history()[0])
    (xs, Fs, infs, ijs), (xd, Fd, infd, ijd) = runs[6], runs[48]
    assert infd["max_row"] > 6 and infd["kmax"] == 48
    assert infs["kmax"] > max(6, infs["max_row"])
    assert np.array_equal(ijs, ijd)
    # FP64: atomics order only; mixed: its float atomics, as between a batch
    # and separate handles (measured on a GB300: FP64 x 1.4e-14, F 4.3e-13;
    # mixed x 6.5e-9, F 1.1e-7)
    tx, tf = (1e-12, 1e-11) if precision == "fp64" else (1e-7, 5e-6)
    record("x", np.abs(xs - xd).max(), tx)
    record("F", _relerr(Fs, Fd), tf)
    assert np.abs(xs - xd).max() <= tx
    assert _relerr(Fs, Fd) <= tf
