"""GPU parity of the optional terms against the FP64 oracle: the short-range
repulsion (Eq. 34), the structural Brownian stress (Eq. 26) with its
per-sample series, and the Green-Kubo integral (Eq. 33).

Same bars as the core parity tests: the FP64 path evaluates the oracle's
expressions (no multiply-add contraction; reciprocal products in the
resistances, a few ulps) and otherwise differs only in the summation order,
so one evaluation agrees to 1e-11 of the largest entry and the
neighbour sets, decided by the same double expression, agree exactly.  The
shell counts of Eq. 26 are integer decisions on the same double gap, so the
structural stress agrees to the same 1e-11.  The mixed path forms gaps and
the repulsion in single precision (noise off): forces within 2e-5 of FP64."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

RTOL_FP64 = 1e-11
EXTRA = dict(rep_A=5.0, rep_cut=10.0, structural=1, shell=0.05)


@pytest.fixture(scope="module")
def susp():
    import paper_2307_13802_gb300 as s
    return s


def _gpu(susp, w, **kw):
    p = dict(w.params)
    args = dict(precision="fp64", eta=p["eta"], rho=p["rho"], kn=p["kn"], kt=p["kt"],
                mu=p["mu"], xi_min=p["xi_min"], xi_max=p["xi_max"], skin=p["skin"],
                shear_rate=p["shear_rate"], kT=p["kT"], seed=p["seed"],
                torque_sign=p["torque_sign"], dt=p["dt"])
    args.update(kw)
    return susp.System(w.radii, w.box, **args)


def _relerr(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / scale if scale > 0 else np.abs(a - b).max()


CASES = [dict(N=500, phi=0.50, pe=10.0, mu=1.0, poly=False),
         dict(N=700, phi=0.56, pe=1.0, mu=0.5, poly=True)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"N{c['N']}-poly{c['poly']}")
@pytest.mark.parametrize("strain", [0.0, -0.41])
def test_one_evaluation_with_repulsion_and_structural_stress(susp, case, strain):
    w = workloads.make(case["N"], case["phi"], case["pe"], case["mu"], poly=case["poly"],
                       pack_seed=13, dyn_seed=14)
    w.x, w.L = w.x * 0.99, w.L * 0.99
    g = _gpu(susp, w, **EXTRA)
    g.set_state(w.x, w.U, w.W)
    g.set_clock(5, strain)
    g.evaluate()
    F, T = g.forces()
    sg = g.stress()
    o = oracle.System(w.radii, w.box, **dict(w.params, **EXTRA))
    o.set_state(w.x, w.U, w.W)
    o.set_strain(strain)
    o.set_k(5)
    o.evaluate()
    Fo, To = o.forces()
    so = o.stress()
    assert np.abs(so["repulsion"]).max() > 0 and np.abs(so["structural"]).max() > 0
    assert _relerr(F, Fo) <= RTOL_FP64
    assert _relerr(T, To) <= RTOL_FP64
    for key in ("contact", "lubrication", "brownian", "repulsion", "structural"):
        assert _relerr(sg[key], so[key]) <= RTOL_FP64, key


@pytest.mark.parametrize("extra", [dict(rep_A=1.0, rep_cut=10.0), dict(structural=1, shell=0.05)],
                         ids=["repulsion", "structural"])
def test_widened_neighbour_list_is_brute_force_exactly(susp, extra):
    w = workloads.make(2000, 0.55, 10.0, 0.0, poly=True, pack_seed=23)
    g = _gpu(susp, w, **extra)
    g.set_state(w.x, w.U, w.W)
    g.set_clock(0, 0.3)
    g.build_neighbors()
    o = oracle.System(w.radii, w.box, **dict(w.params, **extra))
    o.set_state(w.x, w.U, w.W)
    o.set_strain(0.3)
    bp = o.brute_pairs()
    base = oracle.System(w.radii, w.box, **w.params)
    base.set_state(w.x, w.U, w.W)
    base.set_strain(0.3)
    assert len(bp) > len(base.brute_pairs())      # the range did widen
    assert np.array_equal(g.pairs(), bp)


def test_trajectory_with_repulsion_and_series(susp):
    # 400 sheared steps with repulsion, friction and noise; the structural
    # stress of every step is recorded on the GPU and compared with the
    # oracle's step by step
    w = workloads.make(500, 0.52, 10.0, 1.0, pack_seed=33, dyn_seed=34)
    p = dict(w.params, **EXTRA)
    g = _gpu(susp, w, series_cap=1000, **EXTRA)
    g.set_state(w.x, w.U, w.W)
    o = oracle.System(w.radii, w.box, **p)
    o.set_state(w.x, w.U, w.W)
    so_series = []
    for _ in range(400):
        o.step(1)
        so_series.append(o.stress()["structural"][0, 1])
    g.step(400, p["shear_rate"], p["kT"], p["dt"], p["seed"])
    F, T = g.forces()
    Fo, To = o.forces()
    assert _relerr(F, Fo) <= 1e-8 and _relerr(T, To) <= 1e-8
    series, dropped = g.series()
    assert dropped == 0 and len(series) == 400
    so_series = np.array(so_series)
    assert np.abs(so_series).max() > 0
    assert np.abs(series - so_series).max() <= 1e-8 * np.abs(so_series).max()
    n, sums = o.take_stress_sums()
    sg = g.stress()
    assert sg["samples"] == n == 400
    for key in ("repulsion", "structural", "contact"):
        assert _relerr(sg[key], sums[key] / n) <= 1e-8, key
    # the record was reset by the read; capacity overflow is counted
    g.step(10, p["shear_rate"], p["kT"], p["dt"], p["seed"])
    s2, d2 = g.series()
    assert len(s2) == 10 and d2 == 0


def test_series_capacity_and_reset(susp):
    w = workloads.make(300, 0.45, 10.0, 0.0, pack_seed=35, dyn_seed=36)
    p = w.params
    g = _gpu(susp, w, series_cap=50, structural=1)
    g.set_state(w.x, w.U, w.W)
    g.step(70, p["shear_rate"], p["kT"], p["dt"], p["seed"])
    s, dropped = g.series()
    assert len(s) == 50 and dropped == 20
    s, dropped = g.series()
    assert len(s) == 0 and dropped == 0
    plain = _gpu(susp, w)
    plain.set_state(w.x, w.U, w.W)
    with pytest.raises(susp.SuspError, match="no series"):
        plain.series()


def test_green_kubo_matches_the_oracle(susp):
    rng = np.random.Generator(np.random.PCG64(5))
    n, rho = 20_000, 0.95
    x = np.empty(n)
    x[0] = rng.standard_normal()
    for t in range(1, n):
        x[t] = rho * x[t - 1] + np.sqrt(1 - rho * rho) * rng.standard_normal()
    dt, V, kT, M = 0.02, 3.0, 0.7, 300
    Cg, eg, fg = susp.green_kubo(x, M, dt, V, kT)
    Co, eo = oracle.green_kubo(x, M, dt, V, kT)
    fo = oracle.gk_fit(eo, dt)
    assert _relerr(Cg, Co) <= 1e-12
    assert _relerr(eg, eo) <= 1e-12
    assert fg[1] == fo[1]                       # the same grid point
    assert fg[0] == pytest.approx(fo[0], rel=1e-10)


def test_mixed_path_with_repulsion_and_structural_stress(susp):
    w = workloads.make(3000, 0.58, 1000.0, 1.0, pack_seed=53, dyn_seed=54)
    w.x, w.L = w.x * 0.99, w.L * 0.99
    res = {}
    for prec in ("fp64", "mixed"):
        g = _gpu(susp, w, precision=prec, noise=0, **EXTRA)
        g.set_state(w.x, w.U, w.W)
        g.set_clock(3, 0.17)
        g.evaluate()
        res[prec] = (g.forces(), g.stress())
    (F64, T64), s64 = res["fp64"]
    (F32, T32), s32 = res["mixed"]
    assert _relerr(F32, F64) <= 2e-5
    assert _relerr(T32, T64) <= 2e-5
    assert _relerr(s32["repulsion"], s64["repulsion"]) <= 2e-5
    # shell decisions on single-precision gaps: a pair within rounding of a
    # shell edge may be counted differently
    assert _relerr(s32["structural"], s64["structural"]) <= 1e-3
