"""Mixed-precision path against the FP64 path of the same library (which is
itself pinned to the oracle to 1e-11).

With the noise switched off both paths integrate the same deterministic
equations; the mixed one forms pair quantities in single precision
(relative rounding ~6e-8, a few ulps through the resistances) on gaps that
carry ~1e-7 absolute error, and accumulates forces in single precision.  One
evaluation therefore agrees to ~1e-5 of the largest force; short
trajectories agree to the same order.  With noise on the two paths draw the
same Philox words but map them to Gaussians in different precision, so they
are compared statistically (temperature) rather than element by element."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

# one evaluation: measured <= 5.8e-7 of the largest entry on a GB300
RTOL_MIXED = 1e-5


@pytest.fixture(scope="module")
def susp():
    import paper_2307_13802_gb300 as s
    return s


def _sys(susp, w, precision, **kw):
    p = dict(w.params)
    args = dict(precision=precision, eta=p["eta"], rho=p["rho"], kn=p["kn"], kt=p["kt"],
                mu=p["mu"], xi_min=p["xi_min"], xi_max=p["xi_max"], skin=p["skin"],
                shear_rate=p["shear_rate"], kT=p["kT"], seed=p["seed"],
                torque_sign=p["torque_sign"], dt=p["dt"])
    args.update(kw)
    return susp.System(w.radii, w.box, **args)


def _relerr(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("strain", [0.0, 0.2, -0.45])
@pytest.mark.parametrize("poly", [False, True])
def test_mixed_one_evaluation_without_noise(susp, strain, poly, record):
    w = workloads.make(3000, 0.58, 1000.0, 1.0, poly=poly, pack_seed=51, dyn_seed=52)
    w.x = w.x * 0.99
    w.L = w.L * 0.99
    res = {}
    for prec in ("fp64", "mixed"):
        g = _sys(susp, w, prec, noise=0)
        g.set_state(w.x, w.U, w.W)
        g.set_clock(3, strain)
        g.evaluate()
        res[prec] = (g.forces(), g.stress())
    (F64, T64), s64 = res["fp64"]
    (F32, T32), s32 = res["mixed"]
    record("force", _relerr(F32, F64), RTOL_MIXED)
    record("torque", _relerr(T32, T64), RTOL_MIXED)
    for key in ("contact", "lubrication"):
        record(key, _relerr(s32[key], s64[key]), RTOL_MIXED)
    assert _relerr(F32, F64) <= RTOL_MIXED
    assert _relerr(T32, T64) <= RTOL_MIXED
    for key in ("contact", "lubrication"):
        assert _relerr(s32[key], s64[key]) <= RTOL_MIXED, key


def test_mixed_brownian_stress_tracks_fp64_with_noise(susp, record):
    """One evaluation with the pair noise on.  Both paths draw the same Philox
    words; the mixed one maps them through 24-bit uniforms and the fast
    log/sin/cos, so single deviates differ by ~1e-6 relative and rarely (a
    uniform within 2^-24 of 0) by more.  The Brownian stress is a sum over
    thousands of pairs and agrees to 1e-6 of its largest entry (measured on a
    GB300; bar 2e-5); a wrong entry of the 27 virial slots would be off by
    its own size."""
    w = workloads.make(3000, 0.58, 10.0, 1.0, pack_seed=55, dyn_seed=56)
    w.x = w.x * 0.99
    w.L = w.L * 0.99
    res = {}
    for prec in ("fp64", "mixed"):
        g = _sys(susp, w, prec)
        g.set_state(w.x, w.U, w.W)
        g.set_clock(7, 0.3)
        g.evaluate()
        res[prec] = g.stress()
    s64, s32 = res["fp64"], res["mixed"]
    assert np.abs(s64["brownian"]).max() > 0
    for key in ("contact", "lubrication", "brownian"):
        record(key, _relerr(s32[key], s64[key]), RTOL_MIXED if key != "brownian" else 2e-5)
    for key in ("contact", "lubrication"):
        assert _relerr(s32[key], s64[key]) <= RTOL_MIXED, key
    assert _relerr(s32["brownian"], s64["brownian"]) <= 2e-5


@pytest.mark.parametrize("start_strain", [0.1, 0.495])
def test_mixed_trajectory_tracks_fp64_without_noise(susp, start_strain, record):
    # 400 steps with rebuilds (and, from 0.495, a strain flip)
    w = workloads.make(4000, 0.56, 1000.0, 1.0, pack_seed=61, dyn_seed=62)
    p = w.params
    out = {}
    for prec in ("fp64", "mixed"):
        g = _sys(susp, w, prec, noise=0)
        g.set_state(w.x, w.U, w.W)
        g.set_clock(0, start_strain)
        g.step(400, p["shear_rate"], 0.0, p["dt"], p["seed"])
        out[prec] = (g.state(), g.forces(), g.info())
    (x64, U64, W64), (F64, _), i64 = out["fp64"]
    (x32, U32, W32), (F32, _), i32 = out["mixed"]
    assert i32["nbuilds"] >= 2
    assert i32["strain"] == pytest.approx(i64["strain"], abs=1e-12)
    if start_strain > 0.49:
        assert i32["strain"] < 0
    dx = x32 - x64
    dx -= np.rint(dx / w.L) * w.L
    # measured on a GB300: x 5.9e-8, U 7e-8, F 4.3e-6; bars 12-17 times that
    record("x", np.abs(dx).max(), 1e-6)
    record("U", np.abs(U32 - U64).max() / np.abs(U64).max(), 1e-6)
    record("F", _relerr(F32, F64), 5e-5)
    assert np.abs(dx).max() < 1e-6
    assert np.abs(U32 - U64).max() < 1e-6 * np.abs(U64).max()
    assert _relerr(F32, F64) <= 5e-5


def test_mixed_state_round_trip_keeps_double_precision(susp):
    # positions and velocities survive the double-float storage to ~1e-14
    w = workloads.make(2000, 0.5, 10.0, 0.0, pack_seed=71)
    g = _sys(susp, w, "mixed")
    rng = np.random.default_rng(1)
    U = rng.normal(size=(w.N, 3))
    W = rng.normal(size=(w.N, 3))
    g.set_state(w.x, U, W)
    x2, U2, W2 = g.state()
    assert np.abs(x2 - w.x).max() <= 1e-13 * w.L
    assert np.abs(U2 - U).max() <= 1e-13
    assert np.abs(W2 - W).max() <= 1e-13


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_equipartition_at_rest(susp, precision):
    # no shear: full-step kinetic temperature equals kT (exact for the
    # Velocity-Verlet Langevin map with FDT-consistent noise in a frozen
    # configuration; within statistics and the O(dt) drift of the
    # configuration here)
    w = workloads.make(20000 if precision == "mixed" else 4000, 0.45, 1.0, 0.0,
                       pack_seed=81, dyn_seed=82, rate=0.0)
    p = w.params
    kT = 1.0
    g = _sys(susp, w, precision, shear_rate=0.0)
    g.set_state(w.x, np.zeros_like(w.x), np.zeros_like(w.x))
    # the configuration needs ~2 time units to forget the athermal packing
    g.step(20000, 0.0, kT, p["dt"], 5)
    g.stress()
    g.step(20000, 0.0, kT, p["dt"], 5)
    s = g.stress()
    V = w.L ** 3
    Tt = np.trace(s["kinetic"]) * V / (3 * w.N)
    Tr = np.trace(s["kinetic_rot"]) * V / (3 * w.N)
    assert Tt == pytest.approx(kT, rel=0.015)
    assert Tr == pytest.approx(kT, rel=0.015)


def test_mixed_viscosity_within_one_percent_of_fp64(susp, record):
    """The accuracy bar of the mixed path: the relative viscosity and normal
    stress differences of a sheared, frictional, Brownian suspension, averaged
    over 2,000 steps from the same state with the same noise, within 1% of the
    FP64 path.  Over 0.2 strain units the two trajectories stay close, so the
    measured difference is far below the bar (it is printed)."""
    w = workloads.make(10_000, 0.56, 100.0, 1.0, pack_seed=81, dyn_seed=82)
    p = w.params
    res = {}
    for prec in ("fp64", "mixed"):
        g = _sys(susp, w, prec)
        g.set_state(w.x, w.U, w.W)
        g.step(500, p["shear_rate"], p["kT"], p["dt"], p["seed"])
        g.stress()                      # discard the start-up
        g.step(2000, p["shear_rate"], p["kT"], p["dt"], p["seed"])
        res[prec] = g.stress()
    e64, e32 = res["fp64"]["eta_r"], res["mixed"]["eta_r"]
    rel = abs(e32 / e64 - 1.0)
    print(f"eta_r fp64 {e64:.6f} mixed {e32:.6f} rel {rel:.2e}")
    record("eta_r_rel", rel, 1e-2)
    assert e64 > 1.0
    assert rel <= 1e-2
    tot64 = res["fp64"]["contact"] + res["fp64"]["lubrication"]
    tot32 = res["mixed"]["contact"] + res["mixed"]["lubrication"]
    scale = np.abs(tot64).max()
    assert np.abs(tot32 - tot64).max() <= 1e-2 * scale


@pytest.mark.parametrize("sample_every", [1, 3])
def test_stress_samples_do_not_depend_on_how_steps_are_grouped(susp, sample_every):
    """The mixed path reduces a sampled step's stress inside the next step's
    integrator, and a call's last sample after its closing kick.  70 steps as
    one call (captured chunks of 32, 32, 4 and 2 steps run as one sequence
    when every step is sampled, all eager when every third one is) and the
    same steps as 70
    one-step calls must put the same samples into the accumulators and the
    series, in the same order.  20,000 spheres make 79 blocks, so a replica
    spans two reduction chunks.  The two runs differ only by the order of the
    single-precision force atomics: positions part by ~1e-9 over the 70
    steps, and the near-contact resistances (1/xi) turn that into ~1e-6
    relative changes of single pairs.  A lost, repeated or shifted sample
    moves the averages by percents and the series by its own size."""
    w = workloads.make(20_000, 0.55, 10.0, 1.0, pack_seed=91, dyn_seed=92)
    p = w.params
    res = []
    for calls in (1, 70):
        g = _sys(susp, w, "mixed", structural=1, shell=0.05, series_cap=100,
                 sample_every=sample_every)
        g.set_state(w.x, w.U, w.W)
        for _ in range(calls):
            g.step(70 // calls, p["shear_rate"], p["kT"], p["dt"], p["seed"])
        res.append((g.state()[0], g.stress(), g.series()))
    (x1, s1, (q1, d1)), (x2, s2, (q2, d2)) = res
    n_samples = len(range(0, 70, sample_every))
    assert s1["samples"] == s2["samples"] == n_samples
    assert d1 == d2 == 0 and len(q1) == len(q2) == n_samples
    assert np.abs(q1).max() > 0
    assert np.abs(q1 - q2).max() <= 1e-6 * np.abs(q1).max()
    assert np.abs(x1 - x2).max() <= 1e-7
    for key in ("contact", "lubrication", "brownian", "kinetic", "kinetic_rot", "structural"):
        assert _relerr(s1[key], s2[key]) <= 1e-5, key


def test_graph_replay_resumes_after_unaligned_calls_when_sampling_sparsely(susp, record):
    """With the stress sampled every 8th step, calls of 100 steps end off the
    sampling grid; the next call must run eager steps up to the grid and then
    replay captured chunks again, with the samples where an eager run puts
    them."""
    w = workloads.make(6000, 0.55, 100.0, 1.0, pack_seed=95, dyn_seed=96)
    p = w.params
    res = []
    for graphs in (1, 0):
        g = _sys(susp, w, "mixed", sample_every=8, use_graphs=graphs)
        g.set_state(w.x, w.U, w.W)
        steps0 = None
        for call in range(3):
            g.step(100, p["shear_rate"], p["kT"], p["dt"], p["seed"])
            if call == 0:
                steps0 = g.info()["graph_steps"]
        res.append((g.info(), g.stress(), g.forces()[0]))
    (i1, s1, F1), (i0, s0, F0) = res
    # graphs were replayed in the second and third calls too
    assert i1["graph_steps"] >= steps0 + 2 * 64 and i0["graph_steps"] == 0
    assert s1["samples"] == s0["samples"] == len(range(0, 300, 8))
    record("force", _relerr(F1, F0), 1e-4)
    assert _relerr(F1, F0) <= 1e-4
    for key in ("contact", "lubrication"):
        assert _relerr(s1[key], s0[key]) <= 1e-5, key
