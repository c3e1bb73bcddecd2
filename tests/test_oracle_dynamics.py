"""Pins of the oracle's noise, contact model, stresses, box and time
integration against published values, closed forms and invariants."""
import math
import os

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# noise
# --------------------------------------------------------------------------
def test_philox_known_answer_vectors():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t, 16) for t in line.split()])
    assert len(rows) == 3
    for r in rows:
        assert oracle.philox4x32_10(r[0:4], r[4:6]).tolist() == r[6:10]


def test_gaussian_moments():
    # Sec. II.C: the elements of theta, chi, psi, phi are standard normal and
    # mutually uncorrelated.
    n = 40000
    g = np.array([oracle.gaussians6(123456789, k, 5, 17) for k in range(n)])
    se = 1.0 / math.sqrt(n)
    assert np.all(np.abs(g.mean(0)) < 5 * se)
    assert np.all(np.abs(g.var(0) - 1.0) < 5 * math.sqrt(2.0) * se)
    c = np.corrcoef(g.T)
    assert np.max(np.abs(c - np.eye(6))) < 5 * se
    kurt = (g ** 4).mean(0)
    assert np.all(np.abs(kurt - 3.0) < 5 * math.sqrt(96.0) * se)
    # different pairs and one-body counters give different streams
    assert not np.allclose(oracle.gaussians6(1, 3, 5, 17), oracle.gaussians6(1, 3, 5, 5))


def test_one_body_noise_variance():
    # Eqs. 20-21: <F F> = (2kT/dt) 6 pi eta a I, <T T> = (2kT/dt) 8 pi eta a^3 I
    a, kT, dt = 1.3, 2.0, 1e-3
    s = oracle.System([a], [50.0, 50.0, 50.0], shear_rate=0.0, kT=kT, dt=dt,
                      seed=99, lubrication=0, contact=0)
    s.set_state([[1.0, 2.0, 3.0]])
    n = 20000
    F = np.zeros((n, 3)); T = np.zeros((n, 3))
    for k in range(n):
        s.set_k(k)
        s.evaluate()
        f, t = s.forces()
        F[k], T[k] = f[0], t[0]
    c2 = 2 * kT / dt
    vf = c2 * 6 * math.pi * a
    vt = c2 * 8 * math.pi * a ** 3
    tol = 5 * math.sqrt(2.0 / n)
    assert np.all(np.abs(F.var(0) / vf - 1) < tol)
    assert np.all(np.abs(T.var(0) / vt - 1) < tol)


# --------------------------------------------------------------------------
# contact and stresses
# --------------------------------------------------------------------------
def test_head_on_contact_closed_form():
    # Eq. 3 (normal part) for an overlapping pair at rest; stress Sec. II.A.
    kn, delta = 1e4, 0.01
    a = 1.0
    L = 20.0
    s = oracle.System([a, a], [L, L, L], kn=kn, shear_rate=0.0, kT=0.0,
                      noise=0, lubrication=0, onebody=0)
    d = 2 * a - delta
    s.set_state([[5.0, 10.0, 10.0], [5.0 + d, 10.0, 10.0]])
    s.evaluate()
    F, T = s.forces()
    # n points from 0 to 1 (+x); the overlap pushes 0 to -x and 1 to +x
    assert F[0] == pytest.approx([-kn * delta, 0, 0], abs=1e-9)
    assert F[1] == pytest.approx([kn * delta, 0, 0], abs=1e-9)
    assert np.all(T == 0)
    sig = s.stress()["contact"]
    assert sig[0, 0] == pytest.approx(-kn * delta * d / L ** 3, rel=1e-12)
    assert np.count_nonzero(sig) == 1


def test_drag_stresslet_is_einstein():
    # Sec. II.B: sum_i (20/3) pi eta a_i^3 E / V has xy part 2.5 phi eta rate.
    r = workloads.bidisperse_radii(1000, 5)
    for phi in (0.1, 0.45, 0.58):
        L = workloads.box_for_phi(r, phi)
        assert oracle.drag_stress_xy(r, [L, L, L], 0.7, 1.9) == pytest.approx(
            2.5 * phi * 0.7 * 1.9, rel=1e-12)


def test_peclet_number_reproduces_table_1():
    rows = np.loadtxt(os.path.join(GOLDEN, "table1_parameters.txt"))

    def half_unit(v):
        s = f"{v:.10g}"
        mant = s.split("e")[0]
        dec = len(mant.split(".")[1]) if "." in mant else 0
        exp = int(s.split("e")[1]) if "e" in s else 0
        return 0.5 * 10.0 ** (exp - dec)

    for pe, rate, kT, a, rho, kn, eta in rows:
        ts = oracle.timescales(a, rho, kn, eta, kT, rate)
        # the inputs are printed to a few digits: allow their rounding
        tol = half_unit(rate) / rate + half_unit(kT) / kT
        assert abs(ts[4] / pe - 1) <= tol, (pe, ts[4])
        # Pe = 6 pi tau_B / tau_S (Sec. II.F)
        assert ts[4] == pytest.approx(6 * math.pi * ts[2] / ts[3], rel=1e-14)


def _dense(N=300, phi=0.5, seed=7, **kw):
    w = workloads.make(N, phi, 10.0, kw.pop("mu", 0.0), pack_seed=seed,
                       dyn_seed=seed + 1)
    p = dict(w.params)
    p.update(kw)
    s = oracle.System(w.radii, w.box, **p)
    s.set_state(w.x, w.U, w.W)
    return s, w


def test_newton_third_law_pair_forces():
    s, w = _dense(onebody=0)
    s.step(20)
    F, _ = s.forces()
    scale = np.abs(F).max()
    assert np.abs(F.sum(0)).max() <= 1e-12 * scale * w.N


def test_dissipation_without_noise():
    # drag + lubrication are dissipative: sum F.U + T.W <= 0 (no shear, no noise)
    rng = np.random.default_rng(2)
    w = workloads.make(300, 0.5, 10.0, 0.0, pack_seed=9)
    s = oracle.System(w.radii, w.box, **dict(w.params, shear_rate=0.0, kT=0.0,
                                              noise=0, contact=0))
    for _ in range(5):
        U = rng.normal(size=(w.N, 3))
        Wv = rng.normal(size=(w.N, 3))
        s.set_state(w.x, U, Wv)
        s.evaluate()
        F, T = s.forces()
        assert np.sum(F * U) + np.sum(T * Wv) < 0


# --------------------------------------------------------------------------
# box: Lees-Edwards images and the strain flip (Sec. II.E)
# --------------------------------------------------------------------------
def test_lees_edwards_image_invariance():
    # moving a sphere by the lattice vector (tilt, Ly, 0) together with the
    # streaming-velocity jump rate*Ly must leave every force unchanged
    s, w = _dense(N=200, phi=0.5, mu=1.0, kt=5e3)
    s.set_strain(0.3)
    s.evaluate()
    F0, T0 = s.forces()
    x, U, Wv = s.state()
    tilt = s.info()["tilt"]
    sel = x[:, 1] < 4.0          # spheres near the bottom face
    x2, U2 = x.copy(), U.copy()
    x2[sel, 0] += tilt
    x2[sel, 1] += w.L
    U2[sel, 0] += w.params["shear_rate"] * w.L
    s.set_state(x2, U2, Wv)
    s.set_strain(0.3)
    s.evaluate()
    F1, T1 = s.forces()
    scale = np.abs(F0).max()
    assert np.abs(F1 - F0).max() <= 1e-9 * scale
    assert np.abs(T1 - T0).max() <= 1e-9 * np.abs(T0).max()


def test_strain_flip_leaves_forces_unchanged():
    # Sec. II.E: remapping strain 0.5 -> -0.5 changes neither forces nor stress
    s, w = _dense(N=200, phi=0.5)
    s.set_strain(0.4999)
    s.evaluate()
    F0, _ = s.forces()
    sig0 = s.stress()
    s.set_strain(0.4999 - 1.0)
    s.evaluate()
    F1, _ = s.forces()
    sig1 = s.stress()
    assert np.abs(F1 - F0).max() <= 1e-9 * np.abs(F0).max()
    for k in ("contact", "lubrication", "brownian"):
        assert np.abs(sig1[k] - sig0[k]).max() <= 1e-9 * np.abs(sig0[k]).max() + 1e-300


def test_flip_happens_during_run_and_is_seamless():
    # advance through a flip and compare with a run that never flips
    # (strain offset by exactly -1 from the start)
    w = workloads.make(150, 0.45, 10.0, 0.0, pack_seed=21)
    p = dict(w.params, rebuild_every_step=1)
    a = oracle.System(w.radii, w.box, **p)
    b = oracle.System(w.radii, w.box, **p)
    for s in (a, b):
        s.set_state(w.x, w.U, w.W)
    a.set_strain(0.499)
    b.set_strain(0.499 - 1.0)
    a.step(100)          # crosses 0.5 at step 10
    b.step(100)
    assert a.info()["strain"] < 0
    assert a.info()["strain"] == pytest.approx(b.info()["strain"], abs=1e-12)
    xa, _, _ = a.state()
    xb, _, _ = b.state()
    assert np.abs(xa - xb).max() < 1e-8


# --------------------------------------------------------------------------
# Verlet list with skin: same trajectory as a list rebuilt at every step
# --------------------------------------------------------------------------
def test_skin_list_matches_rebuild_every_step_bitwise():
    w = workloads.make(300, 0.5, 1.0, 1.0, pack_seed=31, dyn_seed=32)
    p = dict(w.params, dt=2e-4)
    a = oracle.System(w.radii, w.box, **p)
    b = oracle.System(w.radii, w.box, **dict(p, rebuild_every_step=1))
    for s in (a, b):
        s.set_state(w.x, w.U, w.W)
    a.step(300)
    b.step(300)
    assert a.info()["nbuilds"] < b.info()["nbuilds"]
    xa, Ua, Wa = a.state()
    xb, Ub, Wb = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(Ua, Ub) and np.array_equal(Wa, Wb)


def test_brute_pairs_are_the_list_at_build():
    s, w = _dense(N=250)
    s.build()
    ij, _, _ = s.verlet_list()
    bp = s.brute_pairs()
    assert np.array_equal(ij, bp)


# --------------------------------------------------------------------------
# friction: Coulomb cap (Sec. II.A)
# --------------------------------------------------------------------------
def test_coulomb_cap_holds_every_step():
    mu, kn, kt = 0.5, 1e4, 5e3
    w = workloads.make(300, 0.55, 100.0, mu, pack_seed=41, dyn_seed=42)
    p = dict(w.params, mu=mu, kn=kn, kt=kt, dt=2e-4)
    s = oracle.System(w.radii, w.box, **p)
    s.set_state(w.x, w.U, w.W)
    sliding = 0
    seen = 0
    for _ in range(40):
        s.step(10)
        x, _, _ = s.state()
        ij, hist, contact = s.verlet_list()
        tilt = s.info()["tilt"]
        for (i, j), h, c in zip(ij, hist, contact):
            if not c:
                assert not np.any(h)
                continue
            r = x[j] - x[i]
            sy = np.rint(r[1] / w.L); r[1] -= sy * w.L; r[0] -= sy * tilt
            r[0] -= np.rint(r[0] / w.L) * w.L; r[2] -= np.rint(r[2] / w.L) * w.L
            d = np.linalg.norm(r)
            delta = w.radii[i] + w.radii[j] - d
            assert delta > 0
            ft = kt * np.linalg.norm(h)
            # delta = S - d loses digits to cancellation: allow ulp(S)-level slack
            assert ft <= mu * kn * (delta + 1e-13 * d)
            # history lies in the tangent plane
            assert abs(np.dot(h, r / d)) <= 1e-9 * (np.linalg.norm(h) + 1e-300)
            seen += 1
            sliding += ft >= mu * kn * (delta - 1e-13 * d)
    assert seen > 100 and sliding > 0


# --------------------------------------------------------------------------
# time integration: isolated spheres (Sec. III.B)
# --------------------------------------------------------------------------
def _isolated(N, kT, dt, rate=0.0, seed=5, a=1.0, rho=1.0):
    # spheres on a widely spaced lattice with the pair terms switched off:
    # only the one-body drag and noise act (dt is far above the lubrication
    # stability limit, so a chance encounter must not feel pair forces)
    g = int(math.ceil(N ** (1 / 3)))
    sp = 12.0
    L = g * sp
    idx = np.array([(i, j, k) for k in range(g) for j in range(g) for i in range(g)])[:N]
    x = (idx + 0.5) * sp
    s = oracle.System(np.full(N, a), [L, L, L], shear_rate=rate, kT=kT, dt=dt,
                      rho=rho, seed=seed, skin=0.3, lubrication=0, contact=0)
    return s, x, L


def test_velocity_variance_is_exactly_kT_over_m():
    # For linear drag and the Velocity-Verlet ordering used here, the
    # stationary variance of the full-step velocity is kT/m for any stable dt
    # (exact discrete equipartition); likewise kT/I for the spin.
    N, kT, dt = 512, 1.0, 0.02       # dt * gamma/m = 0.09
    s, x, L = _isolated(N, kT, dt)
    s.set_state(x)
    s.step(200)                       # equilibrate
    s.take_stress_sums()
    s.step(4000)
    n, sums = s.take_stress_sums()
    V = L ** 3
    m = 4.0 / 3.0 * math.pi
    # kinetic tensor = sum m u u / V; equipartition: trace = 3 N kT / V
    ktr = np.trace(sums["kinetic"]) / n * V / (3 * N)
    krot = np.trace(sums["kinetic_rot"]) / n * V / (3 * N)
    # ~N*3*4000/(2*25) effective samples -> sd ~ 0.4 %
    assert ktr == pytest.approx(kT, rel=0.012)
    assert krot == pytest.approx(kT, rel=0.012)
    del m


def test_isolated_msd_matches_closed_form():
    # Eq. 31: <x^2> = 2 kT m/gamma^2 (gamma t/m - 1 + exp(-gamma t/m))
    N, kT, dt = 1000, 1.0, 2e-3
    s, x, L = _isolated(N, kT, dt, seed=17)
    m = 4.0 / 3.0 * math.pi
    gam = 6.0 * math.pi
    # start from equilibrium velocities: the closed form assumes <U^2> = kT/m
    rng = np.random.default_rng(8)
    U0 = rng.normal(scale=math.sqrt(kT / m), size=(N, 3))
    s.set_state(x, U0, None)
    xprev = x.copy()
    unwrapped = x.copy()
    ts = [25, 100, 400, 1200]
    t_done = 0
    for t in ts:
        s.step(t - t_done)
        t_done = t
        xn, _, _ = s.state()
        dx = xn - xprev
        dx -= np.rint(dx / L) * L
        unwrapped += dx
        xprev = xn
        msd = np.mean((unwrapped - x) ** 2)
        tt = t * dt
        ref = 2 * kT * m / gam ** 2 * (gam * tt / m - 1 + math.exp(-gam * tt / m))
        # 3N samples of a Gaussian displacement: sd of the mean ~ sqrt(2/3N)
        assert msd == pytest.approx(ref, rel=5 * math.sqrt(2 / (3 * N)) + 0.01), (t, msd, ref)


def test_shear_drives_isolated_spheres_to_the_flow():
    # Eqs. 5-6 without noise: U -> U_inf(y), Omega -> -rate/2 z
    N, dt, rate = 64, 1e-2, 0.7
    s, x, L = _isolated(N, 0.0, dt, rate=rate)
    s.set_state(x)
    s.step(3000)                     # 30 time units >> m/gamma = 0.22
    xn, U, Wv = s.state()
    assert np.allclose(U[:, 0], rate * (xn[:, 1] - L / 2), atol=1e-9)
    assert np.allclose(U[:, 1:], 0.0, atol=1e-12)
    assert np.allclose(Wv[:, 2], -rate / 2, atol=1e-9)


def test_pair_noise_covariance_in_evaluation():
    # Eq. 19 through the full evaluation: with U = W = 0 the pair force and
    # torques are pure noise; their covariance over evaluation indices k must
    # be (2kT/dt) times the pair resistance (chi-term sign -1 in Eq. 24).
    ai, aj, xi = 1.0, 1.4, 4e-3
    kT, dt = 0.7, 1e-3
    L = 30.0
    d = (ai + aj) * (1 + xi / 2)
    n = np.array([1.0, 2.0, -0.5]); n /= np.linalg.norm(n)
    x = np.array([[10.0, 10.0, 10.0], [10.0, 10.0, 10.0]]) + np.outer([0, 1], d * n)
    s = oracle.System([ai, aj], [L, L, L], shear_rate=0.0, kT=kT, dt=dt,
                      seed=2024, onebody=0, contact=0)
    s.set_state(x)
    K = 20000
    X = np.zeros((K, 12))
    for k in range(K):
        s.set_k(k)
        s.evaluate()
        F, T = s.forces()
        X[k] = np.concatenate([F[0], F[1], T[0], T[1]])
    cov = X.T @ X / K
    R = oracle.resistances(1.0, ai, aj, xi)
    M = np.zeros((12, 12))
    for col in range(12):
        v = np.zeros(12); v[col] = 1.0
        Fi, Ti, Tj = oracle.lubrication(R, n, v[3:6] - v[0:3], v[6:9], v[9:12])
        M[:, col] = -np.concatenate([Fi, -Fi, Ti, Tj])
    ref = 2 * kT / dt * M
    # entrywise standard error of a sample covariance: sqrt((S_aa S_bb + S_ab^2)/K)
    dg = np.diag(ref)
    se = np.sqrt((np.outer(dg, dg) + ref ** 2) / K)
    assert np.all(np.abs(cov - ref) <= 5 * se + 1e-9 * np.abs(ref).max())


def _equipartition_run(i):
    w = workloads.make(100, 0.45, 1.0, 0.0, pack_seed=100 + 7 * i, dyn_seed=101 + 7 * i,
                       rate=0.0)
    s = oracle.System(w.radii, w.box, **dict(w.params, kT=1.0, shear_rate=0.0))
    s.set_state(w.x, np.zeros_like(w.x), np.zeros_like(w.x))
    s.step(20000)
    s.take_stress_sums()
    s.step(40000)
    n, sm = s.take_stress_sums()
    return np.trace(sm["kinetic"]) / n * w.L ** 3 / (3 * w.N)


def test_equipartition_in_a_dense_suspension_at_rest():
    # Pe -> 0 limit (no shear): with lubrication, pair noise, contacts and
    # drag at phi = 0.45 the full-step kinetic temperature is kT within 1.5 %
    # (continuous-time Langevin dynamics with FDT-consistent noise samples
    # the Maxwellian exactly; the discrete scheme is exact for a frozen
    # configuration).  Sixteen independent runs of 100 spheres, 2 time units
    # to forget the athermal packing, 4 of measurement (sd of the mean ~0.5%).
    import concurrent.futures as cf
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=min(8, os.cpu_count() or 1),
                                mp_context=ctx) as ex:
        temps = list(ex.map(_equipartition_run, range(16)))
    assert np.mean(temps) == pytest.approx(1.0, abs=0.015), temps
