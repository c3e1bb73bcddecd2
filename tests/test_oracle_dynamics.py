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


# --------------------------------------------------------------------------
# friction: tangential history and contact torque (Sec. II.A, Eqs. 3-4)
#
# Two spheres of unequal radii touch along a general direction n.  The
# velocities of their surface points at the contact follow from rigid-body
# kinematics, v_c,i = U_i + Omega_i x (a_i n) and v_c,j = U_j + Omega_j x
# (-a_j n); the stored history is the accumulated tangential part of
# v_c,j - v_c,i.  With the positions frozen (n fixed) and the spheres made
# so heavy that the forces do not change their velocities, the history grows
# exactly linearly, so every quantity has a closed form.  The tangential
# spring acts on i at i's contact point (lever arm a_i n) and its reaction on
# j at j's contact point (lever arm -a_j n).
# --------------------------------------------------------------------------
_AI, _AJ, _KN, _KT, _DELTA, _DT = 1.0, 1.4, 1e4, 5e3, 0.01, 1e-4
_N_DIR = np.array([0.3, -0.5, 0.81]) / np.linalg.norm([0.3, -0.5, 0.81])


def _frozen_pair(U, W, mu):
    L = 20.0
    d = _AI + _AJ - _DELTA
    x = np.array([[8.0, 9.0, 7.5], [8.0, 9.0, 7.5]])
    x[1] += d * _N_DIR
    s = oracle.System([_AI, _AJ], [L, L, L], kn=_KN, kt=_KT, mu=mu, rho=1e30,
                      shear_rate=0.0, kT=0.0, dt=_DT, noise=0, lubrication=0,
                      onebody=0, freeze=1)
    s.set_state(x, U, W)
    return s, L


def _contact_slip(U, W):
    """Tangential part of the velocity of j's contact point relative to i's."""
    n = _N_DIR
    vci = U[0] + np.cross(W[0], _AI * n)
    vcj = U[1] + np.cross(W[1], -_AJ * n)
    v = vcj - vci
    return v - np.dot(v, n) * n


@pytest.mark.parametrize("case", ["slide", "spin_i", "spin_j", "general"])
def test_history_grows_as_the_contact_slip_times_t(case):
    rng = np.random.default_rng({"slide": 1, "spin_i": 2, "spin_j": 3, "general": 4}[case])
    U = np.zeros((2, 3))
    W = np.zeros((2, 3))
    if case in ("slide", "general"):
        U = rng.normal(size=(2, 3))
    if case in ("spin_i", "general"):
        W[0] = rng.normal(size=3)
    if case in ("spin_j", "general"):
        W[1] = rng.normal(size=3)
    s, L = _frozen_pair(U, W, mu=1e12)
    nsteps = 37
    s.step(nsteps)
    _, hist, contact = s.verlet_list()
    assert contact[0] == 1
    xi_ref = _contact_slip(U, W) * (nsteps * _DT)
    assert np.linalg.norm(xi_ref) > 1e-4
    assert np.abs(hist[0] - xi_ref).max() <= 1e-12 * np.linalg.norm(xi_ref)
    # forces: normal spring plus the tangential spring k_t xi on i, the
    # reaction on j; torques: lever arm cross force at each contact point
    F, T = s.forces()
    Ft_i = _KT * xi_ref
    Fi_ref = -_KN * _DELTA * _N_DIR + Ft_i
    scale = np.linalg.norm(Fi_ref)
    assert np.abs(F[0] - Fi_ref).max() <= 1e-11 * scale
    assert np.abs(F[1] + Fi_ref).max() <= 1e-11 * scale
    Ti_ref = np.cross(_AI * _N_DIR, Ft_i)
    Tj_ref = np.cross(-_AJ * _N_DIR, -Ft_i)
    tscale = np.linalg.norm(Tj_ref)
    assert np.abs(T[0] - Ti_ref).max() <= 1e-11 * tscale
    assert np.abs(T[1] - Tj_ref).max() <= 1e-11 * tscale
    # contact stress (1/V) F_{i<-j} (x) r_ij
    r = (_AI + _AJ - _DELTA) * _N_DIR
    sig = s.stress()["contact"]
    assert np.abs(sig - np.outer(Fi_ref, r) / L ** 3).max() <= 1e-11 * scale * 2.4 / L ** 3


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_rolling_without_slip_stores_no_history(seed):
    # U_j chosen so that the two contact points move together: the spheres
    # roll on each other (and translate and spin rigidly); nothing slips
    rng = np.random.default_rng(seed)
    W = rng.normal(size=(2, 3))
    U = np.zeros((2, 3))
    U[0] = rng.normal(size=3)
    U[1] = U[0] + np.cross(W[0], _AI * _N_DIR) - np.cross(W[1], -_AJ * _N_DIR)
    assert np.linalg.norm(_contact_slip(U, W)) <= 1e-14
    s, _ = _frozen_pair(U, W, mu=1e12)
    s.step(50)
    _, hist, contact = s.verlet_list()
    assert contact[0] == 1
    vscale = np.abs(U).max() + np.abs(W).max() * _AJ
    assert np.abs(hist[0]).max() <= 1e-14 * vscale * 50 * _DT * 10
    F, T = s.forces()
    assert np.abs(F[0] + _KN * _DELTA * _N_DIR).max() <= 1e-12 * _KN * _DELTA
    assert np.abs(T).max() <= 1e-12 * _KN * _DELTA


def test_capped_friction_opposes_the_slip():
    # a constant slip drives the spring to the Coulomb cap, after which the
    # tangential force has magnitude mu k_n delta and the force on j points
    # against j's slip relative to i
    mu = 0.5
    rng = np.random.default_rng(11)
    U = rng.normal(size=(2, 3))
    W = rng.normal(size=(2, 3)) * 0.3
    vt = _contact_slip(U, W)
    s, _ = _frozen_pair(U, W, mu=mu)
    cap_len = mu * _KN * _DELTA / _KT
    t_cap = cap_len / np.linalg.norm(vt)
    n_before = int(0.5 * t_cap / _DT)
    s.step(n_before)
    _, hist, _ = s.verlet_list()
    assert np.abs(hist[0] - vt * n_before * _DT).max() <= 1e-12 * cap_len
    s.step(int(2 * t_cap / _DT))                     # well past the cap
    _, hist, _ = s.verlet_list()
    F, T = s.forces()
    Ft_j = F[1] - _KN * _DELTA * _N_DIR              # tangential part on j
    assert abs(np.dot(Ft_j, _N_DIR)) <= 1e-12 * _KN * _DELTA
    assert np.linalg.norm(Ft_j) == pytest.approx(mu * _KN * _DELTA, rel=1e-12)
    # the force on j is antiparallel to j's slip
    cosang = np.dot(Ft_j, vt) / (np.linalg.norm(Ft_j) * np.linalg.norm(vt))
    assert cosang == pytest.approx(-1.0, abs=1e-12)
    assert np.linalg.norm(hist[0]) == pytest.approx(cap_len, rel=1e-12)


def _collision_energy_error(dt):
    """Largest relative change of the mechanical energy of a frictional
    glancing collision while the spheres touch: translational and
    rotational kinetic energy of the full-step velocities plus the normal
    and tangential spring energies."""
    ai, aj, kn, kt = 1.0, 1.4, 1e4, 5e3
    rho = 1.0
    L = 30.0
    m = 4.0 / 3.0 * math.pi * rho * np.array([ai ** 3, aj ** 3])
    I = 0.4 * m * np.array([ai ** 2, aj ** 2])
    # the spheres start touching (overlap 0.004) and approaching, so that the
    # history starts from zero at t = 0 whatever dt, and the collision ends
    # when they part
    c = np.array([1.0, 0.9, -0.4]) / np.linalg.norm([1.0, 0.9, -0.4])
    x0 = np.array([[12.0, 15.0, 15.0], [12.0, 15.0, 15.0]])
    x0[1] += (ai + aj - 0.004) * c
    U0 = np.array([[1.0, 0.1, -0.2], [-1.5, -0.3, 0.4]])
    W0 = np.array([[0.0, 0.5, -1.0], [0.7, 0.0, 0.3]])
    s = oracle.System([ai, aj], [L, L, L], kn=kn, kt=kt, mu=1e12, rho=rho,
                      shear_rate=0.0, kT=0.0, dt=dt, noise=0, lubrication=0,
                      onebody=0, skin=0.5)
    s.set_state(x0, U0, W0)

    def energy():
        x, U, W = s.state()
        r = x[1] - x[0]
        d = np.linalg.norm(r)
        delta = max(ai + aj - d, 0.0)
        _, hist, contact = s.verlet_list()
        es = 0.5 * kt * float(np.dot(hist[0], hist[0])) if len(hist) and contact[0] else 0.0
        ek = 0.5 * np.sum(m[:, None] * U ** 2) + 0.5 * np.sum(I[:, None] * W ** 2)
        return ek + 0.5 * kn * delta ** 2 + es, delta

    E0, _ = energy()
    worst, touched, steps = 0.0, 0, 0
    while steps < int(0.3 / dt):
        s.step(1)
        steps += 1
        E, delta = energy()
        if delta > 0:
            touched += 1
            worst = max(worst, abs(E / E0 - 1.0))
        elif touched:
            break
    _, hist, _ = s.verlet_list()
    return worst, touched


def test_frictional_collision_conserves_energy_as_dt_shrinks():
    # With lubrication, drag and noise off and an unbounded Coulomb cap the
    # contact is conservative in continuous time: the tangential spring
    # stores exactly the work that the friction force and the two contact
    # torques do on the spheres.  The discrete history update (rotate, then
    # add the slip of a half-step velocity) is first-order accurate in how the
    # tangent plane turns, and Velocity-Verlet second-order, so the energy
    # error of a glancing collision must shrink at least linearly with dt.
    # A wrong sign of the spin term in the slip, of the tangential force or
    # of a contact torque, or a wrong lever arm, leaves an O(1) error.
    errs = []
    for dt in (2e-4, 1e-4, 5e-5):
        e, n = _collision_energy_error(dt)
        errs.append(e)
        assert n * dt > 0.02          # the spheres stayed in contact for a while
    assert errs[2] < 5e-6, errs
    assert errs[0] / errs[1] > 1.8 and errs[1] / errs[2] > 1.8, errs


def test_history_turns_with_the_contact_without_changing_length():
    # Sec. II.A stores the tangential spring displacement xi in the tangent
    # plane of the contact.  When the contact normal turns while nothing
    # slips, the stored displacement must turn into the new tangent plane and
    # keep its length (the spring energy cannot change without slip).  Here
    # the pair straddles the y boundary of the sheared box: with positions
    # frozen, the growing tilt of the image turns n by about 0.04 rad over 50
    # steps, and j moves with exactly the image velocity rate * Ly so that
    # the contact points do not slip.
    ai, aj, L, rate = 1.0, 1.4, 20.0, 1.0
    xi_pos = np.array([10.0, 0.5, 10.0])
    r0 = np.array([0.05, -2.0, 1.3])                 # min-image r at strain 0
    r0 *= (ai + aj - 0.01) / np.linalg.norm(r0)
    xj_pos = xi_pos + r0 + np.array([0.0, L, 0.0])   # j is the image above
    s = oracle.System([ai, aj], [L, L, L], kn=1e4, kt=5e3, mu=1e12, rho=1e30,
                      shear_rate=rate, kT=0.0, dt=1e-4, noise=0, lubrication=0,
                      onebody=0, freeze=1)
    U = np.zeros((2, 3))
    U[1, 0] = rate * L
    W = np.zeros((2, 3))
    slip = np.array([0.4, 0.3, -0.2])
    s.set_state(np.stack([xi_pos, xj_pos]), U + np.stack([np.zeros(3), slip]), W)
    s.step(30)                                      # build up a history
    s.set_velocities(U, W)                          # from now on nothing slips

    def normal():
        tilt = s.info()["tilt"]
        r = xj_pos - xi_pos - np.array([tilt, L, 0.0])
        return r / np.linalg.norm(r)

    _, h0, c0 = s.verlet_list()
    n0 = normal()
    assert c0[0] == 1 and abs(np.dot(h0[0], n0)) <= 1e-14 * np.linalg.norm(h0[0])
    s.step(50)
    _, h1, c1 = s.verlet_list()
    n1 = normal()
    theta = math.acos(min(1.0, float(np.dot(n0, n1))))
    assert c1[0] == 1 and theta > 0.03
    xi0, xi1 = h0[0], h1[0]
    assert np.linalg.norm(xi0) > 1e-4
    assert np.linalg.norm(xi1) == pytest.approx(np.linalg.norm(xi0), rel=1e-13)
    assert abs(np.dot(xi1, n1)) <= 1e-13 * np.linalg.norm(xi1)
    # it turned with the contact: the rotation taking n0 to n1 takes xi0 to
    # xi1 up to the O(theta^2) by which stepwise turning differs from it
    k = np.cross(n0, n1)
    k /= np.linalg.norm(k)
    rot = (xi0 * math.cos(theta) + np.cross(k, xi0) * math.sin(theta)
           + k * np.dot(k, xi0) * (1 - math.cos(theta)))
    assert np.linalg.norm(xi1 - rot) <= theta ** 2 * np.linalg.norm(xi0)
