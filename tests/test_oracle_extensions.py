"""Pins of the oracle's short-range repulsion (Eq. 34), structural Brownian
stress (Eqs. 25-26) and Green-Kubo integral (Eq. 33) against results fixed
outside the oracle: energy conservation and the closed-form turning point of
a head-on encounter, the stress as the affine-strain derivative of the pair
energy, closed-form shell sums of lattices and single pairs, and the exact
autocorrelation of an AR(1) series."""
import math

import numpy as np
import pytest

import oracle
import workloads

ISOLATE = dict(lubrication=0, onebody=0, noise=0, contact=0, shear_rate=0.0, kT=0.0)


def test_repulsion_conserves_energy_through_a_head_on_encounter():
    # Eq. 34 is the gradient of the pair energy A exp((S - d)/kappa), shifted
    # to zero at the cutoff h = 10 kappa; Velocity-Verlet keeps the total
    # energy to O(dt^2), and the turning point follows from energy alone.
    a, L, A, v = 1.0, 40.0, 1.0, 0.109
    kappa = 0.01 * 2 * a
    s = oracle.System([a, a], [L, L, L], rep_A=A, rep_cut=10.0, dt=1e-4, **ISOLATE)
    x = np.array([[L / 2 - 1.15, L / 2, L / 2], [L / 2 + 1.15, L / 2, L / 2]])
    U = np.array([[v, 0.0, 0.0], [-v, 0.0, 0.0]])
    s.set_state(x, U, np.zeros((2, 3)))
    m = 4.0 / 3.0 * math.pi
    shift = A * math.exp(-10.0)

    def energy():
        xx, UU, _ = s.state()
        h = abs(xx[1, 0] - xx[0, 0]) - 2 * a
        pot = A * math.exp(-h / kappa) - shift if h <= 10 * kappa else 0.0
        return 0.5 * m * (UU ** 2).sum() + pot, h

    E0, _ = energy()
    hmin, worst = 1e9, 0.0
    for _ in range(26000):
        s.step(1)
        E, h = energy()
        hmin = min(hmin, h)
        worst = max(worst, abs(E - E0) / E0)
    assert h > 10 * kappa                               # separated again
    assert worst < 1e-5
    # turning point: A exp(-h/kappa) - shift = relative kinetic energy m v^2
    h_star = -kappa * math.log((m * v * v + shift) / A)
    assert hmin == pytest.approx(h_star, rel=1e-5)
    _, Uf, _ = s.state()
    assert Uf[0, 0] == pytest.approx(-v, rel=1e-6)     # elastic rebound


def _affine_energy(rs, S, A, cut, defo):
    kappa = 0.01 * S
    r = rs + rs @ defo.T
    d = np.linalg.norm(r, axis=1)
    h = d - S
    e = A * np.exp(-h / kappa) - A * np.exp(-cut)
    return np.where(h <= cut * kappa, e, 0.0).sum()


def test_repulsion_stress_is_the_strain_derivative_of_the_pair_energy():
    # sigma_ab V = dU / d eps_ab for the affine map r -> (1 + eps) r of all
    # pair vectors (r_a += eps r_b); pairs and energies are formed here with
    # numpy from the positions alone.
    w = workloads.make(120, 0.50, 10.0, 0.0, pack_seed=91, dyn_seed=92)
    A, cut = 0.7, 10.0
    s = oracle.System(w.radii, w.box, rep_A=A, rep_cut=cut, **ISOLATE)
    s.set_state(w.x, w.U, w.W)
    s.evaluate()
    sig = s.stress()["repulsion"]
    x, L = w.x, w.L
    i, j = np.triu_indices(w.N, 1)
    r = x[j] - x[i]
    r -= L * np.round(r / L)
    S = w.radii[i] + w.radii[j]
    near = np.linalg.norm(r, axis=1) - S <= 0.01 * cut * S * 1.5
    r, S = r[near], S[near]
    assert near.sum() > 20
    V = L ** 3
    eps = 1e-6
    for a_, b_ in ((0, 1), (1, 0), (0, 0), (2, 2), (1, 2)):
        D = np.zeros((3, 3))
        D[a_, b_] = eps
        dU = (_affine_energy(r, S, A, cut, D) - _affine_energy(r, S, A, cut, -D)) / (2 * eps)
        assert sig[a_, b_] * V == pytest.approx(dU, rel=1e-6, abs=1e-9)


def _lattice(n, b):
    g = (np.arange(n) + 0.5) * b
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


@pytest.mark.parametrize("h0,count", [(0.02, 1), (-0.01, 1), (0.0499, 1), (0.0501, 0), (0.06, 0)])
def test_structural_stress_of_a_cubic_lattice(h0, count):
    # every sphere of a simple cubic lattice has its six axis neighbours at
    # gap h0; inside the shell (h0 <= 0.05 a) each sphere counts
    # sum_j n n = 2 I with weight a / Delta = 20, so Sigma^B = -kT/V 40 N I
    n, a, kT = 4, 1.0, 2.0
    b = 2 * a + h0
    x = _lattice(n, b)
    N, L = len(x), n * b
    s = oracle.System(np.full(N, a), [L, L, L], structural=1, shell=0.05,
                      **dict(ISOLATE, kT=kT))
    s.set_state(x)
    s.evaluate()
    sig = s.stress()["structural"]
    expect = -kT / L ** 3 * 40.0 * N * count * np.eye(3)
    assert np.allclose(sig, expect, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("h,weight", [(0.04, 2), (0.06, 1), (0.0699, 1), (0.08, 0)])
def test_structural_shell_is_counted_from_each_side(h, weight):
    # radii 1 and 1.4: the pair lies in the shell of the large sphere up to
    # h = 0.07 and in that of the small one up to h = 0.05
    kT, L = 1.5, 30.0
    x = np.array([[10.0, 12.0, 9.0], [10.0 + 2.4 + h, 12.0, 9.0]])
    s = oracle.System([1.0, 1.4], [L, L, L], structural=1, shell=0.05,
                      **dict(ISOLATE, kT=kT))
    s.set_state(x)
    s.evaluate()
    sig = s.stress()["structural"] * L ** 3 / kT
    expect = np.zeros((3, 3))
    expect[0, 0] = -20.0 * weight
    assert np.allclose(sig, expect, atol=1e-12)


def test_green_kubo_of_an_ar1_series():
    # x_{t+1} = rho x_t + sqrt(1 - rho^2) z has C(tau) = rho^tau exactly, so
    # eta(t_M) = V/kT dt (sum_{tau<=M} rho^tau - (1 + rho^M)/2)
    rho, n, dt, V, kT, M = 0.9, 400_000, 0.01, 2.0, 0.5, 200
    rng = np.random.Generator(np.random.PCG64(7))
    z = rng.standard_normal(n)
    x = np.empty(n)
    x[0] = z[0]
    c = math.sqrt(1 - rho * rho)
    for t in range(1, n):
        x[t] = rho * x[t - 1] + c * z[t]
    C, eta = oracle.green_kubo(x, M, dt, V, kT)
    taus = np.arange(M)
    assert np.abs(C - rho ** taus).max() < 0.03
    exact = V / kT * dt * (np.sum(rho ** taus) - 0.5 * (1 + rho ** (M - 1)))
    assert eta[-1] == pytest.approx(exact, rel=0.05)
    assert eta[0] == 0.0 and np.all(np.diff(eta[:30]) > 0)


def test_green_kubo_fit_recovers_an_exponential_approach():
    dt, M = 0.01, 300
    t = np.arange(M) * dt
    eta = 3.0 * (1.0 - np.exp(-t / 0.37))
    e_phi, tau = oracle.gk_fit(eta, dt)
    step = (10.0 * M) ** (1.0 / 399)        # grid ratio
    assert e_phi == pytest.approx(3.0, rel=5e-3)
    assert 0.37 / step <= tau <= 0.37 * step


def test_a_tagged_cluster_reproduces_the_force_on_its_centre():
    # the forces on a sphere come from the spheres within the interaction
    # range only, and the noise from (seed, k, tags): a cluster carrying the
    # global tags reproduces the full system's force and torque on it
    w = workloads.make(400, 0.52, 10.0, 0.0, pack_seed=95, dyn_seed=96)
    full = oracle.System(w.radii, w.box, **w.params)
    full.set_state(w.x, w.U, w.W)
    full.set_k(3)
    full.evaluate()
    F, T = full.forces()
    L = w.L
    for c in (7, 123, 301):
        d = w.x - w.x[c]
        d -= np.rint(d / L) * L
        near = np.linalg.norm(d, axis=1) < (w.radii + w.radii[c]) * 1.025 + 1e-9
        idx = np.flatnonzero(near)             # sorted, includes c
        o = oracle.System(w.radii[idx], w.box, **w.params)
        o.set_tags(idx)
        o.set_state(w.x[idx], w.U[idx], w.W[idx])
        o.set_k(3)
        o.evaluate()
        Fc, Tc = o.forces()
        k = int(np.flatnonzero(idx == c)[0])
        assert np.allclose(Fc[k], F[c], rtol=1e-13, atol=1e-13 * np.abs(F).max())
        assert np.allclose(Tc[k], T[c], rtol=1e-13, atol=1e-13 * np.abs(T).max())
