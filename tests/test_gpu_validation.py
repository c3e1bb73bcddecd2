"""Statistical validation runs on the GPU (Sec. III.A-B): thousands of
replicas in one batch handle reproduce the paper's two single-particle and
two-particle checks.

* Isolated spheres: the mean-square displacement follows Eq. 31,
  <x^2> = 2 kT m / gamma^2 (gamma t / m - 1 + exp(-gamma t / m)).
* Two spheres at rest with lubrication, pair noise and contacts: the pair
  noise is tied to the position-dependent lubrication resistance (Eq. 19),
  so the stationary distribution is Boltzmann's and, with no force at a gap,
  the separations beyond contact are uniformly distributed: the pair
  distribution g(r), hence the potential of mean force -kT ln g, is flat.
  (A noise amplitude not tied to the resistance, or a wrong sign in Eq. 24,
  pulls pairs together or apart near contact and the profile bends.)
  Inside contact the only conservative force is the normal spring, so the
  potential of mean force is (1/2) k_n delta^2 and g(r) falls as
  exp(-k_n delta^2 / 2 kT) with delta = 2a - r (Sec. III.A)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _batch(susp, R, n, L, radii, kw):
    sizes = np.full(R, n, dtype=np.int64)
    boxes = np.tile([L, L, L], (R, 1))
    params = [dict(kw, seed=9000 + r) for r in range(R)]
    return susp.System.batch(sizes, np.tile(radii, R), boxes, params)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_isolated_sphere_msd_follows_eq31(precision):
    import paper_2307_13802_gb300 as susp

    R, L, kT, dt = 8000, 8.5, 1.0, 2e-3
    kw = dict(precision=precision, shear_rate=0.0, kT=kT, dt=dt, lubrication=0, contact=0)
    b = _batch(susp, R, 1, L, [1.0], kw)
    m, gam = 4.0 / 3.0 * math.pi, 6.0 * math.pi
    rng = np.random.default_rng(3)
    x0 = np.full((R, 3), L / 2)
    b.set_state(x0, rng.normal(scale=math.sqrt(kT / m), size=(R, 3)), None)
    prev, unwrapped, done = x0.copy(), x0.copy(), 0
    for t in (25, 100, 400, 1200):
        b.step_batch(t - done, dt)
        done = t
        x, _, _ = b.state()
        dx = x - prev
        dx -= np.rint(dx / L) * L
        unwrapped += dx
        prev = x
        msd = np.mean((unwrapped - x0) ** 2)
        tt = t * dt
        ref = 2 * kT * m / gam ** 2 * (gam * tt / m - 1 + math.exp(-gam * tt / m))
        # 3R Gaussian displacements: sd of the mean ~ sqrt(2 / 3R)
        assert msd == pytest.approx(ref, rel=4 * math.sqrt(2 / (3 * R)) + 0.005), (t, msd, ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_two_sphere_potential_of_mean_force_is_flat(precision):
    # Starts from the equilibrium distribution (the second sphere placed with
    # the Boltzmann weight of the contact spring: uniform outside contact,
    # exp(-kn delta^2 / 2kT) inside) and checks that the dynamics keep it:
    # with a noise amplitude not tied to the resistance the lubrication shell
    # h <= 0.05 would heat or cool and its population would drift.  (Inside
    # contact the overdamped well relaxes on gamma / kn ~ 0.5 time units, so
    # a start without contacts would not reach equilibrium in this run.)
    import paper_2307_13802_gb300 as susp

    R, L, kT, dt, kn = 8000, 8.5, 10.0, 1e-4, 1e4
    dth = math.sqrt(kT / kn)           # thermal overlap scale, 0.032 a
    kw = dict(precision=precision, shear_rate=0.0, kT=kT, dt=dt, mu=0.0, kn=kn)
    b = _batch(susp, R, 2, L, [1.0, 1.0], kw)
    rng = np.random.default_rng(11)
    x = np.empty((R, 2, 3))
    x[:, 0] = L / 2
    for r in range(R):
        while True:
            y = rng.uniform(0.0, L, size=3)
            d = y - L / 2
            d -= np.rint(d / L) * L
            dist = np.linalg.norm(d)
            if dist >= 2.0 or (dist > 2.0 - 6 * dth and
                               rng.uniform() < math.exp(-kn * (2.0 - dist) ** 2 / (2 * kT))):
                break
        x[r, 1] = y
    m = 4.0 / 3.0 * math.pi
    U = rng.normal(scale=math.sqrt(kT / m), size=(R, 2, 3))
    b.set_state(x.reshape(-1, 3), U.reshape(-1, 3), None)
    b.step_batch(500, dt)
    inner = 2.0 - dth * np.array([2.0, 1.5, 1.0, 0.5])
    edges = np.concatenate([inner, [2.0, 2.05, 2.2, 2.5, 3.0, 3.6]])
    nin = len(inner)
    # histograms per group of replicas: the groups are independent, the
    # snapshots of one replica are not (a pair decorrelates over ~0.1-1
    # time units), so the error bars come from the spread over the groups
    G = 16
    counts = np.zeros((G, len(edges) - 1))
    grp = np.arange(R) * G // R
    for _ in range(400):
        b.step_batch(25, dt)
        xs = b.state()[0].reshape(R, 2, 3)
        d = xs[:, 1] - xs[:, 0]
        d -= np.rint(d / L) * L
        r = np.linalg.norm(d, axis=1)
        for gi in range(G):
            counts[gi] += np.histogram(r[grp == gi], bins=edges)[0]
    shell = 4.0 / 3.0 * math.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    gg = counts / shell
    gg /= gg[:, nin + 1:].mean(axis=1, keepdims=True)   # flat level beyond contact
    g = gg.mean(axis=0)
    sd = gg.std(axis=0, ddof=1) / math.sqrt(G)
    print("bins", np.round(edges, 4), "g", np.round(g, 4), "sd", np.round(sd, 4),
          "counts", counts.sum(axis=0).astype(int))
    out = g[nin:]
    assert counts[:, nin:].sum(axis=0).min() > 5_000
    assert np.all(np.abs(out - 1.0) <= 4 * sd[nin:] + 0.005), (out, sd[nin:])
    # inside contact: the bin averages of exp(-kn delta^2 / 2kT) over r^2 dr
    rr = np.linspace(edges[0], 2.0, 20001)
    wgt = rr ** 2 * np.exp(-kn * (2.0 - rr) ** 2 / (2 * kT))

    def trap(y, x):
        return float(np.sum(0.5 * (y[1:] + y[:-1]) * np.diff(x)))

    ref = np.array([trap(wgt[(rr >= lo) & (rr <= hi)], rr[(rr >= lo) & (rr <= hi)])
                    for lo, hi in zip(edges[:nin], edges[1:nin + 1])]) / (shell[:nin] / (4 * math.pi))
    print("contact bins: g", np.round(g[:nin], 4), "Boltzmann", np.round(ref, 4),
          "sd", np.round(sd[:nin], 4))
    assert counts[:, :nin].sum(axis=0).min() > 300
    assert np.all(np.abs(g[:nin] - ref) <= 4 * sd[:nin] + 0.02 * ref), (g[:nin], ref, sd[:nin])
