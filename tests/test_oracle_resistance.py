"""Pins of the oracle's pair hydrodynamics (Sec. II.B, Eqs. 8-18) and pair
noise (Sec. II.C, Eqs. 19, 22-24) against facts fixed outside the oracle:
textbook equal-sphere limits, exchange symmetry, rigid-body motion at
contact, Onsager symmetry / positive semi-definiteness of the resistance and
the fluctuation-dissipation identity."""
import math

import numpy as np
import pytest

import oracle

ETA = 1.0
BETAS = [1.0, 1.2, 1.4, 1.0 / 1.4]
XIS = [1e-3, 1e-2, 0.05]


def test_equal_spheres_reduce_to_textbook_leading_terms():
    # Jeffrey & Onishi / Kim & Karrila near-contact limits for equal spheres:
    # XA11/(6 pi eta a) = 1/(4 xi) + 9/40 ln(1/xi), YA11/(6 pi eta a) = 1/6 ln,
    # YB11/(4 pi eta a^2) = -1/4 ln, YC11/(8 pi eta a^3) = 1/5 ln,
    # YC12/(8 pi eta a^3) = 1/20 ln.
    for a in (1.0, 1.4):
        for xi in XIS:
            R = oracle.resistances(ETA, a, a, xi)
            L = math.log(1.0 / xi)
            assert R[0] / (6 * math.pi * a) == pytest.approx(0.25 / xi + 9.0 / 40.0 * L, rel=1e-13)
            assert R[1] / (6 * math.pi * a) == pytest.approx(L / 6.0, rel=1e-13)
            assert R[2] / (4 * math.pi * a * a) == pytest.approx(-0.25 * L, rel=1e-13)
            assert R[3] == pytest.approx(R[2], rel=1e-13)
            assert R[4] / (8 * math.pi * a ** 3) == pytest.approx(0.2 * L, rel=1e-13)
            assert R[5] / (8 * math.pi * a ** 3) == pytest.approx(0.05 * L, rel=1e-13)
            assert R[6] == pytest.approx(R[5], rel=1e-13)
            assert R[7] == pytest.approx(R[4], rel=1e-13)


@pytest.mark.parametrize("beta", BETAS)
def test_exchange_symmetry(beta):
    # swapping the two spheres maps 11 <-> 22, 12 <-> 21 and leaves X^A, Y^A
    ai, aj = 1.0, beta
    for xi in XIS:
        R = oracle.resistances(ETA, ai, aj, xi)
        S = oracle.resistances(ETA, aj, ai, xi)
        assert S[0] == pytest.approx(R[0], rel=1e-14)   # XA11
        assert S[1] == pytest.approx(R[1], rel=1e-14)   # YA11
        assert S[2] == pytest.approx(R[3], rel=1e-14)   # YB11 <-> YB21
        assert S[4] == pytest.approx(R[7], rel=1e-14)   # YC11 <-> YC22
        assert S[5] == pytest.approx(R[6], rel=1e-14)   # YC12 <-> YC21
        assert R[5] == pytest.approx(R[6], rel=1e-14)   # YC12 = YC21


def _unit(v):
    v = np.asarray(v, dtype=float)
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("beta", BETAS)
def test_rigid_rotation_of_touching_pair_is_force_free(beta):
    # A touching pair (|r| = a_i + a_j) moving as one rigid body (common
    # rotation Omega, U_j - U_i = Omega x r) has no relative surface motion at
    # the contact, so the lubrication force and torques must vanish.
    rng = np.random.default_rng(7)
    ai, aj = 1.0, beta
    for xi in XIS:
        R = oracle.resistances(ETA, ai, aj, xi)
        for _ in range(5):
            n = _unit(rng.normal(size=3))
            Om = rng.normal(size=3)
            dU = np.cross(Om, (ai + aj) * n)
            Fi, Ti, Tj = oracle.lubrication(R, n, dU, Om, Om)
            scale = max(abs(R[1]) * (ai + aj), abs(R[4])) * np.linalg.norm(Om)
            assert np.max(np.abs(Fi)) <= 1e-13 * scale
            assert np.max(np.abs(Ti)) <= 1e-13 * scale
            assert np.max(np.abs(Tj)) <= 1e-13 * scale


def _pair_resistance(R, n):
    """12x12 matrix with (F_i, F_j, T_i, T_j) = -Rmat (U_i, U_j, W_i, W_j),
    built by probing the oracle's lubrication function (Eq. 8, 13, 14)."""
    M = np.zeros((12, 12))
    for col in range(12):
        v = np.zeros(12)
        v[col] = 1.0
        Ui, Uj, Wi, Wj = v[0:3], v[3:6], v[6:9], v[9:12]
        Fi, Ti, Tj = oracle.lubrication(R, n, Uj - Ui, Wi, Wj)
        M[:, col] = -np.concatenate([Fi, -Fi, Ti, Tj])
    return M


def _pair_noise_matrix(R, n, sign):
    """12x6 matrix B with (F_i, F_j, T_i, T_j) = B (theta, chi) for c = 1,
    built by probing the oracle's pair Brownian function (Eqs. 22-24)."""
    B = np.zeros((12, 6))
    for col in range(6):
        g = np.zeros(6)
        g[col] = 1.0
        Fi, Ti, Tj = oracle.pair_brownian(R, n, g[:3], g[3:], 1.0, sign)
        B[:, col] = np.concatenate([Fi, -Fi, Ti, Tj])
    return B


@pytest.mark.parametrize("beta", BETAS)
def test_pair_resistance_symmetric_positive_semidefinite(beta):
    rng = np.random.default_rng(11)
    for xi in XIS:
        R = oracle.resistances(ETA, 1.0, beta, xi)
        n = _unit(rng.normal(size=3))
        M = _pair_resistance(R, n)
        scale = np.max(np.abs(M))
        assert np.max(np.abs(M - M.T)) <= 1e-13 * scale
        ev = np.linalg.eigvalsh(0.5 * (M + M.T))
        assert ev.min() >= -1e-12 * scale


@pytest.mark.parametrize("beta", BETAS)
def test_pair_noise_satisfies_fluctuation_dissipation(beta):
    # Eq. 19: <F_B F_B^T> = (2kT/dt) R, i.e. B B^T = R for the pair block.
    # With the sign of the chi term of T_ji taken as -1 this holds exactly;
    # the printed + sign breaks the off-diagonal torque block.
    rng = np.random.default_rng(3)
    for xi in XIS:
        R = oracle.resistances(ETA, 1.0, beta, xi)
        n = _unit(rng.normal(size=3))
        M = _pair_resistance(R, n)
        B = _pair_noise_matrix(R, n, -1.0)
        scale = np.max(np.abs(M))
        assert np.max(np.abs(B @ B.T - M)) <= 1e-12 * scale
        Bp = _pair_noise_matrix(R, n, +1.0)
        blk = np.abs(M[6:9, 9:12]).max()           # <T_i T_j> block
        assert np.max(np.abs((Bp @ Bp.T - M)[6:9, 9:12])) > 0.5 * blk


def test_regularisation_and_cutoff_in_system():
    # Sec. II.B: xi_eff = 1e-3 below 1e-3, no lubrication above xi = 0.05.
    # Two equal spheres approaching head on along x with unit closing speed.
    def force(gap_xi):
        a = 1.0
        d = 2 * a * (1 + gap_xi / 2)
        s = oracle.System([a, a], [20.0, 20.0, 20.0], shear_rate=0.0, kT=0.0,
                          noise=0, onebody=0, contact=0)
        x = np.array([[5.0, 10.0, 10.0], [5.0 + d, 10.0, 10.0]])
        U = np.array([[0.5, 0, 0], [-0.5, 0, 0]])
        s.set_state(x, U, None)
        s.evaluate()
        F, _ = s.forces()
        return F[0, 0]

    XA = lambda xi: oracle.resistances(1.0, 1.0, 1.0, xi)[0]
    # closing velocity dU = U_j - U_i = -1 along n = +x: force on i is -XA
    assert force(0.02) == pytest.approx(-XA(0.02), rel=1e-12)
    assert force(5e-4) == pytest.approx(-XA(1e-3), rel=1e-12)
    assert force(-0.01) == pytest.approx(-XA(1e-3), rel=1e-12)
    assert force(0.0499) == pytest.approx(-XA(0.0499), rel=1e-12)
    assert force(0.0501) == 0.0
