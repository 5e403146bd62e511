"""Pins of the oracle's convective flux (Sec. 3.2: Roe-type flux with MUSCL/van Leer;
reading K): consistency, the exact capture of a single moving shock and of a stationary
contact (the defining properties of Roe's linearisation), supersonic upwinding and the
rotational symmetry between the x and r directions."""
import math

import numpy as np
import pytest

import oracle as O

G = 1.4
RA = 287.05


def _q_from(p, T, u, v, Yv=0.0, ml=(0, 0, 0, 0), ms=(0, 0, 0, 0), ns=0.0):
    U = O.prim_to_cons_batch(np.array([[p, T, u, v, Yv, *ml, *ms, ns]]))[0]
    rho = U[0]
    q = np.array([rho, u, v, p, Yv, *ml, *ms, ns], dtype=float)
    return q, U


def _physical_flux(U, q, d):
    un = q[1] if d == 0 else q[2]
    p = q[3]
    F = np.zeros(14)
    F[0] = U[0] * un
    F[1] = U[1] * un + (p if d == 0 else 0.0)
    F[2] = U[2] * un + (p if d == 1 else 0.0)
    F[3] = un * (U[3] + p)
    F[4:] = U[0] * un * q[4:]
    return F


@pytest.mark.parametrize("d", [0, 1])
def test_consistency(d):
    rng = np.random.default_rng(3)
    for _ in range(50):
        q, U = _q_from(rng.uniform(5e3, 5e4), rng.uniform(180, 600), rng.uniform(-500, 500),
                       rng.uniform(-300, 300), rng.uniform(0, 0.1),
                       ml=tuple(rng.uniform(0, 1e10) * 0.3**k for k in range(4)),
                       ms=tuple(rng.uniform(0, 1e8) * 2.0**k for k in range(4)),
                       ns=rng.uniform(0, 1e12))
        F = O.roe_flux(q, q, d)
        assert np.allclose(F, _physical_flux(U, q, d), rtol=1e-13, atol=1e-300)


def _shock_states(M1, p1=2.0e4, T1=230.0):
    """Rankine-Hugoniot normal-shock relations of a perfect gas (textbook)."""
    rho1 = p1 / (RA * T1)
    c1 = math.sqrt(G * p1 / rho1)
    u1 = M1 * c1
    r = (G + 1) * M1**2 / ((G - 1) * M1**2 + 2)
    p2 = p1 * (1 + 2 * G / (G + 1) * (M1**2 - 1))
    rho2 = rho1 * r
    u2 = u1 / r
    return (rho1, u1, p1), (rho2, u2, p2), c1


@pytest.mark.parametrize("M1", [1.3, 2.0, 4.0])
@pytest.mark.parametrize("frame", [0.6, -0.7])
@pytest.mark.parametrize("d", [0, 1])
def test_single_moving_shock_is_captured_exactly(M1, frame, d):
    """Roe's linearisation satisfies F_R - F_L = A~ (U_R - U_L); for states joined by one
    shock moving with speed s (|s| above the entropy-fix threshold) the flux is F_L (s > 0)
    or F_R (s < 0) exactly."""
    (r1, u1, p1), (r2, u2, p2), c1 = _shock_states(M1)
    V = frame * c1   # shock speed in the lab frame
    vt = 37.0
    def q_of(rho, u, p):
        un, ut = u + V, vt
        return _q_from(p, p / (rho * RA), un if d == 0 else ut, ut if d == 0 else un)
    qL, UL = q_of(r1, u1, p1)
    qR, UR = q_of(r2, u2, p2)
    F = O.roe_flux(qL, qR, d)
    FL, FR = _physical_flux(UL, qL, d), _physical_flux(UR, qR, d)
    ref = FL if V > 0 else FR
    scale = np.abs(FL[:4]).max()
    assert np.allclose(F[:4], ref[:4], rtol=0, atol=1e-12 * scale)


def test_stationary_contact_is_exact():
    qL, UL = _q_from(3e4, 400.0, 0.0, 12.0)
    qR, UR = _q_from(3e4, 220.0, 0.0, 12.0)
    F = O.roe_flux(qL, qR, 0)
    assert abs(F[0]) < 1e-14 and F[1] == pytest.approx(3e4, rel=1e-14)
    assert abs(F[3]) < 1e-8


@pytest.mark.parametrize("d", [0, 1])
def test_supersonic_upwinding(d):
    """All waves right-running: the flux is the left state's (Roe property, dry gas of
    one composition); passive quantities are always carried from the upwind side."""
    qL, UL = _q_from(2e4, 250.0, 900.0 if d == 0 else 30.0, 30.0 if d == 0 else 900.0)
    qR, UR = _q_from(3e4, 300.0, 850.0 if d == 0 else -10.0, -10.0 if d == 0 else 850.0)
    F = O.roe_flux(qL, qR, d)
    FL = _physical_flux(UL, qL, d)
    assert np.allclose(F[:4], FL[:4], rtol=1e-12, atol=1e-9)
    qL2, _ = _q_from(2e4, 250.0, 900.0, 30.0, 0.02, ml=(1e10, 1e9, 1e8, 1e7), ns=1e11)
    F2 = O.roe_flux(qL2, qR, 0)
    assert np.allclose(F2[4:], F2[0] * qL2[4:], rtol=1e-15, atol=0)


def test_rotational_symmetry():
    rng = np.random.default_rng(5)
    for _ in range(20):
        qL, _ = _q_from(rng.uniform(1e4, 4e4), rng.uniform(200, 500), rng.uniform(-200, 200),
                        rng.uniform(-200, 200), rng.uniform(0, 0.05), ml=(1e9, 1e8, 1e7, 1e6))
        qR, _ = _q_from(rng.uniform(1e4, 4e4), rng.uniform(200, 500), rng.uniform(-200, 200),
                        rng.uniform(-200, 200), rng.uniform(0, 0.05))
        sw = lambda q: q[[0, 2, 1, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13]]
        F0 = O.roe_flux(sw(qL), sw(qR), 0)
        F1 = O.roe_flux(qL, qR, 1)
        assert np.allclose(F1, F0[[0, 2, 1, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13]], rtol=1e-14, atol=1e-300)


def test_mirror_state_gives_a_solid_wall():
    """A face between a state and its mirror image carries no mass, water or energy."""
    qL, _ = _q_from(2.4e4, 260.0, 120.0, 40.0, 0.03, ml=(1e10, 1e9, 1e8, 1e7))
    qR = qL.copy()
    qR[1] = -qR[1]
    F = O.roe_flux(qL, qR, 0)
    assert F[0] == 0.0 and F[3] == 0.0 and np.all(F[4:] == 0.0)


@pytest.mark.parametrize("d", [0, 1])
def test_roe_sound_speed_and_its_guard(d):
    """Reading K's Roe averages: with weights w = sqrt(rho)/(sqrt(rho_L) + sqrt(rho_R)) and
    the mean gamma, the averaged sound speed is
        c~^2 = (gamma~ - 1) (w_L h_L + w_R h_R + w_L w_R |u_R - u_L|^2 / 2),
    h = c^2/(gamma - 1) the sensible enthalpy of each side (c^2 = gamma p / rho), which
    follows from H~ - ef~ - |u~|^2/2 with the latent formation energy averaged like H.
    Hence c~^2 >= min(c_L^2, c_R^2)/2 for every physical pair, and the oracle's 1 % guard on
    c~^2 never acts on them.  Random pairs with jumps in composition (vapour up to 0.2,
    droplets, crystals), temperature (180-900 K) and velocity (up to 800 m/s)."""
    rng = np.random.default_rng(11 + d)
    for _ in range(400):
        qs = []
        for _side in range(2):
            q, _ = _q_from(rng.uniform(5e3, 5e4), rng.uniform(180, 900), rng.uniform(-800, 800),
                           rng.uniform(-800, 800), rng.uniform(0, 0.2),
                           ml=tuple(rng.uniform(0, 1e11) * 0.1**k for k in range(4)),
                           ms=tuple(rng.uniform(0, 1e9) * 1.0**k for k in range(4)),
                           ns=rng.uniform(0, 1e12))
            qs.append(q)
        qL, qR = qs
        c2, c2_used, c2L, c2R = O.roe_c2(qL, qR, d)
        gL, gR = c2L * qL[0] / qL[3], c2R * qR[0] / qR[3]
        sL, sR = math.sqrt(qL[0]), math.sqrt(qR[0])
        wL, wR = sL / (sL + sR), sR / (sL + sR)
        du2 = (qR[1] - qL[1]) ** 2 + (qR[2] - qL[2]) ** 2
        expect = (0.5 * (gL + gR) - 1.0) * (wL * c2L / (gL - 1.0) + wR * c2R / (gR - 1.0) + 0.5 * wL * wR * du2)
        assert c2 == pytest.approx(expect, rel=1e-11)
        assert c2 >= 0.5 * min(c2L, c2R)
        assert c2_used == c2
