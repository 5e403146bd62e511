"""Pins of the oracle's thermophysical closed forms (Sec. 2.1 and Eq. (1); readings B-E)
against published property tables and thermodynamic identities."""
import math

import numpy as np
import pytest

import oracle as O
from conftest import read_golden


@pytest.mark.parametrize("row", read_golden("saturation_pressure.txt"))
def test_sonntag_against_tables(row):
    phase, T, p = row[0], float(row[1]), float(row[2])
    f = O.ln_psat_l if phase == "l" else O.ln_psat_i
    assert math.exp(f(T)) == pytest.approx(p, rel=3e-3)


def test_triple_point_agreement():
    T = 273.16
    pl, pi = math.exp(O.ln_psat_l(T)), math.exp(O.ln_psat_i(T))
    assert abs(pl - pi) / pl < 2e-4
    # below the triple point ice is the stable phase: p_sat,i < p_sat,l
    for T in np.linspace(150.0, 272.0, 40):
        assert O.ln_psat_i(T) < O.ln_psat_l(T)


def test_monotone_and_clausius_clapeyron():
    """d ln p_sat/dT = h/(R_v T^2): ties Sonntag's curves to the latent heats of reading E."""
    Rv = O.const("R_v")
    T = np.linspace(160.0, 330.0, 60)
    lpl = np.array([O.ln_psat_l(t) for t in T])
    assert np.all(np.diff(lpl) > 0)
    for t in (250.0, 273.15, 300.0):
        h = 1e-3
        slope = (O.ln_psat_l(t + h) - O.ln_psat_l(t - h)) / (2 * h)
        assert slope == pytest.approx(O.hfg(t) / (Rv * t * t), rel=1.5e-2)
    t = 273.15
    slope_i = (O.ln_psat_i(t + 1e-3) - O.ln_psat_i(t - 1e-3)) / 2e-3
    assert slope_i == pytest.approx((2.501e6 + 3.337e5) / (Rv * t * t), rel=2e-3)


@pytest.mark.parametrize("which", [0, 1])
def test_tsat_inverts_psat(which):
    f = O.ln_psat_l if which == 0 else O.ln_psat_i
    for T in np.linspace(140.0, 330.0, 39):
        pv = math.exp(f(T))
        assert O.tsat(pv, which) == pytest.approx(T, rel=1e-12)


@pytest.mark.parametrize("row", read_golden("surface_tension.txt"))
def test_surface_tension_iapws(row):
    T, s = float(row[0]), float(row[1])
    assert O.sigma_lg(T) * 1e3 == pytest.approx(s, abs=0.011)


def test_latent_heats_from_formation_energies():
    assert O.hfg(273.15) == pytest.approx(2.501e6, rel=1e-14)
    # h_l - h_s at the reference = 3.337e5 (c_l T - c_s T - e0_s)
    assert 4186.0 * 273.15 - (2100.0 * 273.15 + O.const("e0_s")) == pytest.approx(3.337e5, rel=1e-12)


def _cons(p, T, u=0.0, v=0.0, Yv=0.0, ml=(0, 0, 0, 0), ms=(0, 0, 0, 0), ns=0.0):
    return O.prim_to_cons_batch(np.array([[p, T, u, v, Yv, *ml, *ms, ns]]))[0]


def test_dry_air_is_textbook_ideal_gas():
    U = _cons(24e3, 220.0, 100.0, 20.0)
    rho, u, v, p, T, Yv, Yl, Ys, c2 = O.cons_to_prim_batch(U)[0]
    assert p == pytest.approx(24e3, rel=1e-14) and T == pytest.approx(220.0, rel=1e-14)
    assert rho == pytest.approx(24e3 / (287.05 * 220.0), rel=1e-14)
    assert c2 == pytest.approx(1.4 * p / rho, rel=1e-14)
    # E = cv T + |u|^2/2 with cv = R/(gamma-1)
    assert U[3] / U[0] == pytest.approx(287.05 / 0.4 * 220.0 + 0.5 * (100.0**2 + 20.0**2), rel=1e-14)


def test_condensation_at_fixed_energy_releases_latent_heat():
    """Moving dY of vapour to liquid at constant rho and rho*E raises T by
    (h_fg - R_v T) dY / c_v: the latent heat lives in the formation energies."""
    Rv = O.const("R_v")
    T0 = 250.0
    U = _cons(30e3, T0, Yv=0.02)
    P0 = O.cons_to_prim_batch(U)[0]
    dY = 1e-7
    U2 = U.copy()
    U2[4] -= U[0] * dY
    # liquid mass fraction dY as a monodisperse population of 1 um droplets
    r = 1e-6
    n = dY / (4.0 / 3.0 * math.pi * 1000.0 * r**3)
    for k in range(4):
        U2[5 + k] = U[0] * n * (r / 1e-6) ** k
    P1 = O.cons_to_prim_batch(U2)[0]
    Yv = 0.02
    cv = (1 - Yv) * 287.05 / 0.4 + Yv * O.const("cv_v")
    dT_expect = (O.hfg(T0) - Rv * T0) * dY / cv
    assert P1[4] - P0[4] == pytest.approx(dT_expect, rel=1e-3)
