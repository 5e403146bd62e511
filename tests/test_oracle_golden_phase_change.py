"""Pins of the oracle's phase-change closed forms against values evaluated independently
from the paper's equations (tests/golden/make_phase_change_golden.py: mpmath at 50 digits,
exact rationals for Koop's polynomial), plus the asymptotic structure of Young's law.

- Eqs. (3), (4), (9), (10): r_crit, the barrier dG*/kT, ln J_hom, ln J_het on the (S, T)
  grid {1.5, 3, 5, 10, 20} x {200, 220, 240 K}.
- Eq. (5): the Kantrowitz factor phi with alpha_crit read as Young's heat-transfer
  coefficient at r_crit.
- Eq. (16): Young's growth rate, liquid and ice, Kn from 40 to 0.01, in both directions of
  the phase change; its Knudsen dependence (affine in 1/r for beta = 0) and the
  free-molecular limit.
- Koop et al. (2000) Eq. (7): log10 J of homogeneous freezing over Delta a_w in [0.26, 0.34].

A dropped term, a wrong sign or a single mistyped coefficient in any of these functions
moves its values far outside the tolerances below."""
import math

import numpy as np
import pytest

import oracle as O
from conftest import read_golden
from synth import cases

P_GAS = 24e3


def _state(p, T, Yv, ml=(0, 0, 0, 0), ms=(0, 0, 0, 0), ns=0.0):
    return O.prim_to_cons_batch(np.array([[p, T, 0.0, 0.0, Yv, *ml, *ms, ns]]))[0]


def _case(**kw):
    c, _ = cases.mixing_layer_case(seeded=False)
    c.update(kw)
    return c


CNT = read_golden("cnt_kantrowitz.txt")


@pytest.mark.parametrize("row", CNT, ids=[f"S{r[0]}-T{float(r[1]):.0f}" for r in CNT])
def test_nucleation_closed_forms_and_kantrowitz_factor(row):
    S, T, Yv, rc, barrier, lnJhom, lnJhet, phi = (float(v) for v in row)
    U = _state(P_GAS, T, Yv)
    U[13] = 1.0                              # soot at the reference number: gate = 1
    _, aux = O.source_batch(_case(n_soot=1.0), U, 1e-15)
    assert aux[0, 0] == pytest.approx(math.log(S), rel=1e-13)
    assert aux[0, 5] == pytest.approx(rc, rel=1e-12)
    assert aux[0, 2] == pytest.approx(lnJhom, abs=1e-12 * barrier)
    assert aux[0, 3] == pytest.approx(lnJhet, abs=1e-12 * barrier)
    assert 2.0 * (aux[0, 3] - aux[0, 2]) == pytest.approx(barrier, rel=1e-11)
    assert aux[0, 6] == pytest.approx(phi, rel=1e-12)


def test_kantrowitz_factor_is_nearly_proportional_to_vapour_density():
    """Eq. (5): phi = q_c rho_v sqrt(R T / 2 pi) (h^2/(R T^2) - h/T) / alpha_crit.  Critical
    nuclei are far smaller than the mean free path (Kn_c ~ 10-100), where Young's
    alpha_crit = lambda / (r_c + 3.78 (1 - nu) lbar / (2 Pr)) depends on r_c only weakly.  So
    at fixed T, phi / S (S ~ rho_v) stays within 20 % over S = 1.5 .. 20 and falls slowly
    as S grows (r_c shrinks, so alpha_crit grows), and it grows with T (the bracket and
    sqrt(R T) grow faster than alpha_crit)."""
    by_T = {}
    for row in CNT:
        S, T, phi = float(row[0]), float(row[1]), float(row[7])
        assert phi > 0
        by_T.setdefault(T, []).append((S, phi / S))
    prev = 0.0
    for T in sorted(by_T):
        v = np.array([x for _, x in sorted(by_T[T])])
        assert v.max() / v.min() < 1.2, (T, v)
        assert np.all(np.diff(v) < 0), (T, v)
        assert v.min() > prev
        prev = v.max()


YOUNG = read_golden("young_growth.txt")


@pytest.mark.parametrize("row", YOUNG, ids=[f"{r[0]}-S{r[1]}-T{float(r[2]):.0f}-r{r[3]}" for r in YOUNG])
def test_young_growth_rate(row):
    phase = row[0]
    S, T, r, n, Yv, G, Kn = (float(v) for v in row[1:])
    mom = tuple(n * (r / 1e-6) ** k for k in range(4))
    if phase == "l":
        U = _state(P_GAS, T, Yv, ml=mom)
    else:
        U = _state(P_GAS, T, Yv, ms=mom)
    _, aux = O.source_batch(_case(freezing=0), U, 1e-15)   # stage limiter inactive at this dt
    g = aux[0, 7] if phase == "l" else aux[0, 8]
    assert g == pytest.approx(G, rel=1e-11), (g, G, Kn)


def _gas_inputs(T, p, Yv):
    """A fixed set of gas inputs for direct calls of the growth law (values only need to be
    plausible: the test checks the law's dependence on r, not the property models)."""
    return dict(lam_g=0.0205, lbar=2.4e-7, gam_g=1.4, cp_g=1004.0)


def test_young_knudsen_dependence_is_affine_in_inverse_radius():
    """Eq. (16) with beta = 0: lambda dT (1 - r_c/r) / (rho h G r) = 1 + 3.78 (1 - nu) Kn/Pr
    with Kn = lbar/(2r), an affine function of 1/r whose intercept is exactly 1 (the
    continuum limit) and whose slope is 3.78 (1 - nu) lbar / (2 Pr).  The slope is
    proportional to lbar and, through nu, depends on alpha, T_sat, gamma, c_p only."""
    T, Tsat, lnS = 230.0, 232.0, 0.12
    sig, rho_d, h = O.sigma_lg(T), 1000.0, O.hfg(T)
    gi = _gas_inputs(T, P_GAS, 1e-3)
    Rv = O.const("R_v")
    rc = 2 * sig / (rho_d * Rv * T * lnS)
    radii = np.geomspace(3 * rc, 1e-4, 25)

    def den(r, lbar):
        G = O.growth(r, T, Tsat, lnS, sig, rho_d, h, gi["lam_g"], lbar, gi["gam_g"], gi["cp_g"])
        return gi["lam_g"] * (Tsat - T) * (1 - rc / r) / (rho_d * h * G * r)

    for lbar in (1e-8, 2.4e-7, 5e-6):
        d = np.array([den(r, lbar) for r in radii])
        slope, icpt = np.polyfit(1.0 / radii, d, 1)
        assert icpt == pytest.approx(1.0, abs=1e-9)
        resid = d - (icpt + slope / radii)
        assert np.max(np.abs(resid) / d) < 1e-11
        nu_from_slope = 1.0 - slope * 2.0 * 0.71 / (3.78 * lbar)
        # nu is a property of the gas state, not of lbar
        if lbar == 1e-8:
            nu0 = nu_from_slope
        assert nu_from_slope == pytest.approx(nu0, rel=1e-7)
    # Young's nu for water at these conditions: R T_sat / h (alpha - 1/2 - ...) is
    # O(0.04) x (11 - 0.5 - 0.86 c_p T_sat / h) ~ 0.39 (alpha = 11 dominates)
    assert 0.3 < nu0 < 0.5


def test_young_free_molecular_limit_is_size_independent():
    """Kn >> 1: den ~ 3.78 (1 - nu) lbar/(2 Pr r), so G (1 - r_c/r)^-1 tends to a constant
    independent of r (free-molecular growth), and doubling lbar halves it."""
    T, Tsat, lnS = 230.0, 232.0, 0.12
    sig, rho_d, h = O.sigma_lg(T), 1000.0, O.hfg(T)
    gi = _gas_inputs(T, P_GAS, 1e-3)
    rc = 2 * sig / (rho_d * O.const("R_v") * T * lnS)

    def g(r, lbar):
        return O.growth(r, T, Tsat, lnS, sig, rho_d, h, gi["lam_g"], lbar, gi["gam_g"], gi["cp_g"]) / (1 - rc / r)

    lbar = 1e-3    # Kn = 2e4 at 2 r_c, 2e3 at 20 r_c: the 1/Kn corrections are 2e-5 and 2e-4
    a, b = g(2 * rc, lbar), g(20 * rc, lbar)
    assert a == pytest.approx(b, rel=5e-4)
    assert g(2 * rc, 2 * lbar) == pytest.approx(0.5 * a, rel=1e-4)


KOOP = read_golden("koop_2000.txt")


@pytest.mark.parametrize("row", KOOP, ids=[r[0] for r in KOOP])
def test_koop_polynomial(row):
    x, l10 = float(row[0]), float(row[1])
    # the cubic's terms reach 3e3, so FP64 evaluation carries about 1e-12 absolute error
    assert O.koop_log10J(x) == pytest.approx(l10, abs=2e-11)


def test_koop_range_and_monotonicity():
    """The fit increases with Delta a_w over its validity range; below 0.26 the rate is zero
    (log10 J = -inf) and above 0.34 it holds the range-end value (reading H)."""
    xs = np.linspace(0.26, 0.34, 81)
    v = np.array([O.koop_log10J(x) for x in xs])
    assert np.all(np.diff(v) > 0)
    assert O.koop_log10J(0.2599) == -math.inf
    assert O.koop_log10J(0.36) == O.koop_log10J(0.34)
