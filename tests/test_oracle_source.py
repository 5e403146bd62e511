"""Pins of the oracle's phase-change source (Sec. 2.2, Eqs. (1)-(21); readings D, F-J):
brute force on the Gibbs energy of Eq. (2), the molecular (Becker-Doering) form of the CNT
prefactor, special cases of the growth law, and mass conservation of every source."""
import math

import numpy as np
import pytest

import oracle as O
from synth import cases

NA, KB, MW = 6.02214076e23, 1.380649e-23, 0.018015
PI = math.pi


def _state(p, T, Yv, ml=(0, 0, 0, 0), ms=(0, 0, 0, 0), ns=0.0, u=0.0):
    return O.prim_to_cons_batch(np.array([[p, T, u, 0.0, Yv, *ml, *ms, ns]]))[0]


def _yv_for_S(S, T, p):
    """Vapour mass fraction giving liquid saturation ratio S at (T, p)."""
    Ra, Rv = 287.05, O.const("R_v")
    pv = S * math.exp(O.ln_psat_l(T))
    return pv * Ra / (Rv * (p - pv) + pv * Ra)


def _case(**kw):
    c, _ = cases.mixing_layer_case(seeded=False)
    c.update(kw)
    return c


GRID = [(S, T) for S in (1.5, 3.0, 5.0, 10.0, 20.0) for T in (200.0, 220.0, 240.0)]


@pytest.mark.parametrize("S,T", GRID)
def test_kelvin_radius_and_barrier_by_brute_force(S, T):
    """Eq. (3) is the maximum of Eq. (2): find max_r dG(r) numerically, compare r* with
    the oracle's r_crit and dG(r*)/kT with the barrier implied by ln J_het - ln J_hom."""
    p = 24e3
    Yv = _yv_for_S(S, T, p)
    U = _state(p, T, Yv, ns=0.0)
    rho = U[0]
    c = _case(n_soot=1.0)   # soot at the reference number per volume: gate = 1
    U[13] = 1.0
    Q, aux = O.source_batch(c, U, 1e-9)
    lnS, rc, lnJhom, lnJhet = aux[0, 0], aux[0, 5], aux[0, 2], aux[0, 3]
    assert lnS == pytest.approx(math.log(S), rel=1e-10)
    sig = O.sigma_lg(T)
    Rv = O.const("R_v")
    dG = lambda r: 4.0 / 3.0 * PI * r**3 * 1000.0 * (-Rv * T * lnS) + 4.0 * PI * r * r * sig
    # golden-section search for the maximum of dG on (0, 1e-7)
    a, b = 1e-12, 1e-7
    gr = (math.sqrt(5.0) - 1.0) / 2.0
    for _ in range(200):
        x1, x2 = b - gr * (b - a), a + gr * (b - a)
        if dG(x1) > dG(x2):
            b = x2
        else:
            a = x1
    rstar = 0.5 * (a + b)
    assert rc == pytest.approx(rstar, rel=1e-6)
    barrier = dG(rstar) / (KB * T)
    # f(90 deg) = 1/2 (Eq. (9)): ln J_het - ln J_hom = (1 - f) dG*/kT
    assert (lnJhet - lnJhom) == pytest.approx(0.5 * barrier, rel=1e-9)


@pytest.mark.parametrize("S,T", GRID)
def test_cnt_prefactor_molecular_form(S, T):
    """The prefactor of Eq. (4), q_c sqrt(2 sigma N_A^3/(pi M^3)) rho_g^2/rho_l, equals the
    Becker-Doering/Frenkel molecular form n_v^2 v_m sqrt(2 sigma/(pi m)) with m the molecular
    mass, n_v the vapour number density and v_m the molecular volume of the liquid."""
    p = 24e3
    Yv = _yv_for_S(S, T, p)
    U = _state(p, T, Yv)
    rho = U[0]
    c = _case(n_soot=1.0)
    U[13] = 1.0   # n_soot per volume = 1 = reference -> gate 1
    _, aux = O.source_batch(c, U, 1e-9)
    lnA = 2.0 * aux[0, 3] - aux[0, 2]     # ln J_het = lnA - dG/2kT, ln J_hom = lnA - dG/kT
    m = MW / NA
    rhov = rho * Yv
    nv = rhov / m
    vm = m / 1000.0
    lnA_mol = math.log(nv * nv * vm * math.sqrt(2.0 * O.sigma_lg(T) / (PI * m)))
    assert lnA == pytest.approx(lnA_mol, abs=1e-9)


@pytest.mark.parametrize("S", [0.2, 0.9, 1.0])
def test_no_nucleation_at_or_below_saturation(S):
    T, p = 220.0, 24e3
    U = _state(p, T, _yv_for_S(S, T, p), ns=1e12)
    Q, aux = O.source_batch(_case(), U, 1e-5)
    assert aux[0, 2] == -math.inf and aux[0, 3] == -math.inf
    assert np.all(Q == 0.0)   # no population: exactly zero source
    assert aux[0, 4] == 0.0


def test_het_nucleation_gated_by_soot():
    """Without soot only homogeneous nucleation occurs (Sec. 4.3, hydrogen case)."""
    T, p = 220.0, 24e3
    U = _state(p, T, _yv_for_S(8.0, T, p), ns=0.0)
    Q0, aux0 = O.source_batch(_case(), U, 1e-9)
    assert aux0[0, 3] == -math.inf and aux0[0, 2] > -math.inf


def _gas(T, p, Yv):
    """Gas-phase transport inputs of the growth law (reading G)."""
    Ra, Rv = 287.05, O.const("R_v")
    cp = (1 - Yv) * (Ra / 0.4 + Ra) + Yv * 1859.0
    cv = (1 - Yv) * Ra / 0.4 + Yv * O.const("cv_v")
    mu = 1.716e-5 * (T / 273.15) ** 1.5 * (273.15 + 110.4) / (T + 110.4)
    lam = mu * cp / 0.71
    lbar = 1.5 * mu * math.sqrt(((1 - Yv) * Ra + Yv * Rv) * T) / p
    return lam, lbar, cp / cv, cp


def test_growth_vanishes_at_critical_radius_and_has_the_right_sign():
    T, p, Yv = 230.0, 24e3, 0.002
    pv = p * Yv * O.const("R_v") / ((1 - Yv) * 287.05 + Yv * O.const("R_v"))
    lnS = math.log(pv) - O.ln_psat_l(T)
    Ts = O.tsat(pv, 0)
    sig = O.sigma_lg(T)
    h = O.hfg(T)
    lam, lbar, gam, cp = _gas(T, p, Yv)
    rc = 2 * sig / (1000.0 * O.const("R_v") * T * lnS)
    g = lambda r, lnS_=lnS, Ts_=Ts: O.growth(r, T, Ts_, lnS_, sig, 1000.0, h, lam, lbar, gam, cp)
    assert abs(g(rc)) < 1e-12 * abs(g(10 * rc))
    assert g(2 * rc) > 0 and g(1e-6) > 0 and g(0.5 * rc) < 0
    # sub-saturated: every droplet evaporates
    assert g(1e-7, -0.2, O.tsat(pv * math.exp(-0.2 - lnS), 0)) < 0


def test_growth_continuum_limit_is_heat_conduction():
    """Kn -> 0: Eq. (16) reduces to conduction-limited growth lam dT (1 - rc/r)/(rho h r)."""
    T, p, Yv = 230.0, 24e3, 0.002
    pv = p * Yv * O.const("R_v") / ((1 - Yv) * 287.05 + Yv * O.const("R_v"))
    lnS = math.log(pv) - O.ln_psat_l(T)
    Ts = O.tsat(pv, 0)
    sig, h = O.sigma_lg(T), O.hfg(T)
    lam, _, gam, cp = _gas(T, p, Yv)
    r = 5e-6
    rc = 2 * sig / (1000.0 * O.const("R_v") * T * lnS)
    gc = O.growth(r, T, Ts, lnS, sig, 1000.0, h, lam, 1e-30, gam, cp)
    assert gc == pytest.approx(lam * (Ts - T) * (1 - rc / r) / (1000.0 * h * r), rel=1e-12)


def test_growth_regular_at_saturation():
    """The Delta T / ln S form of reading G is continuous through S = 1."""
    T, p = 230.0, 24e3
    lam, lbar, gam, cp = _gas(T, p, 0.001)
    sig, h = O.sigma_lg(T), O.hfg(T)
    pv0 = math.exp(O.ln_psat_l(T))
    vals = []
    for e in (-2e-8, -5e-9, 5e-9, 2e-8):
        pv = pv0 * math.exp(e)
        vals.append(O.growth(1e-7, T, O.tsat(pv, 0), math.log(pv) - O.ln_psat_l(T), sig, 1000.0, h,
                             lam, lbar, gam, cp))
    assert np.all(np.isfinite(vals))
    assert abs(vals[1] - vals[2]) < 1e-3 * abs(vals[0] - vals[3]) + 1e-6 * abs(vals[0])


def test_growth_moment_source_is_exact_for_a_monodisperse_population():
    """For mu_k = n r^k the r20 closure (Eq. (21)) is exact: the source of the k-th moment
    must be k n r^(k-1) G(r), with G from Eq. (16); checks indices, moment scaling and the
    per-volume factor rho of Eq. (26)."""
    T, p, Yv = 230.0, 24e3, 0.0015
    r, n = 3e-7, 1e9
    ml = tuple(n * (r / 1e-6) ** k for k in range(4))
    U = _state(p, T, Yv, ml=ml)
    rho = U[0]
    c = _case(freezing=0)
    Q, aux = O.source_batch(c, U, 1e-12)
    G = aux[0, 7]
    assert G != 0.0
    for k in range(1, 4):
        expect = rho * k * n * r ** (k - 1) * G / 1e-6**k
        assert Q[0, 5 + k] == pytest.approx(expect, rel=1e-12)
    assert Q[0, 5] == 0.0 or aux[0, 0] > 0
    # nucleation at S < 1 is off, so Q_0 = 0 exactly
    if aux[0, 0] <= 0:
        assert Q[0, 5] == 0.0


def test_nucleation_moment_source_and_eq6_mass():
    """Newly nucleated droplets sit at r_crit (Eq. (20)): Q_k ~ J r_crit^k, and the liquid
    mass gain equals Eq. (6): (4/3) pi r_crit^3 rho_l J/(1+phi)."""
    T, p = 220.0, 24e3
    U = _state(p, T, _yv_for_S(12.0, T, p))
    c = _case()
    Q, aux = O.source_batch(c, U, 1e-12)
    rc, phi = aux[0, 5], aux[0, 6]
    Jhom = math.exp(aux[0, 2])
    for k in range(3):
        assert Q[0, 6 + k] / Q[0, 5 + k] == pytest.approx(rc / 1e-6, rel=1e-12)
    dYl = 4.0 / 3.0 * PI * 1000.0 * Q[0, 8] * 1e-18
    assert dYl == pytest.approx(4.0 / 3.0 * PI * rc**3 * 1000.0 * Jhom / (1.0 + phi), rel=1e-12)
    assert phi > 0


def _random_states(n, seed=7):
    rng = np.random.default_rng(seed)
    P = np.zeros((n, 14))
    P[:, 0] = rng.uniform(8e3, 40e3, n)
    P[:, 1] = rng.uniform(190.0, 300.0, n)
    P[:, 2] = rng.uniform(-50, 400, n)
    P[:, 4] = 10 ** rng.uniform(-5, -1, n)
    for base, rho_d in ((5, 1000.0), (9, 917.0)):
        Y = 10 ** rng.uniform(-14, -2.5, n)            # condensed mass fraction
        r = 10 ** rng.uniform(-9, -5.5, n)
        sg = np.exp(rng.uniform(0, 0.4, n) ** 2)       # lognormal spread: mu2 mu0 >= mu1^2
        nn = Y / (4.0 / 3.0 * PI * rho_d * r**3 * sg**4.5)
        for k in range(4):
            P[:, base + k] = nn * (r / 1e-6) ** k * sg ** (k * k / 2.0)
    P[:, 13] = 10 ** rng.uniform(8, 13, n)
    return O.prim_to_cons_batch(P)


@pytest.mark.parametrize("dt", [1e-7, 1e-5, 1e-3])
def test_every_source_conserves_water_and_never_creates_mass(dt):
    """Eqs. (18), (25): the vapour sink is the condensed gain negated, cell by cell; rho,
    momentum, energy and soot have no source (reading E: latent heat is in the formation
    energies)."""
    U = _random_states(3000)
    c = _case()
    Q, aux = O.source_batch(c, U, dt)
    assert np.all(np.isfinite(Q))
    water = Q[:, 4] + 4.0 / 3.0 * PI * (1000.0 * Q[:, 8] + 917.0 * Q[:, 12]) * 1e-18
    scale = np.abs(Q[:, 4]) + 4.0 / 3.0 * PI * (1000.0 * np.abs(Q[:, 8]) + 917.0 * np.abs(Q[:, 12])) * 1e-18
    assert np.all(np.abs(water) <= 1e-13 * scale + 1e-300)
    assert np.all(Q[:, [0, 1, 2, 3, 13]] == 0.0)
    # positivity limiters (reading J): the source alone never drives a phase negative
    new = U + dt * Q
    assert np.all(new[:, 4] >= -1e-14 * U[:, 4])
    assert np.all(new[:, 8] >= -1e-12 * np.abs(U[:, 8]))
    assert np.all(new[:, 12] >= -1e-12 * np.abs(U[:, 12]))
    assert aux[:, 4].sum() > 100


def _freezing_state(T, p, r, n, ns):
    """Droplets of radius r (n per kg) in vapour exactly at ice saturation (liquid
    subsaturated: the droplets evaporate slowly while they freeze)."""
    ml = tuple(n * (r / 1e-6) ** k for k in range(4))
    Ra, Rv = 287.05, O.const("R_v")
    pv = math.exp(O.ln_psat_i(T))
    Yv = pv * Ra / (Rv * (p - pv) + pv * Ra)
    return _state(p, T, Yv, ml=ml, ns=ns)


def test_freezing_transfers_mass_without_loss():
    """Eqs. (12)-(15) with reading H, checked without restating the source's formulas:
    - frozen droplets become crystals of equal mass: the ice mass gained equals the liquid
      mass lost by freezing, and the crystals' mean radius mu1/mu0 is r (rho_l/rho_s)^(1/3);
    - the homogeneous part of the per-droplet rate scales with the droplet volume (x8 for
      twice the radius) and equals Koop's rate coefficient (cm^-3 s^-1 -> m^-3 s^-1) times
      that volume;
    - the immersion part does not depend on the droplet size and equals
      k_imm n_s 4 pi <r_p^2> chi, with <r_p^2> of the lognormal soot spectrum by quadrature
      and chi = min(1, n_soot / mu0);
    - over many short stages the droplet number decays as exp(-omega t), the solution of the
      first-order freezing kinetics."""
    T, p, r, n = 225.0, 24e3, 2e-7, 1e9
    c = _case(freezing=1)
    dt = 1e-12
    # homogeneous freezing alone (no soot): volume scaling and Koop's coefficient
    Q1, a1 = O.source_batch(c, _freezing_state(T, p, r, n, 0.0), dt)
    Q2, a2 = O.source_batch(c, _freezing_state(T, p, 2 * r, n, 0.0), dt)
    assert a2[0, 10] / a1[0, 10] == pytest.approx(8.0, rel=1e-12)
    daw = 1.0 - math.exp(O.ln_psat_i(T) - O.ln_psat_l(T))
    assert a1[0, 10] == pytest.approx(1e6 * 10 ** O.koop_log10J(daw) * 4.0 / 3.0 * PI * r**3, rel=1e-12)
    # immersion part alone at 250 K, where Delta a_w = 0.20 lies below Koop's range (no
    # homogeneous freezing): soot per kg ns with chi = min(1, ns / n)
    rm, sg = c["soot_rm"], c["soot_sigma"]
    x = np.linspace(-10, 10, 20001)
    pdf = np.exp(-0.5 * x * x) / math.sqrt(2 * PI)
    rp2 = np.trapezoid(pdf * (rm * np.exp(math.log(sg) * x)) ** 2, x)     # <r_p^2> by quadrature
    for ns_per_kg in (0.25 * n, 4.0 * n):
        om = []
        for rr in (r, 2 * r):
            U = _freezing_state(250.0, p, rr, n, 0.0)
            U[13] = U[0] * ns_per_kg
            om.append(O.source_batch(c, U, dt)[1][0, 10])
        assert om[0] == pytest.approx(om[1], rel=1e-12)                    # size-independent
        assert om[0] == pytest.approx(1.0 * 1e8 * 4.0 * PI * rp2 * min(1.0, ns_per_kg / n), rel=1e-9)
    # mass transfer: ice gained = liquid lost to freezing, crystals at r (rho_l/rho_s)^(1/3)
    U = _freezing_state(T, p, r, n, 1e12)
    Q, aux = O.source_batch(c, U, dt)
    cf = O.source_batch(dict(c, freezing=0), U, dt)[0]
    dliq_freeze = 1000.0 * (Q[0, 8] - cf[0, 8])      # rho_l d(mu3) from freezing alone
    dice = 917.0 * Q[0, 12]
    assert dice > 0 and dice == pytest.approx(-dliq_freeze, rel=1e-9)
    assert Q[0, 10] / Q[0, 9] * 1e-6 == pytest.approx(r * (1000.0 / 917.0) ** (1.0 / 3.0), rel=1e-12)
    # number decay over many short stages against exp(-omega t)
    omega = aux[0, 10]
    t_end = 0.5 / omega
    m = 2000
    h = t_end / m
    cnum = dict(c)
    V = U.copy()
    for _ in range(m):
        Qs, _ = O.source_batch(cnum, V, h)
        V = V + h * Qs[0]                            # no transport: the cell's own kinetics
    # the liquid also evaporates slightly (subsaturated): compare number, which only
    # freezing changes (evaporation of a present population keeps mu0)
    assert V[5] / U[5] == pytest.approx(math.exp(-omega * t_end), rel=2e-3)


def test_koop_threshold_temperature():
    """The Koop fit with a_w = 1 and Sonntag's a_w^ice gives J = 1e9..1e12 cm^-3 s^-1 near
    235-237 K, the homogeneous freezing limit of pure water droplets."""
    daw = 1 - math.exp(O.ln_psat_i(236.0) - O.ln_psat_l(236.0))
    assert 8.0 < O.koop_log10J(daw) < 13.0


@pytest.mark.parametrize("S", [1.05, 1.5, 0.7])
@pytest.mark.parametrize("dt", [1e-6, 1e-4, 1e-2])
def test_growth_stage_never_overshoots_equilibrium(S, dt):
    """Reading J: over one stage the growth exchange follows the exponential solution of the
    linearised relaxation, so a dense supersaturated (subsaturated) population condenses
    (evaporates) towards saturation without crossing it, for any stage length."""
    T, p = 230.0, 24e3
    Yv = _yv_for_S(S, T, p)
    r, n = 5e-7, 1e10
    ml = tuple(n * (r / 1e-6) ** k for k in range(4))
    U = _state(p, T, Yv, ml=ml)
    c = _case(freezing=0)
    Q, aux = O.source_batch(c, U, dt)
    lnS0 = aux[0, 0]
    U1 = U + dt * Q
    _, aux1 = O.source_batch(c, U1, dt)
    lnS1 = aux1[0, 0]
    kelvin = 2 * O.sigma_lg(T) / (1000.0 * O.const("R_v") * T * r)   # equilibrium ln S of the drops
    assert abs(lnS1 - kelvin) <= abs(lnS0 - kelvin) * (1 + 1e-9)
    assert (lnS1 - kelvin) * (lnS0 - kelvin) >= -1e-3 * abs(lnS0 - kelvin) ** 2


def test_growth_limiter_reduces_to_explicit_rate_for_short_stages():
    T, p = 230.0, 24e3
    U = _state(p, T, _yv_for_S(1.3, T, p), ml=tuple(1e8 * (1e-7 / 1e-6) ** k for k in range(4)))
    c = _case(freezing=0)
    _, a1 = O.source_batch(c, U, 1e-14)
    _, a2 = O.source_batch(c, U, 1e-13)
    assert a1[0, 7] == pytest.approx(a2[0, 7], rel=1e-9)


def test_lognormal_spectrum_from_moments_is_exact():
    """Derived quantities 13-16: a lognormal population (N, r_m, sigma_g) has moments
    mu_k = N r_m^k exp(k^2 ln^2 sigma_g / 2); the reconstruction returns r_m and sigma_g."""
    c, uf = cases.closed_box_case(nx=4, nr=2)
    o = O.Oracle(c, uf)
    U = o.init_state()
    for rm, sg, rmi, sgi in ((0.2, 1.6, 1.5, 1.3), (0.015, 1.1, 3.0, 2.0)):
        s2, s2i = np.log(sg) ** 2, np.log(sgi) ** 2
        U2 = U.copy()
        for k in range(4):
            U2[5 + k] = U2[0] * 1e10 * rm ** k * np.exp(k * k * s2 / 2)
            U2[9 + k] = U2[0] * 1e8 * rmi ** k * np.exp(k * k * s2i / 2)
        got = [o.derived(U2, w)[0, 0] for w in (13, 14, 15, 16)]
        assert np.allclose(got, [rm, sg, rmi, sgi], rtol=1e-12), got
