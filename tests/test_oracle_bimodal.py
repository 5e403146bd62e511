"""Pins of the oracle's bimodal liquid (Sec. 2.2: two independent liquid moment sets, one
per nucleation mechanism; reading P).  The second set lives in fields 14..17.

What fixes it without a reference implementation:
  - without soot there is no heterogeneous nucleation, and the bimodal run is the
    single-set run bit for bit (the second set stays exactly empty);
  - transport is linear in the moments and the flow sees only the total liquid, so a
    population split into two equal halves moves exactly like the whole;
  - a closed box conserves mass, water and energy with both sets active;
  - nucleation splits into the two sets in the ratio of Eqs. (4) and (10),
    J_hom / J_het = exp(-(1 - f) dG*/kT) / gate, both at the Kelvin radius of Eq. (3);
  - immersion freezing (Eqs. (14)-(15)) takes only droplets of heterogeneous origin, at
    the per-droplet rate k n_s 4 pi <r_p^2> chi of reading H;
  - one population behaves the same in either set (same growth law, Eq. (16));
  - the lognormal spectrum of each set is recovered from its moments.
"""
import math

import numpy as np
import pytest

import oracle as O
from synth import cases

PI = math.pi


def _state(p, T, Yv, ml=(0, 0, 0, 0), ms=(0, 0, 0, 0), ns=0.0, mh=(0, 0, 0, 0)):
    """Bimodal conserved state (18 fields): the first liquid set ml, ice ms, second set mh."""
    u = O.prim_to_cons_batch(np.array([[p, T, 0.0, 0.0, Yv, *ml, *ms, ns]]))[0]
    rho = u[0]
    # moving liquid between the sets does not change rho: Y_l is the sum of both
    out = np.zeros(18)
    out[:14] = u
    if any(mh):
        tot = np.array(ml, float) + np.array(mh, float)
        u2 = O.prim_to_cons_batch(np.array([[p, T, 0.0, 0.0, Yv, *tot, *ms, ns]]))[0]
        out[:14] = u2
        out[5:9] = u2[0] * np.array(ml, float)
        out[14:18] = u2[0] * np.array(mh, float)
        rho = u2[0]
    return out, rho


def _yv_for_S(S, T, p):
    Ra, Rv = 287.05, O.const("R_v")
    pv = S * math.exp(O.ln_psat_l(T))
    return pv * Ra / (Rv * (p - pv) + pv * Ra)


def _case(**kw):
    c, _ = cases.mixing_layer_case(seeded=False)
    c.update(kw)
    return c


def test_without_soot_the_bimodal_run_is_the_single_set_run():
    c, uf = cases.mixing_layer_case(nx=48, nr=20)
    c = dict(c, n_soot=0.0)
    o1 = O.Oracle(c, uf)
    U1 = o1.init_state()
    d1 = o1.step(U1, 20, 0.5)
    o2 = O.Oracle(dict(c, bimodal=1), uf)
    U2 = o2.init_state()
    assert U2.shape == (18, 20, 48)
    d2 = o2.step(U2, 20, 0.5)
    assert d1[-1, 7] > 100                       # phase change is running
    assert np.array_equal(U2[:14], U1)
    assert not np.any(U2[14:])
    assert np.array_equal(d1, d2)


@pytest.mark.parametrize("phase_change,viscous", [(0, 1), (1, 0)])
def test_halves_of_a_population_move_like_the_whole(phase_change, viscous):
    """Seeded droplets split into two equal sets: every step is linear in the moments
    (upwind passive fluxes, van Leer slopes, diffusion, growth at the same r20), and halving
    is exact in binary arithmetic, so the halves match the whole bit for bit."""
    c, uf = cases.mixing_layer_case(nx=48, nr=20)
    c = dict(c, Yv_core=1e-3, freezing=0, phase_change=phase_change, viscous=viscous, nu_t=0.05)
    o1 = O.Oracle(c, uf)
    U1 = o1.init_state()
    o2 = O.Oracle(dict(c, bimodal=1), uf)
    U2 = np.zeros(o2.shape)
    U2[:14] = U1
    U2[5:9] = U1[5:9] / 2
    U2[14:18] = U1[5:9] / 2
    d1 = o1.step(U1, 20, 0.5)
    o2.step(U2, 20, 0.5)
    if phase_change:
        assert d1[-1, 7] > 100 and np.all(d1[:, 23] < -300)   # growth / evaporation, no nucleation
    assert np.array_equal(U2[:5], U1[:5]) and np.array_equal(U2[9:14], U1[9:14])
    assert np.array_equal(U2[5:9], U2[14:18])
    assert np.array_equal(2 * U2[5:9], U1[5:9])


def test_closed_box_conserves_with_two_liquid_sets():
    c, uf = cases.closed_box_case()
    o = O.Oracle(dict(c, bimodal=1), uf)
    U = o.init_state()
    d = o.step(U, 100, 0.5)
    assert U[14].sum() > 1e-3 * U[5].sum() > 0       # both sets are populated
    for k in (1, 2, 3):                              # mass, water, energy
        assert abs(d[-1, k] / d[0, k] - 1.0) < 1e-12, k


@pytest.mark.parametrize("S,T", [(3.0, 220.0), (10.0, 220.0), (20.0, 240.0), (5.0, 200.0)])
def test_nucleation_splits_by_mechanism(S, T):
    p = 24e3
    Yv = _yv_for_S(S, T, p)
    U, rho = _state(p, T, Yv)
    c = _case(n_soot=1.0e12, freezing=0)
    ns_vol = 3.0e11                                   # soot per m^3: gate 0.3
    U[13] = ns_vol
    Qb, aux = O.source_batch(dict(c, bimodal=1), U, 1e-9)
    Qu, _ = O.source_batch(c, U[:14], 1e-9)
    Qb, Qu = Qb[0], Qu[0]
    # Kelvin radius and barrier, Eq. (3), with the oracle's surface tension (pinned elsewhere)
    sig, Rv, KB = O.sigma_lg(T), O.const("R_v"), 1.380649e-23
    lnS = math.log(S)
    rc = 2.0 * sig / (1000.0 * Rv * T * lnS)
    dGkT = 4.0 / 3.0 * PI * sig * rc * rc / (KB * T)
    # Eqs. (4)/(10): J_hom / J_het,eff = exp(-(1 - f) dG*/kT) / gate, f(90 deg) = 1/2
    want = -0.5 * dGkT - math.log(ns_vol / 1.0e12)
    if Qb[5] > 0.0 and Qb[14] > 0.0:
        assert math.log(Qb[5] / Qb[14]) == pytest.approx(want, rel=1e-9, abs=1e-9)
    else:   # one rate underflows: the other carries the whole source
        assert want < -700.0 and Qb[5] == 0.0 and Qb[14] > 0.0
    for k in range(1, 4):   # both sets nucleate at r_crit (in um)
        for f0 in (5, 14):
            if Qb[f0] > 0.0:
                assert Qb[f0 + k] / Qb[f0] == pytest.approx((rc * 1e6) ** k, rel=1e-9)
    # the single set takes the sum; the vapour sink and the ice do not see the split
    assert Qb[5] + Qb[14] == pytest.approx(Qu[5], rel=1e-14)
    assert Qb[4] == pytest.approx(Qu[4], rel=1e-14)
    assert aux[0, 5] == pytest.approx(rc, rel=1e-12)


def test_immersion_freezes_only_droplets_of_heterogeneous_origin():
    """Two identical populations at 250 K (Koop's homogeneous rate is zero there, Delta a_w <
    0.26): the first set does not freeze, the second freezes by immersion at the rate
    omega = k_imm n_s 4 pi <r_p^2> chi, chi = n_soot / mu0 (< 1 here), over the stage as
    N_f = mu0 (1 - exp(-omega dt)) / dt (readings H, J)."""
    T, p = 250.0, 24e3
    daw = 1.0 - math.exp(O.ln_psat_i(T) - O.ln_psat_l(T))
    assert daw < 0.26
    Yv = _yv_for_S(0.999, T, p)
    n0, r = 1.0e8, 0.5                       # per kg, um
    pop = (n0, n0 * r, n0 * r * r, n0 * r ** 3)
    U, rho = _state(p, T, Yv, ml=pop, mh=pop)
    ns_kg = 2.0e7                            # soot per kg: chi = 0.2
    U[13] = rho * ns_kg
    c = _case(n_soot=1.0e12, freezing=1, soot_rm=15e-9, soot_sigma=1.6)
    dt = 1e-4
    Q, aux = O.source_batch(dict(c, bimodal=1), U, dt)
    Q = Q[0]
    rp2 = (15e-9) ** 2 * math.exp(2.0 * math.log(1.6) ** 2)   # lognormal <r^2>
    omega = 1.0 * 1.0e8 * 4.0 * PI * rp2 * (ns_kg / n0)
    Nf = n0 * (-math.expm1(-omega * dt) / dt)
    assert Q[9] == pytest.approx(rho * Nf, rel=1e-12)          # ice number gain
    assert Q[5] == 0.0                                         # first set: no number change
    assert Q[14] == pytest.approx(-rho * Nf, rel=1e-12)        # second set loses what froze
    assert aux[0, 10] == 0.0                                   # omega of the first set


def test_one_population_has_the_same_source_in_either_set():
    """Growth (evaporation here), homogeneous and immersion freezing of one population: in the
    second set (alone) it gets the source the single-set model gives it."""
    T, p = 232.0, 24e3
    Yv = _yv_for_S(0.95, T, p)
    pop = (3.0e9, 3.0e9 * 0.3, 3.0e9 * 0.1, 3.0e9 * 0.04)
    ice = (1.0e7, 1.0e7 * 1.5, 1.0e7 * 2.5, 1.0e7 * 4.0)
    Ub, rho = _state(p, T, Yv, ms=ice, mh=pop)
    Uu = O.prim_to_cons_batch(np.array([[p, T, 0.0, 0.0, Yv, *pop, *ice, 0.0]]))[0]
    assert Uu[0] == rho
    Ub[13] = Uu[13] = rho * 1.0e9
    c = _case(n_soot=1.0e12, freezing=1)
    for dt in (1e-6, 1e-3):
        Qb = O.source_batch(dict(c, bimodal=1), Ub, dt)[0][0]
        Qu = O.source_batch(c, Uu, dt)[0][0]
        assert Qu[12] > 0.0 and Qu[8] < 0.0             # ice grows, droplets evaporate and freeze
        assert np.array_equal(Qb[14:18], Qu[5:9])
        assert np.array_equal(Qb[9:13], Qu[9:13])
        assert Qb[4] == Qu[4] and not np.any(Qb[5:9])


def test_heterogeneous_spectrum_from_moments_is_exact():
    c, uf = cases.closed_box_case(nx=4, nr=2)
    o = O.Oracle(dict(c, bimodal=1), uf)
    U = o.init_state()
    for rm, sg, rmh, sgh in ((0.015, 1.2, 0.2, 1.6), (0.05, 1.05, 1.0, 2.2)):
        s2, s2h = np.log(sg) ** 2, np.log(sgh) ** 2
        U2 = U.copy()
        for k in range(4):
            U2[5 + k] = U2[0] * 1e12 * rm ** k * np.exp(k * k * s2 / 2)
            U2[14 + k] = U2[0] * 1e9 * rmh ** k * np.exp(k * k * s2h / 2)
        got = [o.derived(U2, w)[0, 0] for w in (13, 14, 17, 18)]
        assert np.allclose(got, [rm, sg, rmh, sgh], rtol=1e-12), got
    # a single-set case has no second spectrum
    o1 = O.Oracle(c, uf)
    assert not np.any(o1.derived(o1.init_state(), 17))


def test_flux_sees_only_the_total_liquid():
    """Roe flux (Sec. 3.2): moving liquid from one set to the other changes no flow flux, and
    each set is a passive scalar upwinded with the mass flux (reading A4)."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        qL = np.zeros(18)
        qR = np.zeros(18)
        for q in (qL, qR):
            q[0], q[1], q[2], q[3], q[4] = rng.uniform(0.3, 1.2), rng.uniform(-200, 200), rng.uniform(-50, 50), \
                rng.uniform(2e4, 3e4), rng.uniform(0, 0.05)
            q[5:9] = rng.uniform(0, 1e9) * np.array([1, 0.2, 0.05, 0.01])
            q[13] = rng.uniform(0, 1e9)
        for d in (0, 1):
            F1 = O.roe_flux(qL, qR, d)
            qL2, qR2 = qL.copy(), qR.copy()
            qL2[14:18], qR2[14:18] = qL[5:9] / 2, qR[5:9] / 2
            qL2[5:9], qR2[5:9] = qL[5:9] / 2, qR[5:9] / 2
            F2 = O.roe_flux(qL2, qR2, d)
            assert np.array_equal(F1[:5], F2[:5]) and np.array_equal(F1[9:14], F2[9:14])
            qu = qL2 if F2[0] >= 0 else qR2
            assert np.array_equal(F2[14:18], F2[0] * qu[14:18])
            assert np.array_equal(F2[5:9], F2[14:18])
            F14 = O.roe_flux(qL[:14], qR[:14], d)
            assert np.array_equal(F14, F1[:14])
