"""Pins of the oracle's viscous and diffusive fluxes (Sec. 3.1 Eqs. (25)-(26), central
differences of Sec. 3.2; the turbulent viscosity is a case constant):

* the vapour diffusivity's scaling D ~ T^1.94 / p and its reference value;
* the face flux is zero for equal states and antisymmetric under exchange of the states;
* diffusion of a passive scalar (soot per kg) along x from a Gaussian: the variance grows
  as 2 D t with D = nu_t / Sc_t, Sc_t = 0.7;
* axisymmetric diffusion of an axial-velocity mode u = A J0(k r) in a closed cylinder with
  slip walls decays as exp(-nu k^2 t), k R the first zero of J1 (the Bessel eigenfunction
  of the cylindrical Laplacian);
* mass, water and energy stay constant in a closed box with phase change and diffusion;
* the viscous flag gates everything (nu_t alone changes nothing)."""
import numpy as np
import pytest

import oracle as O
from synth import cases

special = pytest.importorskip("scipy.special")


def test_vapour_diffusivity_scaling():
    assert O.dv_mol(273.15, 101325.0) == pytest.approx(2.11e-5, rel=1e-14)
    r = O.dv_mol(220.0, 24000.0) / O.dv_mol(300.0, 80000.0)
    assert r == pytest.approx((220.0 / 300.0) ** 1.94 * (80000.0 / 24000.0), rel=1e-13)


def test_face_flux_zero_for_equal_states_and_antisymmetric():
    rng = np.random.default_rng(1)
    q = np.array([0.4, 120.0, 3.0, 3.0e4, 0.01, 1e9, 2e8, 4e7, 8e6, 1e7, 1e7, 1e7, 1e7, 1e12])
    assert np.all(O.diffusive_flux(q, q, 0.01, 0.5) == 0.0)
    for _ in range(5):
        qa = q * (1.0 + 0.1 * rng.standard_normal(14))
        qb = q * (1.0 + 0.1 * rng.standard_normal(14))
        Gab = O.diffusive_flux(qa, qb, 0.01, 0.5)
        Gba = O.diffusive_flux(qb, qa, 0.01, 0.5)
        assert np.allclose(Gab, -Gba, rtol=1e-13, atol=0.0)
        assert Gab[0] == 0.0


def _box(nx, nr, lx, lr, nu_t, T=250.0, p=30000.0):
    c, _ = cases.closed_box_case(nx=nx, nr=nr)
    c.update(lx=lx, lr=lr, phase_change=0, freezing=0, viscous=1, nu_t=nu_t, seed_l_n=0.0, seed_s_n=0.0,
             T_amb=T, p_amb=p, mix_width=0.0)
    return c


def _state(o, p, T, u, v, ns):
    """Conserved (14, nr, nx) state from primitive fields of shape (nr, nx), dry air."""
    nr, nx = o.nr, o.nx
    P = np.zeros((nr * nx, 14))
    P[:, 0] = p
    P[:, 1] = T
    P[:, 2] = np.broadcast_to(u, (nr, nx)).ravel()
    P[:, 3] = np.broadcast_to(v, (nr, nx)).ravel()
    P[:, 13] = np.broadcast_to(ns, (nr, nx)).ravel()
    U = O.prim_to_cons_batch(P)
    return np.ascontiguousarray(U.T.reshape(14, nr, nx))


def test_passive_scalar_gaussian_spreads_at_2Dt():
    nx, nr, lx, nu_t = 200, 2, 2.0, 2.0
    c = _box(nx, nr, lx, 0.1, nu_t)
    o = O.Oracle(c)
    x = (np.arange(nx) + 0.5) * (lx / nx)
    s0 = 0.08
    ns = 1e12 * np.exp(-0.5 * ((x - 1.0) / s0) ** 2)
    U = _state(o, 30000.0, 250.0, 0.0, 0.0, ns[None, :])

    def variance(U):
        n = U[13, 0] / U[0, 0]
        m = np.sum(n * x) / np.sum(n)
        return np.sum(n * (x - m) ** 2) / np.sum(n)

    v0 = variance(U)
    d = o.step(U, 400, 0.5)
    t = d[:, 0].sum()
    D = nu_t / 0.7
    assert (variance(U) - v0) / (2.0 * D * t) == pytest.approx(1.0, rel=1e-2)


def test_axial_velocity_bessel_mode_decays_at_nu_k2():
    # a long box: the end walls stop the axial flow, and the pressure waves they launch stay
    # near the ends during the run, so the amplitude is measured in the middle columns
    nx, nr, L, R, nu_t, A = 40, 48, 10.0, 1.0, 1.0, 0.5
    c = _box(nx, nr, L, R, nu_t)
    o = O.Oracle(c)
    r = (np.arange(nr) + 0.5) * (R / nr)
    k = special.jn_zeros(1, 1)[0] / R          # slip wall: d/dr J0(kR) = -k J1(kR) = 0
    mode = special.j0(k * r)
    U = _state(o, 30000.0, 250.0, (A * mode)[:, None], 0.0, 0.0)
    mid = slice(nx // 2 - 8, nx // 2 + 8)

    def amplitude(U):
        u = (U[1] / U[0])[:, mid].mean(axis=1)
        return np.sum(u * mode * r) / np.sum(mode * mode * r)

    a0 = amplitude(U)
    d = o.step(U, 240, 0.5)
    t = d[:, 0].sum()
    assert 340.0 * t < 0.25 * L                # the end-wall waves have not reached the middle
    rho = U[0].mean()
    T = 250.0
    mu = 1.716e-5 * (T / 273.15) ** 1.5 * (273.15 + 110.4) / (T + 110.4)   # Sutherland
    nu = nu_t + mu / rho
    rate = -np.log(amplitude(U) / a0) / t
    assert rate / (nu * k * k) == pytest.approx(1.0, rel=1e-2)


def test_closed_box_with_diffusion_conserves_mass_water_energy():
    c, uf = cases.closed_box_case(nx=32, nr=16)
    c.update(viscous=1, nu_t=0.05)
    o = O.Oracle(c, uf)
    U = o.init_state()
    d = o.step(U, 60, 0.5)
    assert np.all(d[:, 8] == 0) and d[:, 7].max() > 0
    for k in (1, 2, 3):
        assert np.max(np.abs(d[:, k] - d[0, k])) <= 1e-12 * abs(d[0, k]), k


def test_viscous_flag_gates_the_terms():
    c, uf = cases.mixing_layer_case(nx=24, nr=12)
    U0 = O.Oracle(c, uf).init_state()
    runs = []
    for extra in ({}, {"nu_t": 0.3}, {"nu_t": 0.3, "viscous": 1}):
        o = O.Oracle(dict(c, **extra), uf)
        U = U0.copy()
        o.step(U, 5, 0.5)
        runs.append(U)
    assert np.array_equal(runs[0], runs[1])
    assert not np.array_equal(runs[0], runs[2])


def test_radial_velocity_linear_in_r_has_no_viscous_force():
    """v = a r is annihilated by the radial component of the vector Laplacian
    (d/dr (1/r d(r v)/dr) = 0): the r-weighted face fluxes and the -mu v / r^2 volume term
    cancel, cell by cell, away from the outer wall."""
    nx, nr, R, nu_t = 4, 24, 1.0, 0.5
    c = _box(nx, nr, 0.5, R, nu_t)
    o_v = O.Oracle(c)
    o_i = O.Oracle(dict(c, viscous=0))
    r = (np.arange(nr) + 0.5) * (R / nr)
    U = _state(o_v, 30000.0, 250.0, 0.0, (2.0 * r)[:, None], 0.0)
    Lv, _ = o_v.residual(U, 1e-6)
    Li, _ = o_i.residual(U, 1e-6)
    visc = (Lv - Li)[2]                          # viscous part of the rho v residual
    ref = 0.5 * 0.4 * 2.0 / r[:, None]           # size of either of the two cancelling terms
    assert np.max(np.abs(visc[:-2]) / ref[:-2]) < 1e-9
    assert np.max(np.abs(visc[-1])) > 1e-3 * ref[-1, 0]   # the slip wall breaks it, as it should
