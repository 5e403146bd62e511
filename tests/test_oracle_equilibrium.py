"""Pins of the oracle's equilibrium phase-change model (the comparison model of Sec. 4.3:
phase change is instantaneous once saturation is reached):

* water and energy of every cell are conserved by the source, to rounding;
* where condensate remains, the vapour is exactly saturated over it (S = 1) at the new
  temperature, which the formation energies raise by the latent heat of the condensate;
* subsaturated water is all vapour; a dry cell is untouched;
* applying the model to its own result changes nothing (a fixed point);
* more total water at the same energy gives more condensate;
* a closed box stays conserved to 1e-12."""
import numpy as np
import pytest

import oracle as O
from synth import cases

YL3 = 4.0 / 3.0 * np.pi * 1000.0 * 1e-18
YS3 = 4.0 / 3.0 * np.pi * 917.0 * 1e-18


def _case(**kw):
    c, _ = cases.mixing_layer_case()
    return dict(c, equilibrium=1, **kw)


def _state(p, T, Yv, ml3=0.0, ms3=0.0, u=50.0):
    ml = [ml3] * 4
    ms = [ms3] * 4
    row = [p, T, u, 0.0, Yv] + ml + ms + [1e12]
    return O.prim_to_cons_batch(np.array([row]))


def _apply(c, U, dt=1e-6):
    Q, aux = O.source_batch(c, U, dt)
    return U + dt * Q, aux


def _water(U):
    return U[:, 4] + YL3 * U[:, 8] + YS3 * U[:, 12]


@pytest.mark.parametrize("T,Yv", [(250.0, 0.01), (240.0, 0.004), (230.0, 0.002), (300.0, 0.1)])
def test_supersaturated_cells_end_saturated_conserving_water_and_energy(T, Yv):
    c = _case()
    U = _state(30000.0, T, Yv)
    Ue, aux = _apply(c, U)
    assert aux[0, 4] == 1.0
    assert _water(Ue)[0] == pytest.approx(_water(U)[0], rel=1e-14)
    assert Ue[0, 3] == U[0, 3] and Ue[0, 0] == U[0, 0]
    P = O.cons_to_prim_batch(Ue)[0]      # rho, u, v, p, T, Yv, Yl, Ys, c2
    Teq = P[4]
    assert Teq > T                        # latent heat released
    ice = P[7] > 0.0
    assert (P[6] > 0.0) != ice            # one condensed phase
    assert ice == (Teq < 235.15)
    _, aux2 = _apply(c, Ue)                 # ln S_l, ln S_i of the new state
    assert abs(aux2[0, 1 if ice else 0]) < 1e-10


def test_subsaturated_condensate_evaporates_and_dry_cell_is_untouched():
    c = _case()
    U = _state(30000.0, 280.0, 0.001, ml3=1e6)        # warm, little water: all evaporates
    Ue, aux = _apply(c, U)
    P = O.cons_to_prim_batch(Ue)[0]
    assert P[6] == 0.0 and P[7] == 0.0
    assert _water(Ue)[0] == pytest.approx(_water(U)[0], rel=1e-14)
    Ud = _state(30000.0, 220.0, 0.0)
    Q, aux = O.source_batch(c, Ud, 1e-6)
    assert np.all(Q == 0.0) and aux[0, 4] == 0.0


def test_equilibrium_is_a_fixed_point():
    c = _case()
    U = _state(30000.0, 250.0, 0.01)
    U1, _ = _apply(c, U)
    U2, _ = _apply(c, U1)
    assert np.allclose(U2, U1, rtol=1e-10, atol=0.0)


def test_more_water_more_condensate():
    c = _case()
    yc = []
    for Yv in (0.004, 0.006, 0.008, 0.012):
        Ue, _ = _apply(c, _state(30000.0, 250.0, Yv))
        P = O.cons_to_prim_batch(Ue)[0]
        yc.append(P[6] + P[7])
    assert np.all(np.diff(yc) > 0.0)


def test_closed_box_with_equilibrium_conserves():
    c, uf = cases.closed_box_case(nx=32, nr=16)
    c = dict(c, equilibrium=1)
    o = O.Oracle(c, uf)
    U = o.init_state()
    d = o.step(U, 40, 0.5)
    assert np.all(d[:, 8] == 0) and d[:, 7].max() > 0
    for k in (1, 2, 3):
        assert np.max(np.abs(d[:, k] - d[0, k])) <= 1e-12 * abs(d[0, k]), k
