"""Pins of the tabulated water properties (Sec. 3.2: tables built before the run, second-
order Taylor interpolation at run time), against the closed forms they are built from:

* at the nodes the expansion returns the closed form (and its derivative) exactly;
* between nodes the error stays below the Taylor remainder |f'''| h^3 / 6 (h = 0.25 K,
  the largest distance to the nearest node), and reaches a fair fraction of it, which
  a first-order (missing curvature) expansion would exceed by orders of magnitude;
* T_sat from the tabulated curve agrees with the closed-form Newton;
* a solver run with tables differs from the closed-form run only at the table's error."""
import numpy as np
import pytest

import oracle as O
from synth import cases

CLOSED = (O.ln_psat_l, O.ln_psat_i, O.sigma_lg)
T_NODES = 150.0 + 0.5 * np.arange(981)


def _third_derivative(f, T, h=1e-2):
    return (f(T + 2 * h) - 2 * f(T + h) + 2 * f(T - h) - f(T - 2 * h)) / (2 * h ** 3)


@pytest.mark.parametrize("which", [0, 1, 2])
def test_nodes_reproduce_the_closed_form(which):
    f = CLOSED[which]
    for T in T_NODES[::37]:
        assert O.table_eval(which, T) == pytest.approx(f(T), rel=1e-15, abs=1e-15)
        d = (f(T + 1e-4) - f(T - 1e-4)) / 2e-4
        assert O.table_eval(which, T, 1) == pytest.approx(d, rel=1e-6)


@pytest.mark.parametrize("which", [0, 1, 2])
def test_error_is_third_order_taylor_remainder(which):
    f = CLOSED[which]
    T = np.arange(150.0, 640.0, 0.0173)
    err = np.array([abs(O.table_eval(which, t) - f(t)) for t in T])
    f3 = np.array([abs(_third_derivative(f, t)) for t in T])
    bound = f3 * 0.25 ** 3 / 6.0
    assert np.all(err <= 1.05 * bound + 1e-15)
    assert err.max() >= 0.05 * bound.max()       # really the cubic remainder, not smaller
    print("max table error", err.max(), "max remainder bound", bound.max())


def test_tsat_from_tables():
    for pv in (0.5, 3.0, 40.0, 600.0, 3000.0):
        for which in (0, 1):
            # the tabulated curve crosses ln pv within its own error of the closed form's
            Tc = O.tsat(pv, which)
            f = CLOSED[which]
            dT = abs(O.table_eval(which, Tc) - f(Tc)) / abs(O.table_eval(which, Tc, 1))
            assert dT < 1e-6


def test_solver_with_tables_matches_closed_forms_to_table_error():
    c, uf = cases.freezing_case(nx=48, nr=20)
    runs = []
    for tab in (0, 1):
        o = O.Oracle(dict(c, tables=tab), uf)
        U = o.init_state()
        d = o.step(U, 30, 0.5)
        assert np.all(d[:, 8] == 0)
        runs.append((U, d))
    (U0, d0), (U1, d1) = runs
    assert not np.array_equal(U0, U1)
    rel = np.abs(U1 - U0).max(axis=(1, 2)) / np.maximum(np.abs(U0).max(axis=(1, 2)), 1e-300)
    assert np.all(rel < 1e-5), rel
    assert np.array_equal(d0[:, 7], d1[:, 7])
