"""The FP32 + surrogate step (BF16 tensor cores inside the fused stage): it runs, conserves
water exactly as the plain FP32 path does, reports its fallbacks, and its rates and
trajectories are compared with the FP64 plain source and the FP64 oracle."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from synth import cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2504_20742_gb300 as P
    return P


@pytest.fixture(scope="module")
def sur(P):
    from paper_2504_20742_gb300 import surrogate as S
    return S.Surrogate.load(S.default_path())


def _solver(P, sur, c, uf, prec):
    s = P.Solver(c, uf, precision=prec)
    s.init_state(0.5)
    if prec == P.CT_FP32_MLP:
        s.attach_surrogate(sur.blob())
    return s


def test_surrogate_step_conserves_and_reports_fallbacks(P, sur):
    c, uf = cases.closed_box_case()
    s = _solver(P, sur, c, uf, P.CT_FP32_MLP)
    s.step(1, 0.5)
    d0 = s.diagnostics()
    s.step(60, 0.5)
    d = s.diagnostics()
    assert d[8] == 0 and d[7] > 0
    for k in (1, 2, 3):
        assert abs(d[k] - d0[k]) <= 2e-6 * abs(d0[k]), k     # FP32 state, FP64 sums
    assert 0 <= d[26] <= d[7]


def _visited(P):
    from paper_2504_20742_gb300 import surrogate as S
    rows = []
    for c, uf, n in ((cases.nozzle_case(nx=400), None, 600), (cases.mixing_layer_case(nx=96, nr=40)[0],
                                                               cases.mixing_layer_case(nx=96, nr=40)[1], 60)):
        U = S.sample_active_states(c, uf, nsteps=n, every=3)
        rows.append(S.dataset(c, U))
    return (torch.cat([r[q] for r in rows]) for q in range(3))


def test_surrogate_rates_on_visited_states(P, sur):
    """The rates the FP32 + surrogate step takes on states visited by FP64 runs of the nozzle
    and a hydrogen-like mixing layer.  Nucleation is the plain path's closed form (Eqs. 3-5,
    10: the rates, the Kelvin radius and the Kantrowitz factor), so log10 J is exact; the
    network supplies the growth rates asinh(G / 1 um/s) and the logs of the stage relaxation
    rates.  The shipped network's errors on these states: 0.05-0.11 on average (5-11 %), up to
    0.21 for 90 % of them; the test holds them there (mean 0.15, p90 0.3) and prints them."""
    X, Y, M = _visited(P)
    blob = sur.blob()
    Yp = torch.empty_like(Y)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    P.ct_mlp_infer(blob, X.contiguous(), X.shape[0], Yp, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    for q, name in ((2, "asinh G_l"), (3, "asinh G_s"), (4, "ln 1/tau_l"), (5, "ln 1/tau_s")):
        mm = M[:, q] > 0
        assert int(mm.sum()) > 1000
        d = (Yp[mm, q] - Y[mm, q]).abs().cpu().numpy()
        print(f"{name}: mean |error| {d.mean():.3f}, p90 {np.quantile(d, 0.9):.3f}, max {d.max():.2f}, n {d.size}")
        assert d.mean() <= 0.15 and np.quantile(d, 0.9) <= 0.3, name


def _number_errors(U, Uo, f):
    ref, got = Uo[f].ravel(), U[f].ravel()
    m = ref > 1e-6 * ref.max()
    return abs(got.sum() / ref.sum() - 1.0), np.abs(got[m] - ref[m]).sum() / np.abs(ref[m]).sum()


def test_surrogate_number_density_on_the_nozzle_at_steady_state(P, sur):
    """The condensing nozzle's configured run (400 cells, 20,000 steps to steady state): the
    FP32 + surrogate liquid number density against the FP64 oracle, in total and cell by
    cell (relative L1 over cells above 1e-6 of the maximum), within 2 %; the plain FP32 path
    within 1e-3."""
    c = cases.nozzle_case(nx=400)
    o = O.Oracle(c)
    Uo = o.init_state()
    o.step(Uo, 20000, 0.5)
    res = {}
    for name, prec in (("fp32", P.CT_FP32), ("fp32_mlp", P.CT_FP32_MLP)):
        s = _solver(P, sur, c, None, prec)
        s.step(20000, 0.5)
        d = s.diagnostics()
        assert d[8] == 0
        res[name] = _number_errors(s.state64(), Uo, 5) + (d[26] / max(d[7], 1.0),)
    print("nozzle, 20000 steps, liquid number vs the FP64 oracle (total, cell-wise L1, fallback share):", res)
    assert res["fp32"][0] <= 1e-3 and res["fp32"][1] <= 1e-3
    assert res["fp32_mlp"][0] <= 2e-2 and res["fp32_mlp"][1] <= 2e-2


def test_surrogate_number_density_on_the_freezing_plume(P, sur):
    """The freezing plume (evaporating droplets, homogeneous and immersion freezing, ice
    growth), 100 steps: liquid and ice number density within 2 % of the FP64 oracle, in
    total and cell by cell."""
    c, uf = cases.freezing_case()
    o = O.Oracle(c, uf)
    Uo = o.init_state()
    o.step(Uo, 100, 0.5)
    s = _solver(P, sur, c, uf, P.CT_FP32_MLP)
    s.step(100, 0.5)
    d = s.diagnostics()
    assert d[8] == 0 and d[7] > 100
    U = s.state64()
    for f, name in ((5, "liquid"), (9, "ice")):
        tot, l1 = _number_errors(U, Uo, f)
        print(f"freezing plume, 100 steps, {name} number vs the FP64 oracle: total {tot:.2e}, cell-wise L1 {l1:.2e}")
        assert tot <= 2e-2 and l1 <= 2e-2, (name, tot, l1)


def test_surrogate_gain_on_an_active_workload(P, sur):
    """What the network buys: step time of the FP32 path and of the FP32 + surrogate path on
    a hydrogen-like mixing plume whose source fires in about half of the cells, same state
    and steps.  On GB300 the plain FP32 source (FP32 with FP64 islands) is cheaper than the
    network's evaluation: the surrogate step takes about 1.5 times as long.  The test holds
    the measured ratio to that finding (below 1.8) and prints it."""
    c, uf = cases.mixing_layer_case(nx=1024, nr=256)
    times = {}
    for name, prec in (("fp32", P.CT_FP32), ("fp32_mlp", P.CT_FP32_MLP)):
        s = _solver(P, sur, c, uf, prec)
        s.autotune(reps=2)
        s.step(3, 0.5)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.step(20, 0.5)
        e1.record(s.stream)
        e1.synchronize()
        d = s.diagnostics()
        assert d[8] == 0
        times[name] = (e0.elapsed_time(e1) / 20, d[7] / (1024 * 256), d[26])
    ratio = times["fp32_mlp"][0] / times["fp32"][0]
    print("ms/step, active fraction, fallbacks:", times, "surrogate / plain FP32 step time:", ratio)
    assert times["fp32_mlp"][1] > 0.3
    assert ratio < 1.8
