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


def test_surrogate_rates_on_visited_states(P, sur):
    """log10 J_hom of the BF16 tensor-core network against the FP64 plain source on states
    visited by FP64 runs of the nozzle and a hydrogen-like mixing layer, where J >= 1."""
    from paper_2504_20742_gb300 import surrogate as S
    rows = []
    for c, uf, n in ((cases.nozzle_case(nx=400), None, 600), (cases.mixing_layer_case(nx=96, nr=40)[0],
                                                               cases.mixing_layer_case(nx=96, nr=40)[1], 60)):
        U = S.sample_active_states(c, uf, nsteps=n, every=3)
        X, Y, M = S.dataset(c, U)
        rows.append((X, Y, M))
    X = torch.cat([r[0] for r in rows])
    Y = torch.cat([r[1] for r in rows])
    M = torch.cat([r[2] for r in rows])
    blob = sur.blob()
    Yp = torch.empty_like(Y)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    P.ct_mlp_infer(blob, X.contiguous(), X.shape[0], Yp, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    m = (M[:, 6] > 0) & (Y[:, 6] >= 0)
    assert int(m.sum()) > 1000
    e10 = ((Yp[m, 6] - Y[m, 6]).abs() / np.log(10.0)).cpu().numpy()
    print(f"log10 J_hom error where J >= 1: mean {e10.mean():.3f}, p90 {np.quantile(e10, 0.9):.3f}, "
          f"p99 {np.quantile(e10, 0.99):.3f}, n {e10.size}")
    assert e10.mean() <= 0.1
    assert np.quantile(e10, 0.9) <= 0.25


def test_surrogate_trajectory_vs_oracle_on_nozzle(P, sur):
    """The 400-cell condensing nozzle, 300 steps: the FP32 + surrogate state against
    the FP64 oracle, and the plain FP32 state against it, field by field."""
    c = cases.nozzle_case(nx=400)
    o = O.Oracle(c)
    Uo = o.init_state()
    o.step(Uo, 300, 0.5)
    res = {}
    for name, prec in (("fp32", P.CT_FP32), ("fp32_mlp", P.CT_FP32_MLP)):
        s = _solver(P, sur, c, None, prec)
        s.step(300, 0.5)
        assert s.diagnostics()[8] == 0
        U = s.state64()
        rho_err = np.max(np.abs(U[0] - Uo[0]) / Uo[0])
        n_tot = (U[5] * 1).sum()
        n_ref = Uo[5].sum()
        y_ref = Uo[8].sum()
        res[name] = (rho_err, abs(n_tot / n_ref - 1.0), abs(U[8].sum() / y_ref - 1.0))
    print("nozzle 300 steps, errors vs FP64 oracle (rho max rel, liquid number total, liquid mass total):", res)
    assert res["fp32"][0] < 1e-3 and res["fp32"][2] < 1e-2
    assert res["fp32_mlp"][0] < 5e-2


def test_surrogate_gain_on_an_active_workload(P, sur):
    """What the network buys: step time of the FP32 path and of the FP32 + surrogate path on
    a hydrogen-like mixing plume whose source fires in many cells, same state and steps."""
    c, uf = cases.mixing_layer_case(nx=1024, nr=256)
    times = {}
    for name, prec in (("fp32", P.CT_FP32), ("fp32_mlp", P.CT_FP32_MLP)):
        s = _solver(P, sur, c, uf, prec)
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
    print("ms/step, active fraction, fallbacks:", times,
          "speedup of the surrogate path:", times["fp32"][0] / times["fp32_mlp"][0])
    assert times["fp32_mlp"][1] > 0.02
