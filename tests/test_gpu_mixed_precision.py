"""The mixed-precision plume at full size: 4096 x 1024 cells, FP32 transport with FP64
islands.  Against the FP64 oracle itself after 100 steps (a minute of the oracle on 16
host cores), field by field; and against the GPU FP64 path after the configuration's 2000
steps (the oracle would take about 20 minutes of host time for those; the FP64 path is
held to the oracle at 1e-9 elsewhere).  The kerosene plume has no supersaturated cell in
these runs (ln S_l stays below -0.4), so the FP32 screen leaves its FP64 islands idle;
the FP32 tests of the nozzle and the freezing plume exercise them.

What to expect: the bulk fields agree to the FP32 rounding accumulated over the run.  The
axisymmetric pressure source and the r-face pressure fluxes cancel only to FP32 rounding in
the parallel jet, so rho v carries rounding-level noise, which moves a little core water
and soot across the initially sharp core/bypass contact where the FP64 run keeps exactly
nothing: a leak of about 1e-4 of the core value, large against the zero FP64 value there."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_helpers import FIELD_NAMES, FLOOR_FP32, field_rel_err, report
from synth import cases

pytestmark = pytest.mark.gpu

STEPS = 2000


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2504_20742_gb300 as P
    return P


def _run(P, c, uf, prec, steps=STEPS):
    s = P.Solver(c, uf, precision=prec)
    s.init_state(0.5)
    s.autotune(reps=1)
    for _ in range(steps // 500):
        s.step(500, 0.5)
    s.step(steps % 500, 0.5)
    d = s.diagnostics()
    assert d[8] == 0 and d[27] == steps
    U = s.state64()
    del s
    torch.cuda.empty_cache()
    return U, d


def test_fp32_plume_4096x1024_against_fp64_after_2000_steps(P):
    c, uf = cases.plume_case_mixed_precision()
    U64, d64 = _run(P, c, uf, P.CT_FP64)
    U32, d32 = _run(P, c, uf, P.CT_FP32)
    err = field_rel_err(U32, U64, FLOOR_FP32)
    a = U32.reshape(14, -1) - U64.reshape(14, -1)
    scale = np.maximum(np.abs(U64.reshape(14, -1)).max(1), 1e-300)
    scale[2] = max(scale[1], scale[2])              # rho v on the momentum scale
    err_max = np.abs(a).max(1) / scale
    print(f"FP32 vs FP64, 4096x1024 plume, {STEPS} steps, per cell (floor 1e-3 max):", report(err))
    print(f"  max |error| / max |field|:", report(err_max))
    tot = [abs(d32[k] - d64[k]) / abs(d64[k]) for k in (1, 2, 3)]
    print("  totals (mass, water, energy) rel diff:", tot, "dt rel diff", abs(d32[0] - d64[0]) / d64[0])
    for f in (0, 1, 3):                               # bulk fields, cell by cell
        assert err[f] < 1e-3, (FIELD_NAMES[f], err[f])
    assert np.all(err_max < 1e-3), report(err_max)    # every field against its own scale
    for t in tot:
        assert t <= 1e-5


def test_fp32_plume_4096x1024_against_the_oracle_after_100_steps(P):
    import oracle as O
    c, uf = cases.plume_case_mixed_precision()
    U32, d32 = _run(P, c, uf, P.CT_FP32, steps=100)
    o = O.Oracle(c, uf)
    Uo = o.init_state()
    do = o.step(Uo, 100, 0.5)
    err = field_rel_err(U32, Uo, FLOOR_FP32)
    a = U32.reshape(14, -1) - Uo.reshape(14, -1)
    scale = np.maximum(np.abs(Uo.reshape(14, -1)).max(1), 1e-300)
    scale[2] = max(scale[1], scale[2])
    err_max = np.abs(a).max(1) / scale
    print("FP32 vs oracle, 4096x1024 plume, 100 steps, per cell (floor 1e-3 max):", report(err))
    print("  max |error| / max |field|:", report(err_max))
    for f in (0, 1, 3):
        assert err[f] < 1e-4, (FIELD_NAMES[f], err[f])
    assert np.all(err_max < 1e-4), report(err_max)
    for k in (1, 2, 3):
        assert abs(d32[k] - do[-1, k]) <= 1e-6 * abs(do[-1, k]), k
    assert d32[0] == pytest.approx(do[-1, 0], rel=1e-5)
