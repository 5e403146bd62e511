"""The mixed-precision plume at full size: 4096 x 1024 cells, FP32 transport with FP64
islands against the FP64 path after 2000 steps, field by field.  The FP64 path is held to
the oracle at 1e-9 elsewhere (the oracle itself would take about 20 minutes of host time
for this run), so it stands in for the oracle here."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_helpers import FIELD_NAMES, field_rel_err, report
from synth import cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2504_20742_gb300 as P
    return P


def test_fp32_plume_4096x1024_against_fp64_after_2000_steps(P):
    c, uf = cases.plume_case_mixed_precision()
    out = {}
    for prec in (P.CT_FP64, P.CT_FP32):
        s = P.Solver(c, uf, precision=prec)
        s.init_state(0.5)
        s.autotune(reps=1)
        for _ in range(4):
            s.step(500, 0.5)
        d = s.diagnostics()
        assert d[8] == 0 and d[27] == 2000
        out[prec] = (s.state64(), d)
        del s
        torch.cuda.empty_cache()
    U64, d64 = out[P.CT_FP64]
    U32, d32 = out[P.CT_FP32]
    err = field_rel_err(U32, U64)
    print("FP32 vs FP64, 4096x1024 plume, 2000 steps:", report(err))
    print("totals (mass, water, energy) rel diff:",
          [abs(d32[k] - d64[k]) / abs(d64[k]) for k in (1, 2, 3)], "dt rel diff", abs(d32[0] - d64[0]) / d64[0])
    assert np.all(err < 1e-3), report(err)
    for k in (1, 2, 3):
        assert abs(d32[k] - d64[k]) <= 1e-5 * abs(d64[k])
