"""bench.py without a GPU: the reference arm (the oracle on the host cores) prints one JSON
line with the keys the measurement contract asks for, and the per-cell tables the roofline
takes its traffic from name tile shapes that have kernels of that precision."""
import importlib.util
import json
import os
import subprocess
import sys

from conftest import ROOT


def _bench_module():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    d = json.loads(lines[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] >= 3
    assert d["higher_is_better"] is True and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["workload"] and d["config"]["cells"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_traffic_tables_name_shapes_with_kernels():
    from paper_2504_20742_gb300 import build
    build.build()
    import paper_2504_20742_gb300 as P
    b = _bench_module()
    n = P.ct_tile_shape_count()
    for table, prec in ((b.FP64_TRAFFIC_PER_CELL_LAUNCH, P.CT_FP64), (b.FP32_TRAFFIC_PER_CELL_LAUNCH, P.CT_FP32)):
        assert table
        for shape, per_cell in table.items():
            assert 0 <= shape < n
            assert P.ct_tile_shape_ctas(shape, prec) > 0, (shape, prec)
            assert per_cell > 0
    assert b.FP64_FLOPS_PER_CELL_STAGE > 0 and b.FP64_VISC_FLOPS_PER_CELL_STAGE > b.FP64_FLOPS_PER_CELL_STAGE
