"""Host-side tests of the CUDA library (no GPU needed): it loads, exports every entry point
declared in include/contrail.h, and rejects invalid arguments before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def P():
    from paper_2504_20742_gb300 import build
    build.build()
    import paper_2504_20742_gb300 as P
    return P


def test_exports_every_declared_symbol(P):
    hdr = open(os.path.join(ROOT, "include", "contrail.h")).read()
    names = set(re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*(ct_[a-z_0-9]+)\s*\(", hdr, re.M))
    assert {"ct_setup", "ct_step", "ct_init_state", "ct_diagnostics"} <= names
    lib = ctypes.CDLL(P.lib_path())
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert P.ct_version().startswith("contrail-gb300")


def test_binding_covers_every_declared_symbol(P):
    """The Python binding has a function of the same name, with a ctypes signature, for
    every entry point the header declares."""
    from paper_2504_20742_gb300 import _lib
    hdr = open(os.path.join(ROOT, "include", "contrail.h")).read()
    names = set(re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*(ct_[a-z_0-9]+)\s*\(", hdr, re.M))
    assert sorted(names - set(_lib._SIGS)) == []
    assert sorted(n for n in names if not callable(getattr(_lib, n, None))) == []


def test_workspace_size_and_case_validation(P):
    from synth import cases
    c, _ = cases.plume_case()
    assert P.ct_workspace_bytes(c, P.CT_FP64) > 256 * 14 * 8
    bad = dict(c, nx=1)
    assert P.ct_workspace_bytes(bad, P.CT_FP64) == 0
    assert "nx" in P.ct_last_error()
    assert P.ct_workspace_bytes(c, 7) == 0
    # FP32 + surrogate on a case the column sweep steps: the surrogate queue (a cell index
    # and 14 rates per cell, 4096 reduction records) on top of the FP32 workspace
    n = c["nx"] * c["nr"]
    extra = P.ct_workspace_bytes(c, P.CT_FP32_MLP) - P.ct_workspace_bytes(c, P.CT_FP32)
    assert 60 * n + 4096 * 27 * 8 <= extra <= 60 * n + 4096 * 27 * 8 + 3 * 256
    visc = dict(c, viscous=1, nu_t=0.1)          # the sweep does not step it: no queue
    assert P.ct_workspace_bytes(visc, P.CT_FP32_MLP) == P.ct_workspace_bytes(visc, P.CT_FP32)


def test_invalid_arguments_are_rejected_without_a_gpu(P):
    from synth import cases
    c, _ = cases.plume_case(nx=64, nr=16)
    with pytest.raises(P.ContrailError) as e:
        P.ct_step(c, P.CT_FP64, 0x1000, 0x1000, 0x2000, 1, 0.5)
    assert e.value.status == 1
    with pytest.raises(P.ContrailError):
        P.ct_step(c, P.CT_FP64, 0x1000, 0x3000, 0x2000, -1, 0.5)
    with pytest.raises(P.ContrailError):
        P.ct_step(c, P.CT_FP64, 0x1000, 0x3000, 0x2000, 1, 1.5)
    with pytest.raises(P.ContrailError) as e:
        P.ct_setup(c, P.CT_FP64, None, 0x1000, 16, None)
    assert e.value.status == 6
    with pytest.raises(P.ContrailError):
        P.ct_setup(c, P.CT_FP64, None, 0x1001, 1 << 30, None)
    with pytest.raises(P.ContrailError):
        P.ct_derived(c, P.CT_FP64, 0x1000, 99, 1e-6, 0x2000)
    P.ct_reconstruct_faces(None, None, None, 0, None, None)   # n = 0: nothing to do
    with pytest.raises(P.ContrailError) as e:
        P.ct_reconstruct_faces(0x1000, 0x1000, 0x1000, -1, 0x2000, 0x3000)
    assert e.value.status == 1
    with pytest.raises(P.ContrailError):
        P.ct_reconstruct_faces(0x1000, None, 0x1000, 4, 0x2000, 0x3000)
    for field in (-1, 14):                     # read_field: field index checked first
        with pytest.raises(P.ContrailError) as e:
            P.ct_read_field(c, P.CT_FP64, 0x1000, field)
        assert e.value.status == 1
    assert P.ct_train_workspace_bytes(0, 64, 1) == 0 and P.ct_train_workspace_bytes(100, 64, 0) == 0
    assert P.ct_train_workspace_bytes(1000, 256, 4) >= 1000 * 26 * 4
    with pytest.raises(P.ContrailError) as e:          # invalid configuration, before any copy
        P.ct_train_surrogate(0x1000, 0x2000, 0x3000, 100, dict(epochs=0, batch=10, lr=1e-3, lr_final=0.0),
                             0x4000, 0x5000, 0x6000, 1 << 20)
    assert e.value.status == 1


def test_binding_has_no_oracle_dependency():
    src = open(os.path.join(ROOT, "paper_2504_20742_gb300", "_lib.py")).read()
    src += open(os.path.join(ROOT, "paper_2504_20742_gb300", "solver.py")).read()
    assert "oracle" not in src and "synth" not in src


def test_tile_shapes_and_registry_without_a_gpu(P):
    from synth import cases
    n = P.ct_tile_shape_count()
    shapes = [P.ct_tile_shape(s) for s in range(n)]
    ctas = [P.ct_tile_shape_ctas(s, P.CT_FP32) for s in range(n)]
    ctas64 = [P.ct_tile_shape_ctas(s, P.CT_FP64) for s in range(n)]
    assert shapes[0] == (32, 8) and len(set(zip(shapes, ctas, ctas64))) == n
    assert set(ctas) == {0, 1, 2, 3, 4} and set(ctas64) == {0, 1, 2} and P.ct_tile_shape_ctas(n, P.CT_FP32) == 0
    assert P.ct_tile_shape_ctas(0, 7) == 0
    c, _ = cases.plume_case(nx=64, nr=16)
    # a shape takes a precision exactly when it has kernels for it
    for k in range(n):
        for prec, have in ((P.CT_FP64, ctas64[k]), (P.CT_FP32, ctas[k])):
            if have:
                P.ct_set_tile_shape(c, prec, k)
                P.ct_set_tile_shape(c, prec, -1)
            else:
                with pytest.raises(P.ContrailError) as e:
                    P.ct_set_tile_shape(c, prec, k)
                assert e.value.status == 1
    with pytest.raises(P.ContrailError):
        P.ct_set_tile_shape(c, P.CT_FP32, n)
    # the FP64 two-CTA shape carries the plain FP64 kernels only
    k2 = ctas64.index(2)
    P.ct_set_tile_shape(c, P.CT_FP64, k2)
    P.ct_set_tile_shape(c, P.CT_FP64, -1)
    with pytest.raises(P.ContrailError):
        P.ct_set_tile_shape(c, P.CT_FP32, k2)
    # the three-CTA shapes carry the plain FP32 kernels only
    k3 = ctas.index(3)
    P.ct_set_tile_shape(c, P.CT_FP32, k3)
    P.ct_set_tile_shape(c, P.CT_FP32, -1)
    for prec in (P.CT_FP64, P.CT_FP32_MLP):
        with pytest.raises(P.ContrailError):
            P.ct_set_tile_shape(c, prec, k3)
    # the column-sweep shape (28-cell strips): plain FP32 axisymmetric cases without the
    # diffusive fluxes only
    ks = shapes.index((28, 64))
    assert ctas[ks] == 4 and ctas64[ks] == 0
    P.ct_set_tile_shape(c, P.CT_FP32, ks)
    P.ct_set_tile_shape(c, P.CT_FP32, -1)
    for bad in (dict(c, viscous=1, nu_t=0.1), cases.nozzle_case(nx=64), dict(c, bimodal=1)):
        with pytest.raises(P.ContrailError):
            P.ct_set_tile_shape(bad, P.CT_FP32, ks)
    # the workspace holds the partials of the shape with the most tiles
    ragged, _ = cases.plume_case(nx=40, nr=24)
    tiles = max(-(-40 // tx) * -(-24 // ty) for tx, ty in shapes)
    assert P.ct_workspace_bytes(ragged, P.CT_FP32) >= tiles * 26 * 8


def test_batch_sizes_and_validation_without_a_gpu(P):
    from synth import cases
    bc = [c for c, _ in cases.batch_cases(n=8)]
    elems = sum(14 * c["nx"] * c["nr"] for c in bc)
    assert P.ct_batch_state_elems(bc) == elems
    ws = P.ct_batch_workspace_bytes(bc)
    assert ws >= sum(P.ct_workspace_bytes(c, P.CT_FP32) for c in bc)
    # every case the batched column sweep can step holds its surrogate queue
    assert ws >= sum(P.ct_workspace_bytes(c, P.CT_FP32_MLP) for c in bc)
    noz = cases.nozzle_case()
    assert P.ct_batch_workspace_bytes(bc + [noz]) == 0
    assert "geom" in P.ct_last_error()
    assert P.ct_batch_workspace_bytes([]) == 0
    with pytest.raises(P.ContrailError) as e:
        P.ct_batch_create(bc, P.CT_FP64, None, 0x100, ws, None)
    assert e.value.status == 1
    with pytest.raises(P.ContrailError) as e:
        P.ct_batch_create(bc, P.CT_FP32, None, 0x100, ws - 1, None)
    assert e.value.status == 6
    with pytest.raises(P.ContrailError):
        P.ct_batch_create(bc, P.CT_FP32, None, 0x101, ws, None)


def test_static_scratch_covers_the_grids_its_header_names(P):
    """The allocation-free step's static scratch (CT_STATIC_SCRATCH_BYTES, read from the
    header) holds the workspace of every plume grid up to 4096 x 1024 cells (the FP32 size:
    the static path keeps no stored primitives in either precision), and not that of an
    8192 x 2048 plume (rejected with CT_ERR_SIZE)."""
    from synth import cases
    hdr = open(os.path.join(ROOT, "include", "contrail.h")).read()
    m = re.search(r"#define\s+CT_STATIC_SCRATCH_BYTES\s+\((\d+)u\s*<<\s*(\d+)\)", hdr)
    limit = int(m.group(1)) << int(m.group(2))
    for nx, nr in ((4096, 1024), (4096, 1000), (1024, 256), (2048, 512), (37, 5)):
        c, _ = cases.plume_case(nx=nx, nr=nr)
        need = P.ct_workspace_bytes(c, P.CT_FP32)
        assert 0 < need <= limit, (nx, nr, need, limit)
    big, _ = cases.plume_case(nx=8192, nr=2048)
    assert P.ct_workspace_bytes(big, P.CT_FP32) > limit
    with pytest.raises(P.ContrailError) as e:
        P.ct_step_static(big, P.CT_FP64, None, 0x1000, 0x2000, 1, 0.5)
    assert e.value.status == 6 and "static scratch" in str(e.value)
