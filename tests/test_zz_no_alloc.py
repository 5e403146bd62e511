"""The allocation-free entry point ct_step_static, for callers that cannot allocate device
memory (their allocator belongs to a host framework, or they may only use the buffers they
were handed).  It keeps the step's scratch in the library's static device array; its
results must match ct_step with a caller workspace, on two calls in a row that share that
array.  Collected last on purpose (file name), so that a run stopping at the first failure
has run every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2504_20742_gb300 import build
    build.build()
    import paper_2504_20742_gb300 as P
    return P


def _field_rel_err(a, b):
    a = a.reshape(14, -1)
    b = b.reshape(14, -1)
    out = []
    for f in range(14):
        m = np.max(np.abs(b[f])) if f != 2 else max(np.max(np.abs(b[1])), np.max(np.abs(b[2])))
        out.append(0.0 if m == 0 else np.max(np.abs(a[f] - b[f]) / (np.abs(b[f]) + 1e-3 * m)))
    return max(out)


@pytest.mark.parametrize("precision,name", [(0, "freezing"), (1, "freezing"), (0, "plume"), (1, "plume4096")])
def test_static_scratch_step_matches_workspace_step(P, precision, name):
    n = 20
    if name == "freezing":
        c, uf = cases.freezing_case(nx=96, nr=40)
    elif name == "plume":
        c, uf = cases.plume_case(nx=256, nr=64)
    else:   # the largest grid the static scratch is sized for
        c, uf = cases.plume_case(nx=4096, nr=1024)
        n = 3
    cfl = 0.5
    # reference: the workspace path, two runs of n steps from the same start
    ref = P.Solver(c, uf, precision=precision)
    ref.init_state(cfl)
    U0 = ref.U.clone()
    ref.load_state(U0, cfl)
    ref.step(n, cfl)
    ref1 = ref.U.clone()
    ref.load_state(ref1, cfl)
    ref.step(n, cfl)
    ref2 = ref.U.clone()
    torch.cuda.synchronize()
    # allocation-free path: two calls in a row through the C ABI, sharing the static scratch
    U = U0.clone()
    U1 = torch.empty_like(U)
    ufac = torch.tensor(np.asarray(uf, dtype=np.float64), device=U.device)
    P.ct_step_static(c, precision, ufac, U, U1, n, cfl)
    torch.cuda.synchronize()
    first = U.clone()
    P.ct_step_static(c, precision, ufac, U, U1, n, cfl)
    torch.cuda.synchronize()
    tol = 1e-9 if precision == 0 else 1e-6
    e1 = _field_rel_err(first.double().cpu().numpy(), ref1.double().cpu().numpy())
    e2 = _field_rel_err(U.double().cpu().numpy(), ref2.double().cpu().numpy())
    assert e1 <= tol and e2 <= tol, (e1, e2)


def test_static_scratch_rejects_oversized_cases(P):
    c, uf = cases.plume_case(nx=8192, nr=2048)     # 88,064 tiles of 16x12: beyond the 6 MiB scratch
    U = torch.zeros(1, device="cuda")
    U1 = torch.zeros(1, device="cuda")
    with pytest.raises(P.ContrailError) as e:
        P.ct_step_static(c, 0, None, U, U1, 1, 0.5)
    assert e.value.status == 6 and "static scratch" in str(e.value)
