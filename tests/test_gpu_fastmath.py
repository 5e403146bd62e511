"""The Newton reciprocal of the FP64 transport arithmetic against IEEE division: CUDA's
own 1/x and NumPy's on the same inputs, over normal doubles of both signs spanning 1e-300
to 1e300.  Bound: 4 ulp relative error."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from conftest import ROOT
from synth import cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    d = tempfile.mkdtemp()
    so = os.path.join(d, "rcp_check.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared", "-Xcompiler", "-fPIC",
                    "-o", so, os.path.join(ROOT, "tests", "kernels", "rcp_check.cu")], check=True)
    L = ctypes.CDLL(so)
    L.rcp_check.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int]
    return L


def test_newton_reciprocal_within_4_ulp(lib):
    n = 1 << 20
    u = cases.splitmix64_uniform(123, 2 * n).reshape(2, n)
    x = (10.0 ** (600.0 * u[0] - 300.0)) * np.where(u[1] < 0.5, -1.0, 1.0)
    x[:8] = [1.0, -1.0, 3.0, 0.1, 1e-300, 1e300, 2.0 ** -1000, 7.0]
    X = torch.tensor(x, dtype=torch.float64, device="cuda")
    R = torch.empty_like(X)
    D = torch.empty_like(X)
    torch.cuda.synchronize()
    assert lib.rcp_check(X.data_ptr(), R.data_ptr(), D.data_ptr(), n) == 0
    r, dv = R.cpu().numpy(), D.cpu().numpy()
    exact = 1.0 / x
    assert np.array_equal(dv, exact)                      # CUDA's division is IEEE-rounded
    rel = np.abs(r - exact) / np.abs(exact)
    ulp = rel / np.finfo(np.float64).eps
    print("Newton reciprocal: max error %.2f ulp, mean %.3f ulp" % (ulp.max(), ulp.mean()))
    assert ulp.max() <= 4.0
