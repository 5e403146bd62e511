"""The FP64 van Leer reconstruction of the stage kernels (Sec. 3.2), through
ct_reconstruct_faces, against the plain formula evaluated in NumPy: the decision dm*dp > 0
taken in IEEE FP64 and hs = dm*dp/(dm+dp) by IEEE division.  The kernels take the decision
on the integer pipe (bitwise-equal neighbours, signs, exponent ranges) and fall back to the
product only outside [2^-511, 2^511); the inputs therefore span signed zeros, subnormal,
tiny and huge differences around those bounds, infinities and NaN, besides random cells.
Where no slope is taken the face states must be bit for bit a0 and a0 + 0; where one is,
they may differ from the IEEE-division form by the Newton reciprocal's few ulp."""
import itertools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2504_20742_gb300 as P
from synth import cases

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


def _special_triples():
    v = [0.0, -0.0, 5e-324, -5e-324, 1e-310, 2.0 ** -1022, 2.0 ** -600, -2.0 ** -541, 2.0 ** -540,
         2.0 ** -512, 2.0 ** -511, -2.0 ** -510, 1e-160, 1e-20, 0.5, 1.0, 1.0 + 2.0 ** -52, 3.0, -1.0,
         -3.0, 1e20, 2.0 ** 510, 2.0 ** 511, -2.0 ** 512, 1e300, np.inf, -np.inf, np.nan]
    t = np.array(list(itertools.product(v, repeat=3)), dtype=np.float64)
    return t[:, 0], t[:, 1], t[:, 2]


def _random_triples(n):
    u = cases.splitmix64_uniform(2504, 6 * n).reshape(6, n)
    a0 = 10.0 ** (40.0 * u[0] - 20.0) * np.where(u[1] < 0.5, -1.0, 1.0)
    rm = 10.0 ** (-17.0 * u[2]) * (2.0 * u[3] - 1.0)
    rp = 10.0 ** (-17.0 * u[4]) * (2.0 * u[5] - 1.0)
    am = a0 * (1.0 + rm)
    a1 = a0 * (1.0 + rp)
    am[u[3] < 0.1] = a0[u[3] < 0.1]          # equal neighbours
    a1[u[5] > 0.9] = a0[u[5] > 0.9]
    return am, a0, a1


def _plain(am, a0, a1):
    with np.errstate(all="ignore"):
        dm, dp = a0 - am, a1 - a0
        act = dm * dp > 0.0
        hs = np.where(act, dm * (dp / (dm + dp)), 0.0)
        lo = np.where(act, a0 - hs, a0)
        hi = np.where(act, a0 + hs, a0 + 0.0)
        s = np.abs(dm + dp)
    return act, hs, lo, hi, s


def _device(am, a0, a1):
    n = am.size
    dev = [torch.tensor(x, dtype=torch.float64, device="cuda") for x in (am, a0, a1)]
    lo = torch.empty(n, dtype=torch.float64, device="cuda")
    hi = torch.empty_like(lo)
    P.ct_reconstruct_faces(dev[0], dev[1], dev[2], n, lo, hi)
    torch.cuda.synchronize()
    return lo.cpu().numpy(), hi.cpu().numpy()


def _bits_equal(x, y):
    nan = np.isnan(x) & np.isnan(y)
    return nan | (x.view(np.int64) == y.view(np.int64))


@pytest.mark.parametrize("kind", ["special", "random"])
def test_van_leer_faces_match_the_plain_formula(kind):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    am, a0, a1 = _special_triples() if kind == "special" else _random_triples(1 << 18)
    lo, hi = _device(am, a0, a1)
    act, hs, lo_ref, hi_ref, s = _plain(am, a0, a1)
    # no slope: the face states are a0 and a0 + 0, bit for bit
    bad = ~act & ~(_bits_equal(lo, lo_ref) & _bits_equal(hi, hi_ref))
    assert not bad.any(), f"{bad.sum()} zero-slope cells differ, first at {np.argmax(bad)}"
    # a slope, with dm + dp finite and normal (where the Newton reciprocal is valid): within
    # the reciprocal's error of the IEEE-division form
    ok_range = act & np.isfinite(s) & (s >= 2.0 ** -1022) & (s < 2.0 ** 1022)
    with np.errstate(all="ignore"):
        tl = 8.0 * EPS * np.abs(hs) + np.spacing(np.abs(lo_ref))
        th = 8.0 * EPS * np.abs(hs) + np.spacing(np.abs(hi_ref))
        good = (np.abs(lo - lo_ref) <= tl) & (np.abs(hi - hi_ref) <= th)
    good |= np.isnan(lo) & np.isnan(lo_ref) & np.isnan(hi) & np.isnan(hi_ref)
    bad = ok_range & ~good
    assert not bad.any(), f"{bad.sum()} sloped cells differ, first at {np.argmax(bad)}"
    n_act = int(act.sum())
    assert n_act > 0 and n_act < act.size   # both branches were exercised
