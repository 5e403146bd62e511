"""ctypes wrapper of contrail_oracle.c (test infrastructure; see the package docstring).

`build()` compiles the C oracle with gcc (-O2 -ffp-contract=off, OpenMP over rows) into
oracle/_build/.  The wrapper only marshals numpy arrays; all arithmetic is in the C file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "contrail_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

sys.path.insert(0, os.path.dirname(_HERE))
from synth.cases import CASE_KEYS  # noqa: E402

NF = 14
NF_BI = 18        # fields of a state with the bimodal liquid
NDIAG = 32
AUX_NAMES = ("lnS_l", "lnS_i", "lnJ_hom", "lnJ_het", "active", "r_crit", "phi", "G_l", "G_s",
             "koop_log10J", "omega")


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrCase(C.Structure):
    _fields_ = [(k, C.c_int32 if t == "i" else C.c_double) for k, t in CASE_KEYS]


def nfields(c: dict) -> int:
    """Fields of a case's state: 14, or 18 with the bimodal liquid."""
    return NF_BI if int(c.get("bimodal", 0)) else NF


def _case(c: dict) -> OrCase:
    if int(c.get("bimodal", 0)) and int(c.get("equilibrium", 0)):
        raise ValueError("the equilibrium model carries one condensate: not with the bimodal liquid")
    s = OrCase()
    for k, t in CASE_KEYS:
        setattr(s, k, int(c[k]) if t == "i" else float(c[k]))
    return s


_lib = None
_dp = C.POINTER(C.c_double)


def _L():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        d = C.c_double
        for name in ("or_ln_psat_l", "or_ln_psat_i", "or_sigma_lg", "or_hfg", "or_hsg",
                     "or_koop_log10J"):
            getattr(lib, name).restype = d
            getattr(lib, name).argtypes = [d]
        lib.or_tsat.restype = d
        lib.or_tsat.argtypes = [d, C.c_int]
        lib.or_growth.restype = d
        lib.or_growth.argtypes = [d] * 11
        lib.or_roe_flux.restype = None
        lib.or_roe_flux.argtypes = [_dp, _dp, C.c_int, _dp]
        lib.or_create.restype = C.c_void_p
        lib.or_create.argtypes = [C.POINTER(OrCase), _dp]
        lib.or_destroy.argtypes = [C.c_void_p]
        lib.or_init_state.argtypes = [C.c_void_p, _dp]
        lib.or_step.restype = C.c_int
        lib.or_step.argtypes = [C.c_void_p, _dp, C.c_int, d, _dp]
        lib.or_compute_dt.restype = d
        lib.or_compute_dt.argtypes = [C.c_void_p, _dp, d]
        lib.or_derived.argtypes = [C.c_void_p, _dp, C.c_int, d, _dp]
        lib.or_source_batch.argtypes = [C.POINTER(OrCase), _dp, C.c_int, d, _dp, _dp]
        lib.or_prim_to_cons_batch.argtypes = [_dp, C.c_int, _dp]
        lib.or_cons_to_prim_batch.argtypes = [_dp, C.c_int, _dp]
        lib.or_boundary_states.argtypes = [C.c_void_p, _dp, _dp]
        lib.or_residual.argtypes = [C.c_void_p, _dp, d, _dp, _dp]
        lib.or_const.restype = d
        lib.or_const.argtypes = [C.c_int]
        lib.or_table_eval.restype = d
        lib.or_table_eval.argtypes = [C.c_int, d, C.c_int]
        lib.or_dv_mol.restype = d
        lib.or_dv_mol.argtypes = [d, d]
        lib.or_diffusive_flux.argtypes = [_dp, _dp, d, d, _dp]
        lib.or_diffusive_flux_n.argtypes = [_dp, _dp, d, d, C.c_int, _dp]
        lib.or_roe_flux_n.argtypes = [_dp, _dp, C.c_int, C.c_int, _dp]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def ln_psat_l(T: float) -> float:
    return _L().or_ln_psat_l(T)


def ln_psat_i(T: float) -> float:
    return _L().or_ln_psat_i(T)


def tsat(pv: float, which: int = 0) -> float:
    return _L().or_tsat(pv, which)


def sigma_lg(T: float) -> float:
    return _L().or_sigma_lg(T)


def growth(r, T, Tsat, lnS, sig, rho_d, h, lam_g, lbar, gam_g, cp_g) -> float:
    return _L().or_growth(r, T, Tsat, lnS, sig, rho_d, h, lam_g, lbar, gam_g, cp_g)


def koop_log10J(daw: float) -> float:
    return _L().or_koop_log10J(daw)


def const(which: str) -> float:
    idx = ("R_v", "R_a", "cv_a", "cv_v", "e0_v", "e0_s", "f_theta", "mu_min").index(which)
    return _L().or_const(idx)


def hfg(T: float) -> float:
    return _L().or_hfg(T)


def table_eval(which: int, T: float, der: int = 0) -> float:
    """Tabulated property (0 ln p_sat,l, 1 ln p_sat,i, 2 sigma_lg) or its derivative."""
    return _L().or_table_eval(which, T, der)


def dv_mol(T: float, p: float) -> float:
    return _L().or_dv_mol(T, p)


def diffusive_flux(qa, qb, h: float, nu_t: float) -> np.ndarray:
    """Viscous/diffusive face flux G between primitive vectors qa (minus side), qb."""
    qa = np.ascontiguousarray(qa, dtype=np.float64)
    qb = np.ascontiguousarray(qb, dtype=np.float64)
    G = np.zeros(len(qa))
    _L().or_diffusive_flux_n(_ptr(qa), _ptr(qb), h, nu_t, len(qa), _ptr(G))
    return G


def roe_flux(qL, qR, direction: int) -> np.ndarray:
    qL = np.ascontiguousarray(qL, dtype=np.float64)
    qR = np.ascontiguousarray(qR, dtype=np.float64)
    F = np.zeros(len(qL))
    _L().or_roe_flux_n(_ptr(qL), _ptr(qR), direction, len(qL), _ptr(F))
    return F


def source_batch(case: dict, U: np.ndarray, dt: float):
    """Q (n x nf) and aux (n x 11) of conserved states U (n x nf; nf = 18 for the bimodal
    liquid, else 14)."""
    nf = nfields(case)
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(-1, nf)
    n = U.shape[0]
    Q = np.zeros((n, nf))
    aux = np.zeros((n, 11))
    cs = _case(case)
    _L().or_source_batch(C.byref(cs), _ptr(U), n, dt, _ptr(Q), _ptr(aux))
    return Q, aux


def prim_to_cons_batch(P: np.ndarray) -> np.ndarray:
    """Rows (p, T, u, v, Y_v, ml0..3, ms0..3, ns) -> conserved rows (n x 14)."""
    P = np.ascontiguousarray(P, dtype=np.float64).reshape(-1, NF)
    U = np.zeros_like(P)
    _L().or_prim_to_cons_batch(_ptr(P), P.shape[0], _ptr(U))
    return U


def cons_to_prim_batch(U: np.ndarray) -> np.ndarray:
    """Conserved rows -> (rho, u, v, p, T, Y_v, Y_l, Y_s, c^2) rows."""
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(-1, NF)
    P = np.zeros((U.shape[0], 9))
    _L().or_cons_to_prim_batch(_ptr(U), U.shape[0], _ptr(P))
    return P


class Oracle:
    """One case on the CPU.  State arrays are (nf, nr, nx) float64, x fastest (nf = 14, or 18
    with the bimodal liquid)."""

    def __init__(self, case: dict, ufac_rows=None):
        self.case = dict(case)
        self.nx = int(case["nx"])
        self.nr = int(case["nr"]) if case["geom"] == 1 else 1
        self.nf = nfields(case)
        self._cs = _case(case)
        if ufac_rows is None:
            ufac_rows = np.ones(self.nr)
        self._ufac = np.ascontiguousarray(ufac_rows, dtype=np.float64)
        self._h = _L().or_create(C.byref(self._cs), _ptr(self._ufac))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.or_destroy(self._h)
            self._h = None

    @property
    def shape(self):
        return (self.nf, self.nr, self.nx)

    def init_state(self) -> np.ndarray:
        U = np.zeros(self.shape)
        _L().or_init_state(self._h, _ptr(U))
        return U

    def step(self, U: np.ndarray, nsteps: int, cfl: float) -> np.ndarray:
        """Advance U in place by nsteps; returns the per-step diagnostics (nsteps x 32)."""
        assert U.shape == self.shape and U.dtype == np.float64 and U.flags.c_contiguous
        diag = np.zeros((nsteps, NDIAG))
        _L().or_step(self._h, _ptr(U), nsteps, cfl, _ptr(diag))
        return diag

    def dt(self, U: np.ndarray, cfl: float) -> float:
        return _L().or_compute_dt(self._h, _ptr(np.ascontiguousarray(U)), cfl)

    def derived(self, U: np.ndarray, which: int, dt: float = 1e-6) -> np.ndarray:
        out = np.zeros((self.nr, self.nx))
        _L().or_derived(self._h, _ptr(np.ascontiguousarray(U)), which, dt, _ptr(out))
        return out

    def residual(self, U: np.ndarray, dt: float):
        L = np.zeros(self.shape)
        b = np.zeros(3)
        _L().or_residual(self._h, _ptr(np.ascontiguousarray(U)), dt, _ptr(L), _ptr(b))
        return L, b

    def boundary_states(self):
        inflow = np.zeros((self.nr, self.nf))
        amb = np.zeros(self.nf)
        _L().or_boundary_states(self._h, _ptr(inflow), _ptr(amb))
        return inflow, amb


def roe_c2(qL: np.ndarray, qR: np.ndarray, direction: int) -> np.ndarray:
    """Roe sound speed squared of a face before and after its 1 % guard, and both sides'
    c^2 (face primitive vectors of 14 or 18 fields)."""
    qL = np.ascontiguousarray(qL, dtype=np.float64)
    qR = np.ascontiguousarray(qR, dtype=np.float64)
    out = np.zeros(4)
    lib = _L()
    lib.or_roe_c2.argtypes = [_dp, _dp, C.c_int, C.c_int, _dp]
    lib.or_roe_c2(_ptr(qL), _ptr(qR), direction, qL.shape[0], _ptr(out))
    return out
