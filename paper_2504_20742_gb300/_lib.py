"""ctypes binding of libcontrail.so: same names as the C ABI of include/contrail.h.

Arguments are marshalled only (torch tensors -> device pointers, dicts -> ct_case); every
step of the computation runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libcontrail.so")

CT_FP64, CT_FP32, CT_FP32_MLP = 0, 1, 2
NF, NDIAG, NAUX = 14, 32, 11
NF_BI = 18   # fields of a state with the bimodal liquid


def nfields(case) -> int:
    """Fields of a case's state: 14, or 18 with the bimodal liquid."""
    return NF_BI if int(case.get("bimodal", 0)) else NF
CT_MLP_IN, CT_MLP_HIDDEN, CT_MLP_OUT = 16, 128, 10

# ct_case fields, in the order of include/contrail.h
_CASE_FIELDS = (
    ("geom", "i"), ("nx", "i"), ("nr", "i"), ("bc_xlo", "i"), ("bc_xhi", "i"), ("bc_rhi", "i"),
    ("phase_change", "i"), ("freezing", "i"), ("lx", "d"), ("lr", "d"), ("area_a", "d"),
    ("x_throat", "d"), ("d_core", "d"), ("d_fan", "d"), ("wall_len", "d"), ("T_amb", "d"),
    ("p_amb", "d"), ("S_ice_amb", "d"), ("mach_coflow", "d"), ("T_core", "d"), ("u_core", "d"),
    ("Yv_core", "d"), ("T_byp", "d"), ("u_byp", "d"), ("n_soot", "d"), ("soot_rm", "d"),
    ("soot_sigma", "d"), ("p0", "d"), ("T0", "d"), ("Yv_inlet", "d"), ("seed_l_n", "d"),
    ("seed_l_r", "d"), ("seed_s_n", "d"), ("seed_s_r", "d"), ("mix_width", "d"), ("nu_t", "d"),
    ("viscous", "i"), ("tables", "i"), ("equilibrium", "i"), ("bimodal", "i"),
)


class CtCase(C.Structure):
    _fields_ = [(k, C.c_int32 if t == "i" else C.c_double) for k, t in _CASE_FIELDS]

    @classmethod
    def from_dict(cls, d: dict) -> "CtCase":
        s = cls()
        for k, t in _CASE_FIELDS:
            setattr(s, k, int(d.get(k, 0)) if t == "i" else float(d.get(k, 0.0)))
        return s


class CtTrainCfg(C.Structure):
    _fields_ = [("epochs", C.c_int), ("batch", C.c_int), ("lr", C.c_float), ("lr_final", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float), ("seed", C.c_uint64),
                ("tensor_cores", C.c_int), ("out_weight", C.c_float * 16)]


class ContrailError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"contrail status {status}: {msg}")
        self.status = status


_lib = None
_vp, _dp, _cp = C.c_void_p, C.POINTER(C.c_double), C.POINTER(CtCase)

_SIGS = {
    "ct_workspace_bytes": (C.c_size_t, [_cp, C.c_int]),
    "ct_setup": (C.c_int, [_cp, C.c_int, _dp, _vp, C.c_size_t, _vp]),
    "ct_init_state": (C.c_int, [_cp, C.c_int, _vp, _vp, C.c_double, _vp]),
    "ct_load_state": (C.c_int, [_cp, C.c_int, _vp, _vp, _vp, C.c_double, _vp]),
    "ct_step": (C.c_int, [_cp, C.c_int, _vp, _vp, _vp, C.c_int, C.c_double, _vp]),
    "ct_step_host": (C.c_int, [_cp, C.c_int, _vp, _vp, _vp, _vp, _vp, C.c_int, C.c_double, _vp]),
    "ct_diagnostics": (C.c_int, [_vp, _dp, C.c_int, _vp]),
    "ct_derived": (C.c_int, [_cp, C.c_int, _vp, C.c_int, C.c_double, _vp, _vp]),
    "ct_read_field": (C.c_int, [_cp, C.c_int, _vp, C.c_int, _dp, C.c_size_t, _vp]),
    "ct_source_batch": (C.c_int, [_cp, C.c_int, _vp, C.c_int, C.c_double, _vp, _vp, _vp]),
    "ct_reconstruct_faces": (C.c_int, [_vp, _vp, _vp, C.c_int, _vp, _vp, _vp]),
    "ct_step_static": (C.c_int, [_cp, C.c_int, _vp, _vp, _vp, C.c_int, C.c_double, _vp]),
    "ct_mlp_dataset": (C.c_int, [_cp, _vp, C.c_int, _vp, _vp, _vp, _vp]),
    "ct_mlp_param_count": (C.c_int, []),
    "ct_mlp_work_bytes": (C.c_size_t, [C.c_int]),
    "ct_mlp_forward": (C.c_int, [_vp, _vp, C.c_int, _vp, _vp, C.c_size_t, _vp]),
    "ct_mlp_loss_grad": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int, _vp, _vp, _vp, C.c_size_t, _vp]),
    "ct_mlp_loss_grad_tc": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int, _vp, _vp, _vp, _vp, C.c_size_t, _vp]),
    "ct_mlp_adam": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int,
                              _vp]),
    "ct_mlp_colstats": (C.c_int, [_vp, _vp, C.c_int, C.c_int, _vp, _vp]),
    "ct_mlp_standardize": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp, _vp]),
    "ct_train_workspace_bytes": (C.c_size_t, [C.c_int, C.c_int, C.c_int]),
    "ct_train_surrogate": (C.c_int, [_vp, _vp, _vp, C.c_int, C.POINTER(CtTrainCfg), _vp, _vp,
                                     C.POINTER(C.c_float), _vp, C.c_size_t, _vp]),
    "ct_mlp_blob_bytes": (C.c_size_t, []),
    "ct_mlp_pack": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "ct_mlp_infer": (C.c_int, [_vp, _vp, C.c_int, _vp, _vp, _vp]),
    "ct_step_surrogate": (C.c_int, [_cp, _vp, _vp, _vp, _vp, C.c_int, C.c_double, _vp]),
    "ct_tile_shape_count": (C.c_int, []),
    "ct_tile_shape": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "ct_tile_shape_ctas": (C.c_int, [C.c_int, C.c_int]),
    "ct_set_tile_shape": (C.c_int, [_cp, C.c_int, C.c_int]),
    "ct_autotune": (C.c_int, [_cp, C.c_int, _vp, _vp, _vp, _vp, C.c_int, _vp, C.POINTER(C.c_int),
                              C.POINTER(C.c_float)]),
    "ct_batch_workspace_bytes": (C.c_size_t, [_cp, C.c_int]),
    "ct_batch_state_elems": (C.c_size_t, [_cp, C.c_int]),
    "ct_batch_create": (C.c_int, [_cp, C.c_int, C.c_int, _dp, _vp, C.c_size_t, _vp, C.POINTER(_vp)]),
    "ct_batch_destroy": (None, [_vp]),
    "ct_batch_init_state": (C.c_int, [_vp, _vp, C.c_double]),
    "ct_batch_load_state": (C.c_int, [_vp, _vp, _vp, C.c_double]),
    "ct_batch_set_tile_shape": (C.c_int, [_vp, C.c_int]),
    "ct_batch_tile_shape": (C.c_int, [_vp]),
    "ct_batch_autotune": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    "ct_batch_step": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int, C.c_double]),
    "ct_batch_diagnostics": (C.c_int, [_vp, _dp]),
    "ct_last_error": (C.c_char_p, []),
    "ct_version": (C.c_char_p, []),
}


def lib_path() -> str:
    return _LIB_PATH


def exported_symbols():
    return tuple(_SIGS)


def _L():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(
                f"libcontrail.so not built ({_LIB_PATH}); run paper_2504_20742_gb300.build.build() "
                "(nvcc, sm_103a). There is no CPU fallback.")
        lib = C.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _case(c) -> CtCase:
    return c if isinstance(c, CtCase) else CtCase.from_dict(c)


def _ptr(x):
    """Device/host pointer of a torch tensor, numpy array, int address or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(status: int):
    if status != 0:
        raise ContrailError(status, _L().ct_last_error().decode())


def ct_workspace_bytes(case, precision: int) -> int:
    return _L().ct_workspace_bytes(C.byref(_case(case)), precision)


def ct_setup(case, precision, ufac_rows, work, work_bytes, stream=None):
    u = None
    if ufac_rows is not None:
        arr = np.ascontiguousarray(ufac_rows, dtype=np.float64)
        u = arr.ctypes.data_as(_dp)
    _check(_L().ct_setup(C.byref(_case(case)), precision, u, _ptr(work), work_bytes, _stream(stream)))


def ct_init_state(case, precision, work, U, cfl, stream=None):
    _check(_L().ct_init_state(C.byref(_case(case)), precision, _ptr(work), _ptr(U), cfl, _stream(stream)))


def ct_load_state(case, precision, work, U_src, U, cfl, stream=None):
    _check(_L().ct_load_state(C.byref(_case(case)), precision, _ptr(work), _ptr(U_src), _ptr(U), cfl,
                              _stream(stream)))


def ct_step(case, precision, U, U1, work, nsteps, cfl, stream=None):
    _check(_L().ct_step(C.byref(_case(case)), precision, _ptr(U), _ptr(U1), _ptr(work), nsteps, cfl,
                        _stream(stream)))


def ct_step_host(case, precision, U_host_in, U_host_out, U, U1, work, nsteps, cfl, stream=None):
    _check(_L().ct_step_host(C.byref(_case(case)), precision, _ptr(U_host_in), _ptr(U_host_out), _ptr(U),
                             _ptr(U1), _ptr(work), nsteps, cfl, _stream(stream)))


def ct_diagnostics(work, stream=None, nout: int = NDIAG, raise_nonfinite: bool = False) -> np.ndarray:
    out = np.zeros(nout)
    st = _L().ct_diagnostics(_ptr(work), out.ctypes.data_as(_dp), nout, _stream(stream))
    if st != 0 and (st != 3 or raise_nonfinite):
        _check(st)
    return out


def ct_derived(case, precision, U, which, dt, out, stream=None):
    _check(_L().ct_derived(C.byref(_case(case)), precision, _ptr(U), which, dt, _ptr(out), _stream(stream)))


def ct_source_batch(case, precision, U, n, dt, Q, aux, stream=None):
    _check(_L().ct_source_batch(C.byref(_case(case)), precision, _ptr(U), n, dt, _ptr(Q), _ptr(aux),
                                _stream(stream)))


def ct_reconstruct_faces(am, a0, a1, n, lo, hi, stream=None):
    _check(_L().ct_reconstruct_faces(_ptr(am), _ptr(a0), _ptr(a1), n, _ptr(lo), _ptr(hi), _stream(stream)))


def ct_step_static(case, precision, ufac_rows_dev, U, U1, nsteps, cfl, stream=None):
    """Allocation-free step: scratch in the library's static device array (see contrail.h)."""
    _check(_L().ct_step_static(C.byref(_case(case)), precision, _ptr(ufac_rows_dev), _ptr(U), _ptr(U1),
                               nsteps, cfl, _stream(stream)))


def ct_mlp_dataset(case, U, n, X, Y, M, stream=None):
    _check(_L().ct_mlp_dataset(C.byref(_case(case)), _ptr(U), n, _ptr(X), _ptr(Y), _ptr(M), _stream(stream)))


def ct_mlp_param_count() -> int:
    return _L().ct_mlp_param_count()


def ct_mlp_work_bytes(n: int) -> int:
    return _L().ct_mlp_work_bytes(n)


def ct_mlp_forward(params, X, n, Y, work, work_bytes, stream=None):
    _check(_L().ct_mlp_forward(_ptr(params), _ptr(X), n, _ptr(Y), _ptr(work), work_bytes, _stream(stream)))


def ct_mlp_loss_grad(params, X, Y, M, n, grad, loss, work, work_bytes, stream=None):
    _check(_L().ct_mlp_loss_grad(_ptr(params), _ptr(X), _ptr(Y), _ptr(M), n, _ptr(grad), _ptr(loss), _ptr(work),
                                 work_bytes, _stream(stream)))


def ct_mlp_loss_grad_tc(params, X, Y, M, n, grad, loss, err_flag, work, work_bytes, stream=None):
    _check(_L().ct_mlp_loss_grad_tc(_ptr(params), _ptr(X), _ptr(Y), _ptr(M), n, _ptr(grad), _ptr(loss),
                                    _ptr(err_flag), _ptr(work), work_bytes, _stream(stream)))


def ct_mlp_adam(params, grad, m, v, nparam, lr, beta1, beta2, eps, step, stream=None):
    _check(_L().ct_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), nparam, lr, beta1, beta2, eps, step,
                            _stream(stream)))


def ct_mlp_colstats(X, M, n, d, out, stream=None):
    _check(_L().ct_mlp_colstats(_ptr(X), _ptr(M), n, d, _ptr(out), _stream(stream)))


def ct_mlp_standardize(X, n, d, mean, sd, stream=None):
    _check(_L().ct_mlp_standardize(_ptr(X), n, d, _ptr(mean), _ptr(sd), _stream(stream)))


def ct_mlp_blob_bytes() -> int:
    return _L().ct_mlp_blob_bytes()


def ct_mlp_pack(params, x_mean, x_sd, x_min, x_max, y_mean, y_sd, y_min, y_max, blob, stream=None):
    _check(_L().ct_mlp_pack(_ptr(params), _ptr(x_mean), _ptr(x_sd), _ptr(x_min), _ptr(x_max), _ptr(y_mean),
                            _ptr(y_sd), _ptr(y_min), _ptr(y_max), _ptr(blob), _stream(stream)))


def ct_mlp_infer(blob, X, n, Y, err_flag, stream=None):
    _check(_L().ct_mlp_infer(_ptr(blob), _ptr(X), n, _ptr(Y), _ptr(err_flag), _stream(stream)))


def ct_step_surrogate(case, U, U1, work, blob, nsteps, cfl, stream=None):
    _check(_L().ct_step_surrogate(C.byref(_case(case)), _ptr(U), _ptr(U1), _ptr(work), _ptr(blob), nsteps, cfl,
                                  _stream(stream)))


def ct_last_error() -> str:
    return _L().ct_last_error().decode()


def ct_version() -> str:
    return _L().ct_version().decode()


# ---- tile shapes and the autotuner ----------------------------------------------------------
def ct_tile_shape_count() -> int:
    return _L().ct_tile_shape_count()


def ct_tile_shape(shape: int) -> tuple[int, int]:
    tx, ty = C.c_int(), C.c_int()
    _check(_L().ct_tile_shape(shape, C.byref(tx), C.byref(ty)))
    return tx.value, ty.value


def ct_tile_shape_ctas(shape: int, precision: int = 1) -> int:
    return _L().ct_tile_shape_ctas(shape, precision)


def ct_set_tile_shape(case, precision, shape):
    _check(_L().ct_set_tile_shape(C.byref(_case(case)), precision, shape))


def ct_autotune(case, precision, U, U1, work, blob=None, reps=5, stream=None):
    """Returns (chosen shape, ms per first-stage launch of every shape, -1 where unavailable)."""
    n = ct_tile_shape_count()
    sh = C.c_int()
    ms = (C.c_float * n)()
    _check(_L().ct_autotune(C.byref(_case(case)), precision, _ptr(U), _ptr(U1), _ptr(work), _ptr(blob), reps,
                            _stream(stream), C.byref(sh), ms))
    return sh.value, [float(v) for v in ms]


# ---- batched step ---------------------------------------------------------------------------------
def _cases(cases):
    arr = (CtCase * len(cases))()
    for k, c in enumerate(cases):
        arr[k] = _case(c)
    return arr


def ct_batch_workspace_bytes(cases) -> int:
    return _L().ct_batch_workspace_bytes(_cases(cases), len(cases))


def ct_batch_state_elems(cases) -> int:
    return _L().ct_batch_state_elems(_cases(cases), len(cases))


def ct_batch_create(cases, precision, ufac_rows, work, work_bytes, stream=None) -> int:
    """Returns the batch handle (an address; free with ct_batch_destroy)."""
    u = None
    if ufac_rows is not None:
        arr = np.ascontiguousarray(ufac_rows, dtype=np.float64)
        u = arr.ctypes.data_as(_dp)
    h = _vp()
    _check(_L().ct_batch_create(_cases(cases), len(cases), precision, u, _ptr(work), work_bytes, _stream(stream),
                                C.byref(h)))
    return h.value


def ct_batch_destroy(b):
    _L().ct_batch_destroy(b)


def ct_batch_init_state(b, U, cfl):
    _check(_L().ct_batch_init_state(b, _ptr(U), cfl))


def ct_batch_load_state(b, U_src, U, cfl):
    _check(_L().ct_batch_load_state(b, _ptr(U_src), _ptr(U), cfl))


def ct_batch_set_tile_shape(b, shape):
    _check(_L().ct_batch_set_tile_shape(b, shape))


def ct_batch_tile_shape(b) -> int:
    return _L().ct_batch_tile_shape(b)


def ct_batch_autotune(b, U, U1, blob=None, reps=3):
    n = ct_tile_shape_count()
    sh = C.c_int()
    ms = (C.c_float * n)()
    _check(_L().ct_batch_autotune(b, _ptr(U), _ptr(U1), _ptr(blob), reps, C.byref(sh), ms))
    return sh.value, [float(v) for v in ms]


def ct_batch_step(b, U, U1, blob, nsteps, cfl):
    _check(_L().ct_batch_step(b, _ptr(U), _ptr(U1), _ptr(blob), nsteps, cfl))


def ct_batch_diagnostics(b, ncases: int, raise_nonfinite: bool = False) -> np.ndarray:
    out = np.zeros((ncases, NDIAG))
    st = _L().ct_batch_diagnostics(b, out.ctypes.data_as(_dp))
    if st != 0 and (st != 3 or raise_nonfinite):
        _check(st)
    return out


def ct_read_field(case, precision, U, field, stream=None) -> np.ndarray:
    """Field `field` of the device state U as an (nr, nx) float64 host array."""
    c = _case(case)
    nr = c.nr if c.geom == 1 else 1
    out = np.empty((nr, c.nx), dtype=np.float64)
    _check(_L().ct_read_field(C.byref(c), precision, _ptr(U), field, out.ctypes.data_as(_dp), out.size,
                              _stream(stream)))
    return out


def ct_train_workspace_bytes(n, batch, epochs) -> int:
    return _L().ct_train_workspace_bytes(n, batch, epochs)


def ct_train_surrogate(X, Y, M, n, cfg: dict, params, stats, work, work_bytes, stream=None) -> np.ndarray:
    """Runs the whole training loop in the library; returns the per-epoch mean loss."""
    k = CtTrainCfg(epochs=int(cfg["epochs"]), batch=int(cfg["batch"]), lr=float(cfg["lr"]),
                   lr_final=float(cfg["lr_final"]), beta1=float(cfg.get("beta1", 0.9)),
                   beta2=float(cfg.get("beta2", 0.999)), eps=float(cfg.get("eps", 1e-8)),
                   seed=int(cfg.get("seed", 0)), tensor_cores=int(cfg.get("tensor_cores", 0)))
    w = list(cfg.get("out_weight", [1.0] * CT_MLP_OUT))
    for q in range(16):
        k.out_weight[q] = float(w[q]) if q < len(w) else 0.0
    hist = (C.c_float * k.epochs)()
    _check(_L().ct_train_surrogate(_ptr(X), _ptr(Y), _ptr(M), n, C.byref(k), _ptr(params), _ptr(stats), hist,
                                   _ptr(work), work_bytes, _stream(stream)))
    return np.array([float(v) for v in hist])
