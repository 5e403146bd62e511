"""Shared helpers of the GPU tests (comparison metrics; no method arithmetic)."""
import numpy as np

FIELD_NAMES = ("rho", "rho_u", "rho_v", "rho_E", "rho_Yv", "ml0", "ml1", "ml2", "ml3",
               "ms0", "ms1", "ms2", "ms3", "rho_ns", "mh0", "mh1", "mh2", "mh3")


def field_rel_err(Ug, Uo, floor_frac=1e-3):
    """Per field: max over cells of |g - o| / (|o| + floor_frac * scale_f), with scale_f the
    field's max |o| (the momentum scale max|rho u| for rho v, which is zero up to rounding
    in a parallel jet).  Cells above floor_frac * scale_f are held to the relative
    tolerance; the rest to an absolute one of tolerance * floor_frac * scale_f."""
    nf = Uo.shape[0]   # 14, or 18 with the bimodal liquid
    Ug = Ug.reshape(nf, -1)
    Uo = Uo.reshape(nf, -1)
    out = np.zeros(nf)
    mom = max(np.max(np.abs(Uo[1])), np.max(np.abs(Uo[2])))
    for f in range(nf):
        m = np.max(np.abs(Uo[f])) if f != 2 else mom
        if m == 0.0:
            out[f] = np.max(np.abs(Ug[f]))
            continue
        out[f] = np.max(np.abs(Ug[f] - Uo[f]) / (np.abs(Uo[f]) + floor_frac * m))
    return out


def report(errs):
    return ", ".join(f"{n}={e:.1e}" for n, e in zip(FIELD_NAMES, errs))
