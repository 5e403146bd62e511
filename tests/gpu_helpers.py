"""Shared helpers of the GPU tests (comparison metrics; no method arithmetic)."""
import numpy as np

FIELD_NAMES = ("rho", "rho_u", "rho_v", "rho_E", "rho_Yv", "ml0", "ml1", "ml2", "ml3",
               "ms0", "ms1", "ms2", "ms3", "rho_ns", "mh0", "mh1", "mh2", "mh3")

# Floors of the FP64 parity metric, as fractions of a field's largest |value|.  Cells above
# 1e-5 of the field's maximum are held to the relative tolerance; below it, to an absolute
# one of tolerance x 1e-5 x max (1e-14 x max at the 1e-9 tolerance, some 50 units in the
# last place of the field scale: the rounding that upwind fluxes of field-scale quantities
# leave in nearly empty cells, such as soot or core water diffused across the initially
# sharp core/bypass contact, or a crystal population at its edge).  rho v is judged on the
# momentum scale max(|rho u|, |rho v|) with a floor of 1e-3: in a parallel jet it is
# rounding noise of the momentum (about 1e-13 of it), and relative errors of noise are not
# a property of either implementation.
FLOOR_FP64 = 1e-5
FLOOR_RHO_V = 1e-3
# The FP32 comparisons keep a 1e-3 floor for every field: below it, FP32 rounding of the
# field scale (about 6e-8 of max per operation) dominates any relative measure.
FLOOR_FP32 = 1e-3


def field_rel_err(Ug, Uo, floor_frac=FLOOR_FP64, floor_frac_v=FLOOR_RHO_V):
    """Per field: max over cells of |g - o| / (|o| + floor_f), floor_f = floor_frac x the
    field's max |o| (for rho v: floor_frac_v x the momentum scale max(|rho u|, |rho v|))."""
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
        fl = floor_frac_v if f == 2 else floor_frac
        out[f] = np.max(np.abs(Ug[f] - Uo[f]) / (np.abs(Uo[f]) + fl * m))
    return out


def report(errs):
    return ", ".join(f"{n}={e:.1e}" for n, e in zip(FIELD_NAMES, errs))
