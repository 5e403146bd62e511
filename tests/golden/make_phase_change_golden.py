"""Write the phase-change golden fixtures of this folder from the paper's equations.

Every value is evaluated with mpmath at 50 significant digits (or exact rational arithmetic
for Koop's polynomial) from the equations as the paper and the cited publications print
them, with the readings written out here a second time, independently of the oracle's C
code.  Inputs that have golden tables of their own (the Sonntag saturation curves, the IAPWS
surface tension, the six-step Newton saturation temperature) are taken from `oracle/`, which
is the only module this script calls.

  cnt_kantrowitz.txt  Eqs. (3), (4), (5), (10): r_crit, dG*/kT, ln J_hom, ln J_het and the
                      Kantrowitz factor phi, on the (S, T) grid {1.5, 3, 5, 10, 20} x
                      {200, 220, 240 K} at 24 kPa, pure vapour in dry air.
  young_growth.txt    Eq. (16): Young's growth rate of droplets and ice crystals from the
                      free-molecular (Kn = 40) to the continuum (Kn = 0.01) regime, super- and
                      subsaturated.
  koop_2000.txt       Koop, Luo, Tsias & Peter (2000), Nature 406, 611, Eq. (7): log10 of
                      the homogeneous ice nucleation rate coefficient (cm^-3 s^-1) as a cubic
                      in the water-activity shift, over the fit's validity range.

Run from the repository root:  python tests/golden/make_phase_change_golden.py
"""
from __future__ import annotations

import os
import sys
from fractions import Fraction

import mpmath as mp

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import oracle as O  # noqa: E402

mp.mp.dps = 50
F = mp.mpf

# constants (SI) as the readings state them
NA = F("6.02214076e23")
KB = F("1.380649e-23")
RU = F("8.314462618")
MW = F("0.018015")
RV = RU / MW
RA = F("287.05")
CVA = RA / F("0.4")           # gamma of dry air 1.4 exactly
CPA = CVA + RA
CPV = F(1859)
CVV = CPV - RV
CL, CS = F(4186), F(2100)
RHOL, RHOS = F(1000), F(917)
TREF = F("273.15")
HLV0, HSL0 = F("2.501e6"), F("3.337e5")
QC = F(1)                     # condensation coefficient (the paper leaves it open)
THETA = mp.pi / 2             # contact angle 90 degrees
ALPHA, BETA = F(11), F(0)     # Young's parameters as the paper uses them
PR = F("0.71")
SIGMA_SV = F("0.106")
P_GAS = F(24000)


def h_fg(T):
    """h_v - h_l: 2.501e6 J/kg at 273.15 K, slope c_p,v - c_l (formation-energy reading)."""
    return HLV0 + (CPV - CL) * (T - TREF)


def h_sg(T):
    """h_v - h_s: h_fg plus h_l - h_s = 3.337e5 J/kg at 273.15 K, slope c_l - c_s."""
    return h_fg(T) + HSL0 + (CL - CS) * (T - TREF)


def sutherland(T):
    return F("1.716e-5") * (T / TREF) ** F("1.5") * (TREF + F("110.4")) / (T + F("110.4"))


def gas(T, p, Yv, Ycond):
    """Gas-phase properties of Young's law: lambda, mean free path, gamma, c_p (per kg of
    gas: dry air + vapour)."""
    Ya = 1 - Yv - Ycond
    Yg = Ya + Yv
    cp = (Ya * CPA + Yv * CPV) / Yg
    cv = (Ya * CVA + Yv * CVV) / Yg
    Rg = (Ya * RA + Yv * RV) / Yg
    mu = sutherland(T)
    lam = mu * cp / PR
    lbar = F("1.5") * mu * mp.sqrt(Rg * T) / p
    return lam, lbar, cp / cv, cp


def young_nu(Tsat, h, gam, cp):
    """nu of Eq. (16)."""
    return RV * Tsat / h * (ALPHA - F("0.5") - (2 - QC) / (2 * QC) * (gam + 1) / (2 * gam) * cp * Tsat / h)


def young_den(r, lbar, nu):
    Kn = lbar / (2 * r)
    return 1 / (1 + 2 * BETA * Kn) + F("3.78") * (1 - nu) * Kn / PR


def yv_for_S(S, T, p):
    """Vapour mass fraction of dry air + vapour with p_v = S p_sat,l(T)."""
    pv = S * mp.exp(F(repr(O.ln_psat_l(float(T)))))
    return pv * RA / (RV * (p - pv) + pv * RA), pv


def cnt_rows():
    rows = []
    f_theta = (2 + mp.cos(THETA)) * (1 - mp.cos(THETA)) ** 2 / 4
    for S in (F("1.5"), F(3), F(5), F(10), F(20)):
        for T in (F(200), F(220), F(240)):
            Yv, pv = yv_for_S(S, T, P_GAS)
            sig = F(repr(O.sigma_lg(float(T))))
            lnS = mp.log(S)
            rc = 2 * sig / (RHOL * RV * T * lnS)                                      # Eq. (3)
            dG = F(4) / 3 * mp.pi * sig * rc ** 2                                      # Eq. (3)
            rhov = pv / (RV * T)                                                       # rho_g read as the vapour density
            A = QC * mp.sqrt(2 * sig * NA ** 3 / (mp.pi * MW ** 3)) * rhov ** 2 / RHOL  # Eq. (4) prefactor
            lnJhom = mp.log(A) - dG / (KB * T)
            lnJhet = mp.log(A) - f_theta * dG / (KB * T)                              # Eqs. (9), (10)
            # Eq. (5) with alpha_crit = Young's heat-transfer coefficient lambda/(r den) at r_crit
            lam, lbar, gam, cp = gas(T, P_GAS, Yv, F(0))
            h = h_fg(T)
            Tsat = F(repr(O.tsat(float(pv), 0)))
            nu = young_nu(Tsat, h, gam, cp)
            alpha = lam / (rc * young_den(rc, lbar, nu))
            phi = QC * rhov / alpha * mp.sqrt(RV * T / (2 * mp.pi)) * (h ** 2 / (RV * T ** 2) - h / T)
            rows.append((S, T, Yv, rc, dG / (KB * T), lnJhom, lnJhet, phi))
    return rows


def young_rows():
    """(phase, S, T, r, n per kg) -> G from Eq. (16) of a monodisperse population of n
    particles per kg at radius r; the gas (dry air + vapour with p_v = S p_sat over the
    phase) holds the condensate as well, at 24 kPa."""
    rows = []
    for phase in ("l", "i"):
        for S, T in ((F("1.3"), F(230)), (F("0.8"), F(230)), (F("1.1"), F(250))):
            for r in (F("3e-9"), F("1e-8"), F("1e-7"), F("1e-6"), F("1e-5")):
                n = F("1e6")
                if phase == "l":
                    lnpsat = F(repr(O.ln_psat_l(float(T))))
                    sig, rho_d, h = F(repr(O.sigma_lg(float(T)))), RHOL, h_fg(T)
                else:
                    lnpsat = F(repr(O.ln_psat_i(float(T))))
                    sig, rho_d, h = SIGMA_SV, RHOS, h_sg(T)
                pv0 = S * mp.exp(lnpsat)
                Yv_gas = pv0 * RA / (RV * (P_GAS - pv0) + pv0 * RA)
                Ycond = F(4) / 3 * mp.pi * rho_d * n * r ** 3
                Yv = Yv_gas * (1 - Ycond)                 # per kg of the whole mixture
                Ya = 1 - Yv - Ycond
                rho = P_GAS / ((Ya * RA + Yv * RV) * T)
                pv = rho * Yv * RV * T                    # Eq. (1): vapour partial pressure
                lnS = mp.log(pv) - lnpsat
                Tsat = F(repr(O.tsat(float(pv), 0 if phase == "l" else 1)))
                lam, lbar, gam, cp = gas(T, P_GAS, Yv, Ycond)
                nu = young_nu(Tsat, h, gam, cp)
                rc = 2 * sig / (rho_d * RV * T * lnS)
                G = lam * (Tsat - T) * (1 - rc / r) / (rho_d * h * r * young_den(r, lbar, nu))
                rows.append((phase, S, T, r, n, Yv, G, lbar / (2 * r)))
    return rows


# Koop et al. (2000), Eq. (7): log10 J = -906.7 + 8502 x - 26924 x^2 + 29180 x^3, x = Delta a_w
KOOP = (Fraction("-906.7"), Fraction(8502), Fraction(-26924), Fraction(29180))


def koop_rows():
    rows = []
    for x in ("0.26", "0.27", "0.28", "0.29", "0.30", "0.305", "0.31", "0.32", "0.33", "0.34"):
        d = Fraction(x)
        v = sum(c * d ** k for k, c in enumerate(KOOP))
        rows.append((x, v))
    return rows


def fmt(v):
    return mp.nstr(v, 20, min_fixed=0, max_fixed=0)


def main():
    with open(os.path.join(HERE, "cnt_kantrowitz.txt"), "w") as fh:
        fh.write("# Classical nucleation (Eqs. 3, 4, 9, 10) and the Kantrowitz factor (Eq. 5) of the paper,\n"
                 "# mpmath at 50 digits (make_phase_change_golden.py).  p = 24 kPa, dry air + vapour with\n"
                 "# p_v = S p_sat,l(T), no condensate; rho_g = vapour density; q_c = 1; theta = 90 deg;\n"
                 "# alpha_crit = lambda_g / (r_crit (1/(1+2 beta Kn) + 3.78 (1-nu) Kn/Pr)), Kn = lbar/(2 r_crit).\n"
                 "# Columns: S T[K] Y_v r_crit[m] dG*/kT ln(J_hom[m^-3 s^-1]) ln(J_het) phi\n")
        for row in cnt_rows():
            fh.write(" ".join(fmt(v) for v in row) + "\n")
    with open(os.path.join(HERE, "young_growth.txt"), "w") as fh:
        fh.write("# Young's growth law (Eq. 16 of the paper; alpha = 11, beta = 0, q_c = 1, Pr = 0.71,\n"
                 "# Kn = lbar/(2 r), lbar = 1.5 mu sqrt(R_g T)/p, Sutherland mu, lambda = mu c_p/Pr),\n"
                 "# mpmath at 50 digits (make_phase_change_golden.py).  Monodisperse population of n per kg\n"
                 "# at radius r in dry air + vapour at 24 kPa; S is the saturation ratio over the phase.\n"
                 "# Ice: rho_s = 917, h_sg, sigma_sv = 0.106, T_sat over ice.\n"
                 "# Columns: phase(l|i) S T[K] r[m] n[1/kg] Y_v G[m/s] Kn\n")
        for row in young_rows():
            fh.write(row[0] + " " + " ".join(fmt(v) for v in row[1:]) + "\n")
    with open(os.path.join(HERE, "koop_2000.txt"), "w") as fh:
        fh.write("# Koop, Luo, Tsias & Peter (2000), Nature 406, 611-614, Eq. (7): homogeneous ice\n"
                 "# nucleation rate coefficient of aqueous droplets, log10(J / cm^-3 s^-1) = -906.7 + 8502 x\n"
                 "# - 26924 x^2 + 29180 x^3 with x = Delta a_w, valid for 0.26 < x < 0.34.  Exact rational\n"
                 "# evaluation of the published coefficients (make_phase_change_golden.py).\n"
                 "# Columns: Delta_a_w log10_J\n")
        for x, v in koop_rows():
            fh.write(f"{x} {fmt(mp.mpf(v.numerator) / v.denominator)}\n")


if __name__ == "__main__":
    main()
