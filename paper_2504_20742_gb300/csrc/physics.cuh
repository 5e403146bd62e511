// physics.cuh -- device thermophysics and phase-change source of the contrail step.
//
// Closed forms of Sec. 2.1-2.2 of Tegethoff & Wheeler (arXiv 2504.20742), written for the
// GPU: templated on the state precision T (double or float) with the FP64 islands the
// mixed-precision path keeps (ln S, the nucleation exponent and exp(-dG*/kT)).  Moments are
// handled in scaled radius units (1 um) throughout, so that FP32 stays in range.
#pragma once
#include <type_traits>
#include <cuda_runtime.h>
#include <math.h>

#include "fastmath.cuh"

namespace ct {

constexpr int NF = 14;
// Bimodal liquid (Sec. 2.2: one moment set per nucleation mechanism): fields 14..17 hold
// the droplets of heterogeneous origin, 5..8 those of homogeneous origin.
constexpr int NF_BI = 18;
template <bool BI>
constexpr int nf_of() { return BI ? NF_BI : NF; }
constexpr int NAUX = 11;

// ---- constants (SI) ------------------------------------------------------------------
namespace k {
constexpr double NA = 6.02214076e23;
constexpr double KB = 1.380649e-23;
constexpr double RU = 8.314462618;
constexpr double MW = 0.018015;
constexpr double RV = RU / MW;                 // vapour gas constant
constexpr double RA = 287.05;                  // dry-air pseudo-component
constexpr double CVA = RA / 0.4;               // gamma_air = 1.4
constexpr double CPA = CVA + RA;
constexpr double CPV = 1859.0;
constexpr double CVV = CPV - RV;
constexpr double CL = 4186.0;
constexpr double CS = 2100.0;
constexpr double RHOL = 1000.0;
constexpr double RHOS = 917.0;
constexpr double TREF = 273.15;
constexpr double HLV0 = 2.501e6;               // h_v - h_l at TREF
constexpr double HSL0 = 3.337e5;               // h_l - h_s at TREF
constexpr double E0V = HLV0 - (CPV - CL) * TREF;   // vapour formation energy
constexpr double E0S = (CL - CS) * TREF - HSL0;    // ice formation energy
constexpr double PI = 3.14159265358979323846;
constexpr double FOUR_PI_3 = 4.0 * PI / 3.0;
constexpr double YL3 = FOUR_PI_3 * RHOL * 1e-18;   // Y_l per scaled mu3 (um^3/kg)
constexpr double YS3 = FOUR_PI_3 * RHOS * 1e-18;
constexpr double QC = 1.0;                     // condensation coefficient
constexpr double FTHETA = 0.5;                 // Eq. (9) at theta = 90 deg
constexpr double ALPHA_Y = 11.0, BETA_Y = 0.0; // Eq. (16)
constexpr double PR = 0.71;
constexpr double NS_SITE = 1.0e8;              // Eq. (14)
constexpr double K_IMM = 1.0;                  // s^-1
constexpr double SIGMA_SV = 0.106;
constexpr double MU_MIN = 1.0e-6;
constexpr double LN100 = 4.605170185988091368;   // hPa -> Pa
constexpr double RHOL_OVER_RHOS_CBRT = 1.0293037494292043;   // (1000/917)^(1/3)
}  // namespace k

// ---- precision-dependent arithmetic ------------------------------------------------------
// The FP64 path keeps IEEE division (parity with the CPU oracle); the FP32 path uses the
// fast approximate division (2 ulp), whose error is far below the FP32 state's own rounding.
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
template <class T>
__device__ __forceinline__ T frcp(T a) { return fdiv(T(1), a); }
// Transport arithmetic (primitive recovery, reconstruction, Roe flux): FP64 divisions by
// the Newton reciprocal of fastmath.cuh (a few ulp); the source terms keep IEEE division.
__device__ __forceinline__ float tdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double tdiv(double a, double b) { return a * rcp_nr(b); }
__device__ __forceinline__ float trcp(float a) { return __fdividef(1.0f, a); }
__device__ __forceinline__ double trcp(double a) { return rcp_nr(a); }
// finiteness from the exponent bits (integer pipe, not the FP64 one)
__device__ __forceinline__ bool finite_bits(float x) { return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u; }
__device__ __forceinline__ bool finite_bits(double x) {
  return ((unsigned long long)__double_as_longlong(x) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}
// Explicit precision overloads: a templated call must never promote float to double (the
// FP64 pipe of GB300 is a small fraction of its FP32 rate).
__device__ __forceinline__ float m_log(float x) { return logf(x); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double m_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float m_exp(float x) { return expf(x); }
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
__device__ __forceinline__ float m_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double m_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_cbrt(float x) { return cbrtf(x); }
__device__ __forceinline__ double m_cbrt(double x) { return cbrt(x); }
__device__ __forceinline__ float m_floor(float x) { return floorf(x); }
__device__ __forceinline__ double m_floor(double x) { return floor(x); }
// Sound speed from c^2 for the CFL time step: the FP32 path takes c^2 rsqrt(c^2) (no IEEE
// square root); every kernel that computes a time step uses this one form.
__device__ __forceinline__ float sound_speed(float c2) { return c2 * rsqrtf(c2); }
__device__ __forceinline__ double sound_speed(double c2) { return sqrt(c2); }
__device__ __forceinline__ float m_fabs(float x) { return fabsf(x); }
__device__ __forceinline__ double m_fabs(double x) { return fabs(x); }

// ---- Sonntag (1994) saturation pressures, ln of p in Pa --------------------------------
template <class R>
__device__ __forceinline__ R ln_psat_liq(R T) {
  return R(-6096.9385) / T + R(16.635794 + k::LN100) + T * (R(-2.711193e-2) + T * R(1.673952e-5)) +
         R(2.433502) * m_log(T);
}
template <class R>
__device__ __forceinline__ R ln_psat_ice(R T) {
  return R(-6024.5282) / T + R(24.7219 + k::LN100) + T * (R(1.0613868e-2) + T * R(-1.3198825e-5)) -
         R(0.49382577) * m_log(T);
}
template <class R>
__device__ __forceinline__ R dln_psat_liq(R T) {
  R it = R(1) / T;
  return R(6096.9385) * it * it + R(-2.711193e-2) + R(2.0 * 1.673952e-5) * T + R(2.433502) * it;
}
template <class R>
__device__ __forceinline__ R dln_psat_ice(R T) {
  R it = R(1) / T;
  return R(6024.5282) * it * it + R(1.0613868e-2) - R(2.0 * 1.3198825e-5) * T - R(0.49382577) * it;
}

// Saturation temperature at vapour pressure pv: Newton, Clausius-Clapeyron start, 6 steps.
template <class R, bool ICE>
__device__ __forceinline__ R t_sat(R lnpv) {
  const R h0 = ICE ? R(k::HLV0 + k::HSL0) : R(k::HLV0);
  R T = R(1) / (R(1.0 / k::TREF) - R(k::RV) * (lnpv - R(6.415424237852311)) / h0);  // ln 611.2
#pragma unroll
  for (int it = 0; it < 6; ++it) {
    R f = (ICE ? ln_psat_ice(T) : ln_psat_liq(T)) - lnpv;
    R df = ICE ? dln_psat_ice(T) : dln_psat_liq(T);
    T -= f / df;
  }
  return T;
}

// IAPWS (1994) surface tension of liquid water, N/m.
template <class R>
__device__ __forceinline__ R sigma_liq(R T) {
  R tau = R(1) - T * R(1.0 / 647.096);
  return R(0.2358) * m_exp(R(1.256) * m_log(tau)) * (R(1) - R(0.625) * tau);
}

// Koop et al. (2000): log10 J (cm^-3 s^-1) from Delta a_w, clamped to [0.26, 0.34].
template <class R>
__device__ __forceinline__ R koop_log10(R daw) {
  R d = daw > R(0.34) ? R(0.34) : daw;
  return R(-906.7) + d * (R(8502.0) + d * (R(-26924.0) + d * R(29180.0)));
}

// ---- primitive recovery (Eq. (23), ideal mixture with formation energies) --------------
template <class T>
struct Prim {
  T rho, u, v, p, Tg, Yv, Yl, Ys, ml[4], ms[4], ns, cv, Rg, c2;
  T mh[4];   // bimodal liquid: droplets of heterogeneous origin (set only when BI)
};

// Arithmetic with its rounding pinned (the compiler neither fuses nor splits these), so that
// a function built from them gives the same bits in every kernel it is inlined into.
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return fmaf(a, b, c); }

// Moment fields of the state vector: liquid 5..8, ice 9..12 and, with the bimodal liquid,
// the second liquid set 14..17.
__host__ __device__ constexpr bool is_moment(int f) { return (f >= 5 && f <= 12) || f >= 14; }
// true when every moment field of the NFX-field vector got(f) is +0 or -0 (integer pipe)
template <int NFX, class Get>
__device__ __forceinline__ bool moments_zero(const Get& got) {
  long long z = 0;
#pragma unroll
  for (int f = 0; f < NFX; ++f)
    if (is_moment(f)) z |= __double_as_longlong(double(got(f)));
  return (z << 1) == 0;
}

// BI: the state has the 18 fields of the bimodal liquid; Y_l is the sum of both sets.
// Every operation has its rounding pinned: the primitive variables a kernel stores for the
// next stage are then bit for bit those the next stage would compute itself.  ZERO: the
// moment fields are +-0 (no liquid, no ice), and the terms they enter drop out exactly
// (x - 0 = x, fma(0, c, x) = x for x != 0, and (+-0) / rho keeps the zero's sign), so the
// same bits come with fewer operations.
template <class T, bool BI, bool ZERO>
__device__ __forceinline__ void cons_to_prim_impl(const T* U, Prim<T>& w) {
  const T rho = U[0];
  // rho c_v straight from the conserved partial densities, then one reciprocal serves
  // 1/rho = (rho c_v) X and 1/c_v = rho^2 X, X = 1/(rho rho c_v)
  T rcv;
  if constexpr (ZERO) {
    rcv = rn_fma(U[4], T(k::CVV), rn_mul(rn_sub(rho, U[4]), T(k::CVA)));
  } else {
    const T rYl = rn_mul(T(k::YL3), BI ? rn_add(U[8], U[17]) : U[8]), rYs = rn_mul(T(k::YS3), U[12]);
    const T rYa = rn_sub(rn_sub(rn_sub(rho, U[4]), rYl), rYs);
    rcv = rn_fma(rYs, T(k::CS), rn_fma(rYl, T(k::CL), rn_fma(U[4], T(k::CVV), rn_mul(rYa, T(k::CVA)))));
  }
  const T X = trcp(rn_mul(rho, rcv));
  const T ir = rn_mul(rcv, X);
  w.rho = rho;
  w.u = rn_mul(U[1], ir);
  w.v = rn_mul(U[2], ir);
  w.Yv = rn_mul(U[4], ir);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    w.ml[q] = ZERO ? U[5 + q] : rn_mul(U[5 + q], ir);
    w.ms[q] = ZERO ? U[9 + q] : rn_mul(U[9 + q], ir);
  }
  w.ns = rn_mul(U[13], ir);
  if constexpr (BI) {
#pragma unroll
    for (int q = 0; q < 4; ++q) w.mh[q] = ZERO ? U[14 + q] : rn_mul(U[14 + q], ir);
    w.Yl = rn_mul(T(k::YL3), rn_add(w.ml[3], w.mh[3]));
  } else {
    w.Yl = ZERO ? w.ml[3] : rn_mul(T(k::YL3), w.ml[3]);
  }
  w.Ys = ZERO ? w.ms[3] : rn_mul(T(k::YS3), w.ms[3]);
  const T Ya = ZERO ? rn_sub(T(1), w.Yv) : rn_sub(rn_sub(rn_sub(T(1), w.Yv), w.Yl), w.Ys);
  const T ke = rn_mul(T(0.5), rn_fma(w.u, w.u, rn_mul(w.v, w.v)));
  const T e = rn_fma(U[3], ir, -ke);
  w.cv = rn_mul(rcv, ir);
  const T icv = rn_mul(rn_mul(rho, rho), X);
  w.Tg = ZERO ? rn_mul(rn_fma(-w.Yv, T(k::E0V), e), icv)
              : rn_mul(rn_fma(-w.Ys, T(k::E0S), rn_fma(-w.Yv, T(k::E0V), e)), icv);
  w.Rg = rn_fma(w.Yv, T(k::RV), rn_mul(Ya, T(k::RA)));
  w.p = rn_mul(rn_mul(rho, w.Rg), w.Tg);
  w.c2 = rn_mul(rn_mul(rn_fma(w.Rg, icv, T(1)), w.p), ir);
}
// FP64 takes the shorter form where the moments are zero (the FP64 pipe is the bottleneck
// of the FP64 kernels); FP32 always the full one.
template <class T, bool BI = false>
__device__ __forceinline__ void cons_to_prim(const T* U, Prim<T>& w) {
  if constexpr (std::is_same<T, double>::value) {
    if (moments_zero<nf_of<BI>()>([&](int f) { return U[f]; })) {
      cons_to_prim_impl<T, BI, true>(U, w);
      return;
    }
  }
  cons_to_prim_impl<T, BI, false>(U, w);
}

// Conserved state from (p, T, u, v, Y_v, scaled moments, soot per kg).
template <class T>
__device__ __forceinline__ void prim_to_cons(double p, double Tg, double u, double v, double Yv,
                                             const double* ml, const double* ms, double ns, T* U) {
  const double Yl = k::YL3 * ml[3], Ys = k::YS3 * ms[3];
  const double Ya = 1.0 - Yv - Yl - Ys;
  const double Rg = Ya * k::RA + Yv * k::RV;
  const double rho = p / (Rg * Tg);
  const double cv = Ya * k::CVA + Yv * k::CVV + Yl * k::CL + Ys * k::CS;
  const double e = cv * Tg + Yv * k::E0V + Ys * k::E0S;
  U[0] = T(rho);
  U[1] = T(rho * u);
  U[2] = T(rho * v);
  U[3] = T(rho * (e + 0.5 * (u * u + v * v)));
  U[4] = T(rho * Yv);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    U[5 + q] = T(rho * ml[q]);
    U[9 + q] = T(rho * ms[q]);
  }
  U[13] = T(rho * ns);
}

// ---- phase-change source (Sec. 2.2; Eqs. (1)-(21)) -------------------------------------
struct SrcCase {
  double n_soot_ref;   // exit soot number per m^3 (0: no heterogeneous nucleation)
  double rp2;          // lognormal soot <r_p^2> (m^2)
  int phase_change, freezing;
  int tables;          // water properties from the tables below
  int equilibrium;     // equilibrium phase change instead of the kinetic model
  const double* tab;   // TAB_N x 3 nodes per property (FP64)
  const float* tabf;   // the same in FP32
};

// ---- tabulated water properties (Sec. 3.2: tables before the run, second-order Taylor
// expansion at run time) -----------------------------------------------------------------
// Properties 0 ln p_sat,l, 1 ln p_sat,i, 2 sigma_lg on nodes T_k = 150 K + 0.5 K k,
// k < TAB_N (up to 640 K); each node stores the value, the first derivative and half the
// second derivative of the closed form.  A query expands about the nearest node.
constexpr int TAB_N = 981;
template <class R>
__device__ __forceinline__ R tab_prop(const R* __restrict__ tab, int which, R T, bool der) {
  int kk = (int)m_floor((T - R(150)) * R(2) + R(0.5));
  kk = kk < 0 ? 0 : (kk > TAB_N - 1 ? TAB_N - 1 : kk);
  const R d = T - (R(150) + R(0.5) * R(kk));
  const R* c = tab + ((size_t)which * TAB_N + kk) * 3;
  const R c1 = __ldg(c + 1), c2 = __ldg(c + 2);
  return der ? c1 + R(2) * c2 * d : __ldg(c) + d * (c1 + d * c2);
}
__device__ __forceinline__ const double* tab_of(const SrcCase& sc, double) { return sc.tab; }
__device__ __forceinline__ const float* tab_of(const SrcCase& sc, float) { return sc.tabf; }
template <class R>
__device__ __forceinline__ R prop_lnpl(const SrcCase& sc, R T) {
  return sc.tables ? tab_prop(tab_of(sc, R(0)), 0, T, false) : ln_psat_liq(T);
}
template <class R>
__device__ __forceinline__ R prop_lnpi(const SrcCase& sc, R T) {
  return sc.tables ? tab_prop(tab_of(sc, R(0)), 1, T, false) : ln_psat_ice(T);
}
template <class R>
__device__ __forceinline__ R prop_sigma(const SrcCase& sc, R T) {
  return sc.tables ? tab_prop(tab_of(sc, R(0)), 2, T, false) : sigma_liq(T);
}
// T_sat of reading D with the tabulated curve and its derivative (same start and steps)
template <class R, bool ICE>
__device__ __forceinline__ R prop_tsat(const SrcCase& sc, R lnpv) {
  if (!sc.tables) return t_sat<R, ICE>(lnpv);
  const R h0 = ICE ? R(k::HLV0 + k::HSL0) : R(k::HLV0);
  R T = R(1) / (R(1.0 / k::TREF) - R(k::RV) * (lnpv - R(6.415424237852311)) / h0);
  const R* tab = tab_of(sc, R(0));
#pragma unroll
  for (int it = 0; it < 6; ++it) T -= (tab_prop(tab, ICE ? 1 : 0, T, false) - lnpv) / tab_prop(tab, ICE ? 1 : 0, T, true);
  return T;
}

// Young's growth law, Eq. (16), split as G = cond * D: cond = lambda / den (m/s per K) and
// the driving potential D = Delta T (1 - r_crit/r) (K), with
// Delta T * r_crit written through Delta T / ln S so that S = 1 is regular.
template <class T>
struct Growth {
  T cond, D;
};
template <class T>
__device__ __forceinline__ Growth<T> young_growth(T r, T Tg, T Tsat, T lnS, T sig, T rho_d, T h, T lam,
                                                  T lbar, T gam, T cp) {
  const T Kn = lbar / (T(2) * r);
  const T ih = T(1) / h;
  const T nu = T(k::RV) * Tsat * ih *
               (T(k::ALPHA_Y - 0.5) - T((2.0 - k::QC) / (2.0 * k::QC)) * (gam + T(1)) / (T(2) * gam) * cp * Tsat * ih);
  const T dT = Tsat - Tg;
  const T dT_lnS = m_fabs(lnS) < T(1e-8) ? T(k::RV) * Tg * Tsat * ih : dT / lnS;
  const T dT_rc = dT_lnS * T(2) * sig / (rho_d * T(k::RV) * Tg);
  const T den = rho_d * h * r * (T(1) / (T(1) + T(2 * k::BETA_Y) * Kn) + T(3.78) * (T(1) - nu) * Kn * T(1.0 / k::PR));
  Growth<T> g;
  g.cond = lam / den;
  g.D = dT - dT_rc / r;
  return g;
}

// |dD/dY| of the linearised vapour-condensate exchange at fixed density and energy:
// saturation curve slope R_v Tsat^2/h per ln p_v, latent heating (h - R_v T)/c_v per unit Y.
template <class T>
__device__ __forceinline__ T relax_slope(T Tsat, T Tg, T h, T Yv, T cv) {
  const T a = T(k::RV) * Tsat * Tsat / h;
  return m_fabs(a / Yv + (T(1) - a / Tg) * (h - T(k::RV) * Tg) / cv);
}

// Expensive part of the source (what the surrogate stands in for): the effective nucleation
// rate J/(1+phi) (m^-3 s^-1) and critical radius (um), the raw growth rates G(r20) (um/s) and
// the relaxation rates 1/tau of the linearised vapour exchange (1/s) of both phases.
template <class T>
struct Rates {
  T Jeff, rc_um, Gl, Gs, xl, xs;
  T Jh, Gh, xh;   // bimodal: heterogeneous nucleation, growth and relaxation of the second set
};

// Cheap part of the source, shared by the plain and the surrogate paths: relaxation
// limiter, freezing, moment assembly (Eq. 21), vapour sink (Eqs. 18, 25) and the
// flux-aware limiters of reading J.  U: conserved stage input of the cell; acc (may be
// null): its flux-only residual, so that the limiters act on A = U + dt acc.  BI: the
// bimodal liquid, whose second set (fields 14..17) takes the heterogeneous nucleation
// r.Jh, grows at r.Gh and alone freezes by immersion.
template <class T, bool BI = false>
__device__ __forceinline__ void source_tail(const Prim<T>& w, const T* U, const T* acc, T dt, const SrcCase& sc,
                                            bool pres_l, bool pres_s, double lnSl, double lnSi, Rates<T> r, T* Q,
                                            double* aux, bool pres_h = false) {
  const T Tg = w.Tg, rho = w.rho;
  // growth over the stage: the exponential solution of the linearised exchange
  const T xsum = BI ? dt * (r.xl + r.xh + r.xs) : dt * (r.xl + r.xs);
  if (xsum > T(0)) {
    const T theta = -m_expm1(-xsum) / xsum;
    r.Gl *= theta;
    r.Gs *= theta;
    if (BI) r.Gh *= theta;
  }
  if (aux) { aux[7] = double(r.Gl) * 1e-6; aux[8] = double(r.Gs) * 1e-6; }

  // freezing, Eqs. (12)-(15) (reading H); with the bimodal liquid only droplets of
  // heterogeneous origin carry a soot particle for immersion freezing
  T Nf = T(0), rv = T(0), rf = T(0), Nfh = T(0), rvh = T(0), rfh = T(0);
  if (sc.freezing && (pres_l || (BI && pres_h)) && Tg < T(k::TREF)) {
    const T daw = T(1) - T(m_exp(lnSl - lnSi));   // 1 - p_sat,i / p_sat,l
    T Js = T(0);
    if (daw >= T(0.26)) {
      const T l10 = koop_log10(daw);
      Js = m_exp(l10 * T(2.302585092994045684)) * T(1e6);
      if (aux) aux[9] = double(l10);
    }
    if (pres_l) {
      rv = m_cbrt(w.ml[3] / w.ml[0]);   // um
      const T rvm = rv * T(1e-6);
      T omega;
      if (BI) {   // droplets of homogeneous origin hold no soot
        omega = Js * T(k::FOUR_PI_3) * rvm * rvm * rvm;
      } else {
        T chi = w.ns / w.ml[0];
        chi = chi > T(1) ? T(1) : chi;
        omega = Js * T(k::FOUR_PI_3) * rvm * rvm * rvm + T(k::K_IMM * k::NS_SITE * 4.0 * k::PI * sc.rp2) * chi;
      }
      if (aux) aux[10] = double(omega);
      Nf = w.ml[0] * (-m_expm1(-omega * dt) / dt);   // first-order decay over the stage
      rf = rv * T(k::RHOL_OVER_RHOS_CBRT);
    }
    if (BI && pres_h) {
      rvh = m_cbrt(w.mh[3] / w.mh[0]);
      const T rvm = rvh * T(1e-6);
      T chi = w.ns / w.mh[0];
      chi = chi > T(1) ? T(1) : chi;
      const T omega = Js * T(k::FOUR_PI_3) * rvm * rvm * rvm + T(k::K_IMM * k::NS_SITE * 4.0 * k::PI * sc.rp2) * chi;
      Nfh = w.mh[0] * (-m_expm1(-omega * dt) / dt);
      rfh = rvh * T(k::RHOL_OVER_RHOS_CBRT);
    }
  }

  // moment sources (per kg, scaled units), Eq. (21)
  const T jr = r.Jeff / rho;
  T dml[4], dms[4], dmh[4];
  {
    const T jrh = BI ? r.Jh / rho : T(0);
    T rck = T(1), rvk = T(1), rfk = T(1), rvhk = T(1), rfhk = T(1);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      dml[q] = (q ? T(q) * w.ml[q - 1] * r.Gl : T(0)) + jr * rck - Nf * rvk;
      if (BI) {
        dmh[q] = (q ? T(q) * w.mh[q - 1] * r.Gh : T(0)) + jrh * rck - Nfh * rvhk;
        dms[q] = (q ? T(q) * w.ms[q - 1] * r.Gs : T(0)) + Nf * rfk + Nfh * rfhk;
      } else {
        dms[q] = (q ? T(q) * w.ms[q - 1] * r.Gs : T(0)) + Nf * rfk;
      }
      rck *= r.rc_um;
      rvk *= rv;
      rfk *= rf;
      rvhk *= rvh;
      rfhk *= rfh;
    }
  }
  // limiters on the flux-updated stage state (reading J)
  auto A = [&](int f) { return acc ? U[f] + dt * acc[f] : U[f]; };
  const T ir = T(1) / rho;
  const T idt = T(1) / dt;
  if (A(8) * ir + dt * dml[3] <= T(0)) {
#pragma unroll
    for (int q = 0; q < 4; ++q) dml[q] = -(A(5 + q) * ir) * idt;
  }
  if (BI && A(17) * ir + dt * dmh[3] <= T(0)) {
#pragma unroll
    for (int q = 0; q < 4; ++q) dmh[q] = -(A(14 + q) * ir) * idt;
  }
  if (A(12) * ir + dt * dms[3] <= T(0)) {
#pragma unroll
    for (int q = 0; q < 4; ++q) dms[q] = -(A(9 + q) * ir) * idt;
  }
  T dYv = BI ? -(T(k::YL3) * (dml[3] + dmh[3]) + T(k::YS3) * dms[3]) : -(T(k::YL3) * dml[3] + T(k::YS3) * dms[3]);
  const T av = A(4) * ir;
  if (av + dt * dYv < T(0)) {
    const T th = av > T(0) ? av / (-dt * dYv) : T(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      dml[q] *= th;
      dms[q] *= th;
      if (BI) dmh[q] *= th;
    }
    dYv *= th;
  }
  Q[4] = rho * dYv;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    Q[5 + q] = rho * dml[q];
    Q[9 + q] = rho * dms[q];
    if (BI) Q[14 + q] = rho * dmh[q];
  }
}

// Saturation state of a cell (Eq. 1, FP64): ln S over liquid and ice, ln p_v, populations.
template <class T>
struct Sat {
  double lnSl, lnSi, lnpv;
  bool pres_l, pres_s, active;
  bool pres_h;   // bimodal: second liquid set present
};

template <class T>
__device__ __forceinline__ bool populations(const Prim<T>& w, bool& pres_l, bool& pres_s) {
  pres_l = w.ml[0] > T(k::MU_MIN) && w.ml[1] > T(0) && w.ml[2] > T(0) && w.ml[3] > T(0);
  pres_s = w.ms[0] > T(k::MU_MIN) && w.ms[1] > T(0) && w.ms[2] > T(0) && w.ms[3] > T(0);
  return pres_l || pres_s;
}
template <class T>
__device__ __forceinline__ bool present_h(const Prim<T>& w) {
  return w.mh[0] > T(k::MU_MIN) && w.mh[1] > T(0) && w.mh[2] > T(0) && w.mh[3] > T(0);
}

// FP32 screen: a cell clearly below liquid saturation with no population has an exactly
// zero source; only cells near or above saturation pay for the FP64 island.
template <class T>
__device__ __forceinline__ bool clearly_inactive(const Prim<T>& w) {
  const float Tf = float(w.Tg);
  float pvf = float(w.rho) * float(w.Yv) * float(k::RV) * Tf;
  pvf = pvf < 1e-30f ? 1e-30f : pvf;
  // Sonntag's ln p_sat,l with the fast log and division: their errors (about 1e-5 in ln S
  // here) are far below the margin, and the screen runs in every cell of every stage
  const float lnps = __fdividef(-6096.9385f, Tf) + float(16.635794 + k::LN100) +
                     Tf * (-2.711193e-2f + Tf * 1.673952e-5f) + 2.433502f * __logf(Tf);
  return __logf(pvf) - lnps < -1e-3f;
}

template <class T, bool BI = false>
__device__ __forceinline__ Sat<T> saturation(const Prim<T>& w, const SrcCase& sc) {
  Sat<T> s;
  populations(w, s.pres_l, s.pres_s);
  s.pres_h = BI && present_h(w);
  // Eq. (1) in FP64: ln S = ln p_v - ln p_sat(T)
  double pv = double(w.rho) * double(w.Yv) * k::RV * double(w.Tg);
  pv = pv < 1e-30 ? 1e-30 : pv;
  s.lnpv = m_log(pv);
  s.lnSl = s.lnpv - prop_lnpl<double>(sc, double(w.Tg));
  s.lnSi = s.lnpv - prop_lnpi<double>(sc, double(w.Tg));
  s.active = s.lnSl > 0.0 || s.pres_l || s.pres_s || s.pres_h;
  return s;
}

// Gas-phase properties of a cell for Young's law and the Kantrowitz factor (reading G):
// c_p, gamma, conductivity, mean free path of the gas (dry air and vapour), latent heats.
template <class T>
struct Gas {
  T cp_g, gam_g, lam, lbar, hfg, hsg;
};
template <class T>
__device__ __forceinline__ Gas<T> gas_props(const Prim<T>& w) {
  const T Tg = w.Tg;
  const T Yg = T(1) - w.Yl - w.Ys;
  const T Ya = Yg - w.Yv;
  const T iYg = T(1) / Yg;
  Gas<T> g;
  g.cp_g = (Ya * T(k::CPA) + w.Yv * T(k::CPV)) * iYg;
  const T cv_g = (Ya * T(k::CVA) + w.Yv * T(k::CVV)) * iYg;
  g.gam_g = g.cp_g / cv_g;
  const T Rg_g = (Ya * T(k::RA) + w.Yv * T(k::RV)) * iYg;
  const T mu_g = T(1.716e-5 * (273.15 + 110.4)) * Tg * m_sqrt(Tg * T(1.0 / 273.15)) * T(1.0 / 273.15) / (Tg + T(110.4));
  g.lam = mu_g * g.cp_g * T(1.0 / k::PR);
  g.lbar = T(1.5) * mu_g * m_sqrt(Rg_g * Tg) / w.p;
  g.hfg = T(k::CPV - k::CL) * Tg + T(k::E0V);
  g.hsg = T(k::CPV - k::CS) * Tg + T(k::E0V - k::E0S);
  return g;
}

// Kantrowitz factor phi of Eq. (5), with alpha_crit from Young's heat-transfer law at r_crit
// (reading F); rc, rhov from cnt_rates, Tsat_l the liquid saturation temperature.
template <class T>
__device__ __forceinline__ T kantrowitz_phi(const Prim<T>& w, const Gas<T>& g, double rc, double rhov, T Tsat_l) {
  const T Tg = w.Tg;
  const T rcT = T(rc);
  const T ih = T(1) / g.hfg;
  const T nu = T(k::RV) * Tsat_l * ih *
               (T(k::ALPHA_Y - 0.5) - T(0.5) * (g.gam_g + T(1)) / (T(2) * g.gam_g) * g.cp_g * Tsat_l * ih);
  const T Knc = g.lbar / (T(2) * rcT);
  const T alpha_c = g.lam / (rcT * (T(1) + T(3.78) * (T(1) - nu) * Knc * T(1.0 / k::PR)));
  return T(k::QC) * T(rhov) / alpha_c * m_sqrt(T(k::RV) * Tg * T(1.0 / (2.0 * k::PI))) *
         (g.hfg * g.hfg / (T(k::RV) * Tg * Tg) - g.hfg / Tg);
}

// Classical nucleation, Eqs. (3), (4), (9), (10), with the soot gate of J_het (reading F):
// the Kelvin radius, the vapour density and the two rates, in FP64 (ln S, the barrier and
// its exponential are the FP64 islands of the FP32 path).  Only for ln S_l > 0.  lnJ2 gets
// ln J_hom and ln J_het,eff (-inf without soot).
struct Cnt {
  double rc, rhov, Jhom, Jhet, Jsum;
};
template <class T>
__device__ __forceinline__ Cnt cnt_rates(const Prim<T>& w, double lnSl, const SrcCase& sc, double* lnJ2) {
  const T Tg = w.Tg, rho = w.rho;
  Cnt c;
  const T sig = prop_sigma<T>(sc, Tg);
  const double sigd = double(sig);
  c.rc = 2.0 * sigd / (k::RHOL * k::RV * double(Tg) * lnSl);
  const double dGkT = k::FOUR_PI_3 * sigd * c.rc * c.rc / (k::KB * double(Tg));
  c.rhov = double(rho) * double(w.Yv);
  // ln A = ln q_c + 1/2 ln(2 sigma N_A^3 / (pi M^3)) + 2 ln rho_v - ln rho_l
  const double lnA = 0.5 * m_log(2.0 * sigd) + 0.5 * m_log(k::NA * k::NA * k::NA / (k::PI * k::MW * k::MW * k::MW)) +
                     2.0 * m_log(c.rhov) - m_log(k::RHOL);
  const double lnJhom = lnA - dGkT;
  const double lnJhet = lnA - k::FTHETA * dGkT;
  c.Jhom = m_exp(lnJhom);
  c.Jsum = c.Jhom;
  c.Jhet = 0.0;
  lnJ2[0] = lnJhom;
  const double nsv = double(rho) * double(w.ns);
  if (sc.n_soot_ref > 0.0 && nsv > 0.0) {
    const double gate = nsv / sc.n_soot_ref;
    c.Jhet = m_exp(lnJhet) * gate;
    c.Jsum += c.Jhet;
    lnJ2[1] = lnJhet + m_log(gate);
  }
  return c;
}

// Plain rates, Sec. 2.2.  ext (optional, the surrogate's training targets): 0 ln Jeff,
// 1 ln r_crit/um, 2 G_l raw (um/s), 3 G_s raw, 4 1/tau_l, 5 1/tau_s, 6 ln J_hom,
// 7 ln J_het,eff, 8 ln(1+phi), 9 T_sat,l - T.
template <class T, bool BI = false>
__device__ __forceinline__ Rates<T> plain_rates(const Prim<T>& w, const Sat<T>& st, const SrcCase& sc, double* lnJ2,
                                                double* aux, double* ext) {
  const T Tg = w.Tg;
  Rates<T> r = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
  const Gas<T> gs = gas_props<T>(w);
  const T cp_g = gs.cp_g, gam_g = gs.gam_g, lam = gs.lam, lbar = gs.lbar, hfg = gs.hfg, hsg = gs.hsg;
  const T lnpv_t = T(st.lnpv);
  const double lnSl = st.lnSl, lnSi = st.lnSi;

  // nucleation, Eqs. (3)-(6), (10); soot-gated heterogeneous rate
  T Tsat_l = T(0);
  bool have_tsat_l = false;
  if (lnSl > 0.0) {
    const Cnt c = cnt_rates<T>(w, lnSl, sc, lnJ2);
    const double rc = c.rc, rhov = c.rhov, Jhom = c.Jhom, Jhet = c.Jhet, Jsum = c.Jsum;
    // Eq. (5) with alpha_crit from Young's law at r_crit (reading F)
    Tsat_l = prop_tsat<T, false>(sc, lnpv_t);
    have_tsat_l = true;
    const T phi = kantrowitz_phi<T>(w, gs, rc, rhov, Tsat_l);
    if (BI) {   // one moment set per mechanism
      r.Jeff = T(Jhom) / (T(1) + phi);
      r.Jh = T(Jhet) / (T(1) + phi);
    } else {
      r.Jeff = T(Jsum) / (T(1) + phi);
    }
    r.rc_um = T(rc * 1e6);
    if (aux) { aux[2] = lnJ2[0]; aux[3] = lnJ2[1]; aux[5] = rc; aux[6] = double(phi); }
    if (ext) {
      ext[0] = m_log(Jsum) - m_log(1.0 + double(phi));
      ext[1] = m_log(rc * 1e6);
      ext[6] = lnJ2[0];
      ext[7] = lnJ2[1];
      ext[8] = m_log(1.0 + double(phi));
    }
  }

  // growth at r20, Eqs. (16), (21) -- G in um/s, relaxation rates of reading J
  if (st.pres_l) {
    if (!have_tsat_l) Tsat_l = prop_tsat<T, false>(sc, lnpv_t);
    const T r20 = m_sqrt(w.ml[2] / w.ml[0]) * T(1e-6);
    const Growth<T> g = young_growth<T>(r20, Tg, Tsat_l, T(lnSl), prop_sigma<T>(sc, Tg), T(k::RHOL), hfg, lam, lbar, gam_g, cp_g);
    r.Gl = g.cond * g.D * T(1e6);
    r.xl = T(4.0 * k::PI * k::RHOL * 1e-12) * w.ml[2] * g.cond * relax_slope(Tsat_l, Tg, hfg, w.Yv, w.cv);
  }
  if (BI && st.pres_h) {
    if (!have_tsat_l && !st.pres_l) Tsat_l = prop_tsat<T, false>(sc, lnpv_t);
    const T r20 = m_sqrt(w.mh[2] / w.mh[0]) * T(1e-6);
    const Growth<T> g = young_growth<T>(r20, Tg, Tsat_l, T(lnSl), prop_sigma<T>(sc, Tg), T(k::RHOL), hfg, lam, lbar, gam_g, cp_g);
    r.Gh = g.cond * g.D * T(1e6);
    r.xh = T(4.0 * k::PI * k::RHOL * 1e-12) * w.mh[2] * g.cond * relax_slope(Tsat_l, Tg, hfg, w.Yv, w.cv);
  }
  if (st.pres_s) {
    const T Tsat_i = prop_tsat<T, true>(sc, lnpv_t);
    const T r20 = m_sqrt(w.ms[2] / w.ms[0]) * T(1e-6);
    const Growth<T> g = young_growth<T>(r20, Tg, Tsat_i, T(lnSi), T(k::SIGMA_SV), T(k::RHOS), hsg, lam, lbar, gam_g, cp_g);
    r.Gs = g.cond * g.D * T(1e6);
    r.xs = T(4.0 * k::PI * k::RHOS * 1e-12) * w.ms[2] * g.cond * relax_slope(Tsat_i, Tg, hsg, w.Yv, w.cv);
  }
  if (ext) {
    ext[2] = double(r.Gl);
    ext[3] = double(r.Gs);
    ext[4] = double(r.xl);
    ext[5] = double(r.xs);
    if (!have_tsat_l) Tsat_l = prop_tsat<T, false>(sc, lnpv_t);
    ext[9] = double(Tsat_l - Tg);
  }
  return r;
}

// ---- surrogate inputs and targets ---------------------------------------------------------
constexpr float MLP_G0 = 1.0f;       // um/s, scale of asinh(G/G0)
constexpr float MLP_LNJ_FLOOR = -30.0f;   // J below 1e-13 m^-3 s^-1 is physically zero

// 16 inputs of a cell: ln p, T, the CNT barrier shape 1/max(ln S_l, 1/4)^2 (the barrier of
// Eq. 3 scales as 1/ln^2 S), ln Y_v, ln of the 8 scaled moments, ln soot per m^3,
// ln <r_p^2>/um^2, ln S_l, ln S_i (the last two from the FP64 island).
template <class T>
__device__ __forceinline__ void mlp_features(const Prim<T>& w, const Sat<T>& st, double rp2, float* x) {
  x[0] = logf(float(w.p));
  x[1] = float(w.Tg);
  {
    const float ls = fmaxf(float(st.lnSl), 0.25f);
    x[2] = 1.0f / (ls * ls);
  }
  x[3] = logf(fmaxf(float(w.Yv), 1e-12f));
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    x[4 + q] = logf(fmaxf(float(w.ml[q]), 1e-30f));
    x[8 + q] = logf(fmaxf(float(w.ms[q]), 1e-30f));
  }
  x[12] = logf(fmaxf(float(w.rho) * float(w.ns), 1.0f));
  x[13] = logf(float(rp2 * 1e12) + 1e-30f);
  x[14] = float(st.lnSl);
  x[15] = float(st.lnSi);
}

// Source of one cell (plain method).  w: primitives of the stage input; the limiters keep
// the flux-updated state A = U + dt acc non-negative; Q gets fields 4..12.  aux (optional):
// ln S_l, ln S_i, ln J_hom, ln J_het,eff, active, r_crit, phi, G_l, G_s, Koop log10 J, omega.
// Returns true for an active cell.
// ---- equilibrium phase change (the comparison model of Sec. 4.3) ---------------------------
// The water of the flux-updated stage state is brought to equilibrium with its density,
// velocity, total energy and total water fixed: vapour above saturation over the condensed
// phase condenses, condensate below it evaporates.  Liquid above 235.15 K (homogeneous
// freezing), ice below; monodisperse condensate of radius 1 um.  The temperature solves the
// energy balance by eight Newton steps from the all-vapour temperature; all in FP64.
constexpr double T_FRZ = 235.15;
__device__ __forceinline__ double sat_fraction(const SrcCase& sc, double rho, double T, bool ice, double& dy) {
  const double lnp = ice ? prop_lnpi<double>(sc, T) : prop_lnpl<double>(sc, T);
  const double dlnp = sc.tables ? tab_prop(sc.tab, ice ? 1 : 0, T, true)
                                : (ice ? dln_psat_ice<double>(T) : dln_psat_liq<double>(T));
  const double y = exp(lnp) / (rho * k::RV * T);
  dy = y * (dlnp - 1.0 / T);
  return y;
}
// returns the temperature; sets the vapour and condensate fractions and the phase
static __device__ __noinline__ double equilibrium_split(const SrcCase& sc, double rho, double e, double W, double& Yv,
                                                 double& Yc, bool& ice) {
  const double Ya = 1.0 - W;
  const double Tv = (e - W * k::E0V) / (Ya * k::CVA + W * k::CVV);
  double dy;
  ice = Tv < T_FRZ;
  if (W <= sat_fraction(sc, rho, Tv, ice, dy)) {
    Yv = W;
    Yc = 0.0;
    return Tv;
  }
  for (int pass = 0; pass < 2; ++pass) {
    const bool ic = pass == 1;
    const double cc = ic ? k::CS : k::CL, ec = ic ? k::E0S : 0.0;
    double T = Tv;
    for (int it = 0; it < 8; ++it) {
      const double y = sat_fraction(sc, rho, T, ic, dy);
      const double g = Ya * k::CVA * T + y * (k::CVV * T + k::E0V) + (W - y) * (cc * T + ec) - e;
      const double dg = Ya * k::CVA + y * k::CVV + (W - y) * cc + dy * (k::CVV * T + k::E0V - cc * T - ec);
      T -= g / dg;
    }
    if (ic || T >= T_FRZ) {
      const double y = sat_fraction(sc, rho, T, ic, dy);
      ice = ic;
      if (y >= W) {
        Yv = W;
        Yc = 0.0;
        return Tv;
      }
      Yv = y;
      Yc = W - y;
      return T;
    }
  }
  Yv = W;
  Yc = 0.0;
  return Tv;
}
template <class T>
__device__ __forceinline__ bool equilibrium_source(const T* U, const T* acc, T dt, const SrcCase& sc, T* Q,
                                                   double* aux) {
  double X[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) X[f] = acc ? double(U[f]) + double(dt) * double(acc[f]) : double(U[f]);
  Prim<double> x;
  cons_to_prim<double>(X, x);
  if (aux) {
    double pv = x.rho * x.Yv * k::RV * x.Tg;
    pv = pv < 1e-30 ? 1e-30 : pv;
    aux[0] = log(pv) - prop_lnpl<double>(sc, x.Tg);
    aux[1] = log(pv) - prop_lnpi<double>(sc, x.Tg);
  }
  const double W = x.Yv + x.Yl + x.Ys;
  const double e = x.cv * x.Tg + x.Yv * k::E0V + x.Ys * k::E0S;
  double Yv, Yc;
  bool ice;
  const double Teq = equilibrium_split(sc, x.rho, e, W, Yv, Yc, ice);
  // a condensate below 1e-15 per kg counts as none (rounding residues of the explicit stage)
  const bool had = x.Yl + x.Ys > 1e-15;
  const bool active = Yc > 1e-15 || had;
  if (aux) aux[4] = active ? 1.0 : 0.0;
  if (!active) return false;
  if (aux) aux[5] = Teq;
  const double idt = 1.0 / double(dt);
  const double n = Yc / (ice ? k::YS3 : k::YL3);   // scaled moments of 1 um condensate
  Q[4] = T((x.rho * Yv - X[4]) * idt);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    Q[5 + q] = T(((ice ? 0.0 : x.rho * n) - X[5 + q]) * idt);
    Q[9 + q] = T(((ice ? x.rho * n : 0.0) - X[9 + q]) * idt);
  }
  return true;
}

template <class T, bool BI = false>
__device__ __forceinline__ bool phase_source(const Prim<T>& w, const T* U, const T* acc, T dt, const SrcCase& sc,
                                             T* Q, double* lnJ2, double* aux, double* ext = nullptr) {
#pragma unroll
  for (int f = 4; f < 13; ++f) Q[f] = T(0);
  if (BI) {
#pragma unroll
    for (int f = 14; f < 18; ++f) Q[f] = T(0);
  }
  if (aux) {
#pragma unroll
    for (int a = 0; a < NAUX; ++a) aux[a] = 0.0;
    aux[2] = aux[3] = aux[9] = -INFINITY;
  }
  lnJ2[0] = lnJ2[1] = -INFINITY;
  if (!sc.phase_change) return false;
  if constexpr (!BI) {   // one condensate population: not with the bimodal liquid
    if (sc.equilibrium) return equilibrium_source<T>(U, acc, dt, sc, Q, aux);
  }
  if (!aux && !ext) {
    // the FP32 screen's margin (1e-3 in ln S_l) is far above its rounding error, so a
    // screened cell is inactive in FP64 too: both paths give the same (zero) source
    bool pl, ps;
    if (!populations(w, pl, ps) && !(BI && present_h(w)) && clearly_inactive(w)) return false;
  }
  const Sat<T> st = saturation<T, BI>(w, sc);
  if (aux) { aux[0] = st.lnSl; aux[1] = st.lnSi; aux[4] = st.active ? 1.0 : 0.0; }
  if (!st.active) return false;
  const Rates<T> r = plain_rates<T, BI>(w, st, sc, lnJ2, aux, ext);
  source_tail<T, BI>(w, U, acc, dt, sc, st.pres_l, st.pres_s, st.lnSl, st.lnSi, r, Q, aux, st.pres_h);
  return true;
}

}  // namespace ct
