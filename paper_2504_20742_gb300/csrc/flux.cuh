// flux.cuh -- MUSCL/van Leer reconstruction and Roe flux with Harten's entropy fix
// (Sec. 3.2 of Tegethoff & Wheeler, arXiv 2504.20742; the paper's PGIRoe scheme is not
// published in detail, so this is Roe's flux for the frozen ideal mixture with formation
// energies, passive quantities carried by the upwind mass flux).
#pragma once
#include <type_traits>

#include "pair.cuh"
#include "physics.cuh"

namespace ct {

// Half of van Leer's limited slope psi(r) (q_i - q_{i-1}), psi(r) = (r+|r|)/(1+|r|): in its
// harmonic-mean form the slope is 2 dm dp/(dm+dp) when dm and dp share a sign and 0
// otherwise, so the half slope is dm (dp/(dm+dp)) when dm dp > 0.  The quotient lies in
// (0, 1), which keeps the fast FP32 division in range.  (A product that underflows to
// zero gives a zero slope.)
template <class T>
__device__ __forceinline__ T vl_half_slope(T dm, T dp) {
  return dm * dp > T(0) ? dm * tdiv(dp, dm + dp) : T(0);
}
// The same for two fields at once (pair.cuh).  FP32: paired products and the two
// reciprocals, the sign test applied as a select.  FP64: field by field, so that the
// Newton reciprocal (several FP64 instructions, the bottleneck of the FP64 kernels) is
// skipped where the slope is zero.
__device__ __forceinline__ float2 vl_half_slope2(float2 dm, float2 dp) {
  const float2 s = p_add(dm, dp);
  const float2 q = p_mul(dp, p_make(trcp(s.x), trcp(s.y)));
  const float2 hs = p_mul(dm, q);
  const float2 pr = p_mul(dm, dp);
  return p_make(pr.x > 0.0f ? hs.x : 0.0f, pr.y > 0.0f ? hs.y : 0.0f);
}
__device__ __forceinline__ double2 vl_half_slope2(double2 dm, double2 dp) {
  return p_make(vl_half_slope(dm.x, dp.x), vl_half_slope(dm.y, dp.y));
}

// States of a cell's two faces in one direction, lo = a0 - hs and hi = a0 + hs, from the
// cell value a0, its neighbours am (minus side) and a1 (plus side) and the van Leer half
// slope hs above.  FP64: the same values bit for bit, with the decisions taken on the
// integer pipe (the FP64 pipe is the bottleneck of the FP64 kernels).  Three bitwise-equal
// values have zero differences and slope; differences of opposite signs have a product
// <= 0; same-signed differences whose magnitudes lie in [2^-511, 2^511) have a product that
// is positive and normal.  The rest (zeros, tiny or huge values, NaN) take the product test
// itself.  With a zero slope, hi = a0 + 0, which turns -0 into +0.
__device__ __forceinline__ void vl_faces(double am, double a0, double a1, double& lo, double& hi) {
  const long long bm = __double_as_longlong(am), b0 = __double_as_longlong(a0), b1 = __double_as_longlong(a1);
  lo = a0;
  hi = b0 == (long long)0x8000000000000000ULL ? 0.0 : a0;
  if (bm == b0 && b1 == b0) return;
  const double dm = a0 - am, dp = a1 - a0;
  const int hm = __double2hiint(dm), hp = __double2hiint(dp);
  if ((hm ^ hp) < 0) return;
  const unsigned em = ((unsigned)hm >> 20) & 0x7ffu, ep = ((unsigned)hp >> 20) & 0x7ffu;
  if ((em - 0x200u < 0x3feu && ep - 0x200u < 0x3feu) || dm * dp > 0.0) {
    const double hs = dm * tdiv(dp, dm + dp);
    lo = a0 - hs;
    hi = a0 + hs;
  }
}
__device__ __forceinline__ void vl_faces2(double2 am, double2 a0, double2 a1, double2& lo, double2& hi) {
  vl_faces(am.x, a0.x, a1.x, lo.x, hi.x);
  vl_faces(am.y, a0.y, a1.y, lo.y, hi.y);
}
__device__ __forceinline__ void vl_faces2(float2 am, float2 a0, float2 a1, float2& lo, float2& hi) {
  const float2 hs = vl_half_slope2(p_sub(a0, am), p_sub(a1, a0));
  hi = p_add(a0, hs);
  lo = p_sub(a0, hs);
}

// a < b.  FP64 on the integer pipe, through order-preserving keys of the bit patterns: the
// same result for all values but NaN and the pair (-0, +0), which it orders.
template <class T>
__device__ __forceinline__ bool less(T a, T b) {
  return a < b;
}
__device__ __forceinline__ long long order_key(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 ? b : b ^ 0x7fffffffffffffffLL;
}
template <>
__device__ __forceinline__ bool less(double a, double b) {
  return order_key(a) < order_key(b);
}

// Thermodynamics of a reconstructed face state (frozen composition): gamma, total enthalpy,
// formation energy and frozen sound speed squared.  One reciprocal, E = 1/(rho R_g c_v),
// gives T = p c_v E, R_g/c_v = rho R_g^2 E, and H = (c_v + R_g) T + e_f + |u|^2/2.
// Where the state carries no liquid and no ice (the third moments are +-0) the terms of Y_l
// and Y_s drop out exactly (x - 0 = x and fma(0, c, x) = x for x != 0), so that case skips
// them: FP64 tests the moments' bits per state; FP32 takes the short form when the caller
// knows the moments are zero (DRY).
template <class T>
struct FaceThermo {
  T g, H, ef, c2;
};
template <class T, bool BI = false, bool DRY = false>
__device__ __forceinline__ FaceThermo<T> face_thermo(const T* q) {
  T Ya, cv, ef;
  bool zero = DRY;
  if constexpr (std::is_same<T, double>::value) {
    const long long z3 = __double_as_longlong(q[8]) | __double_as_longlong(q[12]) |
                         (BI ? __double_as_longlong(q[17]) : 0LL);
    zero = (z3 << 1) == 0;
  }
  if (zero) {
    Ya = rn_sub(T(1), q[4]);
    cv = rn_fma(q[4], T(k::CVV), rn_mul(Ya, T(k::CVA)));
    ef = rn_mul(q[4], T(k::E0V));
  } else {
    const T Yl = rn_mul(T(k::YL3), BI ? rn_add(q[8], q[17]) : q[8]), Ys = rn_mul(T(k::YS3), q[12]);
    Ya = rn_sub(rn_sub(rn_sub(T(1), q[4]), Yl), Ys);
    cv = rn_fma(Ys, T(k::CS), rn_fma(Yl, T(k::CL), rn_fma(q[4], T(k::CVV), rn_mul(Ya, T(k::CVA)))));
    ef = rn_fma(Ys, T(k::E0S), rn_mul(q[4], T(k::E0V)));
  }
  // the rest with its rounding pinned too, so that the kernels that inline this function
  // all get the same bits whatever their surroundings
  const T Rg = rn_fma(q[4], T(k::RV), rn_mul(Ya, T(k::RA)));
  const T rR = rn_mul(q[0], Rg);
  const T E = trcp(rn_mul(rR, cv));
  const T Tg = rn_mul(rn_mul(q[3], cv), E);
  FaceThermo<T> t;
  t.ef = ef;
  t.g = rn_fma(rn_mul(Rg, rR), E, T(1));
  t.H = rn_fma(T(0.5), rn_fma(q[1], q[1], rn_mul(q[2], q[2])), rn_fma(rn_add(cv, Rg), Tg, t.ef));
  t.c2 = rn_mul(rn_mul(t.g, Rg), Tg);
  return t;
}

// pairs of state fields (one liquid set) that hold only particle moments: (6, 7) .. (10, 11)
__host__ __device__ constexpr bool moment_pair(int k2) { return k2 >= 3 && k2 <= 5; }

// Reconstructed face primitive vector: 0 rho, 1 u, 2 v, 3 p, 4 Y_v, 5..8 ml, 9..12 ms, 13 ns
// (bimodal: 14..17 the second liquid set).  Roe flux in direction DIR (0: normal velocity u,
// 1: normal velocity v) -> F[NFX].
// DRY (FP32): the moment fields of both states are +0.
template <class T, int DIR, int NFX = NF, bool DRY = false>
__device__ __forceinline__ void roe_flux(const T* qL, const T* qR, T* F) {
  constexpr bool BI = NFX == NF_BI;
  const FaceThermo<T> tL = face_thermo<T, BI, DRY>(qL), tR = face_thermo<T, BI, DRY>(qR);
  const T gL = tL.g, gR = tR.g, HL = tL.H, HR = tR.H, efL = tL.ef, efR = tR.ef, c2L = tL.c2, c2R = tR.c2;
  const T unL = DIR == 0 ? qL[1] : qL[2], utL = DIR == 0 ? qL[2] : qL[1];
  const T unR = DIR == 0 ? qR[1] : qR[2], utR = DIR == 0 ? qR[2] : qR[1];
  const T mL = qL[0] * unL, mR = qR[0] * unR;
  // Roe averages.  The weights sqrt(rho_L) / (sqrt(rho_L) + sqrt(rho_R)) and its mirror,
  // multiplied through by sqrt(rho_L), need one root: rt = sqrt(rho_L rho_R), w_L =
  // rho_L / (rho_L + rt), w_R = rt / (rho_L + rt).
  const T rt = m_sqrt(qL[0] * qR[0]);
  const T isum = trcp(qL[0] + rt);
  const T wL = qL[0] * isum, wR = rt * isum;
  const T un = wL * unL + wR * unR;
  const T ut = wL * utL + wR * utR;
  const T H = wL * HL + wR * HR;
  const T ef = wL * efL + wR * efR;
  const T gam = T(0.5) * (gL + gR);
  const T q2 = un * un + ut * ut;
  T c2 = (gam - T(1)) * (H - T(0.5) * q2 - ef);
  const T c2min = T(0.01) * (less(c2L, c2R) ? c2L : c2R);
  c2 = less(c2, c2min) ? c2min : c2;
  const T rc = m_rsqrt(c2);
  const T c = c2 * rc;
  const T ic2 = rc * rc;
  const T dp = qR[3] - qL[3];
  const T dun = unR - unL;
  const T a1 = (dp - rt * c * dun) * T(0.5) * ic2;
  const T a5 = (dp + rt * c * dun) * T(0.5) * ic2;
  const T a2 = (qR[0] - qL[0]) - dp * ic2;
  const T a3 = rt * (utR - utL);
  const T delta = T(0.1) * (m_fabs(un) + c);
  T l1 = m_fabs(un - c), l5 = m_fabs(un + c);
  const T l2 = m_fabs(un);
  if (less(l1, delta)) l1 = fdiv(l1 * l1 + delta * delta, T(2) * delta);
  if (less(l5, delta)) l5 = fdiv(l5 * l5 + delta * delta, T(2) * delta);
  const T w1 = l1 * a1, w2 = l2 * a2, w3 = l2 * a3, w5 = l5 * a5;
  const T D0 = w1 + w2 + w5;
  const T D1 = w1 * (un - c) + w2 * un + w5 * (un + c);
  const T D2 = (w1 + w2 + w5) * ut + w3;
  const T D3 = w1 * (H - un * c) + w2 * T(0.5) * q2 + w3 * ut + w5 * (H + un * c);
  const T fm = T(0.5) * (mL + mR - D0);
  const T fn = T(0.5) * (mL * unL + qL[3] + mR * unR + qR[3] - D1);
  const T ft = T(0.5) * (mL * utL + mR * utR - D2);
  const T fe = T(0.5) * (mL * HL + mR * HR - D3);
  F[0] = fm;
  F[1] = DIR == 0 ? fn : ft;
  F[2] = DIR == 0 ? ft : fn;
  F[3] = fe;
  // passive quantities: the mass flux times the upwind value
  if constexpr (std::is_same<T, double>::value) {
    // FP64: upwind side from the bits of fm (fm >= 0, -0 included), and the moment fields,
    // zero wherever there is no liquid or ice, without multiplications when all are +0 on
    // that side (fm * +0 is a zero with the sign of fm)
    const long long bf = __double_as_longlong(fm);
    const bool up = bf >= 0 || bf == (long long)0x8000000000000000ULL;
    const auto qu = [&](int f) { return up ? qL[f] : qR[f]; };
    F[4] = fm * qu(4);
    F[13] = fm * qu(13);
    long long z = 0;
#pragma unroll
    for (int f = 5; f < NFX; ++f)
      if (f != 13) z |= __double_as_longlong(qu(f));
    if (z == 0) {
      const double s0 = __longlong_as_double(bf & (long long)0x8000000000000000ULL);
#pragma unroll
      for (int f = 5; f < NFX; ++f)
        if (f != 13) F[f] = s0;
    } else {
#pragma unroll
      for (int f = 5; f < NFX; ++f)
        if (f != 13) F[f] = fm * qu(f);
    }
  } else {
    // fields 4.. in pairs; the upwind values selected one by one (a selected pointer would
    // put both face states in local memory).  DRY: the moment pairs (6, 7) .. (10, 11) are
    // +0 on both sides, so no selection is needed
    const bool up = fm >= T(0);
    const auto fm2 = p_make(fm, fm);
#pragma unroll
    for (int k = 2; k < NFX / 2; ++k) {
      const auto v = (DRY && moment_pair(k))
                         ? p_mul(fm2, p_make(T(0), T(0)))
                         : p_mul(fm2, p_make(up ? qL[2 * k] : qR[2 * k], up ? qL[2 * k + 1] : qR[2 * k + 1]));
      F[2 * k] = v.x;
      F[2 * k + 1] = v.y;
    }
  }
}

// ---- viscous and diffusive face fluxes (Sec. 3.1 Eqs. (25)-(26), central differences) ----
// Turbulent viscosity nu_t is a case constant (the Spalart-Allmaras model is out of scope).
// mu_e = mu(T) + rho nu_t, lambda_e = mu c_p / Pr + rho c_p nu_t / Pr_t (Pr_t = 0.9),
// D_v = 2.11e-5 (T/273.15)^1.94 (101325/p) + nu_t/Sc_t, D_p = nu_t/Sc_t (Sc_t = 0.7).
namespace visc {
constexpr double PR_T = 0.9, SC_T = 0.7, DV0 = 2.11e-5;
}
template <class T>
struct Transport {
  T mu_e, lam_e, Dv, Dp;
};
template <class T>
__device__ __forceinline__ T sutherland(T Tg) {
  return T(1.716e-5 * (273.15 + 110.4)) * Tg * m_sqrt(Tg * T(1.0 / 273.15)) * T(1.0 / 273.15) / (Tg + T(110.4));
}
template <class T>
__device__ __forceinline__ Transport<T> transport(T rho, T Tg, T p, T cp, T nu_t) {
  Transport<T> t;
  const T mu = sutherland(Tg);
  t.mu_e = mu + rho * nu_t;
  t.lam_e = cp * (mu * T(1.0 / k::PR) + rho * nu_t * T(1.0 / visc::PR_T));
  t.Dp = nu_t * T(1.0 / visc::SC_T);
  t.Dv = T(visc::DV0 * 101325.0) * m_exp(T(1.94) * m_log(Tg * T(1.0 / 273.15))) / p + t.Dp;
  return t;
}
// temperature and c_p of a cell from its primitive vector (moments scaled per kg)
template <class T>
__device__ __forceinline__ void cell_T_cp(T rho, T p, T Yv, T ml3, T ms3, T& Tg, T& cp) {
  const T Yl = T(k::YL3) * ml3, Ys = T(k::YS3) * ms3;
  const T Ya = T(1) - Yv - Yl - Ys;
  Tg = tdiv(p, rho * (Ya * T(k::RA) + Yv * T(k::RV)));
  cp = Ya * T(k::CPA) + Yv * T(k::CPV) + Yl * T(k::CL) + Ys * T(k::CS);
}

// G (along +n) between the cells on the minus side (a) and the plus side (b), centres 1/ih
// apart; q(f, side) returns primitive f (0 rho, 1 u, 2 v, 3 p, 4 Y_v, 5..12 moments,
// 13 soot, bimodal 14..17 the second liquid set).  The face's total flux is the Roe flux
// minus G.  The energy flux carries conduction, the work mu_e grad(|u|^2/2) and the
// enthalpy of the diffusing water (against dry air).
template <class T, int NFX = NF, class Q>
__device__ __forceinline__ void sub_diffusive_flux(const Q& q, T ih, T nu_t, T* F) {
  constexpr bool BI = NFX == NF_BI;
  T Ta, cpa_, Tb, cpb;
  cell_T_cp(q(0, 0), q(3, 0), q(4, 0), BI ? q(8, 0) + q(17, 0) : q(8, 0), q(12, 0), Ta, cpa_);
  cell_T_cp(q(0, 1), q(3, 1), q(4, 1), BI ? q(8, 1) + q(17, 1) : q(8, 1), q(12, 1), Tb, cpb);
  const T rho = T(0.5) * (q(0, 0) + q(0, 1)), Tf = T(0.5) * (Ta + Tb), pf = T(0.5) * (q(3, 0) + q(3, 1));
  const Transport<T> tr = transport(rho, Tf, pf, T(0.5) * (cpa_ + cpb), nu_t);
  const T ua = q(1, 0), ub = q(1, 1), va = q(2, 0), vb = q(2, 1);
  const T Gu = tr.mu_e * (ub - ua) * ih, Gv = tr.mu_e * (vb - va) * ih;
  const T rDv = rho * tr.Dv * ih, rDp = rho * tr.Dp * ih;
  const T Gy = rDv * (q(4, 1) - q(4, 0));
  F[1] -= Gu;
  F[2] -= Gv;
  F[4] -= Gy;
  T Gl = T(0), Gs = T(0), gl3 = T(0);
#pragma unroll
  for (int f = 5; f < NFX; ++f) {
    const T g = rDp * (q(f, 1) - q(f, 0));
    if (f == 8) { Gl = T(k::YL3) * g; gl3 = g; }
    if (f == 12) Gs = T(k::YS3) * g;
    if (f == 17) Gl = T(k::YL3) * (gl3 + g);
    F[f] -= g;
  }
  const T ka = T(0.5) * (ua * ua + va * va), kb = T(0.5) * (ub * ub + vb * vb);
  const T hva = T(k::CPV - k::CPA) * Tf + T(k::E0V), hla = T(k::CL - k::CPA) * Tf, hsa = T(k::CS - k::CPA) * Tf + T(k::E0S);
  F[3] -= tr.lam_e * (Tb - Ta) * ih + tr.mu_e * (kb - ka) * ih + hva * Gy + hla * Gl + hsa * Gs;
}

// rate of a cell's explicit diffusion limit, 2 nu_max (1/dx^2 + 1/dr^2), and its mu_e
template <class T>
__device__ __forceinline__ T viscous_rate(const Prim<T>& w, T nu_t, T ih2sum, T& mu_e) {
  const T Ya = T(1) - w.Yv - w.Yl - w.Ys;
  const T cp = Ya * T(k::CPA) + w.Yv * T(k::CPV) + w.Yl * T(k::CL) + w.Ys * T(k::CS);
  const Transport<T> tr = transport(w.rho, w.Tg, w.p, cp, nu_t);
  mu_e = tr.mu_e;
  const T irho = trcp(w.rho);
  T nu = tr.mu_e * irho;
  const T kap = tr.lam_e * irho * trcp(w.cv);
  nu = kap > nu ? kap : nu;
  nu = tr.Dv > nu ? tr.Dv : nu;
  nu = tr.Dp > nu ? tr.Dp : nu;
  return T(2) * nu * ih2sum;
}

}  // namespace ct
