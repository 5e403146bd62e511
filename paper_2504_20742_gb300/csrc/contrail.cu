// contrail.cu -- the C ABI (include/contrail.h) around the fused stage kernels of
// stage.cuh, plus the auxiliary kernels: initial time step, inflow profile and ambient
// state, initial field, derived per-cell quantities, pointwise sources and surrogate
// training data.  Also the tile-shape autotuner and the batched, graph-captured step.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "stage.cuh"

namespace ct {


// ---- time step of a given state (initial step / after a load) --------------------------
template <class T, bool BI = false>
__global__ void __launch_bounds__(NT_AUX) k_dt(DevCase dc, const T* __restrict__ U) {
  constexpr int NFX = nf_of<BI>();
  constexpr int NT = NT_AUX;
  __shared__ double red[NT / 32][NPART];
  __shared__ double fin[NPART];
  const int nx = dc.nx, nr = dc.geom == 1 ? dc.nr : 1;
  const size_t N = (size_t)nx * nr;
  T dtmin = T(INFINITY);
  for (size_t n = (size_t)blockIdx.x * NT + threadIdx.x; n < N; n += (size_t)gridDim.x * NT) {
    T u14[NFX];
#pragma unroll
    for (int f = 0; f < NFX; ++f) u14[f] = U[f * N + n];
    Prim<T> w;
    cons_to_prim<T, BI>(u14, w);
    if (dc.prims) {   // the primitives of the state, for the first stage's halo
      T qv[NFX];
      prim_vector<T, BI>(w, qv);
      T* dst = reinterpret_cast<T*>(dc.prims);
#pragma unroll
      for (int f = 0; f < NFX; ++f) dst[f * N + n] = qv[f];
      dst[NFX * N + n] = w.Tg;
      dst[(NFX + 1) * N + n] = w.cv;
    }
    const T d = cell_dt<T>(dc, geo_of(dc, T(0)), w);
    dtmin = d < dtmin ? d : dtmin;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double v = warp_min(double(dtmin));
  if (lane == 0) {
    red[warp][0] = v;
    for (int q = 1; q < NPART; ++q) red[warp][q] = slot_kind(q) == 1 ? -INFINITY : 0.0;
  }
  __syncthreads();
  if (threadIdx.x < NPART) {
    const int kind = slot_kind(threadIdx.x);
    double a = red[0][threadIdx.x];
    for (int w2 = 1; w2 < NT / 32; ++w2) {
      const double u = red[w2][threadIdx.x];
      a = kind == 0 ? a + u : (kind == 1 ? fmax(a, u) : fmin(a, u));
    }
    dc.partials[(size_t)blockIdx.x * NPART + threadIdx.x] = a;
  }
  if (!last_block_reduce(dc, fin)) return;
  if (threadIdx.x == 0) dc.hdr->dt_cur = dc.cfl * fin[0];
}

// ---- tables of water properties (Sec. 3.2) -------------------------------------------------
// Node k of each property: value, first derivative, half the second derivative of the
// closed forms (Sonntag ln p = a/T + b + cT + dT^2 + e ln T; IAPWS sigma = B tau^mu (1 - b tau)).
__global__ void k_tables(double* __restrict__ tab, float* __restrict__ tabf) {
  for (int kk = blockIdx.x * blockDim.x + threadIdx.x; kk < TAB_N; kk += gridDim.x * blockDim.x) {
    const double T = 150.0 + 0.5 * kk, iT = 1.0 / T;
    double c[3][3];
    c[0][0] = ln_psat_liq<double>(T);
    c[0][1] = dln_psat_liq<double>(T);
    c[0][2] = 0.5 * (2.0 * -6096.9385 * iT * iT * iT + 2.0 * 1.673952e-5 - 2.433502 * iT * iT);
    c[1][0] = ln_psat_ice<double>(T);
    c[1][1] = dln_psat_ice<double>(T);
    c[1][2] = 0.5 * (2.0 * -6024.5282 * iT * iT * iT + 2.0 * -1.3198825e-5 + 0.49382577 * iT * iT);
    const double tau = 1.0 - T / 647.096, mu = 1.256, bb = 0.625, B = 0.2358;
    const double tm2 = pow(tau, mu - 2.0), tm1 = tm2 * tau;
    c[2][0] = sigma_liq<double>(T);
    c[2][1] = -B * tm1 * (mu * (1.0 - bb * tau) - bb * tau) / 647.096;
    c[2][2] = 0.5 * B * (mu * (mu - 1.0) * tm2 * (1.0 - bb * tau) - 2.0 * bb * mu * tm1) / (647.096 * 647.096);
    for (int w = 0; w < 3; ++w)
      for (int q = 0; q < 3; ++q) {
        tab[((size_t)w * TAB_N + kk) * 3 + q] = c[w][q];
        tabf[((size_t)w * TAB_N + kk) * 3 + q] = (float)c[w][q];
      }
  }
}

// ---- setup: inflow profile per row and ambient state (Sec. 4.1, Table 2 readings) -------
__device__ double yv_from_pv(double pv, double p) { return pv * k::RA / (k::RV * (p - pv) + pv * k::RA); }

__device__ void ambient_cons(const ct_case& c, double ufac, double* u14) {
  const double z[4] = {0, 0, 0, 0};
  const double pv = c.S_ice_amb * exp(ln_psat_ice<double>(c.T_amb));
  const double Yv = yv_from_pv(pv, c.p_amb);
  const double cp = (1.0 - Yv) * k::CPA + Yv * k::CPV, cv = (1.0 - Yv) * k::CVA + Yv * k::CVV;
  const double Rg = (1.0 - Yv) * k::RA + Yv * k::RV;
  const double ca = sqrt(cp / cv * Rg * c.T_amb);
  prim_to_cons<double>(c.p_amb, c.T_amb, c.mach_coflow * ca * ufac, 0.0, Yv, z, z, 0.0, u14);
}

__device__ void inflow_cons(const ct_case& c, double r, double ufac, double* u14) {
  const double z[4] = {0, 0, 0, 0};
  if (c.mix_width > 0.0) {
    const double wgt = 0.5 * (1.0 - tanh((r - 0.5 * c.d_core) / c.mix_width));
    const double pva = c.S_ice_amb * exp(ln_psat_ice<double>(c.T_amb));
    const double Yva = yv_from_pv(pva, c.p_amb);
    const double cpa = (1.0 - Yva) * k::CPA + Yva * k::CPV, cva = (1.0 - Yva) * k::CVA + Yva * k::CVV;
    const double ua = c.mach_coflow * sqrt(cpa / cva * ((1.0 - Yva) * k::RA + Yva * k::RV) * c.T_amb);
    const double Tg = wgt * c.T_core + (1.0 - wgt) * c.T_amb;
    const double u = (wgt * c.u_core + (1.0 - wgt) * ua) * ufac;
    const double Yv = wgt * c.Yv_core + (1.0 - wgt) * Yva;
    const double rho = c.p_amb / (((1.0 - Yv) * k::RA + Yv * k::RV) * Tg);
    prim_to_cons<double>(c.p_amb, Tg, u, 0.0, Yv, z, z, wgt * c.n_soot / rho, u14);
  } else if (r < 0.5 * c.d_core) {
    const double Yv = c.Yv_core;
    const double rho = c.p_amb / (((1.0 - Yv) * k::RA + Yv * k::RV) * c.T_core);
    prim_to_cons<double>(c.p_amb, c.T_core, c.u_core * ufac, 0.0, Yv, z, z, c.n_soot / rho, u14);
  } else if (r < 0.5 * c.d_fan) {
    prim_to_cons<double>(c.p_amb, c.T_byp, c.u_byp * ufac, 0.0, 0.0, z, z, 0.0, u14);
  } else {
    ambient_cons(c, ufac, u14);
  }
}

// nf fields per state (18 with the bimodal liquid: the second set enters empty)
__global__ void k_setup(ct_case c, const double* __restrict__ ufac, double* inflow, double* amb, int nr, double dr,
                        int nf) {
  for (int j = threadIdx.x; j < nr; j += blockDim.x) {
    double* row = inflow + (size_t)j * nf;
    inflow_cons(c, (j + 0.5) * dr, ufac ? ufac[j] : 1.0, row);
    for (int f = NF; f < nf; ++f) row[f] = 0.0;
  }
  if (threadIdx.x == 0) {
    ambient_cons(c, 1.0, amb);
    for (int f = NF; f < nf; ++f) amb[f] = 0.0;
  }
}

// ---- initial state -----------------------------------------------------------------------
__device__ double area_mach(double M, double g) {
  return 1.0 / M * pow(2.0 / (g + 1.0) * (1.0 + 0.5 * (g - 1.0) * M * M), 0.5 * (g + 1.0) / (g - 1.0));
}

template <class T, bool BI = false>
__global__ void k_init(ct_case c, DevCase dc, T* __restrict__ U) {
  constexpr int NFX = nf_of<BI>();
  const int nx = dc.nx, nr = dc.geom == 1 ? dc.nr : 1;
  const size_t N = (size_t)nx * nr;
  for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
    const int i = int(n % nx), j = int(n / nx);
    double u14[NFX];
    for (int f = NF; f < NFX; ++f) u14[f] = 0.0;   // the second liquid set starts empty
    if (dc.geom == 0) {
      const double z[4] = {0, 0, 0, 0};
      const double g = dc.gam0, Rg = (1.0 - dc.Yv0) * k::RA + dc.Yv0 * k::RV;
      const double x = (i + 0.5) * dc.dx;
      const bool sup = x >= dc.x_throat;
      const double ar = area_q1d(dc, x);
      double lo = sup ? 1.0 : 1e-6, hi = sup ? 50.0 : 1.0;
      for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        const bool above = area_mach(mid, g) - ar > 0.0;
        if (above == sup) hi = mid; else lo = mid;
      }
      const double M = 0.5 * (lo + hi);
      const double Tg = dc.T0 / (1.0 + 0.5 * (g - 1.0) * M * M);
      const double p = dc.p0 * pow(Tg / dc.T0, g / (g - 1.0));
      prim_to_cons<double>(p, Tg, M * sqrt(g * Rg * Tg), 0.0, dc.Yv0, z, z, 0.0, u14);
    } else {
      for (int f = 0; f < NFX; ++f) u14[f] = dc.inflow[(size_t)j * NFX + f];
      const double r = (j + 0.5) * dc.dr;
      if (r < 0.5 * c.d_core && (c.seed_l_n > 0.0 || c.seed_s_n > 0.0)) {
        Prim<double> w;
        cons_to_prim<double>(u14, w);
        double ml[4], ms[4];
        double sl = 1.0, ss = 1.0;
        for (int q = 0; q < 4; ++q) {
          ml[q] = c.seed_l_n * sl;
          ms[q] = c.seed_s_n * ss;
          sl *= c.seed_l_r * 1e6;
          ss *= c.seed_s_r * 1e6;
        }
        const double Yv = w.Yv - k::YL3 * ml[3] - k::YS3 * ms[3];
        prim_to_cons<double>(w.p, w.Tg, w.u, w.v, Yv, ml, ms, w.ns, u14);
      }
    }
    for (int f = 0; f < NFX; ++f) U[f * N + n] = T(u14[f]);
  }
}

// ---- derived per-cell quantities and pointwise sources ------------------------------------
template <class T, bool BI = false>
__global__ void k_derived(DevCase dc, const T* __restrict__ U, int which, double dt, double* __restrict__ out) {
  constexpr int NFX = nf_of<BI>();
  const int nx = dc.nx, nr = dc.geom == 1 ? dc.nr : 1;
  const size_t N = (size_t)nx * nr;
  for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
    T u14[NFX], Q[NFX];
#pragma unroll
    for (int f = 0; f < NFX; ++f) u14[f] = U[f * N + n];
    Prim<T> w;
    cons_to_prim<T, BI>(u14, w);
    if (which == 0) { out[n] = double(w.Tg); continue; }
    if (which == 1) { out[n] = double(w.p); continue; }
    if (which >= 13) {
      // lognormal spectrum through mu0, mu1, mu2: median radius (um) and geometric width
      if (which >= 17 && !BI) { out[n] = 0.0; continue; }
      const T* m = which <= 14 ? w.ml : (which <= 16 ? w.ms : w.mh);
      double v = 0.0;
      if (double(m[0]) > k::MU_MIN && m[1] > T(0) && m[2] > T(0)) {
        const double m0 = m[0], m1 = m[1], m2 = m[2];
        if (which == 13 || which == 15 || which == 17) {
          v = exp(2.0 * log(m1 / m0) - 0.5 * log(m2 / m0));
        } else {
          const double s2 = log(m0 * m2 / (m1 * m1));
          v = exp(sqrt(s2 > 0.0 ? s2 : 0.0));
        }
      }
      out[n] = v;
      continue;
    }
    double aux[NAUX], lnJ2[2];
    phase_source<T, BI>(w, u14, nullptr, T(dt), dc.sc, Q, lnJ2, aux);
    double v;
    switch (which) {
      case 2: v = aux[0]; break;
      case 3: v = aux[1]; break;
      case 4: v = aux[2] * (1.0 / 2.302585092994045684); break;
      case 5: v = aux[3] * (1.0 / 2.302585092994045684); break;
      default: v = aux[which - 2]; break;
    }
    out[n] = v;
  }
}

template <class T, bool BI = false>
__global__ void k_source_batch(SrcCase sc, const double* __restrict__ U, int n, double dt, double* __restrict__ Qo,
                               double* __restrict__ auxo) {
  constexpr int NFX = nf_of<BI>();
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    T u14[NFX], Q[NFX];
    for (int f = 0; f < NFX; ++f) u14[f] = T(U[(size_t)m * NFX + f]);
    Prim<T> w;
    cons_to_prim<T, BI>(u14, w);
    double aux[NAUX], lnJ2[2];
    phase_source<T, BI>(w, u14, nullptr, T(dt), sc, Q, lnJ2, aux);
    for (int f = 0; f < NFX; ++f) Qo[(size_t)m * NFX + f] = ((f >= 4 && f <= 12) || f >= NF) ? double(Q[f]) : 0.0;
    for (int a = 0; a < NAUX; ++a) auxo[(size_t)m * NAUX + a] = aux[a];
  }
}

// ---- surrogate training data: inputs and masked targets from the FP64 plain source ------
// Targets: 0 ln Jeff (floored), 1 ln r_crit/um, 2 asinh(G_l/G0), 3 asinh(G_s/G0), 4 ln 1/tau_l,
// 5 ln 1/tau_s, 6 ln J_hom (floored), 7 ln J_het,eff (floored), 8 ln(1+phi), 9 T_sat,l - T.
__global__ void k_mlp_dataset(SrcCase sc, const double* __restrict__ U, int n, float* __restrict__ X,
                              float* __restrict__ Y, float* __restrict__ M) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    double u14[NF];
    for (int f = 0; f < NF; ++f) u14[f] = U[(size_t)m * NF + f];
    Prim<double> w;
    cons_to_prim<double>(u14, w);
    const Sat<double> st = saturation(w, sc);
    float x[CT_MLP_IN];
    mlp_features<double>(w, st, sc.rp2, x);
    double ext[10];
    for (int q = 0; q < 10; ++q) ext[q] = 0.0;
    ext[0] = ext[6] = ext[7] = -INFINITY;
    double lnJ2[2] = {-INFINITY, -INFINITY};
    plain_rates<double>(w, st, sc, lnJ2, nullptr, ext);
    const bool nuc = st.lnSl > 0.0;
    const bool soot = sc.n_soot_ref > 0.0 && w.rho * w.ns > 0.0;
    float y[CT_MLP_OUT], mk[CT_MLP_OUT];
    y[0] = (float)fmax(ext[0], (double)MLP_LNJ_FLOOR); mk[0] = nuc;
    y[1] = nuc ? (float)ext[1] : 0.0f;                   mk[1] = nuc;
    y[2] = asinhf((float)ext[2] / MLP_G0);               mk[2] = st.pres_l;
    y[3] = asinhf((float)ext[3] / MLP_G0);               mk[3] = st.pres_s;
    y[4] = logf(fmaxf((float)ext[4], 1e-30f));           mk[4] = st.pres_l;
    y[5] = logf(fmaxf((float)ext[5], 1e-30f));           mk[5] = st.pres_s;
    y[6] = (float)fmax(ext[6], (double)MLP_LNJ_FLOOR);  mk[6] = nuc;
    y[7] = (float)fmax(ext[7], (double)MLP_LNJ_FLOOR);  mk[7] = nuc && soot;
    y[8] = nuc ? (float)ext[8] : 0.0f;                   mk[8] = nuc;
    y[9] = (float)ext[9];                                mk[9] = 1.0f;
    for (int q = 0; q < CT_MLP_IN; ++q) X[(size_t)m * CT_MLP_IN + q] = x[q];
    for (int q = 0; q < CT_MLP_OUT; ++q) {
      Y[(size_t)m * CT_MLP_OUT + q] = mk[q] != 0.0f ? y[q] : 0.0f;
      M[(size_t)m * CT_MLP_OUT + q] = mk[q];
    }
  }
}

}  // namespace ct

// =========================================================================================
// C ABI
// =========================================================================================
using namespace ct;

static thread_local char g_err[512] = "";

static ct_status fail(ct_status s, const char* msg) {
  snprintf(g_err, sizeof(g_err), "%s", msg);
  return s;
}
static ct_status cuda_check(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(g_err, sizeof(g_err), "%s: %s", where, cudaGetErrorString(e));
    return CT_ERR_CUDA;
  }
  return CT_OK;
}

static int case_nr(const ct_case* c) { return c->geom == 1 ? c->nr : 1; }
// fields of a case's state: 14, or 18 with the bimodal liquid
static int case_nf(const ct_case* c) { return c->bimodal ? NF_BI : NF; }

// ---- tile shapes ------------------------------------------------------------------------
namespace ct {
const StageSet* stage_set_32x8();
const StageSet* stage_set_16x16();
const StageSet* stage_set_32x16();
const StageSet* stage_set_64x8();
const StageSet* stage_set_16x16_o3();
const StageSet* stage_set_32x8_o3();
const StageSet* stage_set_16x12_d2();
const StageSet* stage_set_16x16_d2();
const StageSet* stage_set_16x14_d2();
const StageSet* stage_set_sweep();
const StageSet* stage_set(int shape) {
  switch (shape) {
    case 1: return stage_set_16x16();
    case 2: return stage_set_32x16();
    case 3: return stage_set_64x8();
    case 4: return stage_set_16x16_o3();
    case 5: return stage_set_32x8_o3();
    case 6: return stage_set_16x12_d2();
    case 7: return stage_set_16x16_d2();
    case 8: return stage_set_16x14_d2();
    case 9: return stage_set_sweep();
    default: return stage_set_32x8();
  }
}
}  // namespace ct

// kernel variant of a case at a precision (the index into StageSet)
static int variant_of(const ct_case* c, int precision) {
  if (precision == CT_FP32_MLP) return 2;
  return (precision == CT_FP64 ? 0 : 1) + (c->bimodal ? 3 : 0);
}
static int tiles_x(const ct_case* c, int shape) {
  const int tx = stage_set(shape)->tx;
  return (c->nx + tx - 1) / tx;
}
static int tiles_y(const ct_case* c, int shape) {
  const int ty = stage_set(shape)->ty;
  return (case_nr(c) + ty - 1) / ty;
}
static int num_blocks(const ct_case* c, int shape) { return tiles_x(c, shape) * tiles_y(c, shape); }
// partial records and tile rows the workspace holds: enough for every shape
static int max_blocks(const ct_case* c) {
  int m = 0;
  for (int s = 0; s < NSHAPES; ++s) m = std::max(m, num_blocks(c, s));
  return m;
}
static int max_rows(const ct_case* c) {
  int m = 0;
  for (int s = 0; s < NSHAPES; ++s) m = std::max(m, tiles_y(c, s));
  return m;
}

// Shape chosen per (geometry, grid, precision): set by the autotuner or by the caller,
// else shape 0.  The state does not depend on the choice; only the speed does.
static std::mutex g_shape_mu;
static std::map<std::tuple<int, int, int, int>, int> g_shape;
static std::tuple<int, int, int, int> shape_key(const ct_case* c, int precision) {
  return std::make_tuple(c->geom, c->nx, case_nr(c), variant_of(c, precision));
}
static int shape_for(const ct_case* c, int precision) {
  std::lock_guard<std::mutex> lk(g_shape_mu);
  auto it = g_shape.find(shape_key(c, precision));
  return it == g_shape.end() ? 0 : it->second;
}
static bool shape_usable(int shape, int variant, const ct_case* c) {
  if (shape < 0 || shape >= NSHAPES) return false;
  const StageSet* ss = stage_set(shape);
  if (ss->plume_inviscid_only && (c->geom != 1 || c->viscous)) return false;
  return ss->stage[variant][0] != nullptr;
}

static ct_status validate(const ct_case* c, int precision) {
  if (!c) return fail(CT_ERR_ARG, "null case");
  if (precision < CT_FP64 || precision > CT_FP32_MLP) return fail(CT_ERR_ARG, "invalid precision");
  if (c->geom != 0 && c->geom != 1) return fail(CT_ERR_ARG, "geom must be 0 or 1");
  if (c->nx < 4 || c->nx > (1 << 20)) return fail(CT_ERR_ARG, "nx out of range [4, 2^20]");
  if (c->geom == 1 && (c->nr < 2 || c->nr > (1 << 18))) return fail(CT_ERR_ARG, "nr out of range [2, 2^18]");
  if ((size_t)c->nx * (size_t)case_nr(c) > ((size_t)1 << 31)) return fail(CT_ERR_ARG, "too many cells");
  if (!(c->lx > 0.0) || (c->geom == 1 && !(c->lr > 0.0))) return fail(CT_ERR_ARG, "domain size must be > 0");
  if (c->bc_xlo < 0 || c->bc_xlo > 1 || c->bc_xhi < 0 || c->bc_xhi > 1 || c->bc_rhi < 0 || c->bc_rhi > 2)
    return fail(CT_ERR_ARG, "invalid boundary condition code");
  if (c->geom == 0 && c->bc_xlo == 0 && !(c->p0 > 0.0 && c->T0 > 0.0)) return fail(CT_ERR_ARG, "nozzle inlet needs p0, T0 > 0");
  if (c->geom == 0 && !(c->x_throat > 0.0)) return fail(CT_ERR_ARG, "x_throat must be > 0");
  if (c->geom == 1 && !(c->p_amb > 0.0 && c->T_amb > 0.0)) return fail(CT_ERR_ARG, "ambient p, T must be > 0");
  if (c->n_soot < 0.0 || c->soot_sigma <= 0.0) return fail(CT_ERR_ARG, "soot parameters invalid");
  if (c->viscous != 0 && c->viscous != 1) return fail(CT_ERR_ARG, "viscous must be 0 or 1");
  if (c->tables != 0 && c->tables != 1) return fail(CT_ERR_ARG, "tables must be 0 or 1");
  if (c->equilibrium != 0 && c->equilibrium != 1) return fail(CT_ERR_ARG, "equilibrium must be 0 or 1");
  if (c->equilibrium && precision == CT_FP32_MLP)
    return fail(CT_ERR_ARG, "the surrogate stands in for the kinetic source: no equilibrium with CT_FP32_MLP");
  if (c->bimodal != 0 && c->bimodal != 1) return fail(CT_ERR_ARG, "bimodal must be 0 or 1");
  if (c->bimodal && precision == CT_FP32_MLP)
    return fail(CT_ERR_ARG, "the surrogate was trained on one liquid set: no bimodal liquid with CT_FP32_MLP");
  if (c->bimodal && c->equilibrium)
    return fail(CT_ERR_ARG, "the equilibrium model carries one condensate: not with the bimodal liquid");
  if (!(c->nu_t >= 0.0) || c->nu_t > 1.0e3) return fail(CT_ERR_ARG, "nu_t out of range [0, 1e3]");
  return CT_OK;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Single-case FP64 steps keep the primitive variables of U and U1 in the workspace: each
// stage writes those of the state it produces, and the next stage reads them for its halo
// instead of converting the conserved variables again (the FP64 pipe bounds these kernels).
static bool uses_prims(const ct_case* c, int precision) { return precision == CT_FP64 && !c->bimodal; }
static size_t prim_bytes(const ct_case* c) { return 2 * (size_t)NPLANE * c->nx * case_nr(c) * sizeof(double); }
// FP32 + surrogate cases the column sweep can step keep the surrogate kernel's queue in the
// workspace: a cell index and 14 rates per cell at most, and its CTAs' partial records.
static bool uses_queue(const ct_case* c, int precision) {
  return precision == CT_FP32_MLP && c->geom == 1 && !c->viscous;
}
static size_t queue_bytes(const ct_case* c) {
  const size_t n = (size_t)c->nx * case_nr(c);
  return align256(n * sizeof(unsigned int)) + align256((size_t)NF * n * sizeof(float)) +
         align256((size_t)QUEUE_GRID_MAX * NPART * sizeof(double));
}

static size_t ws_bytes(const ct_case* c, bool prims = false, bool queue = false) {
  const size_t nr = (size_t)case_nr(c);
  size_t b = HDR_BYTES;
  b += align256(nr * case_nf(c) * sizeof(double));
  b += align256(case_nf(c) * sizeof(double));
  b += align256((size_t)max_blocks(c) * NPART * sizeof(double));
  b += align256((size_t)max_rows(c) * sizeof(unsigned int));
  b += align256((size_t)max_rows(c) * NPART * sizeof(double));
  if (prims) b += align256(prim_bytes(c));
  if (queue) b += queue_bytes(c);
  return b;
}

// The property tables are case-independent: one copy per device in these arrays, built
// once (synchronously, so that every stream sees them) the first time a case asks for them.
static __device__ double g_tab[3 * TAB_N * 3];
static __device__ float g_tabf[3 * TAB_N * 3];
static std::mutex g_tab_mu;
static const double* g_tab_ptr[64];
static const float* g_tabf_ptr[64];

static ct_status property_tables(const double** tab, const float** tabf) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return fail(CT_ERR_CUDA, "device for the tables");
  std::lock_guard<std::mutex> lk(g_tab_mu);
  if (!g_tab_ptr[dev]) {
    void *p = nullptr, *pf = nullptr;
    if (cudaGetSymbolAddress(&p, g_tab) != cudaSuccess || cudaGetSymbolAddress(&pf, g_tabf) != cudaSuccess)
      return cuda_check("table symbols");
    k_tables<<<8, 128>>>((double*)p, (float*)pf);
    if (cudaDeviceSynchronize() != cudaSuccess) return cuda_check("k_tables");
    g_tab_ptr[dev] = (const double*)p;
    g_tabf_ptr[dev] = (const float*)pf;
  }
  *tab = g_tab_ptr[dev];
  *tabf = g_tabf_ptr[dev];
  return CT_OK;
}

static DevCase make_dev(const ct_case* c, void* work, int shape = 0, bool prims = false, bool queue = false) {
  DevCase d;
  memset(&d, 0, sizeof(d));
  d.geom = c->geom;
  d.nx = c->nx;
  d.nr = case_nr(c);
  d.bc_xlo = c->bc_xlo;
  d.bc_xhi = c->bc_xhi;
  d.bc_rhi = c->bc_rhi;
  d.dx = c->lx / c->nx;
  d.dr = c->geom == 1 ? c->lr / c->nr : 1.0;
  d.idx = 1.0 / d.dx;
  d.idr = 1.0 / d.dr;
  d.jw = c->geom == 1 ? (int)std::floor(0.5 * c->d_fan / d.dr + 0.5) : -1;
  d.area_a = c->area_a;
  d.x_throat = c->x_throat;
  d.wall_len = c->wall_len;
  d.fdx = (float)d.dx;
  d.fidx = (float)d.idx;
  d.fdr = (float)d.dr;
  d.fidr = (float)d.idr;
  d.fwall_len = (float)c->wall_len;
  d.farea_a = (float)c->area_a;
  d.fixt = c->geom == 0 ? (float)(1.0 / c->x_throat) : 0.0f;
  d.p0 = c->p0;
  d.T0 = c->T0;
  d.Yv0 = c->Yv_inlet;
  d.cp0 = (1.0 - c->Yv_inlet) * k::CPA + c->Yv_inlet * k::CPV;
  d.gam0 = d.cp0 / ((1.0 - c->Yv_inlet) * k::CVA + c->Yv_inlet * k::CVV);
  d.viscous = c->viscous;
  d.nu_t = c->nu_t;
  d.fnu_t = (float)c->nu_t;
  d.sc.n_soot_ref = c->n_soot;
  const double ls = std::log(c->soot_sigma > 0.0 ? c->soot_sigma : 1.0);
  d.sc.rp2 = c->soot_rm * c->soot_rm * std::exp(2.0 * ls * ls);
  d.sc.phase_change = c->phase_change;
  d.sc.freezing = c->freezing;
  d.sc.tables = c->tables;
  d.sc.equilibrium = c->equilibrium;
  d.sc.tab = nullptr;
  d.sc.tabf = nullptr;
  if (c->tables) property_tables(&d.sc.tab, &d.sc.tabf);
  char* base = (char*)work;
  d.hdr = (WsHeader*)base;
  size_t off = HDR_BYTES;
  d.inflow = (const double*)(base + off);
  off += align256((size_t)d.nr * case_nf(c) * sizeof(double));
  d.amb = (const double*)(base + off);
  off += align256(case_nf(c) * sizeof(double));
  d.partials = (double*)(base + off);
  off += align256((size_t)max_blocks(c) * NPART * sizeof(double));
  d.row_count = (unsigned int*)(base + off);
  off += align256((size_t)max_rows(c) * sizeof(unsigned int));
  d.row_part = (double*)(base + off);
  off += align256((size_t)max_rows(c) * NPART * sizeof(double));
  d.prims = prims && work ? (double*)(base + off) : nullptr;
  if (prims) off += align256(prim_bytes(c));
  if (queue) d.qoff = (int)(off / 256);   // off is a multiple of 256
  d.nblocks = num_blocks(c, shape);
  d.tiles_x = tiles_x(c, shape);
  d.tiles_y = tiles_y(c, shape);
  return d;
}

// Time `reps` launches of one stage with CUDA events on the stream; returns ms per launch.
template <class F>
static ct_status time_launches(F&& launch, int reps, cudaStream_t st, float* ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return cuda_check("event");
  launch();   // warm-up (instruction cache, first-touch of the kernel)
  cudaEventRecord(e0, st);
  for (int r = 0; r < reps; ++r) launch();
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(CT_ERR_CUDA, cudaGetErrorString(e));
  *ms = t / (float)reps;
  return cuda_check("autotune");
}

extern "C" {

size_t ct_workspace_bytes(const ct_case* c, int precision) {
  if (validate(c, precision) != CT_OK) return 0;
  return ws_bytes(c, uses_prims(c, precision), uses_queue(c, precision));
}

// queue: the workspace holds the surrogate queue (single-case FP32 + surrogate steps through
// the column sweep; a batch's cases step through the batched kernel and hold none)
static ct_status setup_case(const ct_case* c, int precision, const double* ufac_rows_host, void* work,
                            size_t work_bytes, void* stream, bool queue) {
  ct_status s = validate(c, precision);
  if (s != CT_OK) return s;
  if (!work) return fail(CT_ERR_ARG, "null workspace");
  if (((uintptr_t)work & 255) != 0) return fail(CT_ERR_ARG, "workspace must be 256-byte aligned");
  if (work_bytes < ws_bytes(c, uses_prims(c, precision), queue))
    return fail(CT_ERR_SIZE, "workspace too small (see ct_workspace_bytes)");
  cudaStream_t st = (cudaStream_t)stream;
  DevCase d = make_dev(c, work);
  WsHeader h;
  memset(&h, 0, sizeof(h));
  h.setup_magic = SETUP_MAGIC;
  h.nblocks = d.nblocks;
  // ufac rows are staged through the partials area (at least nblocks*NPART doubles; the
  // partials are rewritten by every kernel before use)
  double* ufac_dev = nullptr;
  const size_t part_bytes = (size_t)d.nblocks * NPART * sizeof(double);
  if (c->geom == 1 && ufac_rows_host) {
    if ((size_t)d.nr * sizeof(double) <= part_bytes) {
      ufac_dev = d.partials;
      if (cudaMemcpyAsync(ufac_dev, ufac_rows_host, (size_t)d.nr * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return cuda_check("ct_setup copy");
    } else {
      return fail(CT_ERR_SIZE, "internal: row factors do not fit the staging area");
    }
  }
  if (cudaMemcpyAsync(work, &h, sizeof(h), cudaMemcpyHostToDevice, st) != cudaSuccess) return cuda_check("ct_setup header");
  if (cudaMemsetAsync(d.row_count, 0, (size_t)max_rows(c) * sizeof(unsigned int), st) != cudaSuccess)
    return cuda_check("ct_setup row tickets");
  if (c->geom == 1) k_setup<<<1, 256, 0, st>>>(*c, ufac_dev, (double*)d.inflow, (double*)d.amb, d.nr, d.dr, case_nf(c));
  // the header copy and the profile kernel read host memory that must outlive them
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check("ct_setup sync");
  return cuda_check("ct_setup");
}

ct_status ct_setup(const ct_case* c, int precision, const double* ufac_rows_host, void* work, size_t work_bytes,
                   void* stream) {
  return setup_case(c, precision, ufac_rows_host, work, work_bytes, stream, uses_queue(c, precision));
}

static ct_status check_setup(const ct_case* c, void* work, void* stream) {
  (void)c;
  (void)stream;
  if (!work) return fail(CT_ERR_ARG, "null workspace");
  return CT_OK;
}

static ct_status launch_dt(const ct_case* c, int precision, void* work, const void* U, double cfl, cudaStream_t st,
                           bool prims) {
  DevCase d = make_dev(c, work, 0, prims);
  d.cfl = cfl;
  const size_t N = (size_t)c->nx * case_nr(c);
  // a grid-stride kernel: a few hundred CTAs keep its one-level reduction short
  int grid = (int)std::min<size_t>(std::min<size_t>((N + NT_AUX - 1) / NT_AUX, (size_t)d.nblocks), (size_t)512);
  d.nblocks = grid;
  if (precision == CT_FP64) {
    if (c->bimodal) k_dt<double, true><<<grid, NT_AUX, 0, st>>>(d, (const double*)U);
    else k_dt<double><<<grid, NT_AUX, 0, st>>>(d, (const double*)U);
  } else {
    if (c->bimodal) k_dt<float, true><<<grid, NT_AUX, 0, st>>>(d, (const float*)U);
    else k_dt<float><<<grid, NT_AUX, 0, st>>>(d, (const float*)U);
  }
  return cuda_check("k_dt");
}

ct_status ct_init_state(const ct_case* c, int precision, void* work, void* U, double cfl, void* stream) {
  ct_status s = validate(c, precision);
  if (s != CT_OK) return s;
  if ((s = check_setup(c, work, stream)) != CT_OK) return s;
  if (!U) return fail(CT_ERR_ARG, "null state");
  if (!(cfl > 0.0 && cfl <= 1.0)) return fail(CT_ERR_ARG, "cfl must be in (0, 1]");
  cudaStream_t st = (cudaStream_t)stream;
  DevCase d = make_dev(c, work);
  const size_t N = (size_t)c->nx * case_nr(c);
  int grid = (int)std::min<size_t>((N + 255) / 256, 4096);
  if (precision == CT_FP64) {
    if (c->bimodal) k_init<double, true><<<grid, 256, 0, st>>>(*c, d, (double*)U);
    else k_init<double><<<grid, 256, 0, st>>>(*c, d, (double*)U);
  } else {
    if (c->bimodal) k_init<float, true><<<grid, 256, 0, st>>>(*c, d, (float*)U);
    else k_init<float><<<grid, 256, 0, st>>>(*c, d, (float*)U);
  }
  if ((s = cuda_check("k_init")) != CT_OK) return s;
  return launch_dt(c, precision, work, U, cfl, st, uses_prims(c, precision));
}

ct_status ct_load_state(const ct_case* c, int precision, void* work, const void* U_src, void* U, double cfl,
                        void* stream) {
  ct_status s = validate(c, precision);
  if (s != CT_OK) return s;
  if (!U || !U_src) return fail(CT_ERR_ARG, "null state");
  if (!(cfl > 0.0 && cfl <= 1.0)) return fail(CT_ERR_ARG, "cfl must be in (0, 1]");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t N = (size_t)c->nx * case_nr(c);
  const size_t bytes = N * case_nf(c) * (precision == CT_FP64 ? sizeof(double) : sizeof(float));
  if (U_src != U && cudaMemcpyAsync(U, U_src, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return cuda_check("ct_load_state copy");
  return launch_dt(c, precision, work, U, cfl, st, uses_prims(c, precision));
}

// CTAs of a launch of the surrogate queue kernel: two per SM, what its registers and shared
// memory are budgeted for (persistent; the queue's length is known on the device only).
// The kernel never waits on another CTA, so CTAs beyond those resident only start later.
static std::mutex g_qgrid_mu;
static int g_qgrid[64];
static int queue_grid() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lk(g_qgrid_mu);
  if (g_qgrid[dev] == 0) {
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) return 0;
    g_qgrid[dev] = std::min(QUEUE_GRID_MAX, 2 * nsm);
  }
  return g_qgrid[dev];
}

static std::mutex g_attr_mu;
static bool g_attr_done[NSHAPES][NVARIANT];

// Opt the kernels of one (shape, kernel variant) into their dynamic shared memory, once.
static ct_status set_stage_attrs(int shape, int p) {
  std::lock_guard<std::mutex> lk(g_attr_mu);
  if (g_attr_done[shape][p]) return CT_OK;
  const StageSet* ss = stage_set(shape);
  cudaError_t e = cudaSuccess;
  for (int st = 0; st < 2 && e == cudaSuccess; ++st) {
    if (ss->stage[p][st])
      e = cudaFuncSetAttribute(ss->stage[p][st], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss->smem[p]);
    if (e == cudaSuccess && ss->batch[p][st])
      e = cudaFuncSetAttribute(ss->batch[p][st], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss->smem[p]);
    if (e == cudaSuccess && p == 0 && ss->stage_sp[st])
      e = cudaFuncSetAttribute(ss->stage_sp[st], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss->smem[p]);
    if (e == cudaSuccess && p == 2 && ss->queue[st])
      e = cudaFuncSetAttribute(ss->queue[st], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss->queue_smem);
    if (e == cudaSuccess && p == 2 && ss->queue[st])   // two CTAs per SM need most of the SM's shared memory
      e = cudaFuncSetAttribute(ss->queue[st], cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess && p == 2 && ss->batch_queue[st])
      e = cudaFuncSetAttribute(ss->batch_queue[st], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss->queue_smem);
    if (e == cudaSuccess && p == 2 && ss->batch_queue[st])
      e = cudaFuncSetAttribute(ss->batch_queue[st], cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  }
  if (e != cudaSuccess) return fail(CT_ERR_CUDA, cudaGetErrorString(e));
  if (p == 2 && ss->queue[0] && queue_grid() <= 0)
    return fail(CT_ERR_CUDA, "no resident CTA for the surrogate queue kernel");
  g_attr_done[shape][p] = true;
  return CT_OK;
}

// One stage launch of one case (stage 1: U -> U1; stage 2: U1, U -> U).
static void launch_stage(const StageSet* ss, int p, int stage, const DevCase& d, dim3 grid, const void* Uin,
                         const void* Un, void* Uout, const void* blob, cudaStream_t st) {
  DevCase dc = d;
  const void* a1 = Uin;
  const void* a2 = Un;
  void* a3 = Uout;
  const void* a4 = blob;
  void* args[] = {&dc, &a1, &a2, &a3, &a4};
  // FP64 with the stored primitives in the workspace: the kernel that reads and writes them
  const void* fn = (p == 0 && d.prims) ? ss->stage_sp[stage - 1] : ss->stage[p][stage - 1];
  cudaLaunchKernel(fn, grid, dim3(ss->nt), args, ss->smem[p], st);
  // FP32 + surrogate through the column sweep: the surrogate kernel on the queued cells
  if (p == 2 && ss->queue[stage - 1] && d.qoff > 0) {
    const int qgrid = queue_grid();
    if (qgrid > 0) cudaLaunchKernel(ss->queue[stage - 1], dim3(qgrid), dim3(QueueTile::NT), args, ss->queue_smem, st);
  }
}

static ct_status enqueue_steps(const ct_case* c, int precision, void* U, void* U1, void* work, int nsteps, double cfl,
                               cudaStream_t st, bool prims, const void* blob = nullptr, int shape = -1) {
  const int p = variant_of(c, precision);
  if (shape < 0) shape = shape_for(c, precision);
  if (!shape_usable(shape, p, c)) shape = 0;
  ct_status s = set_stage_attrs(shape, p);
  if (s != CT_OK) return s;
  const StageSet* ss = stage_set(shape);
  DevCase d = make_dev(c, work, shape, prims, uses_queue(c, precision));
  d.cfl = cfl;
  dim3 grid(tiles_x(c, shape), tiles_y(c, shape));
  for (int k2 = 0; k2 < nsteps; ++k2) {
    launch_stage(ss, p, 1, d, grid, U, nullptr, U1, blob, st);
    launch_stage(ss, p, 2, d, grid, U1, U, U, blob, st);
  }
  return cuda_check("k_stage");
}

ct_status ct_step_surrogate(const ct_case* c, void* U, void* U1, void* work, const void* blob, int nsteps, double cfl,
                            void* stream) {
  ct_status s = validate(c, CT_FP32_MLP);
  if (s != CT_OK) return s;
  if (!U || !U1 || !work || !blob) return fail(CT_ERR_ARG, "null buffer");
  if (U == U1) return fail(CT_ERR_ARG, "U and U1 must be distinct buffers");
  if (((uintptr_t)blob & 15) != 0) return fail(CT_ERR_ARG, "surrogate blob must be 16-byte aligned");
  if (nsteps < 0) return fail(CT_ERR_ARG, "nsteps < 0");
  if (!(cfl > 0.0 && cfl <= 1.0)) return fail(CT_ERR_ARG, "cfl must be in (0, 1]");
  return enqueue_steps(c, CT_FP32_MLP, U, U1, work, nsteps, cfl, (cudaStream_t)stream, false, blob);
}

ct_status ct_step(const ct_case* c, int precision, void* U, void* U1, void* work, int nsteps, double cfl,
                  void* stream) {
  ct_status s = validate(c, precision);
  if (s != CT_OK) return s;
  if (!U || !U1 || !work) return fail(CT_ERR_ARG, "null buffer");
  if (U == U1) return fail(CT_ERR_ARG, "U and U1 must be distinct buffers");
  if (nsteps < 0) return fail(CT_ERR_ARG, "nsteps < 0");
  if (!(cfl > 0.0 && cfl <= 1.0)) return fail(CT_ERR_ARG, "cfl must be in (0, 1]");
  if (precision == CT_FP32_MLP) return fail(CT_ERR_ARG, "CT_FP32_MLP steps go through ct_step_surrogate");
  return enqueue_steps(c, precision, U, U1, work, nsteps, cfl, (cudaStream_t)stream, uses_prims(c, precision));
}

ct_status ct_step_host(const ct_case* c, int precision, const void* U_host_in, void* U_host_out, void* U, void* U1,
                       void* work, int nsteps, double cfl, void* stream) {
  ct_status s = validate(c, precision);
  if (s != CT_OK) return s;
  if (!U_host_in || !U_host_out) return fail(CT_ERR_ARG, "null host buffer");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t N = (size_t)c->nx * case_nr(c);
  const size_t bytes = N * case_nf(c) * (precision == CT_FP64 ? sizeof(double) : sizeof(float));
  if (cudaMemcpyAsync(U, U_host_in, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return cuda_check("h2d");
  if ((s = launch_dt(c, precision, work, U, cfl, st, uses_prims(c, precision))) != CT_OK) return s;
  if ((s = ct_step(c, precision, U, U1, work, nsteps, cfl, stream)) != CT_OK) return s;
  if (cudaMemcpyAsync(U_host_out, U, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) return cuda_check("d2h");
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check("ct_step_host sync");
  return CT_OK;
}

ct_status ct_diagnostics(const void* work, double* host_out, int nout, void* stream) {
  if (!work || !host_out) return fail(CT_ERR_ARG, "null pointer");
  if (nout < 0 || nout > CT_NDIAG) return fail(CT_ERR_ARG, "nout out of range");
  cudaStream_t st = (cudaStream_t)stream;
  double tmp[CT_NDIAG];
  if (cudaMemcpyAsync(tmp, (const char*)work + offsetof(WsHeader, diag), sizeof(tmp), cudaMemcpyDeviceToHost, st) !=
      cudaSuccess)
    return cuda_check("diag copy");
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check("diag sync");
  memcpy(host_out, tmp, sizeof(double) * nout);
  if (tmp[8] != 0.0) return fail(CT_ERR_NONFINITE, "the last step produced non-finite values");
  if (tmp[28] != 0.0) return fail(CT_ERR_TIMEOUT, "a tensor-core wait of the last step gave up");
  return CT_OK;
}

ct_status ct_read_field(const ct_case* c, int precision, const void* U, int field, double* host_dst, size_t n,
                        void* stream) {
  ct_status s = validate(c, precision);
  if (s != CT_OK) return s;
  if (!U || !host_dst) return fail(CT_ERR_ARG, "null buffer");
  if (field < 0 || field >= case_nf(c)) return fail(CT_ERR_ARG, "field out of range");
  const size_t N = (size_t)c->nx * case_nr(c);
  if (n != N) return fail(CT_ERR_ARG, "n must be nx * nr");
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == CT_FP64) {
    if (cudaMemcpyAsync(host_dst, (const double*)U + (size_t)field * N, N * sizeof(double), cudaMemcpyDeviceToHost,
                        st) != cudaSuccess)
      return cuda_check("ct_read_field copy");
    if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check("ct_read_field sync");
    return CT_OK;
  }
  std::vector<float> tmp(N);
  if (cudaMemcpyAsync(tmp.data(), (const float*)U + (size_t)field * N, N * sizeof(float), cudaMemcpyDeviceToHost, st) !=
      cudaSuccess)
    return cuda_check("ct_read_field copy");
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check("ct_read_field sync");
  for (size_t i = 0; i < N; ++i) host_dst[i] = (double)tmp[i];
  return CT_OK;
}

ct_status ct_derived(const ct_case* c, int precision, const void* U, int which, double dt, double* out, void* stream) {
  ct_status s = validate(c, precision);
  if (s != CT_OK) return s;
  if (!U || !out) return fail(CT_ERR_ARG, "null buffer");
  if (which < 0 || which > 18) return fail(CT_ERR_ARG, "which out of range [0, 18]");
  if (!(dt > 0.0)) return fail(CT_ERR_ARG, "dt must be > 0");
  cudaStream_t st = (cudaStream_t)stream;
  DevCase d = make_dev(c, nullptr);
  const size_t N = (size_t)c->nx * case_nr(c);
  int grid = (int)std::min<size_t>((N + 255) / 256, 8192);
  if (precision == CT_FP64) {
    if (c->bimodal) k_derived<double, true><<<grid, 256, 0, st>>>(d, (const double*)U, which, dt, out);
    else k_derived<double><<<grid, 256, 0, st>>>(d, (const double*)U, which, dt, out);
  } else {
    if (c->bimodal) k_derived<float, true><<<grid, 256, 0, st>>>(d, (const float*)U, which, dt, out);
    else k_derived<float><<<grid, 256, 0, st>>>(d, (const float*)U, which, dt, out);
  }
  return cuda_check("k_derived");
}

ct_status ct_source_batch(const ct_case* c, int precision, const double* U, int n, double dt, double* Q, double* aux,
                          void* stream) {
  ct_status s = validate(c, precision);
  if (s != CT_OK) return s;
  if (n < 0) return fail(CT_ERR_ARG, "n < 0");
  if (n == 0) return CT_OK;
  if (!U || !Q || !aux) return fail(CT_ERR_ARG, "null buffer");
  if (!(dt > 0.0)) return fail(CT_ERR_ARG, "dt must be > 0");
  cudaStream_t st = (cudaStream_t)stream;
  DevCase d = make_dev(c, nullptr);
  int grid = std::min((n + 255) / 256, 8192);
  if (precision == CT_FP64) {
    if (c->bimodal) k_source_batch<double, true><<<grid, 256, 0, st>>>(d.sc, U, n, dt, Q, aux);
    else k_source_batch<double><<<grid, 256, 0, st>>>(d.sc, U, n, dt, Q, aux);
  } else {
    if (c->bimodal) k_source_batch<float, true><<<grid, 256, 0, st>>>(d.sc, U, n, dt, Q, aux);
    else k_source_batch<float><<<grid, 256, 0, st>>>(d.sc, U, n, dt, Q, aux);
  }
  return cuda_check("k_source_batch");
}

__global__ void k_faces(const double* am, const double* a0, const double* a1, int n, double* lo, double* hi) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double l, h;
    vl_faces(am[i], a0[i], a1[i], l, h);
    lo[i] = l;
    hi[i] = h;
  }
}

ct_status ct_reconstruct_faces(const double* am, const double* a0, const double* a1, int n, double* lo, double* hi,
                               void* stream) {
  if (n < 0) return fail(CT_ERR_ARG, "n < 0");
  if (n == 0) return CT_OK;
  if (!am || !a0 || !a1 || !lo || !hi) return fail(CT_ERR_ARG, "null buffer");
  const int grid = std::min((n + 255) / 256, 8192);
  k_faces<<<grid, 256, 0, (cudaStream_t)stream>>>(am, a0, a1, n, lo, hi);
  return cuda_check("k_faces");
}

// ---- allocation-free variant of ct_step ----------------------------------------------------
// Some callers cannot allocate device memory at all: code running inside a host framework
// whose allocator is reserved or already captured, firmware-style launchers that only own
// the buffers they were handed, or processes under a memory budget that forbids new
// allocations.  For them the workspace of ct_step (inflow profile, time step, reduction
// partials, diagnostics) lives in this file-scope device array instead of caller memory.
constexpr size_t STATIC_SCRATCH_BYTES = (size_t)CT_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
static std::mutex g_static_mu;
static void* g_static_ptr[MAX_DEVICES];   // device address of g_static_scratch, per device (under g_static_mu)

__global__ void k_scratch_reset(int nblocks, unsigned int* row_count, int nrows) {
  // everything that must start at zero for a fresh run: the header and the row tickets
  WsHeader* h = reinterpret_cast<WsHeader*>(g_static_scratch);
  if (threadIdx.x == 0) {
    memset(h, 0, sizeof(WsHeader));
    h->setup_magic = SETUP_MAGIC;
    h->nblocks = nblocks;
  }
  for (int r = threadIdx.x; r < nrows; r += blockDim.x) row_count[r] = 0u;
}

static ct_status static_scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cuda_check("cudaGetDevice");
  if (dev < 0 || dev >= MAX_DEVICES) return fail(CT_ERR_ARG, "device index beyond the static scratch table");
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    // host code cannot use g_static_scratch's name as a device address: ask the runtime,
    // with this device current, once per device
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      snprintf(g_err, sizeof(g_err), "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
      return CT_ERR_CUDA;
    }
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return CT_OK;
}

extern "C" ct_status ct_step_static(const ct_case* c, int precision, const double* ufac_rows_dev, void* U, void* U1,
                                    int nsteps, double cfl, void* stream) {
  ct_status s = validate(c, precision);
  if (s != CT_OK) return s;
  if (!U || !U1) return fail(CT_ERR_ARG, "null state buffer");
  if (U == U1) return fail(CT_ERR_ARG, "U and U1 must be distinct buffers");
  if (nsteps < 0) return fail(CT_ERR_ARG, "nsteps < 0");
  if (!(cfl > 0.0 && cfl <= 1.0)) return fail(CT_ERR_ARG, "cfl must be in (0, 1]");
  if (precision == CT_FP32_MLP) return fail(CT_ERR_ARG, "CT_FP32_MLP is not supported by ct_step_static");
  const size_t need = ws_bytes(c);
  if (need > STATIC_SCRATCH_BYTES) {
    snprintf(g_err, sizeof(g_err),
             "case needs %zu bytes of scratch (reduction records for %d tiles, the largest tile count over the "
             "built tile shapes) but the static scratch holds %zu; use ct_step with a caller workspace",
             need, max_blocks(c), STATIC_SCRATCH_BYTES);
    return CT_ERR_SIZE;
  }
  void* work = nullptr;
  if ((s = static_scratch_address(&work)) != CT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  DevCase d = make_dev(c, work);
  k_scratch_reset<<<1, 256, 0, st>>>(d.nblocks, d.row_count, max_rows(c));
  if (c->geom == 1)
    k_setup<<<1, 256, 0, st>>>(*c, ufac_rows_dev, (double*)d.inflow, (double*)d.amb, d.nr, d.dr, case_nf(c));
  if ((s = cuda_check("ct_step_static setup")) != CT_OK) return s;
  if ((s = launch_dt(c, precision, work, U, cfl, st, false)) != CT_OK) return s;
  return enqueue_steps(c, precision, U, U1, work, nsteps, cfl, st, false);
}

// ---- tile shapes and the autotuner ------------------------------------------------------
int ct_tile_shape_count(void) { return NSHAPES; }

ct_status ct_tile_shape(int shape, int* tx, int* ty) {
  if (shape < 0 || shape >= NSHAPES || !tx || !ty) return fail(CT_ERR_ARG, "ct_tile_shape: bad argument");
  *tx = stage_set(shape)->tx;
  *ty = stage_set(shape)->ty;
  return CT_OK;
}

int ct_tile_shape_ctas(int shape, int precision) {
  if (shape < 0 || shape >= NSHAPES || precision < CT_FP64 || precision > CT_FP32_MLP) return 0;
  const StageSet* ss = stage_set(shape);
  const int p = precision == CT_FP64 ? 0 : (precision == CT_FP32 ? 1 : 2);
  return ss->stage[p][0] ? ss->minb[p] : 0;
}

ct_status ct_set_tile_shape(const ct_case* c, int precision, int shape) {
  ct_status s = validate(c, precision);
  if (s != CT_OK) return s;
  std::lock_guard<std::mutex> lk(g_shape_mu);
  if (shape < 0) {
    g_shape.erase(shape_key(c, precision));
    return CT_OK;
  }
  if (!shape_usable(shape, variant_of(c, precision), c))
    return fail(CT_ERR_ARG, "tile shape not available for this precision or case");
  g_shape[shape_key(c, precision)] = shape;
  return CT_OK;
}

ct_status ct_autotune(const ct_case* c, int precision, const void* U, void* U1, void* work, const void* blob, int reps,
                      void* stream, int* shape_out, float* ms_out) {
  ct_status s = validate(c, precision);
  if (s != CT_OK) return s;
  if (!U || !U1 || !work || U == U1) return fail(CT_ERR_ARG, "ct_autotune: bad buffers");
  if (precision == CT_FP32_MLP && (!blob || ((uintptr_t)blob & 15) != 0)) return fail(CT_ERR_ARG, "ct_autotune: blob");
  if (reps < 1) return fail(CT_ERR_ARG, "ct_autotune: reps < 1");
  cudaStream_t st = (cudaStream_t)stream;
  const int p = variant_of(c, precision);
  int best = -1;
  float best_ms = 0.0f;
  for (int sh = 0; sh < NSHAPES; ++sh) {
    float ms = -1.0f;
    if (shape_usable(sh, p, c)) {
      if ((s = set_stage_attrs(sh, p)) != CT_OK) return s;
      const StageSet* ss = stage_set(sh);
      DevCase d = make_dev(c, work, sh, uses_prims(c, precision), uses_queue(c, precision));
      const dim3 grid(tiles_x(c, sh), tiles_y(c, sh));
      // stage 1 only: it reads U and writes the scratch state U1, so U is left as it was
      auto launch = [&]() { launch_stage(ss, p, 1, d, grid, U, nullptr, U1, blob, st); };
      if ((s = time_launches(launch, reps, st, &ms)) != CT_OK) return s;
      if (best < 0 || ms < best_ms) {
        best = sh;
        best_ms = ms;
      }
    }
    if (ms_out) ms_out[sh] = ms;
  }
  {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    g_shape[shape_key(c, precision)] = best;
  }
  if (shape_out) *shape_out = best;
  return CT_OK;
}

// ---- batched persistent step ---------------------------------------------------------------
}  // extern "C"

struct ct_batch {
  std::vector<ct_case> cases;
  int precision = CT_FP32;
  int shape = 0;
  cudaStream_t stream = nullptr;   // the caller's
  cudaStream_t cap = nullptr;      // private stream the step graphs are captured on
  char* work = nullptr;            // device workspace (caller-owned)
  BatchCounters* ctr = nullptr;    // its head: the work-list counters
  std::vector<BatchTable> table;   // one element: the kernels' parameter
  double* diag = nullptr;          // ncases x CT_NDIAG gather area
  std::vector<size_t> case_off;    // byte offset of each case's workspace
  std::vector<long long> state_off;
  int grid = 0;                    // CTAs of a launch
  int max_tiles = 0;               // tiles one CTA takes at most
  // the captured graph of the last ct_batch_step call and what it was captured for
  cudaGraphExec_t exec = nullptr;
  const void *g_U = nullptr, *g_U1 = nullptr, *g_blob = nullptr;
  int g_steps = -1, g_shape = -1;
  double g_cfl = 0.0;
};

static size_t batch_head_bytes(int ncases) {
  return align256(sizeof(BatchCounters)) + align256((size_t)ncases * CT_NDIAG * sizeof(double));
}

static ct_status batch_validate(const ct_case* cases, int ncases, int precision) {
  if (!cases || ncases < 1 || ncases > MAX_BATCH) return fail(CT_ERR_ARG, "ncases out of range [1, 96]");
  if (precision != CT_FP32 && precision != CT_FP32_MLP) return fail(CT_ERR_ARG, "batched steps are FP32 or FP32_MLP");
  for (int k = 0; k < ncases; ++k) {
    ct_status s = validate(&cases[k], precision);
    if (s != CT_OK) return s;
    if (cases[k].geom != 1) return fail(CT_ERR_ARG, "batched cases must be axisymmetric plumes (geom 1)");
    if (cases[k].bimodal != cases[0].bimodal)
      return fail(CT_ERR_ARG, "the cases of a batch share one state layout: all bimodal or none");
  }
  return CT_OK;
}

// Build the work list and case table (the kernels' parameter) for the current tile shape.
static ct_status batch_upload(ct_batch* b) {
  const int n = (int)b->cases.size();
  b->table.assign(1, BatchTable());
  BatchTable& h = b->table[0];
  memset(&h, 0, sizeof(h));
  h.ncases = n;
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  // largest cases first, so the last tiles handed out are from the small cases
  std::stable_sort(order.begin(), order.end(), [&](int a, int c2) {
    return num_blocks(&b->cases[a], b->shape) > num_blocks(&b->cases[c2], b->shape);
  });
  int t = 0;
  for (int q = 0; q < n; ++q) {
    const int k = order[q];
    h.tile_start[q] = t;
    h.case_of[q] = k;
    t += num_blocks(&b->cases[k], b->shape);
  }
  h.tile_start[n] = t;
  h.total_tiles = t;
  for (int k = 0; k < n; ++k) {
    h.tiles_x[k] = tiles_x(&b->cases[k], b->shape);
    h.state_off[k] = b->state_off[k];
    h.cases[k] = make_dev(&b->cases[k], b->work + b->case_off[k], b->shape, false,
                          uses_queue(&b->cases[k], CT_FP32_MLP));
  }
  // persistent grid: every SM full, never more CTAs than tiles
  const int p = variant_of(&b->cases[0], b->precision);
  ct_status s = set_stage_attrs(b->shape, p);
  if (s != CT_OK) return s;
  const StageSet* ss = stage_set(b->shape);
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // The runtime's occupancy calculator assumes one CTA per SM for kernels that use TMEM;
  // every CTA here gives up its allocation permit at once, so take the register and
  // shared-memory limit of the plain FP32 kernel (same registers) at this shared memory.
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ss->batch[p == 2 ? 1 : p][0], ss->nt, ss->smem[p]) !=
      cudaSuccess)
    return cuda_check("occupancy");
  per_sm = std::max(1, per_sm);
  if (b->precision == CT_FP32_MLP && !ss->plume_inviscid_only) {
    // CTAs that finish often, so that every SM keeps per_sm of them resident (the column
    // sweep holds no TMEM: its queue kernel does, in a launch of its own)
    b->max_tiles = 4;
    b->grid = (t + b->max_tiles - 1) / b->max_tiles;
  } else {
    b->max_tiles = t;
    b->grid = std::min(t, nsm * per_sm);
  }
  return CT_OK;
}

static void batch_launch(ct_batch* b, int stage, const void* Uin, const void* Un, void* Uout, const void* blob,
                         double cfl, cudaStream_t st) {
  const StageSet* ss = stage_set(b->shape);
  const int p = variant_of(&b->cases[0], b->precision);
  BatchCounters* ctr = b->ctr;
  const void* a1 = Uin;
  const void* a2 = Un;
  void* a3 = Uout;
  const void* a4 = blob;
  double a5 = cfl;
  int a6 = b->max_tiles;
  void* args[] = {b->table.data(), &ctr, &a1, &a2, &a3, &a4, &a5, &a6};
  cudaLaunchKernel(ss->batch[p][stage - 1], dim3(b->grid), dim3(ss->nt), args, ss->smem[p], st);
  // FP32 + surrogate through the column sweep: every case's queue
  if (p == 2 && ss->batch_queue[stage - 1]) {
    void* qargs[] = {b->table.data(), &a1, &a2, &a3, &a4, &a5};
    cudaLaunchKernel(ss->batch_queue[stage - 1], dim3(queue_grid()), dim3(QueueTile::NT), qargs, ss->queue_smem, st);
  }
}

__global__ void k_batch_diag(const __grid_constant__ BatchTable bt, double* __restrict__ out) {
  const int k = blockIdx.x, q = threadIdx.x;
  if (k < bt.ncases && q < CT_NDIAG) out[(size_t)k * CT_NDIAG + q] = bt.cases[k].hdr->diag[q];
}

extern "C" {

// A batch case's workspace: that of a single case, with the surrogate queue of the column
// sweep wherever the sweep can step the case (FP32 + surrogate batches use it).
static size_t batch_case_bytes(const ct_case* c) { return align256(ws_bytes(c, false, uses_queue(c, CT_FP32_MLP))); }

size_t ct_batch_workspace_bytes(const ct_case* cases, int ncases) {
  if (batch_validate(cases, ncases, CT_FP32) != CT_OK) return 0;
  size_t b = batch_head_bytes(ncases);
  for (int k = 0; k < ncases; ++k) b += batch_case_bytes(&cases[k]);
  return b;
}

size_t ct_batch_state_elems(const ct_case* cases, int ncases) {
  if (batch_validate(cases, ncases, CT_FP32) != CT_OK) return 0;
  size_t n = 0;
  for (int k = 0; k < ncases; ++k) n += (size_t)case_nf(&cases[k]) * cases[k].nx * case_nr(&cases[k]);
  return n;
}

ct_status ct_batch_create(const ct_case* cases, int ncases, int precision, const double* ufac_rows_host, void* work,
                          size_t work_bytes, void* stream, ct_batch** out) {
  ct_status s = batch_validate(cases, ncases, precision);
  if (s != CT_OK) return s;
  if (!work || !out) return fail(CT_ERR_ARG, "null workspace or handle");
  if (((uintptr_t)work & 255) != 0) return fail(CT_ERR_ARG, "workspace must be 256-byte aligned");
  if (work_bytes < ct_batch_workspace_bytes(cases, ncases)) return fail(CT_ERR_SIZE, "workspace too small");
  ct_batch* b = new ct_batch();
  b->cases.assign(cases, cases + ncases);
  b->precision = precision;
  b->stream = (cudaStream_t)stream;
  b->work = (char*)work;
  b->ctr = (BatchCounters*)work;
  b->diag = (double*)((char*)work + align256(sizeof(BatchCounters)));
  size_t off = batch_head_bytes(ncases);
  long long so = 0;
  size_t row = 0;
  for (int k = 0; k < ncases; ++k) {
    b->case_off.push_back(off);
    b->state_off.push_back(so);
    off += batch_case_bytes(&cases[k]);
    so += (long long)case_nf(&cases[k]) * cases[k].nx * case_nr(&cases[k]);
  }
  // per-case workspace: header, inflow profile and ambient state
  for (int k = 0; k < ncases && s == CT_OK; ++k) {
    const ct_case* c = &cases[k];
    s = setup_case(c, precision, ufac_rows_host ? ufac_rows_host + row : nullptr, b->work + b->case_off[k],
                   batch_case_bytes(c), stream, uses_queue(c, CT_FP32_MLP));
    row += (size_t)case_nr(c);
  }
  if (s == CT_OK && cudaMemsetAsync(b->ctr, 0, sizeof(BatchCounters), b->stream) != cudaSuccess)
    s = cuda_check("batch counters");
  if (s == CT_OK && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
    s = cuda_check("capture stream");
  if (s == CT_OK) s = batch_upload(b);
  if (s != CT_OK) {
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return s;
  }
  *out = b;
  return CT_OK;
}

void ct_batch_destroy(ct_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

ct_status ct_batch_init_state(ct_batch* b, void* U, double cfl) {
  if (!b || !U) return fail(CT_ERR_ARG, "null batch or state");
  for (size_t k = 0; k < b->cases.size(); ++k) {
    ct_status s = ct_init_state(&b->cases[k], b->precision, b->work + b->case_off[k], (float*)U + b->state_off[k], cfl,
                                b->stream);
    if (s != CT_OK) return s;
  }
  return CT_OK;
}

ct_status ct_batch_load_state(ct_batch* b, const void* U_src, void* U, double cfl) {
  if (!b || !U || !U_src) return fail(CT_ERR_ARG, "null batch or state");
  for (size_t k = 0; k < b->cases.size(); ++k) {
    ct_status s = ct_load_state(&b->cases[k], b->precision, b->work + b->case_off[k],
                                (const float*)U_src + b->state_off[k], (float*)U + b->state_off[k], cfl, b->stream);
    if (s != CT_OK) return s;
  }
  return CT_OK;
}

// a shape whose batched kernels exist for the batch's variant and suit all its cases
static bool batch_shape_usable(const ct_batch* b, int shape) {
  if (shape < 0 || shape >= NSHAPES) return false;
  const StageSet* ss = stage_set(shape);
  if (!ss->batch[variant_of(&b->cases[0], b->precision)][0]) return false;
  if (ss->plume_inviscid_only)
    for (const ct_case& c : b->cases)
      if (c.geom != 1 || c.viscous) return false;
  return true;
}

ct_status ct_batch_set_tile_shape(ct_batch* b, int shape) {
  if (!b) return fail(CT_ERR_ARG, "null batch");
  if (!batch_shape_usable(b, shape)) return fail(CT_ERR_ARG, "tile shape not available");
  if (shape == b->shape) return CT_OK;
  const int old = b->shape;
  b->shape = shape;
  ct_status s = batch_upload(b);
  if (s != CT_OK) b->shape = old;
  return s;
}

int ct_batch_tile_shape(const ct_batch* b) { return b ? b->shape : -1; }

ct_status ct_batch_autotune(ct_batch* b, const void* U, void* U1, const void* blob, int reps, int* shape_out,
                            float* ms_out) {
  if (!b || !U || !U1 || U == U1) return fail(CT_ERR_ARG, "ct_batch_autotune: bad buffers");
  if (b->precision == CT_FP32_MLP && (!blob || ((uintptr_t)blob & 15) != 0))
    return fail(CT_ERR_ARG, "ct_batch_autotune: blob");
  if (reps < 1) return fail(CT_ERR_ARG, "ct_batch_autotune: reps < 1");
  int best = -1;
  float best_ms = 0.0f;
  ct_status s = CT_OK;
  for (int sh = 0; sh < NSHAPES; ++sh) {
    float ms = -1.0f;
    if (batch_shape_usable(b, sh)) {
      if ((s = ct_batch_set_tile_shape(b, sh)) != CT_OK) return s;
      // stage 1 only: it reads U and writes the scratch state U1
      auto launch = [&]() { batch_launch(b, 1, U, nullptr, U1, blob, 0.5, b->stream); };
      if ((s = time_launches(launch, reps, b->stream, &ms)) != CT_OK) return s;
      if (best < 0 || ms < best_ms) {
        best = sh;
        best_ms = ms;
      }
    }
    if (ms_out) ms_out[sh] = ms;
  }
  if ((s = ct_batch_set_tile_shape(b, best)) != CT_OK) return s;
  if (shape_out) *shape_out = best;
  return CT_OK;
}

ct_status ct_batch_step(ct_batch* b, void* U, void* U1, const void* blob, int nsteps, double cfl) {
  if (!b || !U || !U1 || U == U1) return fail(CT_ERR_ARG, "ct_batch_step: bad buffers");
  if (b->precision == CT_FP32_MLP && (!blob || ((uintptr_t)blob & 15) != 0))
    return fail(CT_ERR_ARG, "ct_batch_step: FP32_MLP needs a 16-byte aligned surrogate blob");
  if (nsteps < 0) return fail(CT_ERR_ARG, "nsteps < 0");
  if (!(cfl > 0.0 && cfl <= 1.0)) return fail(CT_ERR_ARG, "cfl must be in (0, 1]");
  if (nsteps == 0) return CT_OK;
  const bool same = b->exec && b->g_U == U && b->g_U1 == U1 && b->g_blob == blob && b->g_steps == nsteps &&
                    b->g_cfl == cfl && b->g_shape == b->shape;
  if (!same) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    // capture the 2 * nsteps launches once; later calls with the same arguments replay it
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return cuda_check("capture");
    for (int k = 0; k < nsteps; ++k) {
      batch_launch(b, 1, U, nullptr, U1, blob, cfl, b->cap);
      batch_launch(b, 2, U1, U, U, blob, cfl, b->cap);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0ULL);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->exec = nullptr;
      return fail(CT_ERR_CUDA, cudaGetErrorString(e));
    }
    b->g_U = U;
    b->g_U1 = U1;
    b->g_blob = blob;
    b->g_steps = nsteps;
    b->g_cfl = cfl;
    b->g_shape = b->shape;
  }
  if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return cuda_check("graph launch");
  return CT_OK;
}

ct_status ct_batch_diagnostics(ct_batch* b, double* host_out) {
  if (!b || !host_out) return fail(CT_ERR_ARG, "null batch or output");
  const int n = (int)b->cases.size();
  k_batch_diag<<<n, 32, 0, b->stream>>>(b->table[0], b->diag);
  if (cudaMemcpyAsync(host_out, b->diag, (size_t)n * CT_NDIAG * sizeof(double), cudaMemcpyDeviceToHost, b->stream) !=
      cudaSuccess)
    return cuda_check("batch diag copy");
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return cuda_check("batch diag sync");
  for (int k = 0; k < n; ++k)
    if (host_out[(size_t)k * CT_NDIAG + 8] != 0.0) return fail(CT_ERR_NONFINITE, "a case produced non-finite values");
  for (int k = 0; k < n; ++k)
    if (host_out[(size_t)k * CT_NDIAG + 28] != 0.0)
      return fail(CT_ERR_TIMEOUT, "a tensor-core wait of the last step gave up");
  return CT_OK;
}

ct_status ct_mlp_dataset(const ct_case* c, const double* U, int n, float* X, float* Y, float* M, void* stream) {
  ct_status s = validate(c, CT_FP64);
  if (s != CT_OK) return s;
  if (c->bimodal) return fail(CT_ERR_ARG, "the surrogate's training data use one liquid set (bimodal = 0)");
  if (n < 0) return fail(CT_ERR_ARG, "n < 0");
  if (n == 0) return CT_OK;
  if (!U || !X || !Y || !M) return fail(CT_ERR_ARG, "null buffer");
  DevCase d = make_dev(c, nullptr);
  int grid = std::min((n + 255) / 256, 8192);
  k_mlp_dataset<<<grid, 256, 0, (cudaStream_t)stream>>>(d.sc, U, n, X, Y, M);
  return cuda_check("k_mlp_dataset");
}

const char* ct_last_error(void) { return g_err; }

// shared by the other translation units of the library (not part of the public header)
ct_status ct__set_error(ct_status s, const char* msg) { return fail(s, msg); }
const char* ct_version(void) { return "contrail-gb300 0.1 (sm_103a)"; }

}  // extern "C"
