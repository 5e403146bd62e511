/*
 * contrail_oracle.c -- plain, slow FP64 CPU oracle of the contrail finite-volume step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or execute this
 * file; only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use it.  It
 * shares no code, header, table or constant with the CUDA library: every constant and
 * formula below is written out here a second time, directly from the paper
 * (Tegethoff & Wheeler, "Non-Equilibrium Phase Changes in Aircraft Exhaust", arXiv
 * 2504.20742), with the readings noted at each function where the paper is silent.
 *
 * Equation numbers follow the order of appearance in the paper (its source carries no
 * numbers): Eq. (1) saturation ratio, (3) Kelvin radius and barrier, (4) CNT rate,
 * (5) Kantrowitz correction, (9) f(theta), (10) heterogeneous rate, (12)-(15) freezing,
 * (16) Young growth law, (20)-(21) moment equations with the r20 closure, (22)-(23)
 * conservation law, (25) species transport, (26) moment transport; numerics in Sec. 3.2.
 *
 * Style: one loop per step, plain scalar double arithmetic, no blocking, fusion or
 * reordering beyond what the method states.  Compiled with -O2 -ffp-contract=off.
 * OpenMP (if enabled) only splits independent per-cell/per-face loops over rows;
 * reductions are serial, so results do not depend on the thread count.
 *
 * Bimodal liquid (Sec. 2.2: two independent liquid moment sets, one per nucleation
 * mechanism; reading P): droplets of homogeneous origin keep fields 5..8, droplets of
 * heterogeneous (soot-activated) origin get four more fields 14..17.
 *
 * Parity pins: see tests/test_oracle_*.py (golden values under tests/golden/).  Pinned
 * under a reading, not against numbers the paper prints: alpha_crit of the Kantrowitz
 * factor (Eq. 5), q_c = 1 and the soot gating of J_het.  Pinned against their own
 * publications rather than the paper, which cites but does not print them: the Sonntag,
 * IAPWS and Koop (2000) coefficient sets.  Parity unpinned: everything that needs the
 * paper's REFPROP/IAPWS-95 backend.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------
 * Field layout of the conserved state U (structure of arrays, x fastest):
 *   U[f*N + j*nx + i], N = nx*nr, f = 0..13:
 *   0 rho, 1 rho*u, 2 rho*v, 3 rho*E, 4 rho*Y_v,
 *   5..8  rho*mu_k(liquid)/(1 um)^k, 9..12 rho*mu_k(ice)/(1 um)^k, 13 rho*n_soot.
 * Moments mu_k are specific (per kg of mixture), Eq. (26) transports rho*mu_k.
 * Bimodal cases append 14..17 rho*mu_k of the liquid of heterogeneous origin (reading P),
 * NF_BI = 18 fields; fields 5..8 then hold the liquid of homogeneous origin.
 * ---------------------------------------------------------------------------------- */
#define NF 14
#define NF_BI 18
#define NFMAX 18
#define F_MH 14
#define F_RHO 0
#define F_RU 1
#define F_RV 2
#define F_RE 3
#define F_RYV 4
#define F_ML 5
#define F_MS 9
#define F_NS 13

/* Reading A: constants (SI). */
static const double NA = 6.02214076e23;   /* Avogadro */
static const double KB = 1.380649e-23;    /* Boltzmann */
static const double RU = 8.314462618;     /* universal gas constant */
static const double MW = 0.018015;        /* molar mass of water */
static const double RA = 287.05;          /* dry-air pseudo-component */
static const double CPV = 1859.0;         /* vapour c_p */
static const double CL = 4186.0;          /* liquid water c */
static const double CS = 2100.0;          /* ice c */
static const double RHOL = 1000.0;        /* liquid density */
static const double RHOS = 917.0;         /* ice density */
static const double TREF = 273.15;        /* reference temperature of latent heats */
static const double HLV0 = 2.501e6;       /* h_v - h_l at TREF */
static const double HSL0 = 3.337e5;       /* h_l - h_s at TREF */
static const double QC = 1.0;             /* condensation coefficient q_c (silent -> 1) */
static const double COS_THETA = 0.0;      /* contact angle 90 deg (Sec. 2.2, het. condensation) */
static const double YOUNG_ALPHA = 11.0;   /* Eq. (16): alpha = 11 */
static const double YOUNG_BETA = 0.0;     /* Eq. (16): beta = 0 */
static const double PR = 0.71;            /* Prandtl number of the gas (reading G) */
static const double NS_SITE = 1.0e8;      /* Eq. (14)-(15): n_s = 1e8 m^-2 */
static const double K_IMM = 1.0;          /* immersion rate constant, s^-1 (reading H) */
static const double SIGMA_SV = 0.106;     /* ice-vapour surface tension (reading C) */
static const double MU_MIN = 1.0e-6;      /* population present above this mu0 (per kg) */
static const double PI = 3.14159265358979323846;

static double rv_gas(void) { return RU / MW; }
static double cva(void) { return RA / 0.4; }            /* gamma of dry air = 1.4 */
static double cpa(void) { return RA / 0.4 + RA; }
static double cvv(void) { return CPV - RU / MW; }
/* Reading E: formation energies chosen so that h_v - h_l = HLV0 and h_l - h_s = HSL0 at
 * TREF, with h_v = c_pv T + e0_v, h_l = c_l T, h_s = c_s T + e0_s. */
static double e0v(void) { return HLV0 - (CPV - CL) * TREF; }
static double e0s(void) { return (CL - CS) * TREF - HSL0; }
static double f_theta(void) {   /* Eq. (9) */
  return 0.25 * (2.0 + COS_THETA) * (1.0 - COS_THETA) * (1.0 - COS_THETA);
}

/* ------------------------------------------------------------------------------------
 * Case description (mirrors, independently, the library's ct_case; filled by ctypes).
 * ---------------------------------------------------------------------------------- */
typedef struct {
  int32_t geom;          /* 0 quasi-1D nozzle, 1 axisymmetric plume */
  int32_t nx, nr;
  int32_t bc_xlo;        /* 0 inflow profile / subsonic inlet, 1 wall */
  int32_t bc_xhi;        /* 0 outflow (zero gradient), 1 wall */
  int32_t bc_rhi;        /* 0 far field (ambient), 1 wall, 2 outflow */
  int32_t phase_change;  /* 0: all phase-change sources off */
  int32_t freezing;      /* 0: no freezing (liquid only) */
  double lx, lr;
  double area_a, x_throat;                 /* quasi-1D: A/A_t = 1 + a (x/x_t - 1)^2 */
  double d_core, d_fan, wall_len;          /* plume: nozzle diameters, duct wall length */
  double T_amb, p_amb, S_ice_amb, mach_coflow;
  double T_core, u_core, Yv_core, T_byp, u_byp;
  double n_soot, soot_rm, soot_sigma;      /* soot number per m^3 at exit, lognormal */
  double p0, T0, Yv_inlet;                 /* quasi-1D inlet total conditions */
  double seed_l_n, seed_l_r, seed_s_n, seed_s_r; /* optional initial populations in core */
  double mix_width;      /* > 0: core blends into the ambient through a tanh layer */
  double nu_t;           /* turbulent kinematic viscosity, m^2/s (viscous cases) */
  int32_t viscous;       /* 1: viscous and diffusive fluxes (reading M) */
  int32_t tables;        /* 1: water properties from tables, second-order Taylor (reading N) */
  int32_t equilibrium;   /* 1: equilibrium phase change instead of the kinetic model (reading O) */
  int32_t bimodal;       /* 1: two liquid moment sets, by nucleation mechanism (reading P) */
} or_case;

#define NDIAG 32
/* diag layout per step:
 * 0 dt, 1 total mass, 2 total water, 3 total energy (all after the step),
 * 4 boundary mass inflow over the step, 5 boundary water inflow, 6 boundary energy inflow,
 * 7 number of active cells in stage 2, 8 non-finite count,
 * 9..22 max-norm residual max |U^{n+1}-U^n|/dt per field (bimodal: the heterogeneous
 * liquid's fields 14..17 share the slots of fields 5..8, max of both), 23 max log10 J_hom over cells,
 * 24 max log10 J_het. */

/* ------------------------------------------------------------------------------------
 * Thermophysical closed forms (Sec. 2.1; readings B, C, E, G).
 * ---------------------------------------------------------------------------------- */

/* Reading B: Sonntag (1994) saturation pressure over liquid water, ln of p in Pa. */
double or_ln_psat_l(double T) {
  return -6096.9385 / T + 16.635794 - 2.711193e-2 * T + 1.673952e-5 * T * T +
         2.433502 * log(T) + log(100.0);
}
/* Reading B: Sonntag (1994) saturation pressure over ice, ln of p in Pa. */
double or_ln_psat_i(double T) {
  return -6024.5282 / T + 24.7219 + 1.0613868e-2 * T - 1.3198825e-5 * T * T -
         0.49382577 * log(T) + log(100.0);
}
static double dln_psat_l(double T) {
  return 6096.9385 / (T * T) - 2.711193e-2 + 2.0 * 1.673952e-5 * T + 2.433502 / T;
}
static double dln_psat_i(double T) {
  return 6024.5282 / (T * T) + 1.0613868e-2 - 2.0 * 1.3198825e-5 * T - 0.49382577 / T;
}

/* Reading D: T_sat(p_v) by Newton on ln p_sat(T) = ln p_v, Clausius-Clapeyron start,
 * exactly six iterations.  which = 0 liquid, 1 ice. */
double or_tsat(double pv, int which) {
  double lnpv = log(pv);
  double h0 = which == 0 ? HLV0 : HLV0 + HSL0;
  double T = 1.0 / (1.0 / TREF - rv_gas() * log(pv / 611.2) / h0);
  for (int it = 0; it < 6; ++it) {
    double f = (which == 0 ? or_ln_psat_l(T) : or_ln_psat_i(T)) - lnpv;
    double df = which == 0 ? dln_psat_l(T) : dln_psat_i(T);
    T = T - f / df;
  }
  return T;
}

/* Reading C: IAPWS (1994) surface tension of liquid water against vapour, N/m. */
double or_sigma_lg(double T) {
  double tau = 1.0 - T / 647.096;
  return 0.2358 * pow(tau, 1.256) * (1.0 - 0.625 * tau);
}

/* Sutherland viscosity of air (reading G). */
static double mu_sutherland(double T) {
  return 1.716e-5 * pow(T / 273.15, 1.5) * (273.15 + 110.4) / (T + 110.4);
}

/* Latent heats from the formation energies (reading E). */
double or_hfg(double T) { return (CPV - CL) * T + e0v(); }          /* h_v - h_l */
double or_hsg(double T) { return (CPV - CS) * T + e0v() - e0s(); }  /* h_v - h_s */

/* ------------------------------------------------------------------------------------
 * Primitive state of one cell (Sec. 3.1 Eq. (23); EOS reading E).
 * ---------------------------------------------------------------------------------- */
typedef struct {
  double rho, u, v, p, T;
  double Yv, Yl, Ys, Ya;
  double ml[4], ms[4];      /* specific moments, scaled by (1 um)^k */
  double mh[4];             /* bimodal: liquid of heterogeneous origin (0 otherwise) */
  int bi;                   /* bimodal state (18 fields) */
  double ns;                /* soot number per kg */
  double cv, Rg, gam, ef, c2;
} prim_t;

static double moment_scale(int k) {   /* (1 um)^k */
  double s = 1.0;
  for (int i = 0; i < k; ++i) s *= 1.0e-6;
  return s;
}

/* bi: the state has the 18 fields of the bimodal liquid (reading P) */
static void cons_to_prim(const double *u14, int bi, prim_t *w) {
  double rho = u14[F_RHO];
  w->rho = rho;
  w->u = u14[F_RU] / rho;
  w->v = u14[F_RV] / rho;
  w->Yv = u14[F_RYV] / rho;
  w->bi = bi;
  for (int k = 0; k < 4; ++k) {
    w->ml[k] = u14[F_ML + k] / rho;
    w->ms[k] = u14[F_MS + k] / rho;
    w->mh[k] = bi ? u14[F_MH + k] / rho : 0.0;
  }
  w->ns = u14[F_NS] / rho;
  /* liquid water of both sets */
  w->Yl = 4.0 / 3.0 * PI * RHOL * (bi ? w->ml[3] + w->mh[3] : w->ml[3]) * moment_scale(3);
  w->Ys = 4.0 / 3.0 * PI * RHOS * w->ms[3] * moment_scale(3);
  w->Ya = 1.0 - w->Yv - w->Yl - w->Ys;
  double e = u14[F_RE] / rho - 0.5 * (w->u * w->u + w->v * w->v);
  w->cv = w->Ya * cva() + w->Yv * cvv() + w->Yl * CL + w->Ys * CS;
  w->ef = w->Yv * e0v() + w->Ys * e0s();
  w->T = (e - w->ef) / w->cv;
  w->Rg = w->Ya * RA + w->Yv * rv_gas();
  w->p = rho * w->Rg * w->T;
  w->gam = 1.0 + w->Rg / w->cv;
  w->c2 = w->gam * w->p / rho;
}

/* Conserved state from (rho-free) primitives p, T, u, v, Y_v, moments, soot/kg. */
static void prim_to_cons(double p, double T, double u, double v, double Yv,
                         const double *ml, const double *ms, double ns, double *u14) {
  double Yl = 4.0 / 3.0 * PI * RHOL * ml[3] * moment_scale(3);
  double Ys = 4.0 / 3.0 * PI * RHOS * ms[3] * moment_scale(3);
  double Ya = 1.0 - Yv - Yl - Ys;
  double Rg = Ya * RA + Yv * rv_gas();
  double rho = p / (Rg * T);
  double cv = Ya * cva() + Yv * cvv() + Yl * CL + Ys * CS;
  double e = cv * T + Yv * e0v() + Ys * e0s();
  u14[F_RHO] = rho;
  u14[F_RU] = rho * u;
  u14[F_RV] = rho * v;
  u14[F_RE] = rho * (e + 0.5 * (u * u + v * v));
  u14[F_RYV] = rho * Yv;
  for (int k = 0; k < 4; ++k) {
    u14[F_ML + k] = rho * ml[k];
    u14[F_MS + k] = rho * ms[k];
  }
  u14[F_NS] = rho * ns;
}

/* ------------------------------------------------------------------------------------
 * Viscous and diffusive fluxes (Sec. 3.1 Eqs. (25)-(26); Sec. 3.2 "viscous fluxes are
 * discretized using central differences"; reading M).  The Spalart-Allmaras model is out
 * of scope: the turbulent viscosity is a case constant nu_t.  Effective transport:
 *   mu_e = mu(T) + rho nu_t,   lambda_e = mu(T) c_p / Pr + rho c_p nu_t / Pr_t,
 *   D_v = D_mol(T, p) + nu_t / Sc_t (vapour),   D_p = nu_t / Sc_t (moments, soot),
 * with D_mol = 2.11e-5 (T/273.15)^1.94 (101325/p) m^2/s (the paper gives the scaling
 * T^1.94/p).  Momentum diffuses in the vector-Laplacian form (mu_e grad u per face; the
 * radial component also loses mu_e v / r^2 per volume), energy by conduction, by the work
 * mu_e grad(|u|^2/2), and by the enthalpy that the diffusing water carries against dry air.
 * Walls are adiabatic, impermeable and slip: nothing diffuses through them.
 * ---------------------------------------------------------------------------------- */
static const double PR_T = 0.9;     /* turbulent Prandtl number (silent) */
static const double SC_T = 0.7;     /* turbulent Schmidt number (Sec. 3.1) */
static const double DV0 = 2.11e-5;  /* vapour diffusivity at 273.15 K and 101325 Pa */

double or_dv_mol(double T, double p) { return DV0 * pow(T / 273.15, 1.94) * (101325.0 / p); }

typedef struct { double rho, u, v, p, T, Yv, Yl, Ys, Ya, cp; } tcell_t;

/* transport state of a cell from its primitive vector (layout of prim_vec) */
static void tcell(const double *q, int bi, tcell_t *t) {
  t->rho = q[0]; t->u = q[1]; t->v = q[2]; t->p = q[3]; t->Yv = q[4];
  t->Yl = 4.0 / 3.0 * PI * RHOL * (bi ? q[8] + q[17] : q[8]) * moment_scale(3);
  t->Ys = 4.0 / 3.0 * PI * RHOS * q[12] * moment_scale(3);
  t->Ya = 1.0 - t->Yv - t->Yl - t->Ys;
  double Rg = t->Ya * RA + t->Yv * rv_gas();
  t->T = t->p / (t->rho * Rg);
  t->cp = t->Ya * cpa() + t->Yv * CPV + t->Yl * CL + t->Ys * CS;
}

/* effective viscosity, conductivity and diffusivities at (rho, T, p, c_p) */
static void transport_coeff(double rho, double T, double p, double cp, double nu_t, double *mu_e,
                            double *lam_e, double *Dv, double *Dp) {
  double mu = mu_sutherland(T);
  *mu_e = mu + rho * nu_t;
  *lam_e = mu * cp / PR + rho * cp * nu_t / PR_T;
  *Dv = or_dv_mol(T, p) + nu_t / SC_T;
  *Dp = nu_t / SC_T;
}

/* Face flux G (along +n) between the cell on the minus side (qa) and on the plus side (qb),
 * centres h apart, nf fields (14, or 18 for the bimodal liquid).  The face's total flux is
 * the Roe flux minus G. */
static void diffusive_flux(const double *qa, const double *qb, double h, double nu_t, int nf, double *G) {
  tcell_t a, b;
  int bi = nf == NF_BI;
  tcell(qa, bi, &a);
  tcell(qb, bi, &b);
  double rho = 0.5 * (a.rho + b.rho), T = 0.5 * (a.T + b.T), p = 0.5 * (a.p + b.p), cp = 0.5 * (a.cp + b.cp);
  double mu_e, lam_e, Dv, Dp;
  transport_coeff(rho, T, p, cp, nu_t, &mu_e, &lam_e, &Dv, &Dp);
  G[F_RHO] = 0.0;
  G[F_RU] = mu_e * (b.u - a.u) / h;
  G[F_RV] = mu_e * (b.v - a.v) / h;
  G[F_RYV] = rho * Dv * (qb[4] - qa[4]) / h;
  for (int f = 5; f < nf; ++f) G[f] = rho * Dp * (qb[f] - qa[f]) / h;
  /* mass fluxes of liquid and ice water, against which dry air diffuses back */
  double Gl = 4.0 / 3.0 * PI * RHOL * (bi ? G[F_ML + 3] + G[F_MH + 3] : G[F_ML + 3]) * moment_scale(3);
  double Gs = 4.0 / 3.0 * PI * RHOS * G[F_MS + 3] * moment_scale(3);
  double hva = (CPV - cpa()) * T + e0v();   /* h_v - h_a */
  double hla = (CL - cpa()) * T;            /* h_l - h_a */
  double hsa = (CS - cpa()) * T + e0s();    /* h_s - h_a */
  double ka = 0.5 * (a.u * a.u + a.v * a.v), kb = 0.5 * (b.u * b.u + b.v * b.v);
  G[F_RE] = lam_e * (b.T - a.T) / h + mu_e * (kb - ka) / h + hva * G[F_RYV] + hla * Gl + hsa * Gs;
}
void or_diffusive_flux(const double *qa, const double *qb, double h, double nu_t, double *G) {
  diffusive_flux(qa, qb, h, nu_t, NF, G);
}
void or_diffusive_flux_n(const double *qa, const double *qb, double h, double nu_t, int nf, double *G) {
  diffusive_flux(qa, qb, h, nu_t, nf, G);
}

/* viscous rate of a cell for the time step: 2 nu_max (1/dx^2 + 1/dr^2), and its mu_e */
static double viscous_rate(const prim_t *w, double nu_t, double idx2_sum, double *mu_e_out) {
  double cp = w->Ya * cpa() + w->Yv * CPV + w->Yl * CL + w->Ys * CS;
  double mu_e, lam_e, Dv, Dp;
  transport_coeff(w->rho, w->T, w->p, cp, nu_t, &mu_e, &lam_e, &Dv, &Dp);
  if (mu_e_out) *mu_e_out = mu_e;
  double nu = mu_e / w->rho;
  double kap = lam_e / (w->rho * w->cv);
  if (kap > nu) nu = kap;
  if (Dv > nu) nu = Dv;
  if (Dp > nu) nu = Dp;
  return 2.0 * nu * idx2_sum;
}

/* ------------------------------------------------------------------------------------
 * Phase-change source of one cell (Sec. 2.2, Eqs. (1)-(21); readings D, F-J).
 * Output Q is the conservative source vector (per unit volume), aux receives
 * 0 ln S_l, 1 ln S_i, 2 ln J_hom (or -inf), 3 ln J_het,eff (or -inf), 4 active flag,
 * 5 r_crit, 6 phi, 7 G_l(r20), 8 G_s(r20), 9 Koop log10 J_s (cm^-3 s^-1, or -inf),
 * 10 per-droplet freezing rate omega.
 * ---------------------------------------------------------------------------------- */
typedef struct {
  double n_soot_ref;   /* exit soot number per m^3 (0: no heterogeneous nucleation) */
  double rp2;          /* lognormal soot <r_p^2> */
  int phase_change, freezing;
  int tables;          /* reading N */
  int equilibrium;     /* reading O */
  int bimodal;         /* reading P */
} src_par_t;

/* ------------------------------------------------------------------------------------
 * Tabulated water properties (Sec. 3.2: properties tabulated before the run and
 * interpolated by a second-order Taylor expansion; reading N).  Nodes every 0.5 K from
 * 150 K to 640 K; each node holds the value and the first and half the second derivative
 * of ln p_sat,l, ln p_sat,i and sigma_lg, from the closed forms of readings B and C.  A
 * query uses the nearest node: f(T) = c0 + d (c1 + d c2), d = T - T_k (|d| <= 0.25 K; out of
 * range, the end node's expansion).
 * ---------------------------------------------------------------------------------- */
#define TAB_N 981
static const double TAB_T0 = 150.0, TAB_DT = 0.5;
static double g_tab[3][TAB_N][3];
static int g_tab_ready = 0;

static void build_tables(void) {
  if (g_tab_ready) return;
  const double al = -6096.9385, cl1 = -2.711193e-2, dl = 1.673952e-5, el = 2.433502;   /* Sonntag, liquid */
  const double ai = -6024.5282, ci1 = 1.0613868e-2, di = -1.3198825e-5, ei = -0.49382577;   /* ice */
  const double Tc = 647.096, B = 0.2358, mu = 1.256, b = 0.625;                       /* IAPWS sigma */
  for (int k = 0; k < TAB_N; ++k) {
    double T = TAB_T0 + TAB_DT * k;
    /* ln p = a/T + b0 + c T + d T^2 + e ln T: f' = -a/T^2 + c + 2 d T + e/T, f'' = 2a/T^3 + 2d - e/T^2 */
    g_tab[0][k][0] = or_ln_psat_l(T);
    g_tab[0][k][1] = -al / (T * T) + cl1 + 2.0 * dl * T + el / T;
    g_tab[0][k][2] = 0.5 * (2.0 * al / (T * T * T) + 2.0 * dl - el / (T * T));
    g_tab[1][k][0] = or_ln_psat_i(T);
    g_tab[1][k][1] = -ai / (T * T) + ci1 + 2.0 * di * T + ei / T;
    g_tab[1][k][2] = 0.5 * (2.0 * ai / (T * T * T) + 2.0 * di - ei / (T * T));
    /* sigma = B tau^mu (1 - b tau), tau = 1 - T/Tc */
    double tau = 1.0 - T / Tc;
    double ds_dtau = B * pow(tau, mu - 1.0) * (mu * (1.0 - b * tau) - b * tau);
    double d2s_dtau2 = B * (mu * (mu - 1.0) * pow(tau, mu - 2.0) * (1.0 - b * tau) - 2.0 * b * mu * pow(tau, mu - 1.0));
    g_tab[2][k][0] = or_sigma_lg(T);
    g_tab[2][k][1] = -ds_dtau / Tc;
    g_tab[2][k][2] = 0.5 * d2s_dtau2 / (Tc * Tc);
  }
  g_tab_ready = 1;
}

/* value (der = 0) or first derivative (der = 1) of tabulated property `which` at T */
static double tab_eval(int which, double T, int der) {
  int k = (int)floor((T - TAB_T0) / TAB_DT + 0.5);
  if (k < 0) k = 0;
  if (k > TAB_N - 1) k = TAB_N - 1;
  double d = T - (TAB_T0 + TAB_DT * k);
  const double *c = g_tab[which][k];
  return der ? c[1] + 2.0 * c[2] * d : c[0] + d * (c[1] + d * c[2]);
}

double or_table_eval(int which, double T, int der) {
  build_tables();
  return tab_eval(which, T, der);
}

static double prop_lnpl(const src_par_t *sp, double T) { return sp->tables ? tab_eval(0, T, 0) : or_ln_psat_l(T); }
static double prop_lnpi(const src_par_t *sp, double T) { return sp->tables ? tab_eval(1, T, 0) : or_ln_psat_i(T); }
static double prop_sigma(const src_par_t *sp, double T) { return sp->tables ? tab_eval(2, T, 0) : or_sigma_lg(T); }

/* T_sat of reading D with the tabulated curve and its derivative (same start, 6 steps) */
static double prop_tsat(const src_par_t *sp, double pv, int which) {
  if (!sp->tables) return or_tsat(pv, which);
  double lnpv = log(pv);
  double h0 = which == 0 ? HLV0 : HLV0 + HSL0;
  double T = 1.0 / (1.0 / TREF - rv_gas() * log(pv / 611.2) / h0);
  for (int it = 0; it < 6; ++it) T = T - (tab_eval(which, T, 0) - lnpv) / tab_eval(which, T, 1);
  return T;
}

/* Young's nu, Eq. (16). */
static double young_nu(double Tsat, double h, double gam_g, double cp_g) {
  double Rv = rv_gas();
  return Rv * Tsat / h *
         (YOUNG_ALPHA - 0.5 - (2.0 - QC) / (2.0 * QC) * (gam_g + 1.0) / (2.0 * gam_g) * cp_g * Tsat / h);
}

/* Young growth law, Eq. (16), with Delta T * r_crit written through Delta T / ln S
 * (reading G) so that S = 1 is regular.  rho_d, h, sig: droplet/crystal density,
 * latent heat and surface tension of the phase. */
double or_growth(double r, double T, double Tsat, double lnS, double sig, double rho_d,
                 double h, double lam_g, double lbar, double gam_g, double cp_g) {
  double Rv = rv_gas();
  double Kn = lbar / (2.0 * r);
  double nu = young_nu(Tsat, h, gam_g, cp_g);
  double dT = Tsat - T;
  double dT_over_lnS = fabs(lnS) < 1.0e-8 ? Rv * T * Tsat / h : dT / lnS;
  double dT_rc = dT_over_lnS * 2.0 * sig / (rho_d * Rv * T);
  double num = lam_g * (dT - dT_rc / r);
  double den = rho_d * h * r * (1.0 / (1.0 + 2.0 * YOUNG_BETA * Kn) + 3.78 * (1.0 - nu) * Kn / PR);
  return num / den;
}

/* Koop et al. (2000) homogeneous freezing rate, log10 of J in cm^-3 s^-1, as a cubic in
 * Delta a_w; reading H clamps Delta a_w to the fit's range [0.26, 0.34]. */
double or_koop_log10J(double daw) {
  if (daw < 0.26) return -INFINITY;
  double d = daw > 0.34 ? 0.34 : daw;
  return -906.7 + 8502.0 * d - 26924.0 * d * d + 29180.0 * d * d * d;
}

/* A (may be NULL) is the cell's conserved state after the flux-only part of the stage
 * update, U + dt (-div F + S_geo); the limiters of reading J keep A + dt Q non-negative.
 * NULL means the cell's own state (a pointwise evaluation without transport). */
/* ------------------------------------------------------------------------------------
 * Equilibrium phase change (Sec. 4.3 compares it with the kinetic model; reading O).
 * The water of a cell is at thermodynamic equilibrium at the end of every stage: with the
 * density, velocity, total energy and total water of the flux-updated state fixed, vapour
 * is in excess of saturation over the condensed phase only if no condensate could take it
 * up.  The condensate is liquid above T_FRZ = 235.15 K (homogeneous freezing) and ice
 * below, monodisperse with radius 1 um (the model carries no size); a condensate below
 * 1e-15 per kg counts as none.  The temperature solves
 * the energy balance e(T) = Y_a c_va T + Y_v (c_vv T + e0v) + Y_c e_c(T) with
 * Y_v = p_sat(T) / (rho R_v T) by eight Newton steps from the all-vapour temperature.
 * ---------------------------------------------------------------------------------- */
static const double T_FRZ = 235.15;
static const double Y_MIN_EQ = 1.0e-15;   /* condensate mass fraction taken as none */

/* saturation vapour mass fraction over liquid (ice = 0) or ice (1) and its T derivative */
static double ysat(const src_par_t *sp, double rho, double T, int ice, double *dydT) {
  double lnp = ice ? prop_lnpi(sp, T) : prop_lnpl(sp, T);
  double dlnp = sp->tables ? tab_eval(ice, T, 1) : (ice ? dln_psat_i(T) : dln_psat_l(T));
  double y = exp(lnp) / (rho * rv_gas() * T);
  if (dydT) *dydT = y * (dlnp - 1.0 / T);
  return y;
}

/* Equilibrium split of total water W at density rho and specific internal energy e:
 * returns T and sets Y_v, Y_c (condensate) and the phase (0 liquid, 1 ice). */
static double equilibrium_split(const src_par_t *sp, double rho, double e, double W, double *Yv, double *Yc,
                                int *ice) {
  double Ya = 1.0 - W;
  double Tv = (e - W * e0v()) / (Ya * cva() + W * cvv());   /* all vapour */
  *ice = Tv < T_FRZ;
  if (W <= ysat(sp, rho, Tv, *ice, NULL)) { *Yv = W; *Yc = 0.0; return Tv; }
  for (int pass = 0; pass < 2; ++pass) {
    int ic = pass == 0 ? 0 : 1;
    double cc = ic ? CS : CL, ec0 = ic ? e0s() : 0.0;
    double T = Tv;
    for (int it = 0; it < 8; ++it) {
      double dy, y = ysat(sp, rho, T, ic, &dy);
      double g = Ya * cva() * T + y * (cvv() * T + e0v()) + (W - y) * (cc * T + ec0) - e;
      double dg = Ya * cva() + y * cvv() + (W - y) * cc + dy * (cvv() * T + e0v() - cc * T - ec0);
      T -= g / dg;
    }
    double y = ysat(sp, rho, T, ic, NULL);
    if (ic == 1 || T >= T_FRZ) {
      if (y >= W) { *Yv = W; *Yc = 0.0; *ice = ic; return Tv; }   /* no condensate after all */
      *Yv = y; *Yc = W - y; *ice = ic;
      return T;
    }
  }
  return Tv;   /* not reached */
}

static void phase_source(const prim_t *w, const double *A, double dt, const src_par_t *sp,
                         double *Q, double *aux) {
  for (int f = 0; f < (sp->bimodal ? NF_BI : NF); ++f) Q[f] = 0.0;
  for (int a = 0; a < 11; ++a) aux[a] = 0.0;
  aux[2] = -INFINITY;
  aux[3] = -INFINITY;
  aux[9] = -INFINITY;
  if (!sp->phase_change) return;
  if (sp->equilibrium) {
    /* the equilibrium state of the flux-updated stage state (or of the cell itself); the
     * model carries one condensate population, so it is not combined with the bimodal
     * liquid */
    double X[NF];
    prim_t x;
    if (A) {
      for (int f = 0; f < NF; ++f) X[f] = A[f];
      cons_to_prim(X, 0, &x);
    } else {
      x = *w;
      prim_to_cons(w->p, w->T, w->u, w->v, w->Yv, w->ml, w->ms, w->ns, X);
    }
    double pv0 = x.rho * x.Yv * rv_gas() * x.T;
    if (pv0 < 1.0e-30) pv0 = 1.0e-30;
    aux[0] = log(pv0) - prop_lnpl(sp, x.T);
    aux[1] = log(pv0) - prop_lnpi(sp, x.T);
    double W = x.Yv + x.Yl + x.Ys;
    double e = x.cv * x.T + x.ef;
    double Yv, Yc;
    int ice;
    double Teq = equilibrium_split(sp, x.rho, e, W, &Yv, &Yc, &ice);
    /* condensate below 1e-15 per kg counts as none: the explicit stage leaves rounding
     * residues where the target is exactly zero */
    int had = x.Yl + x.Ys > Y_MIN_EQ;
    int active = Yc > Y_MIN_EQ || had;
    aux[4] = active ? 1.0 : 0.0;
    if (!active) return;
    /* target conserved water fields: monodisperse condensate of radius 1 um */
    double Xt[NF];
    for (int f = 0; f < NF; ++f) Xt[f] = X[f];
    Xt[F_RYV] = x.rho * Yv;
    double n = Yc / (4.0 / 3.0 * PI * (ice ? RHOS : RHOL) * moment_scale(3));   /* mu_hat, scaled */
    for (int k = 0; k < 4; ++k) {
      Xt[F_ML + k] = ice ? 0.0 : x.rho * n;
      Xt[F_MS + k] = ice ? x.rho * n : 0.0;
    }
    for (int f = F_RYV; f <= F_MS + 3; ++f) Q[f] = (Xt[f] - X[f]) / dt;
    aux[5] = Teq;   /* slot 5 carries the equilibrium temperature in this model */
    return;
  }
  const double Rv = rv_gas();
  double T = w->T, rho = w->rho, p = w->p;

  /* Eq. (1): saturation ratio from the vapour partial pressure (reading D). */
  /* a vapour-free cell keeps a vanishing partial pressure so that ln S stays finite */
  double pv = rho * w->Yv * Rv * T;
  if (pv < 1.0e-30) pv = 1.0e-30;
  double lnpsl = prop_lnpl(sp, T), lnpsi = prop_lnpi(sp, T);
  double lnSl = log(pv) - lnpsl;
  double lnSi = log(pv) - lnpsi;
  aux[0] = lnSl;
  aux[1] = lnSi;

  /* moments in SI units; mh: the liquid of heterogeneous origin (bimodal, reading P) */
  const int bi = sp->bimodal;
  double ml[4], ms[4], mh[4];
  for (int k = 0; k < 4; ++k) {
    ml[k] = w->ml[k] * moment_scale(k);
    ms[k] = w->ms[k] * moment_scale(k);
    mh[k] = bi ? w->mh[k] * moment_scale(k) : 0.0;
  }
  int present_l = ml[0] > MU_MIN && ml[1] > 0.0 && ml[2] > 0.0 && ml[3] > 0.0;
  int present_s = ms[0] > MU_MIN && ms[1] > 0.0 && ms[2] > 0.0 && ms[3] > 0.0;
  int present_h = bi && mh[0] > MU_MIN && mh[1] > 0.0 && mh[2] > 0.0 && mh[3] > 0.0;
  /* Active-cell test: nucleation needs S_l > 1 (Eq. (3) has no real r_crit otherwise),
   * growth and freezing need a population; anything else gives an exactly zero source. */
  int active = lnSl > 0.0 || present_l || present_s || present_h;
  aux[4] = active ? 1.0 : 0.0;
  if (!active) return;

  /* gas-phase properties (reading G) */
  double Yg = w->Ya + w->Yv;
  double cp_g = (w->Ya * cpa() + w->Yv * CPV) / Yg;
  double cv_g = (w->Ya * cva() + w->Yv * cvv()) / Yg;
  double gam_g = cp_g / cv_g;
  double Rg = (w->Ya * RA + w->Yv * Rv) / Yg;
  double mu_g = mu_sutherland(T);
  double lam_g = mu_g * cp_g / PR;
  double lbar = 1.5 * mu_g * sqrt(Rg * T) / p;
  double hfg = or_hfg(T), hsg = or_hsg(T);

  /* Nucleation, Eqs. (3)-(6), (9)-(11); J_het gated by the soot number (reading F).
   * One liquid set takes both rates; the bimodal liquid takes the homogeneous rate into
   * the first set and the heterogeneous rate into the second (reading P). */
  double Jeff = 0.0, Jeff_h = 0.0, rc = 0.0;
  if (lnSl > 0.0) {
    double sig = prop_sigma(sp, T);
    rc = 2.0 * sig / (RHOL * Rv * T * lnSl);
    double dGkT = 4.0 / 3.0 * PI * sig * rc * rc / (KB * T);
    double rhov = rho * w->Yv;
    double lnA = log(QC) + 0.5 * log(2.0 * sig * NA * NA * NA / (PI * MW * MW * MW)) +
                 2.0 * log(rhov) - log(RHOL);
    double lnJhom = lnA - dGkT;
    double lnJhet = lnA - f_theta() * dGkT;
    double Jhom = exp(lnJhom);
    double Jhet = 0.0;
    if (sp->n_soot_ref > 0.0 && w->ns > 0.0) {
      double gate = rho * w->ns / sp->n_soot_ref;
      Jhet = exp(lnJhet) * gate;
      aux[3] = lnJhet + log(gate);
    }
    aux[2] = lnJhom;
    /* Eq. (5), alpha_crit from Young's heat-transfer law at r_crit (reading F). */
    double Tsat = prop_tsat(sp, pv, 0);
    double nu = young_nu(Tsat, hfg, gam_g, cp_g);
    double Knc = lbar / (2.0 * rc);
    double alpha_c = lam_g / (rc * (1.0 / (1.0 + 2.0 * YOUNG_BETA * Knc) + 3.78 * (1.0 - nu) * Knc / PR));
    double phi = QC * rhov / alpha_c * sqrt(Rv * T / (2.0 * PI)) *
                 (hfg * hfg / (Rv * T * T) - hfg / T);
    aux[6] = phi;
    if (bi) {
      Jeff = Jhom / (1.0 + phi);
      Jeff_h = Jhet / (1.0 + phi);
    } else {
      Jeff = (Jhom + Jhet) / (1.0 + phi);
    }
  }
  aux[5] = rc;

  /* Growth, Eq. (16) at r20 = sqrt(mu2/mu0) of each population, Eq. (21). */
  double Gl = 0.0, Gs = 0.0, Gh = 0.0;
  if (present_l) {
    double r20 = sqrt(ml[2] / ml[0]);
    double Tsat = prop_tsat(sp, pv, 0);
    Gl = or_growth(r20, T, Tsat, lnSl, prop_sigma(sp, T), RHOL, hfg, lam_g, lbar, gam_g, cp_g);
  }
  if (present_h) {
    double r20 = sqrt(mh[2] / mh[0]);
    double Tsat = prop_tsat(sp, pv, 0);
    Gh = or_growth(r20, T, Tsat, lnSl, prop_sigma(sp, T), RHOL, hfg, lam_g, lbar, gam_g, cp_g);
  }
  if (present_s) {
    double r20 = sqrt(ms[2] / ms[0]);
    double Tsat = prop_tsat(sp, pv, 1);
    Gs = or_growth(r20, T, Tsat, lnSi, SIGMA_SV, RHOS, hsg, lam_g, lbar, gam_g, cp_g);
  }
  /* Stage relaxation limiter (reading J): the vapour-growth exchange relaxes the driving
   * potential D = Delta T (1 - r_crit/r) of Eq. (16) towards zero at the rate
   * 1/tau = 4 pi rho_d mu2 (lambda/den) |dD/dY|, with dD/dY from the linearised saturation
   * curve and the latent heat of reading E.  Over a stage of length dt the exchanged mass
   * follows the exact exponential solution, i.e. G is scaled by (1 - exp(-x))/x with
   * x = dt/tau (all populations together), so that no stage overshoots the equilibrium. */
  double xsum = 0.0;
  for (int set = 0; set < 2; ++set) {
    const double *m = set == 0 ? ml : mh;
    if (!(set == 0 ? present_l : present_h)) continue;
    double r20 = sqrt(m[2] / m[0]);
    double Tsat = prop_tsat(sp, pv, 0);
    double nu = young_nu(Tsat, hfg, gam_g, cp_g);
    double Kn = lbar / (2.0 * r20);
    double cond = lam_g / (RHOL * hfg * r20 * (1.0 / (1.0 + 2.0 * YOUNG_BETA * Kn) + 3.78 * (1.0 - nu) * Kn / PR));
    double dD = Rv * Tsat * Tsat / hfg / w->Yv + (1.0 - Rv * Tsat * Tsat / (hfg * T)) * (hfg - Rv * T) / w->cv;
    xsum += dt * 4.0 * PI * RHOL * m[2] * cond * fabs(dD);
  }
  if (present_s) {
    double r20 = sqrt(ms[2] / ms[0]);
    double Tsat = prop_tsat(sp, pv, 1);
    double nu = young_nu(Tsat, hsg, gam_g, cp_g);
    double Kn = lbar / (2.0 * r20);
    double cond = lam_g / (RHOS * hsg * r20 * (1.0 / (1.0 + 2.0 * YOUNG_BETA * Kn) + 3.78 * (1.0 - nu) * Kn / PR));
    double dD = Rv * Tsat * Tsat / hsg / w->Yv + (1.0 - Rv * Tsat * Tsat / (hsg * T)) * (hsg - Rv * T) / w->cv;
    xsum += dt * 4.0 * PI * RHOS * ms[2] * cond * fabs(dD);
  }
  if (xsum > 0.0) {
    double theta = -expm1(-xsum) / xsum;
    Gl *= theta;
    Gh *= theta;
    Gs *= theta;
  }
  aux[7] = Gl;
  aux[8] = Gs;

  /* Freezing, Eqs. (12)-(15) (reading H): per-droplet rate omega, frozen number rate, for
   * each liquid population.  Immersion freezing needs a soot particle inside the droplet:
   * one set holds a fraction chi = min(1, n_soot/mu0) of such droplets; in the bimodal
   * liquid only the droplets of heterogeneous origin do (chi = min(1, n_soot/mu0_het)),
   * those of homogeneous origin none (reading P). */
  double Nf[2] = {0.0, 0.0}, rv[2] = {0.0, 0.0}, rf[2] = {0.0, 0.0};
  if (sp->freezing && (present_l || present_h) && T < TREF) {
    double daw = 1.0 - exp(lnpsi - lnpsl);   /* a_w = 1, a_w^ice = p_sat,i / p_sat,l */
    double l10 = or_koop_log10J(daw);
    aux[9] = l10;
    double Js = isinf(l10) ? 0.0 : pow(10.0, l10) * 1.0e6;   /* m^-3 s^-1 */
    for (int set = 0; set < 2; ++set) {
      const double *m = set == 0 ? ml : mh;
      if (!(set == 0 ? present_l : present_h)) continue;
      rv[set] = cbrt(m[3] / m[0]);
      double chi = 0.0;
      if (!bi || set == 1) {
        chi = w->ns / m[0];
        if (chi > 1.0) chi = 1.0;
      }
      double omega = Js * (4.0 / 3.0 * PI * rv[set] * rv[set] * rv[set]) + K_IMM * NS_SITE * 4.0 * PI * sp->rp2 * chi;
      if (set == 0) aux[10] = omega;
      /* freezing over the stage as exact first-order decay of the droplet number (reading J) */
      Nf[set] = m[0] * (-expm1(-omega * dt) / dt);
      rf[set] = rv[set] * cbrt(RHOL / RHOS);
    }
  }

  /* Moment sources, Eq. (21) (liquid nucleates at r_crit, ice at the frozen droplet's
   * radius, Sec. 2.2 moments), per kg of mixture, SI units. */
  double dml[4], dms[4], dmh[4];
  for (int k = 0; k < 4; ++k) {
    double gl = k > 0 ? k * ml[k - 1] * Gl : 0.0;
    double gs = k > 0 ? k * ms[k - 1] * Gs : 0.0;
    double gh = k > 0 ? k * mh[k - 1] * Gh : 0.0;
    dml[k] = gl + Jeff / rho * pow(rc, (double)k) - Nf[0] * pow(rv[0], (double)k);
    dmh[k] = bi ? gh + Jeff_h / rho * pow(rc, (double)k) - Nf[1] * pow(rv[1], (double)k) : 0.0;
    dms[k] = bi ? gs + Nf[0] * pow(rf[0], (double)k) + Nf[1] * pow(rf[1], (double)k) : gs + Nf[0] * pow(rf[0], (double)k);
  }
  /* Limiters (reading J) act on the stage update of the cell: al, ah, as_ and av are the
   * specific moments of the liquid sets and the ice and the vapour fraction after the
   * flux-only update. */
  double al[4], ah[4], as_[4], av;
  if (A) {
    for (int k = 0; k < 4; ++k) {
      al[k] = A[F_ML + k] / rho * moment_scale(k);
      as_[k] = A[F_MS + k] / rho * moment_scale(k);
      ah[k] = bi ? A[F_MH + k] / rho * moment_scale(k) : 0.0;
    }
    av = A[F_RYV] / rho;
  } else {
    for (int k = 0; k < 4; ++k) { al[k] = ml[k]; as_[k] = ms[k]; ah[k] = mh[k]; }
    av = w->Yv;
  }
  /* Complete evaporation / sublimation: a population whose mass would not stay positive is
   * removed entirely within the stage. */
  if (al[3] + dt * dml[3] <= 0.0)
    for (int k = 0; k < 4; ++k) dml[k] = -al[k] / dt;
  if (bi && ah[3] + dt * dmh[3] <= 0.0)
    for (int k = 0; k < 4; ++k) dmh[k] = -ah[k] / dt;
  if (as_[3] + dt * dms[3] <= 0.0)
    for (int k = 0; k < 4; ++k) dms[k] = -as_[k] / dt;
  /* Mass exchange, Eqs. (18), (25): the vapour sink is the condensed gain negated. */
  double dYl = 4.0 / 3.0 * PI * RHOL * (bi ? dml[3] + dmh[3] : dml[3]);
  double dYs = 4.0 / 3.0 * PI * RHOS * dms[3];
  double dYv = -(dYl + dYs);
  /* Vapour positivity: condensation is scaled down so that the vapour stays >= 0. */
  if (av + dt * dYv < 0.0) {
    double th = av > 0.0 ? av / (-dt * dYv) : 0.0;
    for (int k = 0; k < 4; ++k) {
      dml[k] *= th;
      dmh[k] *= th;
      dms[k] *= th;
    }
    dYv *= th;
  }
  Q[F_RYV] = rho * dYv;
  for (int k = 0; k < 4; ++k) {
    Q[F_ML + k] = rho * dml[k] / moment_scale(k);
    Q[F_MS + k] = rho * dms[k] / moment_scale(k);
    if (bi) Q[F_MH + k] = rho * dmh[k] / moment_scale(k);
  }
}

/* ------------------------------------------------------------------------------------
 * Convective flux: MUSCL/van Leer on primitives + Roe with Harten fix (Sec. 3.2,
 * reading K).  dir = 0: normal velocity u, dir = 1: normal velocity v.
 * Face primitive vector: 0 rho, 1 u, 2 v, 3 p, 4 Y_v, 5..8 ml, 9..12 ms, 13 ns
 * (bimodal: 14..17 mh).
 * ---------------------------------------------------------------------------------- */
static void prim_vec(const prim_t *w, double *q) {
  q[0] = w->rho; q[1] = w->u; q[2] = w->v; q[3] = w->p; q[4] = w->Yv;
  for (int k = 0; k < 4; ++k) { q[5 + k] = w->ml[k]; q[9 + k] = w->ms[k]; }
  q[13] = w->ns;
  if (w->bi)
    for (int k = 0; k < 4; ++k) q[14 + k] = w->mh[k];
}

/* van Leer limited slope: psi(r) * (q_i - q_{i-1}) with psi(r) = (r+|r|)/(1+|r|),
 * r = (q_{i+1}-q_i)/(q_i-q_{i-1}), written in its equivalent harmonic-mean form. */
static double vl_slope(double dm, double dp) {
  if (!((dm > 0.0 && dp > 0.0) || (dm < 0.0 && dp < 0.0))) return 0.0;
  return 2.0 * dm * (dp / (dm + dp));
}

typedef struct { double rho, u, v, p, Yv, Yl, Ys, Ya, cv, Rg, gam, ef, H, c2; } face_t;

static void face_state(const double *q, int bi, face_t *s) {
  s->rho = q[0]; s->u = q[1]; s->v = q[2]; s->p = q[3]; s->Yv = q[4];
  s->Yl = 4.0 / 3.0 * PI * RHOL * (bi ? q[8] + q[17] : q[8]) * moment_scale(3);
  s->Ys = 4.0 / 3.0 * PI * RHOS * q[12] * moment_scale(3);
  s->Ya = 1.0 - s->Yv - s->Yl - s->Ys;
  s->cv = s->Ya * cva() + s->Yv * cvv() + s->Yl * CL + s->Ys * CS;
  s->Rg = s->Ya * RA + s->Yv * rv_gas();
  s->gam = 1.0 + s->Rg / s->cv;
  s->ef = s->Yv * e0v() + s->Ys * e0s();
  double T = s->p / (s->rho * s->Rg);
  double e = s->cv * T + s->ef;
  s->H = e + 0.5 * (s->u * s->u + s->v * s->v) + s->p / s->rho;
  s->c2 = s->gam * s->p / s->rho;
}

/* Roe averages of a face (reading K): density, normal and tangential velocity, total
 * enthalpy and formation energy with the weights sqrt(rho) / (sqrt(rho_L) + sqrt(rho_R)),
 * gamma as the arithmetic mean, and the sound speed of the averaged state.  For physical
 * face states (p, rho, T > 0) c2 >= (gamma~ - 1) min(h_L, h_R) >= c_min^2 / 2, since
 * H~ - ef~ - q~^2/2 = w_L h_L + w_R h_R + w_L w_R |du|^2 / 2 with the sensible enthalpy
 * h = c_v T + p/rho; c2 is nevertheless held at or above 1 % of the smaller side's c^2
 * (c2_used), a guard against reconstructed states that rounding has made unphysical. */
typedef struct { double rho, un, ut, H, ef, gam, q2, c2, c2_used; } roe_avg_t;

static void roe_average(const face_t *L, const face_t *R, double unL, double utL, double unR, double utR,
                        roe_avg_t *a) {
  double sL = sqrt(L->rho), sR = sqrt(R->rho);
  double wL = sL / (sL + sR), wR = sR / (sL + sR);
  a->rho = sL * sR;
  a->un = wL * unL + wR * unR;
  a->ut = wL * utL + wR * utR;
  a->H = wL * L->H + wR * R->H;
  a->ef = wL * L->ef + wR * R->ef;
  a->gam = 0.5 * (L->gam + R->gam);
  a->q2 = a->un * a->un + a->ut * a->ut;
  a->c2 = (a->gam - 1.0) * (a->H - 0.5 * a->q2 - a->ef);
  double c2min = 0.01 * (L->c2 < R->c2 ? L->c2 : R->c2);
  a->c2_used = a->c2 < c2min ? c2min : a->c2;
}

/* Roe flux between reconstructed primitive vectors qL, qR of nf fields (14, or 18 for the
 * bimodal liquid); F gets nf components. */
static void roe_flux(const double *qL, const double *qR, int dir, int nf, double *F) {
  face_t L, R;
  face_state(qL, nf == NF_BI, &L);
  face_state(qR, nf == NF_BI, &R);
  double unL = dir == 0 ? L.u : L.v, utL = dir == 0 ? L.v : L.u;
  double unR = dir == 0 ? R.u : R.v, utR = dir == 0 ? R.v : R.u;
  /* physical fluxes in (rho, rho u_n, rho u_t, rho E) */
  double FL[4] = {L.rho * unL, L.rho * unL * unL + L.p, L.rho * unL * utL, L.rho * unL * L.H};
  double FR[4] = {R.rho * unR, R.rho * unR * unR + R.p, R.rho * unR * utR, R.rho * unR * R.H};
  roe_avg_t a;
  roe_average(&L, &R, unL, utL, unR, utR, &a);
  double rho_t = a.rho, un = a.un, ut = a.ut, H = a.H, q2 = a.q2;
  double c2 = a.c2_used;
  double c = sqrt(c2);
  /* wave strengths */
  double drho = R.rho - L.rho, dun = unR - unL, dut = utR - utL, dp = R.p - L.p;
  double a1 = (dp - rho_t * c * dun) / (2.0 * c2);
  double a5 = (dp + rho_t * c * dun) / (2.0 * c2);
  double a2 = drho - dp / c2;
  double a3 = rho_t * dut;
  /* |eigenvalues| with Harten's entropy fix on the acoustic waves */
  double delta = 0.1 * (fabs(un) + c);
  double l1 = fabs(un - c), l5 = fabs(un + c), l2 = fabs(un);
  if (l1 < delta) l1 = (l1 * l1 + delta * delta) / (2.0 * delta);
  if (l5 < delta) l5 = (l5 * l5 + delta * delta) / (2.0 * delta);
  double D[4];
  D[0] = l1 * a1 + l2 * a2 + l5 * a5;
  D[1] = l1 * a1 * (un - c) + l2 * a2 * un + l5 * a5 * (un + c);
  D[2] = l1 * a1 * ut + l2 * a2 * ut + l2 * a3 + l5 * a5 * ut;
  D[3] = l1 * a1 * (H - un * c) + l2 * a2 * 0.5 * q2 + l2 * a3 * ut + l5 * a5 * (H + un * c);
  double Fc[4];
  for (int m = 0; m < 4; ++m) Fc[m] = 0.5 * (FL[m] + FR[m]) - 0.5 * D[m];
  F[F_RHO] = Fc[0];
  F[F_RU] = dir == 0 ? Fc[1] : Fc[2];
  F[F_RV] = dir == 0 ? Fc[2] : Fc[1];
  F[F_RE] = Fc[3];
  /* passive quantities upwinded with the mass flux (reading A4) */
  const double *qu = Fc[0] >= 0.0 ? qL : qR;
  F[F_RYV] = Fc[0] * qu[4];
  for (int k = 0; k < 4; ++k) {
    F[F_ML + k] = Fc[0] * qu[5 + k];
    F[F_MS + k] = Fc[0] * qu[9 + k];
  }
  F[F_NS] = Fc[0] * qu[13];
  for (int f = NF; f < nf; ++f) F[f] = Fc[0] * qu[f];
}
void or_roe_flux(const double *qL, const double *qR, int dir, double *F) { roe_flux(qL, qR, dir, NF, F); }
/* Roe sound speed squared of a face, before (out[0]) and after (out[1]) the 1 % guard, and
 * the two sides' c^2 (out[2], out[3]); for the pins of the averages. */
void or_roe_c2(const double *qL, const double *qR, int dir, int nf, double *out) {
  face_t L, R;
  face_state(qL, nf == NF_BI, &L);
  face_state(qR, nf == NF_BI, &R);
  roe_avg_t a;
  roe_average(&L, &R, dir == 0 ? L.u : L.v, dir == 0 ? L.v : L.u, dir == 0 ? R.u : R.v, dir == 0 ? R.v : R.u, &a);
  out[0] = a.c2;
  out[1] = a.c2_used;
  out[2] = L.c2;
  out[3] = R.c2;
}
void or_roe_flux_n(const double *qL, const double *qR, int dir, int nf, double *F) { roe_flux(qL, qR, dir, nf, F); }

/* ------------------------------------------------------------------------------------
 * Solver context: padded grids with two ghost layers per side.
 * ---------------------------------------------------------------------------------- */
typedef struct {
  or_case c;
  int nf;                     /* fields of the state: 14, or 18 with the bimodal liquid */
  int nx, nr, nxp, nrp;       /* padded sizes */
  double dx, dr;
  src_par_t sp;
  double *inflow;             /* nr x nf conserved inflow states (plume) */
  double amb[NFMAX];          /* ambient conserved state (plume far field) */
  double *Up;                 /* padded conserved state, nf x nrp x nxp */
  double *Wp;                 /* padded primitive vectors, nf x nrp x nxp */
  double *Fx;                 /* x-face fluxes, nf x nr x (nx+1) */
  double *Fr;                 /* r-face fluxes, nf x (nr+1) x nx */
  double *L;                  /* residual, nf x N */
  double *U0, *U1;            /* stage states, nf x N */
  double *aux;                /* per-cell aux (11 values) of the last source evaluation */
  double bflux[3];            /* boundary inflow rates (mass, water, energy) */
  int active_count;
} or_ctx;

static double area_q1d(const or_case *c, double x) {   /* config: A/A_t */
  double s = x / c->x_throat - 1.0;
  return 1.0 + c->area_a * s * s;
}
static double r_center(const or_ctx *g, int j) { return (j + 0.5) * g->dr; }
static double cell_volume(const or_ctx *g, int i, int j) {
  if (g->c.geom == 0) return area_q1d(&g->c, (i + 0.5) * g->dx) * g->dx;
  return r_center(g, j) * g->dr * g->dx;
}

/* Vapour mass fraction of moist air with partial pressure pv at total pressure p. */
static double yv_from_pv(double pv, double p) {
  return pv * RA / (rv_gas() * (p - pv) + pv * RA);
}

/* Ambient state (Sec. 4.1 Table 2 reading: static T, p, ice supersaturation, coflow Mach). */
static void ambient_state(const or_case *c, double ufac, double *u14) {
  double zero[4] = {0, 0, 0, 0};
  double pv = c->S_ice_amb * exp(or_ln_psat_i(c->T_amb));
  double Yv = yv_from_pv(pv, c->p_amb);
  double cp = (1.0 - Yv) * cpa() + Yv * CPV, cv = (1.0 - Yv) * cva() + Yv * cvv();
  double Rg = (1.0 - Yv) * RA + Yv * rv_gas();
  double camb = sqrt(cp / cv * Rg * c->T_amb);
  prim_to_cons(c->p_amb, c->T_amb, c->mach_coflow * camb * ufac, 0.0, Yv, zero, zero, 0.0, u14);
}

/* Inflow profile of row j (plume): core / bypass / ambient coflow, all at ambient static
 * pressure; u scaled by the row's perturbation factor. */
static void inflow_state(const or_case *c, double r, double ufac, double *u14) {
  double zero[4] = {0, 0, 0, 0};
  if (c->mix_width > 0.0) {
    /* pre-mixed layer: T, u, Y_v and soot per volume blend linearly between the core and
     * the ambient stream with weight w(r) = (1 - tanh((r - d_core/2)/width))/2 */
    double w = 0.5 * (1.0 - tanh((r - 0.5 * c->d_core) / c->mix_width));
    double pva = c->S_ice_amb * exp(or_ln_psat_i(c->T_amb));
    double Yva = yv_from_pv(pva, c->p_amb);
    double cpm = (1.0 - Yva) * cpa() + Yva * CPV, cvm = (1.0 - Yva) * cva() + Yva * cvv();
    double Rga = (1.0 - Yva) * RA + Yva * rv_gas();
    double ua = c->mach_coflow * sqrt(cpm / cvm * Rga * c->T_amb);
    double T = w * c->T_core + (1.0 - w) * c->T_amb;
    double u = (w * c->u_core + (1.0 - w) * ua) * ufac;
    double Yv = w * c->Yv_core + (1.0 - w) * Yva;
    double Rg = (1.0 - Yv) * RA + Yv * rv_gas();
    double rho = c->p_amb / (Rg * T);
    prim_to_cons(c->p_amb, T, u, 0.0, Yv, zero, zero, w * c->n_soot / rho, u14);
    return;
  }
  if (r < 0.5 * c->d_core) {
    double Yv = c->Yv_core;
    double Rg = (1.0 - Yv) * RA + Yv * rv_gas();
    double rho = c->p_amb / (Rg * c->T_core);
    double ns = c->n_soot / rho;
    prim_to_cons(c->p_amb, c->T_core, c->u_core * ufac, 0.0, Yv, zero, zero, ns, u14);
  } else if (r < 0.5 * c->d_fan) {
    prim_to_cons(c->p_amb, c->T_byp, c->u_byp * ufac, 0.0, 0.0, zero, zero, 0.0, u14);
  } else {
    ambient_state(c, ufac, u14);
  }
}

/* Quasi-1D subsonic inlet from total conditions with the interior velocity (Sec. 4.1
 * prescribes total conditions at the inlets; isentropic relation of the inlet mixture). */
static void q1d_inlet_state(const or_case *c, double u, double *u14) {
  double zero[4] = {0, 0, 0, 0};
  double Yv = c->Yv_inlet;
  double cp = (1.0 - Yv) * cpa() + Yv * CPV, cv = (1.0 - Yv) * cva() + Yv * cvv();
  double gam = cp / cv;
  if (u < 0.0) u = 0.0;
  double T = c->T0 - u * u / (2.0 * cp);
  double p = c->p0 * pow(T / c->T0, gam / (gam - 1.0));
  prim_to_cons(p, T, u, 0.0, Yv, zero, zero, 0.0, u14);
}

#define UP(g, f, i, j) ((g)->Up[((size_t)(f) * (g)->nrp + (size_t)((j) + 2)) * (g)->nxp + (size_t)((i) + 2)])
#define WP(g, f, i, j) ((g)->Wp[((size_t)(f) * (g)->nrp + (size_t)((j) + 2)) * (g)->nxp + (size_t)((i) + 2)])

or_ctx *or_create(const or_case *c, const double *ufac_rows) {
  or_ctx *g = (or_ctx *)calloc(1, sizeof(or_ctx));
  g->c = *c;
  g->nf = c->bimodal ? NF_BI : NF;
  const int nf = g->nf;
  g->nx = c->nx;
  g->nr = c->geom == 0 ? 1 : c->nr;
  g->c.nr = g->nr;
  g->nxp = g->nx + 4;
  g->nrp = g->nr + 4;
  g->dx = c->lx / g->nx;
  g->dr = c->geom == 0 ? 1.0 : c->lr / g->nr;
  size_t N = (size_t)g->nx * g->nr;
  size_t NP = (size_t)g->nxp * g->nrp;
  g->Up = (double *)calloc(nf * NP, sizeof(double));
  g->Wp = (double *)calloc(nf * NP, sizeof(double));
  g->Fx = (double *)calloc(nf * (size_t)g->nr * (g->nx + 1), sizeof(double));
  g->Fr = (double *)calloc(nf * (size_t)(g->nr + 1) * g->nx, sizeof(double));
  g->L = (double *)calloc(nf * N, sizeof(double));
  g->U0 = (double *)calloc(nf * N, sizeof(double));
  g->U1 = (double *)calloc(nf * N, sizeof(double));
  g->aux = (double *)calloc(11 * N, sizeof(double));
  g->inflow = (double *)calloc(nf * (size_t)g->nr, sizeof(double));
  g->sp.phase_change = c->phase_change;
  g->sp.freezing = c->freezing;
  g->sp.n_soot_ref = c->n_soot;
  g->sp.tables = c->tables;
  g->sp.equilibrium = c->equilibrium;
  g->sp.bimodal = c->bimodal;
  build_tables();
  double ls = log(c->soot_sigma > 0.0 ? c->soot_sigma : 1.0);
  g->sp.rp2 = c->soot_rm * c->soot_rm * exp(2.0 * ls * ls);   /* lognormal E[r^2] */
  if (c->geom == 1) {
    for (int j = 0; j < g->nr; ++j)
      inflow_state(c, r_center(g, j), ufac_rows ? ufac_rows[j] : 1.0, g->inflow + (size_t)j * nf);
    ambient_state(c, 1.0, g->amb);
  }
  return g;
}

void or_destroy(or_ctx *g) {
  if (!g) return;
  free(g->Up); free(g->Wp); free(g->Fx); free(g->Fr); free(g->L);
  free(g->U0); free(g->U1); free(g->aux); free(g->inflow); free(g);
}

/* Isentropic area-Mach relation A/A* (Sec. 4 nozzle initial guess), bisection inverse. */
static double area_mach(double M, double gam) {
  return 1.0 / M * pow(2.0 / (gam + 1.0) * (1.0 + 0.5 * (gam - 1.0) * M * M), 0.5 * (gam + 1.0) / (gam - 1.0));
}
static double mach_from_area(double ar, double gam, int supersonic) {
  double lo = supersonic ? 1.0 : 1.0e-6, hi = supersonic ? 50.0 : 1.0;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    double f = area_mach(mid, gam) - ar;
    /* A/A* decreases with M below 1 and increases above 1 */
    if ((f > 0.0) == (supersonic != 0)) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

/* Initial state (NF x N SoA): plume = inflow profile extended through the domain, with
 * the optional seed populations in the core; nozzle = isentropic area-Mach solution. */
void or_init_state(or_ctx *g, double *U) {
  const or_case *c = &g->c;
  const int nf = g->nf;
  size_t N = (size_t)g->nx * g->nr;
  for (int j = 0; j < g->nr; ++j) {
    for (int i = 0; i < g->nx; ++i) {
      double u14[NFMAX] = {0};   /* a bimodal state starts without heterogeneous liquid */
      if (c->geom == 0) {
        double zero[4] = {0, 0, 0, 0};
        double Yv = c->Yv_inlet;
        double cp = (1.0 - Yv) * cpa() + Yv * CPV, cv = (1.0 - Yv) * cva() + Yv * cvv();
        double gam = cp / cv, Rg = (1.0 - Yv) * RA + Yv * rv_gas();
        double x = (i + 0.5) * g->dx;
        double M = mach_from_area(area_q1d(c, x), gam, x >= c->x_throat);
        double T = c->T0 / (1.0 + 0.5 * (gam - 1.0) * M * M);
        double p = c->p0 * pow(T / c->T0, gam / (gam - 1.0));
        prim_to_cons(p, T, M * sqrt(gam * Rg * T), 0.0, Yv, zero, zero, 0.0, u14);
      } else {
        memcpy(u14, g->inflow + (size_t)j * nf, sizeof(double) * nf);
        if (r_center(g, j) < 0.5 * c->d_core && (c->seed_l_n > 0.0 || c->seed_s_n > 0.0)) {
          prim_t w;
          cons_to_prim(u14, g->nf == NF_BI, &w);
          double ml[4], ms[4];
          for (int k = 0; k < 4; ++k) {
            ml[k] = c->seed_l_n * pow(c->seed_l_r, (double)k) / moment_scale(k);
            ms[k] = c->seed_s_n * pow(c->seed_s_r, (double)k) / moment_scale(k);
          }
          double Yl = 4.0 / 3.0 * PI * RHOL * ml[3] * moment_scale(3);
          double Ys = 4.0 / 3.0 * PI * RHOS * ms[3] * moment_scale(3);
          /* the seeded condensate is taken from the vapour, keeping total water */
          double Yv = w.Yv - Yl - Ys;
          prim_to_cons(w.p, w.T, w.u, w.v, Yv, ml, ms, w.ns, u14);
        }
      }
      for (int f = 0; f < nf; ++f) U[(size_t)f * N + (size_t)j * g->nx + i] = u14[f];
    }
  }
}

/* Copy U into the padded array and fill the ghost layers (boundary conditions, Sec. 4.1
 * and reading A1). */
static void fill_padded(or_ctx *g, const double *U) {
  const or_case *c = &g->c;
  const int nf = g->nf;
  int nx = g->nx, nr = g->nr;
  size_t N = (size_t)nx * nr;
  for (int f = 0; f < nf; ++f)
    for (int j = 0; j < nr; ++j)
      for (int i = 0; i < nx; ++i) UP(g, f, i, j) = U[(size_t)f * N + (size_t)j * nx + i];
  for (int j = 0; j < nr; ++j) {
    for (int gl = 1; gl <= 2; ++gl) {
      /* x low */
      double u14[NFMAX] = {0};
      if (c->bc_xlo == 1) {
        for (int f = 0; f < nf; ++f) u14[f] = UP(g, f, gl - 1, j);
        u14[F_RU] = -u14[F_RU];
      } else if (c->geom == 0) {
        q1d_inlet_state(c, UP(g, F_RU, 0, j) / UP(g, F_RHO, 0, j), u14);
      } else {
        memcpy(u14, g->inflow + (size_t)j * nf, sizeof(double) * nf);
      }
      for (int f = 0; f < nf; ++f) UP(g, f, -gl, j) = u14[f];
      /* x high */
      for (int f = 0; f < nf; ++f) u14[f] = c->bc_xhi == 1 ? UP(g, f, nx - gl, j) : UP(g, f, nx - 1, j);
      if (c->bc_xhi == 1) u14[F_RU] = -u14[F_RU];
      for (int f = 0; f < nf; ++f) UP(g, f, nx - 1 + gl, j) = u14[f];
    }
  }
  if (c->geom == 1) {
    for (int i = 0; i < nx; ++i) {
      for (int gl = 1; gl <= 2; ++gl) {
        /* axis: mirror with rho*v negated */
        for (int f = 0; f < nf; ++f) UP(g, f, i, -gl) = UP(g, f, i, gl - 1);
        UP(g, F_RV, i, -gl) = -UP(g, F_RV, i, -gl);
        /* r high */
        double u14[NFMAX];
        if (c->bc_rhi == 0) {
          memcpy(u14, g->amb, sizeof(double) * nf);
        } else if (c->bc_rhi == 1) {
          for (int f = 0; f < nf; ++f) u14[f] = UP(g, f, i, nr - gl);
          u14[F_RV] = -u14[F_RV];
        } else {
          for (int f = 0; f < nf; ++f) u14[f] = UP(g, f, i, nr - 1);
        }
        for (int f = 0; f < nf; ++f) UP(g, f, i, nr - 1 + gl) = u14[f];
      }
    }
  }
}

static double water_of_flux(const double *F, int nf) {
  double fl = nf == NF_BI ? F[F_ML + 3] + F[F_MH + 3] : F[F_ML + 3];
  return F[F_RYV] + 4.0 / 3.0 * PI * (RHOL * fl + RHOS * F[F_MS + 3]) * moment_scale(3);
}

/* Residual L(U) = -div F + S_geo + Q (Sec. 3.1 Eqs. (22), (25), (26); Sec. 3.2), and the
 * boundary inflow rates of mass, water and energy. */
static void residual(or_ctx *g, const double *U, double dt) {
  const or_case *c = &g->c;
  const int nf = g->nf;
  int nx = g->nx, nr = g->nr;
  size_t N = (size_t)nx * nr;
  fill_padded(g, U);
  /* primitives everywhere, ghosts included (x ghosts for all rows, r ghosts for all cols) */
#pragma omp parallel for schedule(static)
  for (int jj = -2; jj < nr + 2; ++jj) {
    for (int ii = -2; ii < nx + 2; ++ii) {
      int xghost = ii < 0 || ii >= nx, rghost = jj < 0 || jj >= nr;
      if (xghost && rghost) continue;
      if (rghost && c->geom == 0) continue;
      double u14[NFMAX], q[NFMAX];
      for (int f = 0; f < nf; ++f) u14[f] = UP(g, f, ii, jj);
      prim_t w;
      cons_to_prim(u14, g->nf == NF_BI, &w);
      prim_vec(&w, q);
      for (int f = 0; f < nf; ++f) WP(g, f, ii, jj) = q[f];
    }
  }
  /* x faces: face i lies between cells i-1 and i, i = 0..nx */
#pragma omp parallel for schedule(static)
  for (int j = 0; j < nr; ++j) {
    for (int i = 0; i <= nx; ++i) {
      double qL[NFMAX], qR[NFMAX], F[NFMAX];
      for (int f = 0; f < nf; ++f) {
        double am = WP(g, f, i - 2, j), a0 = WP(g, f, i - 1, j), a1 = WP(g, f, i, j), a2 = WP(g, f, i + 1, j);
        qL[f] = a0 + 0.5 * vl_slope(a0 - am, a1 - a0);
        qR[f] = a1 - 0.5 * vl_slope(a1 - a0, a2 - a1);
      }
      roe_flux(qL, qR, 0, nf, F);
      /* walls are adiabatic, impermeable and slip: no diffusive flux through them */
      int xwall = (i == 0 && c->bc_xlo == 1) || (i == nx && c->bc_xhi == 1);
      if (c->viscous && !xwall) {
        double qa[NFMAX], qb[NFMAX], G[NFMAX];
        for (int f = 0; f < nf; ++f) { qa[f] = WP(g, f, i - 1, j); qb[f] = WP(g, f, i, j); }
        diffusive_flux(qa, qb, g->dx, c->nu_t, nf, G);
        for (int f = 0; f < nf; ++f) F[f] -= G[f];
      }
      for (int f = 0; f < nf; ++f) g->Fx[((size_t)f * nr + j) * (nx + 1) + i] = F[f];
    }
  }
  /* r faces: face j lies between cells j-1 and j, j = 0..nr */
  if (c->geom == 1) {
#pragma omp parallel for schedule(static)
    for (int j = 0; j <= nr; ++j) {
      for (int i = 0; i < nx; ++i) {
        double qL[NFMAX], qR[NFMAX], F[NFMAX];
        for (int f = 0; f < nf; ++f) {
          double am = WP(g, f, i, j - 2), a0 = WP(g, f, i, j - 1), a1 = WP(g, f, i, j), a2 = WP(g, f, i, j + 1);
          qL[f] = a0 + 0.5 * vl_slope(a0 - am, a1 - a0);
          qR[f] = a1 - 0.5 * vl_slope(a1 - a0, a2 - a1);
        }
        roe_flux(qL, qR, 1, nf, F);
        int rwall = j == nr && c->bc_rhi == 1;
        if (c->viscous && !rwall) {
          double qa[NFMAX], qb[NFMAX], G[NFMAX];
          for (int f = 0; f < nf; ++f) { qa[f] = WP(g, f, i, j - 1); qb[f] = WP(g, f, i, j); }
          diffusive_flux(qa, qb, g->dr, c->nu_t, nf, G);
          for (int f = 0; f < nf; ++f) F[f] -= G[f];
        }
        for (int f = 0; f < nf; ++f) g->Fr[((size_t)f * (nr + 1) + j) * nx + i] = F[f];
      }
    }
  }
  /* cell residuals */
  int jw = c->geom == 1 ? (int)floor(0.5 * c->d_fan / g->dr + 0.5) : -1;
  int active = 0;
#pragma omp parallel for schedule(static) reduction(+ : active)
  for (int j = 0; j < nr; ++j) {
    for (int i = 0; i < nx; ++i) {
      size_t n = (size_t)j * nx + i;
      double Fw[NFMAX], Fe[NFMAX], Fs[NFMAX], Fn[NFMAX];
      for (int f = 0; f < nf; ++f) {
        Fw[f] = g->Fx[((size_t)f * nr + j) * (nx + 1) + i];
        Fe[f] = g->Fx[((size_t)f * nr + j) * (nx + 1) + i + 1];
        Fs[f] = c->geom == 1 ? g->Fr[((size_t)f * (nr + 1) + j) * nx + i] : 0.0;
        Fn[f] = c->geom == 1 ? g->Fr[((size_t)f * (nr + 1) + j + 1) * nx + i] : 0.0;
      }
      double u14[NFMAX];
      for (int f = 0; f < nf; ++f) u14[f] = U[(size_t)f * N + n];
      prim_t w;
      cons_to_prim(u14, g->nf == NF_BI, &w);
      double x = (i + 0.5) * g->dx;
      if (c->geom == 1 && c->wall_len > 0.0 && x < c->wall_len) {
        /* thin duct wall on the face at r = d_fan/2: each side sees a pressure-only flux */
        if (j == jw - 1) { for (int f = 0; f < nf; ++f) Fn[f] = 0.0; Fn[F_RV] = w.p; }
        if (j == jw) { for (int f = 0; f < nf; ++f) Fs[f] = 0.0; Fs[F_RV] = w.p; }
      }
      /* flux divergence and geometric sources (reading A5) */
      double Lf[NFMAX];
      for (int f = 0; f < nf; ++f) {
        double div;
        if (c->geom == 0) {
          double Aw = area_q1d(c, i * g->dx), Ae = area_q1d(c, (i + 1) * g->dx), Ac = area_q1d(c, x);
          div = (Ae * Fe[f] - Aw * Fw[f]) / (Ac * g->dx);
        } else {
          double rc = r_center(g, j), rs = j * g->dr, rn = (j + 1) * g->dr;
          div = (Fe[f] - Fw[f]) / g->dx + (rn * Fn[f] - rs * Fs[f]) / (rc * g->dr);
        }
        Lf[f] = -div;
      }
      if (c->geom == 0) {
        double Aw = area_q1d(c, i * g->dx), Ae = area_q1d(c, (i + 1) * g->dx), Ac = area_q1d(c, x);
        Lf[F_RU] += w.p * (Ae - Aw) / (Ac * g->dx);
      } else {
        Lf[F_RV] += w.p / r_center(g, j);
        if (c->viscous) {   /* radial component of the vector Laplacian: -mu_e v / r^2 */
          double mu_e, rc = r_center(g, j);
          viscous_rate(&w, c->nu_t, 0.0, &mu_e);
          Lf[F_RV] -= mu_e * w.v / (rc * rc);
        }
      }
      /* phase-change source, limited on the flux-updated stage state */
      double A[NFMAX], Q[NFMAX], aux[11];
      for (int f = 0; f < nf; ++f) A[f] = u14[f] + dt * Lf[f];
      phase_source(&w, A, dt, &g->sp, Q, aux);
      for (int a = 0; a < 11; ++a) g->aux[(size_t)a * N + n] = aux[a];
      active += aux[4] > 0.5;
      for (int f = 0; f < nf; ++f) g->L[(size_t)f * N + n] = Lf[f] + Q[f];
    }
  }
  g->active_count = active;
  /* boundary inflow rates (serial, fixed order) */
  double bm = 0.0, bw = 0.0, be = 0.0;
  for (int j = 0; j < nr; ++j) {
    double Aw, Ae;
    if (c->geom == 0) { Aw = area_q1d(c, 0.0); Ae = area_q1d(c, nx * g->dx); }
    else { Aw = Ae = r_center(g, j) * g->dr; }
    double Fw[NFMAX], Fe[NFMAX];
    for (int f = 0; f < nf; ++f) {
      Fw[f] = g->Fx[((size_t)f * nr + j) * (nx + 1) + 0];
      Fe[f] = g->Fx[((size_t)f * nr + j) * (nx + 1) + nx];
    }
    bm += Aw * Fw[F_RHO] - Ae * Fe[F_RHO];
    bw += Aw * water_of_flux(Fw, nf) - Ae * water_of_flux(Fe, nf);
    be += Aw * Fw[F_RE] - Ae * Fe[F_RE];
  }
  if (c->geom == 1) {
    for (int i = 0; i < nx; ++i) {
      double An = nr * g->dr * g->dx;
      double Fn[NFMAX];
      for (int f = 0; f < nf; ++f) Fn[f] = g->Fr[((size_t)f * (nr + 1) + nr) * nx + i];
      bm -= An * Fn[F_RHO];
      bw -= An * water_of_flux(Fn, nf);
      be -= An * Fn[F_RE];
    }
  }
  g->bflux[0] = bm;
  g->bflux[1] = bw;
  g->bflux[2] = be;
}

/* Global CFL time step (Sec. 3.2: one CFL number controls the whole domain; reading A10). */
double or_compute_dt(or_ctx *g, const double *U, double cfl) {
  const int nf = g->nf;
  int nx = g->nx, nr = g->nr;
  size_t N = (size_t)nx * nr;
  double dtmin = INFINITY;
  for (size_t n = 0; n < N; ++n) {
    double u14[NFMAX];
    for (int f = 0; f < nf; ++f) u14[f] = U[(size_t)f * N + n];
    prim_t w;
    cons_to_prim(u14, g->nf == NF_BI, &w);
    double c = sqrt(w.c2);
    double rate = (fabs(w.u) + c) / g->dx;
    if (g->c.geom == 1) rate += (fabs(w.v) + c) / g->dr;
    if (g->c.viscous) {
      double s2 = 1.0 / (g->dx * g->dx) + (g->c.geom == 1 ? 1.0 / (g->dr * g->dr) : 0.0);
      rate += viscous_rate(&w, g->c.nu_t, s2, NULL);
    }
    double dt = cfl / rate;
    if (dt < dtmin) dtmin = dt;
  }
  return dtmin;
}

static void totals(or_ctx *g, const double *U, double *M, double *W, double *E) {
  int nx = g->nx, nr = g->nr;
  size_t N = (size_t)nx * nr;
  double m = 0.0, w = 0.0, e = 0.0;
  for (int j = 0; j < nr; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t n = (size_t)j * nx + i;
      double V = cell_volume(g, i, j);
      m += V * U[(size_t)F_RHO * N + n];
      double l3 = U[(size_t)(F_ML + 3) * N + n];
      if (g->nf == NF_BI) l3 += U[(size_t)(F_MH + 3) * N + n];
      w += V * (U[(size_t)F_RYV * N + n] +
                4.0 / 3.0 * PI * (RHOL * l3 + RHOS * U[(size_t)(F_MS + 3) * N + n]) * moment_scale(3));
      e += V * U[(size_t)F_RE * N + n];
    }
  *M = m; *W = w; *E = e;
}

/* One explicit SSP-RK2 (Heun) step with the same dt and the source in both stages
 * (Sec. 3.2, readings J, K):  U1 = U + dt L(U);  U <- U/2 + (U1 + dt L(U1))/2. */
int or_step(or_ctx *g, double *U, int nsteps, double cfl, double *diag) {
  const int nf = g->nf;
  int nx = g->nx, nr = g->nr;
  size_t N = (size_t)nx * nr;
  for (int s = 0; s < nsteps; ++s) {
    double dt = or_compute_dt(g, U, cfl);
    double *d = diag ? diag + (size_t)s * NDIAG : NULL;
    memcpy(g->U0, U, sizeof(double) * nf * N);
    residual(g, g->U0, dt);
    double b1[3] = {g->bflux[0], g->bflux[1], g->bflux[2]};
    for (size_t m = 0; m < nf * N; ++m) g->U1[m] = g->U0[m] + dt * g->L[m];
    residual(g, g->U1, dt);
    double b2[3] = {g->bflux[0], g->bflux[1], g->bflux[2]};
    for (size_t m = 0; m < nf * N; ++m) U[m] = 0.5 * g->U0[m] + 0.5 * (g->U1[m] + dt * g->L[m]);
    if (d) {
      memset(d, 0, sizeof(double) * NDIAG);
      d[0] = dt;
      totals(g, U, &d[1], &d[2], &d[3]);
      for (int k = 0; k < 3; ++k) d[4 + k] = 0.5 * dt * (b1[k] + b2[k]);
      d[7] = g->active_count;
      double nonfinite = 0.0;
      for (size_t m = 0; m < nf * N; ++m) nonfinite += !isfinite(U[m]);
      d[8] = nonfinite;
      for (int f = 0; f < nf; ++f) {
        double m = 0.0;
        for (size_t n = 0; n < N; ++n) {
          double r = fabs(U[(size_t)f * N + n] - g->U0[(size_t)f * N + n]) / dt;
          if (r > m) m = r;
        }
        /* the heterogeneous liquid's fields share the slots of the first liquid set */
        int slot = f < NF ? f : F_ML + (f - F_MH);
        if (m > d[9 + slot]) d[9 + slot] = m;
      }
      double mh = -INFINITY, mt = -INFINITY;
      for (size_t n = 0; n < N; ++n) {
        if (g->aux[2 * N + n] > mh) mh = g->aux[2 * N + n];
        if (g->aux[3 * N + n] > mt) mt = g->aux[3 * N + n];
      }
      d[23] = mh / log(10.0);
      d[24] = mt / log(10.0);
    }
  }
  return 0;
}

/* Per-cell diagnostic fields of state U: which = 0 T, 1 p, 2 ln S_l, 3 ln S_i,
 * 4 log10 J_hom, 5 log10 J_het,eff, 6 active flag, 7 r_crit, 8 phi, 9 G_l, 10 G_s,
 * 11 Koop log10 J_s, 12 omega (9 and 12 of the first liquid set), 13/14 lognormal median
 * radius and sigma_g of the (first) liquid set, 15/16 of the ice, 17/18 of the liquid of
 * heterogeneous origin (bimodal; 0 otherwise).  Source quantities use dt for the limiters
 * only. */
void or_derived(or_ctx *g, const double *U, int which, double dt, double *out) {
  const int nf = g->nf;
  int nx = g->nx, nr = g->nr;
  size_t N = (size_t)nx * nr;
  for (size_t n = 0; n < N; ++n) {
    double u14[NFMAX], Q[NFMAX], aux[11];
    for (int f = 0; f < nf; ++f) u14[f] = U[(size_t)f * N + n];
    prim_t w;
    cons_to_prim(u14, nf == NF_BI, &w);
    if (which == 0) { out[n] = w.T; continue; }
    if (which == 1) { out[n] = w.p; continue; }
    if (which >= 13) {
      /* lognormal size distribution with the cell's mu0, mu1, mu2 (Sec. 4.3's droplet
       * spectra): mu_k = N r_m^k exp(k^2 s^2 / 2) gives ln r_m = 2 ln(mu1/mu0) - ln(mu2/mu0)/2
       * and s^2 = ln(mu0 mu2 / mu1^2); radius in um, 0 without a population */
      const double *m = which <= 14 ? w.ml : (which <= 16 ? w.ms : w.mh);
      double v = 0.0;
      if (m[0] > MU_MIN && m[1] > 0.0 && m[2] > 0.0) {
        if (which == 13 || which == 15 || which == 17) v = exp(2.0 * log(m[1] / m[0]) - 0.5 * log(m[2] / m[0]));
        else {
          double s2 = log(m[0] * m[2] / (m[1] * m[1]));
          v = exp(sqrt(s2 > 0.0 ? s2 : 0.0));
        }
      }
      out[n] = v;
      continue;
    }
    phase_source(&w, NULL, dt, &g->sp, Q, aux);
    switch (which) {
      case 2: out[n] = aux[0]; break;
      case 3: out[n] = aux[1]; break;
      case 4: out[n] = aux[2] / log(10.0); break;
      case 5: out[n] = aux[3] / log(10.0); break;
      default: out[n] = aux[which - 2]; break;
    }
  }
}

/* Source of a batch of cells given conserved states (n x nf, row-major; nf = 18 for the
 * bimodal liquid, else 14), for pins and for the surrogate's training targets: Q out
 * (n x nf), aux out (n x 11). */
void or_source_batch(const or_case *c, const double *U, int n, double dt, double *Q, double *aux) {
  const int nf = c->bimodal ? NF_BI : NF;
  src_par_t sp;
  sp.phase_change = c->phase_change;
  sp.freezing = c->freezing;
  sp.n_soot_ref = c->n_soot;
  sp.tables = c->tables;
  sp.equilibrium = c->equilibrium;
  sp.bimodal = c->bimodal;
  build_tables();
  double ls = log(c->soot_sigma > 0.0 ? c->soot_sigma : 1.0);
  sp.rp2 = c->soot_rm * c->soot_rm * exp(2.0 * ls * ls);
  for (int m = 0; m < n; ++m) {
    prim_t w;
    cons_to_prim(U + (size_t)m * nf, c->bimodal, &w);
    phase_source(&w, NULL, dt, &sp, Q + (size_t)m * nf, aux + (size_t)m * 11);
  }
}

/* Conserved state from primitives (n rows of p, T, u, v, Y_v, ml0..3, ms0..3, ns). */
void or_prim_to_cons_batch(const double *P, int n, double *U) {
  for (int m = 0; m < n; ++m) {
    const double *q = P + (size_t)m * NF;
    prim_to_cons(q[0], q[1], q[2], q[3], q[4], q + 5, q + 9, q[13], U + (size_t)m * NF);
  }
}

/* Primitive quantities of conserved states: n rows -> (rho, u, v, p, T, Yv, Yl, Ys, c2). */
void or_cons_to_prim_batch(const double *U, int n, double *P) {
  for (int m = 0; m < n; ++m) {
    prim_t w;
    cons_to_prim(U + (size_t)m * NF, 0, &w);
    double *o = P + (size_t)m * 9;
    o[0] = w.rho; o[1] = w.u; o[2] = w.v; o[3] = w.p; o[4] = w.T;
    o[5] = w.Yv; o[6] = w.Yl; o[7] = w.Ys; o[8] = w.c2;
  }
}

/* Inflow and ambient states as built by the oracle (for BC tests). */
void or_boundary_states(or_ctx *g, double *inflow, double *amb) {
  if (inflow) memcpy(inflow, g->inflow, sizeof(double) * g->nf * g->nr);
  if (amb) memcpy(amb, g->amb, sizeof(double) * g->nf);
}

/* One residual evaluation (no time update) of state U, for pins: L out (nf x N),
 * bflux out (3). */
void or_residual(or_ctx *g, const double *U, double dt, double *L, double *bflux) {
  size_t N = (size_t)g->nx * g->nr;
  residual(g, U, dt);
  memcpy(L, g->L, sizeof(double) * g->nf * N);
  if (bflux) memcpy(bflux, g->bflux, sizeof(double) * 3);
}

int or_num_fields(void) { return NF; }
int or_num_diag(void) { return NDIAG; }
double or_const(int which) {
  switch (which) {
    case 0: return rv_gas();
    case 1: return RA;
    case 2: return cva();
    case 3: return cvv();
    case 4: return e0v();
    case 5: return e0s();
    case 6: return f_theta();
    case 7: return MU_MIN;
    default: return NAN;
  }
}
