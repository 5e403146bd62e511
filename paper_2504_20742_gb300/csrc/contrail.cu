// contrail.cu -- fused finite-volume stage kernels and the C ABI (include/contrail.h).
//
// One SSP-RK2 step (Sec. 3.2 of Tegethoff & Wheeler, arXiv 2504.20742) is two launches of
// one fused stage kernel.  Each CTA owns a TX x TY tile of cells and, in shared memory,
// the primitive variables of the tile plus a two-cell halo (boundary ghosts are built on
// the fly).  It computes the x-face and r-face Roe fluxes once per face, the flux
// divergence with the axisymmetric / area geometric sources, the per-cell phase-change
// source (limited on the flux-updated state), the RK combine, and block partials of the
// CFL time step and of the conservation diagnostics.  The last CTA to finish reduces
// the partials in a fixed order (deterministic) and publishes the next time step to the
// workspace, so that N steps run without any host round trip.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <cmath>

#include "../../include/contrail.h"
#include "flux.cuh"
#include "mlp_tc.cuh"
#include "physics.cuh"

namespace ct {

// ---- workspace layout ------------------------------------------------------------------
constexpr int NPART = 26;   // per-block partial record
// partial slots: 0 dt min, 1 M, 2 W, 3 E, 4..6 boundary inflow rate (mass, water, energy),
// 7 active, 8 non-finite, 9..22 max |dU/dt| per field, 23 max ln J_hom, 24 max ln J_het,
// 25 surrogate fallback count.
struct WsHeader {
  double dt_cur;          // time step of the next step
  double cfl;
  double b1[4];           // stage-1 boundary inflow rates
  double diag[CT_NDIAG];  // last completed step
  double steps;
  unsigned int counter;   // last-block-done ticket
  unsigned int setup_magic;
  int nblocks;
  int pad;
};
constexpr unsigned int SETUP_MAGIC = 0x43544231u;
constexpr size_t HDR_BYTES = 1024;
static_assert(sizeof(WsHeader) <= HDR_BYTES, "header");

struct DevCase {
  int geom, nx, nr, bc_xlo, bc_xhi, bc_rhi, jw, nblocks;
  double dx, dr, idx, idr, cfl;
  double area_a, x_throat, wall_len;
  double p0, T0, Yv0, cp0, gam0;       // nozzle inlet mixture
  float fdx, fidx, fdr, fidr, fwall_len, farea_a, fixt;   // FP32 copies of the geometry
  SrcCase sc;
  const double* inflow;   // nr x NF (plume)
  const double* amb;      // NF
  WsHeader* hdr;
  double* partials;       // nblocks x NPART
};

// Tile of TX x TY cells per CTA; NT = (TX+1)*TY... rounded to whole warps so that the
// x-face (33 x 8) and r-face (32 x 9) passes each take a single round of the CTA.
constexpr int TX = 32, TY = 8, NT = 288, NCELL = TX * TY;
constexpr int HX = TX + 4, HY = TY + 4;

// Geometry in the state precision (no double->float conversions inside FP32 kernels).
template <class T>
struct Geo {
  T dx, idx, dr, idr, wall_len, area_a, ixt;
};
__device__ __forceinline__ Geo<float> geo_of(const DevCase& d, float) {
  return {d.fdx, d.fidx, d.fdr, d.fidr, d.fwall_len, d.farea_a, d.fixt};
}
__device__ __forceinline__ Geo<double> geo_of(const DevCase& d, double) {
  return {d.dx, d.idx, d.dr, d.idr, d.wall_len, d.area_a, 1.0 / d.x_throat};
}

// ---- boundary ghost cells (Sec. 4.1; reading A1) ---------------------------------------
// Conserved state at (i, j), i in [-2, nx+1], j in [-2, nr+1], not both outside.
// Out of line on purpose: keeps the nozzle inlet's FP64 arithmetic from being hoisted into
// the interior path of the FP32 kernels.
template <class T>
__device__ __noinline__ void load_ghost(const DevCase& dc, const T* __restrict__ U, size_t N, int i, int j,
                                        T* u14) {
  const int nx = dc.nx, nr = dc.nr;
  if (i < 0) {
    if (dc.bc_xlo == 1) {   // wall: mirror
      const size_t n = (size_t)j * nx + (-i - 1);
#pragma unroll
      for (int f = 0; f < NF; ++f) u14[f] = U[f * N + n];
      u14[1] = -u14[1];
    } else if (dc.geom == 0) {   // total-condition subsonic inlet, interior velocity
      const size_t n = (size_t)j * nx;
      double u = double(U[N + n]) / double(U[n]);
      u = u < 0.0 ? 0.0 : u;
      const double Tg = dc.T0 - u * u / (2.0 * dc.cp0);
      const double p = dc.p0 * pow(Tg / dc.T0, dc.gam0 / (dc.gam0 - 1.0));
      const double z[4] = {0, 0, 0, 0};
      prim_to_cons<T>(p, Tg, u, 0.0, dc.Yv0, z, z, 0.0, u14);
    } else {   // plume inflow profile
#pragma unroll
      for (int f = 0; f < NF; ++f) u14[f] = T(dc.inflow[j * NF + f]);
    }
    return;
  }
  if (i >= nx) {
    const int ii = dc.bc_xhi == 1 ? 2 * nx - 1 - i : nx - 1;
    const size_t n = (size_t)j * nx + ii;
#pragma unroll
    for (int f = 0; f < NF; ++f) u14[f] = U[f * N + n];
    if (dc.bc_xhi == 1) u14[1] = -u14[1];
    return;
  }
  if (j < 0) {   // axis: mirror with rho*v negated
    const size_t n = (size_t)(-j - 1) * nx + i;
#pragma unroll
    for (int f = 0; f < NF; ++f) u14[f] = U[f * N + n];
    u14[2] = -u14[2];
    return;
  }
  if (j >= nr) {
    if (dc.bc_rhi == 0) {
#pragma unroll
      for (int f = 0; f < NF; ++f) u14[f] = T(dc.amb[f]);
    } else {
      const int jj = dc.bc_rhi == 1 ? 2 * nr - 1 - j : nr - 1;
      const size_t n = (size_t)jj * nx + i;
#pragma unroll
      for (int f = 0; f < NF; ++f) u14[f] = U[f * N + n];
      if (dc.bc_rhi == 1) u14[2] = -u14[2];
    }
    return;
  }
  const size_t n = (size_t)j * nx + i;
#pragma unroll
  for (int f = 0; f < NF; ++f) u14[f] = U[f * N + n];
}

__device__ __forceinline__ double area_q1d(const DevCase& dc, double x) {
  const double s = x / dc.x_throat - 1.0;
  return 1.0 + dc.area_a * s * s;
}

// ---- reductions -------------------------------------------------------------------------
template <class V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <class V>
__device__ __forceinline__ V warp_max(V v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    V w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}
template <class V>
__device__ __forceinline__ V warp_min(V v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    V w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  return v;
}
// kind: 0 sum, 1 max, 2 min
__device__ __forceinline__ int slot_kind(int q) { return q == 0 ? 2 : ((q >= 9 && q <= 24) ? 1 : 0); }

// Last CTA: reduce the partial records of all CTAs in a fixed order; returns true in the
// CTA that did it (red[] then holds the totals).
__device__ bool last_block_reduce(const DevCase& dc, double* red_smem) {
  __shared__ unsigned int ticket;
  __threadfence();   // every thread that wrote partials makes them visible device-wide
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(&dc.hdr->counter, 1u);
  __syncthreads();
  if (ticket != (unsigned int)(dc.nblocks - 1)) return false;
  __threadfence();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  for (int q = warp; q < NPART; q += nwarps) {
    const int kind = slot_kind(q);
    double acc = kind == 0 ? 0.0 : (kind == 1 ? -INFINITY : INFINITY);
    for (int b = lane; b < dc.nblocks; b += 32) {
      const double v = __ldcg(&dc.partials[(size_t)b * NPART + q]);
      acc = kind == 0 ? acc + v : (kind == 1 ? fmax(acc, v) : fmin(acc, v));
    }
    acc = kind == 0 ? warp_sum(acc) : (kind == 1 ? warp_max(acc) : warp_min(acc));
    if (lane == 0) red_smem[q] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) dc.hdr->counter = 0u;
  return true;
}

// ---- the fused stage kernel ---------------------------------------------------------------
// STAGE 1: Uout = Uin + dt L(Uin).  STAGE 2: Uout = (Un + Uin + dt L(Uin))/2 (Uout may be Un).
constexpr int NFACE = (TX + 1) * TY > TX * (TY + 1) ? (TX + 1) * TY : TX * (TY + 1);
template <class T>
constexpr size_t stage_smem() { return sizeof(T) * (size_t)NF * (HX * HY + 3 * NFACE); }
// shared memory of the surrogate phase, reusing the (then dead) stencil buffers:
// activations, streamed weights, outputs, blob header, TMEM slot, mbarrier
constexpr size_t SM_A = 0, SM_W = SM_A + mlp::ABYTES, SM_OUT = SM_W + 32768, SM_HDR = SM_OUT + 128 * 10 * 4,
                 SM_TSLOT = SM_HDR + mlp::NFLOAT * 4, SM_MBAR = SM_TSLOT + 16, SM_RES = SM_MBAR + 16,
                 SURR_SMEM = SM_RES + 288 * 10 * 4;
constexpr size_t stage_smem_surr() { return stage_smem<float>() > SURR_SMEM ? stage_smem<float>() : SURR_SMEM; }

// Surrogate cells of one tile (called by all threads, only when the tile has at least one):
// compaction into 128-row tiles and the BF16 tensor-core network.  Each surrogate cell's
// thread finds its 10 outputs (raw units, held to the training range of their targets) in
// res[10 * threadIdx.x ...] afterwards.  x: the cell's 16 raw inputs (kind == 2 only).
__device__ __noinline__ void surrogate_tile(const unsigned char* __restrict__ blob, int kind, const float* x, int& nbad,
                                            unsigned char* smem) {
  __shared__ int wcnt[NT / 32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float* ghdr = reinterpret_cast<const float*>(blob);
  const unsigned mask = __ballot_sync(0xffffffffu, kind == 2);
  if (lane == 0) wcnt[warp] = __popc(mask);
  __syncthreads();
  int off = 0, total = 0;
  for (int w2 = 0; w2 < NT / 32; ++w2) {
    off += w2 < warp ? wcnt[w2] : 0;
    total += wcnt[w2];
  }
  const int row = off + __popc(mask & ((1u << lane) - 1u));
  unsigned char* A = smem + SM_A;
  unsigned char* W = smem + SM_W;
  float* outs = reinterpret_cast<float*>(smem + SM_OUT);
  float* hdr = reinterpret_cast<float*>(smem + SM_HDR);
  float* res = reinterpret_cast<float*>(smem + SM_RES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + SM_TSLOT);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + SM_MBAR);
  for (int q = tid; q < mlp::NFLOAT; q += NT) hdr[q] = ghdr[q];
  if (warp == 0) {
    tc::tmem_alloc(tc::smem_addr(tslot), 128);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(tc::smem_addr(mbar), 1);
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  uint32_t phase = 0;
  bool ok = true;
  for (int c0 = 0; c0 < total; c0 += 128) {
    const bool mine = kind == 2 && row >= c0 && row < c0 + 128;
    if (mine) {
      float v[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = (x[q] - hdr[mlp::F_XMEAN + q]) * hdr[mlp::F_XISD + q];
      mlp::store_row16(A, row - c0, 0, 16, v);
    }
    float o[10];
    ok = mlp::run_tile<true>(A, W, hdr + mlp::F_BIAS, tmem, tc::smem_addr(mbar), phase, o, blob + mlp::WOFF,
                             total - c0) && ok;
    if (tid < 128) {
#pragma unroll
      for (int q = 0; q < 10; ++q) outs[tid * 10 + q] = o[q] * hdr[mlp::F_YSD + q] + hdr[mlp::F_YMEAN + q];
    }
    __syncthreads();
    if (mine) {
#pragma unroll
      for (int q = 0; q < 10; ++q)
        res[tid * 10 + q] = fminf(fmaxf(outs[(row - c0) * 10 + q], hdr[mlp::F_YMIN + q]), hdr[mlp::F_YMAX + q]);
    }
    __syncthreads();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 128);
  if (!ok && tid == 0) nbad += 1;   // a tensor-core wait timed out: the step reports failure
}

// Source of the FP32 + surrogate path (called by all threads): active cells inside the
// surrogate's training hull take their rates from the network, the others the plain source
// (counted as fallbacks); both feed the plain path's tail, so conservation and the limiters
// are exact.  Adds the source to acc.
template <class T>
__device__ __forceinline__ void surrogate_source(const DevCase& dc, const unsigned char* __restrict__ blob, bool cell,
                                                 const Prim<T>& w, const T* u14, T* acc, T dt, int& nactive,
                                                 int& nfallback, int& nbad, T& lnJh, T& lnJt, unsigned char* smem) {
  const float* ghdr = reinterpret_cast<const float*>(blob);
  int kind = 0;   // 0 inactive, 1 plain source (outside the hull), 2 surrogate
  Sat<T> st;
  st.lnSl = st.lnSi = st.lnpv = 0.0;
  st.pres_l = st.pres_s = st.active = false;
  T Q[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) Q[f] = T(0);
  double lnJ2[2] = {-INFINITY, -INFINITY};
  float x[CT_MLP_IN];
  if (cell && dc.sc.phase_change) {
    bool pl, ps;
    const bool pops = populations(w, pl, ps);
    if (pops || !clearly_inactive(w)) {
      st = saturation(w);
      if (st.active) {
        mlp_features<T>(w, st, dc.sc.rp2, x);
        bool inside = true;
#pragma unroll
        for (int q = 0; q < CT_MLP_IN; ++q)
          inside = inside && x[q] >= ghdr[mlp::F_HMIN + q] && x[q] <= ghdr[mlp::F_HMAX + q];
        kind = inside ? 2 : 1;
      }
    }
  }
  if (kind == 1) {
    const Rates<T> r = plain_rates<T>(w, st, dc.sc, lnJ2, nullptr, nullptr);
    source_tail<T>(w, u14, acc, dt, dc.sc, st.pres_l, st.pres_s, st.lnSl, st.lnSi, r, Q, nullptr);
    nfallback = 1;
  }
  // the stencil buffers are dead from here on; tiles without a surrogate cell skip the rest
  if (__syncthreads_or(kind == 2)) {
    surrogate_tile(blob, kind, x, nbad, smem);
    if (kind == 2) {
      const float* y = reinterpret_cast<const float*>(smem + SM_RES) + 10 * threadIdx.x;
      const bool nuc = st.lnSl > 0.0;
      Rates<T> r;
      r.Jeff = nuc ? T(__expf(y[0])) : T(0);
      // the Kelvin radius of Eq. (3) is a closed form: evaluated, not predicted
      r.rc_um = nuc ? T(2.0f * sigma_liq<float>(float(w.Tg)) * 1e6f /
                        (float(k::RHOL * k::RV) * float(w.Tg) * float(st.lnSl)))
                    : T(0);
      r.Gl = st.pres_l ? T(MLP_G0 * sinhf(y[2])) : T(0);
      r.Gs = st.pres_s ? T(MLP_G0 * sinhf(y[3])) : T(0);
      r.xl = st.pres_l ? T(__expf(y[4])) : T(0);
      r.xs = st.pres_s ? T(__expf(y[5])) : T(0);
      if (nuc) {
        lnJ2[0] = y[6];
        if (dc.sc.n_soot_ref > 0.0 && w.rho * w.ns > T(0)) lnJ2[1] = y[7];
      }
      source_tail<T>(w, u14, acc, dt, dc.sc, st.pres_l, st.pres_s, st.lnSl, st.lnSi, r, Q, nullptr);
    }
  }
  if (cell) {
    nactive = kind != 0 ? 1 : 0;
    lnJh = T(lnJ2[0]);
    lnJt = T(lnJ2[1]);
#pragma unroll
    for (int f = 4; f < 13; ++f) acc[f] += Q[f];
  }
}

template <class T, int STAGE, bool SURR>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1)
    k_stage(DevCase dc, const T* __restrict__ Uin, const T* Un, T* Uout, const unsigned char* __restrict__ blob) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T (*qs)[HY][HX] = reinterpret_cast<T (*)[HY][HX]>(smem_raw);                      // primitives
  T (*fb)[NFACE] = reinterpret_cast<T (*)[NFACE]>(smem_raw + sizeof(T) * NF * HX * HY);   // face fluxes
  T (*fL)[NFACE] = fb + NF;        // reconstructed left state of each face
  T (*fR)[NFACE] = fb + 2 * NF;    // reconstructed right state of each face
  __shared__ double red[NT / 32][NPART];
  __shared__ double fin[NPART];

  const int nx = dc.nx, nr = dc.geom == 1 ? dc.nr : 1;
  const size_t N = (size_t)nx * nr;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int tid = threadIdx.x;
  const double dtd = dc.hdr->dt_cur;
  const T dt = T(dtd);
  const Geo<T> g = geo_of(dc, T(0));

  // phase A: halo primitives
  for (int p = tid; p < HX * HY; p += NT) {
    const int hi = p % HX, hj = p / HX;
    const int i = i0 + hi - 2, j = j0 + hj - 2;
    const bool xin = i >= 0 && i < nx, rin = j >= 0 && j < nr;
    bool need = (xin || rin) && i >= -2 && i <= nx + 1 && j >= -2 && j <= nr + 1;
    if (dc.geom == 0) need = need && j == 0;
    if (!need) continue;
    T u14[NF];
    if (xin && rin) {
      const size_t n = (size_t)j * nx + i;
#pragma unroll
      for (int f = 0; f < NF; ++f) u14[f] = Uin[f * N + n];
    } else {
      load_ghost<T>(dc, Uin, N, i, j, u14);
    }
    Prim<T> w;
    cons_to_prim<T>(u14, w);
    qs[0][hj][hi] = w.rho;
    qs[1][hj][hi] = w.u;
    qs[2][hj][hi] = w.v;
    qs[3][hj][hi] = w.p;
    qs[4][hj][hi] = w.Yv;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      qs[5 + q][hj][hi] = w.ml[q];
      qs[9 + q][hj][hi] = w.ms[q];
    }
    qs[13][hj][hi] = w.ns;
  }
  __syncthreads();

  // phase B1: limited x slopes, once per cell, written as the states of its two faces
  // (tile-local cell c in [-1, TX]; face f lies between cells f-1 and f)
  for (int p = tid; p < (TX + 2) * TY; p += NT) {
    const int c = p % (TX + 2) - 1, hj = p / (TX + 2);
    const int i = i0 + c, j = j0 + hj;
    if (i > nx || j >= nr) continue;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const T am = qs[f][hj + 2][c + 1], a0 = qs[f][hj + 2][c + 2], a1 = qs[f][hj + 2][c + 3];
      const T hs = T(0.5) * vl_slope(a0 - am, a1 - a0);
      if (c < TX) fL[f][hj * (TX + 1) + c + 1] = a0 + hs;
      if (c >= 0) fR[f][hj * (TX + 1) + c] = a0 - hs;
    }
  }
  __syncthreads();

  // phase B2: x-face Roe fluxes
  for (int p = tid; p < (TX + 1) * TY; p += NT) {
    const int fx = p % (TX + 1), hj = p / (TX + 1);
    const int i = i0 + fx, j = j0 + hj;
    if (i > nx || j >= nr) continue;
    T qL[NF], qR[NF], F[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      qL[f] = fL[f][p];
      qR[f] = fR[f][p];
    }
    roe_flux<T, 0>(qL, qR, F);
#pragma unroll
    for (int f = 0; f < NF; ++f) fb[f][p] = F[f];
  }
  __syncthreads();

  const int ci = tid % TX, cj = tid / TX;
  const int i = i0 + ci, j = j0 + cj;
  const bool cell = tid < NCELL && i < nx && j < nr;
  T acc[NF];
  T bm = T(0), bw = T(0), be = T(0);   // boundary inflow rates of this cell's faces
  T area_w = T(0), area_e = T(0), vol = T(0);
  if (cell) {
    const int w = cj * (TX + 1) + ci, e = w + 1;
    T cw, ce;
    if (dc.geom == 0) {
      const T xw = T(i) * g.dx, xe = T(i + 1) * g.dx, xc = (T(i) + T(0.5)) * g.dx;
      const T sw = xw * g.ixt - T(1), se = xe * g.ixt - T(1), sc = xc * g.ixt - T(1);
      area_w = T(1) + g.area_a * sw * sw;
      area_e = T(1) + g.area_a * se * se;
      const T Ac = T(1) + g.area_a * sc * sc;
      const T iv = frcp(Ac * g.dx);
      cw = area_w * iv;
      ce = area_e * iv;
      vol = Ac * g.dx;
    } else {
      cw = ce = g.idx;
      area_w = area_e = (T(j) + T(0.5)) * g.dr * g.dr;
      vol = area_w * g.dx;
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) acc[f] = cw * fb[f][w] - ce * fb[f][e];
    if (i == 0) {
      bm += area_w * fb[0][w];
      bw += area_w * (fb[4][w] + T(k::YL3) * fb[8][w] + T(k::YS3) * fb[12][w]);
      be += area_w * fb[3][w];
    }
    if (i == nx - 1) {
      bm -= area_e * fb[0][e];
      bw -= area_e * (fb[4][e] + T(k::YL3) * fb[8][e] + T(k::YS3) * fb[12][e]);
      be -= area_e * fb[3][e];
    }
  }

  if (dc.geom == 1) {
    __syncthreads();
    // phase D1: limited r slopes (tile-local row c in [-1, TY]) -> states of the r faces
    for (int p = tid; p < TX * (TY + 2); p += NT) {
      const int hi = p % TX, c = p / TX - 1;
      const int ii = i0 + hi, jj = j0 + c;
      if (ii >= nx || jj > nr) continue;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const T am = qs[f][c + 1][hi + 2], a0 = qs[f][c + 2][hi + 2], a1 = qs[f][c + 3][hi + 2];
        const T hs = T(0.5) * vl_slope(a0 - am, a1 - a0);
        if (c < TY) fL[f][(c + 1) * TX + hi] = a0 + hs;
        if (c >= 0) fR[f][c * TX + hi] = a0 - hs;
      }
    }
    __syncthreads();
    // phase D2: r-face Roe fluxes (face fy lies between tile rows fy-1 and fy)
    for (int p = tid; p < TX * (TY + 1); p += NT) {
      const int hi = p % TX, fy = p / TX;
      const int ii = i0 + hi, jj = j0 + fy;
      if (ii >= nx || jj > nr) continue;
      T qL[NF], qR[NF], F[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        qL[f] = fL[f][p];
        qR[f] = fR[f][p];
      }
      roe_flux<T, 1>(qL, qR, F);
#pragma unroll
      for (int f = 0; f < NF; ++f) fb[f][p] = F[f];
    }
    __syncthreads();
  }

  // phase E: residual, source, update, partial reductions
  T pM = T(0), pW = T(0), pE = T(0);
  T dtmin = T(INFINITY);
  T rmax[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) rmax[f] = T(0);
  T lnJh = T(-INFINITY), lnJt = T(-INFINITY);
  int nactive = 0, nbad = 0, nfallback = 0;
  T u14[NF];
  Prim<T> w;
  if (cell) {
    const size_t n = (size_t)j * nx + i;
#pragma unroll
    for (int f = 0; f < NF; ++f) u14[f] = Uin[f * N + n];
    cons_to_prim<T>(u14, w);
    if (dc.geom == 1) {
      const T ijh = frcp(T(j) + T(0.5));
      const T cs = T(j) * ijh * g.idr, cn = T(j + 1) * ijh * g.idr;
      const bool wall = g.wall_len > T(0) && (T(i) + T(0.5)) * g.dx < g.wall_len;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        T Fs = fb[f][cj * TX + ci], Fn = fb[f][(cj + 1) * TX + ci];
        if (wall && j == dc.jw - 1) Fn = f == 2 ? w.p : T(0);
        if (wall && j == dc.jw) Fs = f == 2 ? w.p : T(0);
        acc[f] += cs * Fs - cn * Fn;
      }
      acc[2] += w.p * ijh * g.idr;
      if (j == nr - 1) {
        const T An = T(nr) * g.dr * g.dx;
        const int e = (cj + 1) * TX + ci;
        bm -= An * fb[0][e];
        bw -= An * (fb[4][e] + T(k::YL3) * fb[8][e] + T(k::YS3) * fb[12][e]);
        be -= An * fb[3][e];
      }
    } else {
      acc[1] += w.p * fdiv(area_e - area_w, vol);
    }
    // phase-change source limited on the flux-updated state
    T Q[NF];
    double lnJ2[2];
    if (!SURR) {
      const bool act = phase_source<T>(w, u14, acc, dt, dc.sc, Q, lnJ2, nullptr);
      nactive = act ? 1 : 0;
      lnJh = T(lnJ2[0]);
      lnJt = T(lnJ2[1]);
#pragma unroll
      for (int f = 4; f < 13; ++f) acc[f] += Q[f];
    }
  }
  if (SURR) surrogate_source<T>(dc, blob, cell, w, u14, acc, dt, nactive, nfallback, nbad, lnJh, lnJt, smem_raw);
  if (cell) {
    const size_t n = (size_t)j * nx + i;
    // RK combine
    T out[NF];
    if (STAGE == 1) {
#pragma unroll
      for (int f = 0; f < NF; ++f) out[f] = u14[f] + dt * acc[f];
    } else {
      const T idt = frcp(dt);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const T un = Un[f * N + n];
        out[f] = T(0.5) * un + T(0.5) * (u14[f] + dt * acc[f]);
        rmax[f] = m_fabs(out[f] - un) * idt;
      }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      Uout[f * N + n] = out[f];
      nbad += isfinite(out[f]) ? 0 : 1;
    }
    if (STAGE == 2) {
      Prim<T> wn;
      cons_to_prim<T>(out, wn);
      const T c = m_sqrt(wn.c2);
      T rate = (m_fabs(wn.u) + c) * g.idx;
      if (dc.geom == 1) rate += (m_fabs(wn.v) + c) * g.idr;
      dtmin = T(1) / rate;   // times cfl at the end
      pM = vol * out[0];
      pW = vol * (out[4] + T(k::YL3) * out[8] + T(k::YS3) * out[12]);
      pE = vol * out[3];
    }
  }

  // block partials: warp shuffles in the state precision, FP64 from the warp level on
  const int warp = tid >> 5, lane = tid & 31;
  {
    T v;
    v = warp_min(dtmin); if (lane == 0) red[warp][0] = double(v);
    v = warp_sum(pM); if (lane == 0) red[warp][1] = double(v);
    v = warp_sum(pW); if (lane == 0) red[warp][2] = double(v);
    v = warp_sum(pE); if (lane == 0) red[warp][3] = double(v);
    v = warp_sum(bm); if (lane == 0) red[warp][4] = double(v);
    v = warp_sum(bw); if (lane == 0) red[warp][5] = double(v);
    v = warp_sum(be); if (lane == 0) red[warp][6] = double(v);
    int a = warp_sum(nactive); if (lane == 0) red[warp][7] = a;
    a = warp_sum(nbad); if (lane == 0) red[warp][8] = a;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      v = warp_max(rmax[f]);
      if (lane == 0) red[warp][9 + f] = double(v);
    }
    v = warp_max(lnJh); if (lane == 0) red[warp][23] = double(v);
    v = warp_max(lnJt); if (lane == 0) red[warp][24] = double(v);
    a = warp_sum(nfallback); if (lane == 0) red[warp][25] = a;
  }
  __syncthreads();
  if (tid < NPART) {
    const int kind = slot_kind(tid);
    double acc2 = red[0][tid];
    for (int w2 = 1; w2 < NT / 32; ++w2) {
      const double v = red[w2][tid];
      acc2 = kind == 0 ? acc2 + v : (kind == 1 ? fmax(acc2, v) : fmin(acc2, v));
    }
    const int b = blockIdx.y * gridDim.x + blockIdx.x;
    dc.partials[(size_t)b * NPART + tid] = acc2;
  }
  if (!last_block_reduce(dc, fin)) return;
  if (tid == 0) {
    WsHeader* h = dc.hdr;
    if (STAGE == 1) {
      h->b1[0] = fin[4];
      h->b1[1] = fin[5];
      h->b1[2] = fin[6];
    } else {
      double* d = h->diag;
      d[0] = dtd;
      d[1] = fin[1];
      d[2] = fin[2];
      d[3] = fin[3];
      d[4] = 0.5 * dtd * (h->b1[0] + fin[4]);
      d[5] = 0.5 * dtd * (h->b1[1] + fin[5]);
      d[6] = 0.5 * dtd * (h->b1[2] + fin[6]);
      d[7] = fin[7];
      d[8] = fin[8];
      for (int f = 0; f < NF; ++f) d[9 + f] = fin[9 + f];
      d[23] = fin[23] * (1.0 / 2.302585092994045684);
      d[24] = fin[24] * (1.0 / 2.302585092994045684);
      const double dtn = dc.cfl * fin[0];
      d[25] = dtn;
      d[26] = fin[25];
      h->steps += 1.0;
      d[27] = h->steps;
      h->dt_cur = dtn;
    }
  }
}

// ---- time step of a given state (initial step / after a load) --------------------------
template <class T>
__global__ void __launch_bounds__(NT) k_dt(DevCase dc, const T* __restrict__ U) {
  __shared__ double red[NT / 32][NPART];
  __shared__ double fin[NPART];
  const int nx = dc.nx, nr = dc.geom == 1 ? dc.nr : 1;
  const size_t N = (size_t)nx * nr;
  T dtmin = T(INFINITY);
  for (size_t n = (size_t)blockIdx.x * NT + threadIdx.x; n < N; n += (size_t)gridDim.x * NT) {
    T u14[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) u14[f] = U[f * N + n];
    Prim<T> w;
    cons_to_prim<T>(u14, w);
    const T c = m_sqrt(w.c2);
    T rate = (m_fabs(w.u) + c) * T(dc.idx);
    if (dc.geom == 1) rate += (m_fabs(w.v) + c) * T(dc.idr);
    const T d = T(1) / rate;
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

__global__ void k_setup(ct_case c, const double* __restrict__ ufac, double* inflow, double* amb, int nr, double dr) {
  for (int j = threadIdx.x; j < nr; j += blockDim.x)
    inflow_cons(c, (j + 0.5) * dr, ufac ? ufac[j] : 1.0, inflow + (size_t)j * NF);
  if (threadIdx.x == 0) ambient_cons(c, 1.0, amb);
}

// ---- initial state -----------------------------------------------------------------------
__device__ double area_mach(double M, double g) {
  return 1.0 / M * pow(2.0 / (g + 1.0) * (1.0 + 0.5 * (g - 1.0) * M * M), 0.5 * (g + 1.0) / (g - 1.0));
}

template <class T>
__global__ void k_init(ct_case c, DevCase dc, T* __restrict__ U) {
  const int nx = dc.nx, nr = dc.geom == 1 ? dc.nr : 1;
  const size_t N = (size_t)nx * nr;
  for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
    const int i = int(n % nx), j = int(n / nx);
    double u14[NF];
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
      for (int f = 0; f < NF; ++f) u14[f] = dc.inflow[(size_t)j * NF + f];
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
    for (int f = 0; f < NF; ++f) U[f * N + n] = T(u14[f]);
  }
}

// ---- derived per-cell quantities and pointwise sources ------------------------------------
template <class T>
__global__ void k_derived(DevCase dc, const T* __restrict__ U, int which, double dt, double* __restrict__ out) {
  const int nx = dc.nx, nr = dc.geom == 1 ? dc.nr : 1;
  const size_t N = (size_t)nx * nr;
  for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
    T u14[NF], Q[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) u14[f] = U[f * N + n];
    Prim<T> w;
    cons_to_prim<T>(u14, w);
    if (which == 0) { out[n] = double(w.Tg); continue; }
    if (which == 1) { out[n] = double(w.p); continue; }
    double aux[NAUX], lnJ2[2];
    phase_source<T>(w, u14, nullptr, T(dt), dc.sc, Q, lnJ2, aux);
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

template <class T>
__global__ void k_source_batch(SrcCase sc, const double* __restrict__ U, int n, double dt, double* __restrict__ Qo,
                               double* __restrict__ auxo) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    T u14[NF], Q[NF];
    for (int f = 0; f < NF; ++f) u14[f] = T(U[(size_t)m * NF + f]);
    Prim<T> w;
    cons_to_prim<T>(u14, w);
    double aux[NAUX], lnJ2[2];
    phase_source<T>(w, u14, nullptr, T(dt), sc, Q, lnJ2, aux);
    for (int f = 0; f < NF; ++f) Qo[(size_t)m * NF + f] = (f >= 4 && f <= 12) ? double(Q[f]) : 0.0;
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
    const Sat<double> st = saturation(w);
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
static int tiles_x(const ct_case* c) { return (c->nx + TX - 1) / TX; }
static int tiles_y(const ct_case* c) { return (case_nr(c) + TY - 1) / TY; }
static int num_blocks(const ct_case* c) { return tiles_x(c) * tiles_y(c); }

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
  return CT_OK;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

static size_t ws_bytes(const ct_case* c) {
  const size_t nr = (size_t)case_nr(c);
  size_t b = HDR_BYTES;
  b += align256(nr * NF * sizeof(double));
  b += align256(NF * sizeof(double));
  b += align256((size_t)num_blocks(c) * NPART * sizeof(double));
  return b;
}

static DevCase make_dev(const ct_case* c, void* work) {
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
  d.sc.n_soot_ref = c->n_soot;
  const double ls = std::log(c->soot_sigma > 0.0 ? c->soot_sigma : 1.0);
  d.sc.rp2 = c->soot_rm * c->soot_rm * std::exp(2.0 * ls * ls);
  d.sc.phase_change = c->phase_change;
  d.sc.freezing = c->freezing;
  char* base = (char*)work;
  d.hdr = (WsHeader*)base;
  size_t off = HDR_BYTES;
  d.inflow = (const double*)(base + off);
  off += align256((size_t)d.nr * NF * sizeof(double));
  d.amb = (const double*)(base + off);
  off += align256(NF * sizeof(double));
  d.partials = (double*)(base + off);
  d.nblocks = num_blocks(c);
  return d;
}

extern "C" {

size_t ct_workspace_bytes(const ct_case* c, int precision) {
  if (validate(c, precision) != CT_OK) return 0;
  return ws_bytes(c);
}

ct_status ct_setup(const ct_case* c, int precision, const double* ufac_rows_host, void* work, size_t work_bytes,
                   void* stream) {
  ct_status s = validate(c, precision);
  if (s != CT_OK) return s;
  if (!work) return fail(CT_ERR_ARG, "null workspace");
  if (((uintptr_t)work & 255) != 0) return fail(CT_ERR_ARG, "workspace must be 256-byte aligned");
  if (work_bytes < ws_bytes(c)) return fail(CT_ERR_SIZE, "workspace too small (see ct_workspace_bytes)");
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
  if (c->geom == 1) k_setup<<<1, 256, 0, st>>>(*c, ufac_dev, (double*)d.inflow, (double*)d.amb, d.nr, d.dr);
  // the header copy and the profile kernel read host memory that must outlive them
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check("ct_setup sync");
  return cuda_check("ct_setup");
}

static ct_status check_setup(const ct_case* c, void* work, void* stream) {
  (void)c;
  (void)stream;
  if (!work) return fail(CT_ERR_ARG, "null workspace");
  return CT_OK;
}

static ct_status launch_dt(const ct_case* c, int precision, void* work, const void* U, double cfl, cudaStream_t st) {
  DevCase d = make_dev(c, work);
  d.cfl = cfl;
  const size_t N = (size_t)c->nx * case_nr(c);
  int grid = (int)std::min<size_t>((N + NT - 1) / NT, (size_t)d.nblocks);
  d.nblocks = grid;
  if (precision == CT_FP64) k_dt<double><<<grid, NT, 0, st>>>(d, (const double*)U);
  else k_dt<float><<<grid, NT, 0, st>>>(d, (const float*)U);
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
  if (precision == CT_FP64) k_init<double><<<grid, 256, 0, st>>>(*c, d, (double*)U);
  else k_init<float><<<grid, 256, 0, st>>>(*c, d, (float*)U);
  if ((s = cuda_check("k_init")) != CT_OK) return s;
  return launch_dt(c, precision, work, U, cfl, st);
}

ct_status ct_load_state(const ct_case* c, int precision, void* work, const void* U_src, void* U, double cfl,
                        void* stream) {
  ct_status s = validate(c, precision);
  if (s != CT_OK) return s;
  if (!U || !U_src) return fail(CT_ERR_ARG, "null state");
  if (!(cfl > 0.0 && cfl <= 1.0)) return fail(CT_ERR_ARG, "cfl must be in (0, 1]");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t N = (size_t)c->nx * case_nr(c);
  const size_t bytes = N * NF * (precision == CT_FP64 ? sizeof(double) : sizeof(float));
  if (U_src != U && cudaMemcpyAsync(U, U_src, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return cuda_check("ct_load_state copy");
  return launch_dt(c, precision, work, U, cfl, st);
}

static bool g_attr_done[3] = {false, false, false};

static ct_status set_stage_attrs(int precision) {
  const int p = precision == CT_FP64 ? 0 : (precision == CT_FP32 ? 1 : 2);
  if (g_attr_done[p]) return CT_OK;
  cudaError_t e;
  if (p == 0) {
    e = cudaFuncSetAttribute(k_stage<double, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)stage_smem<double>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_stage<double, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)stage_smem<double>());
  } else if (p == 1) {
    e = cudaFuncSetAttribute(k_stage<float, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)stage_smem<float>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_stage<float, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)stage_smem<float>());
  } else {
    e = cudaFuncSetAttribute(k_stage<float, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)stage_smem_surr());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_stage<float, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)stage_smem_surr());
  }
  if (e != cudaSuccess) return fail(CT_ERR_CUDA, cudaGetErrorString(e));
  g_attr_done[p] = true;
  return CT_OK;
}

static ct_status enqueue_steps(const ct_case* c, int precision, void* U, void* U1, void* work, int nsteps, double cfl,
                               cudaStream_t st, const void* blob = nullptr) {
  ct_status s = set_stage_attrs(precision);
  if (s != CT_OK) return s;
  DevCase d = make_dev(c, work);
  d.cfl = cfl;
  dim3 grid(tiles_x(c), tiles_y(c));
  const unsigned char* b = (const unsigned char*)blob;
  for (int k2 = 0; k2 < nsteps; ++k2) {
    if (precision == CT_FP64) {
      const size_t sm = stage_smem<double>();
      k_stage<double, 1, false><<<grid, NT, sm, st>>>(d, (const double*)U, nullptr, (double*)U1, nullptr);
      k_stage<double, 2, false><<<grid, NT, sm, st>>>(d, (const double*)U1, (const double*)U, (double*)U, nullptr);
    } else if (precision == CT_FP32) {
      const size_t sm = stage_smem<float>();
      k_stage<float, 1, false><<<grid, NT, sm, st>>>(d, (const float*)U, nullptr, (float*)U1, nullptr);
      k_stage<float, 2, false><<<grid, NT, sm, st>>>(d, (const float*)U1, (const float*)U, (float*)U, nullptr);
    } else {
      const size_t sm = stage_smem_surr();
      k_stage<float, 1, true><<<grid, NT, sm, st>>>(d, (const float*)U, nullptr, (float*)U1, b);
      k_stage<float, 2, true><<<grid, NT, sm, st>>>(d, (const float*)U1, (const float*)U, (float*)U, b);
    }
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
  return enqueue_steps(c, CT_FP32_MLP, U, U1, work, nsteps, cfl, (cudaStream_t)stream, blob);
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
  return enqueue_steps(c, precision, U, U1, work, nsteps, cfl, (cudaStream_t)stream);
}

ct_status ct_step_host(const ct_case* c, int precision, const void* U_host_in, void* U_host_out, void* U, void* U1,
                       void* work, int nsteps, double cfl, void* stream) {
  ct_status s = validate(c, precision);
  if (s != CT_OK) return s;
  if (!U_host_in || !U_host_out) return fail(CT_ERR_ARG, "null host buffer");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t N = (size_t)c->nx * case_nr(c);
  const size_t bytes = N * NF * (precision == CT_FP64 ? sizeof(double) : sizeof(float));
  if (cudaMemcpyAsync(U, U_host_in, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return cuda_check("h2d");
  if ((s = launch_dt(c, precision, work, U, cfl, st)) != CT_OK) return s;
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
  return CT_OK;
}

ct_status ct_derived(const ct_case* c, int precision, const void* U, int which, double dt, double* out, void* stream) {
  ct_status s = validate(c, precision);
  if (s != CT_OK) return s;
  if (!U || !out) return fail(CT_ERR_ARG, "null buffer");
  if (which < 0 || which > 12) return fail(CT_ERR_ARG, "which out of range [0, 12]");
  if (!(dt > 0.0)) return fail(CT_ERR_ARG, "dt must be > 0");
  cudaStream_t st = (cudaStream_t)stream;
  DevCase d = make_dev(c, nullptr);
  const size_t N = (size_t)c->nx * case_nr(c);
  int grid = (int)std::min<size_t>((N + 255) / 256, 8192);
  if (precision == CT_FP64) k_derived<double><<<grid, 256, 0, st>>>(d, (const double*)U, which, dt, out);
  else k_derived<float><<<grid, 256, 0, st>>>(d, (const float*)U, which, dt, out);
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
  if (precision == CT_FP64) k_source_batch<double><<<grid, 256, 0, st>>>(d.sc, U, n, dt, Q, aux);
  else k_source_batch<float><<<grid, 256, 0, st>>>(d.sc, U, n, dt, Q, aux);
  return cuda_check("k_source_batch");
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
static void* g_static_ptr[MAX_DEVICES];   // device address of g_static_scratch, per device

__global__ void k_scratch_reset(int nblocks) {
  // everything of the header that must start at zero for a fresh run
  WsHeader* h = reinterpret_cast<WsHeader*>(g_static_scratch);
  if (threadIdx.x == 0) {
    memset(h, 0, sizeof(WsHeader));
    h->setup_magic = SETUP_MAGIC;
    h->nblocks = nblocks;
  }
}

static ct_status static_scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cuda_check("cudaGetDevice");
  if (dev < 0 || dev >= MAX_DEVICES) return fail(CT_ERR_ARG, "device index beyond the static scratch table");
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
             "case needs %zu bytes of scratch but the static scratch holds %zu (about %d tiles of %dx%d cells); "
             "use ct_step with a caller workspace",
             need, STATIC_SCRATCH_BYTES, (int)((STATIC_SCRATCH_BYTES - HDR_BYTES) / (NPART * sizeof(double))), TX, TY);
    return CT_ERR_SIZE;
  }
  void* work = nullptr;
  if ((s = static_scratch_address(&work)) != CT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  DevCase d = make_dev(c, work);
  k_scratch_reset<<<1, 32, 0, st>>>(d.nblocks);
  if (c->geom == 1) k_setup<<<1, 256, 0, st>>>(*c, ufac_rows_dev, (double*)d.inflow, (double*)d.amb, d.nr, d.dr);
  if ((s = cuda_check("ct_step_static setup")) != CT_OK) return s;
  if ((s = launch_dt(c, precision, work, U, cfl, st)) != CT_OK) return s;
  return enqueue_steps(c, precision, U, U1, work, nsteps, cfl, st);
}

ct_status ct_mlp_dataset(const ct_case* c, const double* U, int n, float* X, float* Y, float* M, void* stream) {
  ct_status s = validate(c, CT_FP64);
  if (s != CT_OK) return s;
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
