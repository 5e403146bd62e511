// stage.cuh -- the fused finite-volume stage (one SSP-RK2 stage of Sec. 3.2 of Tegethoff &
// Wheeler, arXiv 2504.20742), templated on the tile shape, and its two launch forms: one CTA
// per tile of one case (k_stage), and persistent CTAs over a work list of the tiles of many
// cases (k_batch_stage).
//
// Each CTA owns a TX x TY tile of cells and, in shared memory, the primitive variables of
// the tile plus a two-cell halo (boundary ghosts are built on the fly).  It computes the
// x-face and r-face Roe fluxes once per face, the flux divergence with the axisymmetric /
// area geometric sources, the per-cell phase-change source (limited on the flux-updated
// state), the RK combine, and block partials of the CFL time step and of the conservation
// diagnostics.  The partials are reduced by the last CTAs to arrive, per tile row and then
// per case, in a fixed order (deterministic); the case's last CTA publishes the next time
// step to the workspace, so that N steps run without any host round trip.  Per-cell results do not depend on the tile shape.
#pragma once
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
constexpr int NPART = 27;   // per-block partial record
// partial slots: 0 dt min, 1 M, 2 W, 3 E, 4..6 boundary inflow rate (mass, water, energy),
// 7 active, 8 non-finite, 9..22 max |dU/dt| per field, 23 max ln J_hom, 24 max ln J_het,
// 25 surrogate fallback count, 26 tensor-core wait timeouts.  Stage 1 fills only 4..6 and
// 26 (the others are written as zero).
struct WsHeader {
  double dt_cur;          // time step of the next step
  double cfl;
  double b1[4];           // stage-1 boundary inflow rates (0..2) and timeouts (3)
  double diag[CT_NDIAG];  // last completed step
  double steps;
  unsigned int counter;   // last-block-done ticket
  unsigned int setup_magic;
  int nblocks;
  int pad;
  unsigned int qcount;    // cells queued for the surrogate kernel in the current stage
  unsigned int qticket;   // that kernel's last-block-done ticket
  double pre[NPART];      // the column sweep's record of a stage whose queue is pending
};
constexpr unsigned int SETUP_MAGIC = 0x43544231u;
constexpr size_t HDR_BYTES = 1024;
static_assert(sizeof(WsHeader) <= HDR_BYTES, "header");

struct DevCase {
  int geom, nx, nr, bc_xlo, bc_xhi, bc_rhi, jw, nblocks;
  int tiles_x, tiles_y;   // tile grid of the shape in use (nblocks = tiles_x * tiles_y)
  int viscous;            // viscous and diffusive fluxes
  int qoff;               // FP32 + surrogate through the column sweep: the surrogate queue's
                          // place in the workspace, in 256-byte units from its start (0: none)
  double nu_t;            // turbulent kinematic viscosity
  float fnu_t;
  double dx, dr, idx, idr, cfl;
  double area_a, x_throat, wall_len;
  double p0, T0, Yv0, cp0, gam0;       // nozzle inlet mixture
  float fdx, fidx, fdr, fidr, fwall_len, farea_a, fixt;   // FP32 copies of the geometry
  SrcCase sc;
  const double* inflow;   // nr x nf (plume; nf = 18 for the bimodal liquid, else 14)
  const double* amb;      // nf
  WsHeader* hdr;
  double* partials;       // nblocks x NPART, tile by * tiles_x + bx
  unsigned int* row_count;  // tiles_y arrival tickets (zero between launches)
  double* row_part;       // tiles_y x NPART row records
  // FP64 single-case steps: primitive planes (0 rho, 1 u, 2 v, 3 p, 4 Y_v, 5..12 moments per
  // kg, 13 soot per kg, 14 T, 15 c_v) of U (first NPLANE x N block) and of U1 (second block),
  // written by the kernel that produces each state and read by the next stage; null: every
  // stage converts its halo cells and its own cells itself
  double* prims;
};

// The surrogate queue of a workspace (stage_sweep.cuh): for at most N cells, their indices,
// their 14 rates (field-major, stride N), then the queue kernel's partial records.
__device__ __forceinline__ unsigned int* queue_cells(const DevCase& dc) {
  return reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(dc.hdr) + (size_t)dc.qoff * 256);
}
__device__ __forceinline__ size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }
__device__ __forceinline__ float* queue_rates(const DevCase& dc, size_t N) {
  return reinterpret_cast<float*>(reinterpret_cast<char*>(queue_cells(dc)) + round256(N * sizeof(unsigned int)));
}
__device__ __forceinline__ double* queue_partials(const DevCase& dc, size_t N) {
  return reinterpret_cast<double*>(reinterpret_cast<char*>(queue_rates(dc, N)) + round256((size_t)NF * N * sizeof(float)));
}

// Tile of TX x TY cells per CTA with a two-cell halo (HX x HY).  NT threads: the larger of
// the x-face ((TX+1) x TY) and r-face (TX x (TY+1)) counts rounded up to whole warps, so that
// each face pass takes a single round of the CTA.  minb: CTAs per SM the register budget is
// set for: M32 for the FP32 kernels of tiles up to 320 threads (2: 96 registers; 3: 72
// registers, more warps to hide latency at the price of spills), else one; M64 for the FP64
// kernels.
template <int TX_, int TY_, int M32 = 2, int M64 = 1>
struct Tile {
  static constexpr int TX = TX_, TY = TY_, HX = TX + 4, HY = TY + 4, NCELL = TX * TY;
  static constexpr int NFACE = (TX + 1) * TY > TX * (TY + 1) ? (TX + 1) * TY : TX * (TY + 1);
  static constexpr int NT = (NFACE + 31) / 32 * 32;
  // The r slopes of rows -1..TY outnumber the threads for the 32-wide tiles; then the threads
  // without a cell take row -1 during the x divergence (see stage_tile).
  static constexpr bool ROWM1_EARLY = TX * (TY + 2) > NT && NT - NCELL >= TX;
  // Face buffers: left and right reconstructed states; each face's flux overwrites its left
  // state (the thread that read it writes it).  Row -1's r slopes, written during the x
  // divergence while the x fluxes are still read, go to a side buffer of TX faces.
  static constexpr int NFBUF = 2;
  static constexpr int NSIDE = ROWM1_EARLY ? TX : 0;
  template <class T>
  static constexpr int minb() { return sizeof(T) == 4 ? (NT <= 320 ? M32 : 1) : M64; }
  template <class T, int NFX = NF>
  static constexpr size_t smem() { return sizeof(T) * (size_t)NFX * (HX * HY + NFBUF * NFACE + NSIDE); }
};
// thread count of the auxiliary kernels (time step of a given state)
constexpr int NT_AUX = 288;

// Geometry in the state precision (no double->float conversions inside FP32 kernels).
template <class T>
struct Geo {
  T dx, idx, dr, idr, wall_len, area_a, ixt, nu_t;
};
__device__ __forceinline__ Geo<float> geo_of(const DevCase& d, float) {
  return {d.fdx, d.fidx, d.fdr, d.fidr, d.fwall_len, d.farea_a, d.fixt, d.fnu_t};
}
__device__ __forceinline__ Geo<double> geo_of(const DevCase& d, double) {
  return {d.dx, d.idx, d.dr, d.idr, d.wall_len, d.area_a, 1.0 / d.x_throat, d.nu_t};
}

// Stable time step of a cell for CFL number 1 (reading A10; the diffusion limit with the
// viscous fluxes).  The stage kernel and the time-step kernel both use this one function,
// so that a step after a reload takes exactly the time step a continued run takes.
template <class T>
__device__ __forceinline__ T cell_dt(const DevCase& dc, const Geo<T>& g, const Prim<T>& w) {
  const T c = sound_speed(w.c2);
  T rate = (m_fabs(w.u) + c) * g.idx;
  if (dc.geom == 1) rate += (m_fabs(w.v) + c) * g.idr;
  if (dc.viscous) {
    T mu_e;
    rate += viscous_rate<T>(w, g.nu_t, g.idx * g.idx + (dc.geom == 1 ? g.idr * g.idr : T(0)), mu_e);
  }
  return trcp(rate);
}

// ---- boundary ghost cells (Sec. 4.1; reading A1) ---------------------------------------
// Conserved state at (i, j), i in [-2, nx+1], j in [-2, nr+1], not both outside.
// Out of line on purpose: keeps the nozzle inlet's FP64 arithmetic from being hoisted into
// the interior path of the FP32 kernels.
template <class T, int NFX = NF>
__device__ __noinline__ void load_ghost(const DevCase& dc, const T* __restrict__ U, size_t N, int i, int j,
                                        T* u14) {
  const int nx = dc.nx, nr = dc.nr;
  if (i < 0) {
    if (dc.bc_xlo == 1) {   // wall: mirror
      const size_t n = (size_t)j * nx + (-i - 1);
#pragma unroll
      for (int f = 0; f < NFX; ++f) u14[f] = U[f * N + n];
      u14[1] = -u14[1];
    } else if (dc.geom == 0) {   // total-condition subsonic inlet, interior velocity
      const size_t n = (size_t)j * nx;
      double u = double(U[N + n]) / double(U[n]);
      u = u < 0.0 ? 0.0 : u;
      const double Tg = dc.T0 - u * u / (2.0 * dc.cp0);
      const double p = dc.p0 * pow(Tg / dc.T0, dc.gam0 / (dc.gam0 - 1.0));
      const double z[4] = {0, 0, 0, 0};
      prim_to_cons<T>(p, Tg, u, 0.0, dc.Yv0, z, z, 0.0, u14);
#pragma unroll
      for (int f = NF; f < NFX; ++f) u14[f] = T(0);   // no liquid of heterogeneous origin
    } else {   // plume inflow profile
#pragma unroll
      for (int f = 0; f < NFX; ++f) u14[f] = T(dc.inflow[j * NFX + f]);
    }
    return;
  }
  if (i >= nx) {
    const int ii = dc.bc_xhi == 1 ? 2 * nx - 1 - i : nx - 1;
    const size_t n = (size_t)j * nx + ii;
#pragma unroll
    for (int f = 0; f < NFX; ++f) u14[f] = U[f * N + n];
    if (dc.bc_xhi == 1) u14[1] = -u14[1];
    return;
  }
  if (j < 0) {   // axis: mirror with rho*v negated
    const size_t n = (size_t)(-j - 1) * nx + i;
#pragma unroll
    for (int f = 0; f < NFX; ++f) u14[f] = U[f * N + n];
    u14[2] = -u14[2];
    return;
  }
  if (j >= nr) {
    if (dc.bc_rhi == 0) {
#pragma unroll
      for (int f = 0; f < NFX; ++f) u14[f] = T(dc.amb[f]);
    } else {
      const int jj = dc.bc_rhi == 1 ? 2 * nr - 1 - j : nr - 1;
      const size_t n = (size_t)jj * nx + i;
#pragma unroll
      for (int f = 0; f < NFX; ++f) u14[f] = U[f * N + n];
      if (dc.bc_rhi == 1) u14[2] = -u14[2];
    }
    return;
  }
  const size_t n = (size_t)j * nx + i;
#pragma unroll
  for (int f = 0; f < NFX; ++f) u14[f] = U[f * N + n];
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
// Warp sums of three values a, b, c with the additions of warp_sum in a transposed order:
// at the first two levels each lane adds only the part of the set it keeps (lanes below 16
// keep a and b, the others c; then lanes with bit 3 clear keep the first of their two), so
// 6 additions replace 15 and each sum is formed by the same additions as warp_sum's (bit
// for bit).  The sum of a ends in lane 0, b in lane 8, c in lane 16.
template <class V>
__device__ __forceinline__ V warp_sum3(V a, V b, V c) {
  const int lane = threadIdx.x & 31;
  const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0;
  V k0 = h16 ? c : a, k1 = h16 ? V(0) : b;
  k0 += __shfl_xor_sync(0xffffffffu, h16 ? a : c, 16);
  k1 += __shfl_xor_sync(0xffffffffu, h16 ? b : V(0), 16);
  V v = h8 ? k1 : k0;
  v += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
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
// Single-instruction warp reductions (redux.sync) through order-preserving integer keys.
__device__ __forceinline__ int warp_count(int v) { return __reduce_add_sync(0xffffffffu, v); }
// maximum / minimum of non-negative floats (their bit patterns order as unsigned integers)
__device__ __forceinline__ float warp_max_nonneg(float v) {
  return __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(v)));
}
__device__ __forceinline__ float warp_min_nonneg(float v) {
  return __uint_as_float(__reduce_min_sync(0xffffffffu, __float_as_uint(v)));
}
// maximum of any floats: negative values have their magnitude bits flipped
__device__ __forceinline__ float warp_max_any(float v) {
  const int i = __float_as_int(v);
  const int k = __reduce_max_sync(0xffffffffu, i >= 0 ? i : i ^ 0x7fffffff);
  return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff);
}
// The same for doubles, whose 64-bit keys compare as (high word, low word): the extreme high
// word first, then the extreme low word among the lanes that hold it.  Two redux.sync and no
// FP64 instruction, where a shuffle tree takes five FP64 comparisons.
__device__ __forceinline__ double key_double(unsigned hi, unsigned lo) {
  return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}
__device__ __forceinline__ double warp_max_nonneg(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
  return key_double(mh, __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u));
}
__device__ __forceinline__ double warp_min_nonneg(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned mh = __reduce_min_sync(0xffffffffu, hi);
  return key_double(mh, __reduce_min_sync(0xffffffffu, hi == mh ? lo : 0xffffffffu));
}
__device__ __forceinline__ double warp_max_any(double v) {
  long long b = __double_as_longlong(v);
  b = b >= 0 ? b : b ^ 0x7fffffffffffffffLL;   // order-preserving signed key
  const int hi = (int)(b >> 32);
  const unsigned lo = (unsigned)b;
  const int mh = __reduce_max_sync(0xffffffffu, hi);
  const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
  long long k = (long long)(((unsigned long long)(unsigned)mh << 32) | ml);
  k = k >= 0 ? k : k ^ 0x7fffffffffffffffLL;
  return __longlong_as_double(k);
}

// kind: 0 sum, 1 max, 2 min
__device__ __forceinline__ int slot_kind(int q) { return q == 0 ? 2 : ((q >= 9 && q <= 24) ? 1 : 0); }

// Reduce n partial records (NPART slots each, consecutive) at `base` into out[NPART]
// (shared memory), in a fixed order: lane-strided over the records, then a warp tree.
// All threads call this; it ends with a barrier.
__device__ inline void reduce_records(const double* base, int n, double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  for (int q = warp; q < NPART; q += nwarps) {
    const int kind = slot_kind(q);
    double acc = kind == 0 ? 0.0 : (kind == 1 ? -INFINITY : INFINITY);
    for (int b = lane; b < n; b += 32) {
      const double v = __ldcg(&base[(size_t)b * NPART + q]);
      acc = kind == 0 ? acc + v : (kind == 1 ? fmax(acc, v) : fmin(acc, v));
    }
    acc = kind == 0 ? warp_sum(acc) : (kind == 1 ? warp_max(acc) : warp_min(acc));
    if (lane == 0) out[q] = acc;
  }
  __syncthreads();
}

// Called by all threads after threads 0..NPART-1 wrote this CTA's partial record.  Returns
// true in the last CTA to arrive (out[] then holds the totals of the dc.nblocks records).
// One level: for launches of a few hundred CTAs (the time-step kernel).
__device__ inline bool last_block_reduce(const DevCase& dc, double* out) {
  __shared__ unsigned int ticket;
  if (threadIdx.x < NPART) __threadfence();   // the record's writers publish it
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(&dc.hdr->counter, 1u);
  __syncthreads();
  if (ticket != (unsigned int)(dc.nblocks - 1)) return false;
  __threadfence();
  reduce_records(dc.partials, dc.nblocks, out);
  if (threadIdx.x == 0) dc.hdr->counter = 0u;
  return true;
}

// Two levels, for the stage kernels: the last tile of each tile row to arrive reduces that
// row's records into a row record, and the last row to complete reduces the row records.
// Both orders are fixed, so the totals are deterministic; no CTA waits for another, and
// the serial part on the critical path is one row of records instead of all of them.
// `by`: this tile's row.  Returns true in the CTA that completed the case.
__device__ inline bool tile_reduce(const DevCase& dc, int by, double* out) {
  __shared__ unsigned int ticket;
  if (threadIdx.x < NPART) __threadfence();   // the record's writers publish it
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(&dc.row_count[by], 1u);
  __syncthreads();
  if (ticket != (unsigned int)(dc.tiles_x - 1)) return false;
  __threadfence();
  reduce_records(dc.partials + (size_t)by * dc.tiles_x * NPART, dc.tiles_x, out);
  if (threadIdx.x < NPART) {
    dc.row_part[(size_t)by * NPART + threadIdx.x] = out[threadIdx.x];
    __threadfence();
  }
  if (threadIdx.x == 0) dc.row_count[by] = 0u;   // every tile of the row has arrived
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(&dc.hdr->counter, 1u);
  __syncthreads();
  if (ticket != (unsigned int)(dc.tiles_y - 1)) return false;
  __threadfence();
  reduce_records(dc.row_part, dc.tiles_y, out);
  if (threadIdx.x == 0) dc.hdr->counter = 0u;
  return true;
}

// Publish a stage's reduced record (thread 0 of the block that reduced it): stage 1 the
// boundary inflow rates and the timeouts, stage 2 the diagnostics record and the next time
// step (cfl times the stable step).
__device__ inline void publish_stage(WsHeader* h, const double* fin, int stage, double dtd, double cfl) {
  if (stage == 1) {
    h->b1[0] = fin[4];
    h->b1[1] = fin[5];
    h->b1[2] = fin[6];
    h->b1[3] = fin[26];
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
    const double dtn = cfl * fin[0];
    d[25] = dtn;
    d[26] = fin[25];
    h->steps += 1.0;
    d[27] = h->steps;
    d[28] = h->b1[3] + fin[26];
    h->dt_cur = dtn;
  }
}

// ---- the fused stage kernel ---------------------------------------------------------------
// shared memory of the surrogate phase, reusing the (then dead) stencil buffers:
// activations, streamed weights, outputs, blob header, per-thread results
constexpr size_t SM_A = 0, SM_W = SM_A + mlp::ABYTES, SM_OUT = SM_W + 32768, SM_HDR = SM_OUT + 128 * 10 * 4,
                 SM_RES = SM_HDR + mlp::NFLOAT * 4;
// the surrogate queue kernel of the column sweep (stage_sweep.cuh): threads, shared memory,
// CTAs of a launch at most (the room of its partial records in the workspace)
struct QueueTile {
  static constexpr int NT = 256;
};
constexpr size_t QUEUE_SMEM = SM_RES + (size_t)QueueTile::NT * 40;
constexpr int QUEUE_GRID_MAX = 4096;
template <class TL>
constexpr size_t stage_smem_surr() {
  return TL::template smem<float>() > SM_RES + (size_t)TL::NT * 40 ? TL::template smem<float>()
                                                                     : SM_RES + (size_t)TL::NT * 40;
}

// Tensor-core resources of a CTA: 128 TMEM columns and the MMA-completion mbarrier (outside
// the overlaid stencil buffers).  The stage kernels take them once at the start
// (ready = true); the surrogate routine can also take and free them around a single call
// (ready = false), since a CTA that has relinquished its allocation permit may not
// allocate again.
static __shared__ uint64_t s_tc_mbar;   // MMA completion
static __shared__ uint64_t s_tc_wbar;   // weight bulk copies
static __shared__ uint32_t s_tc_slot;
struct TcCtx {
  uint32_t tmem, phase, wphase;
  bool ready;
};
__device__ __forceinline__ uint32_t tc_acquire() {
  if ((threadIdx.x >> 5) == 0) {
    tc::tmem_alloc(tc::smem_addr(&s_tc_slot), 128);
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    tc::mbar_init(tc::smem_addr(&s_tc_mbar), 1);
    tc::mbar_init(tc::smem_addr(&s_tc_wbar), 1);
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  return s_tc_slot;
}
__device__ __forceinline__ void tc_release(uint32_t tmem) {
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(tmem, 128);
}

// Surrogate cells of one tile (called by all threads, only when the tile has at least one):
// compaction into 128-row tiles and the BF16 tensor-core network.  Each surrogate cell's
// thread finds its 10 outputs (raw units, held to the training range of their targets) in
// res[10 * threadIdx.x ...] afterwards.  x: the cell's 16 raw inputs (kind == 2 only).
template <class TL>
__device__ __noinline__ void surrogate_tile(const unsigned char* __restrict__ blob, int kind, const float* x,
                                            int& ntimeout, unsigned char* smem, TcCtx* tcx) {
  constexpr int NT = TL::NT;
  __shared__ int wcnt[NT / 32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float* ghdr = reinterpret_cast<const float*>(blob);
  const unsigned mask = __ballot_sync(0xffffffffu, kind == 2);
  if (lane == 0) wcnt[warp] = __popc(mask);
  unsigned char* A = smem + SM_A;
  unsigned char* W = smem + SM_W;
  float* outs = reinterpret_cast<float*>(smem + SM_OUT);
  float* hdr = reinterpret_cast<float*>(smem + SM_HDR);
  float* res = reinterpret_cast<float*>(smem + SM_RES);
  for (int q = tid; q < mlp::NFLOAT; q += NT) hdr[q] = ghdr[q];
  uint32_t tmem, phase = 0, wphase = 0;
  if (tcx->ready) {
    tmem = tcx->tmem;
    phase = tcx->phase;
    wphase = tcx->wphase;
    __syncthreads();
  } else {
    tmem = tc_acquire();   // includes the barrier
  }
  int off = 0, total = 0;
  for (int w2 = 0; w2 < NT / 32; ++w2) {
    off += w2 < warp ? wcnt[w2] : 0;
    total += wcnt[w2];
  }
  const int row = off + __popc(mask & ((1u << lane) - 1u));
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
    ok = mlp::run_tile<true>(A, W, hdr + mlp::F_BIAS, tmem, tc::smem_addr(&s_tc_mbar), phase, o, blob + mlp::WOFF,
                             total - c0, tc::smem_addr(&s_tc_wbar), &wphase) && ok;
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
  if (tcx->ready) {
    tcx->phase = phase;
    tcx->wphase = wphase;
  } else {
    tc_release(tmem);
  }
  if (!ok && tid == 0) ntimeout += 1;   // a tensor-core wait gave up: the step reports it
}

// Source of the FP32 + surrogate path (called by all threads): active cells inside the
// surrogate's training hull take their rates from the network, the others the plain source
// (counted as fallbacks); both feed the plain path's tail, so conservation and the limiters
// are exact.  Adds the source to acc.
template <class TL, class T>
__device__ __forceinline__ void surrogate_source(const DevCase& dc, const unsigned char* __restrict__ blob, bool cell,
                                                 const Prim<T>& w, const T* u14, T* acc, T dt, int& nactive,
                                                 int& nfallback, int& ntimeout, T& lnJh, T& lnJt,
                                                 unsigned char* smem, TcCtx* tcx) {
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
      st = saturation(w, dc.sc);
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
    surrogate_tile<TL>(blob, kind, x, ntimeout, smem, tcx);
    if (kind == 2) {
      const float* y = reinterpret_cast<const float*>(smem + SM_RES) + 10 * threadIdx.x;
      const bool nuc = st.lnSl > 0.0;
      Rates<T> r;
      r.Jeff = r.rc_um = T(0);
      if (nuc) {
        // nucleation is the plain path's closed form: the rates and the Kelvin radius of
        // Eqs. 3, 4, 10 (exponent in FP64) and the Kantrowitz factor of Eq. 5 (T_sat by the
        // Newton iteration, Young's law at r_crit); the network supplies growth and relaxation
        const Cnt c = cnt_rates<T>(w, st.lnSl, dc.sc, lnJ2);
        const T Tsat_l = prop_tsat<T, false>(dc.sc, T(st.lnpv));
        const T phi = kantrowitz_phi<T>(w, gas_props<T>(w), c.rc, c.rhov, Tsat_l);
        r.Jeff = T(c.Jsum) / (T(1) + phi);
        r.rc_um = T(c.rc * 1e6);
      }
      r.Gl = st.pres_l ? T(MLP_G0 * sinhf(y[2])) : T(0);
      r.Gs = st.pres_s ? T(MLP_G0 * sinhf(y[3])) : T(0);
      r.xl = st.pres_l ? T(__expf(y[4])) : T(0);
      r.xs = st.pres_s ? T(__expf(y[5])) : T(0);
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


// planes of stored primitive variables per state: the stencil's fields, T and c_v
constexpr int NPLANE = NF + 2;

// The primitive vector of the stencil (fields of the state, conserved -> primitive).
template <class T, bool BI>
__device__ __forceinline__ void prim_vector(const Prim<T>& w, T* qv) {
  qv[0] = w.rho;
  qv[1] = w.u;
  qv[2] = w.v;
  qv[3] = w.p;
  qv[4] = w.Yv;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    qv[5 + q] = w.ml[q];
    qv[9 + q] = w.ms[q];
  }
  qv[13] = w.ns;
  if (BI) {
#pragma unroll
    for (int q = 0; q < 4; ++q) qv[14 + q] = w.mh[q];
  }
}

// One stage on tile (bx, by) of a case; `tile` = by * tiles_x + bx indexes the partial
// records.  All threads of the CTA call this.  STAGE 1: Uout = Uin + dt L(Uin).
// STAGE 2: Uout = (Un + Uin + dt L(Uin))/2 (Uout may be Un); the last tile of the case to
// finish reduces the partials and publishes cfl * (stable step) as the next time step.
// SP: the primitive planes of dc.prims are in use (the input state's are read for the
// interior halo cells instead of converting them, the output state's are written).
template <class TL, class T, int STAGE, bool SURR, bool BI = false, bool SP = false>
__device__ __forceinline__ void stage_tile(const DevCase& dc, int bx, int by, int tile, const T* __restrict__ Uin,
                                           const T* Un, T* Uout, const unsigned char* __restrict__ blob,
                                           unsigned char* smem_raw, double cfl, TcCtx* tcx) {
  constexpr int TX = TL::TX, TY = TL::TY, HX = TL::HX, HY = TL::HY, NT = TL::NT, NCELL = TL::NCELL;
  constexpr int NFACE = TL::NFACE;
  constexpr int NFX = nf_of<BI>();   // fields of the state (18 with the bimodal liquid)
  // Shared memory holds the fields in pairs (pair.cuh): pair k = fields 2k, 2k+1 side by side.
  using V = typename PairOf<T>::V;
  constexpr int NP = NFX / 2;
  V (*qs2)[HY][HX] = reinterpret_cast<V (*)[HY][HX]>(smem_raw);                       // primitives
  V (*fL2)[NFACE] = reinterpret_cast<V (*)[NFACE]>(smem_raw + sizeof(T) * NFX * HX * HY);  // left states
  V (*fR2)[NFACE] = fL2 + NP;                                       // right states
  V (*fb2)[NFACE] = fL2;                                            // face fluxes
  // left states of the r faces of row 0 from the early row -1 slopes (32-wide tiles)
  V (*fLm1)[TL::NSIDE > 0 ? TL::NSIDE : 1] =
      reinterpret_cast<V (*)[TL::NSIDE > 0 ? TL::NSIDE : 1]>(fR2 + NP);
  // scalar views: field f of a cell or face
  const auto qs = [&](int f, int hj, int hi) -> T {
    const V v = qs2[f >> 1][hj][hi];
    return (f & 1) ? v.y : v.x;
  };
  const auto fb = [&](int f, int face) -> T {
    const V v = fb2[f >> 1][face];
    return (f & 1) ? v.y : v.x;
  };
  constexpr bool IS64 = std::is_same<T, double>::value;
  // warp partials in the state precision: the FP32 kernels convert to FP64 once per slot and
  // CTA (conversions run on the FP64 pipe, a small fraction of the FP32 rate on GB300)
  __shared__ T red[NT / 32][NPART];
  __shared__ T s_dt;
  __shared__ double fin[NPART];

  const int nx = dc.nx, nr = dc.geom == 1 ? dc.nr : 1;
  const size_t N = (size_t)nx * nr;
  const int i0 = bx * TX, j0 = by * TY;
  const int tid = threadIdx.x;
  const double dtd = dc.hdr->dt_cur;
  if (tid == 0) s_dt = T(dtd);   // one conversion per CTA; published by phase A's barrier
  const Geo<T> g = geo_of(dc, T(0));
  // FP64, axisymmetric: the geometry of the tile's rows (1/(j + 1/2), the r-face weights,
  // the x-face area per radian, the cell volume per radian) and the duct-wall test of its
  // columns, once per row and column with the expressions the cells would evaluate
  // themselves (the same bits), published by phase A's barrier.  The FP32 kernels keep the
  // per-cell form: their shared memory is the tighter budget.
  __shared__ T s_row[IS64 ? TY : 1][5];
  __shared__ bool s_wall[IS64 ? TX : 1];
  if (IS64 && dc.geom == 1) {
    for (int r = tid; r < TY; r += NT) {
      const int j = j0 + r;
      const T ijh = trcp(T(j) + T(0.5));
      const T area = (T(j) + T(0.5)) * g.dr * g.dr;
      s_row[r][0] = ijh;
      s_row[r][1] = T(j) * ijh * g.idr;
      s_row[r][2] = T(j + 1) * ijh * g.idr;
      s_row[r][3] = area;
      s_row[r][4] = area * g.dx;
    }
    for (int c = tid; c < TX; c += NT) s_wall[c] = g.wall_len > T(0) && (T(i0 + c) + T(0.5)) * g.dx < g.wall_len;
  }

  // phase A: halo primitives.  A thread owns up to NA halo cells; the interior loads of all
  // of them are issued before any is converted, so their latencies overlap.  FP32, one
  // liquid set: zb collects the bits of the halo's moment fields (5..12).
  constexpr bool DRY_OK = !IS64 && !BI;
  unsigned zb = 0;
  {
    constexpr int NA = (HX * HY + NT - 1) / NT;
    T u14[NA][NFX];
    int kind[NA];   // 0 skip, 1 interior, 2 ghost
#pragma unroll
    for (int r = 0; r < NA; ++r) {
      const int p = tid + r * NT;
      const int hi = p % HX, hj = p / HX;
      const int i = i0 + hi - 2, j = j0 + hj - 2;
      const bool xin = i >= 0 && i < nx, rin = j >= 0 && j < nr;
      bool need = p < HX * HY && (xin || rin) && i >= -2 && i <= nx + 1 && j >= -2 && j <= nr + 1;
      if (dc.geom == 0) need = need && j == 0;
      kind[r] = !need ? 0 : (xin && rin ? 1 : 2);
      if (kind[r] == 1) {
        const size_t n = (size_t)j * nx + i;
        // SP: the primitives of the input state, written by the kernel that produced it
        const T* src = SP ? reinterpret_cast<const T*>(dc.prims) + (STAGE == 1 ? 0 : (size_t)NPLANE * N) : Uin;
#pragma unroll
        for (int f = 0; f < NFX; ++f) u14[r][f] = src[f * N + n];
      }
    }
#pragma unroll
    for (int r = 0; r < NA; ++r) {
      if (kind[r] == 0) continue;
      const int p = tid + r * NT;
      const int hi = p % HX, hj = p / HX;
      if (kind[r] == 2) {   // out of line, through its own array: u14 stays in registers
        T g14[NFX];
        load_ghost<T, NFX>(dc, Uin, N, i0 + hi - 2, j0 + hj - 2, g14);
#pragma unroll
        for (int f = 0; f < NFX; ++f) u14[r][f] = g14[f];
      }
      T qv[NFX];
      if (SP && kind[r] == 1) {
#pragma unroll
        for (int f = 0; f < NFX; ++f) qv[f] = u14[r][f];
      } else {
        Prim<T> w;
        cons_to_prim<T, BI>(u14[r], w);
        prim_vector<T, BI>(w, qv);
      }
#pragma unroll
      for (int k2 = 0; k2 < NP; ++k2) qs2[k2][hj][hi] = p_make(qv[2 * k2], qv[2 * k2 + 1]);
      if constexpr (DRY_OK) {
#pragma unroll
        for (int f = 5; f < 13; ++f) zb |= __float_as_uint(float(qv[f]));
      }
    }
  }
  // A dry tile: every moment field of the halo's primitive vectors is +0 (dry air, most of
  // a plume outside its mixing layer).  Its reconstruction skips the three all-moment pairs,
  // whose slopes are zero and face states +0, and its Roe fluxes the condensate terms of the
  // face thermodynamics, which vanish exactly: the bits of the full formulas.
  const bool dry = DRY_OK ? __syncthreads_and(zb == 0u) != 0 : (__syncthreads(), false);

  const T dt = s_dt;

  // phase B1: limited x slopes, once per cell, written as the states of its two faces
  // (tile-local cell c in [-1, TX]; face f lies between cells f-1 and f)
  const auto phase_b1 = [&](auto dry_tag) {
    constexpr bool DRY = decltype(dry_tag)::value;
    for (int p = tid; p < (TX + 2) * TY; p += NT) {
      const int c = p % (TX + 2) - 1, hj = p / (TX + 2);
      const int i = i0 + c, j = j0 + hj;
      if (i > nx || j >= nr) continue;
#pragma unroll
      for (int k2 = 0; k2 < NP; ++k2) {
        if (DRY && moment_pair(k2)) continue;   // +0 face states, not stored
        const V am = qs2[k2][hj + 2][c + 1], a0 = qs2[k2][hj + 2][c + 2], a1 = qs2[k2][hj + 2][c + 3];
        V flo, fhi;
        vl_faces2(am, a0, a1, flo, fhi);
        if (c < TX) fL2[k2][hj * (TX + 1) + c + 1] = fhi;
        if (c >= 0) fR2[k2][hj * (TX + 1) + c] = flo;
      }
    }
  };
  if (dry)
    phase_b1(std::true_type{});
  else
    phase_b1(std::false_type{});
  __syncthreads();

  // phase B2: x-face Roe fluxes
  const auto phase_b2 = [&](auto dry_tag) {
    constexpr bool DRY = decltype(dry_tag)::value;
  for (int p = tid; p < (TX + 1) * TY; p += NT) {
    const int fx = p % (TX + 1), hj = p / (TX + 1);
    const int i = i0 + fx, j = j0 + hj;
    if (i > nx || j >= nr) continue;
    T qL[NFX], qR[NFX], F[NFX];
#pragma unroll
    for (int k2 = 0; k2 < NP; ++k2) {
      if (DRY && moment_pair(k2)) {
        qL[2 * k2] = qL[2 * k2 + 1] = qR[2 * k2] = qR[2 * k2 + 1] = T(0);
        continue;
      }
      const V a = fL2[k2][p], b = fR2[k2][p];
      qL[2 * k2] = a.x;
      qL[2 * k2 + 1] = a.y;
      qR[2 * k2] = b.x;
      qR[2 * k2 + 1] = b.y;
    }
    roe_flux<T, 0, NFX, DRY>(qL, qR, F);
    // walls are adiabatic, impermeable and slip: nothing diffuses through them
    if (dc.viscous && !((i == 0 && dc.bc_xlo == 1) || (i == nx && dc.bc_xhi == 1))) {
      const auto q = [&](int f, int side) -> T { return qs(f, hj + 2, fx + 1 + side); };
      sub_diffusive_flux<T, NFX>(q, g.idx, g.nu_t, F);
    }
#pragma unroll
    for (int k2 = 0; k2 < NP; ++k2) fb2[k2][p] = p_make(F[2 * k2], F[2 * k2 + 1]);
  }
  };
  if (dry)
    phase_b2(std::true_type{});
  else
    phase_b2(std::false_type{});
  __syncthreads();

  const int ci = tid % TX, cj = tid / TX;
  const int i = i0 + ci, j = j0 + cj;
  const bool cell = tid < NCELL && i < nx && j < nr;
  // limited r slope of tile-local row c in [-1, TY] at column hi -> states of its r faces
  const auto r_slope = [&](int hi, int c, auto dry_tag) {
    constexpr bool DRY = decltype(dry_tag)::value;
    const int ii = i0 + hi, jj = j0 + c;
    if (ii >= nx || jj > nr) return;
#pragma unroll
    for (int k2 = 0; k2 < NP; ++k2) {
      if (DRY && moment_pair(k2)) continue;   // +0 face states, not stored
      const V am = qs2[k2][c + 1][hi + 2], a0 = qs2[k2][c + 2][hi + 2], a1 = qs2[k2][c + 3][hi + 2];
      V flo, fhi;
      vl_faces2(am, a0, a1, flo, fhi);
      if (TL::ROWM1_EARLY && c < 0) fLm1[k2][hi] = fhi;
      else if (c < TY) fL2[k2][(c + 1) * TX + hi] = fhi;
      if (c >= 0) fR2[k2][c * TX + hi] = flo;
    }
  };
  // The r slopes of rows -1..TY outnumber the threads for the 32-wide tiles; the threads
  // without a cell take row -1 during the x divergence (the x face states are dead by then),
  // so that phase D1 is a single round.
  constexpr bool ROWM1_EARLY = TL::ROWM1_EARLY;
  T acc[NFX];
  // water carried by a face flux: vapour, liquid (both sets) and ice
  const auto water_flux = [&](int f) -> T {
    const T l3 = BI ? fb(8, f) + fb(17, f) : fb(8, f);
    return fb(4, f) + T(k::YL3) * l3 + T(k::YS3) * fb(12, f);
  };
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
      const T iv = trcp(Ac * g.dx);
      cw = area_w * iv;
      ce = area_e * iv;
      vol = Ac * g.dx;
    } else {
      cw = ce = g.idx;
      if constexpr (IS64) {
        area_w = area_e = s_row[cj][3];
        vol = s_row[cj][4];
      } else {
        area_w = area_e = (T(j) + T(0.5)) * g.dr * g.dr;
        vol = area_w * g.dx;
      }
    }
    if constexpr (IS64) {
      // FP64: where the x fluxes of every moment field are zero, so is their divergence.
      // (A zero's sign cannot reach the update: a zero term is added to a non-zero one, or
      // to a state that is +0 as every state this code writes.)
#pragma unroll
      for (int f = 0; f < NFX; ++f)
        if (!is_moment(f)) acc[f] = fma(cw, fb(f, w), -ce * fb(f, e));
      if (moments_zero<NFX>([&](int f) { return fb(f, w); }) && moments_zero<NFX>([&](int f) { return fb(f, e); })) {
#pragma unroll
        for (int f = 0; f < NFX; ++f)
          if (is_moment(f)) acc[f] = T(0);
      } else {
#pragma unroll
        for (int f = 0; f < NFX; ++f)
          if (is_moment(f)) acc[f] = fma(cw, fb(f, w), -ce * fb(f, e));
      }
    } else {
      const V cw2 = p_make(cw, cw), nce2 = p_make(-ce, -ce);
#pragma unroll
      for (int k2 = 0; k2 < NP; ++k2) {
        const V a = p_fma(cw2, fb2[k2][w], p_mul(nce2, fb2[k2][e]));
        acc[2 * k2] = a.x;
        acc[2 * k2 + 1] = a.y;
      }
    }
    if (i == 0) {
      bm += area_w * fb(0, w);
      bw += area_w * water_flux(w);
      be += area_w * fb(3, w);
    }
    if (i == nx - 1) {
      bm -= area_e * fb(0, e);
      bw -= area_e * water_flux(e);
      be -= area_e * fb(3, e);
    }
  }

  if (dc.geom == 1) {
    if (ROWM1_EARLY && tid >= NCELL && tid - NCELL < TX) {
      if (dry)
        r_slope(tid - NCELL, -1, std::true_type{});
      else
        r_slope(tid - NCELL, -1, std::false_type{});
    }
    __syncthreads();
    // phase D1: limited r slopes (tile-local row c in [-1, TY]) -> states of the r faces
    if (dry) {
      for (int p = tid + (ROWM1_EARLY ? TX : 0); p < TX * (TY + 2); p += NT) r_slope(p % TX, p / TX - 1, std::true_type{});
    } else {
      for (int p = tid + (ROWM1_EARLY ? TX : 0); p < TX * (TY + 2); p += NT) r_slope(p % TX, p / TX - 1, std::false_type{});
    }
    __syncthreads();
    // phase D2: r-face Roe fluxes (face fy lies between tile rows fy-1 and fy)
    const auto phase_d2 = [&](auto dry_tag) {
      constexpr bool DRY = decltype(dry_tag)::value;
    for (int p = tid; p < TX * (TY + 1); p += NT) {
      const int hi = p % TX, fy = p / TX;
      const int ii = i0 + hi, jj = j0 + fy;
      if (ii >= nx || jj > nr) continue;
      T qL[NFX], qR[NFX], F[NFX];
#pragma unroll
      for (int k2 = 0; k2 < NP; ++k2) {
        if (DRY && moment_pair(k2)) {
          qL[2 * k2] = qL[2 * k2 + 1] = qR[2 * k2] = qR[2 * k2 + 1] = T(0);
          continue;
        }
        const V a = (TL::ROWM1_EARLY && p < TX) ? fLm1[k2][p] : fL2[k2][p], b = fR2[k2][p];
        qL[2 * k2] = a.x;
        qL[2 * k2 + 1] = a.y;
        qR[2 * k2] = b.x;
        qR[2 * k2 + 1] = b.y;
      }
      roe_flux<T, 1, NFX, DRY>(qL, qR, F);
      if (dc.viscous && !(jj == nr && dc.bc_rhi == 1)) {
        const auto q = [&](int f, int side) -> T { return qs(f, fy + 1 + side, hi + 2); };
        sub_diffusive_flux<T, NFX>(q, g.idr, g.nu_t, F);
      }
#pragma unroll
      for (int k2 = 0; k2 < NP; ++k2) fb2[k2][p] = p_make(F[2 * k2], F[2 * k2 + 1]);
    }
    };
    if (dry)
      phase_d2(std::true_type{});
    else
      phase_d2(std::false_type{});
    __syncthreads();
  }

  // phase E: residual, source, update, partial reductions
  T pM = T(0), pW = T(0), pE = T(0);
  T dtmin = T(INFINITY);
  T rmax[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) rmax[f] = T(0);
  T lnJh = T(-INFINITY), lnJt = T(-INFINITY);
  int nactive = 0, nbad = 0, nfallback = 0, ntimeout = 0;
  T u14[NFX];
  Prim<T> w;
  if (cell) {
    const size_t n = (size_t)j * nx + i;
#pragma unroll
    for (int f = 0; f < NFX; ++f) u14[f] = Uin[f * N + n];
    if (SP) {   // the cell's primitives: the stencil's from shared memory, T and c_v stored
      w.rho = qs(0, cj + 2, ci + 2);
      w.u = qs(1, cj + 2, ci + 2);
      w.v = qs(2, cj + 2, ci + 2);
      w.p = qs(3, cj + 2, ci + 2);
      w.Yv = qs(4, cj + 2, ci + 2);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        w.ml[q] = qs(5 + q, cj + 2, ci + 2);
        w.ms[q] = qs(9 + q, cj + 2, ci + 2);
      }
      w.ns = qs(13, cj + 2, ci + 2);
      w.Yl = rn_mul(T(k::YL3), w.ml[3]);   // as the conversion forms them
      w.Ys = rn_mul(T(k::YS3), w.ms[3]);
      const T* src = reinterpret_cast<const T*>(dc.prims) + (STAGE == 1 ? 0 : (size_t)NPLANE * N);
      w.Tg = src[NFX * N + n];
      w.cv = src[(NFX + 1) * N + n];
      w.Rg = w.c2 = T(0);   // not used by the cell update
    } else {
      cons_to_prim<T, BI>(u14, w);
    }
    if (dc.geom == 1) {
      T ijh, cs, cn;
      bool wall;
      if constexpr (IS64) {
        ijh = s_row[cj][0];
        cs = s_row[cj][1];
        cn = s_row[cj][2];
        wall = s_wall[ci];
      } else {
        ijh = trcp(T(j) + T(0.5));
        cs = T(j) * ijh * g.idr;
        cn = T(j + 1) * ijh * g.idr;
        wall = g.wall_len > T(0) && (T(i) + T(0.5)) * g.dx < g.wall_len;
      }
      // the duct wall's faces carry the pressure in rho*v (field 2) and nothing else
      const bool wall_s = wall && j == dc.jw, wall_n = wall && j == dc.jw - 1;
      if constexpr (IS64) {
        const int fs = cj * TX + ci, fn = (cj + 1) * TX + ci;
        const auto Fs = [&](int f) -> T { return wall_s ? (f == 2 ? w.p : T(0)) : fb(f, fs); };
        const auto Fn = [&](int f) -> T { return wall_n ? (f == 2 ? w.p : T(0)) : fb(f, fn); };
#pragma unroll
        for (int f = 0; f < NFX; ++f)
          if (!is_moment(f)) acc[f] = acc[f] + fma(cs, Fs(f), -cn * Fn(f));
        if (!(moments_zero<NFX>(Fs) && moments_zero<NFX>(Fn))) {   // as in the x divergence
#pragma unroll
          for (int f = 0; f < NFX; ++f)
            if (is_moment(f)) acc[f] = acc[f] + fma(cs, Fs(f), -cn * Fn(f));
        }
      } else {
        const V cs2 = p_make(cs, cs), ncn2 = p_make(-cn, -cn);
#pragma unroll
        for (int k2 = 0; k2 < NP; ++k2) {
          V Fs = fb2[k2][cj * TX + ci], Fn = fb2[k2][(cj + 1) * TX + ci];
          if (wall_n) Fn = p_make(k2 == 1 ? w.p : T(0), T(0));
          if (wall_s) Fs = p_make(k2 == 1 ? w.p : T(0), T(0));
          const V a = p_add(p_make(acc[2 * k2], acc[2 * k2 + 1]), p_fma(cs2, Fs, p_mul(ncn2, Fn)));
          acc[2 * k2] = a.x;
          acc[2 * k2 + 1] = a.y;
        }
      }
      acc[2] += w.p * ijh * g.idr;
      if (dc.viscous) {   // radial component of the vector Laplacian: -mu_e v / r^2
        T mu_e;
        viscous_rate<T>(w, g.nu_t, T(0), mu_e);
        acc[2] -= mu_e * w.v * (ijh * ijh) * (g.idr * g.idr);
      }
      if (j == nr - 1) {
        const T An = T(nr) * g.dr * g.dx;
        const int e = (cj + 1) * TX + ci;
        bm -= An * fb(0, e);
        bw -= An * water_flux(e);
        be -= An * fb(3, e);
      }
    } else {
      acc[1] += w.p * tdiv(area_e - area_w, vol);
    }
    // phase-change source limited on the flux-updated state
    T Q[NFX];
    double lnJ2[2];
    if (!SURR) {
      const bool act = phase_source<T, BI>(w, u14, acc, dt, dc.sc, Q, lnJ2, nullptr);
      nactive = act ? 1 : 0;
      // inactive cells keep -inf without a conversion, and their source is +0: adding it
      // could only turn a -0 into +0, which the update cannot tell apart
      if (act) {
        lnJh = T(lnJ2[0]);
        lnJt = T(lnJ2[1]);
#pragma unroll
        for (int f = 4; f < 13; ++f) acc[f] += Q[f];
        if (BI) {
#pragma unroll
          for (int f = 14; f < 18; ++f) acc[f] += Q[f];
        }
      }
    }
  }
  if (SURR)
    surrogate_source<TL, T>(dc, blob, cell, w, u14, acc, dt, nactive, nfallback, ntimeout, lnJh, lnJt, smem_raw,
                            tcx);
  if (cell) {
    const size_t n = (size_t)j * nx + i;
    // RK combine
    T out[NFX];
    const V dt2 = p_make(dt, dt);
    // FP64: moment fields that are +0 in the input states with a zero rate stay +0 (exactly
    // what the update gives), and their residual is 0
    bool mz = false;
    if constexpr (IS64) {
      const auto bits0 = [&](const T* v) {
        long long z = 0;
#pragma unroll
        for (int f = 0; f < NFX; ++f)
          if (is_moment(f)) z |= __double_as_longlong(v[f]);
        return z == 0;
      };
      mz = bits0(u14) && moments_zero<NFX>([&](int f) { return acc[f]; });
      if (STAGE == 2) {
        if (mz) {
          T unm[NFX];
#pragma unroll
          for (int f = 0; f < NFX; ++f)
            if (is_moment(f)) unm[f] = Un[f * N + n];
          mz = bits0(unm);
        }
      }
    }
    if (STAGE == 1) {
      if constexpr (IS64) {
#pragma unroll
        for (int f = 0; f < NFX; ++f)
          if (!is_moment(f)) out[f] = fma(dt, acc[f], u14[f]);
        if (mz) {
#pragma unroll
          for (int f = 0; f < NFX; ++f)
            if (is_moment(f)) out[f] = T(0);
        } else {
#pragma unroll
          for (int f = 0; f < NFX; ++f)
            if (is_moment(f)) out[f] = fma(dt, acc[f], u14[f]);
        }
      } else {
#pragma unroll
        for (int k2 = 0; k2 < NP; ++k2) {
          const V o = p_fma(dt2, p_make(acc[2 * k2], acc[2 * k2 + 1]), p_make(u14[2 * k2], u14[2 * k2 + 1]));
          out[2 * k2] = o.x;
          out[2 * k2 + 1] = o.y;
        }
      }
    } else if (IS64) {
#pragma unroll
      for (int f = 0; f < NFX; ++f) {
        if (is_moment(f)) continue;
        const T un = Un[f * N + n];
        out[f] = fma(T(0.5), un, T(0.5) * fma(dt, acc[f], u14[f]));
        if (f < NF) rmax[f] = m_fabs(out[f] - un);   // divided by dt once per CTA
      }
      if (mz) {
#pragma unroll
        for (int f = 0; f < NFX; ++f)
          if (is_moment(f)) {
            out[f] = T(0);
            if (f < NF) rmax[f] = T(0);   // the second set's slots keep their maximum
          }
      } else {
#pragma unroll
        for (int f = 0; f < NFX; ++f) {
          if (!is_moment(f)) continue;
          const T un = Un[f * N + n];
          out[f] = fma(T(0.5), un, T(0.5) * fma(dt, acc[f], u14[f]));
          const T rf = m_fabs(out[f] - un);
          if (f < NF) {
            rmax[f] = rf;
          } else {   // the second liquid set shares the residual slots of the first
            rmax[f - 9] = rf > rmax[f - 9] ? rf : rmax[f - 9];
          }
        }
      }
    } else {
      const V half2 = p_make(T(0.5), T(0.5));
      T unv[NFX];
#pragma unroll
      for (int f = 0; f < NFX; ++f) unv[f] = Un[f * N + n];
#pragma unroll
      for (int k2 = 0; k2 < NP; ++k2) {
        const V un2 = p_make(unv[2 * k2], unv[2 * k2 + 1]);
        const V t = p_fma(dt2, p_make(acc[2 * k2], acc[2 * k2 + 1]), p_make(u14[2 * k2], u14[2 * k2 + 1]));
        const V o = p_fma(half2, un2, p_mul(half2, t));
        out[2 * k2] = o.x;
        out[2 * k2 + 1] = o.y;
      }
#pragma unroll
      for (int f = 0; f < NFX; ++f) {
        const T un = unv[f];
        const T rf = m_fabs(out[f] - un);   // divided by dt once per CTA
        if (f < NF) {
          rmax[f] = rf;
        } else {   // the second liquid set shares the residual slots of the first
          rmax[f - 9] = rf > rmax[f - 9] ? rf : rmax[f - 9];
        }
      }
    }
#pragma unroll
    for (int f = 0; f < NFX; ++f) {
      Uout[f * N + n] = out[f];
      nbad += finite_bits(out[f]) ? 0 : 1;
    }
    if (STAGE == 2 || SP) {
      Prim<T> wn;
      cons_to_prim<T, BI>(out, wn);
      if (SP) {   // the primitives of the output state, for the next stage
        T qv[NFX];
        prim_vector<T, BI>(wn, qv);
        T* dst = reinterpret_cast<T*>(dc.prims) + (STAGE == 1 ? (size_t)NPLANE * N : 0);
#pragma unroll
        for (int f = 0; f < NFX; ++f) dst[f * N + n] = qv[f];
        dst[NFX * N + n] = wn.Tg;
        dst[(NFX + 1) * N + n] = wn.cv;
      }
      if (STAGE == 2) dtmin = cell_dt<T>(dc, g, wn);   // times cfl at the end
    }
    if (STAGE == 2) {
      pM = vol * out[0];
      pW = vol * (out[4] + T(k::YL3) * (BI ? out[8] + out[17] : out[8]) + T(k::YS3) * out[12]);
      pE = vol * out[3];
    }
  }

  // block partials: warp and CTA sums in the state precision, FP64 from the CTA level on
  const int warp = tid >> 5, lane = tid & 31;
  {
    T v;
    int a;
    // boundary fluxes: only tiles on the inflow, outflow or far-field boundary have any
    if (i0 == 0 || i0 + TX >= nx || (dc.geom == 1 && j0 + TY >= nr)) {
      v = warp_sum3(bm, bw, be);
      if (lane == 0) red[warp][4] = v;
      if (lane == 8) red[warp][5] = v;
      if (lane == 16) red[warp][6] = v;
    } else if (lane == 0) {
      red[warp][4] = red[warp][5] = red[warp][6] = T(0);
    }
    if (SURR) {
      a = warp_count(ntimeout);
      if (lane == 0) red[warp][26] = T(a);
    } else if (lane == 0) {
      red[warp][26] = T(0);
    }
    if (STAGE == 2) {
      v = warp_min_nonneg(dtmin); if (lane == 0) red[warp][0] = v;
      v = warp_sum3(pM, pW, pE);
      if (lane == 0) red[warp][1] = v;
      if (lane == 8) red[warp][2] = v;
      if (lane == 16) red[warp][3] = v;
      a = warp_count(nactive); if (lane == 0) red[warp][7] = T(a);
      a = warp_count(nbad); if (lane == 0) red[warp][8] = T(a);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        v = warp_max_nonneg(rmax[f]);
        if (lane == 0) red[warp][9 + f] = v;
      }
      v = warp_max_any(lnJh); if (lane == 0) red[warp][23] = v;
      v = warp_max_any(lnJt); if (lane == 0) red[warp][24] = v;
      a = warp_count(nfallback); if (lane == 0) red[warp][25] = T(a);
    } else if (lane == 0) {
      // stage 1 needs the boundary inflow and the timeouts only
      for (int q = 0; q < NPART; ++q)
        if (q < 4 || q > 6) red[warp][q] = q == 26 ? red[warp][q] : T(0);
    }
  }
  __syncthreads();
  if (tid < NPART) {
    const int kind = slot_kind(tid);
    T acc2 = red[0][tid];
    for (int w2 = 1; w2 < NT / 32; ++w2) {
      const T v = red[w2][tid];
      acc2 = kind == 0 ? acc2 + v : (kind == 1 ? (v > acc2 ? v : acc2) : (v < acc2 ? v : acc2));
    }
    // residual max-norms |dU| / dt: rounding is monotone, so scaling the maximum gives the
    // maximum of the scaled values
    if (STAGE == 2 && tid >= 9 && tid < 9 + NF) acc2 *= trcp(dt);
    dc.partials[(size_t)tile * NPART + tid] = double(acc2);
  }
  if (!tile_reduce(dc, by, fin)) return;
  if (tid == 0) publish_stage(dc.hdr, fin, STAGE, dtd, cfl);
}

// Register budget from __launch_bounds__: the register file is split between the SM's four
// schedulers, so 18 warps (two CTAs of 288 threads) leave 96 registers per thread and 9
// warps (one FP64 CTA) 168; a larger cap fails at launch.
template <class TL, class T, int STAGE, bool SURR, bool BI = false, bool SP = false>
__global__ void __launch_bounds__(TL::NT, TL::template minb<T>())
    k_stage(DevCase dc, const T* __restrict__ Uin, const T* Un, T* Uout, const unsigned char* __restrict__ blob) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TcCtx tcx;
  tcx.ready = false;
  if (SURR) {
    // Take the tensor-core resources up front, also in tiles that will not need them: the
    // SM does not start a second CTA of a kernel that uses TMEM until the first has given
    // up its allocation permit, so a lazy allocation would halve the CTAs per SM.
    tcx.tmem = tc_acquire();
    tcx.phase = 0;
    tcx.wphase = 0;
    tcx.ready = true;
  }
  stage_tile<TL, T, STAGE, SURR, BI, SP>(dc, blockIdx.x, blockIdx.y, blockIdx.y * gridDim.x + blockIdx.x, Uin, Un, Uout, blob,
                                 smem_raw, dc.cfl, &tcx);
  if (SURR) tc_release(tcx.tmem);
}

// ---- batched persistent stage ----------------------------------------------------------------
// Many independent cases of uneven size in one launch.  The work list is the concatenation
// of the cases' tiles (largest cases first); persistent CTAs take tiles from an atomic
// counter, so a CTA that drew a cheap tile takes the next one at once.  Each case keeps its
// own workspace (time step, partials, diagnostics): its last tile reduces it as in the
// single-case kernel.  The last CTA to leave resets the counter for the next launch.
// max_tiles bounds the tiles one CTA takes.  The surrogate variant uses a small bound: the
// SM places a further CTA of a kernel that holds TMEM only when one of its CTAs finishes,
// so CTAs that never finished would keep one CTA per SM for the whole launch.
constexpr int MAX_BATCH = 96;
// The work list and the case table travel as the kernel's parameter (__grid_constant__,
// about 28 KB): every field a tile reads is a constant-cache load indexed by the case, with
// no copy into shared memory and no registers to hold it.
struct BatchTable {
  int ncases, total_tiles;
  int tile_start[MAX_BATCH + 1];   // first work-list tile of each slot
  int case_of[MAX_BATCH];          // case index of each work-list slot
  int tiles_x[MAX_BATCH];          // per case
  long long state_off[MAX_BATCH];  // element offset of the case's first plane
  DevCase cases[MAX_BATCH];
};
static_assert(sizeof(BatchTable) + 128 <= 32764, "kernel parameter space");
struct BatchCounters {
  unsigned int next_tile;
  unsigned int exited;
};

template <class TL, class T, int STAGE, bool SURR, bool BI = false>
__global__ void __launch_bounds__(TL::NT, TL::template minb<T>())
    k_batch_stage(const __grid_constant__ BatchTable bt, BatchCounters* __restrict__ ctr, const T* __restrict__ Uin,
                  const T* Un, T* Uout, const unsigned char* __restrict__ blob, double cfl, int max_tiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_t, s_slot;
  const int tid = threadIdx.x;
  const int ncases = bt.ncases, total = bt.total_tiles;
  TcCtx tcx;
  tcx.ready = false;
  if (SURR) {
    tcx.tmem = tc_acquire();   // includes the barrier
    tcx.phase = 0;
    tcx.wphase = 0;
    tcx.ready = true;
  }
  for (int taken = 0; taken < max_tiles; ++taken) {
    if (tid == 0) {
      const int t = (int)atomicAdd(&ctr->next_tile, 1u);
      int lo = 0, hi = ncases;   // slot with tile_start[slot] <= t < tile_start[slot + 1]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (bt.tile_start[mid] <= t) lo = mid; else hi = mid;
      }
      s_t = t;
      s_slot = lo;
    }
    __syncthreads();
    const int t = s_t, slot = s_slot;
    if (t >= total) break;
    const int k = bt.case_of[slot];
    const int lt = t - bt.tile_start[slot], tx = bt.tiles_x[k];
    const long long off = bt.state_off[k];
    stage_tile<TL, T, STAGE, SURR, BI>(bt.cases[k], lt % tx, lt / tx, lt, Uin + off, Un ? Un + off : nullptr, Uout + off,
                                   blob, smem_raw, cfl, &tcx);
    __syncthreads();
  }
  if (SURR) tc_release(tcx.tmem);
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&ctr->exited, 1u) == gridDim.x - 1) {   // every CTA has left the loop
      ctr->next_tile = 0u;
      ctr->exited = 0u;
      __threadfence();
    }
  }
}

// ---- kernels of one tile shape, as seen by the host ---------------------------------------
// Kernel variant index p: 0 FP64, 1 FP32, 2 FP32 + surrogate, 3 FP64 with the bimodal
// liquid, 4 FP32 with the bimodal liquid.  A null entry: that combination does not fit the
// shared memory of an SM.
constexpr int NVARIANT = 5;
struct StageSet {
  int tx, ty, nt;
  size_t smem[NVARIANT];
  int minb[NVARIANT];
  const void* stage[NVARIANT][2];   // k_stage, stages 1 and 2
  const void* stage_sp[2];          // FP64 k_stage with the stored primitives (variant 0)
  const void* batch[NVARIANT][2];   // k_batch_stage (FP32 variants only)
  bool plume_inviscid_only;         // kernels for axisymmetric cases without diffusive fluxes only
  const void* queue[2];             // FP32 + surrogate: the kernel after each stage kernel (or null)
  const void* batch_queue[2];       // the same after each batched stage kernel
  size_t queue_smem;                // their dynamic shared memory
};
constexpr size_t SMEM_LIMIT = 227 * 1024 - 4096;   // opt-in limit minus the static shared memory

template <class TL>
StageSet make_stage_set() {
  StageSet s;
  memset(&s, 0, sizeof(s));
  s.tx = TL::TX;
  s.ty = TL::TY;
  s.nt = TL::NT;
  s.smem[0] = TL::template smem<double>();
  s.smem[1] = TL::template smem<float>();
  s.smem[2] = stage_smem_surr<TL>();
  s.minb[0] = TL::template minb<double>();
  s.minb[1] = s.minb[2] = TL::template minb<float>();
  if constexpr (TL::template smem<double>() <= SMEM_LIMIT) {
    s.stage[0][0] = (const void*)k_stage<TL, double, 1, false>;
    s.stage[0][1] = (const void*)k_stage<TL, double, 2, false>;
    s.stage_sp[0] = (const void*)k_stage<TL, double, 1, false, false, true>;
    s.stage_sp[1] = (const void*)k_stage<TL, double, 2, false, false, true>;
  }
  s.stage[1][0] = (const void*)k_stage<TL, float, 1, false>;
  s.stage[1][1] = (const void*)k_stage<TL, float, 2, false>;
  s.stage[2][0] = (const void*)k_stage<TL, float, 1, true>;
  s.stage[2][1] = (const void*)k_stage<TL, float, 2, true>;
  s.batch[1][0] = (const void*)k_batch_stage<TL, float, 1, false>;
  s.batch[1][1] = (const void*)k_batch_stage<TL, float, 2, false>;
  s.batch[2][0] = (const void*)k_batch_stage<TL, float, 1, true>;
  s.batch[2][1] = (const void*)k_batch_stage<TL, float, 2, true>;
  return s;
}

// The bimodal variants (3, 4) of a shape, instantiated in a translation unit of their own.
template <class TL>
void add_bimodal_variants(StageSet& s) {
  s.smem[3] = TL::template smem<double, NF_BI>();
  s.smem[4] = TL::template smem<float, NF_BI>();
  s.minb[3] = TL::template minb<double>();
  s.minb[4] = TL::template minb<float>();
  if constexpr (TL::template smem<double, NF_BI>() <= SMEM_LIMIT) {
    s.stage[3][0] = (const void*)k_stage<TL, double, 1, false, true>;
    s.stage[3][1] = (const void*)k_stage<TL, double, 2, false, true>;
  }
  if constexpr (TL::template smem<float, NF_BI>() <= SMEM_LIMIT) {
    s.stage[4][0] = (const void*)k_stage<TL, float, 1, false, true>;
    s.stage[4][1] = (const void*)k_stage<TL, float, 2, false, true>;
    s.batch[4][0] = (const void*)k_batch_stage<TL, float, 1, false, true>;
    s.batch[4][1] = (const void*)k_batch_stage<TL, float, 2, false, true>;
  }
}

// Plain FP32 kernels only (variant 1, single-case and batched), for the shapes whose
// registers are budgeted for three CTAs per SM: the FP64 kernels would be those of the
// two-CTA shape, and the surrogate and bimodal FP32 kernels do not fit three CTAs' shared
// memory.
template <class TL>
StageSet make_stage_set_fp32() {
  StageSet s;
  memset(&s, 0, sizeof(s));
  s.tx = TL::TX;
  s.ty = TL::TY;
  s.nt = TL::NT;
  s.smem[1] = TL::template smem<float>();
  s.minb[1] = TL::template minb<float>();
  s.stage[1][0] = (const void*)k_stage<TL, float, 1, false>;
  s.stage[1][1] = (const void*)k_stage<TL, float, 2, false>;
  s.batch[1][0] = (const void*)k_batch_stage<TL, float, 1, false>;
  s.batch[1][1] = (const void*)k_batch_stage<TL, float, 2, false>;
  return s;
}

// Plain FP64 kernels only (variant 0), for a shape whose registers and shared memory are
// budgeted for two FP64 CTAs per SM.
template <class TL>
StageSet make_stage_set_fp64() {
  StageSet s;
  memset(&s, 0, sizeof(s));
  s.tx = TL::TX;
  s.ty = TL::TY;
  s.nt = TL::NT;
  s.smem[0] = TL::template smem<double>();
  s.minb[0] = TL::template minb<double>();
  s.stage[0][0] = (const void*)k_stage<TL, double, 1, false>;
  s.stage[0][1] = (const void*)k_stage<TL, double, 2, false>;
  s.stage_sp[0] = (const void*)k_stage<TL, double, 1, false, false, true>;
  s.stage_sp[1] = (const void*)k_stage<TL, double, 2, false, false, true>;
  return s;
}

// the tile shapes the library is built with (one translation unit each)
constexpr int NSHAPES = 10;
// 0: 32x8 (default), 1: 16x16, 2: 32x16, 3: 64x8, 4: 16x16 and 5: 32x8 with three FP32 CTAs
// per SM, 6: 16x12, 7: 16x16 and 8: 16x14 with two FP64 CTAs per SM
const StageSet* stage_set(int shape);

}  // namespace ct
