// stage_sweep.cuh -- the FP32 stage of an axisymmetric plume as column sweeps.
//
// The same SSP-RK2 stage as stage_tile (Sec. 3.2: MUSCL/van Leer, Roe fluxes, axisymmetric
// source, phase-change source, RK combine, partials), organised for the instruction issue
// of sm_103a instead of shared-memory staging of faces.  A warp owns a strip of 28 cells in
// x (lanes 2..29; lanes 0, 1, 30 and 31 carry the two-column halo) and sweeps R rows in r,
// one row per iteration, with no CTA barrier:
//   - x direction inside the warp: neighbour values from a three-row ring of primitive
//     vectors in shared memory, the right face state and the west flux by shuffles, one
//     x-face flux per lane;
//   - r direction along the sweep: per lane, the upper face state of the row below and the
//     flux of its south face wait in shared memory from one row to the next, so every r face
//     is reconstructed and fluxed once;
//   - a cell that the FP32 source screen keeps takes its phase-change source after the row's
//     fluxes are stored (its divergence parked in the lane's slot), where the FP64 island
//     finds few values live.
// Every cell value is computed by the same expressions in the same order as in stage_tile,
// so the state is bitwise that of the other tile shapes; only the summation order of the
// FP64 totals differs (compensated FP32 sums per lane, FP64 from the warp on).  Dry rows
// (the particle moments +0 in all 32 columns; level 2: the soot too) skip the reconstruction
// of the all-moment field pairs (and the soot pair), whose face states are then +0, and the
// Y_l, Y_s terms of the face thermodynamics, which drop out exactly: the bits of the full
// formulas.  Variant: FP32, axisymmetric, without the diffusive fluxes, one liquid set;
// plain source, or (Q) FP32 + surrogate through a queue that k_sweep_queue works off.  Both
// have a batched persistent form (k_batch_sweep, k_batch_queue).
#pragma once
#include "stage.cuh"

namespace ct {

template <int W_, int R_, int MINB_>
struct SweepTile {
  static constexpr int W = W_, R = R_, MINB = MINB_;
  static constexpr int TX = 28, TY = W * R, NT = 32 * W;
};

// Kahan-compensated FP32 running sum of one lane's cells
struct KSum {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

__device__ __forceinline__ float2 shfl_up2(float2 v) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
}
__device__ __forceinline__ float2 shfl_down2(float2 v) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
}

// Q (FP32 + surrogate): the cells the screen keeps are not finished here but queued, with
// their flux divergence, for k_sweep_queue, which runs the surrogate on them; the stage's
// record then waits in the header (pre) for that kernel to complete and publish it.
// One strip tile (bx, by) of a case; `tile` = by * tiles_x + bx indexes the partial records.
template <class ST, int STAGE, bool Q>
__device__ __forceinline__ void sweep_tile(const DevCase& dc, int bx, int by, int tile, const float* __restrict__ Uin,
                                           const float* Un, float* Uout, double cfl) {
  using T = float;
  using V = float2;
  constexpr int NP = NF / 2;
  constexpr int R = ST::R;
  __shared__ double red[ST::W][NPART];
  __shared__ double fin[NPART];
  // per warp, per lane: the primitive vectors of three consecutive rows (a ring indexed by
  // row mod 3), row j's upper r-face state, the flux of the face below row j, row j's x
  // divergence, and (lane 0) the running residual maxima
  __shared__ float2 s_q[ST::W][3][NP][32];
  __shared__ float2 s_fhi[ST::W][NP][32], s_fs[ST::W][NP][32], s_acc[ST::W][NP][32];
  __shared__ float s_rmax[ST::W][NF];
  // per warp, per lane: the temperature of the three rows of the ring (the cell update's
  // source screen takes the primitive variables from the ring instead of recomputing them)
  __shared__ float s_T[ST::W][3][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nx = dc.nx, nr = dc.nr;
  const size_t N = (size_t)nx * nr;
  const int i0 = bx * ST::TX;
  const int i = i0 - 2 + lane;                       // this lane's column
  const int jb = by * ST::TY + warp * R;             // the warp's first row
  const int je = min(jb + R, nr);                    // one past its last row
  const double dtd = dc.hdr->dt_cur;
  const T dt = T(dtd);
  const Geo<T> g = geo_of(dc, T(0));
  const bool xin = i >= 0 && i < nx;
  const bool cell_col = lane >= 2 && lane < 30 && i < nx;   // the lane owns cells of this column
  const bool wall = g.wall_len > T(0) && (T(i) + T(0.5)) * g.dx < g.wall_len;
  const bool edge = i0 == 0 || i0 + ST::TX >= nx;           // the strip touches x = 0 or x = L_x
  const int lm = lane > 0 ? lane - 1 : 0, lp = lane < 31 ? lane + 1 : 31;
  const auto slot = [](int j) { return (j + 3) % 3; };   // j >= -2

  // primitive vector (stage_tile's phase A) of cell (i, j) of the stencil; zero where no
  // cell of the strip needs it (corners, columns beyond the halo).  Returns whether the row
  // is dry (1: every moment field (5..12) of the primitive vectors of the warp's 32 columns
  // is +0; 2: the soot field too, as in the air around a plume's core) or not (0).
  const auto load_q = [&](int j, V* q, T& Tg) -> int {
    const bool rin = j >= 0 && j < nr;
    if ((xin || rin) && i >= -2 && i <= nx + 1 && j >= -2 && j <= nr + 1) {
      T u14[NF];
      if (xin && rin) {
        const size_t n = (size_t)j * nx + i;
#pragma unroll
        for (int f = 0; f < NF; ++f) u14[f] = Uin[f * N + n];
      } else {   // out of line, through its own array: u14 stays in registers
        T g14[NF];
        load_ghost<T, NF>(dc, Uin, N, i, j, g14);
#pragma unroll
        for (int f = 0; f < NF; ++f) u14[f] = g14[f];
      }
      Prim<T> w;
      cons_to_prim<T, false>(u14, w);
      T qv[NF];
      prim_vector<T, false>(w, qv);
#pragma unroll
      for (int k2 = 0; k2 < NP; ++k2) q[k2] = p_make(qv[2 * k2], qv[2 * k2 + 1]);
      Tg = w.Tg;
    } else {
#pragma unroll
      for (int k2 = 0; k2 < NP; ++k2) q[k2] = p_make(T(0), T(0));
      Tg = T(0);
    }
    unsigned zb = 0;
#pragma unroll
    for (int k2 = 2; k2 < NP; ++k2) zb |= (k2 == 2 ? 0u : __float_as_uint(q[k2].x)) | (k2 == 6 ? 0u : __float_as_uint(q[k2].y));
    const unsigned zs = __float_as_uint(q[6].y);   // soot
    const int dry = __all_sync(0xffffffffu, zb == 0u) ? 1 : 0;
    return dry + (__all_sync(0xffffffffu, (zb | zs) == 0u) ? 1 : 0);
  };

  // running partials of this lane's cells
  KSum sM, sW, sE;
  T bm = T(0), bw = T(0), be = T(0);
  T dtmin = T(INFINITY);
  T lnJh = T(-INFINITY), lnJt = T(-INFINITY);
  int nactive = 0, nbad = 0;
  if (lane < NF) s_rmax[warp][lane] = T(0);

  // dry rows around the current row j: bit 0 row j-1, bit 1 row j, bit 2 row j+1, bit 3
  // row j+2 (warp-uniform)
  unsigned rowdry = 0, rowsoot = 0;   // rowsoot: the same bits for the soot-free rows
  if (jb < je) {
    // rows jb-2 .. jb+1: the upper face state of row jb-1, row jb's lower face state, and the
    // flux of the face between rows jb-1 and jb; rows jb-1 .. jb+1 stay in the ring
    {
      V qm[NP], q0[NP], q1[NP], q2[NP];
      T Tm, T0, T1, T2;
      load_q(jb - 2, qm, Tm);
      const int l0 = load_q(jb - 1, q0, T0), l1 = load_q(jb, q1, T1), l2 = load_q(jb + 1, q2, T2);
      rowdry = (l0 > 0 ? 1u : 0u) | (l1 > 0 ? 2u : 0u) | (l2 > 0 ? 4u : 0u);
      rowsoot = (l0 > 1 ? 1u : 0u) | (l1 > 1 ? 2u : 0u) | (l2 > 1 ? 4u : 0u);
      s_T[warp][slot(jb - 1)][lane] = T0;
      s_T[warp][slot(jb)][lane] = T1;
      s_T[warp][slot(jb + 1)][lane] = T2;
      T qL[NF], qR[NF], F[NF];
#pragma unroll
      for (int k2 = 0; k2 < NP; ++k2) {
        V lo, hi;
        vl_faces2(qm[k2], q0[k2], q1[k2], lo, hi);     // row jb-1
        qL[2 * k2] = hi.x;
        qL[2 * k2 + 1] = hi.y;
        vl_faces2(q0[k2], q1[k2], q2[k2], lo, hi);     // row jb
        qR[2 * k2] = lo.x;
        qR[2 * k2 + 1] = lo.y;
        s_fhi[warp][k2][lane] = hi;
        s_q[warp][slot(jb - 1)][k2][lane] = q0[k2];
        s_q[warp][slot(jb)][k2][lane] = q1[k2];
        s_q[warp][slot(jb + 1)][k2][lane] = q2[k2];
      }
      roe_flux<T, 1, NF>(qL, qR, F);
#pragma unroll
      for (int k2 = 0; k2 < NP; ++k2) s_fs[warp][k2][lane] = p_make(F[2 * k2], F[2 * k2 + 1]);
    }
    __syncwarp();
    // invariant at the top of iteration j: rows j-1, j, j+1 in the ring; row j's upper face
    // state and the flux of the face between rows j-1 and j in shared memory
    for (int j = jb; j < je; ++j) {
      const int sj = slot(j), sj1 = slot(j + 1), sj2 = slot(j + 2);
      // x direction, row j: slopes from the neighbours' values, the face i+1/2 per lane,
      // the divergence from the west neighbour's face.  A dry row: the all-moment pairs have
      // zero slopes and +0 face states (vl_faces2 of three +0 values gives hi = +0, lo = +0)
      const auto xphase = [&](auto dry_tag) {
        constexpr int LEVEL = decltype(dry_tag)::value;
        constexpr bool DRY = LEVEL > 0;
        T qL[NF], qR[NF], F[NF];
#pragma unroll
        for (int k2 = 0; k2 < NP; ++k2) {
          if ((DRY && moment_pair(k2)) || (LEVEL == 2 && k2 == NP - 1)) {
            qL[2 * k2] = qL[2 * k2 + 1] = qR[2 * k2] = qR[2 * k2 + 1] = T(0);
            continue;
          }
          V lo, hi;
          vl_faces2(s_q[warp][sj][k2][lm], s_q[warp][sj][k2][lane], s_q[warp][sj][k2][lp], lo, hi);
          const V r = shfl_down2(lo);
          qL[2 * k2] = hi.x;
          qL[2 * k2 + 1] = hi.y;
          qR[2 * k2] = r.x;
          qR[2 * k2 + 1] = r.y;
        }
        roe_flux<T, 0, NF, DRY>(qL, qR, F);
        const V cw2 = p_make(g.idx, g.idx), nce2 = p_make(-g.idx, -g.idx);
#pragma unroll
        for (int k2 = 0; k2 < NP; ++k2) {
          const V fe = p_make(F[2 * k2], F[2 * k2 + 1]);
          s_acc[warp][k2][lane] = p_fma(cw2, shfl_up2(fe), p_mul(nce2, fe));
        }
        if (edge) {   // boundary inflow rates of the inflow and outflow columns
          const T area = (T(j) + T(0.5)) * g.dr * g.dr;
          const T w0 = __shfl_up_sync(0xffffffffu, F[0], 1), w3 = __shfl_up_sync(0xffffffffu, F[3], 1);
          const T w4 = __shfl_up_sync(0xffffffffu, F[4], 1), w8 = __shfl_up_sync(0xffffffffu, F[8], 1);
          const T w12 = __shfl_up_sync(0xffffffffu, F[12], 1);
          if (cell_col) {
            if (i == 0) {
              bm += area * w0;
              bw += area * (w4 + T(k::YL3) * w8 + T(k::YS3) * w12);
              be += area * w3;
            }
            if (i == nx - 1) {
              bm -= area * F[0];
              bw -= area * (F[4] + T(k::YL3) * F[8] + T(k::YS3) * F[12]);
              be -= area * F[3];
            }
          }
        }
      };
      if (rowsoot & 2u)
        xphase(std::integral_constant<int, 2>{});
      else if (rowdry & 2u)
        xphase(std::integral_constant<int, 1>{});
      else
        xphase(std::integral_constant<int, 0>{});
      // r direction: row j+2 into the ring (over row j-1), row j+1's slope, face j+1/2.
      // Rows j-1 .. j+2 dry: the all-moment pairs of both face states are +0 (row j's upper
      // face state came from rows j-1 .. j+1)
      V Fn[NP];
      V qc[NP];
      T Tc;
      {
        const int lc = load_q(j + 2, qc, Tc);
        rowdry |= lc > 0 ? 8u : 0u;
        rowsoot |= lc > 1 ? 8u : 0u;
      }
      const auto rphase = [&](auto dry_tag) {
        constexpr int LEVEL = decltype(dry_tag)::value;
        constexpr bool DRY = LEVEL > 0;
        T qL[NF], qR[NF], F[NF];
#pragma unroll
        for (int k2 = 0; k2 < NP; ++k2) {
          if ((DRY && moment_pair(k2)) || (LEVEL == 2 && k2 == NP - 1)) {
            qL[2 * k2] = qL[2 * k2 + 1] = qR[2 * k2] = qR[2 * k2 + 1] = T(0);
            s_fhi[warp][k2][lane] = p_make(T(0), T(0));
            continue;
          }
          V lo, hi;
          vl_faces2(s_q[warp][sj][k2][lane], s_q[warp][sj1][k2][lane], qc[k2], lo, hi);
          const V fl = s_fhi[warp][k2][lane];
          qL[2 * k2] = fl.x;
          qL[2 * k2 + 1] = fl.y;
          qR[2 * k2] = lo.x;
          qR[2 * k2 + 1] = lo.y;
          s_fhi[warp][k2][lane] = hi;   // row j+1's upper face state, for the next iteration
        }
        __syncwarp();                   // every lane has read row j's values above
#pragma unroll
        for (int k2 = 0; k2 < NP; ++k2) s_q[warp][sj2][k2][lane] = qc[k2];
        s_T[warp][sj2][lane] = Tc;
        roe_flux<T, 1, NF, DRY>(qL, qR, F);
#pragma unroll
        for (int k2 = 0; k2 < NP; ++k2) Fn[k2] = p_make(F[2 * k2], F[2 * k2 + 1]);
      };
      if ((rowsoot & 15u) == 15u)
        rphase(std::integral_constant<int, 2>{});
      else if ((rowdry & 15u) == 15u)
        rphase(std::integral_constant<int, 1>{});
      else
        rphase(std::integral_constant<int, 0>{});
      // cell (i, j): r divergence, sources, RK combine, partials (stage_tile's phase E).  A cell
      // the FP32 screen does not rule out takes its phase-change source after the row's other
      // work, its divergence parked in s_acc: there the FP64 island runs with few values live
      // and needs no spills, and the screened cells never pay for its registers.
      T rf[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) rf[f] = T(0);
      // RK combine, output and partials of cell n = (i, j) whose rates (flux divergence and
      // sources) are in a
      const auto finish = [&](size_t n, const T* u14, const T* a) {
        T out[NF];
        const V dt2 = p_make(dt, dt);
        if (STAGE == 1) {
#pragma unroll
          for (int k2 = 0; k2 < NP; ++k2) {
            const V o = p_fma(dt2, p_make(a[2 * k2], a[2 * k2 + 1]), p_make(u14[2 * k2], u14[2 * k2 + 1]));
            out[2 * k2] = o.x;
            out[2 * k2 + 1] = o.y;
          }
        } else {
          const V half2 = p_make(T(0.5), T(0.5));
#pragma unroll
          for (int k2 = 0; k2 < NP; ++k2) {
            const V un2 = p_make(Un[(2 * k2) * N + n], Un[(2 * k2 + 1) * N + n]);
            const V t = p_fma(dt2, p_make(a[2 * k2], a[2 * k2 + 1]), p_make(u14[2 * k2], u14[2 * k2 + 1]));
            const V o = p_fma(half2, un2, p_mul(half2, t));
            out[2 * k2] = o.x;
            out[2 * k2 + 1] = o.y;
            rf[2 * k2] = m_fabs(o.x - un2.x);
            rf[2 * k2 + 1] = m_fabs(o.y - un2.y);
          }
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          Uout[f * N + n] = out[f];
          nbad += finite_bits(out[f]) ? 0 : 1;
        }
        if (STAGE == 2) {
          Prim<T> wn;
          cons_to_prim<T, false>(out, wn);
          const T cdt = cell_dt<T>(dc, g, wn);
          dtmin = cdt < dtmin ? cdt : dtmin;
          const T vol = (T(j) + T(0.5)) * g.dr * g.dr * g.dx;
          sM.add(vol * out[0]);
          sW.add(vol * (out[4] + T(k::YL3) * out[8] + T(k::YS3) * out[12]));
          sE.add(vol * out[3]);
        }
      };
      bool pending = false;
      if (cell_col) {
        const size_t n = (size_t)j * nx + i;
        T u14[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) u14[f] = Uin[f * N + n];
        // the primitive variables the update and the screen use, from the ring: the bits
        // cons_to_prim gave for this cell's values when the row entered it
        Prim<T> w;
        {
          T qv[NF];
#pragma unroll
          for (int k2 = 0; k2 < NP; ++k2) {
            const V a = s_q[warp][sj][k2][lane];
            qv[2 * k2] = a.x;
            qv[2 * k2 + 1] = a.y;
          }
          w.rho = qv[0];
          w.p = qv[3];
          w.Yv = qv[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            w.ml[q] = qv[5 + q];
            w.ms[q] = qv[9 + q];
          }
          w.Tg = s_T[warp][sj][lane];
        }
        T acc[NF];
        const T ijh = trcp(T(j) + T(0.5));
        const T cs = T(j) * ijh * g.idr;
        const T cn = T(j + 1) * ijh * g.idr;
        const bool wall_s = wall && j == dc.jw, wall_n = wall && j == dc.jw - 1;
        {
          const V cs2 = p_make(cs, cs), ncn2 = p_make(-cn, -cn);
#pragma unroll
          for (int k2 = 0; k2 < NP; ++k2) {
            V fs = s_fs[warp][k2][lane], fn = Fn[k2];
            if (wall_n) fn = p_make(k2 == 1 ? w.p : T(0), T(0));
            if (wall_s) fs = p_make(k2 == 1 ? w.p : T(0), T(0));
            const V a = p_add(s_acc[warp][k2][lane], p_fma(cs2, fs, p_mul(ncn2, fn)));
            acc[2 * k2] = a.x;
            acc[2 * k2 + 1] = a.y;
          }
        }
        acc[2] += w.p * ijh * g.idr;
        if (j == nr - 1) {
          const T An = T(nr) * g.dr * g.dx;
          bm -= An * Fn[0].x;
          bw -= An * (Fn[2].x + T(k::YL3) * Fn[4].x + T(k::YS3) * Fn[6].x);
          be -= An * Fn[1].y;
        }
        // phase_source's own screen: no phase change, or (kinetic model) no population and
        // clearly below liquid saturation, gives a zero source
        bool pl, ps;
        pending = dc.sc.phase_change && (dc.sc.equilibrium || populations(w, pl, ps) || !clearly_inactive(w));
        if (pending) {
#pragma unroll
          for (int k2 = 0; k2 < NP; ++k2) s_acc[warp][k2][lane] = p_make(acc[2 * k2], acc[2 * k2 + 1]);
        } else {
          finish(n, u14, acc);
        }
      }
#pragma unroll
      for (int k2 = 0; k2 < NP; ++k2) s_fs[warp][k2][lane] = Fn[k2];
      if constexpr (Q) {
        // queue the row's kept cells: one atomic per warp, slots in lane order
        const unsigned pm = __ballot_sync(0xffffffffu, pending);
        if (pm != 0u) {
          unsigned base = 0u;
          if (lane == 0) base = atomicAdd(&dc.hdr->qcount, (unsigned)__popc(pm));
          base = __shfl_sync(0xffffffffu, base, 0);
          if (pending) {
            const unsigned k = base + (unsigned)__popc(pm & ((1u << lane) - 1u));
            queue_cells(dc)[k] = (unsigned)((size_t)j * nx + i);
            float* qacc = queue_rates(dc, N);
#pragma unroll
            for (int k2 = 0; k2 < NP; ++k2) {
              const V a = s_acc[warp][k2][lane];
              qacc[(size_t)(2 * k2) * N + k] = a.x;
              qacc[(size_t)(2 * k2 + 1) * N + k] = a.y;
            }
          }
        }
      } else if (pending) {
        const size_t n = (size_t)j * nx + i;
        T u14[NF], acc[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) u14[f] = Uin[f * N + n];
#pragma unroll
        for (int k2 = 0; k2 < NP; ++k2) {
          const V a = s_acc[warp][k2][lane];
          acc[2 * k2] = a.x;
          acc[2 * k2 + 1] = a.y;
        }
        Prim<T> w;
        cons_to_prim<T, false>(u14, w);
        T Qs[NF];
        double lnJ2[2];
        if (phase_source<T, false>(w, u14, acc, dt, dc.sc, Qs, lnJ2, nullptr)) {
          nactive += 1;
          lnJh = fmaxf(lnJh, T(lnJ2[0]));
          lnJt = fmaxf(lnJt, T(lnJ2[1]));
#pragma unroll
          for (int f = 4; f < 13; ++f) acc[f] += Qs[f];
        }
        finish(n, u14, acc);
      }
      if (STAGE == 2) {   // residual maxima of the row: one warp reduction per field
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const T m = warp_max_nonneg(rf[f]);
          if (lane == 0) s_rmax[warp][f] = m > s_rmax[warp][f] ? m : s_rmax[warp][f];
        }
      }
      rowdry >>= 1;
      rowsoot >>= 1;
      __syncwarp();
    }
  }

  // warp partials in FP64 (one conversion per lane), CTA record in a fixed order
  {
    const double b0 = warp_sum(double(bm)), b1 = warp_sum(double(bw)), b2 = warp_sum(double(be));
    if (lane == 0) {
      for (int q = 0; q < NPART; ++q) red[warp][q] = 0.0;
      red[warp][4] = b0;
      red[warp][5] = b1;
      red[warp][6] = b2;
    }
    if (STAGE == 2) {
      const double m = warp_sum(double(sM.s) - double(sM.c));
      const double wt = warp_sum(double(sW.s) - double(sW.c));
      const double e = warp_sum(double(sE.s) - double(sE.c));
      const T dmin = warp_min_nonneg(dtmin);
      const int na = warp_count(nactive), nb = warp_count(nbad);
      const T jh = warp_max_any(lnJh), jt = warp_max_any(lnJt);
      if (lane == 0) {
        red[warp][0] = double(dmin);
        red[warp][1] = m;
        red[warp][2] = wt;
        red[warp][3] = e;
        red[warp][7] = double(na);
        red[warp][8] = double(nb);
        // residual max-norms |dU|/dt: the maximum scaled once (rounding is monotone)
#pragma unroll
        for (int f = 0; f < NF; ++f) red[warp][9 + f] = double(s_rmax[warp][f] * trcp(dt));
        red[warp][23] = double(jh);
        red[warp][24] = double(jt);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < NPART) {
    const int q = threadIdx.x, kind = slot_kind(q);
    double a = red[0][q];
    for (int w2 = 1; w2 < ST::W; ++w2) {
      const double v = red[w2][q];
      a = kind == 0 ? a + v : (kind == 1 ? (v > a ? v : a) : (v < a ? v : a));
    }
    dc.partials[(size_t)tile * NPART + q] = a;
  }
  if (!tile_reduce(dc, by, fin)) return;
  if (threadIdx.x == 0) {
    if (Q) {
      for (int q = 0; q < NPART; ++q) dc.hdr->pre[q] = fin[q];
    } else {
      publish_stage(dc.hdr, fin, STAGE, dtd, cfl);
    }
  }
}

template <class ST, int STAGE, bool Q = false>
__global__ void __launch_bounds__(ST::NT, ST::MINB)
    k_sweep(DevCase dc, const float* __restrict__ Uin, const float* Un, float* Uout,
            const unsigned char* __restrict__ blob) {
  sweep_tile<ST, STAGE, Q>(dc, blockIdx.x, blockIdx.y, blockIdx.y * gridDim.x + blockIdx.x, Uin, Un, Uout, dc.cfl);
}

// The batched persistent form (k_batch_stage's work list: CTAs take strip tiles of any case
// from an atomic counter, largest cases first; the last CTA to leave resets the counter).
template <class ST, int STAGE, bool Q>
__global__ void __launch_bounds__(ST::NT, ST::MINB)
    k_batch_sweep(const __grid_constant__ BatchTable bt, BatchCounters* __restrict__ ctr, const float* __restrict__ Uin,
                  const float* Un, float* Uout, const unsigned char* __restrict__ blob, double cfl, int max_tiles) {
  __shared__ int s_t, s_slot;
  const int tid = threadIdx.x;
  const int ncases = bt.ncases, total = bt.total_tiles;
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
    sweep_tile<ST, STAGE, Q>(bt.cases[k], lt % tx, lt / tx, lt, Uin + off, Un ? Un + off : nullptr, Uout + off, cfl);
    __syncthreads();
  }
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&ctr->exited, 1u) == gridDim.x - 1) {   // every CTA has left the loop
      ctr->next_tile = 0u;
      ctr->exited = 0u;
      __threadfence();
    }
  }
}

// ---- the surrogate kernel of the FP32 + surrogate step through the column sweep ----------
// The cells k_sweep<..., Q = true> queued (those its screen keeps), 256 at a time, take the
// fused path's source (surrogate_source: the features, the BF16 tensor-core network inside
// the training hull, the plain source outside it, the exact tail), then the RK combine, the
// output and the partials; the last CTA merges its record with the sweep's and publishes
// the stage.  A persistent grid: the queue's length is known on the device only.
// The queue of one case (all threads of every CTA of the launch; tcx: the CTA's tensor-core
// resources, taken once per launch; pub: the CTA that publishes the stage when nothing is
// queued).
template <int STAGE>
__device__ __forceinline__ void queue_case(const DevCase& dc, const float* __restrict__ Uin, const float* Un,
                                           float* Uout, const unsigned char* __restrict__ blob, double cfl,
                                           TcCtx* tcx, unsigned char* smem_raw, int pub) {
  using T = float;
  using V = float2;
  constexpr int NT = QueueTile::NT, NP = NF / 2;
  __shared__ double red[NT / 32][NPART];
  __shared__ double fin[NPART];
  __shared__ unsigned int s_ticket;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nx = dc.nx;
  const size_t N = (size_t)nx * dc.nr;
  const unsigned count = dc.hdr->qcount;
  const double dtd = dc.hdr->dt_cur;
  if (count == 0u) {   // nothing queued: the sweep's record is the stage's (merging adds nothing)
    if ((int)blockIdx.x == pub && tid == 0) publish_stage(dc.hdr, dc.hdr->pre, STAGE, dtd, cfl);
    return;
  }
  const T dt = T(dtd);
  const Geo<T> g = geo_of(dc, T(0));
  KSum sM, sW, sE;
  T dtmin = T(INFINITY);
  T rmax[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) rmax[f] = T(0);
  T lnJh = T(-INFINITY), lnJt = T(-INFINITY);
  int nactive = 0, nbad = 0, nfallback = 0, ntimeout = 0;
  for (unsigned base = blockIdx.x * NT; base < count; base += gridDim.x * NT) {   // uniform
    const unsigned k = base + tid;
    const bool cell = k < count;
    size_t n = 0;
    T u14[NF], acc[NF];
    Prim<T> w{};
    if (cell) {
      n = queue_cells(dc)[k];
      const float* qacc = queue_rates(dc, N);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        u14[f] = Uin[f * N + n];
        acc[f] = qacc[(size_t)f * N + k];
      }
      cons_to_prim<T, false>(u14, w);
    } else {
#pragma unroll
      for (int f = 0; f < NF; ++f) u14[f] = acc[f] = T(0);
    }
    int na = 0, nf = 0;
    T jh = T(-INFINITY), jt = T(-INFINITY);
    surrogate_source<QueueTile, T>(dc, blob, cell, w, u14, acc, dt, na, nf, ntimeout, jh, jt, smem_raw, tcx);
    if (cell) {
      nactive += na;
      nfallback += nf;
      lnJh = fmaxf(lnJh, jh);
      lnJt = fmaxf(lnJt, jt);
      // the sweep's RK combine, output and partials
      T out[NF];
      const V dt2 = p_make(dt, dt);
      if (STAGE == 1) {
#pragma unroll
        for (int k2 = 0; k2 < NP; ++k2) {
          const V o = p_fma(dt2, p_make(acc[2 * k2], acc[2 * k2 + 1]), p_make(u14[2 * k2], u14[2 * k2 + 1]));
          out[2 * k2] = o.x;
          out[2 * k2 + 1] = o.y;
        }
      } else {
        const V half2 = p_make(T(0.5), T(0.5));
#pragma unroll
        for (int k2 = 0; k2 < NP; ++k2) {
          const V un2 = p_make(Un[(2 * k2) * N + n], Un[(2 * k2 + 1) * N + n]);
          const V t = p_fma(dt2, p_make(acc[2 * k2], acc[2 * k2 + 1]), p_make(u14[2 * k2], u14[2 * k2 + 1]));
          const V o = p_fma(half2, un2, p_mul(half2, t));
          out[2 * k2] = o.x;
          out[2 * k2 + 1] = o.y;
          const T r0 = m_fabs(o.x - un2.x), r1 = m_fabs(o.y - un2.y);
          rmax[2 * k2] = r0 > rmax[2 * k2] ? r0 : rmax[2 * k2];
          rmax[2 * k2 + 1] = r1 > rmax[2 * k2 + 1] ? r1 : rmax[2 * k2 + 1];
        }
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        Uout[f * N + n] = out[f];
        nbad += finite_bits(out[f]) ? 0 : 1;
      }
      if (STAGE == 2) {
        Prim<T> wn;
        cons_to_prim<T, false>(out, wn);
        const T cdt = cell_dt<T>(dc, g, wn);
        dtmin = cdt < dtmin ? cdt : dtmin;
        const int j = (int)(n / (size_t)nx);
        const T vol = (T(j) + T(0.5)) * g.dr * g.dr * g.dx;
        sM.add(vol * out[0]);
        sW.add(vol * (out[4] + T(k::YL3) * out[8] + T(k::YS3) * out[12]));
        sE.add(vol * out[3]);
      }
    }
  }
  // warp records in FP64, the CTA's record in a fixed order (the sweep's layout)
  {
    const int nt = warp_count(ntimeout);
    if (lane == 0) {
      for (int q = 0; q < NPART; ++q) red[warp][q] = 0.0;
      red[warp][26] = double(nt);
    }
    if (STAGE == 2) {
      const double m = warp_sum(double(sM.s) - double(sM.c));
      const double wt = warp_sum(double(sW.s) - double(sW.c));
      const double e = warp_sum(double(sE.s) - double(sE.c));
      const T dmin = warp_min_nonneg(dtmin);
      const int na = warp_count(nactive), nb = warp_count(nbad), nfb = warp_count(nfallback);
      const T jh = warp_max_any(lnJh), jt = warp_max_any(lnJt);
      T rm[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) rm[f] = warp_max_nonneg(rmax[f]);
      if (lane == 0) {
        red[warp][0] = double(dmin);
        red[warp][1] = m;
        red[warp][2] = wt;
        red[warp][3] = e;
        red[warp][7] = double(na);
        red[warp][8] = double(nb);
#pragma unroll
        for (int f = 0; f < NF; ++f) red[warp][9 + f] = double(rm[f] * trcp(dt));
        red[warp][23] = double(jh);
        red[warp][24] = double(jt);
        red[warp][25] = double(nfb);
      }
    }
  }
  __syncthreads();
  if (tid < NPART) {
    const int kind = slot_kind(tid);
    double a = red[0][tid];
    for (int w2 = 1; w2 < NT / 32; ++w2) {
      const double v = red[w2][tid];
      a = kind == 0 ? a + v : (kind == 1 ? (v > a ? v : a) : (v < a ? v : a));
    }
    queue_partials(dc, N)[(size_t)blockIdx.x * NPART + tid] = a;
  }
  // the last CTA to finish merges the records with the sweep's and publishes the stage
  __threadfence();
  __syncthreads();
  if (tid == 0) s_ticket = atomicAdd(&dc.hdr->qticket, 1u);
  __syncthreads();
  if (s_ticket != gridDim.x - 1) return;
  __threadfence();
  reduce_records(queue_partials(dc, N), gridDim.x, fin);
  if (tid == 0) {
    WsHeader* h = dc.hdr;
    double m[NPART];
    for (int q = 0; q < NPART; ++q) {
      const int kind = slot_kind(q);
      const double a = h->pre[q], b = fin[q];
      m[q] = kind == 0 ? a + b : (kind == 1 ? (b > a ? b : a) : (b < a ? b : a));
    }
    publish_stage(h, m, STAGE, dtd, cfl);
    h->qcount = 0u;
    h->qticket = 0u;
  }
}

template <int STAGE>
__global__ void __launch_bounds__(QueueTile::NT, 2)
    k_sweep_queue(DevCase dc, const float* __restrict__ Uin, const float* Un, float* Uout,
                  const unsigned char* __restrict__ blob) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (dc.hdr->qcount == 0u) {   // nothing queued: publish the sweep's record, take no TMEM
    if (blockIdx.x == 0 && threadIdx.x == 0) publish_stage(dc.hdr, dc.hdr->pre, STAGE, dc.hdr->dt_cur, dc.cfl);
    return;
  }
  // tensor-core resources up front (a CTA that has given up its allocation permit may not
  // allocate again)
  TcCtx tcx;
  tcx.tmem = tc_acquire();
  tcx.phase = 0;
  tcx.wphase = 0;
  tcx.ready = true;
  queue_case<STAGE>(dc, Uin, Un, Uout, blob, dc.cfl, &tcx, smem_raw, 0);
  tc_release(tcx.tmem);
}

// The batched form: the queues of every case of a batch in turn (cases without one skip).
template <int STAGE>
__global__ void __launch_bounds__(QueueTile::NT, 2)
    k_batch_queue(const __grid_constant__ BatchTable bt, const float* __restrict__ Uin, const float* Un, float* Uout,
                  const unsigned char* __restrict__ blob, double cfl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // nothing queued in any case: each case's record is published by one CTA, no TMEM taken.
  // (Every CTA reads the counts before any is reset: a count is reset only after all CTAs
  // have passed that case.)
  int any = 0;
  for (int k = threadIdx.x; k < bt.ncases; k += blockDim.x)
    any |= (bt.cases[k].qoff != 0 && bt.cases[k].hdr->qcount != 0u) ? 1 : 0;
  if (!__syncthreads_or(any)) {
    if (threadIdx.x == 0)
      for (int k = blockIdx.x; k < bt.ncases; k += gridDim.x)
        if (bt.cases[k].qoff != 0)
          publish_stage(bt.cases[k].hdr, bt.cases[k].hdr->pre, STAGE, bt.cases[k].hdr->dt_cur, cfl);
    return;
  }
  TcCtx tcx;
  tcx.tmem = tc_acquire();
  tcx.phase = 0;
  tcx.wphase = 0;
  tcx.ready = true;
  for (int k = 0; k < bt.ncases; ++k) {
    if (bt.cases[k].qoff == 0) continue;
    const long long off = bt.state_off[k];
    queue_case<STAGE>(bt.cases[k], Uin + off, Un ? Un + off : nullptr, Uout + off, blob, cfl, &tcx, smem_raw,
                      k % (int)gridDim.x);
    __syncthreads();
  }
  tc_release(tcx.tmem);
}

template <class ST>
StageSet make_stage_set_sweep() {
  StageSet s;
  memset(&s, 0, sizeof(s));
  s.tx = ST::TX;
  s.ty = ST::TY;
  s.nt = ST::NT;
  s.smem[1] = 0;
  s.minb[1] = ST::MINB;
  s.stage[1][0] = (const void*)k_sweep<ST, 1>;
  s.stage[1][1] = (const void*)k_sweep<ST, 2>;
  // FP32 + surrogate: the sweep queues the cells the screen keeps for k_sweep_queue
  s.smem[2] = 0;
  s.minb[2] = ST::MINB;
  s.stage[2][0] = (const void*)k_sweep<ST, 1, true>;
  s.stage[2][1] = (const void*)k_sweep<ST, 2, true>;
  s.queue[0] = (const void*)k_sweep_queue<1>;
  s.queue[1] = (const void*)k_sweep_queue<2>;
  s.queue_smem = QUEUE_SMEM;
  // batches: the persistent sweep over every case's strips, and the queues of every case
  s.batch[1][0] = (const void*)k_batch_sweep<ST, 1, false>;
  s.batch[1][1] = (const void*)k_batch_sweep<ST, 2, false>;
  s.batch[2][0] = (const void*)k_batch_sweep<ST, 1, true>;
  s.batch[2][1] = (const void*)k_batch_sweep<ST, 2, true>;
  s.batch_queue[0] = (const void*)k_batch_queue<1>;
  s.batch_queue[1] = (const void*)k_batch_queue<2>;
  s.plume_inviscid_only = true;
  return s;
}

}  // namespace ct
