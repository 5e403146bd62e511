// mlp_tc.cuh -- BF16 tensor-core inference of the source surrogate (16 -> 4x128 SiLU -> 10)
// on tiles of 128 rows: the five layers run as tcgen05.mma chains (M = 128, K = 16 or 128,
// N = 128 or 16) with FP32 accumulation in TMEM; between layers, one warpgroup reads the
// accumulator back (tcgen05.ld), adds the bias, applies SiLU, rounds to BF16 and writes the
// next layer's operand into shared memory.
#pragma once
#include <cuda_bf16.h>

#include "tc.cuh"

namespace ct {
namespace mlp {

// Device blob: a float header, then the BF16 weights in K-major core-matrix order.
constexpr int F_XMEAN = 0, F_XISD = 16, F_YMEAN = 32, F_YSD = 48, F_HMIN = 64, F_HMAX = 80, F_YMIN = 96,
              F_YMAX = 112, F_BIAS = 128;
constexpr int NFLOAT = F_BIAS + 4 * 128 + 16;   // 656
constexpr int WOFF = 2688;                      // byte offset of the weights (128-byte aligned)
__host__ __device__ constexpr int kdim(int l) { return l == 0 ? 16 : 128; }
__host__ __device__ constexpr int ndim(int l) { return l == 4 ? 16 : 128; }      // padded output width
__host__ __device__ constexpr int wbytes(int l) { return ndim(l) * kdim(l) * 2; }
__host__ __device__ constexpr int woff(int l) {
  int o = 0;
  for (int q = 0; q < l; ++q) o += wbytes(q);
  return o;
}
constexpr int WBYTES = woff(5);                 // 106,496
constexpr int BLOB_BYTES = WOFF + WBYTES;       // 109,184
constexpr int ABYTES = 128 * 128 * 2;           // activation operand, 32 KB

// z sigmoid(z) = (z/2)(1 + tanh(z/2)) with the hardware tanh approximation (one
// special-function operation; its relative error, below 2^-10, is under the BF16 rounding
// that follows)
__device__ __forceinline__ float silu(float z) {
  const float h = 0.5f * z;
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(h));
  return fmaf(h, t, h);
}

// Write 16 values of row `row` (columns c16*16 .. +15) as BF16 into a K-major operand with K
// columns (two 16-byte core-matrix rows).
__device__ __forceinline__ void store_row16(unsigned char* buf, int row, int c16, int K, const float* v) {
  uint4 a, b;
  __nv_bfloat162 t;
  t = __floats2bfloat162_rn(v[0], v[1]);   a.x = *reinterpret_cast<uint32_t*>(&t);
  t = __floats2bfloat162_rn(v[2], v[3]);   a.y = *reinterpret_cast<uint32_t*>(&t);
  t = __floats2bfloat162_rn(v[4], v[5]);   a.z = *reinterpret_cast<uint32_t*>(&t);
  t = __floats2bfloat162_rn(v[6], v[7]);   a.w = *reinterpret_cast<uint32_t*>(&t);
  t = __floats2bfloat162_rn(v[8], v[9]);   b.x = *reinterpret_cast<uint32_t*>(&t);
  t = __floats2bfloat162_rn(v[10], v[11]); b.y = *reinterpret_cast<uint32_t*>(&t);
  t = __floats2bfloat162_rn(v[12], v[13]); b.z = *reinterpret_cast<uint32_t*>(&t);
  t = __floats2bfloat162_rn(v[14], v[15]); b.w = *reinterpret_cast<uint32_t*>(&t);
  *reinterpret_cast<uint4*>(buf + tc::cm_offset(row, c16 * 16, K)) = a;
  *reinterpret_cast<uint4*>(buf + tc::cm_offset(row, c16 * 16 + 8, K)) = b;
}

// Run the network on one 128-row tile whose standardised inputs are already in `A`
// (K = 16 layout).  All threads of the CTA call this; threads 0..127 (warps 0-3) own rows
// 0..127 and return the 10 standardised outputs of their row in `out`.  `W`: weights in
// shared memory; `bias`: the 4x128 + 16 biases; `tmem`: 128 allocated TMEM columns;
// `mbar`/`phase`: the MMA-completion barrier.  Returns false if a wait timed out.
// STREAM: W is a 32 KB shared buffer; each layer's weights arrive there from the global
// blob weights Wg by one bulk copy (completion on `wbar`/`wphase`), issued as soon as the
// previous layer's MMAs have finished, so that the copy overlaps that layer's epilogue
// (keeps the fused step at 2 CTAs/SM).
// nrows: rows of the tile that carry data; 32-row groups beyond it skip the epilogue.  With
// 8 or more warps, warps w and w+4 share the lane quarter of TMEM and split the columns.
template <bool STREAM = false>
__device__ __forceinline__ bool run_tile(unsigned char* A, unsigned char* W, const float* bias, uint32_t tmem,
                                         uint32_t mbar, uint32_t& phase, float* out,
                                         const unsigned char* __restrict__ Wg = nullptr, int nrows = 128,
                                         uint32_t wbar = 0, uint32_t* wphase = nullptr) {
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;
  const int quarter = warp & 3;                  // TMEM lanes 32*quarter .. +31
  const int half = nwarps >= 8 ? (warp >> 2) : 0;   // column half handled by this warp
  const bool epi = warp < (nwarps >= 8 ? 8 : 4) && 32 * quarter < nrows;
  const int row = 32 * quarter + (tid & 31);
  bool ok = true;
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (STREAM && tid == 0) {   // layer 0's weights
    tc::mbar_arrive_expect_tx(wbar, (uint32_t)wbytes(0));
    tc::bulk_g2s(tc::smem_addr(W), Wg + woff(0), (uint32_t)wbytes(0), wbar);
  }
  for (int l = 0; l < 5; ++l) {
    const int K = kdim(l), N = ndim(l);
    if (tid == 0) {
      if (STREAM) {
        if (!tc::mbar_wait(wbar, *wphase)) ok = false;
        *wphase ^= 1u;
      }
      const uint32_t a0 = tc::smem_addr(A), b0 = tc::smem_addr(STREAM ? W : W + woff(l));
      const uint32_t sbo = (uint32_t)(K / 8) * 128u;
      const uint32_t idesc = tc::idesc_bf16_f32(128, N);
      for (int s = 0; s < K / 16; ++s)
        tc::mma_bf16(tmem, tc::smem_desc(a0 + 256u * s, 128u, sbo), tc::smem_desc(b0 + 256u * s, 128u, sbo), idesc,
                     s > 0 ? 1u : 0u);
      tc::mma_commit(mbar);
    }
    if (!tc::mbar_wait(mbar, phase)) ok = false;
    phase ^= 1u;
    tc::fence_after_sync();
    if (STREAM && tid == 0 && l < 4) {   // W is free again: fetch the next layer's weights
      tc::mbar_arrive_expect_tx(wbar, (uint32_t)wbytes(l + 1));
      tc::bulk_g2s(tc::smem_addr(W), Wg + woff(l + 1), (uint32_t)wbytes(l + 1), wbar);
    }
    if (epi) {
      const uint32_t lane_addr = tmem + ((uint32_t)(32 * quarter) << 16);
      if (l < 4) {
        const int c_lo = nwarps >= 8 ? 4 * half : 0, c_hi = nwarps >= 8 ? c_lo + 4 : 8;
        for (int c = c_lo; c < c_hi; ++c) {
          float v[16];
          tc::tmem_ld16(lane_addr + 16u * c, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = silu(v[i] + bias[l * 128 + 16 * c + i]);
          store_row16(A, row, c, 128, v);
        }
      } else if (half == 0) {
        float v[16];
        tc::tmem_ld16(lane_addr, v);
#pragma unroll
        for (int i = 0; i < 10; ++i) out[i] = v[i] + bias[4 * 128 + i];
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  }
  return ok;
}

}  // namespace mlp
}  // namespace ct
