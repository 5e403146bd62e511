// pair.cuh -- two state fields at a time.  The stencil phases of the stage kernel treat the
// fields in pairs (fields 2k and 2k+1 side by side in shared memory): in FP32 every add,
// multiply and fused multiply-add of a pair is one paired instruction of sm_100-class GPUs
// (FADD2 / FMUL2 / FFMA2, round to nearest like their scalar forms) and every shared-memory
// access one 64-bit access; in FP64 a pair is two scalar operations.
#pragma once
#include <cuda_runtime.h>

#include "fastmath.cuh"

namespace ct {

template <class T>
struct PairOf;
template <>
struct PairOf<float> {
  using V = float2;
};
template <>
struct PairOf<double> {
  using V = double2;
};

__device__ __forceinline__ float2 p_make(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ double2 p_make(double x, double y) { return make_double2(x, y); }

__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b as one rounding of b * (-1) + a, i.e. exactly the scalar difference
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }

__device__ __forceinline__ double2 p_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 p_mul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 p_fma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 p_sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

}  // namespace ct
