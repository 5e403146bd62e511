// fastmath.cuh -- reciprocal for the FP64 transport arithmetic.
//
// rcp_nr(s): Newton-Raphson iteration for 1/s, x_{k+1} = x_k + x_k (1 - s x_k), whose
// relative error e_{k+1} = -e_k^2 squares at each step, started from the hardware's
// approximate reciprocal (PTX rcp.approx.ftz.f64, relative error below 2^-20).  Two steps
// bring the error below the FP64 rounding of the last fused multiply-adds (a few ulp) at
// four FP64 operations, against about nine for an IEEE-rounded division.  Valid for normal
// s (subnormal s flush to zero and give an infinite seed); the transport code calls it only
// with normal, finite arguments.
#pragma once
#include <cuda_runtime.h>

namespace ct {

__device__ __forceinline__ double rcp_nr(double s) {
  double x;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(s));
  double e = fma(-s, x, 1.0);
  x = fma(x, e, x);
  e = fma(-s, x, 1.0);
  return fma(x, e, x);
}

}  // namespace ct
