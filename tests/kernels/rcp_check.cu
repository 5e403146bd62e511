// Test kernel: the transport path's Newton reciprocal (paper_2504_20742_gb300/csrc/fastmath.cuh)
// and CUDA's IEEE division on the same inputs.
#include <cuda_runtime.h>

#include "../../paper_2504_20742_gb300/csrc/fastmath.cuh"

__global__ void k_rcp(const double* __restrict__ x, double* __restrict__ r_nr, double* __restrict__ r_div, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    r_nr[i] = ct::rcp_nr(x[i]);
    r_div[i] = 1.0 / x[i];
  }
}

extern "C" int rcp_check(const double* x, double* r_nr, double* r_div, int n) {
  k_rcp<<<(n + 255) / 256, 256>>>(x, r_nr, r_div, n);
  return (int)cudaDeviceSynchronize();
}
