// mlp_infer.cu -- packing of a trained surrogate into its device blob, and a standalone
// persistent tensor-core inference kernel over a batch of raw inputs (the same tile routine
// as the fused FP32_MLP step).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/contrail.h"
#include "mlp_tc.cuh"

extern "C" ct_status ct__set_error(ct_status s, const char* msg);

namespace ct {
namespace mlp {

// params: flat FP32 (per layer W out x in, then b); stats: 16-float arrays.
__global__ void k_pack(const float* __restrict__ params, const float* __restrict__ x_mean,
                       const float* __restrict__ x_sd, const float* __restrict__ x_min, const float* __restrict__ x_max,
                       const float* __restrict__ y_mean, const float* __restrict__ y_sd, const float* __restrict__ y_min,
                       const float* __restrict__ y_max, unsigned char* __restrict__ blob) {
  float* hdr = reinterpret_cast<float*>(blob);
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  for (int i = tid; i < 16; i += nt) {
    hdr[F_XMEAN + i] = x_mean[i];
    hdr[F_XISD + i] = x_sd[i] > 0.0f ? 1.0f / x_sd[i] : 1.0f;
    hdr[F_YMEAN + i] = i < CT_MLP_OUT ? y_mean[i] : 0.0f;
    hdr[F_YSD + i] = i < CT_MLP_OUT ? y_sd[i] : 0.0f;
    hdr[F_HMIN + i] = x_min[i];
    hdr[F_HMAX + i] = x_max[i];
    hdr[F_YMIN + i] = i < CT_MLP_OUT ? y_min[i] : 0.0f;
    hdr[F_YMAX + i] = i < CT_MLP_OUT ? y_max[i] : 0.0f;
  }
  // flat parameter offsets
  int po = 0;
  for (int l = 0; l < 5; ++l) {
    const int K = kdim(l), Nout = l == 4 ? CT_MLP_OUT : 128, Np = ndim(l);
    const float* Wl = params + po;
    const float* bl = Wl + Nout * K;
    __nv_bfloat16* wb = reinterpret_cast<__nv_bfloat16*>(blob + WOFF + woff(l));
    for (int e = tid; e < Np * K; e += nt) {
      const int n = e / K, k = e % K;
      const float v = n < Nout ? Wl[n * K + k] : 0.0f;
      wb[tc::cm_offset(n, k, K) / 2] = __float2bfloat16_rn(v);
    }
    for (int n = tid; n < Np; n += nt) hdr[F_BIAS + 128 * l + n] = n < Nout ? bl[n] : 0.0f;
    po += Nout * K + Nout;
  }
}

constexpr size_t INFER_SMEM = (size_t)WBYTES + ABYTES + NFLOAT * sizeof(float) + 64;

__global__ void __launch_bounds__(128, 1) k_infer(const unsigned char* __restrict__ blob, const float* __restrict__ X,
                                                 int n, float* __restrict__ Y, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* W = sm;
  unsigned char* A = sm + WBYTES;
  float* hdr = reinterpret_cast<float*>(sm + WBYTES + ABYTES);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + WBYTES + ABYTES + NFLOAT * sizeof(float) + 16);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + WBYTES + ABYTES + NFLOAT * sizeof(float));
  const int tid = threadIdx.x;
  // weights and header into shared memory
  const uint4* src = reinterpret_cast<const uint4*>(blob + WOFF);
  uint4* dst = reinterpret_cast<uint4*>(W);
  for (int i = tid; i < WBYTES / 16; i += blockDim.x) dst[i] = src[i];
  for (int i = tid; i < NFLOAT; i += blockDim.x) hdr[i] = reinterpret_cast<const float*>(blob)[i];
  if (tid < 32) {
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
  const int ntiles = (n + 127) / 128;
  for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
    const int row = t * 128 + tid;
    float v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = row < n ? (X[(size_t)row * 16 + i] - hdr[F_XMEAN + i]) * hdr[F_XISD + i] : 0.0f;
    store_row16(A, tid, 0, 16, v);
    float o[10];
    const bool tile_ok = run_tile<false>(A, W, hdr + F_BIAS, tmem, tc::smem_addr(mbar), phase, o);
    ok = __syncthreads_and(tile_ok ? 1 : 0) != 0;   // CTA-uniform, so the loop stays convergent
    if (row < n) {
#pragma unroll
      for (int i = 0; i < 10; ++i) Y[(size_t)row * 10 + i] = o[i] * hdr[F_YSD + i] + hdr[F_YMEAN + i];
    }
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid < 32) tc::tmem_dealloc(tmem, 128);
}

}  // namespace mlp
}  // namespace ct

using namespace ct::mlp;

extern "C" {

size_t ct_mlp_blob_bytes(void) { return (size_t)BLOB_BYTES; }

ct_status ct_mlp_pack(const float* params, const float* x_mean, const float* x_sd, const float* x_min,
                      const float* x_max, const float* y_mean, const float* y_sd, const float* y_min,
                      const float* y_max, void* blob, void* stream) {
  if (!params || !x_mean || !x_sd || !x_min || !x_max || !y_mean || !y_sd || !y_min || !y_max || !blob)
    return ct__set_error(CT_ERR_ARG, "ct_mlp_pack: null pointer");
  if (((uintptr_t)blob & 15) != 0) return ct__set_error(CT_ERR_ARG, "ct_mlp_pack: blob must be 16-byte aligned");
  k_pack<<<64, 256, 0, (cudaStream_t)stream>>>(params, x_mean, x_sd, x_min, x_max, y_mean, y_sd, y_min, y_max,
                                                (unsigned char*)blob);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CT_OK : ct__set_error(CT_ERR_CUDA, cudaGetErrorString(e));
}

ct_status ct_mlp_infer(const void* blob, const float* X, int n, float* Y, int* err_flag, void* stream) {
  if (!blob || !X || !Y || !err_flag || n < 0) return ct__set_error(CT_ERR_ARG, "ct_mlp_infer: bad argument");
  if (((uintptr_t)blob & 15) != 0) return ct__set_error(CT_ERR_ARG, "ct_mlp_infer: blob must be 16-byte aligned");
  if (n == 0) return CT_OK;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)INFER_SMEM);
    if (e != cudaSuccess) return ct__set_error(CT_ERR_CUDA, cudaGetErrorString(e));
    attr = true;
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int ntiles = (n + 127) / 128;
  const int grid = ntiles < nsm ? ntiles : nsm;
  k_infer<<<grid, 128, INFER_SMEM, (cudaStream_t)stream>>>((const unsigned char*)blob, X, n, Y, err_flag);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CT_OK : ct__set_error(CT_ERR_CUDA, cudaGetErrorString(e));
}

}  // extern "C"
