// mlp.cu -- training kernels of the phase-change source surrogate (16 -> 4x128 SiLU -> 10).
//
// The surrogate stands in for the stiff pointwise rates of Sec. 2.2 (nucleation, growth,
// relaxation) in the FP32 path.  It is trained on the GPU with these kernels: a tiled FP32
// GEMM with transpose variants for the forward pass and both backward products, fused
// bias and SiLU epilogues, a masked mean-squared-error kernel and Adam.  Parameters are one
// flat FP32 vector, per layer W (out x in, row-major) then b (out).  Deterministic: no
// atomics; reductions run in a fixed order.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <vector>

#include "../../include/contrail.h"
#include "mlp_tc.cuh"

namespace ctm {

constexpr int NL = 5;
__host__ __device__ constexpr int dim(int l) { return l == 0 ? CT_MLP_IN : (l == NL ? CT_MLP_OUT : CT_MLP_HIDDEN); }
__host__ __device__ constexpr int w_off(int l) {
  int o = 0;
  for (int q = 0; q < l; ++q) o += dim(q + 1) * dim(q) + dim(q + 1);
  return o;
}
constexpr int NPARAM = w_off(NL);

// ---- tiled SGEMM: C[M,N] = op(A)[M,K] op(B)[K,N] (+ bias[N]) -----------------------------
// op(A)[m][k] = TA ? A[k*lda + m] : A[m*lda + k];  op(B)[k][n] = TB ? B[n*ldb + k] : B[k*ldb + n].
// EPI 0: C = AB (+bias); 1: Z = AB + bias stored to C and SiLU(Z) stored to H.
constexpr int BM = 64, BN = 64, BK = 16, GT = 256;

__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(GT) k_sgemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                              const float* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                                              const float* __restrict__ bias, float* __restrict__ H) {
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;   // rows on x: up to 2^31 blocks
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += GT) {
      int mm, kk;
      if (TA) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
      const int m = m0 + mm, k = k0 + kk;
      float v = 0.0f;
      if (m < M && k < K) v = TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < BN * BK; e += GT) {
      int nn, kk;
      if (TB) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
      const int n = n0 + nn, k = k0 + kk;
      float v = 0.0f;
      if (n < N && k < K) v = TB ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= N) continue;
      float v = acc[i][j] + (bias ? bias[n] : 0.0f);
      C[(size_t)m * ldc + n] = v;
      if (EPI == 1) H[(size_t)m * ldc + n] = silu(v);
    }
  }
}

// ---- BF16 tensor-core GEMM (tcgen05, FP32 accumulation in TMEM) for training -----------------
// C[M,N] = op(A)[M,K] op(B)[K,N] on tiles of 128 x NT (NT = 128 or 16) per CTA: 128 threads
// stage K-chunks of both operands from FP32 global memory as BF16 into shared memory (the
// K-major core-matrix layout of the tensor cores, whatever the global layout), thread 0
// issues the MMAs and commits to an mbarrier, and each thread reads its row of the
// accumulator back from TMEM for the epilogue.  The FP32 masters stay untouched: operands
// are rounded to BF16 as they are staged.  Split-K over gridDim.z: CTA z covers K-rows
// [z*kper, (z+1)*kper) and, with EPI 2, stores its partial tile to P[z] (summed later in a
// fixed order, so results are deterministic).  EPI 0: C = AB (+bias); 1: Z = AB + bias to C,
// SiLU(Z) to H; 2: split-K partial.  A bounded wait that gives up sets *err.
constexpr int TCK = 64;                      // K-chunk staged per round
// dynamic shared memory per CTA: the two operand buffers (32 KB), padded to 56 KB so that
// at most four CTAs share an SM and their 4 x 128 TMEM columns always fit
constexpr int TC_SMEM = 56 * 1024;
constexpr int TC_SPLIT_MAX = 64;             // split-K partial tiles of the weight gradients

template <bool TA, bool TB, int EPI, int NT>
__global__ void __launch_bounds__(128) k_tc_gemm(int M, int N, int K, int kper, const float* __restrict__ A, int lda,
                                                 const float* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                                                 const float* __restrict__ bias, float* __restrict__ H,
                                                 float* __restrict__ P, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char* As = tsm;                       // 128 x TCK bf16
  unsigned char* Bs = tsm + 128 * TCK * 2;       // NT x TCK bf16
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x;
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * NT;
  const int kb = blockIdx.z * kper, ke = min(K, kb + kper);
  if (tid < 32) {
    ct::tc::tmem_alloc(ct::tc::smem_addr(&tmem_slot), 128);
    ct::tc::tmem_relinquish();
  }
  if (tid == 0) {
    ct::tc::mbar_init(ct::tc::smem_addr(&mbar), 1);
    ct::tc::fence_mbar_init();
  }
  ct::tc::fence_before_sync();
  __syncthreads();
  ct::tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;
  const uint32_t mb = ct::tc::smem_addr(&mbar);
  uint32_t phase = 0;
  bool ok = true;
  const uint32_t idesc = ct::tc::idesc_bf16_f32(128, NT);
  int nchunk = 0;
  for (int k0 = kb; k0 < ke; k0 += TCK, ++nchunk) {
    // stage: coalesced along the contiguous global index of each operand
    for (int e = tid; e < 128 * TCK; e += 128) {
      int mm, kk;
      if (TA) { mm = e % 128; kk = e / 128; } else { kk = e % TCK; mm = e / TCK; }
      const int m = m0 + mm, k = k0 + kk;
      float v = 0.0f;
      if (m < M && k < ke) v = TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
      *reinterpret_cast<__nv_bfloat16*>(As + ct::tc::cm_offset(mm, kk, TCK)) = __float2bfloat16_rn(v);
    }
    for (int e = tid; e < NT * TCK; e += 128) {
      int nn, kk;
      if (TB) { kk = e % TCK; nn = e / TCK; } else { nn = e % NT; kk = e / NT; }
      const int n = n0 + nn, k = k0 + kk;
      float v = 0.0f;
      if (n < N && k < ke) v = TB ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n];
      *reinterpret_cast<__nv_bfloat16*>(Bs + ct::tc::cm_offset(nn, kk, TCK)) = __float2bfloat16_rn(v);
    }
    ct::tc::fence_async_smem();
    ct::tc::fence_before_sync();
    __syncthreads();
    ct::tc::fence_after_sync();
    if (tid == 0) {
      const uint32_t a0 = ct::tc::smem_addr(As), b0 = ct::tc::smem_addr(Bs);
      const uint32_t sbo = (uint32_t)(TCK / 8) * 128u;
      for (int s = 0; s < TCK / 16; ++s)
        ct::tc::mma_bf16(tmem, ct::tc::smem_desc(a0 + 256u * s, 128u, sbo), ct::tc::smem_desc(b0 + 256u * s, 128u, sbo),
                         idesc, (nchunk > 0 || s > 0) ? 1u : 0u);
      ct::tc::mma_commit(mb);
    }
    // the chunk's MMAs must finish before the buffers are restaged; a wait that gives up
    // stops the CTA (a collective decision, so that every thread leaves the loop)
    const bool gave_up = !ct::tc::mbar_wait(mb, phase);
    phase ^= 1u;
    ct::tc::fence_after_sync();
    if (__syncthreads_or(gave_up)) {
      ok = false;
      break;
    }
  }
  // epilogue: thread t owns row m0 + t (TMEM lane t); warp w reads lanes 32w .. 32w+31
  const int row = m0 + tid;
  const uint32_t lane_addr = tmem + ((uint32_t)(32 * (tid >> 5)) << 16);
  if (ok && nchunk > 0) {
    for (int c = 0; c < NT / 16; ++c) {
      float v[16];
      ct::tc::tmem_ld16(lane_addr + 16u * c, v);
      if (row < M) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int n = n0 + 16 * c + i;
          if (n >= N) continue;
          if (EPI == 2) {
            P[((size_t)blockIdx.z * M + row) * N + n] = v[i];
          } else {
            const float z = v[i] + (bias ? bias[n] : 0.0f);
            C[(size_t)row * ldc + n] = z;
            if (EPI == 1) H[(size_t)row * ldc + n] = z / (1.0f + __expf(-z));
          }
        }
      }
    }
  } else if (EPI == 2 && row < M) {   // an empty K range contributes zeros
    for (int n = n0; n < min(N, n0 + NT); ++n) P[((size_t)blockIdx.z * M + row) * N + n] = 0.0f;
  }
  if (!ok && tid == 0) {
    atomicExch(err, 1);
    ct::tc::mbar_wait(mb, phase ^ 1u);   // give the abandoned MMAs a bounded time to land
  }
  ct::tc::fence_before_sync();
  __syncthreads();
  if (tid < 32) ct::tc::tmem_dealloc(tmem, 128);
}

// C[m][n] = sum_z P[z][m][n], z in order (the split-K partials of k_tc_gemm)
__global__ void k_splitk_sum(const float* __restrict__ P, int S, int MN, float* __restrict__ C) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MN; i += gridDim.x * blockDim.x) {
    float a = 0.0f;
    for (int z = 0; z < S; ++z) a += P[(size_t)z * MN + i];
    C[i] = a;
  }
}

// column sums of an n x d matrix (bias gradients), fixed-order tree per column
__global__ void k_colsum(const float* __restrict__ G, int n, int d, float* __restrict__ out) {
  __shared__ float s[256];
  const int j = blockIdx.x;
  float a = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += G[(size_t)i * d + j];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = s[0];
}

// dZ = dH * SiLU'(Z), in place on dH
__global__ void k_silu_bwd(float* __restrict__ dH, const float* __restrict__ Z, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float z = Z[i];
    const float s = 1.0f / (1.0f + __expf(-z));
    dH[i] *= s * (1.0f + z * (1.0f - s));
  }
}

// per-output weights of the squared errors (all 1: the plain masked MSE)
struct OutW {
  float w[CT_MLP_OUT];
};

// masked, weighted MSE: dY = 2 w_q m (yhat - y) / count, per-block partial sums of
// w_q m (yhat - y)^2 and m (the mask m is 0 or 1; count = sum m)
__global__ void k_mse(const float* __restrict__ Yh, const float* __restrict__ Y, const float* __restrict__ Mk, size_t n,
                      OutW ow, float* __restrict__ dY, double* __restrict__ part) {
  __shared__ double s0[256], s1[256];
  double a = 0.0, c = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float wq = ow.w[i % CT_MLP_OUT];
    const float r = (Yh[i] - Y[i]) * Mk[i];
    dY[i] = wq * r;
    a += (double)wq * ((double)r * r);
    c += Mk[i];
  }
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = c;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s0[threadIdx.x] += s0[threadIdx.x + o];
      s1[threadIdx.x] += s1[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s0[0];
    part[2 * blockIdx.x + 1] = s1[0];
  }
}

// loss = sum/count; scale dY by 2/count
__global__ void k_mse_finish(const double* __restrict__ part, int nb, float* __restrict__ dY, size_t n,
                             float* __restrict__ loss) {
  __shared__ double inv;
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int b = 0; b < nb; ++b) { a += part[2 * b]; c += part[2 * b + 1]; }
    c = c < 1.0 ? 1.0 : c;
    inv = 2.0 / c;
    if (blockIdx.x == 0 && loss) *loss = (float)(a / c);
  }
  __syncthreads();
  const float s = (float)inv;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) dY[i] *= s;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// per-column statistics of an n x d matrix (optionally masked): mean, std, min, max
__global__ void k_colstats(const float* __restrict__ X, const float* __restrict__ Mk, int n, int d, float* __restrict__ out) {
  const int j = blockIdx.x;
  __shared__ double s[3][256];
  __shared__ float mn[256], mx[256];
  double a = 0.0, b = 0.0, c = 0.0;
  float lo = INFINITY, hi = -INFINITY;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float w = Mk ? Mk[(size_t)i * d + j] : 1.0f;
    if (w == 0.0f) continue;
    const float x = X[(size_t)i * d + j];
    a += x;
    b += (double)x * x;
    c += 1.0;
    lo = fminf(lo, x);
    hi = fmaxf(hi, x);
  }
  s[0][threadIdx.x] = a;
  s[1][threadIdx.x] = b;
  s[2][threadIdx.x] = c;
  mn[threadIdx.x] = lo;
  mx[threadIdx.x] = hi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      for (int q = 0; q < 3; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + o];
      mn[threadIdx.x] = fminf(mn[threadIdx.x], mn[threadIdx.x + o]);
      mx[threadIdx.x] = fmaxf(mx[threadIdx.x], mx[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double cnt = s[2][0] > 0.0 ? s[2][0] : 1.0;
    const double mean = s[0][0] / cnt;
    const double var = s[1][0] / cnt - mean * mean;
    out[j] = (float)mean;
    out[d + j] = (float)sqrt(var > 0.0 ? var : 0.0);
    out[2 * d + j] = mn[0];
    out[3 * d + j] = mx[0];
  }
}

// (x - mean)/std, in place
__global__ void k_standardize(float* __restrict__ X, int n, int d, const float* __restrict__ mean,
                              const float* __restrict__ sd) {
  const size_t tot = (size_t)n * d;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(i % d);
    const float s = sd[j] > 0.0f ? sd[j] : 1.0f;
    X[i] = (X[i] - mean[j]) / s;
  }
}

// batch rows by index: xb = Xn[idx], yb = Yn[idx], mb = M[idx]
__global__ void k_gather_rows(const int* __restrict__ idx, int nb, const float* __restrict__ Xn,
                              const float* __restrict__ Yn, const float* __restrict__ Mk, float* __restrict__ xb,
                              float* __restrict__ yb, float* __restrict__ mb) {
  const size_t tot = (size_t)nb * (CT_MLP_IN + 2 * CT_MLP_OUT);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / (CT_MLP_IN + 2 * CT_MLP_OUT));
    const int c = (int)(e % (CT_MLP_IN + 2 * CT_MLP_OUT));
    const size_t src = (size_t)idx[r];
    if (c < CT_MLP_IN) xb[(size_t)r * CT_MLP_IN + c] = Xn[src * CT_MLP_IN + c];
    else if (c < CT_MLP_IN + CT_MLP_OUT) yb[(size_t)r * CT_MLP_OUT + c - CT_MLP_IN] = Yn[src * CT_MLP_OUT + c - CT_MLP_IN];
    else mb[(size_t)r * CT_MLP_OUT + c - CT_MLP_IN - CT_MLP_OUT] = Mk[src * CT_MLP_OUT + c - CT_MLP_IN - CT_MLP_OUT];
  }
}

// Yn *= M (masked entries carry no information); sd of a column below 1e-6 -> 1
__global__ void k_mask_mul(float* __restrict__ Y, const float* __restrict__ Mk, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) Y[i] *= Mk[i];
}
__global__ void k_fix_sd(float* __restrict__ stats, int d) {
  const int j = threadIdx.x;
  if (j < d && !(stats[d + j] > 1e-6f)) stats[d + j] = 1.0f;
}

// loss bookkeeping of the epoch loop: acc[e] += loss (one thread, fixed order)
__global__ void k_acc_loss(const float* __restrict__ loss, double* __restrict__ acc, int e) {
  if (threadIdx.x == 0 && blockIdx.x == 0) acc[e] += (double)loss[0];
}

// ---- host helpers ---------------------------------------------------------------------------
}  // namespace ctm
extern "C" ct_status ct__set_error(ct_status s, const char* msg);   // contrail.cu (thread-local message)
namespace ctm {

static ct_status fail(ct_status s, const char* m) { return ct__set_error(s, m); }
static ct_status check(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
    return ct__set_error(CT_ERR_CUDA, buf);
  }
  return CT_OK;
}

template <bool TA, bool TB, int EPI>
static void gemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                 const float* bias, float* H, cudaStream_t st) {
  dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN);
  k_sgemm<TA, TB, EPI><<<grid, GT, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, H);
}

// work layout (floats): Z_l (n x out_l) for l = 0..4, H_l (n x out_l) for l = 0..3, two
// n x 128 gradient buffers, the split-K partial tiles of the tensor-core weight gradients
// (TC_SPLIT_MAX x 128 x 128), then 2*256 doubles of loss partials and the tensor-core wait
// flag.
static size_t work_floats(int n) {
  size_t f = 0;
  for (int l = 0; l < NL; ++l) f += (size_t)n * dim(l + 1);
  for (int l = 0; l < NL - 1; ++l) f += (size_t)n * dim(l + 1);
  f += 2 * (size_t)n * CT_MLP_HIDDEN;
  f += (size_t)TC_SPLIT_MAX * 128 * 128;
  return f;
}
static size_t work_bytes(int n) { return work_floats(n) * sizeof(float) + 2 * 256 * sizeof(double) + 512; }

struct Work {
  float* Z[NL];
  float* H[NL - 1];
  float* g0;
  float* g1;
  float* ptc;
  double* part;
  int* err;
};
static Work carve(float* w, int n) {
  Work k;
  float* p = w;
  for (int l = 0; l < NL; ++l) { k.Z[l] = p; p += (size_t)n * dim(l + 1); }
  for (int l = 0; l < NL - 1; ++l) { k.H[l] = p; p += (size_t)n * dim(l + 1); }
  k.g0 = p; p += (size_t)n * CT_MLP_HIDDEN;
  k.g1 = p; p += (size_t)n * CT_MLP_HIDDEN;
  k.ptc = p; p += (size_t)TC_SPLIT_MAX * 128 * 128;
  uintptr_t a = ((uintptr_t)p + 255) & ~(uintptr_t)255;
  k.part = (double*)a;
  k.err = (int*)(k.part + 2 * 256);
  return k;
}

// BF16 tensor-core GEMM launch (k_tc_gemm); N <= 16 takes the 16-wide tile
template <bool TA, bool TB, int EPI, int NT>
static void tc_launch(dim3 grid, int M, int N, int K, int kper, const float* A, int lda, const float* B, int ldb,
                      float* C, int ldc, const float* bias, float* H, float* P, int* err, cudaStream_t st) {
  static bool attr = false;   // idempotent: racing first calls set the same value
  if (!attr) {
    cudaFuncSetAttribute(k_tc_gemm<TA, TB, EPI, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    attr = true;
  }
  k_tc_gemm<TA, TB, EPI, NT><<<grid, 128, TC_SMEM, st>>>(M, N, K, kper, A, lda, B, ldb, C, ldc, bias, H, P, err);
}
template <bool TA, bool TB, int EPI>
static void tc_gemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                    const float* bias, float* H, float* P, int splits, int* err, cudaStream_t st) {
  const int kper = ((K + splits - 1) / splits + TCK - 1) / TCK * TCK;
  const int nt = N > 16 ? 128 : 16;
  dim3 grid((M + 127) / 128, (N + nt - 1) / nt, splits);
  if (nt == 128) tc_launch<TA, TB, EPI, 128>(grid, M, N, K, kper, A, lda, B, ldb, C, ldc, bias, H, P, err, st);
  else tc_launch<TA, TB, EPI, 16>(grid, M, N, K, kper, A, lda, B, ldb, C, ldc, bias, H, P, err, st);
}

static void forward(const float* P, const float* X, int n, const Work& w, cudaStream_t st) {
  const float* h = X;
  for (int l = 0; l < NL; ++l) {
    const int in = dim(l), out = dim(l + 1);
    const float* W = P + w_off(l);
    const float* b = W + out * in;
    if (l < NL - 1) gemm<false, true, 1>(n, out, in, h, in, W, in, w.Z[l], out, b, w.H[l], st);
    else gemm<false, true, 0>(n, out, in, h, in, W, in, w.Z[l], out, b, nullptr, st);
    h = l < NL - 1 ? w.H[l] : nullptr;
  }
}

static OutW ones_w() {
  OutW o;
  for (int q = 0; q < CT_MLP_OUT; ++q) o.w[q] = 1.0f;
  return o;
}

// Masked MSE and its gradient (forward, loss, backward through the five layers).
static void loss_grad(const float* params, const float* X, const float* Y, const float* M, int n, float* grad,
                      float* loss, const Work& w, const OutW& ow, cudaStream_t st) {
  forward(params, X, n, w, st);
  // dL/dyhat into g0 (n x 10)
  const size_t ny = (size_t)n * CT_MLP_OUT;
  const int nb = (int)((ny + 255) / 256 < 256 ? (ny + 255) / 256 : 256);
  k_mse<<<nb, 256, 0, st>>>(w.Z[NL - 1], Y, M, ny, ow, w.g0, w.part);
  k_mse_finish<<<nb, 256, 0, st>>>(w.part, nb, w.g0, ny, loss);
  float* g = w.g0;     // gradient wrt the current layer's output (pre-activation for the last)
  float* gn = w.g1;
  for (int l = NL - 1; l >= 0; --l) {
    const int in = dim(l), out = dim(l + 1);
    const float* W = params + w_off(l);
    float* gW = grad + w_off(l);
    float* gb = gW + out * in;
    if (l < NL - 1) {
      const size_t tot = (size_t)n * out;
      k_silu_bwd<<<(int)((tot + 255) / 256 < 4096 ? (tot + 255) / 256 : 4096), 256, 0, st>>>(g, w.Z[l], tot);
    }
    const float* hin = l == 0 ? X : w.H[l - 1];
    // dW = dZ^T h  (out x in),  db = dZ^T 1
    gemm<true, false, 0>(out, in, n, g, out, hin, in, gW, in, nullptr, nullptr, st);
    k_colsum<<<out, 256, 0, st>>>(g, n, out, gb);
    if (l > 0) gemm<false, false, 0>(n, in, out, g, out, W, in, gn, in, nullptr, nullptr, st);
    float* t = g;
    g = gn;
    gn = t;
  }
}


// The same forward pass and gradient on the tensor cores: every GEMM (forward, input
// gradient, weight gradient) runs in BF16 with FP32 accumulation; biases, SiLU, the loss,
// the bias gradients and the FP32 master weights stay in FP32.
static void forward_tc(const float* P, const float* X, int n, const Work& w, int* err, cudaStream_t st) {
  const float* h = X;
  for (int l = 0; l < NL; ++l) {
    const int in = dim(l), out = dim(l + 1);
    const float* W = P + w_off(l);
    const float* b = W + out * in;
    if (l < NL - 1) tc_gemm<false, true, 1>(n, out, in, h, in, W, in, w.Z[l], out, b, w.H[l], nullptr, 1, err, st);
    else tc_gemm<false, true, 0>(n, out, in, h, in, W, in, w.Z[l], out, b, nullptr, nullptr, 1, err, st);
    h = l < NL - 1 ? w.H[l] : nullptr;
  }
}

static void loss_grad_tc(const float* params, const float* X, const float* Y, const float* M, int n, float* grad,
                         float* loss, const Work& w, int* err, const OutW& ow, cudaStream_t st) {
  forward_tc(params, X, n, w, err, st);
  const size_t ny = (size_t)n * CT_MLP_OUT;
  const int nb = (int)((ny + 255) / 256 < 256 ? (ny + 255) / 256 : 256);
  k_mse<<<nb, 256, 0, st>>>(w.Z[NL - 1], Y, M, ny, ow, w.g0, w.part);
  k_mse_finish<<<nb, 256, 0, st>>>(w.part, nb, w.g0, ny, loss);
  const int splits = n / 256 < 1 ? 1 : (n / 256 > TC_SPLIT_MAX ? TC_SPLIT_MAX : n / 256);
  float* g = w.g0;
  float* gn = w.g1;
  for (int l = NL - 1; l >= 0; --l) {
    const int in = dim(l), out = dim(l + 1);
    const float* W = params + w_off(l);
    float* gW = grad + w_off(l);
    float* gb = gW + out * in;
    if (l < NL - 1) {
      const size_t tot = (size_t)n * out;
      k_silu_bwd<<<(int)((tot + 255) / 256 < 4096 ? (tot + 255) / 256 : 4096), 256, 0, st>>>(g, w.Z[l], tot);
    }
    const float* hin = l == 0 ? X : w.H[l - 1];
    // dW = dZ^T h (out x in): split-K over the batch rows, partials summed in order
    tc_gemm<true, false, 2>(out, in, n, g, out, hin, in, nullptr, 0, nullptr, nullptr, w.ptc, splits, err, st);
    k_splitk_sum<<<(out * in + 255) / 256, 256, 0, st>>>(w.ptc, splits, out * in, gW);
    k_colsum<<<out, 256, 0, st>>>(g, n, out, gb);
    if (l > 0) tc_gemm<false, false, 0>(n, in, out, g, out, W, in, gn, in, nullptr, nullptr, nullptr, 1, err, st);
    float* t = g;
    g = gn;
    gn = t;
  }
}

}  // namespace ctm

using namespace ctm;

extern "C" {

int ct_mlp_param_count(void) { return NPARAM; }

size_t ct_mlp_work_bytes(int n) { return n > 0 ? work_bytes(n) : 0; }

ct_status ct_mlp_forward(const float* params, const float* X, int n, float* Y, void* work, size_t wbytes, void* stream) {
  if (!params || !X || !Y || !work || n <= 0) return fail(CT_ERR_ARG, "ct_mlp_forward: null pointer or n <= 0");
  if (wbytes < work_bytes(n)) return fail(CT_ERR_SIZE, "ct_mlp_forward: work too small (ct_mlp_work_bytes)");
  cudaStream_t st = (cudaStream_t)stream;
  Work w = carve((float*)work, n);
  forward(params, X, n, w, st);
  if (cudaMemcpyAsync(Y, w.Z[NL - 1], sizeof(float) * (size_t)n * CT_MLP_OUT, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return check("ct_mlp_forward copy");
  return check("ct_mlp_forward");
}

ct_status ct_mlp_loss_grad(const float* params, const float* X, const float* Y, const float* M, int n, float* grad,
                           float* loss, void* work, size_t wbytes, void* stream) {
  if (!params || !X || !Y || !M || !grad || !work || n <= 0) return fail(CT_ERR_ARG, "ct_mlp_loss_grad: bad argument");
  if (wbytes < work_bytes(n)) return fail(CT_ERR_SIZE, "ct_mlp_loss_grad: work too small (ct_mlp_work_bytes)");
  loss_grad(params, X, Y, M, n, grad, loss, carve((float*)work, n), ones_w(), (cudaStream_t)stream);
  return check("ct_mlp_loss_grad");
}

ct_status ct_mlp_loss_grad_tc(const float* params, const float* X, const float* Y, const float* M, int n, float* grad,
                              float* loss, int* err_flag, void* work, size_t wbytes, void* stream) {
  if (!params || !X || !Y || !M || !grad || !err_flag || !work || n <= 0)
    return fail(CT_ERR_ARG, "ct_mlp_loss_grad_tc: bad argument");
  if (wbytes < work_bytes(n)) return fail(CT_ERR_SIZE, "ct_mlp_loss_grad_tc: work too small (ct_mlp_work_bytes)");
  loss_grad_tc(params, X, Y, M, n, grad, loss, carve((float*)work, n), err_flag, ones_w(), (cudaStream_t)stream);
  return check("ct_mlp_loss_grad_tc");
}

ct_status ct_mlp_adam(float* params, const float* grad, float* m, float* v, int nparam, float lr, float beta1,
                      float beta2, float eps, int step, void* stream) {
  if (!params || !grad || !m || !v || nparam <= 0 || step < 1) return fail(CT_ERR_ARG, "ct_mlp_adam: bad argument");
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  k_adam<<<(nparam + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, nparam, lr, beta1, beta2, eps, c1, c2);
  return check("ct_mlp_adam");
}

ct_status ct_mlp_colstats(const float* X, const float* M, int n, int d, float* out, void* stream) {
  if (!X || !out || n <= 0 || d <= 0) return fail(CT_ERR_ARG, "ct_mlp_colstats: bad argument");
  k_colstats<<<d, 256, 0, (cudaStream_t)stream>>>(X, M, n, d, out);
  return check("ct_mlp_colstats");
}

ct_status ct_mlp_standardize(float* X, int n, int d, const float* mean, const float* sd, void* stream) {
  if (!X || !mean || !sd || n <= 0 || d <= 0) return fail(CT_ERR_ARG, "ct_mlp_standardize: bad argument");
  const size_t tot = (size_t)n * d;
  k_standardize<<<(int)((tot + 255) / 256 < 8192 ? (tot + 255) / 256 : 8192), 256, 0, (cudaStream_t)stream>>>(X, n, d,
                                                                                                           mean, sd);
  return check("ct_mlp_standardize");
}

}  // extern "C"
namespace ctm {

// ---- the training loop in one call -----------------------------------------------------------
static uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static size_t align_up(size_t b) { return (b + 255) & ~(size_t)255; }

// workspace: Xn (n x in), Yn (n x out), epoch permutation (n ints), batch rows x/y/m, gradient
// and the two Adam moments (NPARAM each), the loss (1 float), per-epoch loss sums (doubles),
// then the network work memory of one batch
static size_t train_ws_bytes(int n, int batch, int epochs) {
  const int rows = batch < n ? batch : n;
  size_t b = 0;
  b += align_up((size_t)n * CT_MLP_IN * sizeof(float));
  b += align_up((size_t)n * CT_MLP_OUT * sizeof(float));
  b += align_up((size_t)n * sizeof(int));
  b += align_up((size_t)rows * (CT_MLP_IN + 2 * CT_MLP_OUT) * sizeof(float));
  b += 3 * align_up((size_t)NPARAM * sizeof(float));
  b += align_up(sizeof(float));
  b += align_up((size_t)(epochs > 0 ? epochs : 1) * sizeof(double));
  b += align_up(work_bytes(rows));
  return b;
}

}  // namespace ctm
using namespace ctm;

extern "C" size_t ct_train_workspace_bytes(int n, int batch, int epochs) {
  if (n <= 0 || batch <= 0 || epochs <= 0) return 0;
  return train_ws_bytes(n, batch, epochs);
}

extern "C" ct_status ct_train_surrogate(const float* X, const float* Y, const float* M, int n, const ct_train_cfg* cfg,
                                        float* params, float* stats, float* loss_hist, void* work, size_t wbytes,
                                        void* stream) {
  if (!X || !Y || !M || !cfg || !params || !stats || !loss_hist || !work || n <= 0)
    return fail(CT_ERR_ARG, "ct_train_surrogate: null pointer or n <= 0");
  if (cfg->epochs <= 0 || cfg->batch <= 0 || !(cfg->lr > 0.0f) || !(cfg->lr_final >= 0.0f) ||
      !(cfg->beta1 >= 0.0f && cfg->beta1 < 1.0f) || !(cfg->beta2 >= 0.0f && cfg->beta2 < 1.0f) || !(cfg->eps > 0.0f))
    return fail(CT_ERR_ARG, "ct_train_surrogate: invalid configuration");
  if (cfg->tensor_cores != 0 && cfg->tensor_cores != 1) return fail(CT_ERR_ARG, "ct_train_surrogate: tensor_cores must be 0 or 1");
  OutW ow;
  float wsum = 0.0f;
  for (int q = 0; q < CT_MLP_OUT; ++q) {
    if (!(cfg->out_weight[q] >= 0.0f)) return fail(CT_ERR_ARG, "ct_train_surrogate: output weights must be >= 0");
    ow.w[q] = cfg->out_weight[q];
    wsum += ow.w[q];
  }
  if (!(wsum > 0.0f)) return fail(CT_ERR_ARG, "ct_train_surrogate: output weights all zero");
  if (wbytes < train_ws_bytes(n, cfg->batch, cfg->epochs))
    return fail(CT_ERR_SIZE, "ct_train_surrogate: workspace too small (ct_train_workspace_bytes)");
  cudaStream_t st = (cudaStream_t)stream;
  const int rows = cfg->batch < n ? cfg->batch : n;
  const int nb = n / rows > 0 ? n / rows : 1;      // batches per epoch; the tail of a shuffle is left out
  unsigned char* p = (unsigned char*)work;
  auto take = [&](size_t bytes) { unsigned char* q = p; p += align_up(bytes); return q; };
  float* Xn = (float*)take((size_t)n * CT_MLP_IN * sizeof(float));
  float* Yn = (float*)take((size_t)n * CT_MLP_OUT * sizeof(float));
  int* perm_d = (int*)take((size_t)n * sizeof(int));
  float* xb = (float*)take((size_t)rows * (CT_MLP_IN + 2 * CT_MLP_OUT) * sizeof(float));
  float* yb = xb + (size_t)rows * CT_MLP_IN;
  float* mb = yb + (size_t)rows * CT_MLP_OUT;
  float* G = (float*)take((size_t)NPARAM * sizeof(float));
  float* m1 = (float*)take((size_t)NPARAM * sizeof(float));
  float* m2 = (float*)take((size_t)NPARAM * sizeof(float));
  float* loss = (float*)take(sizeof(float));
  double* acc = (double*)take((size_t)cfg->epochs * sizeof(double));
  Work w = carve((float*)take(work_bytes(rows)), rows);
  // statistics: inputs unmasked, targets over their mask; standardised copies
  float* sx = stats;                      // 4 x CT_MLP_IN: mean, sd, min, max
  float* sy = stats + 4 * CT_MLP_IN;      // 4 x CT_MLP_OUT
  k_colstats<<<CT_MLP_IN, 256, 0, st>>>(X, nullptr, n, CT_MLP_IN, sx);
  k_colstats<<<CT_MLP_OUT, 256, 0, st>>>(Y, M, n, CT_MLP_OUT, sy);
  k_fix_sd<<<1, 32, 0, st>>>(sx, CT_MLP_IN);
  k_fix_sd<<<1, 32, 0, st>>>(sy, CT_MLP_OUT);
  const size_t nx = (size_t)n * CT_MLP_IN, ny = (size_t)n * CT_MLP_OUT;
  const int g1 = (int)((nx + 255) / 256 < 8192 ? (nx + 255) / 256 : 8192);
  const int g2 = (int)((ny + 255) / 256 < 8192 ? (ny + 255) / 256 : 8192);
  if (cudaMemcpyAsync(Xn, X, nx * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(Yn, Y, ny * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(m1, 0, (size_t)NPARAM * sizeof(float), st) != cudaSuccess ||
      cudaMemsetAsync(m2, 0, (size_t)NPARAM * sizeof(float), st) != cudaSuccess ||
      cudaMemsetAsync(acc, 0, (size_t)cfg->epochs * sizeof(double), st) != cudaSuccess ||
      cudaMemsetAsync(w.err, 0, sizeof(int), st) != cudaSuccess)
    return check("ct_train_surrogate setup");
  k_standardize<<<g1, 256, 0, st>>>(Xn, n, CT_MLP_IN, sx, sx + CT_MLP_IN);
  k_standardize<<<g2, 256, 0, st>>>(Yn, n, CT_MLP_OUT, sy, sy + CT_MLP_OUT);
  k_mask_mul<<<g2, 256, 0, st>>>(Yn, M, ny);
  ct_status s = check("ct_train_surrogate setup");
  if (s != CT_OK) return s;
  // epochs: a Fisher-Yates shuffle from splitmix64 (seed, epoch), batches of `rows` rows,
  // Adam with a cosine learning rate from lr to lr_final over all steps
  std::vector<int> perm(n);
  uint64_t rng = cfg->seed;
  const int total = cfg->epochs * nb;
  const int ggrid = (int)(((size_t)rows * (CT_MLP_IN + 2 * CT_MLP_OUT) + 255) / 256 < 4096
                              ? ((size_t)rows * (CT_MLP_IN + 2 * CT_MLP_OUT) + 255) / 256 : 4096);
  int step = 0;
  for (int e = 0; e < cfg->epochs; ++e) {
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int i = n - 1; i > 0; --i) {
      const int j = (int)(splitmix64(rng) % (uint64_t)(i + 1));
      const int t = perm[i];
      perm[i] = perm[j];
      perm[j] = t;
    }
    // a pageable copy returns once the host buffer has been staged: perm may be refilled
    if (cudaMemcpyAsync(perm_d, perm.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return check("ct_train_surrogate shuffle");
    for (int b = 0; b < nb; ++b) {
      k_gather_rows<<<ggrid, 256, 0, st>>>(perm_d + (size_t)b * rows, rows, Xn, Yn, M, xb, yb, mb);
      if (cfg->tensor_cores) loss_grad_tc(params, xb, yb, mb, rows, G, loss, w, w.err, ow, st);
      else loss_grad(params, xb, yb, mb, rows, G, loss, w, ow, st);
      ++step;
      const double frac = (double)step / (double)total;
      const float lr_t = (float)(cfg->lr_final + 0.5 * (cfg->lr - cfg->lr_final) * (1.0 + std::cos(M_PI * frac)));
      const float c1 = 1.0f - powf(cfg->beta1, (float)step), c2 = 1.0f - powf(cfg->beta2, (float)step);
      k_adam<<<(NPARAM + 255) / 256, 256, 0, st>>>(params, G, m1, m2, NPARAM, lr_t, cfg->beta1, cfg->beta2, cfg->eps,
                                                   c1, c2);
      k_acc_loss<<<1, 32, 0, st>>>(loss, acc, e);
    }
    if ((s = check("ct_train_surrogate epoch")) != CT_OK) return s;
  }
  std::vector<double> h(cfg->epochs);
  int err = 0;
  if (cudaMemcpyAsync(h.data(), acc, (size_t)cfg->epochs * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return check("ct_train_surrogate loss history");
  for (int e = 0; e < cfg->epochs; ++e) loss_hist[e] = (float)(h[e] / nb);
  if (err) return fail(CT_ERR_TIMEOUT, "ct_train_surrogate: a tensor-core wait gave up");
  return CT_OK;
}
