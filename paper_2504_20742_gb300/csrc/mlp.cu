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

#include "../../include/contrail.h"

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

// masked MSE: dY = 2 m (yhat - y) / count, per-block partial sums of m (yhat - y)^2 and m
__global__ void k_mse(const float* __restrict__ Yh, const float* __restrict__ Y, const float* __restrict__ Mk, size_t n,
                      float* __restrict__ dY, double* __restrict__ part) {
  __shared__ double s0[256], s1[256];
  double a = 0.0, c = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float r = (Yh[i] - Y[i]) * Mk[i];
    dY[i] = r;
    a += (double)r * r;
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
// n x 128 gradient buffers, then 2*256 doubles of loss partials.
static size_t work_floats(int n) {
  size_t f = 0;
  for (int l = 0; l < NL; ++l) f += (size_t)n * dim(l + 1);
  for (int l = 0; l < NL - 1; ++l) f += (size_t)n * dim(l + 1);
  f += 2 * (size_t)n * CT_MLP_HIDDEN;
  return f;
}
static size_t work_bytes(int n) { return work_floats(n) * sizeof(float) + 2 * 256 * sizeof(double) + 256; }

struct Work {
  float* Z[NL];
  float* H[NL - 1];
  float* g0;
  float* g1;
  double* part;
};
static Work carve(float* w, int n) {
  Work k;
  float* p = w;
  for (int l = 0; l < NL; ++l) { k.Z[l] = p; p += (size_t)n * dim(l + 1); }
  for (int l = 0; l < NL - 1; ++l) { k.H[l] = p; p += (size_t)n * dim(l + 1); }
  k.g0 = p; p += (size_t)n * CT_MLP_HIDDEN;
  k.g1 = p; p += (size_t)n * CT_MLP_HIDDEN;
  uintptr_t a = ((uintptr_t)p + 255) & ~(uintptr_t)255;
  k.part = (double*)a;
  return k;
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
  cudaStream_t st = (cudaStream_t)stream;
  Work w = carve((float*)work, n);
  forward(params, X, n, w, st);
  // dL/dyhat into g0 (n x 10)
  const size_t ny = (size_t)n * CT_MLP_OUT;
  const int nb = (int)((ny + 255) / 256 < 256 ? (ny + 255) / 256 : 256);
  k_mse<<<nb, 256, 0, st>>>(w.Z[NL - 1], Y, M, ny, w.g0, w.part);
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
  return check("ct_mlp_loss_grad");
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
