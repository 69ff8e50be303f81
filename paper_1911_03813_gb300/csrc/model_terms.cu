// Model terms and outputs of Alg. 2 (lines 3-9), in FP64.
//
// reduce_partials: (w, Y) = sum over the pass's blocks of their FP64 partials, one thread per
//                  entry, blocks summed in index order (deterministic).
// finalize:        one block forms B = A^T A, C = B^{d-1}, u = (B * C) lambda (Lemma 3.4),
//                  f = alpha + lambda^T u - 2 w^T lambda, g_lambda = -2 (w - u) (eq. gradl) and
//                  G_A = -2 d (Y - A D_lambda C) D_lambda (eq. gradb).
// The two inner products of line 7 are summed by one thread in index order, so f is
// reproducible bit for bit.
#include "stmf_internal.h"

namespace stmf {
namespace {

constexpr int RT = 256;

__global__ void reduce_partials_kernel(const double* __restrict__ partials, int grid, int L,
                                       double* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= L) return;
  double s = 0.0;
  for (int g = 0; g < grid; ++g) s += partials[size_t(g) * L + e];
  out[e] = s;
}

__device__ __forceinline__ double ipow_d(double z, int e) {
  double t = 1.0;
  for (int k = 0; k < e; ++k) t *= z;
  return t;
}

// dynamic shared memory: B[r*r] and C[r*r] (r <= 64: at most 64 KB)
__global__ void __launch_bounds__(RT) finalize_kernel(const ModelParams prm) {
  extern __shared__ double dyn[];
  double* Bs = dyn;
  double* Cs = dyn + prm.r * prm.r;
  __shared__ double us[64];
  __shared__ double lam[64];
  __shared__ double fs;
  const int n = prm.n, r = prm.r, d = prm.d;
  const double* w = prm.yw;
  const double* Y = prm.yw + r;
  const double* A = prm.A;
  const int tid = threadIdx.x;

  for (int j = tid; j < r; j += RT) lam[j] = prm.lambda[j];
  // line 4: B = A^T A; line 5: C = B^{d-1}
  for (int e = tid; e < r * r; e += RT) {
    const int j = e / r, k = e % r;
    double b = 0.0;
    for (int i = 0; i < n; ++i) b += A[i + size_t(n) * j] * A[i + size_t(n) * k];
    Bs[e] = b;
    Cs[e] = ipow_d(b, d - 1);
  }
  __syncthreads();
  // line 6: u = (B * C) lambda
  for (int j = tid; j < r; j += RT) {
    double u = 0.0;
    for (int k = 0; k < r; ++k) u += Bs[j * r + k] * Cs[j * r + k] * lam[k];
    us[j] = u;
  }
  __syncthreads();
  if (tid == 0) {
    // line 7: f = alpha + lambda^T u - 2 w^T lambda
    double lu = 0.0, wl = 0.0;
    for (int j = 0; j < r; ++j) {
      lu += lam[j] * us[j];
      wl += w[j] * lam[j];
    }
    const double alpha = prm.alpha ? *prm.alpha : 0.0;
    const double f = alpha + lu - 2.0 * wl;
    fs = f;
    *prm.f = f;
  }
  // line 8: g_lambda = -2 (w - u)
  for (int j = tid; j < r; j += RT) prm.g_lambda[j] = -2.0 * (w[j] - us[j]);
  // line 9: G_A = -2 d (Y - A D_lambda C) D_lambda
  for (int e = tid; e < n * r; e += RT) {
    const int j = e / n, i = e % n;
    double t = 0.0;
    for (int k = 0; k < r; ++k) t += A[i + size_t(n) * k] * lam[k] * Cs[k * r + j];
    prm.G_A[e] = -2.0 * d * (Y[e] - t) * lam[j];
  }
  __syncthreads();
  if (tid == 0 && !isfinite(fs)) stmf_set_status(prm.status, STMF_ENONFINITE);
}

__global__ void reduce_scalar_kernel(const double* __restrict__ partials, int count,
                                     double* __restrict__ out, int32_t* status) {
  // one thread, index order: deterministic
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int g = 0; g < count; ++g) s += partials[g];
    *out = s;
    if (!isfinite(s)) stmf_set_status(status, STMF_ENONFINITE);
  }
}

}  // namespace

cudaError_t model_terms_launch(const ModelParams& prm, cudaStream_t s) {
  const int L = prm.r + prm.n * prm.r;
  reduce_partials_kernel<<<(L + RT - 1) / RT, RT, 0, s>>>(prm.partials, prm.grid, L, prm.yw);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  static bool configured = false;
  if (!configured) {
    e = cudaFuncSetAttribute(finalize_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             2 * 64 * 64 * int(sizeof(double)));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  finalize_kernel<<<1, RT, 2 * prm.r * prm.r * sizeof(double), s>>>(prm);
  return cudaGetLastError();
}

cudaError_t reduce_scalar_launch(const double* partials, int count, double* out,
                                 int32_t* status, cudaStream_t s) {
  reduce_scalar_kernel<<<1, 32, 0, s>>>(partials, count, out, status);
  return cudaGetLastError();
}

}  // namespace stmf
