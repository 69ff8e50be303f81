// Model terms and outputs of Alg. 2 (every step after Y), in FP64.
//
// reduce_kernel:   (w, Y) = sum over the pass's blocks of their FP64 partials (16 threads per
//                  entry, combined in a fixed order, so results are reproducible bit for bit),
//                  and, in extra blocks, B = A^T A (Alg. 2), one warp per entry.
// finalize_kernel: C = B^{d-1} (element-wise), then one thread per entry of
//                  G_A = -2 d (Y - A D_lambda C) D_lambda (eq. gradb); block 0 also forms
//                  u = (B * C) lambda (Lemma 3.4), f = alpha + lambda^T u - 2 w^T lambda
//                  and g_lambda = -2 (w - u) (eq. gradl). The two inner products of f are
//                  summed by one thread in index order.
#include "stmf_internal.h"

namespace stmf {
namespace {

constexpr int RT = 128;

__device__ __forceinline__ double ipow_d(double z, int e) {
  double t = 1.0;
  for (int k = 0; k < e; ++k) t *= z;
  return t;
}

// Block (RE x RY): thread (x, y) sums the partials of blocks y, y + RY, y + 2 RY, ... of entry
// e = blockIdx.x * RE + x, issuing all of its loads before adding; the RY sums are then added in
// y order. The order is fixed, so results are reproducible bit for bit.
constexpr int RE = 32;    // entries per block
constexpr int RY = 16;    // threads per entry
constexpr int RMAX = 20;  // loads per thread (pass grid <= RY * RMAX = 320 blocks)

__global__ void __launch_bounds__(RE * RY) reduce_kernel(const ModelParams prm, int L, int nb) {
  if (prm.skip && *prm.skip) return;
  __shared__ double red[RY][RE];
  const int x = threadIdx.x % RE, y = threadIdx.x / RE;
  if ((int)blockIdx.x < nb) {
    const int e = blockIdx.x * RE + x;
    double s = 0.0;
    if (e < L) {
      const double* p = prm.partials + e;
      double v[RMAX];
#pragma unroll
      for (int k = 0; k < RMAX; ++k) {
        const int g = y + k * RY;
        v[k] = g < prm.grid ? p[size_t(g) * L] : 0.0;
      }
#pragma unroll
      for (int k = 0; k < RMAX; ++k) s += v[k];
    }
    red[y][x] = s;
    __syncthreads();
    if (y == 0 && e < L) {
      double t = red[0][x];
#pragma unroll
      for (int k = 1; k < RY; ++k) t += red[k][x];
      prm.yw[e] = prm.accumulate ? prm.yw[e] + t : t;
    }
    return;
  }
  // B = A^T A: one warp per entry, lanes stride the features, then a fixed-order warp sum
  const int n = prm.n, r = prm.r;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = (blockIdx.x - nb) * (RE * RY / 32) + warp;
  if (e >= r * r) return;
  const int j = e / r, k = e - j * r;
  const double* aj = prm.A + size_t(n) * j;
  const double* ak = prm.A + size_t(n) * k;
  double b = 0.0;
  for (int i = lane; i < n; i += 32) b += aj[i] * ak[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
  if (lane == 0) prm.bmat[e] = b;
}

__global__ void __launch_bounds__(RT) finalize_kernel(const ModelParams prm) {
  if (prm.skip && *prm.skip) return;
  if (prm.poison && *(volatile int32_t*)prm.status != 0) {
    // an earlier step of this evaluation reported an error (e.g. a pass whose bounded wait ran
    // out left its block partials unwritten): the outputs must not look like a valid result
    const double qnan = __longlong_as_double(0x7ff8000000000000LL);
    const int e = blockIdx.x * RT + threadIdx.x;
    if (e < prm.n * prm.r) prm.G_A[e] = qnan;
    if (blockIdx.x == 0) {
      for (int j = threadIdx.x; j < prm.r; j += RT) prm.g_lambda[j] = qnan;
      if (threadIdx.x == 0) *prm.f = qnan;
    }
    return;
  }
  __shared__ double Cs[64 * 64];
  __shared__ double lam[64];
  __shared__ double us[64];
  const int n = prm.n, r = prm.r, d = prm.d;
  const double* w = prm.yw;
  const double* Y = prm.yw + r;
  const int tid = threadIdx.x;
  for (int j = tid; j < r; j += RT) lam[j] = prm.lambda[j];
  for (int e = tid; e < r * r; e += RT) Cs[e] = ipow_d(prm.bmat[e], d - 1);
  __syncthreads();
  const int e = blockIdx.x * RT + tid;
  if (e < n * r) {
    const int j = e / n, i = e - j * n;
    double t = 0.0;
    for (int k = 0; k < r; ++k) t += prm.A[i + size_t(n) * k] * lam[k] * Cs[k * r + j];
    prm.G_A[e] = -2.0 * d * (Y[e] - t) * lam[j];
  }
  if (blockIdx.x != 0) return;
  for (int j = tid; j < r; j += RT) {
    double u = 0.0;
    for (int k = 0; k < r; ++k) u += prm.bmat[j * r + k] * Cs[j * r + k] * lam[k];
    us[j] = u;
    prm.g_lambda[j] = -2.0 * (w[j] - u);
  }
  __syncthreads();
  if (tid == 0) {
    double lu = 0.0, wl = 0.0;
    for (int j = 0; j < r; ++j) {
      lu += lam[j] * us[j];
      wl += w[j] * lam[j];
    }
    const double alpha = prm.alpha ? *prm.alpha : 0.0;
    const double f = alpha + lu - 2.0 * wl;
    *prm.f = f;
    if (!isfinite(f)) stmf_set_status(prm.status, STMF_ENONFINITE);
  }
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
  const int nb = (L + RE - 1) / RE;
  if (prm.grid > RY * RMAX) return cudaErrorInvalidValue;
  const int nbB = (prm.r * prm.r + (RE * RY / 32) - 1) / (RE * RY / 32);
  cudaError_t e = launch_kernel(reduce_kernel, dim3(nb + nbB), dim3(RE * RY), 0, s, prm, L, nb);
  if (e != cudaSuccess) return e;
  return launch_kernel(finalize_kernel, dim3((prm.n * prm.r + RT - 1) / RT), dim3(RT), 0, s, prm);
}

cudaError_t reduce_partials_launch(const ModelParams& prm, cudaStream_t s) {
  const int L = prm.r + prm.n * prm.r;
  const int nb = (L + RE - 1) / RE;
  if (prm.grid > RY * RMAX) return cudaErrorInvalidValue;
  reduce_kernel<<<nb, RE * RY, 0, s>>>(prm, L, nb);
  return cudaGetLastError();
}

cudaError_t finish_launch(const ModelParams& prm, cudaStream_t s) {
  const int nbB = (prm.r * prm.r + (RE * RY / 32) - 1) / (RE * RY / 32);
  reduce_kernel<<<nbB, RE * RY, 0, s>>>(prm, prm.r + prm.n * prm.r, 0);  // B blocks only
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  finalize_kernel<<<(prm.n * prm.r + RT - 1) / RT, RT, 0, s>>>(prm);
  return cudaGetLastError();
}

cudaError_t reduce_scalar_launch(const double* partials, int count, double* out,
                                 int32_t* status, cudaStream_t s) {
  reduce_scalar_kernel<<<1, 32, 0, s>>>(partials, count, out, status);
  return cudaGetLastError();
}

}  // namespace stmf
