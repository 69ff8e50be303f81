// ||X||^2 = nu^T (V^T V)^d nu (Lemma 3.4 applied to X, Sec. 3.3) on the CUDA cores.
//
// The p x p Gram matrix is never formed: persistent blocks walk the upper triangle of
// 64 x 64 sample-tile pairs (I <= J), form the tile G = V_I V_J^T in registers (features staged
// in chunks of at most KC, so any n fits in shared memory), and add
// (2 - [I == J]) * sum_{l in I, k in J} nu_l nu_k G_lk^d to an FP64 block total. Block totals are
// summed in index order by reduce_scalar (deterministic).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "stmf_internal.h"

namespace stmf {
namespace {

constexpr int TG = 64;   // samples per tile
constexpr int KC = 128;  // features per shared-memory chunk
constexpr int NT = 256;  // threads: 16 x 16, each a 4 x 4 block of the tile pair

template <int DT> struct St;
template <> struct St<STMF_F64> { using T = double; };
template <> struct St<STMF_F32> { using T = float; };
template <> struct St<STMF_BF16> { using T = __nv_bfloat16; };
template <> struct St<STMF_E4M3> { using T = __nv_fp8_e4m3; };

template <typename TC> __device__ __forceinline__ TC cv(double x) { return (TC)x; }
template <typename TC> __device__ __forceinline__ TC cv(float x) { return (TC)x; }
template <typename TC> __device__ __forceinline__ TC cv(__nv_bfloat16 x) {
  return (TC)__bfloat162float(x);
}
template <typename TC> __device__ __forceinline__ TC cv(__nv_fp8_e4m3 x) { return (TC)(float)x; }

__host__ __device__ inline int gstride(int n) { return (n % 2 == 0) ? n + 1 : n; }

// pair index q -> (I, J), I <= J, row-major over the upper triangle of a T x T grid
__device__ __forceinline__ void pair_of(int64_t q, int64_t T, int64_t& I, int64_t& J) {
  // rows I hold T - I pairs; first index of row I is I*T - I*(I-1)/2
  double b = 2.0 * double(T) + 1.0;
  int64_t i = (int64_t)floor((b - sqrt(b * b - 8.0 * double(q))) * 0.5);
  if (i < 0) i = 0;
  if (i >= T) i = T - 1;
  auto start = [T](int64_t k) { return k * T - k * (k - 1) / 2; };
  while (i > 0 && start(i) > q) --i;
  while (i + 1 < T && start(i + 1) <= q) ++i;
  I = i;
  J = i + (q - start(i));
}

// features [k0, k0 + kc) of samples s0 .. s0 + TG (zero past `valid`), row stride gs
template <typename TC, int DT>
__device__ void load_tile(TC* dst, const typename St<DT>::T* V, const float* scale, int64_t s0,
                          int valid, int k0, int kc, int gs, int ld) {
  for (int e = threadIdx.x; e < TG * kc; e += NT) {
    const int s = e / kc, i = e - s * kc;
    TC v = (TC)0;
    if (s < valid) {
      v = cv<TC>(V[(s0 + s) * ld + k0 + i]);
      if (DT == STMF_E4M3) v *= (TC)scale[s0 + s];
    }
    dst[s * gs + i] = v;
  }
}

template <typename TC>
__device__ __forceinline__ TC ipow_t(TC z, int e) {
  TC t = z;
  for (int k = 1; k < e; ++k) t *= z;
  return t;
}

template <typename TC, int DT>
__global__ void __launch_bounds__(NT) gram_simt_kernel(const GramParams prm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = prm.n, gs = gstride(n < KC ? n : KC);
  TC* Vi = reinterpret_cast<TC*>(smem_raw);
  TC* Vj = Vi + TG * gs;
  TC* nui = Vj + TG * gs;
  TC* nuj = nui + TG;
  __shared__ double red[NT / 32];
  const auto* V = reinterpret_cast<const typename St<DT>::T*>(prm.V);
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  const int64_t T = (prm.p + TG - 1) / TG;
  const int64_t pairs = T * (T + 1) / 2;
  double total = 0.0;
  for (int64_t q = blockIdx.x; q < pairs; q += gridDim.x) {
    int64_t I, J;
    pair_of(q, T, I, J);
    const int vi = (int)(prm.p - I * TG < TG ? prm.p - I * TG : TG);
    const int vj = (int)(prm.p - J * TG < TG ? prm.p - J * TG : TG);
    TC g[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) g[a][b] = (TC)0;
    for (int k0 = 0; k0 < n; k0 += KC) {  // features in index order, chunk by chunk
      const int kc = n - k0 < KC ? n - k0 : KC;
      __syncthreads();
      load_tile<TC, DT>(Vi, V, prm.scale, I * TG, vi, k0, kc, gs, prm.ld);
      load_tile<TC, DT>(Vj, V, prm.scale, J * TG, vj, k0, kc, gs, prm.ld);
      if (k0 == 0 && tid < TG) {
        nui[tid] = tid < vi ? (TC)(prm.nu ? prm.nu[I * TG + tid] : prm.nu_uniform) : (TC)0;
        nuj[tid] = tid < vj ? (TC)(prm.nu ? prm.nu[J * TG + tid] : prm.nu_uniform) : (TC)0;
      }
      __syncthreads();
      for (int i = 0; i < kc; ++i) {
        TC x[4], y[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) x[a] = Vi[(4 * ty + a) * gs + i];
#pragma unroll
        for (int b = 0; b < 4; ++b) y[b] = Vj[(4 * tx + b) * gs + i];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) g[a][b] += x[a] * y[b];
      }
    }
    TC part = (TC)0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      TC rowsum = (TC)0;
#pragma unroll
      for (int b = 0; b < 4; ++b) rowsum += nuj[4 * tx + b] * ipow_t(g[a][b], prm.d);
      part += nui[4 * ty + a] * rowsum;
    }
    double x = (double)part;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((tid & 31) == 0) red[tid >> 5] = x;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < NT / 32; ++w) t += red[w];
      total += (I == J ? 1.0 : 2.0) * t;
    }
  }
  if (tid == 0) prm.partials[blockIdx.x] = total;
}

template <typename TC>
size_t gram_smem(int n) {
  return sizeof(TC) * (2 * size_t(TG) * gstride(n < KC ? n : KC) + 2 * TG);
}

template <typename TC, int DT>
cudaError_t launch(const GramParams& prm, int grid, cudaStream_t s) {
  const cudaError_t e = smem_limit((const void*)gram_simt_kernel<TC, DT>, 232448 - 1024);
  if (e != cudaSuccess) return e;
  gram_simt_kernel<TC, DT><<<grid, NT, gram_smem<TC>(prm.n), s>>>(prm);
  return cudaGetLastError();
}

}  // namespace

int gram_simt_grid(int dtype, int n, int64_t p, int num_sms) {
  const size_t smem = dtype == STMF_F64 ? gram_smem<double>(n) : gram_smem<float>(n);
  int per_sm = (int)((228 * 1024) / (smem + 2048));
  per_sm = per_sm < 1 ? 1 : (per_sm > 2 ? 2 : per_sm);
  const int64_t T = (p + TG - 1) / TG;
  const int64_t pairs = T * (T + 1) / 2;
  int64_t grid = int64_t(num_sms) * per_sm;
  if (grid > pairs) grid = pairs;
  return (int)(grid < 1 ? 1 : grid);
}

cudaError_t gram_simt_launch(int dtype, const GramParams& prm, int grid, cudaStream_t s) {
  switch (dtype) {
    case STMF_F64: return launch<double, STMF_F64>(prm, grid, s);
    case STMF_F32: return launch<float, STMF_F32>(prm, grid, s);
    case STMF_BF16: return launch<float, STMF_BF16>(prm, grid, s);
    case STMF_E4M3: return launch<float, STMF_E4M3>(prm, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace stmf
