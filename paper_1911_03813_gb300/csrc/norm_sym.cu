// ||X||^2 from the distinct entries of the symmetric moment tensor (Sec. 3.3: the constant term
// of f; the paper notes that the implicit O(n p^2) route can cost more than forming X).
//
// X = sum_l nu_l v_l^{(d)} is symmetric, so its entries are indexed by multisets m of d features:
// X_m = sum_l nu_l prod_{i in m} v_li, and every multiset stands for mult(m) = d! / prod_t c_t!
// index tuples (c_t: how often feature t occurs in m), so ||X||^2 = sum_m mult(m) X_m^2. Forming
// the C(n+d-1, d) distinct entries costs p C(n+d-1, d) multiply-adds against n p^2 / 2 for the
// Gram form, far less when p is large and n d small.
//
// A multiset is a sorted prefix P of d-1 features and a last feature k >= last(P). Block (x, y, z)
// owns prefixes [64 x, 64 x + 64) of the prefix table (ordered by last feature), features
// k in [64 y, 64 y + 64) and the z-th of S equal ranges of sample tiles: per 32-sample tile it
// forms T[l][P] = nu_l prod_{i in P} v_li in shared memory, then X[P][k] += T[l][P] v_lk in 4 x 4
// register blocks (FP32, folded into FP64 every 16 tiles; FP64 throughout for FP64 samples), and
// writes its FP64 partial of X to slab z. A second kernel adds the S slabs in order and sums
// mult(P, k) X[P][k]^2 over k >= last(P), k < n; its block partials are summed in index order
// (deterministic).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <vector>

#include "stmf_internal.h"

namespace stmf {
namespace {

constexpr int NT = 256;
constexpr int TSS = 32;  // samples per tile
constexpr int PT = 64;   // prefixes per block
constexpr int KT = 64;   // last features per block
constexpr int FLUSH = 16;

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

__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}
__device__ __forceinline__ void load4(const double* p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}

__host__ __device__ inline int row_of(int n) {  // padded features per staged sample
  return (n + KT - 1) / KT * KT + 4;
}

// two sample-tile buffers (the next tile streams in while the current one is used, for FP32 and
// FP64 samples), T, two buffers of nu, the block's prefixes
template <typename TC>
size_t smem_of(int n) {
  return sizeof(TC) * (2 * size_t(TSS) * row_of(n) + size_t(TSS) * PT) +
         sizeof(double) * 2 * TSS + sizeof(uint16_t) * PT * 8;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src), "r"(bytes)
               : "memory");
}

template <typename TC, int DT>
__global__ void __launch_bounds__(NT) norm_sym_kernel(const SymParams prm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = prm.n, L = prm.d - 1, row = row_of(n);
  TC* Vs0 = reinterpret_cast<TC*>(smem_raw);           // [2][TSS][row]
  TC* Ts = Vs0 + 2 * TSS * row;                        // [TSS][PT]
  double* nus0 = reinterpret_cast<double*>(Ts + TSS * PT);  // [2][TSS]
  uint16_t* Pidx = reinterpret_cast<uint16_t*>(nus0 + 2 * TSS);  // [PT][8]
  // samples already in the compute type stream in with cp.async, one tile ahead
  constexpr bool kAsync = (DT == STMF_F32 && sizeof(TC) == 4) || (DT == STMF_F64 && sizeof(TC) == 8);
  const int tid = threadIdx.x;
  const int64_t p0 = int64_t(blockIdx.x) * PT;
  const int k0 = blockIdx.y * KT;
  const int nk = int(gridDim.y) * KT;  // slab row length
  double* slab = prm.slabs + size_t(blockIdx.z) * size_t(prm.count) * nk;

  __shared__ int min_last;
  if (tid == 0) min_last = 1 << 30;
  __syncthreads();
  for (int e = tid; e < PT * 8; e += NT) {
    const int q = e >> 3, j = e & 7;
    Pidx[e] = (p0 + q < prm.count && j < 7) ? prm.prefixes[p0 + q].idx[j] : 0;
    if (j == L - 1 && p0 + q < prm.count) atomicMin(&min_last, int(Pidx[e]));
  }
  __syncthreads();
  // every k of this block lies below last(P) for all the block's prefixes: no valid entry (the
  // squaring kernel reads only k >= last(P), so these slab entries are never needed)
  if (k0 + KT <= min_last) return;

  const auto* V = reinterpret_cast<const typename St<DT>::T*>(prm.V);
  const int ty = tid >> 4, tx = tid & 15;  // prefixes 4 ty .. + 3, features k0 + 4 tx .. + 3
  TC acc[4][4];
  double accd[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      acc[a][b] = (TC)0;
      accd[a][b] = 0.0;
    }
  const int64_t tiles = (prm.p + TSS - 1) / TSS;
  const int64_t t_lo = tiles * blockIdx.z / gridDim.z, t_hi = tiles * (blockIdx.z + 1) / gridDim.z;
  // stage tile `tile` into buffer b: features past n and samples past p read as zero
  auto stage = [&](int64_t tile, int b) {
    TC* Vb = Vs0 + b * TSS * row;
    double* nb = nus0 + b * TSS;
    const int64_t s0 = tile * TSS;
    if constexpr (kAsync) {
      constexpr int EC = 16 / sizeof(TC);  // elements per 16-byte chunk
      const int cpr = row / EC;
      for (int e = tid; e < TSS * cpr; e += NT) {
        const int s = e / cpr, c = e - s * cpr;
        const int left = n - c * EC;
        const uint32_t bytes =
            (s0 + s < prm.p && left > 0) ? uint32_t((left >= EC ? EC : left) * sizeof(TC)) : 0u;
        const TC* src = bytes ? reinterpret_cast<const TC*>(V) + (s0 + s) * prm.ld + c * EC
                              : reinterpret_cast<const TC*>(V);
        cp_async16(smem_u32(Vb + s * row + c * EC), src, bytes);
      }
      if (tid < TSS) {
        const bool ok = s0 + tid < prm.p;
        if (prm.nu)
          cp_async8(smem_u32(nb + tid), ok ? prm.nu + s0 + tid : prm.nu, ok ? 8u : 0u);
        else
          nb[tid] = ok ? prm.nu_uniform : 0.0;
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    } else {
      for (int e = tid; e < TSS * row; e += NT) {
        const int s = e / row, i = e - s * row;
        TC v = (TC)0;
        if (i < n && s0 + s < prm.p) {
          v = cv<TC>(V[(s0 + s) * prm.ld + i]);
          if (DT == STMF_E4M3) v *= (TC)prm.scale[s0 + s];
        }
        Vb[e] = v;
      }
      if (tid < TSS)
        nb[tid] = s0 + tid < prm.p ? (prm.nu ? prm.nu[s0 + tid] : prm.nu_uniform) : 0.0;
    }
  };
  if (kAsync && t_lo < t_hi) stage(t_lo, 0);
  int since = 0;
  for (int64_t tile = t_lo; tile < t_hi; ++tile) {
    const int buf = kAsync ? int((tile - t_lo) & 1) : 0;
    const TC* Vs = Vs0 + buf * TSS * row;
    const double* nus = nus0 + buf * TSS;
    __syncthreads();  // the previous tile is done with its buffer and with Ts
    if constexpr (kAsync) {
      if (tile + 1 < t_hi) {
        stage(tile + 1, buf ^ 1);
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      }
    } else {
      stage(tile, 0);
    }
    __syncthreads();
    for (int e = tid; e < TSS * PT; e += NT) {
      const int s = e / PT, q = e - s * PT;
      TC t = (TC)nus[s];
      for (int j = 0; j < L; ++j) t *= Vs[s * row + Pidx[q * 8 + j]];
      Ts[e] = t;
    }
    __syncthreads();
#pragma unroll 4
    for (int s = 0; s < TSS; ++s) {
      TC tv[4], vv[4];
      load4(Ts + s * PT + 4 * ty, tv);
      load4(Vs + s * row + k0 + 4 * tx, vv);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += tv[a] * vv[b];
    }
    if (++since == FLUSH || tile == t_hi - 1) {
      since = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          accd[a][b] += (double)acc[a][b];
          acc[a][b] = (TC)0;
        }
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t q = p0 + 4 * ty + a;
    if (q >= prm.count) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) slab[size_t(q) * nk + k0 + 4 * tx + b] = accd[a][b];
  }
}

// ||X||^2 = sum over prefixes P and k >= last(P), k < n of mult(P, k) (sum of the slabs)^2
__global__ void __launch_bounds__(NT) sym_square_kernel(const SymParams prm, int nk, int S) {
  const int64_t q = int64_t(blockIdx.x) * (NT / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  double part = 0.0;
  if (q < prm.count) {
    const SymPrefix P = prm.prefixes[q];
    const int L = prm.d - 1, last = P.idx[L - 1];
    for (int k = last + lane; k < prm.n; k += 32) {  // every block holding such k wrote it
      double x = 0.0;
      for (int z = 0; z < S; ++z) x += prm.slabs[(size_t(z) * prm.count + q) * nk + k];
      const double m = k == last ? P.base / double(P.run + 1) : P.base;
      part += m * x * x;
    }
  }
  __shared__ double red[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (lane == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += red[w];
    prm.partials[blockIdx.x] = t;
  }
}

template <typename TC, int DT>
cudaError_t launch(const SymParams& prm, dim3 grid, cudaStream_t s) {
  // the opt-in limit covers static shared memory too (the kernel's reduction array)
  const cudaError_t e = smem_limit((const void*)norm_sym_kernel<TC, DT>, 232448 - 1024);
  if (e != cudaSuccess) return e;
  norm_sym_kernel<TC, DT><<<grid, NT, smem_of<TC>(prm.n), s>>>(prm);
  return cudaGetLastError();
}

}  // namespace

double sym_prefix_count(int n, int d) {
  // C(n + d - 2, d - 1) sorted prefixes of d - 1 features
  double c = 1.0;
  for (int j = 1; j <= d - 1; ++j) c = c * double(n - 1 + j) / double(j);
  return c;
}

void sym_prefixes(int n, int d, std::vector<SymPrefix>& out) {
  const int L = d - 1;
  out.clear();
  double dfact = 1.0;
  for (int j = 2; j <= d; ++j) dfact *= j;
  std::vector<int> idx(L, 0);
  while (true) {
    SymPrefix e{};
    double denom = 1.0;
    int run = 1;
    for (int j = 0; j < L; ++j) {
      e.idx[j] = uint16_t(idx[j]);
      if (j > 0 && idx[j] == idx[j - 1]) {
        ++run;
        denom *= run;
      } else {
        run = 1;
      }
    }
    e.run = uint16_t(run);  // length of the run of last(P)
    e.base = dfact / denom;
    out.push_back(e);
    // next sorted tuple (nondecreasing indices), lexicographic
    int j = L - 1;
    while (j >= 0 && idx[j] == n - 1) --j;
    if (j < 0) break;
    ++idx[j];
    for (int t = j + 1; t < L; ++t) idx[t] = idx[j];
  }
  // order by last feature (stable): a block of 64 consecutive prefixes then has nearly equal
  // last(P), and the blocks of features k below all of them have nothing to compute
  std::stable_sort(out.begin(), out.end(), [L](const SymPrefix& a, const SymPrefix& b) {
    return a.idx[L - 1] < b.idx[L - 1];
  });
}

size_t norm_sym_smem(int dtype, int n) {
  return dtype == STMF_F64 ? smem_of<double>(n) : smem_of<float>(n);
}

dim3 norm_sym_grid(long long count, int n, int64_t p, int num_sms) {
  // sample splits (z) until there are ~8 blocks per SM, while the slabs stay under 2 GB
  const long long gx = (count + PT - 1) / PT, gy = (n + KT - 1) / KT;
  const double slab = double(count) * double(gy * KT) * sizeof(double);
  long long S = (8LL * num_sms + gx * gy - 1) / (gx * gy);
  const long long tiles = (p + TSS - 1) / TSS;
  if (S > 16) S = 16;
  if (S > tiles) S = tiles;
  while (S > 1 && S * slab > 2e9) --S;
  if (S < 1) S = 1;
  return dim3((unsigned)gx, (unsigned)gy, (unsigned)S);
}

size_t norm_sym_slab_bytes(long long count, dim3 grid) {
  return size_t(count) * grid.y * KT * grid.z * sizeof(double);
}

int norm_sym_square_blocks(long long count) { return (int)((count + NT / 32 - 1) / (NT / 32)); }

cudaError_t norm_sym_launch(int dtype, const SymParams& prm, dim3 grid, cudaStream_t s) {
  cudaError_t e;
  switch (dtype) {
    case STMF_F64: e = launch<double, STMF_F64>(prm, grid, s); break;
    case STMF_F32: e = launch<float, STMF_F32>(prm, grid, s); break;
    case STMF_BF16: e = launch<float, STMF_BF16>(prm, grid, s); break;
    case STMF_E4M3: e = launch<float, STMF_E4M3>(prm, grid, s); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  sym_square_kernel<<<norm_sym_square_blocks(prm.count), NT, 0, s>>>(prm, int(grid.y) * KT,
                                                                      int(grid.z));
  return cudaGetLastError();
}

}  // namespace stmf
