// The CUDA-core fused pass (kernel template and its launch helpers), shared by the translation
// units that instantiate it: fg_simt.cu (FP32, BF16 and E4M3 samples), fg_simt_f64.cu (FP64
// samples) and fg_simt_rrf.cu (the randomized range finder). Split so the instantiations compile
// in parallel.
//
// Fused pass over the samples on the CUDA cores (FP64 and FP32 storage; also BF16/E4M3 for
// shapes the tensor-core pass does not take).
//
// One persistent block walks sample tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... and
// accumulates, for its tiles only,
//     Y_part = sum_l nu_l (v_l^T A)^{d-1} v_l^T      (Alg. 2, Lemma 3.3, eq. Y)
//     w_part = sum_l nu_l (v_l^T A)^d                (Lemma 3.5: w_j = X a_j^d = a_j^T y_j)
// Each tile is staged in shared memory once and used twice: phase 1 forms Z = V_tile A and the
// weighted powers W = D_nu Z^{d-1}; phase 2 adds V_tile^T W into register accumulators. FP32
// accumulators are folded into the block's FP64 partial slot every `flush_tiles` tiles, so an
// FP32 sum never runs over more than flush_tiles * 64 samples. Partials are combined across
// blocks in FP64 by the model-terms kernel in a fixed order (deterministic results).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "rrf_draw.cuh"
#include "stmf_internal.h"

namespace stmf {
namespace {

constexpr int TS_MAX = 64;  // samples per tile (32 when a 64-sample tile does not fit)
constexpr int NT = 256;     // threads per block
constexpr int MAXACC = 64;  // Y accumulators per thread

template <int DT>
struct Storage;
template <>
struct Storage<STMF_F64> { using T = double; };
template <>
struct Storage<STMF_F32> { using T = float; };
template <>
struct Storage<STMF_BF16> { using T = __nv_bfloat16; };
template <>
struct Storage<STMF_E4M3> { using T = __nv_fp8_e4m3; };

template <typename TC>
__device__ __forceinline__ TC widen(double x) { return (TC)x; }
template <typename TC>
__device__ __forceinline__ TC widen(float x) { return (TC)x; }
template <typename TC>
__device__ __forceinline__ TC widen(__nv_bfloat16 x) { return (TC)__bfloat162float(x); }
template <typename TC>
__device__ __forceinline__ TC widen(__nv_fp8_e4m3 x) { return (TC)(float)x; }

template <typename TC>
__device__ __forceinline__ TC ipow(TC z, int e) {
  TC t = z;
  for (int k = 1; k < e; ++k) t *= z;
  return e == 0 ? (TC)1 : t;
}

__host__ __device__ inline int vstride_of(int n) { return (n % 2 == 0) ? n + 1 : n; }

template <typename TC>
size_t smem_bytes(int n, int rp, int TS) {
  auto up16 = [](size_t b) { return (b + 15) & ~size_t(15); };
  size_t b = up16(sizeof(TC) * size_t(n) * rp);          // As[n][rp]
  b += up16(sizeof(TC) * size_t(TS) * vstride_of(n));    // Vs[TS][vstride]
  b += up16(sizeof(TC) * size_t(TS) * rp);               // Ws[TS][rp]
  b += up16(sizeof(TC) * TS);                            // nus[TS]
  b += up16(sizeof(double) * (NT / 32) * 16);            // wsh[warps][16]
  return b;
}

// RRF = false: the fused pass of Alg. 2. RRF = true: the randomized range finder of eq. rrf,
// Y_part = sum_l v_l omega_l^T with the test matrix drawn in phase 1 (no w).
template <typename TC, int DT, int JB, bool RRF, int TS>
__global__ void __launch_bounds__(NT) fg_simt_kernel(const FgParams prm) {
  constexpr int QG = NT / TS;  // phase 1: groups of column quads (one sample per thread)
  using TS_t = typename Storage<DT>::T;
  if (prm.skip && *prm.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = prm.n, r = prm.r, rp = prm.r_pad, d = prm.d, ld = prm.ld;
  const int vst = vstride_of(n);
  auto up16 = [](size_t b) { return (b + 15) & ~size_t(15); };
  unsigned char* ptr = smem_raw;
  TC* As = reinterpret_cast<TC*>(ptr);
  ptr += up16(sizeof(TC) * size_t(n) * rp);
  TC* Vs = reinterpret_cast<TC*>(ptr);
  ptr += up16(sizeof(TC) * size_t(TS) * vst);
  TC* Ws = reinterpret_cast<TC*>(ptr);
  ptr += up16(sizeof(TC) * size_t(TS) * rp);
  TC* nus = reinterpret_cast<TC*>(ptr);
  ptr += up16(sizeof(TC) * TS);
  double* wsh = reinterpret_cast<double*>(ptr);

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const TS_t* V = reinterpret_cast<const TS_t*>(prm.V);
  double* part = prm.partials + size_t(blockIdx.x) * (size_t(r) + size_t(n) * r);

  // A (FP64, n x r column-major) -> As[i][j] in the compute type, zero-padded to rp columns.
  if constexpr (!RRF) {
    for (int e = tid; e < n * rp; e += NT) {
      const int i = e / rp, j = e - i * rp;
      As[e] = j < r ? (TC)prm.A[i + size_t(n) * j] : (TC)0;
    }
  }
  for (int e = tid; e < (NT / 32) * 16; e += NT) wsh[e] = 0.0;

  const int nJB = rp / JB;
  const int n_items = n * nJB;
  constexpr int ITEMS = MAXACC / JB;
  TC acc[MAXACC];
#pragma unroll
  for (int k = 0; k < MAXACC; ++k) acc[k] = (TC)0;
  TC wacc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) wacc[k] = (TC)0;

  // zero the FP64 Y entries this thread owns (only this thread ever touches them)
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const int it = tid + k * NT;
    if (it < n_items) {
      const int i = it / nJB, jb = it - (it / nJB) * nJB;
#pragma unroll
      for (int c = 0; c < JB; ++c) {
        const int j = jb * JB + c;
        if (j < r) part[r + i + size_t(n) * j] = 0.0;
      }
    }
  }

  const int64_t num_tiles = (prm.p + TS - 1) / TS;
  int since_flush = 0;
  for (int64_t tile = blockIdx.x; tile < num_tiles; tile += gridDim.x) {
    const int64_t s0 = tile * TS;
    const int valid = (int)(prm.p - s0 < TS ? prm.p - s0 : TS);
    __syncthreads();  // the previous tile's phase 2 is done with Vs and Ws
    for (int e = tid; e < TS * n; e += NT) {
      const int s = e / n, i = e - s * n;
      TC v = (TC)0;
      if (s < valid) {
        int64_t row = s0 + s;
        if (prm.idx) {  // sampled rows (Sec. 5): a row outside the storage reads as zero
          row = prm.idx[s0 + s];
          if (row < 0 || row >= prm.rows) {
            if (i == 0) stmf_set_status(prm.status, STMF_EINVAL);
            row = -1;
          }
        }
        if (row >= 0) {
          v = widen<TC>(V[row * ld + i]);
          if (DT == STMF_E4M3) v *= (TC)prm.scale[row];
        }
      }
      Vs[s * vst + i] = v;
    }
    if (tid < TS)
      nus[tid] = tid < valid ? (TC)(prm.nu ? prm.nu[s0 + tid] : prm.nu_uniform) : (TC)0;
    __syncthreads();

    if constexpr (RRF) {
      // phase 1 (range finder): W = the rows of the Gaussian test matrix for these samples
      for (int e = tid; e < TS * rp; e += NT) {
        const int s = e / rp, j = e - (e / rp) * rp;
        TC om = (TC)0;
        if (s < valid && j < r) {
          if constexpr (sizeof(TC) == 4) om = rrf_omega_f32(s0 + s, j, prm.seed);
          else om = (TC)rrf_omega(s0 + s, j, prm.seed);
        }
        Ws[e] = om;
      }
    } else
    // phase 1: z = v_s^T a_j for the thread's sample s and column quads q0, q0 + QG, ...
    {
      const int s = tid % TS;
      const int q0 = tid / TS;  // column quads q0, q0 + QG, ...
      const TC nu_s = nus[s];
      const TC* vrow = Vs + s * vst;
#pragma unroll
      for (int kq = 0; kq < 16 / QG; ++kq) {
        const int q = q0 + QG * kq;
        if (4 * q < rp) {
          TC z0 = 0, z1 = 0, z2 = 0, z3 = 0;
          const TC* acol = As + 4 * q;
          for (int i = 0; i < n; ++i) {
            const TC v = vrow[i];
            const TC* a = acol + i * rp;
            z0 += v * a[0];
            z1 += v * a[1];
            z2 += v * a[2];
            z3 += v * a[3];
          }
          const TC zz[4] = {z0, z1, z2, z3};
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const TC t = ipow(zz[c], d - 1);
            Ws[s * rp + 4 * q + c] = nu_s * t;
            wacc[kq * 4 + c] += nu_s * t * zz[c];
          }
        }
      }
    }
    __syncthreads();

    // phase 2: Y[i][j] += sum_s V[s][i] W[s][j]
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const int it = tid + k * NT;
      if (it < n_items) {
        const int i = it / nJB, jb = it - (it / nJB) * nJB;
        const TC* wcol = Ws + jb * JB;
        for (int s = 0; s < valid; ++s) {
          const TC v = Vs[s * vst + i];
          const TC* w = wcol + s * rp;
#pragma unroll
          for (int c = 0; c < JB; ++c) acc[k * JB + c] += v * w[c];
        }
      }
    }

    ++since_flush;
    const bool last = tile + gridDim.x >= num_tiles;
    if (since_flush == prm.flush_tiles || last) {
      since_flush = 0;
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        const int it = tid + k * NT;
        if (it < n_items) {
          const int i = it / nJB, jb = it - (it / nJB) * nJB;
#pragma unroll
          for (int c = 0; c < JB; ++c) {
            const int j = jb * JB + c;
            if (j < r) part[r + i + size_t(n) * j] += (double)acc[k * JB + c];
            acc[k * JB + c] = (TC)0;
          }
        }
      }
      // w: reduce over the warp's samples, then fold into the warp's FP64 row
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        double x = (double)wacc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) wsh[warp * 16 + k] += x;
        wacc[k] = (TC)0;
      }
    }
  }
  __syncthreads();
  // w_j = sum over the TS / 32 warps that own column quad q0 = (j/4) % QG, slot (j/4) / QG
  for (int j = tid; j < r; j += NT) {
    const int q = j / 4, c = j % 4, q0 = q % QG, kq = q / QG;
    double t = 0.0;
    for (int w = q0 * (TS / 32); w < (q0 + 1) * (TS / 32); ++w) t += wsh[w * 16 + kq * 4 + c];
    part[j] = t;
  }
}

constexpr size_t kSmemMax = 232448;

// Samples per tile: 64, or 32 when a 64-sample tile of the compute type does not fit (FP64 at
// large n). With FP32 compute and n x rp <= NT * MAXACC a 64-sample tile always fits.
template <typename TC>
int tile_of(int n, int rp) {
  return smem_bytes<TC>(n, rp, TS_MAX) <= kSmemMax ? TS_MAX : TS_MAX / 2;
}

template <typename TC, int DT, int JB, bool RRF, int TS>
cudaError_t launch_one(const FgParams& prm, int grid, cudaStream_t s) {
  const size_t smem = smem_bytes<TC>(prm.n, prm.r_pad, TS);
  const cudaError_t e = smem_limit((const void*)fg_simt_kernel<TC, DT, JB, RRF, TS>, kSmemMax);
  if (e != cudaSuccess) return e;
  return launch_kernel(fg_simt_kernel<TC, DT, JB, RRF, TS>, dim3(grid), dim3(NT), smem, s, prm);
}

template <typename TC, int DT, bool RRF, int TS>
cudaError_t launch_ts(const FgParams& prm, int grid, cudaStream_t s) {
  if (prm.r_pad % 16 == 0) return launch_one<TC, DT, 16, RRF, TS>(prm, grid, s);
  if (prm.r_pad % 8 == 0) return launch_one<TC, DT, 8, RRF, TS>(prm, grid, s);
  return launch_one<TC, DT, 4, RRF, TS>(prm, grid, s);
}

template <typename TC, int DT, bool RRF = false>
cudaError_t launch_jb(const FgParams& prm, int grid, cudaStream_t s) {
  if constexpr (sizeof(TC) == 8) {
    if (tile_of<TC>(prm.n, prm.r_pad) != TS_MAX)
      return launch_ts<TC, DT, RRF, TS_MAX / 2>(prm, grid, s);
  }
  return launch_ts<TC, DT, RRF, TS_MAX>(prm, grid, s);
}

// The range finder runs once per fit: one column grouping (JB = 4 divides every padded rank).
template <typename TC, int DT>
cudaError_t launch_rrf(const FgParams& prm, int grid, cudaStream_t s) {
  if constexpr (sizeof(TC) == 8) {
    if (tile_of<TC>(prm.n, prm.r_pad) != TS_MAX)
      return launch_one<TC, DT, 4, true, TS_MAX / 2>(prm, grid, s);
  }
  return launch_one<TC, DT, 4, true, TS_MAX>(prm, grid, s);
}

}  // namespace
}  // namespace stmf
