// Fused pass over FP32 samples on the CUDA cores, register-blocked (r <= 16, n <= 256).
//
// Per persistent block and over that block's tiles of TS samples it accumulates the partial
// sums of Alg. 2's Y (Lemma 3.3, eq. Y) and of Lemma 3.5:
//     Y_part = sum_l nu_l (v_l^T A)^{d-1} v_l,      w_part_j = sum_l nu_l (v_l^T a_j)^d,
// reading every sample from HBM once. The arithmetic is 2 n r FMA per sample per product (Z = V A
// and Y += V^T W); at n = 256, r = 16 that is above the HBM time of the FP32 samples, so the
// kernel is laid out for the FP32 pipe: every thread computes a 4 x 4 register block of its
// product with two 16-byte shared-memory loads per 16 FMA (warp-wide, one of the two is a
// broadcast), and the next tile streams into the other shared-memory buffer with cp.async while
// the current one is used.
//
// Per tile (NW warps; SH = TS / 32 groups of 32 samples, KS = NW / SH feature splits):
//   phase 1  Z = V_t A          warp w: samples [32 (w % SH), +32), features of split w / SH;
//                               lane: samples g, g+8, g+16, g+24 (g = lane / 4) x columns
//                               4 (lane % 4) .. +3; the KS split partials go to shared memory
//   weights  z = sum of the KS split partials (fixed order); W = nu z^{d-1}; w += nu z^d
//   phase 2  Y += V_t^T W       warp: 32 features (lane: 4 features x 4 columns) over its share
//                               of the tile's samples (warps split the samples when n is small)
// Each phase ends at a block barrier. The pass runs 8 warps and two blocks per SM, so that one
// block's barrier waits overlap the other block's arithmetic (measured against 64-sample tiles
// with 16 warps and one block per SM: 8.6 against 9.4 ms at n = 256, r = 16, p = 2^24, and 0.80
// against 1.13 ms at n = 100, r = 10, p = 2.5e6). The tile grows as n shrinks (32 samples for
// n > 128, 64 for n > 64, 128 otherwise), so that each barrier covers the same work per thread.
// Y is folded from FP32 into the block's FP64 partial and w into FP64 registers every
// 64 flush_tiles samples, in a fixed order (results reproducible bit for bit).
#include <cuda_runtime.h>

#include "stmf_internal.h"

namespace stmf {
namespace {

constexpr int RC = 16;  // columns of A handled (r <= 16, zero-padded)

// TS samples per tile, NW warps per block, MB blocks per SM, for n <= NMAX
template <int TS_, int NW_, int MB_, int NMAX_>
struct Cfg {
  static constexpr int NMAX = NMAX_;
  static constexpr int TS = TS_;
  static constexpr int NW = NW_;
  static constexpr int MB = MB_;
  static constexpr int NT = 32 * NW;
  static constexpr int SH = TS / 32;         // phase 1: groups of 32 samples
  static constexpr int KS = NW / SH;         // phase 1: K splits
  static constexpr int EPT = TS * RC / NT;   // weights: (sample, column) entries per thread
  static constexpr int CPT = RC / EPT;       // weights: threads per sample
  static_assert(KS * SH == NW && KS >= 1, "phase 1 splits the features KS ways");
  static_assert(NT == TS * CPT, "one weights thread per (sample, column group)");
};
using CfgN256 = Cfg<32, 8, 2, 256>;   // 128 < n <= 256
using CfgN128 = Cfg<64, 8, 2, 128>;   //  64 < n <= 128
using CfgN64 = Cfg<128, 8, 2, 64>;    //       n <= 64

struct Shape {
  int np;      // features padded to a multiple of 32 (each K split a multiple of 4)
  int pitch;   // floats between consecutive samples in shared memory (np + 4: odd 16-byte count)
  int kq;      // features per K split in phase 1 (np / KS)
  int p2;      // feature warps in phase 2 (power of two >= ceil(np / 32))
  int ss;      // sample splits in phase 2 (NW / p2)
};

template <class C>
Shape shape_of(int n) {
  Shape s;
  s.np = (n + 31) / 32 * 32;
  s.pitch = s.np + 4;
  s.kq = s.np / C::KS;
  const int nfb = (s.np + 31) / 32;
  s.p2 = 1;
  while (s.p2 < nfb) s.p2 <<= 1;
  s.ss = C::NW / s.p2;
  return s;
}

template <class C>
size_t smem_of(const Shape& s) {
  constexpr int TS = C::TS;
  return sizeof(float) * (2 * size_t(TS) * s.pitch  // V tiles (double buffer)
                          + size_t(s.np) * RC       // A
                          + C::KS * TS * RC         // K-split partials of Z (reused at the end)
                          + TS * RC)                // W
         + sizeof(double) * 2 * TS;                 // nu (double buffer)
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

__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ float ipow_f(float z, int e) {
  float t = 1.f;
  for (int k = 0; k < e; ++k) t *= z;
  return t;
}

// Stage tile `tile` (rows s0 .. s0 + TS, or the gathered rows idx[s0 ..]) into buffer `buf`:
// features past n and rows past p (or outside the storage) are zero-filled by cp.async. Thread
// t copies the 16-byte chunks e = t, t + NT, ... of the tile (row e / cpr, chunk e % cpr), walked
// by increments (ds, dc) = (NT / cpr, NT % cpr) from (s, c) = (t / cpr, t % cpr).
struct StageWalk {
  int s, c, ds, dc, cpr;
};

template <class C>
__device__ __forceinline__ void stage_tile(const FgParams& prm, const Shape& sh, const StageWalk& w,
                                           float* Vbuf, double* nubuf, int64_t tile) {
  constexpr int TS = C::TS;
  const float* V = static_cast<const float*>(prm.V);
  const int64_t s0 = tile * TS;
  int s = w.s, c = w.c;
  for (; s < TS; s += w.ds) {
    int64_t row = s0 + s;
    bool ok = row < prm.p;
    if (ok && prm.idx) {
      row = prm.idx[row];
      if (row < 0 || row >= prm.rows) {
        if (c == 0) stmf_set_status(prm.status, STMF_EINVAL);
        ok = false;
      }
    }
    const int left = prm.n - 4 * c;
    const uint32_t bytes = (ok && left > 0) ? uint32_t(left >= 4 ? 16 : 4 * left) : 0u;
    const float* src = bytes ? V + row * prm.ld + 4 * c : V;
    cp_async16(smem_u32(Vbuf + s * sh.pitch + 4 * c), src, bytes);
    c += w.dc;
    if (c >= w.cpr) {
      c -= w.cpr;
      ++s;
    }
  }
  if (threadIdx.x < TS) {
    const int64_t row = s0 + threadIdx.x;
    if (prm.nu) {
      const bool ok = row < prm.p;
      cp_async8(smem_u32(nubuf + threadIdx.x), ok ? prm.nu + row : prm.nu, ok ? 8u : 0u);
    } else {
      nubuf[threadIdx.x] = row < prm.p ? prm.nu_uniform : 0.0;
    }
  }
}

template <class C>
__global__ void __launch_bounds__(C::NT, C::MB) fg_f32_kernel(const FgParams prm, const Shape sh) {
  constexpr int TS = C::TS, NT = C::NT, SH = C::SH, EPT = C::EPT, CPT = C::CPT;
  if (prm.skip && *prm.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Vs = reinterpret_cast<float*>(smem_raw);
  float* As = Vs + 2 * TS * sh.pitch;
  float* Zp = As + sh.np * RC;
  float* Ws = Zp + C::KS * TS * RC;
  double* nus = reinterpret_cast<double*>(Ws + TS * RC);

  const int n = prm.n, r = prm.r, d = prm.d;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // A (FP64, n x r column-major) -> As[k][j] in FP32, zero past n and r
  for (int e = tid; e < sh.np * RC; e += NT) {
    const int k = e / RC, j = e - k * RC;
    As[e] = (k < n && j < r) ? (float)prm.A[k + size_t(n) * j] : 0.f;
  }

  const int64_t num_tiles = (prm.p + TS - 1) / TS;
  const int my_tiles = (int)((num_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
  StageWalk walk;
  walk.cpr = sh.np / 4;
  walk.s = tid / walk.cpr;
  walk.c = tid - walk.s * walk.cpr;
  walk.ds = NT / walk.cpr;
  walk.dc = NT - walk.ds * walk.cpr;

  // phase 1 roles
  const int h1 = warp % SH, q1 = warp / SH;
  const int g1 = lane >> 2, cg = lane & 3;
  // weights role: sample sw, columns EPT cw .. EPT cw + EPT - 1
  const int sw = tid / CPT, cw = tid % CPT;
  // phase 2 roles
  const int fb2 = warp % sh.p2, sp2 = warp / sh.p2;
  const int i2 = 32 * fb2 + 4 * (lane >> 2);  // first of the thread's 4 features
  const bool act2 = 32 * fb2 < sh.np;
  const int sb2 = sp2 * (TS / sh.ss), se2 = sb2 + TS / sh.ss;

  double* part = prm.partials + size_t(blockIdx.x) * (size_t(r) + size_t(n) * r);
  float2 yacc[4][2];  // (feature f, columns 4 cg + 2 c, + 1), packed FP32 FMA
  float wacc[EPT];
  double wd[EPT];
#pragma unroll
  for (int a = 0; a < EPT; ++a) {
    wacc[a] = 0.f;
    wd[a] = 0.0;
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) yacc[a][0] = yacc[a][1] = make_float2(0.f, 0.f);
  bool first_flush = true;

  const int flush_every = (prm.flush_tiles * 64 + TS - 1) / TS;  // every 64 flush_tiles samples
  if (my_tiles > 0) stage_tile<C>(prm, sh, walk, Vs, nus, blockIdx.x);
  cp_async_commit();
  int since_flush = 0;
  for (int it = 0; it < my_tiles; ++it) {
    const int buf = it & 1;
    const float* Vt = Vs + buf * TS * sh.pitch;
    if (it + 1 < my_tiles)
      stage_tile<C>(prm, sh, walk, Vs + (buf ^ 1) * TS * sh.pitch, nus + (buf ^ 1) * TS,
                 blockIdx.x + int64_t(it + 1) * gridDim.x);
    cp_async_commit();
    cp_async_wait<1>();  // this tile's copies (the older group) have landed
    __syncthreads();

    // ---------------------------------------------------------------- phase 1: quarter of Z
    {
      float2 acc[4][2];  // (sample j, columns 4 cg + 2 c, + 1), packed FP32 FMA
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[j][0] = acc[j][1] = make_float2(0.f, 0.f);
      const float* vrow = Vt + (32 * h1 + g1) * sh.pitch;
      const float* arow = As + 4 * cg;
      const int kb = q1 * sh.kq, ke = kb + sh.kq;
#pragma unroll 4
      for (int k0 = kb; k0 < ke; k0 += 4) {
        float4 a[4], v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) a[t] = *reinterpret_cast<const float4*>(arow + (k0 + t) * RC);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          v[j] = *reinterpret_cast<const float4*>(vrow + 8 * j * sh.pitch + k0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float vv[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const float2 vt = make_float2(vv[t], vv[t]);
            acc[j][0] = __ffma2_rn(vt, make_float2(a[t].x, a[t].y), acc[j][0]);
            acc[j][1] = __ffma2_rn(vt, make_float2(a[t].z, a[t].w), acc[j][1]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
        *reinterpret_cast<float4*>(Zp + (q1 * TS + 32 * h1 + g1 + 8 * j) * RC + 4 * cg) =
            make_float4(acc[j][0].x, acc[j][0].y, acc[j][1].x, acc[j][1].y);
    }
    __syncthreads();

    // ---------------------------------------------------------------- weights
    {
      float z[EPT];
#pragma unroll
      for (int c = 0; c < EPT; ++c) z[c] = 0.f;
#pragma unroll
      for (int q = 0; q < C::KS; ++q) {  // K splits added in order
        const float* zp = Zp + (q * TS + sw) * RC + EPT * cw;
#pragma unroll
        for (int c = 0; c < EPT; ++c) z[c] += zp[c];
      }
      const float nu = (float)nus[buf * TS + sw];
      float wv[EPT];
#pragma unroll
      for (int c = 0; c < EPT; ++c) {
        wv[c] = nu * ipow_f(z[c], d - 1);
        wacc[c] = fmaf(wv[c], z[c], wacc[c]);
        Ws[sw * RC + EPT * cw + c] = wv[c];
      }
    }
    __syncthreads();

    // ---------------------------------------------------------------- phase 2: Y += V_t^T W
    if (act2) {
      const float* wcol = Ws + 4 * cg;
#pragma unroll 4
      for (int s = sb2; s < se2; ++s) {
        const float4 v = *reinterpret_cast<const float4*>(Vt + s * sh.pitch + i2);
        const float4 w = *reinterpret_cast<const float4*>(wcol + s * RC);
        const float vv[4] = {v.x, v.y, v.z, v.w};
        const float2 w01 = make_float2(w.x, w.y), w23 = make_float2(w.z, w.w);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const float2 vf = make_float2(vv[f], vv[f]);
          yacc[f][0] = __ffma2_rn(vf, w01, yacc[f][0]);
          yacc[f][1] = __ffma2_rn(vf, w23, yacc[f][1]);
        }
      }
    }
    if (++since_flush == flush_every || it == my_tiles - 1) {
      since_flush = 0;
#pragma unroll
      for (int a = 0; a < EPT; ++a) {
        wd[a] += (double)wacc[a];
        wacc[a] = 0.f;
      }
      // fold Y into the block's FP64 partial (its entries belong to this block alone); the
      // sample splits add in split order, the first fold of split 0 initialises the entries
      for (int sp = 0; sp < sh.ss; ++sp) {
        if (act2 && sp2 == sp) {
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            const int i = i2 + f;
            const float yv[4] = {yacc[f][0].x, yacc[f][0].y, yacc[f][1].x, yacc[f][1].y};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const int j = 4 * cg + c;
              if (i < n && j < r) {
                double* dst = part + r + i + size_t(n) * j;
                *dst = (first_flush && sp == 0) ? (double)yv[c] : *dst + (double)yv[c];
              }
            }
            yacc[f][0] = yacc[f][1] = make_float2(0.f, 0.f);
          }
        }
        if (sh.ss > 1) __syncthreads();
      }
      first_flush = false;
    }
    __syncthreads();  // buffer `buf` and Zp/Ws are free for the next tile's copies and phases
  }
  cp_async_wait<0>();

  // ------------------------------------------------------------------ block partials
  // w: per column, the TS sample slots summed in slot order
  double* red = reinterpret_cast<double*>(Zp);  // NT x EPT doubles fit in the Z partials
#pragma unroll
  for (int c = 0; c < EPT; ++c) red[tid * EPT + c] = wd[c];
  __syncthreads();
  if (tid < r) {
    const int cgj = tid / EPT, c = tid % EPT;
    double s = 0.0;
    for (int q = 0; q < TS; ++q) s += red[(q * CPT + cgj) * EPT + c];
    part[tid] = s;
  }
}

}  // namespace

bool fg_f32_supported(int dtype, int n, int r) {
  return dtype == STMF_F32 && n >= 1 && n <= 256 && r >= 1 && r <= RC;
}

namespace {

template <class C>
int grid_of(int64_t p, int num_sms) {
  // C::MB persistent blocks per SM (shared memory and registers)
  const int64_t tiles = (p + C::TS - 1) / C::TS;
  int64_t grid = int64_t(num_sms) * C::MB;
  if (grid > tiles) grid = tiles;
  return (int)(grid < 1 ? 1 : grid);
}

template <class C>
cudaError_t launch_cfg(const FgParams& prm, int grid, cudaStream_t s) {
  const Shape sh = shape_of<C>(prm.n);
  const size_t smem = smem_of<C>(sh);
  const cudaError_t e = smem_limit((const void*)fg_f32_kernel<C>, int(smem_of<C>(shape_of<C>(C::NMAX))));
  if (e != cudaSuccess) return e;
  return launch_kernel(fg_f32_kernel<C>, dim3(grid), dim3(C::NT), smem, s, prm, sh);
}

}  // namespace

int fg_f32_grid(int n, int64_t p, int num_sms) {
  return n > 128  ? grid_of<CfgN256>(p, num_sms)
         : n > 64 ? grid_of<CfgN128>(p, num_sms)
                  : grid_of<CfgN64>(p, num_sms);
}

cudaError_t fg_f32_launch(const FgParams& prm, int grid, cudaStream_t s) {
  return prm.n > 128  ? launch_cfg<CfgN256>(prm, grid, s)
         : prm.n > 64 ? launch_cfg<CfgN128>(prm, grid, s)
                      : launch_cfg<CfgN64>(prm, grid, s);
}

}  // namespace stmf
