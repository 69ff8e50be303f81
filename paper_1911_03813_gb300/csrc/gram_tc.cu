// ||X||^2 = nu^T (V^T V)^d nu (Lemma 3.4 applied to X, Sec. 3.3) on the tensor cores, for BF16
// samples.
//
// The sample tiles (128 samples each) are paired over the upper triangle j >= i; the p x p Gram
// matrix is never formed. A CTA keeps two I tiles (i_u = 2m + u, u = 0, 1: 256 samples, K-major)
// in shared memory and streams J blocks of 256 samples (tiles 2b and 2b + 1) past them in K
// chunks of 64 features (32 KB) through a ring of TMA stages. Per chunk and I tile one MMA
// instruction covers 128 x 256 x 16 products:
//   MMA   G_u += V_{i_u} V_{2b, 2b+1}^T    M = 128, N = 256, K = 16 (tcgen05 kind::f16, FP32 TMEM)
//   epi   acc_l += nu_l * w * sum_k nu_k (G_u)_lk^d over each tile j of the block, w = 2 above
//         the diagonal (j > i_u), 1 on it, 0 below it
// The tensor cores share the SM's shared-memory bandwidth with the TMA writes that fill it, and
// both shapes here cut that traffic per product: N = 256 reads A once per 256 columns, and every
// staged chunk feeds the MMAs of both I tiles, so each byte copied in serves 256 rows.
// A work item is (m, chunk of JB blocks); items are ordered chunk-major, so the CTAs running at
// one time share the same J blocks in L2, and JB = 16 blocks (4096 samples) keeps the reload of
// the I tiles (between items) rare.
// TMEM holds the two accumulators G_0, G_1 (256 columns each: all 512), one buffer each: G_0 is
// complete (and handed to the epilogue) when its last chunk's MMAs are issued, so the epilogue
// drains it while the MMAs of G_1 run, and drains G_1 while the next block's first chunk runs
// into G_0. Epilogue sums are compensated FP32 (the FP64 pipe is slow on this part) and are
// combined in FP64 once per CTA; CTA totals are summed in index order (deterministic).
//
// Warp roles: warp 0 TMA producer, warp 1 TMEM allocator and MMA issuer, warps 2-17 epilogue
// (four column groups of 64 columns, groups 0-1 on tile 2b and 2-3 on tile 2b + 1; thread = TMEM
// lane = sample of the I tile). Every wait is bounded; a wait that runs out sets STMF_ETIMEOUT and
// the CTA winds down.
#include <cuda.h>
#include <cuda_bf16.h>

#include "stmf_internal.h"
#include "tc_common.cuh"

namespace stmf {
namespace {

constexpr int TM = 128;
constexpr int REG_BYTES = TM * 128;         // 128 samples x 64 features of BF16 (one TMA box)
constexpr int STAGE_BYTES = 2 * REG_BYTES;  // one K chunk of a J block (256 samples)
constexpr int JB = 16;                      // J blocks (of two tiles) per work item
constexpr int CG = 4;                       // epilogue column groups
constexpr int NEPI = 128 * CG;
constexpr int NTHREADS = 64 + NEPI;
constexpr int MAX_STAGES = 4;
constexpr int TMEM_COLS = 512;              // G_0, G_1: 256 columns each
// dynamic shared memory of at least this much keeps one CTA per SM (the CTA takes all of TMEM)
constexpr int MIN_SMEM = 120 * 1024;
constexpr long long WAIT_LIMIT = 4000000000LL;

struct GramTcParams {
  const double* nu;
  double nu_uniform;
  double* partials;
  long long p;
  int n, d, nload, stages, smem_bytes;
  long long T, items;
  int32_t* status;
};

// TB = ceil(T / 2) blocks of two tiles and as many I pairs. Items of chunk row c (blocks
// [JB c, min(JB (c + 1), TB))): the I pairs m <= the row's last block. Every row but the last is
// full (JB (c + 1) items), so row c starts at item JB c (c + 1) / 2; the last row holds all TB.
__host__ __device__ __forceinline__ long long row_start(long long c) {
  return (long long)JB * c * (c + 1) / 2;
}

__host__ __device__ __forceinline__ long long total_items(long long T) {
  const long long TB = (T + 1) / 2;
  const long long nrows = (TB + JB - 1) / JB;
  return row_start(nrows - 1) + TB;
}

__host__ __device__ __forceinline__ void item_of(long long k, long long T, long long& c,
                                                 long long& m) {
  const long long TB = (T + 1) / 2;
  const long long nrows = (TB + JB - 1) / JB;
  long long lo = 0, hi = nrows - 1;
  while (lo < hi) {  // largest c with row_start(c) <= k
    const long long mid = (lo + hi + 1) / 2;
    if (row_start(mid) <= k) lo = mid;
    else hi = mid - 1;
  }
  c = lo;
  m = k - row_start(lo);
}

// J blocks [b0, b1) of item (c, m)
__host__ __device__ __forceinline__ void brange(long long c, long long m, long long T,
                                                long long& b0, long long& b1) {
  const long long TB = (T + 1) / 2;
  const long long c0 = (long long)JB * c;
  b0 = m > c0 ? m : c0;
  b1 = c0 + JB < TB ? c0 + JB : TB;
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// x^DP by repeated squaring (DP known at compile time: 2..8)
template <int DP>
__device__ __forceinline__ float powd(float x) {
  if constexpr (DP == 1) return x;
  else if constexpr (DP % 2 == 0) {
    const float h = powd<DP / 2>(x);
    return h * h;
  } else {
    return x * powd<DP - 1>(x);
  }
}

template <int DP>
__global__ void __launch_bounds__(NTHREADS, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap tmap, const GramTcParams prm) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw = tc::smem_addr(smem_raw);
  unsigned char* base = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const int S = prm.stages, nload = prm.nload;
  const uint32_t itile_bytes = uint32_t(nload) * REG_BYTES;
  unsigned char* sA = base;                          // I tile u: regions [u nload, (u+1) nload)
  unsigned char* sB = sA + 2 * size_t(itile_bytes);  // S stages of one K chunk of a J block
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + size_t(S) * STAGE_BYTES);
  uint64_t* a_full = bars;
  uint64_t* a_empty = bars + 1;
  uint64_t* b_full = bars + 2;
  uint64_t* b_empty = b_full + S;
  uint64_t* d_full = b_empty + S;  // [2] G_u complete
  uint64_t* d_empty = d_full + 2;  // [2] G_u read by the epilogue
  uint64_t* mma_done = d_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  double* red = reinterpret_cast<double*>(mma_done + 2);  // NEPI / 32 warps

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    tc::mbar_init(a_full, 1);
    tc::mbar_init(a_empty, 1);
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&b_full[s], 1);
      tc::mbar_init(&b_empty[s], 1);
    }
    for (int u = 0; u < 2; ++u) {
      tc::mbar_init(&d_full[u], 1);
      tc::mbar_init(&d_empty[u], NEPI / 32);
    }
    tc::mbar_init(mma_done, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0 && lane == 0) tc::prefetch_tmap(&tmap);
  if (warp == 1) tc::tmem_alloc(tmem_slot, TMEM_COLS);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int* abortv = abort_flag;
  int no_abort = 0;
  auto fail = [&]() {
    stmf_set_status(prm.status, STMF_ETIMEOUT);
    *abortv = 1;
  };
  const long long T = prm.T;

  if (warp == 0) {
    // ------------------------------------------------------------------ TMA producer
    if (lane == 0) {
      long long nitem = 0, bs = 0;
      bool ok = true;
      for (long long k = blockIdx.x; k < prm.items && ok; k += gridDim.x, ++nitem) {
        long long c, m, b0, b1;
        item_of(k, T, c, m);
        brange(c, m, T, b0, b1);
        const int nI = 2 * m + 1 < T ? 2 : 1;  // a last, odd I tile has no partner
        if (!tc::mbar_wait(a_empty, uint32_t(nitem & 1) ^ 1u, abortv, WAIT_LIMIT)) {
          ok = false;
          break;
        }
        tc::mbar_arrive_expect_tx(a_full, uint32_t(nI) * itile_bytes);
        for (int u = 0; u < nI; ++u)
          for (int g = 0; g < nload; ++g)
            tc::tma_load_2d(sA + size_t(u * nload + g) * REG_BYTES, &tmap, g * 64,
                            (int32_t)((2 * m + u) * TM), a_full);
        for (long long b = b0; b < b1 && ok; ++b)
          for (int g = 0; g < nload; ++g, ++bs) {
            const int st = int(bs % S);
            if (!tc::mbar_wait(&b_empty[st], uint32_t((bs / S) & 1) ^ 1u, abortv, WAIT_LIMIT)) {
              ok = false;
              break;
            }
            // tiles 2b and 2b + 1 (the second may lie past the last tile: zero-filled)
            tc::mbar_arrive_expect_tx(&b_full[st], STAGE_BYTES);
            for (int h = 0; h < 2; ++h)
              tc::tma_load_2d(sB + size_t(st) * STAGE_BYTES + size_t(h) * REG_BYTES, &tmap,
                              g * 64, (int32_t)((2 * b + h) * TM), &b_full[st]);
          }
      }
      if (!ok) fail();
      // drain: the last A load and the last load of each B stage
      if (nitem > 0) tc::mbar_wait(a_full, uint32_t((nitem - 1) & 1), &no_abort, WAIT_LIMIT);
      for (long long q = bs > S ? bs - S : 0; q < bs; ++q)
        tc::mbar_wait(&b_full[q % S], uint32_t((q / S) & 1), &no_abort, WAIT_LIMIT);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16(128, 256, 0, 0);
      // shared-memory descriptors are linear in the operand address (16-byte units in the low
      // bits; every address here is below 256 KB): one base per operand plus (offset >> 4)
      const uint64_t adesc0 = tc::sdesc_sw128(tc::smem_addr(sA), 16, 1024);
      const uint64_t bdesc0 = tc::sdesc_sw128(tc::smem_addr(sB), 16, 1024);
      long long nitem = 0, bs = 0;
      long long du[2] = {0, 0};  // blocks in which G_u was used
      bool ok = true;
      for (long long k = blockIdx.x; k < prm.items && ok; k += gridDim.x, ++nitem) {
        long long c, m, b0, b1;
        item_of(k, T, c, m);
        brange(c, m, T, b0, b1);
        const int nI = 2 * m + 1 < T ? 2 : 1;
        if (!tc::mbar_wait(a_full, uint32_t(nitem & 1), abortv, WAIT_LIMIT)) {
          ok = false;
          break;
        }
        for (long long b = b0; b < b1 && ok; ++b) {
          for (int g = 0; g < nload && ok; ++g, ++bs) {
            const int st = int(bs % S);
            if (!tc::mbar_wait(&b_full[st], uint32_t((bs / S) & 1), abortv, WAIT_LIMIT)) {
              ok = false;
              break;
            }
            tc::tc_fence_after();
            const uint64_t bd = bdesc0 + uint64_t((uint32_t(st) * STAGE_BYTES) >> 4);
            for (int u = 0; u < nI; ++u) {
              if (g == 0) {  // the epilogue has read G_u of its previous use
                if (!tc::mbar_wait(&d_empty[u], uint32_t(du[u] & 1) ^ 1u, abortv, WAIT_LIMIT)) {
                  ok = false;
                  break;
                }
                tc::tc_fence_after();
              }
              const uint64_t ad = adesc0 + uint64_t((uint32_t(u * nload + g) * REG_BYTES) >> 4);
              const uint32_t dG = tmem + uint32_t(u) * 256;
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                tc::mma_bf16(dG, ad + uint64_t((kk * 32) >> 4), bd + uint64_t((kk * 32) >> 4),
                             idesc, (g | kk) ? 1u : 0u);
              if (g == nload - 1) tc::mma_commit(&d_full[u]);  // G_u of block b complete
            }
            if (!ok) break;
            tc::mma_commit(&b_empty[st]);
          }
          for (int u = 0; u < nI; ++u) ++du[u];
        }
        tc::mma_commit(a_empty);  // the I tiles may be replaced once these MMAs are done
      }
      if (!ok) fail();
      tc::mma_commit(mma_done);
      tc::mbar_wait(mma_done, 0, &no_abort, WAIT_LIMIT);
    }
  } else {
    // ------------------------------------------------------------------ epilogue
    const int ew = warp - 2;
    const int cg = ew >> 2;                 // column group: columns [64 cg, 64 cg + 64)
    const int q = warp & 3;                 // TMEM lane quarter
    const int L = 32 * q + lane;            // sample of each I tile
    const uint32_t lane_off = uint32_t(32 * q) << 16;
    float acc_s = 0.f, acc_c = 0.f;
    long long du[2] = {0, 0};  // blocks in which G_u was used
    bool ok = true;
    const bool uniform = prm.nu == nullptr;
    for (long long k = blockIdx.x; k < prm.items && ok; k += gridDim.x) {
      long long c, m, b0, b1;
      item_of(k, T, c, m);
      brange(c, m, T, b0, b1);
      const int nI = 2 * m + 1 < T ? 2 : 1;
      float nu_l[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const long long sl = (2 * m + u) * TM + L;
        nu_l[u] = sl < prm.p ? (uniform ? 1.f : (float)prm.nu[sl]) : 0.f;
      }
      for (long long b = b0; b < b1 && ok; ++b) {
        const long long j = 2 * b + (cg >> 1);  // this group's tile of the block
        const long long k0 = j * TM + 64 * (cg & 1);  // its first sample
        for (int u = 0; u < nI; ++u) {
          if (!tc::mbar_wait(&d_full[u], uint32_t(du[u]++ & 1), abortv, WAIT_LIMIT)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          float g0[32], g1[32];
          const uint32_t col = tmem + uint32_t(u) * 256 + 64 * cg + lane_off;
          tc::tmem_ld32(col, g0);
          tc::tmem_ld32(col + 32, g1);
          tc::tmem_ld_wait();
          tc::tc_fence_before();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&d_empty[u]);
          const long long i = 2 * m + u;
          if (j < i) continue;  // below the diagonal
          float row = 0.f;
          if (uniform) {
            // samples beyond p are zero-filled by TMA, so their G entries (and powers) vanish
#pragma unroll
            for (int e = 0; e < 32; ++e) row += powd<DP>(g0[e]) + powd<DP>(g1[e]);
          } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              const float n0 = (k0 + e) < prm.p ? (float)prm.nu[k0 + e] : 0.f;
              const float n1 = (k0 + 32 + e) < prm.p ? (float)prm.nu[k0 + 32 + e] : 0.f;
              row += n0 * powd<DP>(g0[e]) + n1 * powd<DP>(g1[e]);
            }
          }
          kahan_add(acc_s, acc_c, (j == i ? 1.f : 2.f) * nu_l[u] * row);
        }
      }
    }
    if (!ok) fail();
    double x = (double)acc_s - (double)acc_c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[ew] = x;
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < NEPI / 32; ++w) t += red[w];
    const double scale = prm.nu ? 1.0 : prm.nu_uniform * prm.nu_uniform;
    prm.partials[blockIdx.x] = t * scale;
  }
  if (warp == 1) tc::tmem_dealloc(tmem, TMEM_COLS);
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  }
  return fn;
}

template <int DP>
cudaError_t launch_d(const CUtensorMap& tmap, const GramTcParams& prm, int grid, cudaStream_t s) {
  const cudaError_t e = smem_limit((const void*)gram_tc_kernel<DP>, 232448);
  if (e != cudaSuccess) return e;
  gram_tc_kernel<DP><<<grid, NTHREADS, prm.smem_bytes, s>>>(tmap, prm);
  return cudaGetLastError();
}

int stages_for(int n) {
  const int nload = (n + 63) / 64;
  const int S = (232448 - 2048 - 2 * nload * REG_BYTES) / STAGE_BYTES;
  return S > MAX_STAGES ? MAX_STAGES : S;
}

}  // namespace

bool gram_tc_supported(int dtype, int n, int64_t p) {
  return dtype == STMF_BF16 && n >= 1 && n <= 256 && p < (int64_t(1) << 31) - 2 * TM &&
         encoder() != nullptr && stages_for(n) >= 3;
}

int gram_tc_grid(int64_t p, int num_sms) {
  const long long items = total_items((p + TM - 1) / TM);
  return (int)(items < num_sms ? items : num_sms);
}

cudaError_t gram_tc_launch(const GramParams& gp, int grid, cudaStream_t s) {
  EncodeFn enc = encoder();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap tmap;
  const cuuint64_t dims[2] = {(cuuint64_t)gp.n, (cuuint64_t)gp.p};
  const cuuint64_t strides[1] = {(cuuint64_t)gp.ld * 2};
  const cuuint32_t box[2] = {64, TM};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(gp.V), dims, strides, box,
          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  GramTcParams prm{};
  prm.nu = gp.nu;
  prm.nu_uniform = gp.nu_uniform;
  prm.partials = gp.partials;
  prm.p = gp.p;
  prm.n = gp.n;
  prm.d = gp.d;
  prm.nload = (gp.n + 63) / 64;
  prm.stages = stages_for(gp.n);
  prm.T = (gp.p + TM - 1) / TM;
  prm.items = total_items(prm.T);
  prm.status = gp.status;
  const int need = 2 * prm.nload * REG_BYTES + prm.stages * STAGE_BYTES + 1024 /*align*/ +
                   1024 /*barriers*/;
  prm.smem_bytes = need > MIN_SMEM ? need : MIN_SMEM;
  switch (gp.d) {
    case 2: return launch_d<2>(tmap, prm, grid, s);
    case 3: return launch_d<3>(tmap, prm, grid, s);
    case 4: return launch_d<4>(tmap, prm, grid, s);
    case 5: return launch_d<5>(tmap, prm, grid, s);
    case 6: return launch_d<6>(tmap, prm, grid, s);
    case 7: return launch_d<7>(tmap, prm, grid, s);
    case 8: return launch_d<8>(tmap, prm, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace stmf
