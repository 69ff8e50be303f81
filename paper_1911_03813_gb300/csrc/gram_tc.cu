// ||X||^2 = nu^T (V^T V)^d nu (Lemma 3.4 applied to X, Sec. 3.3) on the tensor cores, for BF16
// samples.
//
// The sample tiles (128 samples each) are paired over the upper triangle j >= i; the p x p Gram
// matrix is never formed. A work item is (i, J-chunk): the A operand (tile i, 128 x n, K-major)
// stays in shared memory while the chunk's J tiles (up to JC tiles of 128 samples) stream through
// a TMA ring. Items are ordered chunk-major, so the CTAs running at one time share the same J
// tiles in L2. Per pair:
//   MMA   G = V_i V_j^T                 M = 128, N = 128, K = n (tcgen05 kind::f16, FP32 in TMEM)
//   epi   acc_l += nu_l * w_ij * sum_k nu_k G_lk^d,   w_ij = 1 on the diagonal tile, 2 above it
// with a double-buffered TMEM accumulator so the epilogue of one pair overlaps the MMAs of the
// next. Epilogue sums are compensated FP32 (the FP64 pipe is slow on this part) and are combined
// in FP64 once per CTA; CTA totals are summed in index order (deterministic).
//
// Warp roles: warp 0 TMA producer, warp 1 TMEM allocator and MMA issuer, warps 2-17 epilogue
// (four column groups of 32 columns; thread = TMEM lane = sample of tile i). Every wait is
// bounded; a wait that runs out sets STMF_ETIMEOUT and the CTA winds down.
#include <cuda.h>
#include <cuda_bf16.h>

#include "stmf_internal.h"
#include "tc_common.cuh"

namespace stmf {
namespace {

constexpr int TM = 128;
constexpr int REG_BYTES = TM * 128;   // 128 samples x 64 features of BF16
constexpr int JC = 8;                 // J tiles per work item
constexpr int CG = 4;                 // epilogue column groups
constexpr int NEPI = 128 * CG;
constexpr int NTHREADS = 64 + NEPI;
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

// first item of chunk row jc: rows hold min(T, JC (q + 1)) items
__device__ __forceinline__ long long row_start(long long jc, long long T) {
  const long long q0 = T / JC;  // rows with JC (q + 1) <= T
  if (jc <= q0) return (long long)JC * jc * (jc + 1) / 2;
  return (long long)JC * q0 * (q0 + 1) / 2 + (jc - q0) * T;
}

__device__ __forceinline__ void item_of(long long k, long long T, long long& jc, long long& i) {
  const long long nrows = (T + JC - 1) / JC;
  long long lo = 0, hi = nrows - 1;
  while (lo < hi) {  // largest jc with row_start(jc) <= k
    const long long mid = (lo + hi + 1) / 2;
    if (row_start(mid, T) <= k) lo = mid;
    else hi = mid - 1;
  }
  jc = lo;
  i = k - row_start(lo, T);
}

__device__ __forceinline__ void pairs_of(long long jc, long long i, long long T, long long& j0,
                                         long long& j1) {
  const long long c0 = (long long)JC * jc;
  j0 = i > c0 ? i : c0;
  j1 = c0 + JC < T ? c0 + JC : T;
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
  const int S = prm.stages, nload = prm.nload, n = prm.n;
  const uint32_t tile_bytes = uint32_t(nload) * REG_BYTES;
  unsigned char* sA = base;
  unsigned char* sB = sA + tile_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + size_t(S) * tile_bytes);
  uint64_t* a_full = bars;
  uint64_t* a_empty = bars + 1;
  uint64_t* b_full = bars + 2;
  uint64_t* b_empty = b_full + S;
  uint64_t* d_full = b_empty + S;
  uint64_t* d_empty = d_full + 2;
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
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&d_full[b], 1);
      tc::mbar_init(&d_empty[b], NEPI / 32);
    }
    tc::mbar_init(mma_done, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0 && lane == 0) tc::prefetch_tmap(&tmap);
  if (warp == 1) tc::tmem_alloc(tmem_slot, 256);
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
      long long nitem = 0, gp = 0;
      bool ok = true;
      for (long long k = blockIdx.x; k < prm.items && ok; k += gridDim.x, ++nitem) {
        long long jc, i, j0, j1;
        item_of(k, T, jc, i);
        pairs_of(jc, i, T, j0, j1);
        if (!tc::mbar_wait(a_empty, uint32_t(nitem & 1) ^ 1u, abortv, WAIT_LIMIT)) {
          ok = false;
          break;
        }
        tc::mbar_arrive_expect_tx(a_full, tile_bytes);
        for (int g = 0; g < nload; ++g)
          tc::tma_load_2d(sA + size_t(g) * REG_BYTES, &tmap, g * 64, (int32_t)(i * TM), a_full);
        for (long long j = j0; j < j1; ++j, ++gp) {
          const int st = int(gp % S);
          if (!tc::mbar_wait(&b_empty[st], uint32_t((gp / S) & 1) ^ 1u, abortv, WAIT_LIMIT)) {
            ok = false;
            break;
          }
          tc::mbar_arrive_expect_tx(&b_full[st], tile_bytes);
          for (int g = 0; g < nload; ++g)
            tc::tma_load_2d(sB + size_t(st) * tile_bytes + size_t(g) * REG_BYTES, &tmap, g * 64,
                            (int32_t)(j * TM), &b_full[st]);
        }
      }
      if (!ok) fail();
      // drain: the last A load and the last load of each B stage
      if (nitem > 0) tc::mbar_wait(a_full, uint32_t((nitem - 1) & 1), &no_abort, WAIT_LIMIT);
      for (long long q = gp > S ? gp - S : 0; q < gp; ++q)
        tc::mbar_wait(&b_full[q % S], uint32_t((q / S) & 1), &no_abort, WAIT_LIMIT);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16(128, 128, 0, 0);
      const int k1 = (n + 15) / 16;
      const uint32_t sa0 = tc::smem_addr(sA), sb0 = tc::smem_addr(sB);
      long long nitem = 0, gp = 0;
      bool ok = true;
      for (long long k = blockIdx.x; k < prm.items && ok; k += gridDim.x, ++nitem) {
        long long jc, i, j0, j1;
        item_of(k, T, jc, i);
        pairs_of(jc, i, T, j0, j1);
        if (!tc::mbar_wait(a_full, uint32_t(nitem & 1), abortv, WAIT_LIMIT)) {
          ok = false;
          break;
        }
        for (long long j = j0; j < j1; ++j, ++gp) {
          const int st = int(gp % S), db = int(gp & 1);
          if (!tc::mbar_wait(&b_full[st], uint32_t((gp / S) & 1), abortv, WAIT_LIMIT) ||
              !tc::mbar_wait(&d_empty[db], uint32_t((gp >> 1) & 1) ^ 1u, abortv, WAIT_LIMIT)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t bb = sb0 + uint32_t(st) * tile_bytes;
          for (int kk = 0; kk < k1; ++kk) {
            const uint32_t off = (kk >> 2) * REG_BYTES + (kk & 3) * 32;
            tc::mma_bf16(tmem + db * 128, tc::sdesc_sw128(sa0 + off, 16, 1024),
                         tc::sdesc_sw128(bb + off, 16, 1024), idesc, kk > 0 ? 1u : 0u);
          }
          tc::mma_commit(&b_empty[st]);
          tc::mma_commit(&d_full[db]);
        }
        tc::mma_commit(a_empty);  // tile i may be replaced once these MMAs are done
      }
      if (!ok) fail();
      tc::mma_commit(mma_done);
      tc::mbar_wait(mma_done, 0, &no_abort, WAIT_LIMIT);
    }
  } else {
    // ------------------------------------------------------------------ epilogue
    const int ew = warp - 2;
    const int cg = ew >> 2;                 // column group: columns [32 cg, 32 cg + 32)
    const int q = warp & 3;                 // TMEM lane quarter
    const int L = 32 * q + lane;            // sample of tile i
    const uint32_t lane_off = uint32_t(32 * q) << 16;
    float acc_s = 0.f, acc_c = 0.f;
    long long gp = 0;
    bool ok = true;
    const bool uniform = prm.nu == nullptr;
    for (long long k = blockIdx.x; k < prm.items && ok; k += gridDim.x) {
      long long jc, i, j0, j1;
      item_of(k, T, jc, i);
      pairs_of(jc, i, T, j0, j1);
      const long long sl = i * TM + L;
      const float nu_l = uniform ? 1.f : (sl < prm.p ? (float)prm.nu[sl] : 0.f);
      for (long long j = j0; j < j1; ++j, ++gp) {
        const int db = int(gp & 1);
        if (!tc::mbar_wait(&d_full[db], uint32_t((gp >> 1) & 1), abortv, WAIT_LIMIT)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        float g[32];
        tc::tmem_ld32(tmem + db * 128 + 32 * cg + lane_off, g);
        tc::tmem_ld_wait();
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&d_empty[db]);
        float row = 0.f;
        if (uniform) {
          // samples beyond p are zero-filled by TMA, so their G entries (and powers) vanish
#pragma unroll
          for (int c = 0; c < 32; ++c) row += powd<DP>(g[c]);
        } else {
          const long long k0 = j * TM + 32 * cg;
#pragma unroll
          for (int c = 0; c < 32; ++c) {
            const float nk = (k0 + c) < prm.p ? (float)prm.nu[k0 + c] : 0.f;
            row += nk * powd<DP>(g[c]);
          }
        }
        kahan_add(acc_s, acc_c, (j == i ? 1.f : 2.f) * nu_l * row);
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
  if (warp == 1) tc::tmem_dealloc(tmem, 256);
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
  const int tile = nload * REG_BYTES;
  int S = (232448 - 2048 - tile) / tile;
  return S > 6 ? 6 : S;
}

}  // namespace

bool gram_tc_supported(int dtype, int n, int64_t p) {
  return dtype == STMF_BF16 && n >= 1 && n <= 256 && p < (int64_t(1) << 31) - TM &&
         encoder() != nullptr && stages_for(n) >= 2;
}

int gram_tc_grid(int64_t p, int num_sms) {
  const long long T = (p + TM - 1) / TM;
  const long long nrows = (T + JC - 1) / JC;
  // total items: rows hold min(T, JC (q + 1)) items
  long long items = 0;
  for (long long q = 0; q < nrows; ++q) items += (JC * (q + 1) < T ? JC * (q + 1) : T);
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
  const long long nrows = (prm.T + JC - 1) / JC;
  long long items = 0;
  for (long long q = 0; q < nrows; ++q) items += (JC * (q + 1) < prm.T ? JC * (q + 1) : prm.T);
  prm.items = items;
  prm.status = gp.status;
  const int tile = prm.nload * REG_BYTES;
  prm.smem_bytes = tile * (1 + prm.stages) + 1024 /*align*/ + 1024 /*barriers*/;
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
