// Fused pass over BF16 (and E4M3) samples on the 5th-generation tensor cores (tcgen05, TMA,
// TMEM), with two more modes of the same pipeline: the randomized range finder of eq. rrf
// (A0 = V Omega, Omega drawn in the epilogue, no MMA1) and the sampled evaluation of Sec. 5
// (rows idx[0..p) copied into the stages in place of TMA: by gather warps for BF16 samples, by
// the converter warps for E4M3 samples).
//
// Computes, per persistent CTA and over that CTA's sample tiles, the partial sums of Alg. 2's
// Y (Lemma 3.3, eq. Y) and of Lemma 3.5:
//     Y_part = sum_l nu_l (v_l^T A)^{d-1} v_l,      w_part_j = sum_l nu_l (v_l^T a_j)^d,
// reading every sample from HBM exactly once.
//
// Per 128-sample tile (V_t: 128 samples x n features, BF16, staged by TMA with the 128-byte
// swizzle, one 16 KB region per 64 features):
//   MMA1  Z  = V_t [A_hi, A_lo]            M = 128 samples, N = 2 RP, K = n     (TMEM)
//   epi   z = Z_hi + Z_lo;  W = nu z^{d-1} (split into BF16 hi | lo);  w += nu z^d
//   end   w += d sum_i Y_ij (A - A_hi - A_lo)_ij   (first-order correction for the split of A)
//   MMA2  Y += V_t^T [W_hi, W_lo]          M = 128 features (per block), N = 2 RP, K = 128
// The same shared-memory tile is the K-major A operand of MMA1 and the MN-major A operand of
// MMA2. A (FP64) is split once per CTA into BF16 hi/lo halves so that A_hi + A_lo carries ~16
// significant bits; W is split the same way per tile. Both halves ride in one MMA along N, so
// V is read from shared memory once per MMA.
//
// Warp roles (608 threads): warp 0 = TMA producer, warp 1 = TMEM allocator and MMA1 issuer,
// warp 2 = MMA2 issuer, warps 3-18 = epilogue in four warpgroups that split the components
// (thread = TMEM lane = sample of the tile, or feature of the M-block); E4M3 samples add warps
// 19-22 that widen the codes, gathered rows add warps 19-22 that copy the rows (736 threads).
// Pipelines: S shared-memory stages of V; double-buffered Z (TMEM) and W (shared memory); Y
// accumulates in TMEM and is folded into compensated FP32 registers every `flush` tiles (FP64
// from the block partials on), with two TMEM
// buffers so the MMAs never wait for the fold and the epilogue folds whenever the buffer is
// done rather than waiting for it. Every wait is bounded: a wait that runs out sets
// STMF_ETIMEOUT in the status word and all roles wind down, wait for their own copies and MMAs,
// and free TMEM before the CTA exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "rrf_draw.cuh"
#include "stmf_internal.h"
#include "tc_common.cuh"

namespace stmf {
namespace {

constexpr int TM = 128;                // samples per tile
constexpr int REG_BYTES = TM * 128;    // one 64-feature region of a V tile (16 KB)
constexpr int EG = 4;                  // epilogue warpgroups (components split among them)
constexpr int NEPI = 128 * EG;         // epilogue threads
constexpr int NTHREADS = 96 + NEPI;    // producer warp, MMA1 warp, MMA2 warp, epilogue
constexpr int NCONV = 4;               // FP8 samples: warps that widen E4M3 tiles to BF16
constexpr int NTHREADS_FP8 = NTHREADS + 32 * NCONV;
// Z accumulators per tile: MMA1's K steps are split ZC ways and the partial products summed in
// the epilogue with round-to-nearest. The tensor cores' FP32 accumulation truncates, so a long
// run of accumulations biases |z| low (measured at n = 256: 1.6e-6 relative with one
// accumulator, 0.8e-6 with two, 0.4e-6 with four); w = sum nu z^d inherits d times that bias.
// Two accumulators halve it for about 1% of the pass time.
constexpr int ZC = 2;
constexpr long long WAIT_LIMIT = 4000000000LL;  // SM cycles (about 2 s) before a wait gives up

struct TcExtra {
  int nload;      // regions loaded by TMA: ceil(n / 64)
  int nreg;       // regions per stage, even: 2 * ceil(n / 128)
  int stages;
  int flush;      // tiles between folds of Y into FP64
  int tmem_cols;
  int smem_bytes;
  int nq;         // E4M3 samples: 128-feature regions per tile (ceil(n / 128))
  int kpz;        // K steps (16 features each) per Z accumulator (ZC accumulators per tile)
};

// Column order along N (rows of the A and W splits, columns of Z and Y in TMEM): components are
// grouped by epilogue warpgroup, hi and lo side by side, so one TMEM load brings a warpgroup's
// hi and lo values: column of (component j, part) = (j / CPG) 2 CPG + part CPG + j % CPG.
template <int RP>
struct Cfg {
  static constexpr int CPG = RP / EG;         // components per epilogue warpgroup
  static constexpr int N = 2 * RP;            // MMA N: hi and lo of every component
  static constexpr int W_REG = N * 128;       // one 64-sample region of W (N rows)
  static constexpr int A_REG = N * 128;       // one 64-feature region of the A split
};

// Compensated FP32 accumulation (Kahan): s + c carries the running sum to about twice FP32's
// precision without the FP64 pipe, which is a small fraction of FP32 throughput on this part.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

__device__ __forceinline__ float ipow_f(float z, int e) {
  float t = z;
  for (int k = 1; k < e; ++k) t *= z;
  return t;
}

// Two E4M3 codes -> two BF16 values, exactly (E4M3 -> FP16 -> FP32 -> BF16; every E4M3 value
// has at most 4 significant bits and an exponent in -9..8, so no step rounds).
__device__ __forceinline__ uint32_t e4m3x2_to_bf16x2(uint16_t q) {
  const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)q, __NV_E4M3);
  const __half2 hh = *reinterpret_cast<const __half2*>(&hr);
  const __nv_bfloat162 bb = __floats2bfloat162_rn(__low2float(hh), __high2float(hh));
  return *reinterpret_cast<const uint32_t*>(&bb);
}

// 16-byte global -> shared copy of which the first `bytes` are read (the rest zero-filled).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int C>
__device__ __forceinline__ void tmem_load_cols(uint32_t taddr, float (&v)[C]) {
  if constexpr (C == 8) {
    tc::tmem_ld8(taddr, v);
  } else if constexpr (C == 4) {
    tc::tmem_ld4(taddr, v);
  } else {
    static_assert(C == 2, "2, 4 or 8 columns per load");
    tc::tmem_ld2(taddr, v);
  }
}

// FP8 = false: BF16 samples, TMA fills the S-stage ring the MMAs read.
// FP8 = true:  E4M3 samples (v = s q): TMA brings each 128-feature half of an E4M3 tile (16 KB)
//              into the upper 64-feature region of its two BF16 regions in the same S-stage ring,
//              and NCONV converter warps widen it to BF16 in place (every E4M3 value is exactly a
//              BF16 value) before the MMAs read the stage; the scale folds into the weight,
//              nu' = nu s^d: with z = q^T a, the terms of eq. Y and Lemma 3.5 are nu' z^{d-1} q
//              and nu' z^d.
// MODE = kRrf:    the randomized range finder of eq. rrf, Y_part = sum_l v_l omega_l^T: no MMA1
//                 and no w; the epilogue draws row l of the Gaussian test matrix (Philox4x32-10,
//                 FP32 Box-Muller; times s_l for E4M3) as W, and MMA2 accumulates V^T W as above.
//                 MMA2 then waits for the staged tile itself, which MMA1 otherwise orders.
// MODE = kGather: the sampled evaluation of Sec. 5 (Lemma 5.1) on rows idx[0..p): for BF16
//                 samples NCONV gather warps copy the rows into the stages in place of TMA; for
//                 E4M3 samples the converter warps fetch the code rows before widening them.
enum PassMode { kFused = 0, kRrf = 1, kGather = 2 };

template <int RP, bool FP8, int MODE>
__global__ void __launch_bounds__((FP8 || MODE == kGather) ? NTHREADS_FP8 : NTHREADS, 1)
    fg_tc_kernel(const __grid_constant__ CUtensorMap tmap, const FgParams prm, const TcExtra ex) {
  constexpr bool RRF = MODE == kRrf, GATHER = MODE == kGather;
  constexpr int NT = (FP8 || GATHER) ? NTHREADS_FP8 : NTHREADS;
  using C = Cfg<RP>;
  constexpr int N = C::N;
  if (prm.skip && *prm.skip) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw_addr = tc::smem_addr(smem_raw);
  unsigned char* base = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);

  const int S = ex.stages, nreg = ex.nreg, nload = ex.nload;
  const int kpz = ex.kpz;
  const int n = prm.n, r = prm.r, d = prm.d;
  const uint32_t stage_bytes = uint32_t(nreg) * REG_BYTES;
  unsigned char* sV = base;
  unsigned char* sW = sV + size_t(S) * stage_bytes;
  unsigned char* sA = sW + 2 * 2 * C::W_REG;
  const int nq = ex.nq;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA + size_t(nreg) * C::A_REG);
  uint64_t* full = bars;          // TMA landed
  uint64_t* empty = bars + S;     // MMA2 done with the stage
  uint64_t* conv = bars + 2 * S;  // E4M3 samples: the stage is widened to BF16
  uint64_t* zfull = bars + 3 * S;
  uint64_t* zempty = zfull + 2;
  uint64_t* wfull = zempty + 2;
  uint64_t* wempty = wfull + 2;
  uint64_t* yfull = wempty + 2;
  uint64_t* yempty = yfull + 2;
  uint64_t* mma_done = yempty + 2;  // [0]: MMA1 issuer, [1]: MMA2 issuer
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 2);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  double* wred = reinterpret_cast<double*>(mma_done + 3);  // 4 x RP

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], GATHER ? NCONV : 1);  // TMA, or one arrival per gather warp
      tc::mbar_init(&empty[s], 1);
      tc::mbar_init(&conv[s], NCONV);  // one arrival per converter warp
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&zfull[b], 1);
      tc::mbar_init(&zempty[b], NEPI / 32);  // one elected arrival per epilogue warp
      tc::mbar_init(&wfull[b], NEPI / 32);
      tc::mbar_init(&wempty[b], 1);
      tc::mbar_init(&yfull[b], 1);
      tc::mbar_init(&yempty[b], NEPI / 32);
    }
    tc::mbar_init(&mma_done[0], 1);
    tc::mbar_init(&mma_done[1], 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (!GATHER && warp == 0 && lane == 0) tc::prefetch_tmap(&tmap);
  if (warp == 1) tc::tmem_alloc(tmem_slot, ex.tmem_cols);

  // A split: the hi row of component j holds BF16(a_j), its lo row BF16(a_j - BF16(a_j)); K =
  // feature (not used by the range finder).
  {
    const int kext = nreg * 64;
    for (int e = tid; e < (RRF ? 0 : N * kext); e += NT) {
      const int row = e / kext, k = e - row * kext;
      const int grp = row / (2 * C::CPG), part = (row / C::CPG) & 1;
      const int j = grp * C::CPG + row % C::CPG;
      double a = (j < r && k < n) ? prm.A[k + size_t(n) * j] : 0.0;
      const __nv_bfloat16 hi = __double2bfloat16(a);
      const __nv_bfloat16 v = part == 0 ? hi : __double2bfloat16(a - (double)__bfloat162float(hi));
      *reinterpret_cast<__nv_bfloat16*>(sA + (k >> 6) * C::A_REG + tc::sw128_offset(row, k & 63)) = v;
    }
    // regions of each V stage that TMA never loads (features beyond the last 64-block) are zero
    const int zero_regs = nreg - nload;
    if (zero_regs > 0) {
      const int words = zero_regs * REG_BYTES / 16;
      for (int s = 0; s < S; ++s) {
        uint4* z = reinterpret_cast<uint4*>(sV + size_t(s) * stage_bytes + size_t(nload) * REG_BYTES);
        for (int e = tid; e < words; e += NT) z[e] = make_uint4(0, 0, 0, 0);
      }
    }
  }
  tc::fence_proxy_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int64_t num_tiles = (prm.p + TM - 1) / TM;
  const int my_tiles = (int)((num_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
  const int nmb = nreg / 2;
  const int flush = ex.flush;
  volatile int* abortv = abort_flag;
  int no_abort = 0;
  auto fail = [&]() {
    stmf_set_status(prm.status, STMF_ETIMEOUT);
    *abortv = 1;
  };

  if (warp == 0) {
    // ------------------------------------------------------------------ TMA producer
    if (!GATHER && lane == 0) {
      // BF16: tiles go straight to the MMAs; E4M3: the converters widen them in place first
      const int R = S;
      uint64_t* rfull = full;
      uint64_t* rempty = empty;
      const uint32_t rbytes = FP8 ? uint32_t(nq) * REG_BYTES : uint32_t(nload) * REG_BYTES;
      int issued = 0;
      for (int it = 0; it < my_tiles; ++it) {
        const int st = it % R;
        const uint32_t ph = (it / R) & 1;
        if (!tc::mbar_wait(&rempty[st], ph ^ 1, abortv, WAIT_LIMIT)) {
          fail();
          break;
        }
        tc::mbar_arrive_expect_tx(&rfull[st], rbytes);
        const int64_t tile = blockIdx.x + int64_t(it) * gridDim.x;
        if constexpr (FP8) {
          for (int g = 0; g < nq; ++g)  // half g into BF16 region 2g + 1
            tc::tma_load_2d(sV + size_t(st) * stage_bytes + size_t(2 * g + 1) * REG_BYTES, &tmap,
                            g * 128, (int32_t)(tile * TM), &rfull[st]);
        } else {
          for (int g = 0; g < nload; ++g)
            tc::tma_load_2d(sV + size_t(st) * stage_bytes + size_t(g) * REG_BYTES, &tmap, g * 64,
                            (int32_t)(tile * TM), &rfull[st]);
        }
        ++issued;
      }
      // wait for the last copy issued into each stage (already complete unless we aborted)
      for (int k = issued > R ? issued - R : 0; k < issued; ++k)
        tc::mbar_wait(&rfull[k % R], (k / R) & 1, &no_abort, WAIT_LIMIT);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA1 issuer
    // Z(t) = V_t [A_hi | A_lo] as soon as tile t has landed and its Z buffer is free.
    if (!RRF && lane == 0) {
      const uint32_t idesc1 = tc::idesc_bf16(128, N, 0, 0);  // V K-major, A split K-major
      const int k1 = (n + 15) / 16;
      // shared-memory descriptors are linear in the operand address (16-byte units in the low
      // bits; every address here is below 256 KB): one base per operand plus (offset >> 4)
      const uint64_t vdesc0 = tc::sdesc_sw128(tc::smem_addr(sV), 16, 1024);
      const uint64_t adesc0 = tc::sdesc_sw128(tc::smem_addr(sA), 16, 1024);
      bool ok = true;
      for (int t = 0; t < my_tiles; ++t) {
        const int st = t % S, zb = t & 1;
        ok = tc::mbar_wait(FP8 ? &conv[st] : &full[st], (t / S) & 1, abortv, WAIT_LIMIT) &&
             tc::mbar_wait(&zempty[zb], ((t >> 1) & 1) ^ 1, abortv, WAIT_LIMIT);
        if (!ok) break;
        tc::tc_fence_after();
        const uint64_t vd = vdesc0 + uint64_t((uint32_t(st) * stage_bytes) >> 4);
        // accumulator c takes K steps [c kpz, min((c + 1) kpz, k1)); one that gets none (small
        // n) takes step c kpz alone, which lies in the zero padding of both operands, so every
        // accumulator is written
        for (int c = 0; c < ZC; ++c) {
          const uint32_t dZ = tmem + uint32_t(zb * ZC + c) * N;
          const int kb = c * kpz;
          const int ke = kb + kpz < k1 ? kb + kpz : (kb < k1 ? k1 : kb + 1);
          for (int kk = kb; kk < ke; ++kk)
            tc::mma_bf16(dZ, vd + uint64_t(((kk >> 2) * REG_BYTES + (kk & 3) * 32) >> 4),
                         adesc0 + uint64_t(((kk >> 2) * C::A_REG + (kk & 3) * 32) >> 4), idesc1,
                         kk > kb ? 1u : 0u);
        }
        tc::mma_commit(&zfull[zb]);
      }
      if (!ok) fail();
      tc::mma_commit(&mma_done[0]);
      tc::mbar_wait(&mma_done[0], 0, &no_abort, WAIT_LIMIT);
    }
  } else if (warp == 2) {
    // ------------------------------------------------------------------ MMA2 issuer
    // Y += V_t^T [W_hi | W_lo] as soon as W(t) is written; its completion frees the V stage.
    // A separate issuing thread keeps this from queueing behind the next tile's MMA1 issue.
    if (lane == 0) {
      const uint32_t idesc2 = tc::idesc_bf16(128, N, 1, 0);  // V^T MN-major, W K-major
      const uint64_t vdesc0 = tc::sdesc_sw128(tc::smem_addr(sV), REG_BYTES, 1024);
      const uint64_t wdesc0 = tc::sdesc_sw128(tc::smem_addr(sW), 16, 1024);
      bool ok = true;
      for (int t = 0; t < my_tiles; ++t) {
        const int st = t % S, wb = t & 1;
        const int period = t / flush, yb = period & 1;
        const bool first = (t % flush) == 0;
        if (first) ok = tc::mbar_wait(&yempty[yb], ((period >> 1) & 1) ^ 1, abortv, WAIT_LIMIT);
        ok = ok && tc::mbar_wait(&wfull[wb], (t >> 1) & 1, abortv, WAIT_LIMIT);
        if constexpr (RRF)  // no MMA1 has waited for this tile
          ok = ok && tc::mbar_wait(FP8 ? &conv[st] : &full[st], (t / S) & 1, abortv, WAIT_LIMIT);
        if (!ok) break;
        tc::tc_fence_after();
        const uint64_t wd = wdesc0 + uint64_t((uint32_t(wb) * 2 * C::W_REG) >> 4);
        for (int mb = 0; mb < nmb; ++mb) {
          const uint32_t dY = tmem + uint32_t(2 * ZC + yb * 2 + mb) * N;
          const uint64_t vd =
              vdesc0 + uint64_t((uint32_t(st) * stage_bytes + uint32_t(2 * mb) * REG_BYTES) >> 4);
#pragma unroll
          for (int kk = 0; kk < TM / 16; ++kk)
            tc::mma_bf16(dY, vd + uint64_t((kk * 2048) >> 4),
                         wd + uint64_t(((kk >> 2) * C::W_REG + (kk & 3) * 32) >> 4), idesc2,
                         (first && kk == 0) ? 0u : 1u);
        }
        tc::mma_commit(&empty[st]);
        tc::mma_commit(&wempty[wb]);
        if ((t % flush) == flush - 1 || t == my_tiles - 1) tc::mma_commit(&yfull[yb]);
      }
      if (!ok) fail();
      tc::mma_commit(&mma_done[1]);
      tc::mbar_wait(&mma_done[1], 0, &no_abort, WAIT_LIMIT);
    }
  } else if (GATHER && !FP8 && warp >= 3 + NEPI / 32) {
    // ------------------------------------------------------------------ row gather (Sec. 5)
    // Gather warp G copies rows y = G + 4k (k = 0..31) of tile t: row y is sample idx[t TM + y],
    // and one warp instruction copies the whole row, lane l taking its 16-byte chunk l (features
    // 8l .. 8l + 7: region l / 8, chunk l % 8 at position (l % 8) ^ (y & 7) of the 128-byte
    // swizzle TMA would use), so each instruction reads whole 128-byte lines. Features past n and
    // rows past p are zero-filled; a row outside the storage reads as zero and sets STMF_EINVAL.
    // cp.async writes through the generic proxy, so each thread waits for its own copies and
    // fences them to the async proxy (the MMAs) before its warp arrives; two tiles are in flight
    // per warp, and the row indices are read one tile ahead (one per lane).
    if constexpr (GATHER && !FP8) {
      const int G = warp - (3 + NEPI / 32);  // 0 .. NCONV - 1
      const uint16_t* Vg = static_cast<const uint16_t*>(prm.V);
      const int lg = lane >> 3, lc = lane & 7;  // this lane's region and chunk of a row
      const int f0 = 64 * lg + 8 * lc;          // its first feature
      const int valid = n - f0 >= 8 ? 8 : (n - f0 > 0 ? n - f0 : 0);
      const bool active = lg < nload;           // regions past the last loaded one stay zero
      auto row_of = [&](int it_) -> int64_t {   // the row of sample y = G + 4 lane of tile it_
        const int64_t pos = (blockIdx.x + int64_t(it_) * gridDim.x) * TM + G + 4 * lane;
        if (it_ >= my_tiles || pos >= prm.p) return -1;
        const int64_t row = prm.idx[pos];
        if (row < 0 || row >= prm.rows) {
          stmf_set_status(prm.status, STMF_EINVAL);
          return -1;
        }
        return row;
      };
      auto retire = [&](int k) {  // this warp's copies of tile k have landed
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&full[k % S]);
      };
      bool ok = true;
      int64_t row_next = row_of(0);
      int it = 0;
      for (; it < my_tiles; ++it) {
        const int st = it % S;
        ok = tc::mbar_wait(&empty[st], ((it / S) & 1) ^ 1, abortv, WAIT_LIMIT);
        if (!__all_sync(0xffffffffu, ok)) {
          ok = false;
          break;
        }
        const int64_t my_row = row_next;  // row of sample G + 4 lane
        row_next = row_of(it + 1);
        const uint32_t stage0 = tc::smem_addr(sV + size_t(st) * stage_bytes) +
                                uint32_t(lg) * REG_BYTES;
        for (int k = 0; k < 32; ++k) {
          const int y = G + 4 * k;
          const int64_t row = __shfl_sync(0xffffffffu, my_row, k);
          if (active) {
            const int nb = row < 0 ? 0 : valid;
            const uint16_t* src = nb ? Vg + row * prm.ld + f0 : Vg;
            cp_async16(stage0 + uint32_t(y) * 128u + ((uint32_t(lc) ^ uint32_t(y & 7)) << 4), src,
                       uint32_t(2 * nb));
          }
        }
        cp_async_commit();
        if (it >= 1) {
          cp_async_wait<1>();
          retire(it - 1);
        }
      }
      cp_async_wait<0>();  // nothing of this thread's stays in flight past here
      if (ok && it >= 1) retire(it - 1);
      if (!ok) fail();
    }
  } else if (FP8 && warp >= 3 + NEPI / 32) {
    // ------------------------------------------------------------------ E4M3 -> BF16 converters
    // Tile t: E4M3 region g (features [128 g, 128 g + 128), 128-byte rows) becomes BF16 regions
    // 2g and 2g + 1 of MMA buffer t % 2, both in the 128-byte swizzle. Features beyond n are zero
    // (TMA fills them), so the BF16 padding is zero too.
    if constexpr (FP8) {
      // thread ct owns row y = ct of every tile (128 converter threads, 128 samples per tile).
      // Per 128-feature half g: the E4M3 row (128 bytes, 16-byte chunk c at position c ^ (y & 7))
      // sits in BF16 region 2g + 1; all 8 chunks are read first, then features 0-63 become row y
      // of region 2g and features 64-127 overwrite row y of region 2g + 1 in place. Only this
      // thread touches row y, so nothing else can read the bytes it overwrites.
      const int ct = tid - (96 + NEPI);
      const int y = ct;
      auto widen_row = [&](int st) {  // row y of stage st, in place
        unsigned char* stg = sV + size_t(st) * stage_bytes;
        for (int g = 0; g < nq; ++g) {
          unsigned char* lo = stg + size_t(2 * g) * REG_BYTES + y * 128;
          unsigned char* hi = lo + REG_BYTES;  // holds the E4M3 row, becomes features 64-127
          uint4 raw[8];
#pragma unroll
          for (int c = 0; c < 8; ++c)
            raw[c] = *reinterpret_cast<const uint4*>(hi + (((c ^ (y & 7)) & 7) << 4));
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            unsigned char* dst = h == 0 ? lo : hi;
#pragma unroll
            for (int c = 0; c < 4; ++c) {  // E4M3 chunk 4h + c -> BF16 chunks 2c, 2c + 1
              const uint4 q = raw[4 * h + c];
              const uint32_t w[4] = {q.x, q.y, q.z, q.w};
              uint32_t o[8];
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                o[2 * k] = e4m3x2_to_bf16x2((uint16_t)(w[k] & 0xFFFFu));
                o[2 * k + 1] = e4m3x2_to_bf16x2((uint16_t)(w[k] >> 16));
              }
              *reinterpret_cast<uint4*>(dst + ((((2 * c) ^ (y & 7)) & 7) << 4)) =
                  make_uint4(o[0], o[1], o[2], o[3]);
              *reinterpret_cast<uint4*>(dst + ((((2 * c + 1) ^ (y & 7)) & 7) << 4)) =
                  make_uint4(o[4], o[5], o[6], o[7]);
            }
          }
        }
      };
      bool ok = true;
      if constexpr (GATHER) {
        // Sampled E4M3 rows (Sec. 5): the converter warps fetch the code rows themselves. Warp w
        // holds rows y = 32 w + l of every tile (lane l: the row index of sample y, read one
        // tile ahead); one warp instruction copies two rows' codes (lanes 0-15 and 16-31,
        // 16-byte chunk q = codes 16q .. 16q + 15: half q / 8 into region 2 (q / 8) + 1, chunk
        // q % 8 at position (q % 8) ^ (y & 7), where TMA would put it), zero-filling codes past
        // n and rows past p; a row outside the storage reads as zero and sets STMF_EINVAL. Tile
        // t + 1 is requested before tile t is widened: each thread waits for its own copies of
        // t, the warp syncs (its rows are complete), every thread widens its row in place,
        // fences to the async proxy, and the warp arrives.
        const int w = y >> 5, half = lane >> 4, q = lane & 15;
        const bool active = (q >> 3) < nq;
        const uint8_t* V8 = static_cast<const uint8_t*>(prm.V);
        const int f = 16 * q;
        const int fv = n - f >= 16 ? 16 : (n - f > 0 ? n - f : 0);
        auto row_of = [&](int it_) -> int64_t {
          const int64_t pos = (blockIdx.x + int64_t(it_) * gridDim.x) * TM + y;
          if (it_ >= my_tiles || pos >= prm.p) return -1;
          const int64_t row = prm.idx[pos];
          if (row < 0 || row >= prm.rows) {
            stmf_set_status(prm.status, STMF_EINVAL);
            return -1;
          }
          return row;
        };
        auto finish = [&](int k) {
          __syncwarp();
          widen_row(k % S);
          tc::fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&conv[k % S]);
        };
        int64_t row_cur = -1, row_next = row_of(0);
        int it = 0;
        for (; it < my_tiles; ++it) {
          const int st = it % S;
          ok = tc::mbar_wait(&empty[st], ((it / S) & 1) ^ 1, abortv, WAIT_LIMIT);
          if (!__all_sync(0xffffffffu, ok)) {
            ok = false;
            break;
          }
          row_cur = row_next;
          row_next = row_of(it + 1);
          const uint32_t base = tc::smem_addr(sV + size_t(st) * stage_bytes) +
                                uint32_t(2 * (q >> 3) + 1) * REG_BYTES;
#pragma unroll 4
          for (int i = 0; i < 16; ++i) {
            const int yy = 32 * w + 2 * i + half;
            const int64_t row = __shfl_sync(0xffffffffu, row_cur, 2 * i + half);
            if (active) {
              const int nb = row < 0 ? 0 : fv;
              const uint8_t* src = nb ? V8 + row * prm.ld + f : V8;
              cp_async16(base + uint32_t(yy) * 128u + ((uint32_t(q & 7) ^ uint32_t(yy & 7)) << 4),
                         src, uint32_t(nb));
            }
          }
          cp_async_commit();
          if (it >= 1) {
            cp_async_wait<1>();
            finish(it - 1);
          }
        }
        cp_async_wait<0>();  // nothing of this thread's stays in flight past here
        if (ok && it >= 1) finish(it - 1);
      } else {
        for (int it = 0; it < my_tiles; ++it) {
          const int st = it % S;
          if (!tc::mbar_wait(&full[st], (it / S) & 1, abortv, WAIT_LIMIT)) {
            ok = false;
            break;
          }
          widen_row(st);
          tc::fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&conv[st]);
        }
      }
      if (!ok) fail();
    }
  } else {
    // ------------------------------------------------------------------ epilogue
    // EG warpgroups; warpgroup g owns components [g*CPG, (g+1)*CPG) of every sample of the tile
    // (thread = TMEM lane = sample), so the per-tile work of one thread is CPG components.
    constexpr int CPG = C::CPG;
    const int g = (warp - 3) >> 2;
    const int q = warp & 3;            // TMEM lane quarter this warp may access
    const int L = 32 * q + lane;       // sample within the tile / feature within the M-block
    const int j0 = g * CPG;
    const uint32_t lane_off = uint32_t(32 * q) << 16;
    // per-period FP32 sums of w join compensated FP32 totals at the end of each period
    float wacc[CPG], ws[CPG], wc[CPG], ys[2][CPG], yc[2][CPG];
#pragma unroll
    for (int c = 0; c < CPG; ++c) {
      wacc[c] = ws[c] = wc[c] = 0.f;
      ys[0][c] = yc[0][c] = ys[1][c] = yc[1][c] = 0.f;
    }
    // byte offsets of this thread's W entries (rows j and RP + j, column L) in a W buffer
    const uint32_t wcol = uint32_t(L >> 6) * C::W_REG;
    int pending = -1;  // Y period whose fold is outstanding
    // Fold period `per` if its MMAs are done (or wait for them when `force`); clears `pending`
    // once folded. Returns false if a forced wait ran out.
    auto fold = [&](int per, bool force) -> bool {
      const int yb = per & 1;
      const uint32_t par = (per >> 1) & 1;
      if (!tc::mbar_test_wait(&yfull[yb], par)) {
        if (!force) return true;
        if (!tc::mbar_wait(&yfull[yb], par, abortv, WAIT_LIMIT)) return false;
      }
      tc::tc_fence_after();
#pragma unroll
      for (int mb = 0; mb < 2; ++mb) {
        if (mb < nmb) {
          float yv[2 * CPG];  // hi of the group's components, then lo
          tmem_load_cols<2 * CPG>(tmem + uint32_t(2 * ZC + yb * 2 + mb) * N + 2 * j0 + lane_off,
                                  yv);
          tc::tmem_ld_wait();
#pragma unroll
          for (int c = 0; c < CPG; ++c) {
            kahan_add(ys[mb][c], yc[mb][c], yv[c]);
            kahan_add(ys[mb][c], yc[mb][c], yv[CPG + c]);
          }
        }
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&yempty[yb]);
      pending = -1;
      return true;
    };
    // The weight of this thread's sample in tile it (and, for E4M3, its scale) is loaded one
    // tile ahead, so the loads' latency stays off the per-tile chain.
    float nu_next = 0.f, sc_next = 1.f;
    auto load_weight = [&](int it_) {
      const int64_t sidx_ = (blockIdx.x + int64_t(it_) * gridDim.x) * TM + L;
      nu_next = 0.f;
      if (it_ < my_tiles && sidx_ < prm.p) {
        nu_next = prm.nu ? (float)prm.nu[sidx_] : (float)prm.nu_uniform;
        if constexpr (FP8) {  // a gathered sample's scale is its row's (zero for a bad row)
          const int64_t srow = GATHER ? prm.idx[sidx_] : sidx_;
          sc_next = (srow >= 0 && srow < (GATHER ? prm.rows : prm.p)) ? prm.scale[srow] : 0.f;
        }
      }
    };
    load_weight(0);
    bool ok = true;
    for (int it = 0; it < my_tiles; ++it) {
      const int zb = it & 1, wb = it & 1;
      float nu_s = nu_next;
      const float sc_cur = sc_next;
      if constexpr (FP8 && !RRF) {  // nu' = nu s^d (the scale of sample l folded into its weight)
        float sd = sc_cur;
        for (int e = 1; e < d; ++e) sd *= sc_cur;
        nu_s *= sd;
      }
      load_weight(it + 1);
      float wv[CPG];
      if constexpr (RRF) {
        // W row of sample l: omega_lj (s_l omega_lj for E4M3 codes), zero past p and past r
        const int64_t sidx = (blockIdx.x + int64_t(it) * gridDim.x) * TM + L;
#pragma unroll
        for (int c = 0; c < CPG; ++c)
          wv[c] = (sidx < prm.p && j0 + c < r)
                      ? (FP8 ? sc_cur : 1.f) * rrf_omega_f32(sidx, j0 + c, prm.seed)
                      : 0.f;
      } else {
        if (!tc::mbar_wait(&zfull[zb], (it >> 1) & 1, abortv, WAIT_LIMIT)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        // z = sum over the Z accumulators of (hi + lo), rounded to nearest in FP32: each
        // accumulator takes only kpz truncating tensor-core accumulations
        float zv[ZC][2 * CPG];  // per accumulator: hi of the group's components, then lo
#pragma unroll
        for (int c = 0; c < ZC; ++c)
          tmem_load_cols<2 * CPG>(tmem + uint32_t(zb * ZC + c) * N + 2 * j0 + lane_off, zv[c]);
        tc::tmem_ld_wait();
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&zempty[zb]);
#pragma unroll
        for (int c = 0; c < CPG; ++c) {
          float zz = zv[0][c] + zv[0][CPG + c];
#pragma unroll
          for (int k = 1; k < ZC; ++k) zz += zv[k][c] + zv[k][CPG + c];
          const float t = ipow_f(zz, d - 1);
          wv[c] = nu_s * t;
          wacc[c] += wv[c] * zz;
        }
      }
      if (!tc::mbar_wait(&wempty[wb], ((it >> 1) & 1) ^ 1, abortv, WAIT_LIMIT)) {
        ok = false;
        break;
      }
      unsigned char* wbuf = sW + size_t(wb) * 2 * C::W_REG + wcol;
#pragma unroll
      for (int c = 0; c < CPG; ++c) {  // rows 2 j0 + c (hi) and 2 j0 + CPG + c (lo)
        const __nv_bfloat16 hi = __float2bfloat16_rn(wv[c]);
        const __nv_bfloat16 lo = __float2bfloat16_rn(wv[c] - __bfloat162float(hi));
        *reinterpret_cast<__nv_bfloat16*>(wbuf + tc::sw128_offset(2 * j0 + c, L & 63)) = hi;
        *reinterpret_cast<__nv_bfloat16*>(wbuf + tc::sw128_offset(2 * j0 + CPG + c, L & 63)) = lo;
      }
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&wfull[wb]);
      // Fold a finished Y period into FP64 once its MMAs have completed. The fold is polled on
      // later tiles rather than waited for, so the epilogue never stalls behind MMA2; Y is
      // double-buffered, so MMA2 needs this buffer back only a whole period later. A fold that
      // is still outstanding is forced on the tile before the next period ends, at a period's
      // end if one is somehow still pending, and on the CTA's last tile.
      const bool period_end = (it % flush) == flush - 1 || it == my_tiles - 1;
      // the FP32 sum of w over the period joins the compensated total at the period's last
      // tile, a fixed point (the Y fold below happens whenever MMA2 is done, which varies), so
      // the result is the same bit for bit from run to run
      if (period_end) {
#pragma unroll
        for (int c = 0; c < CPG; ++c) {
          kahan_add(ws[c], wc[c], wacc[c]);
          wacc[c] = 0.f;
        }
      }
      if (period_end && pending >= 0 && !fold(pending, true)) {
        ok = false;
        break;
      }
      if (period_end) pending = it / flush;
      if (pending >= 0) {
        const bool force = it == my_tiles - 1 || (it % flush) == flush - 2;
        if (!fold(pending, force)) {
          ok = false;
          break;
        }
      }
    }
    if (!ok) {
      fail();
    } else {
      double* part = prm.partials + size_t(blockIdx.x) * (size_t(r) + size_t(n) * r);
      // First-order correction of w for the split of A: MMA1 contracts with
      // A^ = A_hi + A_lo = A - dA (|dA| <= 2^-17 |A|), so z^ = z - v^T da_j and
      // sum nu z^d = sum nu z^^d + d sum_i Y_ij dA_ij + O(|dA|^2), with Y the block's own partial
      // of eq. Y. The correction is linear in Y, so block partials stay additive.
      double corr[CPG];
#pragma unroll
      for (int c = 0; c < CPG; ++c) corr[c] = 0.0;
#pragma unroll
      for (int mb = 0; mb < 2; ++mb) {
        const int i = 128 * mb + L;
        if (mb < nmb && i < n) {
#pragma unroll
          for (int c = 0; c < CPG; ++c)
            if (j0 + c < r) {
              const double y = (double)ys[mb][c] - (double)yc[mb][c];
              part[r + i + size_t(n) * (j0 + c)] = y;
              if constexpr (!RRF) {
                const double a = prm.A[i + size_t(n) * (j0 + c)];
                const double hi = (double)__bfloat162float(__double2bfloat16(a));
                const double lo = (double)__bfloat162float(__double2bfloat16(a - hi));
                corr[c] += y * ((a - hi) - lo);
              }
            }
        }
      }
#pragma unroll
      for (int c = 0; c < CPG; ++c) {
        double x = (double)ws[c] - (double)wc[c] + double(d) * corr[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) wred[q * RP + j0 + c] = x;
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (tid < r && !*abortv) {
    double* part = prm.partials + size_t(blockIdx.x) * (size_t(r) + size_t(n) * r);
    part[tid] = wred[0 * RP + tid] + wred[1 * RP + tid] + wred[2 * RP + tid] + wred[3 * RP + tid];
  }
  if (warp == 1) tc::tmem_dealloc(tmem, ex.tmem_cols);
}

// ---------------------------------------------------------------------------------- host side
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode() {
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

int rp_of(int r) { return r <= 8 ? 8 : 16; }

TcExtra plan(int n, int r, bool) {  // the same staging serves BF16 and E4M3 samples
  TcExtra ex{};
  ex.nload = (n + 63) / 64;
  ex.nreg = 2 * ((n + 127) / 128);
  const int RP = rp_of(r), N = 2 * RP;
  const int fixed = 2 * 2 * N * 128 + ex.nreg * N * 128 + 1024 /*align*/ + 1024 /*barriers, w*/;
  const int stage = ex.nreg * REG_BYTES;
  int S = (232448 - fixed) / stage;
  if (S > 8) S = 8;
  ex.stages = S;
  ex.flush = 8;  // fewer truncating accumulations of Y in TMEM between FP32 folds
  // MMA1 runs K = n in k1 steps of 16 features, split over ZC accumulators. An accumulator with
  // no step of its own takes step c kpz <= 9, inside the zero padding: the V stage holds
  // nreg * 64 >= 128 features (zero past n) and the A split is zero past n as well.
  const int k1 = (n + 15) / 16;
  ex.kpz = (k1 + ZC - 1) / ZC;
  int cols = (2 * ZC + 4) * N;
  int pow2 = 32;
  while (pow2 < cols) pow2 <<= 1;
  ex.tmem_cols = pow2;
  ex.smem_bytes = fixed + S * stage;
  ex.nq = (n + 127) / 128;
  return ex;
}

template <int RP, bool FP8, int MODE>
cudaError_t launch_rp(const CUtensorMap& tmap, const FgParams& prm, const TcExtra& ex, int grid,
                      cudaStream_t s) {
  const cudaError_t e = smem_limit((const void*)fg_tc_kernel<RP, FP8, MODE>, 232448);
  if (e != cudaSuccess) return e;
  return launch_kernel(fg_tc_kernel<RP, FP8, MODE>, dim3(grid),
                       dim3((FP8 || MODE == kGather) ? NTHREADS_FP8 : NTHREADS),
                       size_t(ex.smem_bytes), s, tmap, prm, ex);
}

}  // namespace

size_t fg_tc_supported(int dtype, int n, int r) {
  if (dtype != STMF_BF16 && dtype != STMF_E4M3) return 0;
  if (r < 1 || r > 16 || n < 1 || n > 256) return 0;
  if (!get_encode()) return 0;
  const TcExtra ex = plan(n, r, dtype == STMF_E4M3);
  return ex.stages >= 2 ? 1 : 0;
}

int fg_tc_grid(int, int, int, int64_t p, int num_sms, int min_tiles) {
  // one CTA per SM, or fewer so that each takes at least min_tiles tiles (a CTA holds a whole SM
  // through its shared memory, so a small pass spread over every SM keeps concurrent passes off
  // the GPU while it runs one or two tiles per SM)
  const int64_t tiles = (p + TM - 1) / TM;
  const int64_t mt = min_tiles > 1 ? min_tiles : 1;
  const int64_t want = (tiles + mt - 1) / mt;
  return (int)(want < num_sms ? want : num_sms);
}

namespace {

template <int MODE>
cudaError_t launch_tc(int dtype, const FgParams& prm, int grid, cudaStream_t s) {
  if (dtype != STMF_BF16 && dtype != STMF_E4M3) return cudaErrorNotSupported;
  if (MODE == kGather && !prm.idx) return cudaErrorNotSupported;
  if (prm.p > (int64_t(1) << 31) - TM) return cudaErrorInvalidValue;
  EncodeFn enc = get_encode();
  if (!enc) return cudaErrorNotSupported;
  const bool fp8 = dtype == STMF_E4M3;
  CUtensorMap tmap;
  // (gathered rows: the map spans the whole storage and goes unused)
  const cuuint64_t dims[2] = {(cuuint64_t)prm.n, (cuuint64_t)(MODE == kGather ? prm.rows : prm.p)};
  const cuuint64_t strides[1] = {(cuuint64_t)prm.ld * (fp8 ? 1 : 2)};
  const cuuint32_t box[2] = {fp8 ? 128u : 64u, TM};  // 128-byte rows either way
  const cuuint32_t estr[2] = {1, 1};
  CUresult cr = enc(&tmap, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                    2, const_cast<void*>(prm.V), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const TcExtra ex = plan(prm.n, prm.r, fp8);
  if (fp8) {
    if (rp_of(prm.r) == 8) return launch_rp<8, true, MODE>(tmap, prm, ex, grid, s);
    return launch_rp<16, true, MODE>(tmap, prm, ex, grid, s);
  }
  if (rp_of(prm.r) == 8) return launch_rp<8, false, MODE>(tmap, prm, ex, grid, s);
  return launch_rp<16, false, MODE>(tmap, prm, ex, grid, s);
}

}  // namespace

cudaError_t fg_tc_launch(int dtype, const FgParams& prm, int grid, cudaStream_t s) {
  return launch_tc<kFused>(dtype, prm, grid, s);
}

cudaError_t fg_tc_rrf_launch(int dtype, const FgParams& prm, int grid, cudaStream_t s) {
  return launch_tc<kRrf>(dtype, prm, grid, s);
}

cudaError_t fg_tc_gather_launch(int dtype, const FgParams& prm, int grid, cudaStream_t s) {
  return launch_tc<kGather>(dtype, prm, grid, s);
}

}  // namespace stmf
