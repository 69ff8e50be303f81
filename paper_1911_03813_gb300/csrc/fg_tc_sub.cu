// Fused pass over samples on the 5th-generation tensor cores (tcgen05, TMA, TMEM), streaming
// each tile through a ring of sub-stages: FP32 samples (n <= 256), and BF16 or E4M3 samples with
// more features than the whole-tile pass holds (n <= 512). For the sampled evaluation of Sec. 5
// on FP32 rows idx[0..p), the converter warps copy the rows into the sub-stages themselves.
//
// Computes the same per-CTA partial sums of Alg. 2 as the whole-tile pass (Lemma 3.3, eq. Y;
// Lemma 3.5):
//     Y_part = sum_l nu_l (v_l^T A)^{d-1} v_l,      w_part_j = sum_l nu_l (v_l^T a_j)^d,
// reading every sample from HBM exactly once. A sub-stage is 32 KB of shared memory: two
// regions of 128 sample rows x 128 bytes (the 128-byte swizzle) holding BF16 values for MMAs:
//   FP32  64 features, two TMA boxes of 32 FP32 features; each value x is split in place into
//         two BF16 terms, b1 = bf16(x) and b2 = bf16(x - b1) (2^-18 relative: x - b1 is exact in
//         FP32 and b2 keeps its leading 8 bits), region g (features 32g .. 32g + 31) becoming
//         row by row [b1 of its 32 features | b2 of them]; z = b1 A + b2 A.
//   BF16  128 features, two TMA boxes of 64 BF16 features, used as they land.
//   E4M3  128 features, one TMA box of 128 codes landing in a ring of 16 KB code slots of its
//         own; the converters read a slot into registers, free it for the next copy at once and
//         write the BF16 values (every E4M3 value is a BF16 value) into both regions of a
//         sub-stage, so a copy's slot is held only while the copy is in flight and not through
//         the tile's MMAs; the per-sample scale s folds into the weight, nu' = nu s^d, so
//         z = q^T a with the codes q.
// Per sub-stage h of a tile:
//   MMA1  Z += V_h A_split(features of h)        M = 128 samples, N = 3 RP (16-padded)
//         (FP32: the b2 products N = 2 RP into their own accumulator)
//   MMA2  Y_h += V_h^T [W_hi, W_lo]               M = 128 rows of the sub-stage, N = 2 RP
// MMA2's block h reads only sub-stage h and releases it when done, so a tile needs at most four
// sub-stages at a time and the ring of six keeps the next tile streaming in. A (FP64) is split
// once per CTA into three BF16 terms A1 + A2 + A3 (2^-25 relative): the split of A is the same
// perturbation for every sample, so unlike the rounding of W and V it does not average out over
// samples, and a two-term split (2^-17) would show in the small entries of G_A. W is split per
// tile into BF16 hi/lo. The tensor cores' FP32 accumulation truncates, so every addition into an
// accumulator biases |z| low by up to an ulp of the running sum: the products go to two
// accumulators (even and odd sub-stages) and, for FP32, the b2 products, 2^-8 of the size, to a
// third, so no accumulator takes more additions than K = 256 split in two.
//
// FP32: each K step of 16 of MMA1 is either all b1 or all b2, and the rows of MMA2 block h are
// [b1 f0-31; b2 f0-31; b1 f32-63; b2 f32-63] of sub-stage h's features; BF16/E4M3: rows are
// features 128h .. 128h + 127.
//
// Warp roles (736 threads): warp 0 = TMA producer, warp 1 = TMEM allocator and MMA1 issuer,
// warp 2 = MMA2 issuer, warps 3-18 = epilogue (four warpgroups that split the components;
// thread = TMEM lane = sample of the tile, or row of an MMA2 block), warps 19-22 = converters
// (FP32 and E4M3; thread = one sample row of both regions, so the in-place rewrite never
// crosses threads). Every wait is bounded: a wait that runs out sets STMF_ETIMEOUT in the
// status word and all roles wind down, wait for their own copies and MMAs, and free TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "stmf_internal.h"
#include "tc_common.cuh"

namespace stmf {
namespace {

constexpr int TM = 128;                  // samples per tile
constexpr int REG_BYTES = TM * 128;      // one region: 128 rows of 128 bytes (16 KB)
constexpr int SUB_BYTES = 2 * REG_BYTES; // one sub-stage (two regions)
constexpr int MAX_SUB = 4;               // sub-stages per tile: n <= 256 (FP32), 512 (BF16, E4M3)
enum SubMode { kF32 = 0, kBF16 = 1, kE4M3 = 2 };
__host__ __device__ constexpr int feats_per_sub(int mode) { return mode == kF32 ? 64 : 128; }
constexpr int EG = 4;                    // epilogue warpgroups
constexpr int NEPI = 128 * EG;
constexpr int NCONV = 4;                 // converter warps: one thread per sample row
constexpr int CONV0 = 96 + NEPI;         // first converter thread
constexpr int NTHREADS = CONV0 + 32 * NCONV;
constexpr long long WAIT_LIMIT = 4000000000LL;  // SM cycles (about 2 s) before a wait gives up

struct SubExtra {
  int nsub;        // sub-stages per tile: ceil(n / features per sub-stage)
  int zbufs;       // Z buffers in TMEM: 2 where they fit beside Y, else 1
  int ring;        // sub-stage slots in shared memory
  int raw;         // E4M3 code slots (16 KB each; 0 for the other storage types)
  int wbufs;       // W buffers: 2, or 1 where a second one would cost a ring slot
  int flush;       // tiles between folds of Y into compensated FP32 registers
  int tmem_cols;
  int smem_bytes;
};

// MMA1 columns (rows of the A split, columns of Z in TMEM) are term-major: column of
// (component j, term k) = k RP + j; rows past 3 RP are zero. The b2 products use the first 2 RP
// rows (A1 and A2 only: b2 A3 is below 2^-24 of z). A warpgroup reads its CPG components of
// each term with one load of CPG columns at a multiple of CPG.
// TMEM: each Z buffer (ZBS columns) holds the b1 accumulators at columns 0 and ZS and the b2
// accumulator at 2 ZS; Y follows the Z buffers, 2 buffers x nsub blocks of N2 columns. Two Z
// buffers (MMA1 of the next tile runs while the epilogue reads this one) fit beside Y for
// n <= 128; above that there is one. Every MMA's columns start at a multiple of 2 RP and every
// load at a multiple of its width.
template <int RP>
struct Cfg32 {
  static constexpr int CPG = RP / EG;
  static constexpr int N1 = (3 * RP + 15) / 16 * 16;  // MMA1 N for b1: three terms
  static constexpr int NB2 = 2 * RP;                  // MMA1 N for b2: two terms
  static constexpr int N2 = 2 * RP;                   // MMA2 N: W hi and lo
  static constexpr int ZS = (N1 + 2 * RP - 1) / (2 * RP) * (2 * RP);  // b1 accumulator stride
  static constexpr int ZBS = 2 * ZS + NB2;            // one Z buffer: 160 or 80 columns
  static constexpr int W_REG = N2 * 128;              // one 64-sample region of W
  static constexpr int A_REG = N1 * 128;              // one 64-feature region of the A split
};

// TMEM columns of a plan: Z buffers, then 2 x nsub Y blocks.
__host__ __device__ constexpr int tmem_need(int zbs, int zbufs, int nsub, int n2) {
  return zbs * zbufs + 2 * nsub * n2;
}

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

// z of one warpgroup's CPG components from a Z buffer at `zaddr`: the b2 accumulator's two
// terms (FP32 samples only: HAS_B2), the second accumulator's three (when there is more than one
// sub-stage) and the first's three, each accumulator's terms summed smallest first, in FP32
// rounded to nearest. ONE_BY_ONE reads the accumulators one at a time (a wait each) so that at
// most three terms are live: the variant with four blocks of Y sums in registers needs that.
template <int CPG, int RP, int ZS, bool ONE_BY_ONE, bool HAS_B2>
__device__ __forceinline__ void tmem_z(uint32_t zaddr, bool two_acc, float (&z)[CPG]) {
  if constexpr (ONE_BY_ONE) {
    float v[3][CPG];
#pragma unroll
    for (int c = 0; c < CPG; ++c) z[c] = 0.f;
    if constexpr (HAS_B2) {
#pragma unroll
      for (int k = 0; k < 2; ++k) tmem_load_cols<CPG>(zaddr + uint32_t(2 * ZS + k * RP), v[k]);
      tc::tmem_ld_wait();
#pragma unroll
      for (int c = 0; c < CPG; ++c) z[c] = v[1][c] + v[0][c];
    }
    if (two_acc) {
#pragma unroll
      for (int k = 0; k < 3; ++k) tmem_load_cols<CPG>(zaddr + uint32_t(ZS + k * RP), v[k]);
      tc::tmem_ld_wait();
#pragma unroll
      for (int c = 0; c < CPG; ++c) z[c] += (v[2][c] + v[1][c]) + v[0][c];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) tmem_load_cols<CPG>(zaddr + uint32_t(k * RP), v[k]);
    tc::tmem_ld_wait();
#pragma unroll
    for (int c = 0; c < CPG; ++c) z[c] += (v[2][c] + v[1][c]) + v[0][c];
  } else {
    float v[8][CPG];
#pragma unroll
    for (int k = 0; k < 3; ++k) tmem_load_cols<CPG>(zaddr + uint32_t(k * RP), v[k]);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (two_acc) tmem_load_cols<CPG>(zaddr + uint32_t(ZS + k * RP), v[3 + k]);
    if constexpr (HAS_B2) {
#pragma unroll
      for (int k = 0; k < 2; ++k)
        tmem_load_cols<CPG>(zaddr + uint32_t(2 * ZS + k * RP), v[6 + k]);
    }
    tc::tmem_ld_wait();
#pragma unroll
    for (int c = 0; c < CPG; ++c) {
      float t = 0.f;
      if constexpr (HAS_B2) t = v[7][c] + v[6][c];
      if (two_acc) t += (v[5][c] + v[4][c]) + v[3][c];
      z[c] = t + ((v[2][c] + v[1][c]) + v[0][c]);
    }
  }
}

// Two E4M3 codes -> two BF16 values, exactly (E4M3 -> FP16 -> FP32 -> BF16; every E4M3 value
// has at most 4 significant bits and an exponent in -9..8, so no step rounds).
__device__ __forceinline__ uint32_t e4m3x2_to_bf16x2(uint16_t q) {
  const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)q, __NV_E4M3);
  const __half2 hh = *reinterpret_cast<const __half2*>(&hr);
  const __nv_bfloat162 bb = __floats2bfloat162_rn(__low2float(hh), __high2float(hh));
  return *reinterpret_cast<const uint32_t*>(&bb);
}

// Eight FP32 values -> their BF16 leading terms (b1) and BF16 remainders (b2), packed in pairs.
__device__ __forceinline__ void split8(const float (&x)[8], uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(x[2 * k], x[2 * k + 1]);
    const uint32_t u = *reinterpret_cast<const uint32_t*>(&b);
    const float r0 = x[2 * k] - __uint_as_float(u << 16);          // exact
    const float r1 = x[2 * k + 1] - __uint_as_float(u & 0xFFFF0000u);
    const __nv_bfloat162 c = __floats2bfloat162_rn(r0, r1);
    h[k] = u;
    l[k] = *reinterpret_cast<const uint32_t*>(&c);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
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

__device__ __forceinline__ void epi_barrier() {
  asm volatile("bar.sync 1, %0;" ::"n"(NEPI) : "memory");
}

// NS: sub-stages per tile the epilogue keeps Y sums for (1, 2 or 4; at least ex.nsub).
// MODE: the storage type of the samples (SubMode).
// GATHER: sampled FP32 rows idx[0..p) (Sec. 5, Lemma 5.1), fetched by the converter warps in
//         place of TMA.
template <int RP, int NS, int MODE, bool GATHER>
__global__ void __launch_bounds__(NTHREADS, 1)
    fg_tc_sub_kernel(const __grid_constant__ CUtensorMap tmap, const FgParams prm,
                     const SubExtra ex) {
  static_assert(!GATHER || MODE == kF32, "gathered rows: FP32 samples");
  constexpr int FS = feats_per_sub(MODE);  // features per sub-stage
  constexpr int AR = FS / 64;              // A-split regions per sub-stage
  constexpr bool CONVERT = MODE != kBF16;  // converter warps rewrite each sub-stage
  using C = Cfg32<RP>;
  constexpr int N1 = C::N1;
  constexpr int N2 = C::N2;
  constexpr int CPG = C::CPG;
  constexpr int ZS = C::ZS;
  const int ZBUF = ex.zbufs;
  const uint32_t YB0 = uint32_t(C::ZBS * ZBUF);  // first Y column
  if (prm.skip && *prm.skip) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw_addr = tc::smem_addr(smem_raw);
  unsigned char* base = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);

  const int R = ex.ring, nsub = ex.nsub, WB = ex.wbufs;
  const int RR = MODE == kE4M3 ? ex.raw : 0;  // E4M3 code slots
  const int NF = MODE == kE4M3 ? RR : R;      // slots the TMA copies land in
  const int n = prm.n, r = prm.r, d = prm.d;
  unsigned char* sV = base;                              // ring of R sub-stages
  unsigned char* sRaw = sV + size_t(R) * SUB_BYTES;      // RR code slots (E4M3)
  unsigned char* sW = sRaw + size_t(RR) * REG_BYTES;     // WB buffers x 2 regions
  unsigned char* sA = sW + size_t(WB) * 2 * C::W_REG;    // nsub x AR regions
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA + size_t(nsub * AR) * C::A_REG);
  uint64_t* full = bars;            // [NF] TMA landed (in a sub-stage, or an E4M3 code slot)
  uint64_t* conv = full + NF;       // [R] rewritten as BF16 (FP32, E4M3)
  uint64_t* empty = conv + R;       // [R] MMA2 done with the sub-stage
  uint64_t* rawfree = empty + R;    // [RR] the converters have read the code slot
  uint64_t* zfull = rawfree + RR;   // [ZBUF]
  uint64_t* zempty = zfull + 2;
  uint64_t* wfull = zempty + 2;
  uint64_t* wempty = wfull + 2;
  uint64_t* yfull = wempty + 2;
  uint64_t* yempty = yfull + 2;
  uint64_t* mma_done = yempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 2);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  double* wred = reinterpret_cast<double*>(mma_done + 3);  // 4 x RP

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < NF; ++s) tc::mbar_init(&full[s], 1);
    for (int s = 0; s < R; ++s) {
      tc::mbar_init(&conv[s], NCONV);
      tc::mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < RR; ++s) tc::mbar_init(&rawfree[s], NCONV);
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&zfull[b], 1);
      tc::mbar_init(&zempty[b], NEPI / 32);
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

  // A split: row k RP + j holds term k of a_j, with A1 = BF16(a), A2 = BF16(a - A1),
  // A3 = BF16(a - A1 - A2) (rows past 3 RP are zero), in regions of 64 features (FP32: region h
  // serves the b1 and the b2 half of sub-stage h)
  {
    const int kext = nsub * FS;
    for (int e = tid; e < N1 * kext; e += NTHREADS) {
      const int row = e / kext, k = e - row * kext;
      const int term = row / RP, j = row % RP;
      const double a = (term < 3 && j < r && k < n) ? prm.A[k + size_t(n) * j] : 0.0;
      const double a1 = (double)__bfloat162float(__double2bfloat16(a));
      const double a2 = (double)__bfloat162float(__double2bfloat16(a - a1));
      const double v = term == 0 ? a1 : term == 1 ? a2 : a - a1 - a2;
      *reinterpret_cast<__nv_bfloat16*>(sA + (k >> 6) * C::A_REG + tc::sw128_offset(row, k & 63)) =
          __double2bfloat16(v);
    }
  }
  tc::fence_proxy_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int64_t num_tiles = (prm.p + TM - 1) / TM;
  const int my_tiles = (int)((num_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
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
      int issued = 0;
      bool ok = true;
      for (int it = 0; it < my_tiles && ok; ++it) {
        const int64_t tile = blockIdx.x + int64_t(it) * gridDim.x;
        for (int h = 0; h < nsub; ++h) {
          const int slot = issued % NF;
          // E4M3: the code slot is free once the converters have read it; otherwise the
          // sub-stage is free once MMA2 is done with it
          uint64_t* freed = MODE == kE4M3 ? &rawfree[slot] : &empty[slot];
          if (!tc::mbar_wait_sleep(freed, ((issued / NF) & 1) ^ 1, abortv, WAIT_LIMIT)) {
            fail();
            ok = false;
            break;
          }
          const int32_t y0 = (int32_t)(tile * TM);
          if constexpr (MODE == kE4M3) {  // 128 codes per row, into a code slot
            tc::mbar_arrive_expect_tx(&full[slot], REG_BYTES);
            tc::tma_load_2d(sRaw + size_t(slot) * REG_BYTES, &tmap, FS * h, y0, &full[slot]);
          } else {  // two boxes of FS / 2 features (128-byte rows)
            unsigned char* dst = sV + size_t(slot) * SUB_BYTES;
            tc::mbar_arrive_expect_tx(&full[slot], SUB_BYTES);
            tc::tma_load_2d(dst, &tmap, FS * h, y0, &full[slot]);
            tc::tma_load_2d(dst + REG_BYTES, &tmap, FS * h + FS / 2, y0, &full[slot]);
          }
          ++issued;
        }
      }
      // wait for the last copy issued into each slot (already complete unless we aborted)
      for (int k = issued > NF ? issued - NF : 0; k < issued; ++k)
        tc::mbar_wait_sleep(&full[k % NF], (k / NF) & 1, &no_abort, WAIT_LIMIT);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA1 issuer
    // Z(t) = sum over sub-stages of b1 A_split(h) (accumulator h % 2) and b2 [A1, A2](h) (the
    // third accumulator), as each sub-stage is split and the Z buffer has been read.
    if (lane == 0) {
      const uint32_t idesc_b1 = tc::idesc_bf16(128, N1, 0, 0);
      const uint32_t idesc_b2 = tc::idesc_bf16(128, C::NB2, 0, 0);
      // Shared-memory descriptors are linear in the operand address (its 16-byte units sit in
      // the low bits and every address here is below 256 KB): one base per operand plus
      // (byte offset >> 4), so the issuing thread spends one add per MMA.
      const uint64_t vdesc0 = tc::sdesc_sw128(tc::smem_addr(sV), 16, 1024);
      const uint64_t adesc0 = tc::sdesc_sw128(tc::smem_addr(sA), 16, 1024);
      bool ok = true;
      int seq = 0;
      for (int t = 0; t < my_tiles && ok; ++t) {
        const int zb = t % ZBUF;
        ok = tc::mbar_wait_sleep(&zempty[zb], ((t / ZBUF) & 1) ^ 1, abortv, WAIT_LIMIT);
        uint32_t written = 0;
        for (int h = 0; h < nsub && ok; ++h, ++seq) {
          const int slot = seq % R;
          ok = tc::mbar_wait_sleep(CONVERT ? &conv[slot] : &full[slot], (seq / R) & 1, abortv,
                                   WAIT_LIMIT);
          if (!ok) break;
          tc::tc_fence_after();
          const uint64_t vd = vdesc0 + uint64_t((uint32_t(slot) * SUB_BYTES) >> 4);
          const uint64_t ad0 = adesc0 + uint64_t((uint32_t(h * AR) * C::A_REG) >> 4);
          if constexpr (MODE == kF32) {
            // K step kk of region g: kk = 0, 1 are b1, kk = 2, 3 b2, of features 32g + 16 (kk % 2)
#pragma unroll
            for (int part = 0; part < 2; ++part) {
              const int acc = part == 0 ? (h & 1) : 2;
              const uint32_t dZ = tmem + uint32_t(zb * C::ZBS + acc * ZS);
              const uint32_t idesc = part == 0 ? idesc_b1 : idesc_b2;
              const uint32_t first = (written >> acc) & 1u;
#pragma unroll
              for (int g = 0; g < 2; ++g)
#pragma unroll
                for (int kk = 0; kk < 2; ++kk)
                  tc::mma_bf16(dZ, vd + uint64_t((g * REG_BYTES + (2 * part + kk) * 32) >> 4),
                               ad0 + uint64_t(((2 * g + kk) * 32) >> 4), idesc,
                               (g | kk) ? 1u : first);
              written |= 1u << acc;
            }
          } else {
            // region g holds features 64g .. 64g + 63 of the sub-stage, A-split region 2h + g
            const int acc = h & 1;
            const uint32_t dZ = tmem + uint32_t(zb * C::ZBS + acc * ZS);
            const uint32_t first = (written >> acc) & 1u;
#pragma unroll
            for (int g = 0; g < 2; ++g)
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                tc::mma_bf16(dZ, vd + uint64_t((g * REG_BYTES + kk * 32) >> 4),
                             ad0 + uint64_t((g * C::A_REG + kk * 32) >> 4), idesc_b1,
                             (g | kk) ? 1u : first);
            written |= 1u << acc;
          }
        }
        if (!ok) break;
        tc::mma_commit(&zfull[zb]);
      }
      if (!ok) fail();
      tc::mma_commit(&mma_done[0]);
      tc::mbar_wait_sleep(&mma_done[0], 0, &no_abort, WAIT_LIMIT);
    }
  } else if (warp == 2) {
    // ------------------------------------------------------------------ MMA2 issuer
    // Y_h += [b1 ; b2]^T [W_hi | W_lo] per sub-stage h once W(t) is written; the completion of
    // block h frees sub-stage h for the producer.
    if (lane == 0) {
      const uint32_t idesc2 = tc::idesc_bf16(128, N2, 1, 0);  // V^T MN-major, W K-major
      const uint64_t vdesc0 = tc::sdesc_sw128(tc::smem_addr(sV), REG_BYTES, 1024);
      const uint64_t wdesc0 = tc::sdesc_sw128(tc::smem_addr(sW), 16, 1024);
      bool ok = true;
      int seq = 0;
      for (int t = 0; t < my_tiles; ++t) {
        const int wb = t % WB;
        const int period = t / flush, yb = period & 1;
        const bool first = (t % flush) == 0;
        if (first) ok = tc::mbar_wait_sleep(&yempty[yb], ((period >> 1) & 1) ^ 1, abortv, WAIT_LIMIT);
        ok = ok && tc::mbar_wait_sleep(&wfull[wb], (t / WB) & 1, abortv, WAIT_LIMIT);
        if (!ok) break;
        tc::tc_fence_after();
        const uint64_t wd = wdesc0 + uint64_t((uint32_t(wb) * 2 * C::W_REG) >> 4);
        for (int h = 0; h < nsub; ++h, ++seq) {
          const int slot = seq % R;
          const uint64_t vd = vdesc0 + uint64_t((uint32_t(slot) * SUB_BYTES) >> 4);
          const uint32_t dY = tmem + YB0 + uint32_t((yb * nsub + h) * N2);
#pragma unroll
          for (int kk = 0; kk < TM / 16; ++kk)
            tc::mma_bf16(dY, vd + uint64_t((kk * 2048) >> 4),
                         wd + uint64_t(((kk >> 2) * C::W_REG + (kk & 3) * 32) >> 4), idesc2,
                         (first && kk == 0) ? 0u : 1u);
          tc::mma_commit(&empty[slot]);
        }
        tc::mma_commit(&wempty[wb]);
        if ((t % flush) == flush - 1 || t == my_tiles - 1) tc::mma_commit(&yfull[yb]);
      }
      if (!ok) fail();
      tc::mma_commit(&mma_done[1]);
      tc::mbar_wait_sleep(&mma_done[1], 0, &no_abort, WAIT_LIMIT);
    }
  } else if (tid >= CONV0) {
    // ------------------------------------------------------------------ converters
    // Thread y owns row y (sample y of the tile) of both regions of every sub-stage; only this
    // thread touches the row, so nothing else reads the bytes it overwrites (16-byte chunk c of
    // row y sits at chunk position c ^ (y & 7) in either layout).
    // FP32: per region, the 32 FP32 values of the row become b1 of the 32 features (BF16 chunks
    //       0-3) and b2 (chunks 4-7).
    // E4M3: the 128 codes of the row (row y of a code slot, the same swizzle) are read into
    //       registers, the slot is released, and once MMA2 is done with the sub-stage's last use
    //       they are written as the BF16 values of features 0-63 (region 0) and 64-127
    //       (region 1).
    if constexpr (CONVERT) {
      const int y = tid - CONV0;
      const uint32_t sw = uint32_t(y & 7);
      // FP32: row y of both regions of sub-stage `slot`, split in place
      auto split_row = [&](int slot) {
        unsigned char* row0 = sV + size_t(slot) * SUB_BYTES + y * 128;
#pragma unroll 1
        for (int rg = 0; rg < 2; ++rg) {
          unsigned char* row = row0 + size_t(rg) * REG_BYTES;
          float x[8][4];
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float4 a = *reinterpret_cast<const float4*>(row + ((c ^ sw) << 4));
            x[c][0] = a.x; x[c][1] = a.y; x[c][2] = a.z; x[c][3] = a.w;
          }
#pragma unroll
          for (int k = 0; k < 4; ++k) {  // features 8k .. 8k + 7 of the region
            const float v[8] = {x[2 * k][0],     x[2 * k][1],     x[2 * k][2],
                                x[2 * k][3],     x[2 * k + 1][0], x[2 * k + 1][1],
                                x[2 * k + 1][2], x[2 * k + 1][3]};
            uint4 hi, lo;
            split8(v, hi, lo);
            *reinterpret_cast<uint4*>(row + ((uint32_t(k) ^ sw) << 4)) = hi;
            *reinterpret_cast<uint4*>(row + ((uint32_t(4 + k) ^ sw) << 4)) = lo;
          }
        }
      };
      bool ok = true;
      if constexpr (GATHER) {
        // Sampled FP32 rows (Sec. 5): the converter warps fetch the rows themselves. Warp w
        // holds rows y = 32 w + l of every tile (lane l: the row index of sample y, read one
        // tile ahead); one warp instruction copies the sub-stage's 256-byte slices of two rows
        // (lanes 0-15 and 16-31, 16-byte chunk q = features 4q .. 4q + 3 of the sub-stage:
        // region q / 8, chunk q % 8 at position (q % 8) ^ (y & 7) of the 128-byte swizzle).
        // Features past n and rows past p are zero-filled; a row outside the storage reads as
        // zero and sets STMF_EINVAL. Sub-stage k + 1 is requested before sub-stage k is split:
        // each thread waits for its own copies of k, the warp syncs (its rows are complete),
        // every thread splits its row, fences to the async proxy, and the warp arrives.
        const int w = y >> 5, half = lane >> 4, q = lane & 15;
        const float* Vg = static_cast<const float*>(prm.V);
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
        auto finish = [&](int seq_) {
          __syncwarp();
          split_row(seq_ % R);
          tc::fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&conv[seq_ % R]);
        };
        int64_t row_cur = -1, row_next = row_of(0);
        int seq = 0;
        for (int it = 0; it < my_tiles && ok; ++it) {
          row_cur = row_next;
          row_next = row_of(it + 1);
          for (int h = 0; h < nsub; ++h, ++seq) {
            const int slot = seq % R;
            ok = tc::mbar_wait_sleep(&empty[slot], ((seq / R) & 1) ^ 1, abortv, WAIT_LIMIT);
            if (!__all_sync(0xffffffffu, ok)) {
              ok = false;
              break;
            }
            const uint32_t base = tc::smem_addr(sV + size_t(slot) * SUB_BYTES);
            const int f = FS * h + 4 * q;
            const int fv = n - f >= 4 ? 4 : (n - f > 0 ? n - f : 0);
#pragma unroll 4
            for (int i = 0; i < 16; ++i) {
              const int yy = 32 * w + 2 * i + half;
              const int64_t row = __shfl_sync(0xffffffffu, row_cur, 2 * i + half);
              const int nb = row < 0 ? 0 : fv;
              const float* src = nb ? Vg + row * prm.ld + f : Vg;
              cp_async16(base + uint32_t(q >> 3) * REG_BYTES + uint32_t(yy) * 128u +
                             ((uint32_t(q & 7) ^ uint32_t(yy & 7)) << 4),
                         src, uint32_t(4 * nb));
            }
            cp_async_commit();
            if (seq >= 1) {
              cp_async_wait<1>();
              finish(seq - 1);
            }
          }
        }
        cp_async_wait<0>();  // nothing of this thread's stays in flight past here
        if (ok && seq >= 1) finish(seq - 1);
      } else {
      int seq = 0;
      for (int it = 0; it < my_tiles && ok; ++it) {
        for (int h = 0; h < nsub; ++h, ++seq) {
          const int slot = seq % R;
          const int fs = seq % NF;
          if (!tc::mbar_wait_sleep(&full[fs], (seq / NF) & 1, abortv, WAIT_LIMIT)) {
            ok = false;
            break;
          }
          if constexpr (MODE == kF32) {
            split_row(slot);
          } else {
            unsigned char* row0 = sV + size_t(slot) * SUB_BYTES + y * 128;
            unsigned char* row1 = row0 + REG_BYTES;
            const unsigned char* src = sRaw + size_t(fs) * REG_BYTES + y * 128;
            uint4 raw[8];
#pragma unroll
            for (int c = 0; c < 8; ++c)
              raw[c] = *reinterpret_cast<const uint4*>(src + ((uint32_t(c) ^ sw) << 4));
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&rawfree[fs]);
            if (!tc::mbar_wait_sleep(&empty[slot], ((seq / R) & 1) ^ 1, abortv, WAIT_LIMIT)) {
              ok = false;
              break;
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {  // codes 16c .. 16c + 15 -> BF16 chunks 2c, 2c + 1
              unsigned char* dst = (c < 4) ? row0 : row1;
              const uint32_t k0 = uint32_t(2 * (c & 3));
              const uint32_t w[4] = {raw[c].x, raw[c].y, raw[c].z, raw[c].w};
              uint32_t o[8];
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                o[2 * k] = e4m3x2_to_bf16x2((uint16_t)(w[k] & 0xFFFFu));
                o[2 * k + 1] = e4m3x2_to_bf16x2((uint16_t)(w[k] >> 16));
              }
              *reinterpret_cast<uint4*>(dst + ((k0 ^ sw) << 4)) = make_uint4(o[0], o[1], o[2], o[3]);
              *reinterpret_cast<uint4*>(dst + (((k0 + 1) ^ sw) << 4)) =
                  make_uint4(o[4], o[5], o[6], o[7]);
            }
          }
          tc::fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&conv[slot]);
        }
      }
      }
      if (!ok) fail();
    }
  } else {
    // ------------------------------------------------------------------ epilogue
    const int g = (warp - 3) >> 2;
    const int q = warp & 3;            // TMEM lane quarter this warp may access
    const int L = 32 * q + lane;       // sample within the tile / row within an MMA2 block
    const int j0 = g * CPG;
    const uint32_t lane_off = uint32_t(32 * q) << 16;
    float wacc[CPG], ws[CPG], wc[CPG], ys[NS][CPG], yc[NS][CPG];
#pragma unroll
    for (int c = 0; c < CPG; ++c) {
      wacc[c] = ws[c] = wc[c] = 0.f;
#pragma unroll
      for (int h = 0; h < NS; ++h) ys[h][c] = yc[h][c] = 0.f;
    }
    const uint32_t wcol = uint32_t(L >> 6) * C::W_REG;
    int pending = -1;
    auto fold = [&](int per, bool force) -> bool {
      const int yb = per & 1;
      const uint32_t par = (per >> 1) & 1;
      if (!tc::mbar_test_wait(&yfull[yb], par)) {
        if (!force) return true;
        if (!tc::mbar_wait_sleep(&yfull[yb], par, abortv, WAIT_LIMIT)) return false;
      }
      tc::tc_fence_after();
#pragma unroll
      for (int h = 0; h < NS; ++h) {
        if (h < nsub) {
          float yv[2 * CPG];
          tmem_load_cols<2 * CPG>(
              tmem + YB0 + uint32_t((yb * nsub + h) * N2 + 2 * j0) + lane_off, yv);
          tc::tmem_ld_wait();
#pragma unroll
          for (int c = 0; c < CPG; ++c) {
            kahan_add(ys[h][c], yc[h][c], yv[c]);
            kahan_add(ys[h][c], yc[h][c], yv[CPG + c]);
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
    float sc_next = 1.f;
    auto weight_of = [&](int it_) -> float {
      const int64_t sidx_ = (blockIdx.x + int64_t(it_) * gridDim.x) * TM + L;
      if (it_ >= my_tiles || sidx_ >= prm.p) return 0.f;
      if constexpr (MODE == kE4M3) sc_next = prm.scale[sidx_];
      return prm.nu ? (float)prm.nu[sidx_] : (float)prm.nu_uniform;
    };
    float nu_next = weight_of(0);
    bool ok = true;
    for (int it = 0; it < my_tiles; ++it) {
      const int wb = it % WB, zb = it % ZBUF;
      float nu_s = nu_next;
      if constexpr (MODE == kE4M3) {  // nu' = nu s^d: the sample's scale folded into its weight
        const float sc = sc_next;
        float sd = sc;
        for (int e = 1; e < d; ++e) sd *= sc;
        nu_s *= sd;
      }
      nu_next = weight_of(it + 1);
      if (!tc::mbar_wait_sleep(&zfull[zb], (it / ZBUF) & 1, abortv, WAIT_LIMIT)) {
        ok = false;
        break;
      }
      tc::tc_fence_after();
      float zsum[CPG];
      tmem_z<CPG, RP, ZS, (NS > 2), MODE == kF32>(tmem + uint32_t(zb * C::ZBS + j0) + lane_off,
                                                  nsub > 1, zsum);
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&zempty[zb]);
      float wv[CPG];
#pragma unroll
      for (int c = 0; c < CPG; ++c) {
        const float zz = zsum[c];
        const float t = ipow_f(zz, d - 1);
        wv[c] = nu_s * t;
        wacc[c] += wv[c] * zz;
      }
      if (!tc::mbar_wait_sleep(&wempty[wb], ((it / WB) & 1) ^ 1, abortv, WAIT_LIMIT)) {
        ok = false;
        break;
      }
      unsigned char* wbuf = sW + size_t(wb) * 2 * C::W_REG + wcol;
#pragma unroll
      for (int c = 0; c < CPG; ++c) {
        const __nv_bfloat16 hi = __float2bfloat16_rn(wv[c]);
        const __nv_bfloat16 lo = __float2bfloat16_rn(wv[c] - __bfloat162float(hi));
        *reinterpret_cast<__nv_bfloat16*>(wbuf + tc::sw128_offset(2 * j0 + c, L & 63)) = hi;
        *reinterpret_cast<__nv_bfloat16*>(wbuf + tc::sw128_offset(2 * j0 + CPG + c, L & 63)) = lo;
      }
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&wfull[wb]);
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
    // FP32: lane quarter q of MMA2 block h holds part q % 2 (b1, b2) of features
    // 64h + 32 (q / 2) + lane: the b2 quarters pass their sums to the b1 quarters of the same
    // warpgroup through shared memory (the ring is idle by now: every copy has landed and every
    // MMA has completed once the last fold is done). Every epilogue thread reaches the barrier,
    // also after a failed wait. BF16 / E4M3: lane L of block h holds feature FS h + L.
    const int fi = MODE == kF32 ? 32 * (q >> 1) + lane : L;  // feature within the sub-stage
    const bool writer = MODE == kF32 ? !(q & 1) : true;
    double* xch = reinterpret_cast<double*>(sV);  // [NS][64][RP]
    if (MODE == kF32 && ok && (q & 1)) {
#pragma unroll
      for (int h = 0; h < NS; ++h)
        if (h < nsub) {
#pragma unroll
          for (int c = 0; c < CPG; ++c)
            xch[(h * 64 + fi) * RP + j0 + c] = (double)ys[h][c] - (double)yc[h][c];
        }
    }
    epi_barrier();
    if (!ok) {
      fail();
    } else {
      double* part = prm.partials + size_t(blockIdx.x) * (size_t(r) + size_t(n) * r);
      // First-order correction of w for the split of A (as in the BF16 pass):
      // sum nu z^d = sum nu z^^d + d sum_i Y_ij dA_ij + O(|dA|^2) with z^ from A1 + A2 + A3.
      double corr[CPG];
#pragma unroll
      for (int c = 0; c < CPG; ++c) corr[c] = 0.0;
      if (writer) {
#pragma unroll
        for (int h = 0; h < NS; ++h) {
          const int i = FS * h + fi;
          if (h < nsub && i < n) {
#pragma unroll
            for (int c = 0; c < CPG; ++c)
              if (j0 + c < r) {
                const double y = ((double)ys[h][c] - (double)yc[h][c]) +
                                 (MODE == kF32 ? xch[(h * 64 + fi) * RP + j0 + c] : 0.0);
                part[r + i + size_t(n) * (j0 + c)] = y;
                const double a = prm.A[i + size_t(n) * (j0 + c)];
                const double a1 = (double)__bfloat162float(__double2bfloat16(a));
                const double a2 = (double)__bfloat162float(__double2bfloat16(a - a1));
                const double a3 = (double)__bfloat162float(__double2bfloat16(a - a1 - a2));
                corr[c] += y * (((a - a1) - a2) - a3);
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

EncodeFn get_encode_sub() {
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

int mode_of(int dtype) {
  return dtype == STMF_F32 ? kF32 : dtype == STMF_BF16 ? kBF16 : dtype == STMF_E4M3 ? kE4M3 : -1;
}

SubExtra plan_sub(int mode, int n, int r) {
  SubExtra ex{};
  const int fs = feats_per_sub(mode);
  ex.nsub = (n + fs - 1) / fs;
  const int RP = rp_of(r), N1 = (3 * RP + 15) / 16 * 16, N2 = 2 * RP;
  const int a_bytes = ex.nsub * (fs / 64) * N1 * 128;
  // W buffers, E4M3 code slots, A split, 1024 bytes of alignment slack and 1024 of barriers and w
  // sums. A second W buffer lets the epilogue write W(t+1) while MMA2 still reads W(t); the ring
  // wants six sub-stages (FP32, BF16: each is held from its copy to its MMA2 block) or two tiles'
  // worth (E4M3: copies land in the code slots, so a sub-stage is held only from its widening
  // on); E4M3 takes as many code slots (copies in flight) as fit beside that.
  static const int kRawE4M3[3] = {4, 3, 2}, kRawNone[1] = {0};
  const int* raw_opts = mode == kE4M3 ? kRawE4M3 : kRawNone;
  const int n_raw = mode == kE4M3 ? 3 : 1;
  const int want = mode == kE4M3 ? 2 * ex.nsub : 6;
  int best = -1;
  for (int k = 0; k < n_raw; ++k) {
    const int rr = raw_opts[k];
    for (int wb = 2; wb >= 1; --wb) {
      const int fixed = wb * 2 * N2 * 128 + a_bytes + rr * REG_BYTES + 1024 + 1024;
      int R = (int(kMaxSmem) - fixed) / SUB_BYTES;
      if (R > 8) R = 8;
      if (R < 1) continue;
      const int score = (R < want ? R : want) * 100 + rr * 10 + wb;
      if (score > best) {
        best = score;
        ex.ring = R;
        ex.raw = rr;
        ex.wbufs = wb;
        ex.smem_bytes = fixed + R * SUB_BYTES;
      }
    }
  }
  ex.flush = 8;
  const int zbs = 2 * ((N1 + 2 * RP - 1) / (2 * RP) * (2 * RP)) + 2 * RP;
  ex.zbufs = tmem_need(zbs, 2, ex.nsub, N2) <= 512 ? 2 : 1;
  const int cols = tmem_need(zbs, ex.zbufs, ex.nsub, N2);
  int pow2 = 32;
  while (pow2 < cols) pow2 <<= 1;
  ex.tmem_cols = pow2;
  return ex;
}

template <int RP, int NS, int MODE, bool GATHER>
cudaError_t launch_sub(const CUtensorMap& tmap, const FgParams& prm, const SubExtra& ex, int grid,
                       cudaStream_t s) {
  const cudaError_t e =
      smem_limit((const void*)fg_tc_sub_kernel<RP, NS, MODE, GATHER>, (int)kMaxSmem);
  if (e != cudaSuccess) return e;
  return launch_kernel(fg_tc_sub_kernel<RP, NS, MODE, GATHER>, dim3(grid), dim3(NTHREADS),
                       size_t(ex.smem_bytes), s, tmap, prm, ex);
}

template <int RP, int MODE, bool GATHER>
cudaError_t launch_sub_ns(const CUtensorMap& tmap, const FgParams& prm, const SubExtra& ex,
                          int grid, cudaStream_t s) {
  if (ex.nsub == 1) return launch_sub<RP, 1, MODE, GATHER>(tmap, prm, ex, grid, s);
  if (ex.nsub == 2) return launch_sub<RP, 2, MODE, GATHER>(tmap, prm, ex, grid, s);
  return launch_sub<RP, 4, MODE, GATHER>(tmap, prm, ex, grid, s);
}

template <int MODE, bool GATHER>
cudaError_t launch_sub_rp(const CUtensorMap& tmap, const FgParams& prm, const SubExtra& ex,
                          int grid, cudaStream_t s) {
  if (rp_of(prm.r) == 8) return launch_sub_ns<8, MODE, GATHER>(tmap, prm, ex, grid, s);
  return launch_sub_ns<16, MODE, GATHER>(tmap, prm, ex, grid, s);
}

}  // namespace

bool fg_tc_sub_supported(int dtype, int n, int r) {
  const int mode = mode_of(dtype);
  if (mode < 0) return false;
  if (r < 1 || r > 16 || n < 1 || n > feats_per_sub(mode) * MAX_SUB) return false;
  if (!get_encode_sub()) return false;
  const SubExtra ex = plan_sub(mode, n, r);
  // the exchange at the end of the FP32 epilogue reuses the ring: MAX_SUB x 64 x 16 doubles
  return ex.ring >= ex.nsub && ex.ring * SUB_BYTES >= MAX_SUB * 64 * 16 * 8;
}

int fg_tc_sub_grid(int64_t p, int num_sms, int min_tiles) {
  // one CTA per SM, or fewer so that each takes at least min_tiles tiles (a CTA holds a whole SM
  // through its shared memory, so a small pass spread over every SM keeps concurrent passes off
  // the GPU while it runs one or two tiles per SM)
  const int64_t tiles = (p + TM - 1) / TM;
  const int64_t mt = min_tiles > 1 ? min_tiles : 1;
  const int64_t want = (tiles + mt - 1) / mt;
  return (int)(want < num_sms ? want : num_sms);
}

namespace {

template <bool GATHER>
cudaError_t launch_any(int dtype, const FgParams& prm, int grid, cudaStream_t s) {
  const int mode = mode_of(dtype);
  if (mode < 0) return cudaErrorNotSupported;
  if (GATHER && (mode != kF32 || !prm.idx)) return cudaErrorNotSupported;
  if (prm.p > (int64_t(1) << 31) - TM) return cudaErrorInvalidValue;
  EncodeFn enc = get_encode_sub();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap tmap;
  const int eb = mode == kF32 ? 4 : mode == kBF16 ? 2 : 1;
  // (gathered rows: the map spans the whole storage and goes unused)
  const cuuint64_t dims[2] = {(cuuint64_t)prm.n, (cuuint64_t)(GATHER ? prm.rows : prm.p)};
  const cuuint64_t strides[1] = {(cuuint64_t)prm.ld * eb};
  const cuuint32_t box[2] = {128u / eb, TM};  // 128-byte rows
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = mode == kF32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : mode == kBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  CUresult cr = enc(&tmap, dt, 2, const_cast<void*>(prm.V), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const SubExtra ex = plan_sub(mode, prm.n, prm.r);
  if constexpr (GATHER) {
    // the converters finish sub-stage k after requesting k + 1, which needs the ring to hold a
    // whole tile beyond it
    if (ex.ring < ex.nsub + 1) return cudaErrorNotSupported;
    return launch_sub_rp<kF32, true>(tmap, prm, ex, grid, s);
  } else {
    if (mode == kF32) return launch_sub_rp<kF32, false>(tmap, prm, ex, grid, s);
    if (mode == kBF16) return launch_sub_rp<kBF16, false>(tmap, prm, ex, grid, s);
    return launch_sub_rp<kE4M3, false>(tmap, prm, ex, grid, s);
  }
}

}  // namespace

cudaError_t fg_tc_sub_launch(int dtype, const FgParams& prm, int grid, cudaStream_t s) {
  return launch_any<false>(dtype, prm, grid, s);
}

cudaError_t fg_tc_sub_gather_launch(int dtype, const FgParams& prm, int grid, cudaStream_t s) {
  return launch_any<true>(dtype, prm, grid, s);
}

bool fg_tc_sub_gather_supported(int dtype, int n, int r) {
  if (dtype != STMF_F32 || !fg_tc_sub_supported(dtype, n, r)) return false;
  const SubExtra ex = plan_sub(kF32, n, r);
  return ex.ring >= ex.nsub + 1;
}

}  // namespace stmf
