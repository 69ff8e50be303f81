// Host side of the CUDA-core fused pass: shared memory, grid, and the launch for FP32, BF16 and
// E4M3 samples (FP64 samples: fg_simt_f64.cu). The kernel is in fg_simt_kernel.cuh.
#include "fg_simt_kernel.cuh"

namespace stmf {

size_t fg_simt_smem(int dtype, int n, int r) {
  const int rp = (r + 3) / 4 * 4;
  // the block's threads hold all n x rp entries of Y in registers: NT * MAXACC of them at most
  if (size_t(n) * size_t(rp) > size_t(NT) * MAXACC) return ~size_t(0);
  return dtype == STMF_F64 ? smem_bytes<double>(n, rp, tile_of<double>(n, rp))
                           : smem_bytes<float>(n, rp, TS_MAX);
}

int fg_simt_grid(int dtype, int n, int r, int64_t p, int num_sms) {
  const int rp = (r + 3) / 4 * 4;
  const int TS = dtype == STMF_F64 ? tile_of<double>(n, rp) : TS_MAX;
  const size_t smem = dtype == STMF_F64 ? smem_bytes<double>(n, rp, TS) : smem_bytes<float>(n, rp, TS);
  // blocks per SM bounded by shared memory (228 KB per SM) and registers (1 or 2 per SM)
  int per_sm = (int)((228 * 1024) / (smem + 1024));
  const int reg_cap = dtype == STMF_F64 ? 1 : 2;
  per_sm = per_sm < 1 ? 1 : (per_sm > reg_cap ? reg_cap : per_sm);
  const int64_t tiles = (p + TS - 1) / TS;
  int64_t grid = int64_t(num_sms) * per_sm;
  if (grid > tiles) grid = tiles;
  return (int)(grid < 1 ? 1 : grid);
}

cudaError_t fg_simt_launch(int dtype, const FgParams& prm, int grid, cudaStream_t s) {
  switch (dtype) {
    case STMF_F64: return fg_simt_launch_f64(prm, grid, s);
    case STMF_F32: return launch_jb<float, STMF_F32>(prm, grid, s);
    case STMF_BF16: return launch_jb<float, STMF_BF16>(prm, grid, s);
    case STMF_E4M3: return launch_jb<float, STMF_E4M3>(prm, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace stmf
