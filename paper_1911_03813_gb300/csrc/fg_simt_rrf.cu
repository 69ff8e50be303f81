// Randomized range finder (eq. rrf) on the CUDA cores: A0 = V Omega with the test matrix drawn in
// the pass (the RRF variant of the kernel in fg_simt_kernel.cuh).
#include "fg_simt_kernel.cuh"

namespace stmf {

int rrf_grid(int, int n, int r, int64_t p, int num_sms, bool f64) {
  // each variant takes the grid of its accumulator type (FP64: one block per SM; FP32: up to two)
  return fg_simt_grid(f64 ? STMF_F64 : STMF_F32, n, r, p, num_sms);
}

cudaError_t rrf_launch(int dtype, const FgParams& prm, int grid, cudaStream_t s, bool f64) {
  if (f64) {
    switch (dtype) {
      case STMF_F64: return launch_rrf<double, STMF_F64>(prm, grid, s);
      case STMF_F32: return launch_rrf<double, STMF_F32>(prm, grid, s);
      case STMF_BF16: return launch_rrf<double, STMF_BF16>(prm, grid, s);
      case STMF_E4M3: return launch_rrf<double, STMF_E4M3>(prm, grid, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (dtype) {
    case STMF_F32: return launch_rrf<float, STMF_F32>(prm, grid, s);
    case STMF_BF16: return launch_rrf<float, STMF_BF16>(prm, grid, s);
    case STMF_E4M3: return launch_rrf<float, STMF_E4M3>(prm, grid, s);
    default: return cudaErrorInvalidValue;  // FP64 samples need the FP64 variant
  }
}

}  // namespace stmf
