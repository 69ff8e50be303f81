// The CUDA-core fused pass for FP64 samples (FP64 arithmetic; 64- or 32-sample tiles).
#include "fg_simt_kernel.cuh"

namespace stmf {

cudaError_t fg_simt_launch_f64(const FgParams& prm, int grid, cudaStream_t s) {
  return launch_jb<double, STMF_F64>(prm, grid, s);
}

}  // namespace stmf
