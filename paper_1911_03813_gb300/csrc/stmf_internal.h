// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "stmf.h"

namespace stmf {

constexpr size_t kMaxSmem = 232448;  // dynamic shared memory per block on sm_103
constexpr int64_t kMaxN = 512;       // features per sample
constexpr int64_t kMaxP = int64_t(1) << 40;  // samples per call

// Checks of a sample descriptor that need no context (pointers, sizes, alignment, dtype and
// scale): nullptr when V is acceptable, else a description of the first problem.
const char* samples_problem(const stmf_samples* V);

// Launch parameters of the fused pass over V (Alg. 2: Y, and the sums behind w).
struct FgParams {
  const void* V;        // sample-major storage, p rows of ld elements
  const float* scale;   // per-sample scales (e4m3) or nullptr
  const double* nu;     // p weights or nullptr (uniform nu_uniform)
  double nu_uniform;
  const double* A;      // n x r column-major FP64
  double* partials;     // [grid][r + n*r]: w partial then Y partial (column-major n x r)
  int64_t p;
  int n, ld, d, r;
  int r_pad;            // r rounded up to a multiple of 4
  int flush_tiles;      // FP32 accumulators are folded into FP64 every flush_tiles tiles
  int32_t* status;      // device status word
  const int32_t* skip;  // when non-null and nonzero at launch, the kernel does nothing
  const int64_t* idx;   // when non-null: sample k of the pass is row idx[k] of the storage
  int64_t rows;         // rows of the storage (bounds of idx)
  uint64_t seed;        // randomized range finder: key of the Philox test matrix
};

// Finalisation of Alg. 2 (the steps after Y) from the reduced (w, Y).
struct ModelParams {
  const double* partials;  // [grid][L] with L = r + n*r
  int grid;
  const double* A;
  const double* lambda;
  const double* alpha;     // device scalar or nullptr
  double* f;
  double* g_lambda;
  double* G_A;
  double* yw;              // reduced w and Y, L doubles (workspace)
  double* bmat;            // B = A^T A, r*r doubles (workspace)
  int n, r, d;
  int32_t* status;
  const int32_t* skip;     // as in FgParams
  int accumulate;          // reduce_partials: yw += sum (instead of yw = sum)
  int poison;              // finalize: write NaN to f, g_lambda and G_A when *status != 0
};

struct GramParams {
  const void* V;
  const float* scale;
  const double* nu;
  double nu_uniform;
  double* partials;  // [grid]
  int64_t p;
  int n, ld, d;
  int32_t* status;
};

// One sorted prefix of d - 1 features of the compressed symmetric moment tensor (norm_sym.cu):
// its feature indices, the length of its last run of equal indices, and d! / prod(run lengths!).
struct SymPrefix {
  uint16_t idx[7];
  uint16_t run;
  double base;
};

struct SymParams {
  const void* V;
  const float* scale;
  const double* nu;
  double nu_uniform;
  const SymPrefix* prefixes;  // [count], ordered by last feature
  long long count;
  double* slabs;     // [grid.z][count][grid.y * 64]: FP64 partial X per sample range
  double* partials;  // [blocks of the squaring kernel]
  int64_t p;
  int n, ld, d;
};

// Host launchers, one per translation unit. Each returns cudaSuccess or the launch error.
// `grid_out` receives the grid size used (partials has grid_out slots).
// dynamic shared memory of the pass; SIZE_MAX when n x r does not fit the block's registers
size_t fg_simt_smem(int dtype, int n, int r);
int fg_simt_grid(int dtype, int n, int r, int64_t p, int num_sms);
cudaError_t fg_simt_launch(int dtype, const FgParams& prm, int grid, cudaStream_t s);
cudaError_t fg_simt_launch_f64(const FgParams& prm, int grid, cudaStream_t s);
// Randomized range finder (eq. rrf): block partials of V Omega into prm.partials (w part zero).
// f64: FP64 products and sums (needs fg_simt_smem(STMF_F64, n, r) <= 232448), else FP32 products
// with FP32 sums folded into FP64 every prm.flush_tiles tiles.
int rrf_grid(int dtype, int n, int r, int64_t p, int num_sms, bool f64);
cudaError_t rrf_launch(int dtype, const FgParams& prm, int grid, cudaStream_t s, bool f64);
// Sum the block partials only (no model terms): yw = sum_g partials[g].
cudaError_t reduce_partials_launch(const ModelParams& prm, cudaStream_t s);
// Alg. 2 from a given yw = [w; vec(Y)] (B = A^T A, then the outputs).
cudaError_t finish_launch(const ModelParams& prm, cudaStream_t s);
// Register-blocked CUDA-core pass for FP32 samples (n <= 256, r <= 16; gathers supported).
bool fg_f32_supported(int dtype, int n, int r);
int fg_f32_grid(int n, int64_t p, int num_sms);
cudaError_t fg_f32_launch(const FgParams& prm, int grid, cudaStream_t s);
// Tensor-core pass that streams tiles as sub-stages (fg_tc_sub.cu): FP32 samples (each split
// into two BF16 terms; n <= 256) and BF16 / E4M3 samples with n <= 512; r <= 16.
bool fg_tc_sub_supported(int dtype, int n, int r);
int fg_tc_sub_grid(int64_t p, int num_sms, int min_tiles = 1);
cudaError_t fg_tc_sub_launch(int dtype, const FgParams& prm, int grid, cudaStream_t s);
// the sampled evaluation of Sec. 5 on the sub-stage pass: rows prm.idx[0..p) of FP32 samples
bool fg_tc_sub_gather_supported(int dtype, int n, int r);
cudaError_t fg_tc_sub_gather_launch(int dtype, const FgParams& prm, int grid, cudaStream_t s);
size_t fg_tc_supported(int dtype, int n, int r);  // nonzero when the tensor-core pass applies
int fg_tc_grid(int dtype, int n, int r, int64_t p, int num_sms, int min_tiles = 1);
cudaError_t fg_tc_launch(int dtype, const FgParams& prm, int grid, cudaStream_t s);
// the range finder of eq. rrf on the same pass (Y partials of V Omega, w = 0; prm.seed)
cudaError_t fg_tc_rrf_launch(int dtype, const FgParams& prm, int grid, cudaStream_t s);
// the sampled evaluation of Sec. 5 on the same pass: rows prm.idx[0..p) of BF16 samples
cudaError_t fg_tc_gather_launch(int dtype, const FgParams& prm, int grid, cudaStream_t s);
cudaError_t model_terms_launch(const ModelParams& prm, cudaStream_t s);
int gram_simt_grid(int dtype, int n, int64_t p, int num_sms);
bool gram_tc_supported(int dtype, int n, int64_t p);
int gram_tc_grid(int64_t p, int num_sms);
cudaError_t gram_tc_launch(const GramParams& prm, int grid, cudaStream_t s);
cudaError_t gram_simt_launch(int dtype, const GramParams& prm, int grid, cudaStream_t s);
cudaError_t reduce_scalar_launch(const double* partials, int count, double* out,
                                 int32_t* status, cudaStream_t s);
// ||X||^2 from the distinct entries of the symmetric moment tensor (norm_sym.cu).
double sym_prefix_count(int n, int d);
void sym_prefixes(int n, int d, std::vector<SymPrefix>& out);
size_t norm_sym_smem(int dtype, int n);
dim3 norm_sym_grid(long long count, int n, int64_t p, int num_sms);
size_t norm_sym_slab_bytes(long long count, dim3 grid);
int norm_sym_square_blocks(long long count);
cudaError_t norm_sym_launch(int dtype, const SymParams& prm, dim3 grid, cudaStream_t s);

// The fused pass that serves a request (r <= 16 for every tensor-core pass): the whole-tile
// tensor-core pass for BF16/E4M3 with n <= 256, the sub-stage tensor-core pass for FP32 with
// n <= 256 and for BF16/E4M3 with n <= 512, else the register-blocked FP32 pass (FP32, r <= 16),
// else the CUDA-core pass. Gathered rows (an index array) take the CUDA-core passes only.
enum PassKind {
  kPassTc = 0, kPassTcSub = 1, kPassF32 = 2, kPassSimt = 3, kPassTcGather = 4, kPassTcSubGather = 5
};
struct PassPlan {
  PassKind kind;
  int grid;
};
// false when no pass holds n x r (the CUDA-core pass's shared memory). min_tiles: the fewest
// 128-sample tiles a CTA of a tensor-core pass takes (1: one CTA per SM whenever p allows).
bool plan_pass(int dtype, int n, int r, int64_t p, int num_sms, bool gather, PassPlan* out,
               int min_tiles = 1);
cudaError_t launch_pass(const PassPlan& pl, int dtype, const FgParams& prm, cudaStream_t s);

inline int elem_bytes(int dtype) {
  switch (dtype) {
    case STMF_F64: return 8;
    case STMF_F32: return 4;
    case STMF_BF16: return 2;
    case STMF_E4M3: return 1;
    default: return 0;
  }
}

}  // namespace stmf

#include <vector>

// A library context (opaque to callers): device, workspace, status word, timing events.
struct stmf_ctx {
  int device = 0;
  int num_sms = 0;
  void* ws = nullptr;        // device workspace (partials, reduced Y/w)
  size_t ws_bytes = 0;
  void* fit_ws = nullptr;    // device workspace of the optimiser state
  size_t fit_ws_bytes = 0;
  int32_t* status = nullptr; // device status word
  std::string last_error;
  bool profiling = false;    // record events around each fused pass
  int min_tiles = 1;         // fewest tiles per CTA of a tensor-core pass (serving slots: more)
  std::vector<cudaEvent_t> ev_pool;  // recorded pairs: [2k] start, [2k+1] end
  size_t ev_used = 0;
  // host-streaming evaluation (stmf_fg_host): staging buffers, copy streams, events
  void* stage[3] = {nullptr, nullptr, nullptr};
  size_t stage_bytes = 0;
  cudaStream_t copy_stream[2] = {nullptr, nullptr};
  cudaEvent_t copied[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t consumed[3] = {nullptr, nullptr, nullptr};
  void* host_small = nullptr;  // device: lambda, A, alpha, yw, outputs
  size_t host_small_bytes = 0;
  // prefix table of the compressed symmetric ||X||^2 for (sym_n, sym_d)
  void* sym_dev = nullptr;
  size_t sym_dev_bytes = 0;
  int sym_n = 0, sym_d = 0;
  long long sym_count = 0;
};

namespace stmf {
// Shared host helpers of the entry points (stmf_api.cu).
stmf_status set_error(stmf_ctx* c, stmf_status st, const std::string& msg);
stmf_status check_samples_arg(stmf_ctx* c, const stmf_samples* V);
stmf_status ensure_workspace(stmf_ctx* c, size_t bytes);
// Enqueue one evaluation of Alg. 2 (fused pass + model terms) with optional skip flag.
stmf_status enqueue_fg(stmf_ctx* c, const stmf_samples* V, const double* nu, int d, int64_t r,
                       const double* lambda, const double* A, const double* alpha, double* f,
                       double* g_lambda, double* G_A, const int32_t* skip, cudaStream_t s,
                       const int64_t* idx = nullptr, int64_t n_idx = 0,
                       double* yw_out = nullptr, double nu_uniform = 0.0,
                       bool accumulate = false);
size_t fg_workspace_bytes(const stmf_ctx* c, const stmf_samples* V, int64_t r);
// The largest fg_workspace_bytes over every storage type for n features and rank r.
size_t fg_workspace_bytes_any(const stmf_ctx* c, int64_t n, int64_t r);

// Bytes of the device optimiser state for D unknowns and m pairs.
size_t fit_state_bytes(long long D, int m);

// One run of the on-device L-BFGS (lbfgs.cu), driven asynchronously: begin() enqueues the set-up
// (and alpha when asked), enqueue_chunk() enqueues opts.chunk evaluations + steps and an async
// copy of the done flag to *done_host, finish() enqueues the export of the iterate into the
// (lambda, A) buffers given to begin() and an async copy of the optimiser state to state_host
// (FitRun::state_size() bytes), from which result_from() fills a stmf_fit_result.
struct FitRun {
  stmf_ctx* ctx = nullptr;
  stmf_samples V{};
  const double* nu = nullptr;
  int d = 0;
  int64_t r = 0;
  stmf_fit_opts opts{};
  double* lam_out = nullptr;
  double* A_out = nullptr;
  cudaStream_t stream = nullptr;
  long long D = 0;
  long long enqueued = 0;
  // From the second chunk on, a chunk (its evaluations, steps and the done-flag copy) is replayed
  // from a CUDA graph recorded once per run: the same launches with the same arguments every time.
  cudaGraphExec_t graph = nullptr;
  bool graph_ok = true;
  int chunks = 0;
  stmf_status begin(stmf_ctx* c, const stmf_samples* V, const double* nu, int d, int64_t r,
                    const stmf_fit_opts* opts, double* lambda, double* A, cudaStream_t s);
  stmf_status enqueue_chunk(int32_t* done_host);
  stmf_status enqueue_body(int32_t* done_host);
  void release();  // destroys the chunk graph (begin and finish call it)
  bool exhausted() const;
  stmf_status finish(void* state_host);
  static size_t state_size();
  static void result_from(const void* state_host, int32_t dev_status, stmf_fit_result* out);
};
}  // namespace stmf

namespace stmf {
// Graph recording (the fit loop, lbfgs.cu): while a recorder is set for the calling thread, the
// kernel launchers append kernel nodes, in order, to its graph instead of launching them. No
// stream capture is involved, so other threads' device-wide synchronisation is unaffected.
struct GraphRecorder {
  cudaGraph_t graph = nullptr;
  cudaGraphNode_t last = nullptr;
  bool ok = true;
};
GraphRecorder*& graph_recorder();

// Raise `kernel`'s dynamic shared-memory limit to `bytes` on the current device, once per
// (kernel, device); safe to call from several host threads.
cudaError_t smem_limit(const void* kernel, int bytes);

template <typename T>
struct NonDeduced {
  using type = T;
};

#ifdef __CUDACC__
// Launch kern<<<grid, block, smem, s>>>(args...), or record it when a recorder is active.
template <typename... P>
cudaError_t launch_kernel(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                          typename NonDeduced<P>::type... args) {
  GraphRecorder* rec = graph_recorder();
  if (rec) {
    void* ptrs[sizeof...(P) > 0 ? sizeof...(P) : 1] = {(void*)&args...};
    cudaKernelNodeParams kp{};
    kp.func = (void*)kern;
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = ptrs;
    cudaGraphNode_t node;
    const cudaError_t e = cudaGraphAddKernelNode(&node, rec->graph, rec->last ? &rec->last : nullptr,
                                                 rec->last ? 1 : 0, &kp);
    if (e != cudaSuccess) {
      rec->ok = false;
      return e;
    }
    rec->last = node;
    return cudaSuccess;
  }
  kern<<<grid, block, smem, s>>>(args...);
  return cudaGetLastError();
}
#endif
}  // namespace stmf

// Record a device-side error in the status word: the first error wins.
#ifdef __CUDACC__
__device__ __forceinline__ void stmf_set_status(int32_t* status, int32_t code) {
  if (status) atomicCAS(status, 0, code);
}
#endif
