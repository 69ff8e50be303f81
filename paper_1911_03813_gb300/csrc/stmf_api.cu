// Host side of the C ABI declared in include/stmf.h: contexts, argument validation, workspace
// management and the launch sequence of each entry point.
#include <cuda_runtime.h>
#include <stdio.h>

#include <cmath>
#include <map>
#include <mutex>
#include <utility>
#include <string>
#include <vector>

#include "stmf_internal.h"

namespace {

using stmf::kMaxN;
using stmf::kMaxSmem;

stmf_status fail(stmf_ctx* c, stmf_status st, const std::string& msg) {
  if (c) c->last_error = msg;
  return st;
}

stmf_status cuda_fail(stmf_ctx* c, cudaError_t e, const char* where) {
  return fail(c, STMF_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// A context's arrays and workspace live on its device: every call runs with that device current.
stmf_status check_device(stmf_ctx* c) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != c->device)
    return fail(c, STMF_EINVAL, "the context's device is not the calling thread's current device");
  return STMF_OK;
}

stmf_status check_samples(stmf_ctx* c, const stmf_samples* V) {
  const char* why = stmf::samples_problem(V);
  if (why) return fail(c, STMF_EINVAL, why);
  return check_device(c);
}

stmf_status ensure_ws(stmf_ctx* c, size_t bytes) {
  if (bytes <= c->ws_bytes) return STMF_OK;
  size_t want = bytes + bytes / 4 + 4096;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaDeviceSynchronize (workspace growth)");
  if (c->ws) cudaFree(c->ws);
  c->ws = nullptr;
  c->ws_bytes = 0;
  e = cudaMalloc(&c->ws, want);
  if (e != cudaSuccess) return fail(c, STMF_ENOMEM, "cudaMalloc of the workspace failed");
  c->ws_bytes = want;
  return STMF_OK;
}

struct FgPlan {
  stmf::PassPlan pass{};
  bool fits = false;           // some pass holds n x r
  size_t partial_doubles = 0;  // grid * L
  size_t L = 0;
};

FgPlan plan_fg(const stmf_ctx* c, const stmf_samples* V, int64_t r, bool gather = false) {
  FgPlan pl;
  pl.fits = stmf::plan_pass(V->dtype, (int)V->n, (int)r, V->p, c->num_sms, gather, &pl.pass,
                            c->min_tiles);
  pl.L = size_t(r) + size_t(V->n) * size_t(r);
  pl.partial_doubles = size_t(pl.pass.grid) * pl.L;
  return pl;
}

size_t fg_ws_bytes(const FgPlan& pl, int64_t r) {
  return (pl.partial_doubles + pl.L + size_t(r) * size_t(r)) * sizeof(double);
}

size_t gram_ws_bytes(int grid) { return size_t(grid) * sizeof(double); }

}  // namespace

cudaError_t stmf::smem_limit(const void* kernel, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> done;  // (kernel, device) -> limit set
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(kernel, dev);
  const auto it = done.find(key);
  if (it != done.end() && it->second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done[key] = bytes;
  return e;
}

bool stmf::plan_pass(int dtype, int n, int r, int64_t p, int num_sms, bool gather,
                     stmf::PassPlan* out, int min_tiles) {
  PassPlan pl{kPassSimt, 0};
  if (gather && fg_tc_supported(dtype, n, r)) {
    // sampled BF16 / E4M3 rows: the tensor-core pass with warps gathering the rows
    pl = {kPassTcGather, fg_tc_grid(dtype, n, r, p, num_sms, min_tiles)};
  } else if (gather && fg_tc_sub_gather_supported(dtype, n, r)) {
    // sampled FP32 rows: the sub-stage pass, its converter warps fetching the rows
    pl = {kPassTcSubGather, fg_tc_sub_grid(p, num_sms, min_tiles)};
  } else if (!gather && fg_tc_supported(dtype, n, r)) {
    pl = {kPassTc, fg_tc_grid(dtype, n, r, p, num_sms, min_tiles)};
  } else if (!gather && fg_tc_sub_supported(dtype, n, r)) {
    pl = {kPassTcSub, fg_tc_sub_grid(p, num_sms, min_tiles)};
  } else if (fg_f32_supported(dtype, n, r)) {
    pl = {kPassF32, fg_f32_grid(n, p, num_sms)};
  } else {
    pl = {kPassSimt, fg_simt_grid(dtype, n, r, p, num_sms)};
  }
  *out = pl;
  return pl.kind != kPassSimt || fg_simt_smem(dtype, n, r) <= kMaxSmem;
}

cudaError_t stmf::launch_pass(const stmf::PassPlan& pl, int dtype, const stmf::FgParams& prm,
                              cudaStream_t s) {
  switch (pl.kind) {
    case kPassTc: return fg_tc_launch(dtype, prm, pl.grid, s);
    case kPassTcGather: return fg_tc_gather_launch(dtype, prm, pl.grid, s);
    case kPassTcSubGather: return fg_tc_sub_gather_launch(dtype, prm, pl.grid, s);
    case kPassTcSub: return fg_tc_sub_launch(dtype, prm, pl.grid, s);
    case kPassF32: return fg_f32_launch(prm, pl.grid, s);
    default: return fg_simt_launch(dtype, prm, pl.grid, s);
  }
}

const char* stmf::samples_problem(const stmf_samples* V) {
  if (!V) return "V is NULL";
  if (!V->data) return "V->data is NULL";
  const int eb = stmf::elem_bytes(V->dtype);
  if (eb == 0) return "V->dtype is not a stmf_dtype";
  if (V->n < 1 || V->n > kMaxN) return "V->n must be in [1, 512]";
  if (V->p < 1) return "V->p must be >= 1";
  if (V->p > stmf::kMaxP) return "V->p is too large";
  if (V->ld < V->n) return "V->ld must be >= V->n";
  if ((V->ld * eb) % 16 != 0) return "V->ld * element size must be a multiple of 16 bytes";
  if ((reinterpret_cast<uintptr_t>(V->data) & 15) != 0) return "V->data must be 16-byte aligned";
  if (V->dtype == STMF_E4M3 && !V->scale) return "E4M3 samples need V->scale";
  if (V->dtype != STMF_E4M3 && V->scale) return "V->scale is only used with E4M3 samples";
  return nullptr;
}

stmf_status stmf::set_error(stmf_ctx* c, stmf_status st, const std::string& msg) {
  return fail(c, st, msg);
}
stmf_status stmf::check_samples_arg(stmf_ctx* c, const stmf_samples* V) {
  return check_samples(c, V);
}
stmf_status stmf::ensure_workspace(stmf_ctx* c, size_t bytes) { return ensure_ws(c, bytes); }
size_t stmf::fg_workspace_bytes(const stmf_ctx* c, const stmf_samples* V, int64_t r) {
  return fg_ws_bytes(plan_fg(c, V, r), r);
}
size_t stmf::fg_workspace_bytes_any(const stmf_ctx* c, int64_t n, int64_t r) {
  size_t most = 0;
  for (int dt : {STMF_F64, STMF_F32, STMF_BF16, STMF_E4M3}) {
    stmf_samples V{};
    V.n = n;
    V.p = int64_t(1) << 30;
    V.dtype = dt;
    const size_t b = fg_ws_bytes(plan_fg(c, &V, r), r);
    if (b > most) most = b;
  }
  return most;
}

stmf_status stmf::enqueue_fg(stmf_ctx* c, const stmf_samples* V_in, const double* nu, int d, int64_t r,
                             const double* lambda, const double* A, const double* alpha, double* f,
                             double* g_lambda, double* G_A, const int32_t* skip, cudaStream_t s,
                             const int64_t* idx, int64_t n_idx, double* yw_out,
                             double nu_uniform, bool accumulate) {
  stmf_status st = check_samples(c, V_in);
  if (st != STMF_OK) return st;
  if (idx && n_idx < 1) return fail(c, STMF_EINVAL, "the number of sampled rows must be >= 1");
  // a sampled pass processes n_idx rows gathered through idx (the CUDA-core pass gathers)
  stmf_samples Vs = *V_in;
  if (idx) Vs.p = n_idx;
  const stmf_samples* V = &Vs;
  if (d < 2 || d > 8) return fail(c, STMF_EINVAL, "d must be in [2, 8]");
  if (r < 1 || r > 64) return fail(c, STMF_EINVAL, "r must be in [1, 64]");
  if (!lambda || !A || (!yw_out && (!f || !g_lambda || !G_A)))
    return fail(c, STMF_EINVAL, "NULL model or output pointer");
  const int n = (int)V->n;
  const FgPlan pl = plan_fg(c, V, r, idx != nullptr);  // gathers take the CUDA-core passes
  if (!pl.fits)
    return fail(c, STMF_EINVAL, "n * r too large for this sample type (shared memory)");
  st = ensure_ws(c, fg_ws_bytes(pl, r));
  if (st != STMF_OK) return st;
  double* partials = static_cast<double*>(c->ws);
  double* yw = partials + pl.partial_doubles;

  stmf::FgParams prm{};
  prm.V = V->data;
  prm.scale = V->scale;
  prm.nu = nu;
  prm.nu_uniform = nu_uniform > 0.0 ? nu_uniform : 1.0 / double(V->p);
  prm.A = A;
  prm.partials = partials;
  prm.p = V->p;
  prm.n = n;
  prm.ld = (int)V->ld;
  prm.d = d;
  prm.r = (int)r;
  prm.r_pad = (int)((r + 3) / 4 * 4);
  prm.flush_tiles = 16;
  prm.status = c->status;
  prm.skip = skip;
  prm.idx = idx;
  prm.rows = V_in->p;
  cudaEvent_t ev_end = nullptr;
  if (c->profiling && !stmf::graph_recorder() && c->ev_used + 2 <= 2 * 65536) {
    while (c->ev_pool.size() < c->ev_used + 2) {
      cudaEvent_t ev;
      if (cudaEventCreate(&ev) != cudaSuccess) break;
      c->ev_pool.push_back(ev);
    }
    if (c->ev_pool.size() >= c->ev_used + 2) {
      cudaEventRecord(c->ev_pool[c->ev_used], s);
      ev_end = c->ev_pool[c->ev_used + 1];
      c->ev_used += 2;
    }
  }
  cudaError_t e = stmf::launch_pass(pl.pass, V->dtype, prm, s);
  if (ev_end) cudaEventRecord(ev_end, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "fused pass launch");

  stmf::ModelParams mp{};
  mp.partials = partials;
  mp.grid = pl.pass.grid;
  mp.A = A;
  mp.lambda = lambda;
  mp.alpha = alpha;
  mp.f = f;
  mp.g_lambda = g_lambda;
  mp.G_A = G_A;
  mp.yw = yw;
  mp.bmat = yw + pl.L;
  mp.n = n;
  mp.r = (int)r;
  mp.d = d;
  mp.status = c->status;
  mp.skip = skip;
  if (yw_out) {  // partial sums only (one shard of a sample-sharded evaluation)
    mp.yw = yw_out;
    mp.accumulate = accumulate ? 1 : 0;
    e = stmf::reduce_partials_launch(mp, s);
  } else {
    e = stmf::model_terms_launch(mp, s);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "model terms launch");
  return STMF_OK;
}


extern "C" {

int stmf_version(void) { return 100; }

const char* stmf_status_string(int s) {
  switch (s) {
    case STMF_OK: return "STMF_OK";
    case STMF_EINVAL: return "STMF_EINVAL";
    case STMF_ENOMEM: return "STMF_ENOMEM";
    case STMF_ECUDA: return "STMF_ECUDA";
    case STMF_ETIMEOUT: return "STMF_ETIMEOUT";
    case STMF_ENONFINITE: return "STMF_ENONFINITE";
    case STMF_ENOTREADY: return "STMF_ENOTREADY";
    case STMF_ECANCELLED: return "STMF_ECANCELLED";
    case STMF_EBUSY: return "STMF_EBUSY";
    case STMF_EUNSUPPORTED: return "STMF_EUNSUPPORTED";
    default: return "unknown status";
  }
}

stmf_status stmf_create(int device, stmf_ctx_t* out) {
  if (!out) return STMF_EINVAL;
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || device < 0 || device >= count) return STMF_EINVAL;
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) return STMF_ECUDA;
  if (!(prop.major == 10 && prop.minor == 3)) return STMF_EUNSUPPORTED;
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return STMF_ECUDA;
  stmf_ctx* c = new stmf_ctx();
  c->device = device;
  c->num_sms = prop.multiProcessorCount;
  e = cudaMalloc(&c->status, sizeof(int32_t));
  if (e != cudaSuccess) {
    delete c;
    return STMF_ENOMEM;
  }
  cudaMemset(c->status, 0, sizeof(int32_t));
  cudaDeviceSynchronize();
  *out = c;
  return STMF_OK;
}

stmf_status stmf_destroy(stmf_ctx_t c) {
  if (!c) return STMF_OK;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  if (c->ws) cudaFree(c->ws);
  if (c->fit_ws) cudaFree(c->fit_ws);
  if (c->status) cudaFree(c->status);
  for (cudaEvent_t ev : c->ev_pool) cudaEventDestroy(ev);
  for (int k = 0; k < 3; ++k) {
    if (c->stage[k]) cudaFree(c->stage[k]);
    if (c->copied[k]) cudaEventDestroy(c->copied[k]);
    if (c->consumed[k]) cudaEventDestroy(c->consumed[k]);
  }
  for (int k = 0; k < 2; ++k)
    if (c->copy_stream[k]) cudaStreamDestroy(c->copy_stream[k]);
  if (c->host_small) cudaFree(c->host_small);
  if (c->sym_dev) cudaFree(c->sym_dev);
  delete c;
  return STMF_OK;
}

const char* stmf_last_error(stmf_ctx_t c) { return c ? c->last_error.c_str() : "NULL context"; }

stmf_status stmf_device_status(stmf_ctx_t c, stmf_stream_t stream, int32_t* out_host) {
  if (!c || !out_host) return fail(c, STMF_EINVAL, "NULL argument");
  if (check_device(c) != STMF_OK) return STMF_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int32_t v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, c->status, sizeof(v), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "stmf_device_status");
  *out_host = v;
  return STMF_OK;
}

stmf_status stmf_reserve(stmf_ctx_t c, const stmf_samples* V, int64_t r) {
  if (!c) return STMF_EINVAL;
  stmf_status st = check_samples(c, V);
  if (st != STMF_OK) return st;
  if (r < 1 || r > 64) return fail(c, STMF_EINVAL, "r must be in [1, 64]");
  const FgPlan pl = plan_fg(c, V, r);
  const int gg = stmf::gram_simt_grid(V->dtype, (int)V->n, V->p, c->num_sms);
  size_t need = fg_ws_bytes(pl, r);
  if (gram_ws_bytes(gg) > need) need = gram_ws_bytes(gg);
  return ensure_ws(c, need);
}

stmf_status stmf_fg(stmf_ctx_t c, const stmf_samples* V, const double* nu, int32_t d, int64_t r,
                    const double* lambda, const double* A, const double* alpha, double* f,
                    double* g_lambda, double* G_A, stmf_stream_t stream) {
  if (!c) return STMF_EINVAL;
  return stmf::enqueue_fg(c, V, nu, d, r, lambda, A, alpha, f, g_lambda, G_A, nullptr,
                          reinterpret_cast<cudaStream_t>(stream));
}

namespace {
__global__ void normalize_columns(const double* Y, int n, int r, double* A0) {
  // one warp per column: A0[:, j] = Y[:, j] / ||Y[:, j]||_2 (lanes stride the rows, fixed order)
  const int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
  if (j >= r) return;
  double ss = 0.0;
  for (int i = lane; i < n; i += 32) ss += Y[i + size_t(n) * j] * Y[i + size_t(n) * j];
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  const double inv = 1.0 / sqrt(ss);
  for (int i = lane; i < n; i += 32) A0[i + size_t(n) * j] = Y[i + size_t(n) * j] * inv;
}
}  // namespace

stmf_status stmf_rrf_start(stmf_ctx_t c, const stmf_samples* V, int64_t r_hat, uint64_t seed,
                           double* A0, stmf_stream_t stream) {
  if (!c) return STMF_EINVAL;
  stmf_status st = check_samples(c, V);
  if (st != STMF_OK) return st;
  if (r_hat < 1 || r_hat > 64) return fail(c, STMF_EINVAL, "r_hat must be in [1, 64]");
  if (!A0) return fail(c, STMF_EINVAL, "A0 is NULL");
  const int n = (int)V->n;
  // BF16 and E4M3 samples with n <= 256 and r_hat <= 16: the tensor-core pass (the test matrix
  // drawn in FP32 as its W, hi/lo BF16 products, FP32 accumulation folded every 8 tiles).
  // FP64 samples: FP64 draws, products and sums on the CUDA cores (an FP64 tile must fit in
  // shared memory). Other samples: FP32 draws and products on the CUDA cores, FP32 sums over 16
  // tiles folded into FP64 (FP64 arithmetic runs at a small fraction of the FP32 rate on this
  // part, and A0 is a random start).
  const bool tcore = stmf::fg_tc_supported(V->dtype, n, (int)r_hat) != 0;
  const bool f64 = V->dtype == STMF_F64;
  if (!tcore && stmf::fg_simt_smem(f64 ? STMF_F64 : STMF_F32, n, (int)r_hat) > kMaxSmem)
    return fail(c, STMF_EINVAL, "n * r_hat too large for the range finder (shared memory)");
  const int grid = tcore ? stmf::fg_tc_grid(V->dtype, n, (int)r_hat, V->p, c->num_sms, c->min_tiles)
                         : stmf::rrf_grid(V->dtype, n, (int)r_hat, V->p, c->num_sms, f64);
  const size_t L = size_t(r_hat) + size_t(n) * size_t(r_hat);
  st = ensure_ws(c, (size_t(grid) * L + L) * sizeof(double));
  if (st != STMF_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  double* partials = static_cast<double*>(c->ws);
  double* yw = partials + size_t(grid) * L;
  stmf::FgParams prm{};
  prm.V = V->data;
  prm.scale = V->scale;
  prm.nu_uniform = 1.0;
  prm.partials = partials;
  prm.p = V->p;
  prm.n = n;
  prm.ld = (int)V->ld;
  prm.d = 2;
  prm.r = (int)r_hat;
  prm.r_pad = (int)((r_hat + 3) / 4 * 4);
  prm.flush_tiles = f64 ? 1 << 30 : 16;  // FP64 accumulators need no intermediate folds
  prm.status = c->status;
  prm.seed = seed;
  cudaError_t e = tcore ? stmf::fg_tc_rrf_launch(V->dtype, prm, grid, s)
                        : stmf::rrf_launch(V->dtype, prm, grid, s, f64);
  if (e != cudaSuccess) return cuda_fail(c, e, "range finder launch");
  stmf::ModelParams mp{};
  mp.partials = partials;
  mp.grid = grid;
  mp.yw = yw;
  mp.n = n;
  mp.r = (int)r_hat;
  e = stmf::reduce_partials_launch(mp, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "range finder reduction launch");
  normalize_columns<<<(int)((r_hat + 7) / 8), 256, 0, s>>>(yw + r_hat, n, (int)r_hat, A0);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "normalisation launch");
  return STMF_OK;
}

stmf_status stmf_fg_partial(stmf_ctx_t c, const stmf_samples* V, const double* nu,
                            int64_t p_total, int32_t d, int64_t r, const double* lambda,
                            const double* A, double* yw, stmf_stream_t stream) {
  if (!c) return STMF_EINVAL;
  if (!yw) return fail(c, STMF_EINVAL, "yw is NULL");
  if (!V || (!nu && p_total < V->p)) return fail(c, STMF_EINVAL, "p_total must be >= V->p");
  return stmf::enqueue_fg(c, V, nu, d, r, lambda, A, nullptr, nullptr, nullptr, nullptr, nullptr,
                          reinterpret_cast<cudaStream_t>(stream), nullptr, 0, yw,
                          nu ? 0.0 : 1.0 / double(p_total));
}

stmf_status stmf_fg_finish(stmf_ctx_t c, const double* yw, int64_t n, int32_t d, int64_t r,
                           const double* lambda, const double* A, const double* alpha, double* f,
                           double* g_lambda, double* G_A, stmf_stream_t stream) {
  if (!c) return STMF_EINVAL;
  if (!yw || !lambda || !A || !f || !g_lambda || !G_A)
    return fail(c, STMF_EINVAL, "NULL argument");
  if (n < 1 || n > kMaxN || r < 1 || r > 64 || d < 2 || d > 8)
    return fail(c, STMF_EINVAL, "n, r or d out of range");
  stmf_status st = check_device(c);
  if (st != STMF_OK) return st;
  st = ensure_ws(c, size_t(r) * size_t(r) * sizeof(double));
  if (st != STMF_OK) return st;
  stmf::ModelParams mp{};
  mp.A = A;
  mp.lambda = lambda;
  mp.alpha = alpha;
  mp.f = f;
  mp.g_lambda = g_lambda;
  mp.G_A = G_A;
  mp.yw = const_cast<double*>(yw);
  mp.bmat = static_cast<double*>(c->ws);
  mp.n = (int)n;
  mp.r = (int)r;
  mp.d = d;
  mp.status = c->status;
  cudaError_t e = stmf::finish_launch(mp, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "finish launch");
  return STMF_OK;
}

stmf_status stmf_fg_host(stmf_ctx_t c, const stmf_samples* V, const double* nu, int32_t d,
                         int64_t r, const double* lambda, const double* A, double alpha,
                         double* f, double* g_lambda, double* G_A, stmf_stream_t stream) {
  if (!c) return STMF_EINVAL;
  if (!V || !V->data || !lambda || !A || !f || !g_lambda || !G_A)
    return fail(c, STMF_EINVAL, "NULL argument");
  const int eb = stmf::elem_bytes(V->dtype);
  if (eb == 0 || V->n < 1 || V->n > kMaxN || V->p < 1 || V->ld < V->n || (V->ld * eb) % 16 != 0)
    return fail(c, STMF_EINVAL, "invalid samples");
  if ((V->dtype == STMF_E4M3) != (V->scale != nullptr))
    return fail(c, STMF_EINVAL, "E4M3 samples need scales (and only they)");
  if (d < 2 || d > 8 || r < 1 || r > 64) return fail(c, STMF_EINVAL, "d or r out of range");
  if (check_device(c) != STMF_OK) return STMF_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n = V->n, p = V->p;
  const size_t row_bytes = size_t(V->ld) * eb;
  // chunks of about 256 MB (a whole number of 128-sample tiles), three staging buffers
  int64_t rows = (int64_t(256) << 20) / int64_t(row_bytes);
  rows = rows < 128 ? 128 : rows / 128 * 128;
  if (rows > p) rows = p;
  const size_t chunk_bytes = size_t(rows) * row_bytes;
  const size_t extra = size_t(rows) * (sizeof(double) + sizeof(float));  // nu and scale slices
  const size_t need_stage = chunk_bytes + extra + 256;
  if (need_stage > c->stage_bytes) {
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(c, STMF_ECUDA, "sync");
    for (int k = 0; k < 3; ++k) {
      if (c->stage[k]) cudaFree(c->stage[k]);
      c->stage[k] = nullptr;
    }
    c->stage_bytes = 0;
    for (int k = 0; k < 3; ++k)
      if (cudaMalloc(&c->stage[k], need_stage) != cudaSuccess)
        return fail(c, STMF_ENOMEM, "cudaMalloc of the staging buffers failed");
    c->stage_bytes = need_stage;
  }
  for (int k = 0; k < 3; ++k) {
    if (!c->copied[k] && cudaEventCreateWithFlags(&c->copied[k], cudaEventDisableTiming) != cudaSuccess)
      return fail(c, STMF_ECUDA, "event");
    if (!c->consumed[k] &&
        cudaEventCreateWithFlags(&c->consumed[k], cudaEventDisableTiming) != cudaSuccess)
      return fail(c, STMF_ECUDA, "event");
  }
  for (int k = 0; k < 2; ++k)
    if (!c->copy_stream[k] &&
        cudaStreamCreateWithFlags(&c->copy_stream[k], cudaStreamNonBlocking) != cudaSuccess)
      return fail(c, STMF_ECUDA, "stream");
  // small device buffers: lambda, A, alpha, yw, f, g_lambda, G_A
  const size_t L = size_t(r) + size_t(n) * r;
  const size_t small = sizeof(double) * (r + n * r + 1 + L + 1 + r + n * r);
  if (small > c->host_small_bytes) {
    if (c->host_small) cudaFree(c->host_small);
    c->host_small = nullptr;
    c->host_small_bytes = 0;
    if (cudaMalloc(&c->host_small, small) != cudaSuccess)
      return fail(c, STMF_ENOMEM, "cudaMalloc failed");
    c->host_small_bytes = small;
  }
  double* d_lam = static_cast<double*>(c->host_small);
  double* d_A = d_lam + r;
  double* d_alpha = d_A + n * r;
  double* d_yw = d_alpha + 1;
  double* d_f = d_yw + L;
  double* d_gl = d_f + 1;
  double* d_GA = d_gl + r;
  cudaMemcpyAsync(d_lam, lambda, sizeof(double) * r, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d_A, A, sizeof(double) * n * r, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d_alpha, &alpha, sizeof(double), cudaMemcpyHostToDevice, s);
  cudaEvent_t start_ev = c->copied[2];
  cudaEventRecord(start_ev, s);  // the copies start after the previous work on `s`
  cudaStreamWaitEvent(c->copy_stream[0], start_ev, 0);
  const int64_t nchunks = (p + rows - 1) / rows;
  for (int64_t ch = 0; ch < nchunks; ++ch) {
    const int k = int(ch % 3);
    cudaStream_t cs = c->copy_stream[0];  // one stream: chunk copies in order at the link rate
    const int64_t lo = ch * rows, cnt = (lo + rows <= p) ? rows : p - lo;
    unsigned char* buf = static_cast<unsigned char*>(c->stage[k]);
    if (ch >= 3) cudaStreamWaitEvent(cs, c->consumed[k], 0);  // the pass over chunk ch-3 is done
    cudaMemcpyAsync(buf, static_cast<const unsigned char*>(V->data) + size_t(lo) * row_bytes,
                    size_t(cnt) * row_bytes, cudaMemcpyHostToDevice, cs);
    double* nu_d = reinterpret_cast<double*>(buf + chunk_bytes);
    float* sc_d = reinterpret_cast<float*>(buf + chunk_bytes + size_t(rows) * sizeof(double));
    if (nu) cudaMemcpyAsync(nu_d, nu + lo, sizeof(double) * cnt, cudaMemcpyHostToDevice, cs);
    if (V->scale)
      cudaMemcpyAsync(sc_d, V->scale + lo, sizeof(float) * cnt, cudaMemcpyHostToDevice, cs);
    cudaEventRecord(c->copied[k], cs);
    cudaStreamWaitEvent(s, c->copied[k], 0);
    stmf_samples chunk = *V;
    chunk.data = buf;
    chunk.p = cnt;
    chunk.scale = V->scale ? sc_d : nullptr;
    stmf_status st = stmf::enqueue_fg(c, &chunk, nu ? nu_d : nullptr, d, r, d_lam, d_A, nullptr,
                                      nullptr, nullptr, nullptr, nullptr, s, nullptr, 0, d_yw,
                                      nu ? 0.0 : 1.0 / double(p), ch > 0);
    if (st != STMF_OK) return st;
    cudaEventRecord(c->consumed[k], s);
  }
  stmf::ModelParams mp{};
  mp.A = d_A;
  mp.lambda = d_lam;
  mp.alpha = d_alpha;
  mp.f = d_f;
  mp.g_lambda = d_gl;
  mp.G_A = d_GA;
  mp.yw = d_yw;
  mp.bmat = static_cast<double*>(c->ws);  // the passes are done with the workspace by now
  mp.n = (int)n;
  mp.r = (int)r;
  mp.d = d;
  mp.status = c->status;
  cudaError_t e = stmf::finish_launch(mp, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "finish launch");
  cudaMemcpyAsync(f, d_f, sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(g_lambda, d_gl, sizeof(double) * r, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(G_A, d_GA, sizeof(double) * n * r, cudaMemcpyDeviceToHost, s);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "stmf_fg_host");
  return STMF_OK;
}

stmf_status stmf_set_pass_tiles(stmf_ctx_t c, int32_t min_tiles) {
  if (!c) return STMF_EINVAL;
  if (min_tiles < 1 || min_tiles > (1 << 20)) return fail(c, STMF_EINVAL, "min_tiles must be in [1, 2^20]");
  c->min_tiles = min_tiles;
  return STMF_OK;
}

stmf_status stmf_profile_enable(stmf_ctx_t c, int32_t enable) {
  if (!c) return STMF_EINVAL;
  c->profiling = enable != 0;
  return STMF_OK;
}

stmf_status stmf_profile_read(stmf_ctx_t c, double* total_ms, int64_t* count) {
  if (!c || !total_ms || !count) return fail(c, STMF_EINVAL, "NULL argument");
  double tot = 0.0;
  for (size_t k = 0; k + 1 < c->ev_used; k += 2) {
    cudaError_t e = cudaEventSynchronize(c->ev_pool[k + 1]);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventSynchronize");
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, c->ev_pool[k], c->ev_pool[k + 1]);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventElapsedTime");
    tot += ms;
  }
  *total_ms = tot;
  *count = (int64_t)(c->ev_used / 2);
  c->ev_used = 0;
  return STMF_OK;
}

namespace {
constexpr double kMaxSymPrefixes = double(1 << 22);  // prefix table of at most 96 MB

// ||X||^2 from the distinct entries of the symmetric moment tensor (norm_sym.cu)
stmf_status norm_x_sym(stmf_ctx* c, const stmf_samples* V, const double* nu, int d,
                       double* alpha_out, cudaStream_t s) {
  const int n = (int)V->n;
  if (stmf::sym_prefix_count(n, d) > kMaxSymPrefixes)
    return fail(c, STMF_EINVAL, "C(n + d - 2, d - 1) too large for the compressed tensor");
  if (stmf::norm_sym_smem(V->dtype, n) > kMaxSmem - 1024)
    return fail(c, STMF_EINVAL, "n too large for the compressed tensor (shared memory)");
  if (c->sym_n != n || c->sym_d != d || !c->sym_dev) {
    c->sym_n = c->sym_d = -1;  // no valid table until the upload below succeeds
    std::vector<stmf::SymPrefix> tab;
    stmf::sym_prefixes(n, d, tab);
    const size_t bytes = tab.size() * sizeof(stmf::SymPrefix);
    // an earlier call may still read the old table
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaDeviceSynchronize (prefix table)");
    if (bytes > c->sym_dev_bytes) {
      if (c->sym_dev) cudaFree(c->sym_dev);
      c->sym_dev = nullptr;
      c->sym_dev_bytes = 0;
      if (cudaMalloc(&c->sym_dev, bytes) != cudaSuccess)
        return fail(c, STMF_ENOMEM, "cudaMalloc of the prefix table failed");
      c->sym_dev_bytes = bytes;
    }
    e = cudaMemcpy(c->sym_dev, tab.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "prefix table upload");
    c->sym_n = n;
    c->sym_d = d;
    c->sym_count = (long long)tab.size();
  }
  const dim3 grid = stmf::norm_sym_grid(c->sym_count, n, V->p, c->num_sms);
  const size_t slab_bytes = stmf::norm_sym_slab_bytes(c->sym_count, grid);
  const int nblk = stmf::norm_sym_square_blocks(c->sym_count);
  stmf_status st = ensure_ws(c, slab_bytes + size_t(nblk) * sizeof(double));
  if (st != STMF_OK) return st;
  stmf::SymParams sp{};
  sp.V = V->data;
  sp.scale = V->scale;
  sp.nu = nu;
  sp.nu_uniform = 1.0 / double(V->p);
  sp.prefixes = static_cast<const stmf::SymPrefix*>(c->sym_dev);
  sp.count = c->sym_count;
  sp.slabs = static_cast<double*>(c->ws);
  sp.partials = sp.slabs + slab_bytes / sizeof(double);
  sp.p = V->p;
  sp.n = n;
  sp.ld = (int)V->ld;
  sp.d = d;
  cudaError_t e = stmf::norm_sym_launch(V->dtype, sp, grid, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "compressed tensor launch");
  e = stmf::reduce_scalar_launch(sp.partials, nblk, alpha_out, c->status, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "compressed tensor reduction launch");
  return STMF_OK;
}
}  // namespace

stmf_status stmf_norm_x(stmf_ctx_t c, const stmf_samples* V, const double* nu, int32_t d,
                        double* alpha_out, stmf_stream_t stream) {
  return stmf_norm_x_method(c, V, nu, d, 0, alpha_out, stream);
}

stmf_status stmf_norm_x_method(stmf_ctx_t c, const stmf_samples* V, const double* nu, int32_t d,
                               int32_t method, double* alpha_out, stmf_stream_t stream) {
  if (!c) return STMF_EINVAL;
  stmf_status st = check_samples(c, V);
  if (st != STMF_OK) return st;
  if (d < 2 || d > 8) return fail(c, STMF_EINVAL, "d must be in [2, 8]");
  if (!alpha_out) return fail(c, STMF_EINVAL, "alpha_out is NULL");
  if (method < 0 || method > 2) return fail(c, STMF_EINVAL, "method must be 0, 1 or 2");
  if (method == 0) {
    // multiply-adds of each form: the compressed tensor ~ prefixes x ceil64(n) x p, the Gram
    // ~ n p^2 / 2; the tensor-core Gram (BF16) runs ~25x the CUDA-core rate
    const double pre = stmf::sym_prefix_count((int)V->n, d);
    const double cs = pre * double((V->n + 63) / 64 * 64) * double(V->p);
    const double cg = double(V->n) * double(V->p) * double(V->p) / 2.0;
    const bool tcg = stmf::gram_tc_supported(V->dtype, (int)V->n, V->p);
    method = (pre <= kMaxSymPrefixes && cs * (tcg ? 25.0 : 1.0) < cg &&
              stmf::norm_sym_smem(V->dtype, (int)V->n) <= kMaxSmem - 1024)
                 ? 2 : 1;
  }
  if (method == 2)
    return norm_x_sym(c, V, nu, d, alpha_out, reinterpret_cast<cudaStream_t>(stream));
  const bool tc = stmf::gram_tc_supported(V->dtype, (int)V->n, V->p);
  const int grid = tc ? stmf::gram_tc_grid(V->p, c->num_sms)
                      : stmf::gram_simt_grid(V->dtype, (int)V->n, V->p, c->num_sms);
  st = ensure_ws(c, gram_ws_bytes(grid));
  if (st != STMF_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  stmf::GramParams gp{};
  gp.V = V->data;
  gp.scale = V->scale;
  gp.nu = nu;
  gp.nu_uniform = 1.0 / double(V->p);
  gp.partials = static_cast<double*>(c->ws);
  gp.p = V->p;
  gp.n = (int)V->n;
  gp.ld = (int)V->ld;
  gp.d = d;
  gp.status = c->status;
  cudaError_t e = tc ? stmf::gram_tc_launch(gp, grid, s)
                     : stmf::gram_simt_launch(V->dtype, gp, grid, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "Gram pass launch");
  e = stmf::reduce_scalar_launch(gp.partials, grid, alpha_out, c->status, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "Gram reduction launch");
  return STMF_OK;
}

}  // extern "C"
