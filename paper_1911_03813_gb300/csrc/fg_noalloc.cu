// stmf_fg_noalloc: the function/gradient evaluation of stmf_fg for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a memory pool or an arena
// owned by another runtime that forbids outside allocations, a host process whose allocator
// hooks must not be re-entered, or a launch path where an allocation would synchronise the
// device at the wrong moment. stmf_fg needs a context, and a context allocates its status word
// and grows its workspace with cudaMalloc. This entry point needs neither: its scratch (the
// per-block partial sums, the reduced Y and w, B = A^T A, and a status word) lives in one fixed
// array in the library's device globals, which every GPU that loads the library holds until the
// process exits.
//
// Set-up: the first call on a device (with that device current) looks up the device address of
// the array with cudaGetSymbolAddress; make that first call before any stream capture. Later
// calls look it up again whenever their stream is not capturing (the lookup is cheap and stays
// correct after a cudaDeviceReset reloads the module); a call on a capturing stream uses the
// address cached by the last call on that device. The call itself allocates nothing and frees
// nothing.
//
// Sharing: every call on a device uses the same array and leaves its contents behind. A call
// writes every block partial it reads, unless a block gave up on a bounded wait; in that case
// it has set an error in the status word, and the model-terms kernel then writes NaN to f,
// g_lambda and G_A rather than a result built from another call's partials. Two calls whose work
// overlaps on the GPU (different streams, or different host threads) race on the array and give
// wrong results: serialise them.
#include <cuda_runtime.h>

#include <mutex>

#include "stmf_internal.h"

namespace {

// 8 MiB of FP64 scratch, plus room for the status word.
constexpr size_t kScratchDoubles = size_t(1) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_fg_scratch[kScratchDoubles + 32];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

stmf_status scratch_for_current_device(cudaStream_t stream, double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return STMF_ECUDA;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return STMF_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (cap == cudaStreamCaptureStatusNone || !g_scratch_addr[dev]) {
    if (cap != cudaStreamCaptureStatusNone) return STMF_EINVAL;  // no address cached yet
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_fg_scratch);
    if (e != cudaSuccess || !p) return STMF_ECUDA;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return STMF_OK;
}

}  // namespace

extern "C" stmf_status stmf_fg_noalloc(const stmf_samples* V, const double* nu, int32_t d,
                                       int64_t r, const double* lambda, const double* A,
                                       const double* alpha, double* f, double* g_lambda,
                                       double* G_A, int32_t* status, stmf_stream_t stream) {
  // argument checks (the same rules, limits and messages as stmf_fg)
  if (stmf::samples_problem(V)) return STMF_EINVAL;
  if (d < 2 || d > 8 || r < 1 || r > 64) return STMF_EINVAL;
  if (!lambda || !A || !f || !g_lambda || !G_A) return STMF_EINVAL;

  int dev = 0, major = 0, minor = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return STMF_ECUDA;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return STMF_ECUDA;
  if (!(major == 10 && minor == 3)) return STMF_EUNSUPPORTED;

  const int n = (int)V->n;
  stmf::PassPlan pass{};
  if (!stmf::plan_pass(V->dtype, n, (int)r, V->p, sms, false, &pass)) return STMF_EINVAL;
  int grid = pass.grid;
  // the partials of `grid` blocks plus the reduced (w, Y) must fit the fixed scratch; the pass is
  // persistent, so fewer blocks only means fewer tiles in flight
  const size_t L = size_t(r) + size_t(n) * size_t(r);
  const size_t max_grid = (kScratchDoubles - size_t(r) * size_t(r)) / L;
  if (max_grid < 2) return STMF_ENOMEM;  // (n + 1) * r too large for the scratch
  if (size_t(grid) > max_grid - 1) grid = int(max_grid - 1);

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  double* scratch = nullptr;
  stmf_status st = scratch_for_current_device(s, &scratch);
  if (st != STMF_OK) return st;
  int32_t* status_word = status;
  if (!status_word) {
    status_word = reinterpret_cast<int32_t*>(scratch + kScratchDoubles);
    if (cudaMemsetAsync(status_word, 0, sizeof(int32_t), s) != cudaSuccess) return STMF_ECUDA;
  }

  stmf::FgParams prm{};
  prm.V = V->data;
  prm.scale = V->scale;
  prm.nu = nu;
  prm.nu_uniform = 1.0 / double(V->p);
  prm.A = A;
  prm.partials = scratch;
  prm.p = V->p;
  prm.n = n;
  prm.ld = (int)V->ld;
  prm.d = d;
  prm.r = (int)r;
  prm.r_pad = (int)((r + 3) / 4 * 4);
  prm.flush_tiles = 16;
  prm.status = status_word;
  pass.grid = grid;
  cudaError_t e = stmf::launch_pass(pass, V->dtype, prm, s);
  if (e != cudaSuccess) return STMF_ECUDA;

  stmf::ModelParams mp{};
  mp.partials = scratch;
  mp.grid = grid;
  mp.A = A;
  mp.lambda = lambda;
  mp.alpha = alpha;
  mp.f = f;
  mp.g_lambda = g_lambda;
  mp.G_A = G_A;
  mp.yw = scratch + size_t(grid) * L;
  mp.bmat = mp.yw + L;
  mp.n = n;
  mp.r = (int)r;
  mp.d = d;
  mp.status = status_word;
  mp.poison = 1;  // an error recorded during this call (or left in a caller's word) gives NaN
  e = stmf::model_terms_launch(mp, s);
  return e == cudaSuccess ? STMF_OK : STMF_ECUDA;
}
