// Sec. 5: stochastic evaluation from sampled columns (Lemma 5.1) and the Adam schedule used with
// it, on the device.
//
// stmf_fg_sampled runs Alg. 2 on the stochastic Kruskal tensor of Lemma 5.1: the s sampled rows
// idx[0..s) of the samples (drawn with replacement by the caller) with weights nu~ = 1/s, whose
// TTSVs are unbiased for those of X. The pass gathers its rows through the index array.
//
// stmf_adam runs Adam (Kingma & Ba, 2015) on x = (lambda, A) with Sec. 5's schedule: each
// iteration steps on the stochastic gradient of its own sample (row t of sample_idx); after every
// `epoch` iterations the shifted objective is estimated on the fixed rows est_idx; the first time
// the estimate does not decrease, the learning rate drops from lr0 to lr1 and the state returns
// to the end of the prior epoch; the second time, the method stops and returns the prior epoch's
// iterate. Reading where Sec. 5 is silent (the same as the CPU oracle's): returning to the prior
// epoch restores the Adam moments and the step counter as well as (lambda, A). All state lives in
// device memory; the decisions run on the device; the host reads a done flag once per epoch.
#include <cuda_runtime.h>

#include <cmath>

#include "stmf_internal.h"

namespace stmf {
namespace {

struct AdamState {
  double f_prev;   // estimate at the end of the last accepted epoch
  double f_now;    // estimate just computed (written by the evaluation)
  double lr;
  long long t, t_saved;
  long long epochs;
  int drops;
  int done;
  double fs, gl0;  // scratch outputs of the step evaluations (f; first g entry unused)
};

struct AdamLayout {
  AdamState* st;
  double *x, *m, *v, *xs, *ms, *vs, *g;  // D each; *s = saved at the end of the prior epoch
  long long D;
};

constexpr int AT = 256;

// x <- x - lr mhat / (sqrt(vhat) + eps) after folding the gradient g into the moments
__global__ void adam_step(AdamLayout L, double beta1, double beta2, double eps) {
  AdamState* st = L.st;
  if (st->done) return;
  const long long t = st->t + 1;
  const double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
  const double lr = st->lr;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.D;
       i += (long long)gridDim.x * blockDim.x) {
    const double g = L.g[i];
    const double m = beta1 * L.m[i] + (1.0 - beta1) * g;
    const double v = beta2 * L.v[i] + (1.0 - beta2) * g * g;
    L.m[i] = m;
    L.v[i] = v;
    L.x[i] -= lr * (m / c1) / (sqrt(v / c2) + eps);
  }
}

__global__ void adam_advance(AdamState* st) {
  if (!st->done) st->t += 1;
}

// End of an epoch: keep the state if the estimate decreased, else restore the prior epoch's
// state and drop the learning rate (first time) or stop (second time).
__global__ void adam_epoch_end(AdamLayout L, double lr1, long long max_epochs) {
  AdamState* st = L.st;
  if (st->done) return;
  __shared__ int keep;
  if (threadIdx.x == 0) {
    st->epochs += 1;
    keep = st->f_now < st->f_prev;
    if (keep) {
      st->f_prev = st->f_now;
      st->t_saved = st->t;
    } else {
      st->t = st->t_saved;
      st->drops += 1;
      st->lr = lr1;
    }
  }
  __syncthreads();
  for (long long i = threadIdx.x; i < L.D; i += blockDim.x) {
    if (keep) {
      L.xs[i] = L.x[i];
      L.ms[i] = L.m[i];
      L.vs[i] = L.v[i];
    } else {
      L.x[i] = L.xs[i];
      L.m[i] = L.ms[i];
      L.v[i] = L.vs[i];
    }
  }
  if (threadIdx.x == 0) {
    if (st->drops >= 2) st->done = 1;
    if (max_epochs > 0 && st->epochs >= max_epochs) st->done = 1;
  }
}

__global__ void adam_init(AdamLayout L, const double* lambda, const double* A, int r, double lr0) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.D;
       i += (long long)gridDim.x * blockDim.x) {
    const double xi = i < r ? lambda[i] : A[i - r];
    L.x[i] = xi;
    L.xs[i] = xi;
    L.m[i] = L.v[i] = L.ms[i] = L.vs[i] = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *L.st = AdamState{};
    L.st->lr = lr0;
  }
}

__global__ void adam_first_estimate(AdamState* st) { st->f_prev = st->f_now; }

__global__ void adam_export(AdamLayout L, double* lambda, double* A, int r) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.D;
       i += (long long)gridDim.x * blockDim.x) {
    if (i < r) lambda[i] = L.x[i];
    else A[i - r] = L.x[i];
  }
}

AdamLayout adam_layout(void* base, long long D) {
  AdamLayout L;
  L.st = static_cast<AdamState*>(base);
  double* p = reinterpret_cast<double*>(static_cast<char*>(base) + 256);
  L.x = p; p += D;
  L.m = p; p += D;
  L.v = p; p += D;
  L.xs = p; p += D;
  L.ms = p; p += D;
  L.vs = p; p += D;
  L.g = p;
  L.D = D;
  return L;
}

}  // namespace
}  // namespace stmf

extern "C" stmf_status stmf_fg_sampled(stmf_ctx_t c, const stmf_samples* V, const int64_t* idx,
                                       int64_t s, int32_t d, int64_t r, const double* lambda,
                                       const double* A, const double* alpha, double* f,
                                       double* g_lambda, double* G_A, stmf_stream_t stream) {
  if (!c) return STMF_EINVAL;
  if (!idx) return stmf::set_error(c, STMF_EINVAL, "idx is NULL");
  return stmf::enqueue_fg(c, V, nullptr, d, r, lambda, A, alpha, f, g_lambda, G_A, nullptr,
                          reinterpret_cast<cudaStream_t>(stream), idx, s);
}

extern "C" stmf_status stmf_adam_default_opts(stmf_adam_opts* o) {
  if (!o) return STMF_EINVAL;
  o->lr0 = 1e-2;
  o->lr1 = 1e-3;
  o->beta1 = 0.9;
  o->beta2 = 0.999;
  o->eps = 1e-8;
  o->epoch = 100;
  o->max_epochs = 0;
  return STMF_OK;
}

extern "C" stmf_status stmf_adam(stmf_ctx_t c, const stmf_samples* V, int32_t d, int64_t r,
                                 const stmf_adam_opts* o, const int64_t* sample_idx,
                                 int64_t iters, int64_t s, const int64_t* est_idx, int64_t est_s,
                                 double* lambda, double* A, stmf_adam_result* out,
                                 stmf_stream_t stream) {
  using namespace stmf;
  if (!c) return STMF_EINVAL;
  stmf_status st = check_samples_arg(c, V);
  if (st != STMF_OK) return st;
  if (!o || !sample_idx || !est_idx || !lambda || !A || !out)
    return set_error(c, STMF_EINVAL, "NULL argument");
  if (d < 2 || d > 8 || r < 1 || r > 64) return set_error(c, STMF_EINVAL, "d or r out of range");
  if (s < 1 || est_s < 1 || iters < 0 || o->epoch < 1 || !(o->lr0 > 0.0) || !(o->lr1 > 0.0))
    return set_error(c, STMF_EINVAL, "invalid Adam arguments");
  cudaStream_t strm = reinterpret_cast<cudaStream_t>(stream);
  const long long D = r + V->n * r;
  const size_t need = 256 + sizeof(double) * size_t(D) * 7;
  if (need > c->fit_ws_bytes) {
    if (cudaDeviceSynchronize() != cudaSuccess) return set_error(c, STMF_ECUDA, "sync");
    if (c->fit_ws) cudaFree(c->fit_ws);
    c->fit_ws = nullptr;
    c->fit_ws_bytes = 0;
    if (cudaMalloc(&c->fit_ws, need) != cudaSuccess)
      return set_error(c, STMF_ENOMEM, "cudaMalloc of the Adam state failed");
    c->fit_ws_bytes = need;
  }
  AdamLayout L = adam_layout(c->fit_ws, D);
  adam_init<<<32, AT, 0, strm>>>(L, lambda, A, (int)r, o->lr0);
  // f at the start, estimated on the fixed rows (shifted objective: alpha = 0)
  st = enqueue_fg(c, V, nullptr, d, r, L.x, L.x + r, nullptr, &L.st->f_now, L.g, L.g + r,
                  nullptr, strm, est_idx, est_s);
  if (st != STMF_OK) return st;
  adam_first_estimate<<<1, 1, 0, strm>>>(L.st);
  const int32_t* skip = &L.st->done;
  int32_t done = 0;
  long long it = 0;
  while (!done && it + o->epoch <= iters) {
    for (long long k = 0; k < o->epoch; ++k, ++it) {
      st = enqueue_fg(c, V, nullptr, d, r, L.x, L.x + r, nullptr, &L.st->fs, L.g, L.g + r, skip,
                      strm, sample_idx + it * s, s);
      if (st != STMF_OK) return st;
      adam_step<<<32, AT, 0, strm>>>(L, o->beta1, o->beta2, o->eps);
      adam_advance<<<1, 1, 0, strm>>>(L.st);
    }
    st = enqueue_fg(c, V, nullptr, d, r, L.x, L.x + r, nullptr, &L.st->f_now, L.g, L.g + r, skip,
                    strm, est_idx, est_s);
    if (st != STMF_OK) return st;
    adam_epoch_end<<<1, AT, 0, strm>>>(L, o->lr1, o->max_epochs);
    if (cudaGetLastError() != cudaSuccess) return set_error(c, STMF_ECUDA, "Adam launch");
    if (cudaMemcpyAsync(&done, &L.st->done, sizeof(int32_t), cudaMemcpyDeviceToHost, strm) !=
            cudaSuccess ||
        cudaStreamSynchronize(strm) != cudaSuccess)
      return set_error(c, STMF_ECUDA, "reading the done flag");
  }
  adam_export<<<32, AT, 0, strm>>>(L, lambda, A, (int)r);
  AdamState h;
  if (cudaMemcpyAsync(&h, L.st, sizeof(h), cudaMemcpyDeviceToHost, strm) != cudaSuccess ||
      cudaStreamSynchronize(strm) != cudaSuccess)
    return set_error(c, STMF_ECUDA, "reading the Adam state");
  out->f_est = h.f_prev;
  out->epochs = h.epochs;
  out->iters = h.t;
  out->drops = h.drops;
  int32_t dev_status = 0;
  cudaMemcpy(&dev_status, c->status, sizeof(int32_t), cudaMemcpyDeviceToHost);
  out->status = dev_status;
  return STMF_OK;
}
