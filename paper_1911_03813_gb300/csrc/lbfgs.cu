// On-device limited-memory BFGS for eq. optFunc (Sec. 4) and the stmf_fit entry point.
//
// Sec. 4 minimises f(lambda, A) with L-BFGS-B, no bounds, memory m = 5, at most 10,000
// iterations and 50,000 function/gradient evaluations, stopping on the gradient norm `pgtol`.
// Without bounds L-BFGS-B is L-BFGS. The paper leaves the rest to the solver's defaults; this
// optimiser takes the same steps as the CPU oracle's (test infrastructure, written separately):
//   direction   two-loop recursion (Nocedal & Wright, Alg. 7.4), H0 = (s^T y / y^T y) I;
//   step        strong-Wolfe bracketing + zoom (ibid., Algs. 3.5/3.6), c1 = 1e-3, c2 = 0.9,
//               zoom trial = safeguarded cubic minimiser (ibid., eq. 3.59) or the midpoint,
//               bracketing doubles the step, first step 1/||p||_2 (later ones 1), at most
//               max_ls evaluations per line search;
//   stopping    ||g||_inf <= pgtol; (f_k - f_k+1) / max(|f_k|, |f_k+1|, 1) <= factr eps;
//               max_iters outer iterations; max_evals evaluations; non-finite values;
//   memory      a pair (s, y) is kept only when s^T y > 1e-10 y^T y.
//
// The optimiser state lives in device memory; one evaluation = the fused pass over V plus the
// model terms (writing f and the gradient of the trial point) followed by `lbfgs_step` (one
// block, FP64), which consumes the evaluation and writes the next trial point. When the method
// stops, it sets `done`, and every later kernel of the queue returns at once; the host enqueues
// evaluations in chunks and reads `done` once per chunk.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "stmf_internal.h"

namespace stmf {
namespace {

enum Phase { PH_INIT = 0, PH_BRACKET = 1, PH_ZOOM = 2, PH_DONE = 3 };
enum Stop { ST_RUN = 0, ST_PGTOL = 1, ST_FACTR = 2, ST_MAXITER = 3, ST_MAXEVAL = 4, ST_LSFAIL = 5,
            ST_NONFINITE = 6 };

struct FitState {
  double f;                    // objective at x
  double ft;                   // objective at the trial point (written by the evaluation)
  double alpha;                // ||X||^2 or 0
  double phi0, dphi0, a_cur;
  double prev_a, prev_f, prev_d;
  double lo_a, lo_f, lo_d;
  double hi_a, hi_f, hi_d;
  double g_inf;
  long long iters, evals;
  int phase, ls_evals, has_lo, has_hi;
  int npairs, head;            // ring of stored pairs: oldest at (head - npairs) mod m
  int stop;
  int done;
};

struct FitLayout {
  FitState* st;
  double *x, *g, *p, *xt, *gt, *prev_g, *lo_g, *S, *Yv, *rho;
  long long D;
  int m;
};

constexpr int LT = 512;  // threads of the step kernel

__device__ double block_sum(double v, double* red) {
  // fixed-order block reduction: warp butterflies, then warp sums in index order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < LT / 32; ++k) t += red[k];
  return t;
}

__device__ double block_max(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double t = red[0];
  for (int k = 1; k < LT / 32; ++k) t = fmax(t, red[k]);
  return t;
}

__device__ double dot(const double* a, const double* b, long long D, double* red) {
  double s = 0.0;
  for (long long i = threadIdx.x; i < D; i += LT) s += a[i] * b[i];
  return block_sum(s, red);
}

// Minimiser of the cubic through (a0, f0, d0) and (a1, f1, d1) (Nocedal & Wright eq. 3.59),
// or NaN when there is none.
__device__ double cubic_step(double a0, double f0, double d0, double a1, double f1, double d1) {
  if (a0 == a1) return nan("");
  const double t1 = d0 + d1 - 3.0 * (f0 - f1) / (a0 - a1);
  const double disc = t1 * t1 - d0 * d1;
  if (!(disc >= 0.0) || !isfinite(disc)) return nan("");
  const double t2 = copysign(sqrt(disc), a1 - a0);
  const double den = d1 - d0 + 2.0 * t2;
  if (den == 0.0 || !isfinite(den)) return nan("");
  return a1 - (a1 - a0) * (d1 + t2 - t1) / den;
}

// Trial point of the zoom: the cubic minimiser if it lies in the middle 80% of [lo, hi],
// else the midpoint.
__device__ double zoom_trial(double lo, double flo, double dlo, double hi, double fhi,
                             double dhi) {
  if (!isfinite(fhi)) return 0.5 * (lo + hi);
  double a = cubic_step(lo, flo, dlo, hi, fhi, dhi);
  const double left = fmin(lo, hi), right = fmax(lo, hi), width = right - left;
  if (!(a >= left + 0.1 * width && a <= right - 0.1 * width)) a = 0.5 * (lo + hi);
  return a;
}

struct StepOpts {
  double pgtol, factr, c1, c2;
  long long max_iters, max_evals;
  int max_ls;
};

enum Action { A_TRIAL = 0, A_ACCEPT_CUR = 1, A_ACCEPT_LO = 2, A_STOP = 3, A_NEWITER = 4 };

// Consume the evaluation at the trial point and produce the next one (see the file comment).
__global__ void __launch_bounds__(LT) lbfgs_step(FitLayout L, StepOpts o) {
  __shared__ double red[LT / 32];
  __shared__ int action, copy_prev_to_lo, copy_cur_to_lo, copy_cur_to_prev, new_iter;
  __shared__ double trial_a, acc_a, acc_f;
  FitState* st = L.st;
  if (st->done) return;
  const long long D = L.D;
  const int tid = threadIdx.x;
  const double eps = 2.220446049250313e-16;

  // ------------------------------------------------------------ 1. the evaluation just made
  const double ft = st->ft;
  double dt = 0.0;
  if (st->phase != PH_INIT) dt = dot(L.gt, L.p, D, red);
  if (tid == 0) {
    st->evals += 1;
    copy_prev_to_lo = copy_cur_to_lo = copy_cur_to_prev = 0;
    new_iter = 0;
    int act = A_TRIAL;
    if (st->phase == PH_INIT) {
      act = A_NEWITER;  // x0 evaluated: x = xt, f = ft, g = gt (copied below)
    } else {
      st->ls_evals += 1;
      const double a = st->a_cur;
      bool zoom_next = false;
      if (st->phase == PH_BRACKET) {
        if (!isfinite(ft) || ft > st->phi0 + o.c1 * a * st->dphi0 ||
            (st->ls_evals > 1 && ft >= st->prev_f)) {
          st->lo_a = st->prev_a; st->lo_f = st->prev_f; st->lo_d = st->prev_d;
          copy_prev_to_lo = 1;
          st->hi_a = a; st->hi_f = ft; st->hi_d = dt;
          st->has_lo = st->has_hi = 1;
          zoom_next = true;
        } else if (fabs(dt) <= -o.c2 * st->dphi0) {
          act = A_ACCEPT_CUR;
        } else if (dt >= 0.0) {
          st->lo_a = a; st->lo_f = ft; st->lo_d = dt;
          copy_cur_to_lo = 1;
          st->hi_a = st->prev_a; st->hi_f = st->prev_f; st->hi_d = st->prev_d;
          st->has_lo = st->has_hi = 1;
          zoom_next = true;
        } else {
          st->prev_a = a; st->prev_f = ft; st->prev_d = dt;
          copy_cur_to_prev = 1;
          st->a_cur = 2.0 * a;
          if (st->evals < o.max_evals && st->ls_evals < o.max_ls) {
            act = A_TRIAL;
          } else {  // out of budget while extrapolating: lo = prev, no zoom
            st->lo_a = st->prev_a; st->lo_f = st->prev_f; st->lo_d = st->prev_d;
            copy_cur_to_lo = 1;  // prev is the point just evaluated
            st->has_lo = 1;
            act = (st->lo_a > 0.0 && st->lo_f < st->phi0) ? A_ACCEPT_LO : A_STOP;
            if (act == A_STOP) st->stop = st->evals >= o.max_evals ? ST_MAXEVAL : ST_LSFAIL;
          }
        }
      } else {  // PH_ZOOM
        if (!isfinite(ft) || ft > st->phi0 + o.c1 * a * st->dphi0 || ft >= st->lo_f) {
          st->hi_a = a; st->hi_f = ft; st->hi_d = dt;
          zoom_next = true;
        } else if (fabs(dt) <= -o.c2 * st->dphi0) {
          act = A_ACCEPT_CUR;
        } else {
          if (dt * (st->hi_a - st->lo_a) >= 0.0) {
            st->hi_a = st->lo_a; st->hi_f = st->lo_f; st->hi_d = st->lo_d;
          }
          st->lo_a = a; st->lo_f = ft; st->lo_d = dt;
          copy_cur_to_lo = 1;
          zoom_next = true;
        }
      }
      if (zoom_next) {
        if (st->evals < o.max_evals && st->ls_evals < o.max_ls) {
          st->a_cur = zoom_trial(st->lo_a, st->lo_f, st->lo_d, st->hi_a, st->hi_f, st->hi_d);
          st->phase = PH_ZOOM;
          act = A_TRIAL;
        } else if (st->lo_a > 0.0 && st->lo_f < st->phi0) {
          act = A_ACCEPT_LO;
        } else {
          act = A_STOP;
          st->stop = st->evals >= o.max_evals ? ST_MAXEVAL : ST_LSFAIL;
        }
      }
    }
    action = act;
    trial_a = st->a_cur;
    if (act == A_ACCEPT_CUR) { acc_a = st->a_cur; acc_f = ft; }
    if (act == A_ACCEPT_LO) { acc_a = st->lo_a; acc_f = st->lo_f; }
  }
  __syncthreads();
  int act = action;
  // vector bookkeeping of the line-search points
  if (copy_prev_to_lo)
    for (long long i = tid; i < D; i += LT) L.lo_g[i] = L.prev_g[i];
  if (copy_cur_to_lo)
    for (long long i = tid; i < D; i += LT) L.lo_g[i] = L.gt[i];
  if (copy_cur_to_prev)
    for (long long i = tid; i < D; i += LT) L.prev_g[i] = L.gt[i];
  __syncthreads();

  if (act == A_TRIAL) {
    const double a = trial_a;
    for (long long i = tid; i < D; i += LT) L.xt[i] = L.x[i] + a * L.p[i];
    return;
  }
  if (act == A_STOP) {
    if (tid == 0) {
      st->done = 1;
      st->phase = PH_DONE;
    }
    return;
  }

  if (act == A_NEWITER) {
    // first evaluation: x = x0 (= xt), f, g
    for (long long i = tid; i < D; i += LT) {
      L.x[i] = L.xt[i];
      L.g[i] = L.gt[i];
    }
    if (tid == 0) st->f = ft;
    __syncthreads();
  } else {
    // ------------------------------------------------------------ 2. accept the step
    const double a = acc_a;
    const double* gnew = act == A_ACCEPT_CUR ? L.gt : L.lo_g;
    // s = (x + a p) - x and y = g_new - g; the pair goes into ring slot `head` only when the
    // curvature test passes (then it becomes the newest pair, replacing the oldest when full)
    const int slot = st->head;
    double sy_part = 0.0, yy_part = 0.0;
    for (long long i = tid; i < D; i += LT) {
      const double si = (L.x[i] + a * L.p[i]) - L.x[i];
      const double yi = gnew[i] - L.g[i];
      sy_part += si * yi;
      yy_part += yi * yi;
    }
    const double sy = block_sum(sy_part, red);
    const double yy = block_sum(yy_part, red);
    const bool keep = sy > 1e-10 * yy;
    double* s = L.S + (long long)slot * D;
    double* y = L.Yv + (long long)slot * D;
    for (long long i = tid; i < D; i += LT) {
      const double xn = L.x[i] + a * L.p[i];
      if (keep) {
        s[i] = xn - L.x[i];
        y[i] = gnew[i] - L.g[i];
      }
      L.x[i] = xn;
      L.g[i] = gnew[i];
    }
    if (tid == 0) {
      if (keep) {
        L.rho[slot] = 1.0 / sy;
        st->head = (slot + 1) % L.m;
        st->npairs = min(st->npairs + 1, L.m);
      }
      const double f_old = st->f;
      st->f = acc_f;
      st->iters += 1;
      new_iter = 1;
      if ((f_old - acc_f) / fmax(fmax(fabs(f_old), fabs(acc_f)), 1.0) <= o.factr * eps) {
        st->stop = ST_FACTR;
        new_iter = 0;
      }
    }
    __syncthreads();
    if (!new_iter) {
      if (tid == 0) {
        st->done = 1;
        st->phase = PH_DONE;
      }
      return;
    }
  }

  // ------------------------------------------------------------ 3. a new outer iteration
  double ginf = 0.0;
  int bad = 0;
  for (long long i = tid; i < D; i += LT) {
    const double gi = L.g[i];
    if (!isfinite(gi)) bad = 1;
    ginf = fmax(ginf, fabs(gi));
  }
  const double nbad = block_sum((double)bad, red);
  ginf = block_max(ginf, red);
  if (tid == 0) {
    int stop = ST_RUN;
    if (!isfinite(st->f) || nbad > 0.0) stop = ST_NONFINITE;
    else if (ginf <= o.pgtol) stop = ST_PGTOL;
    else if (st->iters >= o.max_iters) stop = ST_MAXITER;
    else if (st->evals >= o.max_evals) stop = ST_MAXEVAL;
    st->g_inf = ginf;
    if (stop != ST_RUN) {
      st->stop = stop;
      st->done = 1;
      st->phase = PH_DONE;
    }
    action = stop != ST_RUN;
  }
  __syncthreads();
  if (action) return;

  // two-loop recursion: p = -H g
  __shared__ double alph[64];
  const int m = L.m, np = st->npairs, head = st->head;
  for (long long i = tid; i < D; i += LT) L.p[i] = L.g[i];  // q
  __syncthreads();
  for (int k = np - 1; k >= 0; --k) {  // newest to oldest
    const int slot = (head - np + k + m) % m;
    const double* s = L.S + (long long)slot * D;
    const double* y = L.Yv + (long long)slot * D;
    const double ak = L.rho[slot] * dot(s, L.p, D, red);
    if (tid == 0) alph[k] = ak;
    for (long long i = tid; i < D; i += LT) L.p[i] -= ak * y[i];
    __syncthreads();
  }
  double gamma = 1.0;
  if (np > 0) {
    const int newest = (head - 1 + m) % m;
    const double* s = L.S + (long long)newest * D;
    const double* y = L.Yv + (long long)newest * D;
    const double sy = dot(s, y, D, red);
    const double yy = dot(y, y, D, red);
    gamma = sy / yy;
  }
  for (long long i = tid; i < D; i += LT) L.p[i] *= gamma;
  __syncthreads();
  for (int k = 0; k < np; ++k) {  // oldest to newest
    const int slot = (head - np + k + m) % m;
    const double* s = L.S + (long long)slot * D;
    const double* y = L.Yv + (long long)slot * D;
    const double beta = L.rho[slot] * dot(y, L.p, D, red);
    const double ak = alph[k];
    for (long long i = tid; i < D; i += LT) L.p[i] += s[i] * (ak - beta);
    __syncthreads();
  }
  for (long long i = tid; i < D; i += LT) L.p[i] = -L.p[i];
  __syncthreads();
  double dphi0 = dot(L.g, L.p, D, red);
  int reset = !(dphi0 < 0.0);
  if (reset) {  // not a descent direction: drop the memory and use -g
    for (long long i = tid; i < D; i += LT) L.p[i] = -L.g[i];
    __syncthreads();
    dphi0 = dot(L.g, L.p, D, red);
  }
  const double pp = dot(L.p, L.p, D, red);
  if (tid == 0) {
    if (reset) {
      st->npairs = 0;
      st->head = 0;
    }
    const double a0 = st->npairs == 0 ? 1.0 / sqrt(pp) : 1.0;
    st->dphi0 = dphi0;
    st->phi0 = st->f;
    st->prev_a = 0.0;
    st->prev_f = st->f;
    st->prev_d = dphi0;
    st->a_cur = a0;
    st->ls_evals = 0;
    st->has_lo = st->has_hi = 0;
    st->phase = PH_BRACKET;
    trial_a = a0;
  }
  for (long long i = tid; i < D; i += LT) L.prev_g[i] = L.g[i];
  __syncthreads();
  const double a = trial_a;
  for (long long i = tid; i < D; i += LT) L.xt[i] = L.x[i] + a * L.p[i];
}

__global__ void fit_init(FitLayout L, const double* lambda, const double* A, int r, long long D) {
  for (long long i = blockIdx.x * blockDim.x + threadIdx.x; i < D; i += gridDim.x * blockDim.x)
    L.xt[i] = i < r ? lambda[i] : A[i - r];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    FitState* st = L.st;
    *st = FitState{};
    st->phase = PH_INIT;
  }
}

__global__ void fit_export(FitLayout L, double* lambda, double* A, int r, long long D) {
  for (long long i = blockIdx.x * blockDim.x + threadIdx.x; i < D; i += gridDim.x * blockDim.x) {
    if (i < r) lambda[i] = L.x[i];
    else A[i - r] = L.x[i];
  }
}

}  // namespace

size_t fit_state_bytes(long long D, int m) {
  return 256 + sizeof(double) * (size_t(D) * (7 + 2 * size_t(m)) + size_t(m) + 8);
}

namespace {

FitLayout layout(void* base, long long D, int m) {
  FitLayout L;
  L.st = static_cast<FitState*>(base);
  double* p = reinterpret_cast<double*>(static_cast<char*>(base) + 256);
  L.x = p; p += D;
  L.g = p; p += D;
  L.p = p; p += D;
  L.xt = p; p += D;
  L.gt = p; p += D;
  L.prev_g = p; p += D;
  L.lo_g = p; p += D;
  L.S = p; p += size_t(m) * D;
  L.Yv = p; p += size_t(m) * D;
  L.rho = p;
  L.D = D;
  L.m = m;
  return L;
}

}  // namespace

// ---------------------------------------------------------------------------------- host side

stmf_status FitRun::begin(stmf_ctx* c, const stmf_samples* V_, const double* nu_, int d_,
                          int64_t r_, const stmf_fit_opts* o, double* lambda, double* A,
                          cudaStream_t s) {
  release();
  ctx = c;
  V = *V_;
  nu = nu_;
  d = d_;
  r = r_;
  opts = *o;
  lam_out = lambda;
  A_out = A;
  stream = s;
  D = r + V.n * r;
  stmf_status st = check_samples_arg(c, &V);
  if (st != STMF_OK) return st;
  if (d < 2 || d > 8) return set_error(c, STMF_EINVAL, "d must be in [2, 8]");
  if (r < 1 || r > 64) return set_error(c, STMF_EINVAL, "r must be in [1, 64]");
  if (o->m < 1 || o->m > 64 || o->max_ls < 1 || o->chunk < 1 || o->max_evals < 1 ||
      o->max_iters < 0 || !(o->pgtol >= 0.0) || !(o->factr >= 0.0))
    return set_error(c, STMF_EINVAL, "invalid optimiser options");
  st = ensure_workspace(c, fg_workspace_bytes(c, &V, r));
  if (st != STMF_OK) return st;
  const size_t need = fit_state_bytes(D, o->m);
  if (need > c->fit_ws_bytes) {
    if (cudaDeviceSynchronize() != cudaSuccess) return set_error(c, STMF_ECUDA, "sync");
    if (c->fit_ws) cudaFree(c->fit_ws);
    c->fit_ws = nullptr;
    c->fit_ws_bytes = 0;
    if (cudaMalloc(&c->fit_ws, need) != cudaSuccess)
      return set_error(c, STMF_ENOMEM, "cudaMalloc of the optimiser state failed");
    c->fit_ws_bytes = need;
  }
  FitLayout L = layout(c->fit_ws, D, o->m);
  fit_init<<<32, 256, 0, s>>>(L, lambda, A, (int)r, D);
  if (cudaGetLastError() != cudaSuccess) return set_error(c, STMF_ECUDA, "fit_init launch");
  if (o->alpha_mode) {
    st = stmf_norm_x(c, &V, nu, d, &L.st->alpha, reinterpret_cast<stmf_stream_t>(s));
    if (st != STMF_OK) return st;
  }
  enqueued = 0;
  return STMF_OK;
}

GraphRecorder*& graph_recorder() {
  static thread_local GraphRecorder* rec = nullptr;
  return rec;
}

void FitRun::release() {
  if (graph) cudaGraphExecDestroy(graph);
  graph = nullptr;
  graph_ok = true;
  chunks = 0;
}

stmf_status FitRun::enqueue_chunk(int32_t* done_host) {
  // the first chunk runs as plain launches (kernel attributes get set up on first use); later
  // ones replay a graph of the chunk, recorded once by the launchers themselves (no stream
  // capture)
  if (++chunks >= 2 && graph_ok) {
    if (!graph) {
      cudaGraph_t g = nullptr;
      bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
      if (ok) {
        GraphRecorder rec;
        rec.graph = g;
        graph_recorder() = &rec;
        const stmf_status st = enqueue_body(done_host);
        graph_recorder() = nullptr;
        ok = st == STMF_OK && rec.ok && cudaGraphInstantiate(&graph, g, 0) == cudaSuccess;
        cudaGraphDestroy(g);
      }
      if (!ok) {
        graph = nullptr;
        graph_ok = false;  // plain launches for the rest of this run
        cudaGetLastError();
      }
    }
    if (graph) {
      if (cudaGraphLaunch(graph, stream) != cudaSuccess)
        return set_error(ctx, STMF_ECUDA, "chunk graph launch");
      enqueued += opts.chunk;
      return STMF_OK;
    }
  }
  const stmf_status st = enqueue_body(done_host);
  if (st != STMF_OK) return st;
  enqueued += opts.chunk;
  return STMF_OK;
}

stmf_status FitRun::enqueue_body(int32_t* done_host) {
  FitLayout L = layout(ctx->fit_ws, D, opts.m);
  StepOpts so;
  so.pgtol = opts.pgtol;
  so.factr = opts.factr;
  so.c1 = 1e-3;
  so.c2 = 0.9;
  so.max_iters = opts.max_iters;
  so.max_evals = opts.max_evals;
  so.max_ls = opts.max_ls;
  const int32_t* skip = &L.st->done;
  for (int k = 0; k < opts.chunk; ++k) {
    stmf_status st = enqueue_fg(ctx, &V, nu, d, r, L.xt, L.xt + r, &L.st->alpha, &L.st->ft,
                                L.gt, L.gt + r, skip, stream);
    if (st != STMF_OK) return st;
    if (launch_kernel(lbfgs_step, dim3(1), dim3(LT), 0, stream, L, so) != cudaSuccess)
      return set_error(ctx, STMF_ECUDA, "lbfgs_step launch");
  }
  GraphRecorder* rec = graph_recorder();
  if (rec) {
    cudaGraphNode_t node;
    if (cudaGraphAddMemcpyNode1D(&node, rec->graph, rec->last ? &rec->last : nullptr,
                                 rec->last ? 1 : 0, done_host, &L.st->done, sizeof(int32_t),
                                 cudaMemcpyDeviceToHost) != cudaSuccess) {
      rec->ok = false;
      return set_error(ctx, STMF_ECUDA, "recording the done-flag copy");
    }
    rec->last = node;
  } else if (cudaMemcpyAsync(done_host, &L.st->done, sizeof(int32_t), cudaMemcpyDeviceToHost,
                             stream) != cudaSuccess) {
    return set_error(ctx, STMF_ECUDA, "reading the done flag");
  }
  return STMF_OK;
}

bool FitRun::exhausted() const { return enqueued > opts.max_evals + opts.chunk; }

stmf_status FitRun::finish(void* state_host) {
  release();
  FitLayout L = layout(ctx->fit_ws, D, opts.m);
  fit_export<<<32, 256, 0, stream>>>(L, lam_out, A_out, (int)r, D);
  if (cudaGetLastError() != cudaSuccess) return set_error(ctx, STMF_ECUDA, "fit_export launch");
  if (cudaMemcpyAsync(state_host, L.st, sizeof(FitState), cudaMemcpyDeviceToHost, stream) !=
      cudaSuccess)
    return set_error(ctx, STMF_ECUDA, "reading the optimiser state");
  return STMF_OK;
}

size_t FitRun::state_size() { return sizeof(FitState); }

void FitRun::result_from(const void* state_host, int32_t dev_status, stmf_fit_result* out) {
  const FitState& h = *static_cast<const FitState*>(state_host);
  out->f = h.f;
  out->alpha = h.alpha;
  out->g_inf = h.g_inf;
  out->iters = h.iters;
  out->evals = h.evals;
  out->stop_reason = h.stop;
  out->status = dev_status;
}

size_t fit_workspace_total(const stmf_ctx* c, const stmf_samples* V, int64_t r, int m) {
  return fg_workspace_bytes(c, V, r) + fit_state_bytes(r + V->n * r, m);
}

}  // namespace stmf

extern "C" stmf_status stmf_fit_default_opts(stmf_fit_opts* o) {
  if (!o) return STMF_EINVAL;
  o->m = 5;
  o->max_ls = 20;
  o->pgtol = 1e-5;
  o->factr = 1e7;
  o->max_iters = 10000;
  o->max_evals = 50000;
  o->alpha_mode = 1;
  o->chunk = 16;
  return STMF_OK;
}

extern "C" stmf_status stmf_fit(stmf_ctx_t c, const stmf_samples* V, const double* nu,
                                int32_t d, int64_t r, const stmf_fit_opts* opts,
                                double* lambda, double* A, stmf_fit_result* out,
                                stmf_stream_t stream) {
  using namespace stmf;
  if (!c) return STMF_EINVAL;
  if (!V || !opts || !lambda || !A || !out) return set_error(c, STMF_EINVAL, "NULL argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  FitRun run;
  stmf_status st = run.begin(c, V, nu, d, r, opts, lambda, A, s);
  if (st != STMF_OK) return st;
  int32_t done = 0;
  while (!done) {
    st = run.enqueue_chunk(&done);
    if (st != STMF_OK) return st;
    if (cudaStreamSynchronize(s) != cudaSuccess) return set_error(c, STMF_ECUDA, "sync");
    if (!done && run.exhausted())
      return set_error(c, STMF_ECUDA, "optimiser did not stop within its evaluation budget");
  }
  alignas(16) unsigned char hstate[512];
  st = run.finish(hstate);
  if (st != STMF_OK) return st;
  if (cudaStreamSynchronize(s) != cudaSuccess) return set_error(c, STMF_ECUDA, "sync");
  int32_t dev_status = 0;
  cudaMemcpy(&dev_status, c->status, sizeof(int32_t), cudaMemcpyDeviceToHost);
  FitRun::result_from(hstate, dev_status, out);
  return STMF_OK;
}

