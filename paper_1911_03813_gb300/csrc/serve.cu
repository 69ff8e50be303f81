// Continuously batched fits: stmf_server_create / stmf_submit / stmf_poll / stmf_cancel.
//
// A scheduler thread owns `max_fits` slots, each a library context (preallocated workspaces for
// the largest admitted shape, so no allocation ever synchronises the device), a CUDA stream, an
// event and pinned host words. A request with S starts needs S free slots and its device
// footprint (its own copy of host samples, if any, and S start/result vectors) within the
// budget; requests are admitted first come, first served. Each start runs stmf_fit's on-device
// L-BFGS (FitRun) on its slot's stream in chunks of evaluations; the scheduler never blocks on
// the GPU: it polls each slot's event, enqueues the next chunk, or (once the device reports the
// fit done) the export of the final iterate, then hands the slot to the next start. Requests'
// device memory comes from the stream-ordered allocator (cudaMallocAsync / cudaFreeAsync), so
// admission and completion do not synchronise the device either.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "stmf_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { RQ_QUEUED = 0, RQ_ACTIVE = 1, RQ_FINALIZING = 2, RQ_DONE = 3 };

struct Request {
  uint64_t ticket = 0;
  stmf_request req{};
  std::vector<double> x0;      // start points (host copy)
  int state = RQ_QUEUED;
  stmf_status status = STMF_OK;
  bool cancel = false;
  double t_submit = 0, t_admit = 0, t_done = 0;
  size_t footprint = 0;
  size_t v_bytes = 0, s_bytes = 0;
  void* dmem = nullptr;        // [samples copy][scale copy][S start/result vectors]
  double* xbuf = nullptr;
  long long D = 0;
  int starts_left = 0;
  int best_start = -1;
  stmf_fit_result best{};
  int64_t total_evals = 0;
  cudaEvent_t ready = nullptr;  // inputs are on the device
  cudaEvent_t fin = nullptr;    // result copied and memory released
};

struct Slot {
  stmf_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  int32_t* host_words = nullptr;  // pinned: [0] done flag, [1] device status
  void* state_host = nullptr;     // pinned optimiser state
  Request* req = nullptr;
  int start = -1;
  int phase = 0;                  // 0 idle, 1 chunk in flight, 2 finish in flight
  stmf::FitRun run;
};

size_t elem_size(int dtype) { return (size_t)stmf::elem_bytes(dtype); }

// Fewest 128-sample tiles per CTA in a slot's tensor-core passes. Measured on the serving workload
// (4096 requests, n, p log-uniform in [8, 128] x [1e3, 1e6]): 1 tile (one CTA per SM) 503
// saturated fits/s, 4 tiles 624, 8 704, 16 796, 32 921, 64 1051, 128 1085.
constexpr int kSlotTiles = STMF_SERVER_PASS_TILES;

}  // namespace

struct stmf_server {
  stmf_server_config cfg{};
  std::vector<Slot> slots;
  size_t slot_bytes = 0;
  size_t avail = 0;
  cudaStream_t admin = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::map<uint64_t, std::unique_ptr<Request>> all;
  std::vector<Request*> active;
  uint64_t next_ticket = 1;
  std::atomic<bool> stop{false};
  std::thread thr;
  Clock::time_point t0;
  stmf_server_stats stats{};

  double now() const {
    return std::chrono::duration<double>(Clock::now() - t0).count();
  }
  void run();
  bool admit(Request* r);
  void fail(Request* r, stmf_status st);
  void finalize(Request* r);
  bool progress_slot(Slot& s);
};

void stmf_server::fail(Request* r, stmf_status st) {
  if (r->status == STMF_OK) r->status = st;
  r->cancel = true;  // stop its other starts
}

// Copy the best start's iterate out, release the request's device memory (stream-ordered), and
// mark the request finalizing; it is done once `fin` completes.
void stmf_server::finalize(Request* r) {
  const long long D = r->D;
  const int64_t rr = r->req.r;
  if (r->status == STMF_OK && !r->cancel && r->best_start >= 0) {
    const double* x = r->xbuf + r->best_start * D;
    if (r->req.lambda_out)
      cudaMemcpyAsync(r->req.lambda_out, x, sizeof(double) * rr, cudaMemcpyDeviceToDevice, admin);
    if (r->req.A_out)
      cudaMemcpyAsync(r->req.A_out, x + rr, sizeof(double) * (D - rr), cudaMemcpyDeviceToDevice,
                      admin);
  }
  if (r->dmem) cudaFreeAsync(r->dmem, admin);
  r->dmem = nullptr;
  cudaEventRecord(r->fin, admin);
  r->state = RQ_FINALIZING;
}

bool stmf_server::admit(Request* r) {
  const stmf_request& q = r->req;
  const size_t need = r->footprint;
  int free_slots = 0;
  for (auto& s : slots) free_slots += s.req == nullptr;
  if (free_slots < q.n_starts) return false;
  if (stats.bytes_in_use + need > avail) return false;
  // device memory for the request, inputs copied on the admin stream
  if (cudaMallocAsync(&r->dmem, need, admin) != cudaSuccess) {
    r->dmem = nullptr;
    r->status = STMF_ENOMEM;
    r->state = RQ_DONE;
    r->t_done = now();
    ++stats.failed;
    return true;
  }
  unsigned char* p = static_cast<unsigned char*>(r->dmem);
  if (q.V_on_host) {
    cudaMemcpyAsync(p, q.V.data, r->v_bytes, cudaMemcpyHostToDevice, admin);
    r->req.V.data = p;
    if (q.V.scale) {
      cudaMemcpyAsync(p + r->v_bytes, q.V.scale, r->s_bytes, cudaMemcpyHostToDevice, admin);
      r->req.V.scale = reinterpret_cast<const float*>(p + r->v_bytes);
    }
  }
  r->xbuf = reinterpret_cast<double*>(p + ((r->v_bytes + r->s_bytes + 255) & ~size_t(255)));
  cudaMemcpyAsync(r->xbuf, r->x0.data(), sizeof(double) * r->x0.size(), cudaMemcpyHostToDevice,
                  admin);
  cudaEventRecord(r->ready, admin);
  stats.bytes_in_use += need;
  if (stats.bytes_in_use > stats.peak_bytes_in_use) stats.peak_bytes_in_use = stats.bytes_in_use;
  r->state = RQ_ACTIVE;
  r->t_admit = now();
  r->starts_left = q.n_starts;
  ++stats.admitted;
  int start = 0;
  for (auto& s : slots) {
    if (start == q.n_starts) break;
    if (s.req) continue;
    s.req = r;
    s.start = start;
    cudaStreamWaitEvent(s.stream, r->ready, 0);
    double* x = r->xbuf + start * r->D;
    stmf_status st = s.run.begin(s.ctx, &r->req.V, q.nu, q.d, q.r, &q.opts, x, x + q.r, s.stream);
    if (st == STMF_OK) st = s.run.enqueue_chunk(&s.host_words[0]);
    if (st != STMF_OK) fail(r, st);
    cudaEventRecord(s.ev, s.stream);
    s.phase = 1;
    ++start;
  }
  return true;
}

// Advance one busy slot if its last enqueued work has completed. Returns true on progress.
bool stmf_server::progress_slot(Slot& s) {
  if (!s.req || s.phase == 0) return false;
  const cudaError_t e = cudaEventQuery(s.ev);
  if (e == cudaErrorNotReady) return false;
  Request* r = s.req;
  if (e != cudaSuccess) fail(r, STMF_ECUDA);
  if (s.phase == 1 && !r->cancel) {
    if (s.host_words[0]) {
      stmf_status st = s.run.finish(s.state_host);
      cudaMemcpyAsync(&s.host_words[1], s.ctx->status, sizeof(int32_t), cudaMemcpyDeviceToHost,
                      s.stream);
      cudaMemsetAsync(s.ctx->status, 0, sizeof(int32_t), s.stream);
      if (st != STMF_OK) fail(r, st);
      cudaEventRecord(s.ev, s.stream);
      s.phase = 2;
      return true;
    }
    if (s.run.exhausted()) {
      fail(r, STMF_ECUDA);
    } else {
      stmf_status st = s.run.enqueue_chunk(&s.host_words[0]);
      if (st != STMF_OK) fail(r, st);
      cudaEventRecord(s.ev, s.stream);
      return true;
    }
  }
  if (s.phase == 2 && !r->cancel) {
    stmf_fit_result res{};
    stmf::FitRun::result_from(s.state_host, s.host_words[1], &res);
    r->total_evals += res.evals;
    if (r->best_start < 0 || res.f < r->best.f) {
      r->best = res;
      r->best_start = s.start;
    }
  }
  // the start is over (finished, cancelled or failed): free the slot
  s.req = nullptr;
  s.start = -1;
  s.phase = 0;
  if (--r->starts_left == 0) finalize(r);
  return true;
}

void stmf_server::run() {
  cudaSetDevice(cfg.device);
  while (!stop.load()) {
    bool progress = false;
    {
      std::unique_lock<std::mutex> lock(mu);
      // cancelled queued requests finish at once
      for (auto it = queue.begin(); it != queue.end();) {
        if ((*it)->cancel) {
          Request* r = *it;
          r->status = STMF_ECANCELLED;
          r->state = RQ_DONE;
          r->t_done = now();
          ++stats.cancelled;
          it = queue.erase(it);
          progress = true;
        } else {
          ++it;
        }
      }
      while (!queue.empty()) {
        Request* r = queue.front();
        if (!admit(r)) break;
        queue.pop_front();
        if (r->state == RQ_DONE) cv.notify_all();  // refused at admission
        else active.push_back(r);
        progress = true;
      }
      stats.queued = (int32_t)queue.size();
    }
    for (auto& s : slots) {
      std::lock_guard<std::mutex> lock(mu);
      progress |= progress_slot(s);
    }
    {
      std::lock_guard<std::mutex> lock(mu);
      bool notify = false;
      for (auto it = active.begin(); it != active.end();) {
        Request* r = *it;
        if (r->state == RQ_FINALIZING && cudaEventQuery(r->fin) != cudaErrorNotReady) {
          r->state = RQ_DONE;
          r->t_done = now();
          stats.bytes_in_use -= r->footprint;
          if (r->cancel && r->status == STMF_OK) {
            r->status = STMF_ECANCELLED;
            ++stats.cancelled;
          } else if (r->status != STMF_OK) {
            ++stats.failed;
          } else {
            ++stats.completed;
          }
          it = active.erase(it);
          notify = true;
          progress = true;
        } else {
          ++it;
        }
      }
      int busy = 0;
      for (auto& s : slots) busy += s.req != nullptr;
      stats.active_fits = busy;
      if (busy > stats.peak_active_fits) stats.peak_active_fits = busy;
      if (notify) cv.notify_all();
    }
    if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

extern "C" stmf_status stmf_server_create(const stmf_server_config* cfg, stmf_server_t* out) {
  if (!cfg || !out || cfg->max_fits < 1 || cfg->n_max < 1 || cfg->n_max > 512 || cfg->r_max < 1 ||
      cfg->r_max > 64 || cfg->m_max < 1 || cfg->m_max > 64)
    return STMF_EINVAL;
  *out = nullptr;
  std::unique_ptr<stmf_server> srv(new stmf_server());
  srv->cfg = *cfg;
  srv->t0 = Clock::now();
  if (cudaSetDevice(cfg->device) != cudaSuccess) return STMF_EINVAL;
  // a failure part-way releases whatever was built (destroy skips what was not: no thread yet,
  // null handles)
  auto bail = [&srv](stmf_status st) {
    stmf_server_destroy(srv.release());
    return st;
  };
  // the largest workspaces any request may need (every storage type at n_max, r_max)
  const long long Dmax = cfg->r_max + (long long)cfg->n_max * cfg->r_max;
  srv->slots.resize(cfg->max_fits);
  for (auto& s : srv->slots) {
    stmf_status st = stmf_create(cfg->device, &s.ctx);
    if (st != STMF_OK) return bail(st);
    // many small fits run at once: a tensor-core pass takes whole SMs, so each CTA of a slot's
    // pass takes at least kSlotTiles tiles and the passes of other slots find SMs free
    stmf_set_pass_tiles(s.ctx, kSlotTiles);
    const size_t ws = stmf::fg_workspace_bytes_any(s.ctx, cfg->n_max, cfg->r_max);
    st = stmf::ensure_workspace(s.ctx, ws);
    if (st != STMF_OK) return bail(st);
    const size_t fb = stmf::fit_state_bytes(Dmax, cfg->m_max);
    if (cudaMalloc(&s.ctx->fit_ws, fb) != cudaSuccess) {
      s.ctx->fit_ws = nullptr;
      return bail(STMF_ENOMEM);
    }
    s.ctx->fit_ws_bytes = fb;
    srv->slot_bytes += s.ctx->ws_bytes + fb;
    if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&s.host_words, 2 * sizeof(int32_t)) != cudaSuccess ||
        cudaMallocHost(&s.state_host, stmf::FitRun::state_size()) != cudaSuccess)
      return bail(STMF_ECUDA);
  }
  if (srv->slot_bytes > cfg->mem_budget) return bail(STMF_ENOMEM);
  srv->avail = cfg->mem_budget - srv->slot_bytes;
  srv->stats.slot_bytes = srv->slot_bytes;
  if (cudaStreamCreateWithFlags(&srv->admin, cudaStreamNonBlocking) != cudaSuccess)
    return bail(STMF_ECUDA);
  if (cudaDeviceSynchronize() != cudaSuccess) return bail(STMF_ECUDA);
  stmf_server* raw = srv.get();
  srv->thr = std::thread([raw]() { raw->run(); });
  *out = srv.release();
  return STMF_OK;
}

extern "C" stmf_status stmf_server_destroy(stmf_server_t srv) {
  if (!srv) return STMF_OK;
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    for (auto& kv : srv->all) kv.second->cancel = true;
  }
  srv->stop.store(true);
  if (srv->thr.joinable()) srv->thr.join();
  cudaSetDevice(srv->cfg.device);
  cudaDeviceSynchronize();
  for (auto& kv : srv->all) {
    Request* r = kv.second.get();
    if (r->dmem) cudaFree(r->dmem);
    if (r->ready) cudaEventDestroy(r->ready);
    if (r->fin) cudaEventDestroy(r->fin);
  }
  for (auto& s : srv->slots) {
    s.run.release();
    if (s.ev) cudaEventDestroy(s.ev);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.host_words) cudaFreeHost(s.host_words);
    if (s.state_host) cudaFreeHost(s.state_host);
    if (s.ctx) stmf_destroy(s.ctx);
  }
  if (srv->admin) cudaStreamDestroy(srv->admin);
  delete srv;
  return STMF_OK;
}

extern "C" stmf_status stmf_submit(stmf_server_t srv, const stmf_request* q, uint64_t* ticket) {
  if (!srv || !q || !ticket) return STMF_EINVAL;
  const stmf_samples& V = q->V;
  const int eb = stmf::elem_bytes(V.dtype);
  if (!V.data || eb == 0 || V.n < 1 || V.n > srv->cfg.n_max || V.p < 1 || V.ld < V.n ||
      (V.ld * eb) % 16 != 0 || q->r < 1 || q->r > srv->cfg.r_max || q->d < 2 || q->d > 8 ||
      q->n_starts < 1 || q->n_starts > srv->cfg.max_fits || !q->x0 ||
      q->opts.m < 1 || q->opts.m > srv->cfg.m_max || q->opts.chunk < 1 ||
      ((V.dtype == STMF_E4M3) != (V.scale != nullptr)))
    return STMF_EINVAL;
  std::unique_ptr<Request> r(new Request());
  r->req = *q;
  r->D = q->r + V.n * q->r;
  r->x0.assign(q->x0, q->x0 + q->n_starts * r->D);
  r->v_bytes = q->V_on_host ? size_t(V.p) * V.ld * elem_size(V.dtype) : 0;
  r->s_bytes = (q->V_on_host && V.scale) ? size_t(V.p) * sizeof(float) : 0;
  r->footprint =
      ((r->v_bytes + r->s_bytes + 255) & ~size_t(255)) + sizeof(double) * r->x0.size() + 256;
  if (r->footprint > srv->avail) return STMF_ENOMEM;
  {
    // the request's events belong to the server's device, whatever device the caller has current
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return STMF_ECUDA;
    if (prev != srv->cfg.device && cudaSetDevice(srv->cfg.device) != cudaSuccess)
      return STMF_ECUDA;
    const bool ok = cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming) == cudaSuccess &&
                    cudaEventCreateWithFlags(&r->fin, cudaEventDisableTiming) == cudaSuccess;
    if (prev != srv->cfg.device) cudaSetDevice(prev);
    if (!ok) {
      if (r->ready) cudaEventDestroy(r->ready);
      return STMF_ECUDA;
    }
  }
  std::lock_guard<std::mutex> lock(srv->mu);
  r->ticket = srv->next_ticket++;
  r->t_submit = srv->now();
  *ticket = r->ticket;
  srv->queue.push_back(r.get());
  ++srv->stats.submitted;
  srv->all[r->ticket] = std::move(r);
  return STMF_OK;
}

extern "C" stmf_status stmf_poll(stmf_server_t srv, uint64_t ticket, stmf_request_result* out,
                                 int32_t timeout_ms) {
  if (!srv || !out) return STMF_EINVAL;
  std::unique_lock<std::mutex> lock(srv->mu);
  // the request is looked up again after every wait: a concurrent poll may release it
  auto find = [srv, ticket]() -> Request* {
    auto it = srv->all.find(ticket);
    return it == srv->all.end() ? nullptr : it->second.get();
  };
  auto settled = [&find]() {
    Request* q = find();
    return !q || q->state == RQ_DONE;
  };
  if (!find()) return STMF_EINVAL;
  if (!settled()) {
    if (timeout_ms < 0) srv->cv.wait(lock, settled);
    else if (timeout_ms > 0) srv->cv.wait_for(lock, std::chrono::milliseconds(timeout_ms), settled);
  }
  Request* r = find();
  if (!r) return STMF_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->t_submit = r->t_submit;
  out->t_admit = r->t_admit;
  out->footprint = r->footprint;
  if (r->state != RQ_DONE) {
    out->state = STMF_ENOTREADY;
    return STMF_ENOTREADY;
  }
  out->state = r->status;
  out->best_start = r->best_start;
  out->best = r->best;
  out->total_evals = r->total_evals;
  out->t_done = r->t_done;
  // the result has been delivered: release the ticket (no queue, slot or stream refers to a
  // finished request, and its device memory went back at finalisation)
  if (r->ready) cudaEventDestroy(r->ready);
  if (r->fin) cudaEventDestroy(r->fin);
  srv->all.erase(ticket);
  return STMF_OK;
}

extern "C" stmf_status stmf_cancel(stmf_server_t srv, uint64_t ticket) {
  if (!srv) return STMF_EINVAL;
  std::lock_guard<std::mutex> lock(srv->mu);
  auto it = srv->all.find(ticket);
  if (it == srv->all.end()) return STMF_EINVAL;
  it->second->cancel = true;
  return STMF_OK;
}

extern "C" stmf_status stmf_server_get_stats(stmf_server_t srv, stmf_server_stats* out) {
  if (!srv || !out) return STMF_EINVAL;
  std::lock_guard<std::mutex> lock(srv->mu);
  *out = srv->stats;
  out->now = srv->now();
  return STMF_OK;
}
