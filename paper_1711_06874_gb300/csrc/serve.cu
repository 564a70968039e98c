// Serving loop with continuous batching: requests are queued by tk_submit and
// taken by worker threads, each with its own CUDA stream and workspaces.  A
// free worker takes the oldest request together with every queued request of
// the same bucket (same grid, precision, caps; different eps and kernels),
// as many as the device memory admits, and solves them as one batch; requests
// that arrive meanwhile wait for the next free worker, so batches keep
// forming while others run and their work overlaps on the device.  Results
// (factors and cores) stay in device memory until the caller takes them with
// tk_poll.  A request's result is bitwise the one it gets alone (the batched
// engine does not depend on the batch around an instance).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <memory>
#include <new>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tk_internal.h"

using Clock = std::chrono::steady_clock;

struct tk_server {
  tk_ctx* ctx = nullptr;
  tk_serve_opts opts{};
  std::mutex mu;
  std::condition_variable work_cv;  // queue changed or memory released
  std::condition_variable done_cv;  // a batch finished
  bool stop = false;

  struct Pending {
    uint64_t ticket;
    tk::SolveReq req;
    tk::BucketKey key;
    Clock::time_point t0;
  };
  struct Done {
    tk_result* res = nullptr;
    int status = TK_OK;
    double latency = 0.0;
  };
  std::deque<Pending> queue;
  std::unordered_map<uint64_t, Done> done;
  std::unordered_map<uint64_t, bool> running;
  uint64_t next_ticket = 1;
  size_t in_flight_bytes = 0;
  int in_flight = 0;
  size_t budget = 0;
  tk_serve_stats stats{};
  std::vector<std::thread> workers;

  void worker_main(int wid);
};

namespace {

using namespace tk;

struct WorkerState {
  Workspace pre, post;
  HostPinned pin;
  SideStream side;
  GraphCache graphs;
  cudaStream_t stream = nullptr;
};

}  // namespace

void tk_server::worker_main(int /*wid*/) {
  cudaSetDevice(ctx->device);
  WorkerState w;
  if (cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    w.stream = nullptr;
  }
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    work_cv.wait(lk, [&] { return stop || !queue.empty(); });
    if (queue.empty()) {
      if (stop) break;
      continue;
    }
    // the oldest request fixes the bucket; take every queued request of it
    // that the memory budget admits
    const BucketKey key = queue.front().key;
    const size_t per = bucket_bytes_per_instance(key);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      free_b = budget;
    }
    const size_t room_now = (size_t)(free_b * opts.mem_fraction);
    size_t avail = std::min(budget, room_now);
    avail = (avail > in_flight_bytes) ? avail - in_flight_bytes : 0;
    std::vector<Pending> batch;
    for (auto it = queue.begin(); it != queue.end() && (int)batch.size() < opts.max_batch;) {
      if (it->key == key && (batch.size() + 1) * per <= avail) {
        batch.push_back(*it);
        it = queue.erase(it);
      } else {
        ++it;
      }
    }
    if (batch.empty()) {
      if (in_flight > 0) {  // wait for memory to come back
        work_cv.wait(lk);
        continue;
      }
      batch.push_back(queue.front());  // nothing else runs: try it alone
      queue.pop_front();
    }
    const size_t bytes = batch.size() * per;
    in_flight_bytes += bytes;
    ++in_flight;
    for (auto& p : batch) running[p.ticket] = true;
    stats.batches += 1;
    stats.max_batch_seen = std::max<uint64_t>(stats.max_batch_seen, batch.size());
    stats.bytes_peak = std::max<uint64_t>(stats.bytes_peak, in_flight_bytes);
    lk.unlock();

    std::vector<SolveReq> reqs(batch.size());
    for (size_t i = 0; i < batch.size(); ++i) reqs[i] = batch[i].req;
    std::vector<tk_result*> outs(batch.size(), nullptr);
    int status = TK_OK;
    try {
      if (!w.stream) fail(TK_ECUDA, "cannot create a worker stream");
      solve_bucket(ctx, w.pre, w.post, w.pin, w.side, &w.graphs, nullptr, reqs.data(), (int)reqs.size(), outs.data(), w.stream);
    } catch (const Error& e) {
      status = e.status;
    } catch (...) {
      status = TK_ECUDA;
    }
    if (status != TK_OK) {
      cudaGetLastError();
      for (auto& r : outs)
        if (r) {
          tk_result_free(r);
          r = nullptr;
        }
    }
    const Clock::time_point t1 = Clock::now();

    lk.lock();
    for (size_t i = 0; i < batch.size(); ++i) {
      Done d;
      d.res = outs[i];
      d.status = status;
      d.latency = std::chrono::duration<double>(t1 - batch[i].t0).count();
      running.erase(batch[i].ticket);
      done[batch[i].ticket] = d;
    }
    if (status == TK_OK)
      stats.completed += batch.size();
    else
      stats.failed += batch.size();
    in_flight_bytes -= bytes;
    --in_flight;
    work_cv.notify_all();
    done_cv.notify_all();
  }
  lk.unlock();
  w.graphs.release();
  w.pre.release();
  w.post.release();
  if (w.stream) {
    cudaStreamSynchronize(w.stream);
    cudaStreamDestroy(w.stream);
  }
}

extern "C" {

void tk_default_serve_opts(tk_serve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->workers = 2;
  o->max_batch = 256;
  o->mem_fraction = 0.8;
}

int tk_serve_start(tk_ctx* ctx, const tk_serve_opts* opts) {
  if (!ctx || !opts) return TK_EINVAL;
  if (opts->workers < 1 || opts->workers > 8 || opts->max_batch < 1 || opts->max_batch > 4096 ||
      !(opts->mem_fraction > 0.0 && opts->mem_fraction <= 0.95))
    return TK_EINVAL;
  for (int i = 0; i < 4; ++i)
    if (opts->reserved[i] != 0) return TK_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->server_mu);
  if (ctx->server) return TK_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    cudaGetLastError();
    return TK_ECUDA;
  }
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return TK_ECUDA;
  }
  std::shared_ptr<tk_server> sv;
  try {
    sv = std::make_shared<tk_server>();
  } catch (...) {
    return TK_ENOMEM;
  }
  sv->ctx = ctx;
  sv->opts = *opts;
  sv->budget = (size_t)(free_b * opts->mem_fraction);
  sv->stats.bytes_budget = sv->budget;
  for (int i = 0; i < opts->workers; ++i) sv->workers.emplace_back(&tk_server::worker_main, sv.get(), i);
  ctx->server = sv;
  return TK_OK;
}

static std::shared_ptr<tk_server> server_of(tk_ctx* ctx) {
  std::lock_guard<std::mutex> lock(ctx->server_mu);
  return ctx->server;
}

int tk_serve_stop(tk_ctx* ctx) {
  if (!ctx) return TK_EINVAL;
  std::shared_ptr<tk_server> sv;
  {
    std::lock_guard<std::mutex> lock(ctx->server_mu);
    sv = ctx->server;
    ctx->server.reset();
  }
  if (!sv) return TK_EINVAL;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->work_cv.notify_all();
  for (auto& t : sv->workers) t.join();
  std::lock_guard<std::mutex> lk(sv->mu);
  for (auto& kv : sv->done)
    if (kv.second.res) tk_result_free(kv.second.res);
  sv->done.clear();
  sv->done_cv.notify_all();
  return TK_OK;
}

int tk_submit(tk_ctx* ctx, const tk_kernel* kernel, const tk_grid* grid, const tk_opts* opts, uint64_t* ticket) {
  if (!ctx || !kernel || !grid || !opts || !ticket) return TK_EINVAL;
  std::shared_ptr<tk_server> sv = server_of(ctx);
  if (!sv) return TK_EINVAL;
  const int rc = validate_request(kernel, grid, opts);
  if (rc != TK_OK) return rc;
  if (!fold_applicable(*grid, *opts)) return TK_EINVAL;  // serving runs the folded engine only
  tk_server::Pending p;
  p.req = SolveReq{*kernel, *grid, *opts};
  p.key = bucket_key(p.req);
  p.t0 = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return TK_EINVAL;
    p.ticket = sv->next_ticket++;
    sv->queue.push_back(p);
    sv->stats.submitted += 1;
  }
  sv->work_cv.notify_one();
  *ticket = p.ticket;
  return TK_OK;
}

int tk_poll(tk_ctx* ctx, uint64_t ticket, tk_result** out, double* latency_s, double wait_s) {
  if (!ctx || !out) return TK_EINVAL;
  std::shared_ptr<tk_server> sv = server_of(ctx);
  if (!sv) return TK_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto ready = [&] { return sv->done.count(ticket) > 0; };
  auto known = [&] {
    if (sv->done.count(ticket) || sv->running.count(ticket)) return true;
    for (const auto& p : sv->queue)
      if (p.ticket == ticket) return true;
    return false;
  };
  if (!known()) return TK_ENOTFOUND;
  if (!ready() && wait_s > 0.0)
    sv->done_cv.wait_for(lk, std::chrono::duration<double>(wait_s), [&] { return ready() || sv->stop; });
  if (!ready()) return TK_EBUSY;
  auto it = sv->done.find(ticket);
  const tk_server::Done d = it->second;
  sv->done.erase(it);
  if (latency_s) *latency_s = d.latency;
  *out = d.res;
  return d.status;
}

int tk_serve_read_stats(tk_ctx* ctx, tk_serve_stats* out) {
  if (!ctx || !out) return TK_EINVAL;
  std::shared_ptr<tk_server> sv = server_of(ctx);
  if (!sv) return TK_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  *out = sv->stats;
  out->queued = sv->queue.size();
  out->in_flight_batches = (uint64_t)sv->in_flight;
  return TK_OK;
}

}  // extern "C"
