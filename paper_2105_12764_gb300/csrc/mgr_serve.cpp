// mgr_serve.cpp -- serving loop for decompose / recompose requests.
//
// Continuous batching on one GPU: requests enter a FIFO admission queue; a
// dispatcher thread admits the head request as soon as an execution slot is
// free and its device memory (workspace, plus the resident hierarchy for a
// decomposition) fits the context's memory budget, evicting least recently
// used unpinned resident hierarchies if needed.  Admitted requests are
// launched on a pool of streams, so requests that arrive while others run
// overlap on the device; completion is detected by events, which frees the
// slot and the workspace and admits the next requests.  A decomposition's
// output (its hierarchy) stays resident under a handle when asked, and a
// recomposition reads a resident hierarchy (pinned while the request waits
// or runs).  Device memory comes from the stream-ordered allocator.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "mgr_internal.h"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum { R_QUEUED = 0, R_RUNNING = 1, R_DONE = 2, R_FAILED = 3 };

struct Req {
  uint64_t id = 0;
  mgr_serve_request r{};
  double t_arrival = 0, t_admit = 0, t_done = 0;
  int state = R_QUEUED;
  int rc = MGR_OK;
  int stream = 0;
  cudaEvent_t ev = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* hier = nullptr;  // decompose output
  size_t hier_bytes = 0;
};

struct Hier {
  void* buf = nullptr;
  size_t bytes = 0;
  const mgr_plan* plan = nullptr;
  int pins = 0;
  bool ready = false;
  uint64_t last_use = 0;
};

}  // namespace

struct mgr_server {
  mgr_ctx* ctx = nullptr;
  int slots = 1;
  std::vector<cudaStream_t> streams;
  int next_stream = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> queue;
  std::vector<Req*> running;
  std::map<uint64_t, std::unique_ptr<Req>> reqs;
  std::map<uint64_t, Hier> hiers;
  size_t used = 0;  // bytes of resident hierarchies + in-flight workspaces
  uint64_t next_id = 1, clock = 0;
  bool stop = false;
  std::thread worker;
};

namespace {

size_t field_bytes(const mgr_plan* p) { return size_t(p->count) * p->elem; }

// Free unpinned resident hierarchies, least recently used first, until
// `need` more bytes fit the budget.  Caller holds the lock.
bool make_room(mgr_server* s, size_t need) {
  const size_t budget = s->ctx->budget;
  if (!budget) return true;
  while (s->used + need > budget) {
    uint64_t victim = 0;
    uint64_t best = UINT64_MAX;
    for (auto& kv : s->hiers)
      if (kv.second.ready && kv.second.pins == 0 && kv.second.last_use < best) {
        best = kv.second.last_use;
        victim = kv.first;
      }
    if (!victim) return false;
    Hier& h = s->hiers[victim];
    cudaFreeAsync(h.buf, s->streams[0]);
    s->used -= h.bytes;
    s->hiers.erase(victim);
  }
  return true;
}

void complete(mgr_server* s, Req* r, int rc) {
  r->t_done = now_s();
  r->rc = rc;
  r->state = rc == MGR_OK ? R_DONE : R_FAILED;
  if (r->ws) {
    cudaFreeAsync(r->ws, s->streams[r->stream]);
    s->used -= r->ws_bytes;
    r->ws = nullptr;
  }
  if (r->r.op == MGR_OP_DECOMPOSE) {
    auto it = s->hiers.find(r->id);
    if (it != s->hiers.end()) {
      if (rc == MGR_OK && r->r.keep_resident) {
        it->second.ready = true;
        it->second.last_use = ++s->clock;
      } else {
        cudaFreeAsync(it->second.buf, s->streams[r->stream]);
        s->used -= it->second.bytes;
        s->hiers.erase(it);
      }
    }
  } else {
    auto it = s->hiers.find(r->r.src);
    if (it != s->hiers.end()) {
      it->second.pins--;
      it->second.last_use = ++s->clock;
    }
  }
  if (r->ev) {
    cudaEventDestroy(r->ev);
    r->ev = nullptr;
  }
}

// Try to admit and launch the queue head.  Returns false when it must wait.
bool admit_one(mgr_server* s) {
  Req* r = s->queue.front();
  const mgr_plan* p = r->r.plan;
  const size_t ws = (p->ws_bytes + 255) & ~size_t(255);
  const size_t out = r->r.op == MGR_OP_DECOMPOSE ? field_bytes(p) : 0;
  if (!make_room(s, ws + out)) return false;
  const int si = s->next_stream;
  s->next_stream = (s->next_stream + 1) % int(s->streams.size());
  cudaStream_t st = s->streams[si];
  r->stream = si;
  int rc = MGR_OK;
  if (mgr::fault_injected("admit")) rc = MGR_EBUDGET;
  else if (mgr::fault_injected("alloc")) rc = MGR_ENOMEM;
  if (rc == MGR_OK && ws && cudaMallocAsync(&r->ws, ws, st) != cudaSuccess) rc = MGR_ENOMEM;
  r->ws_bytes = r->ws ? ws : 0;
  s->used += r->ws_bytes;
  const void* src = r->r.in;
  void* dst = r->r.out;
  if (rc == MGR_OK && r->r.op == MGR_OP_DECOMPOSE) {
    if (cudaMallocAsync(&r->hier, out, st) != cudaSuccess) {
      rc = MGR_ENOMEM;
    } else {
      Hier h;
      h.buf = r->hier;
      h.bytes = out;
      h.plan = p;
      s->hiers[r->id] = h;
      s->used += out;
      dst = r->hier;
    }
  } else if (rc == MGR_OK) {
    src = s->hiers[r->r.src].buf;  // pinned at enqueue, so still resident
  }
  if (rc == MGR_OK && mgr::fault_injected("launch")) rc = MGR_ECUDA;
  if (rc == MGR_OK) {
    cudaError_t e = r->r.op == MGR_OP_DECOMPOSE ? mgr::enqueue_decompose(p, src, dst, r->ws, st)
                                                : mgr::enqueue_recompose(p, src, dst, r->ws, st);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(r->ev, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      rc = MGR_ECUDA;
    }
  }
  s->queue.pop_front();
  r->t_admit = now_s();
  if (rc != MGR_OK) {
    complete(s, r, rc);
    s->cv_done.notify_all();
    return true;
  }
  r->state = R_RUNNING;
  s->running.push_back(r);
  return true;
}

void worker_loop(mgr_server* s) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    bool progress = false;
    for (size_t i = 0; i < s->running.size();) {
      Req* r = s->running[i];
      const cudaError_t q = cudaEventQuery(r->ev);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      if (q != cudaSuccess) cudaGetLastError();
      complete(s, r, q == cudaSuccess ? MGR_OK : MGR_ECUDA);
      s->running.erase(s->running.begin() + long(i));
      progress = true;
    }
    if (progress) s->cv_done.notify_all();
    while (!s->queue.empty() && int(s->running.size()) < s->slots) {
      if (admit_one(s)) {
        progress = true;
        continue;
      }
      if (s->running.empty()) {
        // nothing runs and the head still does not fit (the memory is held by
        // hierarchies pinned by later requests): fail it rather than wait forever
        Req* r = s->queue.front();
        s->queue.pop_front();
        r->t_admit = now_s();
        complete(s, r, MGR_EBUDGET);
        s->cv_done.notify_all();
        progress = true;
        continue;
      }
      break;
    }
    if (s->running.empty() && s->queue.empty()) {
      s->cv_work.wait(lk);
    } else if (!progress) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(10));
      lk.lock();
    }
  }
}

}  // namespace

extern "C" {

double mgr_serve_now(void) { return now_s(); }

int mgr_serve_start(mgr_ctx* ctx, int slots, int nstreams, mgr_server** out) {
  if (!ctx || !out || slots < 1 || nstreams < 1 || nstreams > 64) return MGR_EINVAL;
  *out = nullptr;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return MGR_ECUDA;
  auto s = std::make_unique<mgr_server>();
  s->ctx = ctx;
  s->slots = slots;
  // keep freed blocks in the stream-ordered pool instead of returning them
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
    uint64_t thr = ctx->budget ? uint64_t(ctx->budget) : UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  for (int i = 0; i < nstreams; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto x : s->streams) cudaStreamDestroy(x);
      return MGR_ECUDA;
    }
    s->streams.push_back(st);
  }
  mgr_server* raw = s.release();
  raw->worker = std::thread(worker_loop, raw);
  *out = raw;
  return MGR_OK;
}

int mgr_serve_enqueue(mgr_server* s, const mgr_serve_request* req, uint64_t* id) {
  if (!s || !req || !id || !req->plan) return MGR_EINVAL;
  *id = 0;
  const mgr_plan* p = req->plan;
  if (p->ctx != s->ctx) return MGR_EINVAL;
  if (req->op == MGR_OP_DECOMPOSE) {
    if (!req->in) return MGR_EINVAL;
  } else if (req->op == MGR_OP_RECOMPOSE) {
    if (!req->out) return MGR_EINVAL;
  } else {
    return MGR_EINVAL;
  }
  const size_t need = ((p->ws_bytes + 255) & ~size_t(255)) + (req->op == MGR_OP_DECOMPOSE ? field_bytes(p) : 0);
  if (s->ctx->budget && need > s->ctx->budget) return MGR_EBUDGET;
  std::lock_guard<std::mutex> lk(s->mu);
  if (req->op == MGR_OP_RECOMPOSE) {
    auto it = s->hiers.find(req->src);
    if (it == s->hiers.end()) return MGR_ENOTFOUND;
    if (!it->second.ready) return MGR_EPENDING;  // its decomposition has not finished
    if (it->second.plan->count != p->count || it->second.plan->elem != p->elem) return MGR_EINVAL;
    it->second.pins++;  // resident until this request completes
  }
  auto r = std::make_unique<Req>();
  r->id = s->next_id++;
  r->r = *req;
  r->t_arrival = req->arrival > 0 ? req->arrival : now_s();
  *id = r->id;
  s->queue.push_back(r.get());
  s->reqs[r->id] = std::move(r);
  s->cv_work.notify_one();
  return MGR_OK;
}

int mgr_serve_wait(mgr_server* s, uint64_t id, int64_t timeout_us, mgr_serve_result* res) {
  if (!s || !res) return MGR_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return MGR_ENOTFOUND;
  Req* r = it->second.get();
  auto done = [&] { return r->state == R_DONE || r->state == R_FAILED; };
  if (!done()) {
    if (timeout_us == 0) return MGR_EPENDING;
    if (timeout_us < 0) {
      s->cv_done.wait(lk, done);
    } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done)) {
      return MGR_ETIMEDOUT;
    }
  }
  res->status = r->rc;
#ifdef MGR_DEBUG_BOUNDS
  // bounds-checking builds: an out-of-bounds access of the finished request
  if (r->rc == MGR_OK) {
    mgr::DebugRecord rec{};
    if (mgr::debug_take(&rec)) {
      std::lock_guard<std::mutex> dl(mgr::g_dbg_mu);
      mgr::g_dbg_last = rec;
      mgr::g_dbg_have = true;
      res->status = MGR_EDEVICE;
    }
  }
#endif
  res->arrival = r->t_arrival;
  res->admitted = r->t_admit;
  res->done = r->t_done;
  res->handle = (r->r.op == MGR_OP_DECOMPOSE && r->rc == MGR_OK && r->r.keep_resident) ? r->id : 0;
  s->reqs.erase(it);
  return MGR_OK;
}

int mgr_serve_hierarchy(mgr_server* s, uint64_t handle, const void** ptr) {
  if (!s || !ptr) return MGR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->hiers.find(handle);
  if (it == s->hiers.end() || !it->second.ready) return MGR_ENOTFOUND;
  *ptr = it->second.buf;
  return MGR_OK;
}

int mgr_serve_read(mgr_server* s, uint64_t handle, void* dst, mgr_stream_t stream) {
  if (!s || !dst) return MGR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->hiers.find(handle);
  if (it == s->hiers.end() || !it->second.ready) return MGR_ENOTFOUND;
  it->second.last_use = ++s->clock;
  return cudaMemcpyAsync(dst, it->second.buf, it->second.bytes, cudaMemcpyDeviceToDevice,
                         reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? MGR_OK
             : MGR_ECUDA;
}

int mgr_serve_release(mgr_server* s, uint64_t handle) {
  if (!s) return MGR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->hiers.find(handle);
  if (it == s->hiers.end()) return MGR_ENOTFOUND;
  if (it->second.pins > 0 || !it->second.ready) return MGR_EPENDING;
  cudaFreeAsync(it->second.buf, s->streams[0]);
  s->used -= it->second.bytes;
  s->hiers.erase(it);
  return MGR_OK;
}

int mgr_serve_stats(mgr_server* s, size_t* used_bytes, int* queued, int* running, int* resident) {
  if (!s) return MGR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (used_bytes) *used_bytes = s->used;
  if (queued) *queued = int(s->queue.size());
  if (running) *running = int(s->running.size());
  if (resident) *resident = int(s->hiers.size());
  return MGR_OK;
}

int mgr_serve_stop(mgr_server* s) {
  if (!s) return MGR_EINVAL;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    // let admitted and queued work finish
    while (!s->queue.empty() || !s->running.empty()) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(100));
      lk.lock();
      if (s->running.empty() && !s->queue.empty()) s->cv_work.notify_one();
    }
    s->stop = true;
    s->cv_work.notify_all();
  }
  s->worker.join();
  for (auto& kv : s->hiers) cudaFreeAsync(kv.second.buf, s->streams[0]);
  for (auto st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  delete s;
  return MGR_OK;
}

}  // extern "C"
