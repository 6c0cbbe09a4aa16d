// mgr_api.cpp -- C ABI entry points (include/mgr.h): context, plans,
// workspace sizing, argument checks, and the CUDA-graph cache that replays a
// plan's whole launch sequence (all levels) as one graph launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>

#include "mgr_internal.h"

namespace mgr {

cudaError_t raise_smem_limit(const void* fn, size_t bytes) {
  // the default limit (48 KB) covers static and dynamic shared memory together
  constexpr size_t kDefault = 48 * 1024;
  if (bytes == 0) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  struct Limit {
    size_t static_bytes = 0;
    size_t dynamic = 0;  // the dynamic limit set so far (0: the default)
    bool known = false;
  };
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, Limit> limits;
  std::lock_guard<std::mutex> lk(mu);
  Limit& cur = limits[{dev, fn}];
  if (!cur.known) {
    cudaFuncAttributes at{};
    e = cudaFuncGetAttributes(&at, fn);
    if (e != cudaSuccess) return e;
    cur.static_bytes = at.sharedSizeBytes;
    cur.known = true;
  }
  if (bytes + cur.static_bytes <= kDefault || bytes <= cur.dynamic) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  if (e == cudaSuccess) cur.dynamic = bytes;
  return e;
}

unsigned long long debug_take(DebugRecord* first) {
  DebugRecord r[3] = {};
  const unsigned long long n[3] = {debug_take_core(&r[0]), debug_take_batch(&r[1]), debug_take_st(&r[2])};
  unsigned long long total = 0;
  for (int i = 0; i < 3; ++i) {
    if (n[i] && first && total == 0) *first = r[i];
    total += n[i];
  }
  return total;
}

// Bounds-checking builds: the first out-of-bounds access of the last
// operation that reported one (mgr_debug_last).
std::mutex g_dbg_mu;
DebugRecord g_dbg_last{};
bool g_dbg_have = false;

// After an operation is enqueued on `st`: in bounds-checking builds wait for
// it (unless `st` is being captured) and report a recorded out-of-bounds
// access as MGR_EDEVICE; otherwise nothing.
int debug_after(cudaStream_t st) {
#ifdef MGR_DEBUG_BOUNDS
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return MGR_OK;
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return MGR_ECUDA;
  }
  DebugRecord r{};
  if (debug_take(&r)) {
    std::lock_guard<std::mutex> lk(g_dbg_mu);
    g_dbg_last = r;
    g_dbg_have = true;
    return MGR_EDEVICE;
  }
#else
  (void)st;
#endif
  return MGR_OK;
}

bool fault_injected(const char* what) {
  const char* v = std::getenv("MGR_FAULT_INJECT");
  if (!v || !*v) return false;
  const std::string list = std::string(",") + v + ",";
  return list.find(std::string(",") + what + ",") != std::string::npos;
}

}  // namespace mgr

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + nb && pb < pa + na;
}

int check_sticky() {
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    cudaGetLastError();
    return MGR_ECUDA;
  }
  return MGR_OK;
}

// Operation codes of run_op / the graph cache; OP_REC_PACKED and OP_REC_DEQ
// carry the number of classes in bits 8 and up.
enum { OP_DEC = 0, OP_REC = 1, OP_DEC_PACKED = 2, OP_REC_PACKED = 3, OP_DEC_QUANT = 4, OP_REC_DEQ = 5,
       OP_DEC_HOST = 6, OP_REC_HOST = 7 /* graph-cache keys of the pipelined host-buffer operations */ };

// Arguments of the quantized operations (part of the graph-cache key).
struct Extra {
  double tau = 0.0;
  unsigned long long* sat = nullptr;
};

int check_op_args(const mgr_plan* p, const void* in, const void* out, const void* ws, bool alias_ok = true) {
  if (!p || !in || !out) return MGR_EINVAL;
  if (p->desc.ndim == 4) alias_ok = false;  // the spatiotemporal form is out of place
  const size_t bytes = size_t(p->count) * p->elem;
  if ((reinterpret_cast<uintptr_t>(in) % p->elem) || (reinterpret_cast<uintptr_t>(out) % p->elem)) return MGR_EINVAL;
  if ((in != out || !alias_ok) && ranges_overlap(in, bytes, out, bytes)) return MGR_EINVAL;
  if (p->ws_bytes > 0) {
    if (!ws || (reinterpret_cast<uintptr_t>(ws) % kAlign)) return MGR_EINVAL;
    if (ranges_overlap(ws, p->ws_bytes, in, bytes) || ranges_overlap(ws, p->ws_bytes, out, bytes)) return MGR_EINVAL;
  }
  return MGR_OK;
}

cudaError_t enqueue(const mgr_plan* p, int op, const void* in, void* out, void* ws, cudaStream_t st,
                    const Extra& x = Extra{}) {
  std::vector<double> bins;
  if ((op & 0xff) >= OP_DEC_QUANT && mgr::quant_bins(const_cast<mgr_plan*>(p), x.tau, bins) != MGR_OK)
    return cudaErrorInvalidValue;
  switch (op & 0xff) {
    case OP_DEC: return mgr::enqueue_decompose(p, in, out, ws, st);
    case OP_REC: return mgr::enqueue_recompose(p, in, out, ws, st);
    case OP_DEC_PACKED: return mgr::enqueue_decompose_packed(p, in, out, ws, st);
    case OP_REC_PACKED: return mgr::enqueue_recompose_packed(p, in, op >> 8, out, ws, st);
    case OP_DEC_QUANT: return mgr::enqueue_decompose_quantized(p, in, static_cast<int*>(out), bins.data(), x.sat, ws, st);
    default: return mgr::enqueue_recompose_dequantized(p, static_cast<const int*>(in), op >> 8, bins.data(), out, ws, st);
  }
}

bool packed_op(int op) { return (op & 0xff) >= OP_DEC_PACKED; }

// The side streams and events of a forked recomposition graph (graph_mu held).
bool ensure_fork(mgr_plan* p) {
  if (p->side) return true;
  if (!p->side2 && cudaStreamCreateWithFlags(&p->side2, cudaStreamNonBlocking) != cudaSuccess) return false;
  if (cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess) return false;
  p->fork_ev.assign(p->levels + 1, nullptr);
  for (auto& e : p->fork_ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return false;
  return true;
}

// Enqueue while capturing a graph (graph_mu held): recompositions fork their
// load-vector passes onto the plan's side stream.
cudaError_t enqueue_captured(mgr_plan* p, int op, const void* in, void* out, void* ws, cudaStream_t cs, const Extra& x) {
  const int base = op & 0xff;
  const bool rec = base == OP_REC || base == OP_REC_PACKED || base == OP_REC_DEQ;
  if (!rec || p->desc.ndim == 4 || p->levels < 1) return enqueue(p, op, in, out, ws, cs, x);
  if (!ensure_fork(p)) return cudaErrorMemoryAllocation;
  std::vector<double> bins;
  if (base == OP_REC_DEQ && mgr::quant_bins(p, x.tau, bins) != MGR_OK) return cudaErrorInvalidValue;
  const int ncls = base == OP_REC ? p->levels + 1 : (op >> 8);
  const int kind = base == OP_REC ? 0 : (base == OP_REC_PACKED ? 1 : 2);
  return mgr::enqueue_recompose_fork(p, kind, in, ncls, bins.data(), out, ws, cs, mgr::ForkCtx{p->side, p->fork_ev.data(), p->side2});
}

// Arguments of a quantized operation: the field (elem bytes per element) and
// the int32 codes must be aligned and must not overlap.
int check_quant_args(const mgr_plan* p, const void* field, const void* codes, const void* ws, double tau) {
  if (!p || !field || !codes || !(tau > 0.0)) return MGR_EINVAL;
  if ((reinterpret_cast<uintptr_t>(field) % p->elem) || (reinterpret_cast<uintptr_t>(codes) % 4)) return MGR_EINVAL;
  const size_t fb = size_t(p->count) * p->elem, cb = size_t(p->count) * 4;
  if (ranges_overlap(field, fb, codes, cb)) return MGR_EINVAL;
  if (p->ws_bytes > 0) {
    if (!ws || (reinterpret_cast<uintptr_t>(ws) % kAlign)) return MGR_EINVAL;
    if (ranges_overlap(ws, p->ws_bytes, field, fb) || ranges_overlap(ws, p->ws_bytes, codes, cb)) return MGR_EINVAL;
  }
  return MGR_OK;
}

int run_op_graph(mgr_plan* p, int op, const void* in, void* out, void* ws, cudaStream_t st, const Extra& x);

// Launch through a cached CUDA graph of the plan's launch sequence.  When the
// caller's stream is itself being captured the kernels are enqueued directly
// (they become part of the caller's graph).
int run_op(const mgr_plan* cp, int op, const void* in, void* out, void* ws, cudaStream_t st,
           const Extra& x = Extra{}) {
  mgr_plan* p = const_cast<mgr_plan*>(cp);
  if (p && p->desc.ndim == 4 && packed_op(op)) return MGR_EINVAL;  // 4D: nodal layout only
  int rc = (op & 0xff) == OP_DEC_QUANT  ? check_quant_args(p, in, out, ws, x.tau)
           : (op & 0xff) == OP_REC_DEQ ? check_quant_args(p, out, in, ws, x.tau)
                                        : check_op_args(p, in, out, ws, !packed_op(op));
  if (rc != MGR_OK) return rc;
  if ((rc = check_sticky()) != MGR_OK) return rc;
  if (mgr::fault_injected("launch")) return MGR_ECUDA;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return MGR_ECUDA;
  if (cap != cudaStreamCaptureStatusNone) return enqueue(p, op, in, out, ws, st, x) == cudaSuccess ? MGR_OK : MGR_ECUDA;
  const int launched = run_op_graph(p, op, in, out, ws, st, x);
  return launched != MGR_OK ? launched : mgr::debug_after(st);
}

// The cached-graph launch of run_op.
int run_op_graph(mgr_plan* p, int op, const void* in, void* out, void* ws, cudaStream_t st, const Extra& x) {

  std::lock_guard<std::mutex> lk(p->graph_mu);
  cudaGraphExec_t exec = nullptr;
  for (auto& g : p->graphs)
    if (g.op == op && g.in == in && g.out == out && g.ws == ws && g.tau == x.tau && g.aux == x.sat) exec = g.exec;
  if (!exec) {
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return MGR_ECUDA;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = enqueue_captured(p, op, in, out, ws, cs, x);
      e = cudaStreamEndCapture(cs, &graph);
      if (e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return MGR_ECUDA;
    }
    if (p->graphs.size() >= 8) {
      cudaGraphExecDestroy(p->graphs.front().exec);
      p->graphs.erase(p->graphs.begin());
    }
    p->graphs.push_back({op, in, out, ws, x.tau, x.sat, exec});
  }
  return cudaGraphLaunch(exec, st) == cudaSuccess ? MGR_OK : MGR_ECUDA;
}

// page-locked (or registered) host memory
bool host_pinned(const void* ptr) {
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeHost;
}

// A decomposition or recomposition with pinned host buffers as one cached
// graph whose copies overlap its kernels (mgr::PipeCtx).
int run_host_pipe(mgr_plan* p, int op, const void* host_in, void* host_out, void* dev_in, void* dev_out, void* ws,
                  cudaStream_t st) {
  const int key = op == OP_DEC ? OP_DEC_HOST : OP_REC_HOST;
  int rc = check_op_args(p, dev_in, dev_out, ws, false);
  if (rc != MGR_OK) return rc;
  if ((rc = check_sticky()) != MGR_OK) return rc;
  if (mgr::fault_injected("launch")) return MGR_ECUDA;
  std::lock_guard<std::mutex> lk(p->graph_mu);
  cudaGraphExec_t exec = nullptr;
  for (auto& g : p->graphs)
    if (g.op == key && g.in == host_in && g.out == host_out && g.ws == ws && g.din == dev_in && g.dout == dev_out)
      exec = g.exec;
  if (!exec) {
    if (!p->pipe_h2d) {
      if (cudaStreamCreateWithFlags(&p->pipe_h2d, cudaStreamNonBlocking) != cudaSuccess ||
          cudaStreamCreateWithFlags(&p->pipe_d2h, cudaStreamNonBlocking) != cudaSuccess)
        return MGR_ECUDA;
      p->pipe_ev.assign(mgr::kPipeEvents, nullptr);
      for (auto& e : p->pipe_ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return MGR_ECUDA;
    }
    if (op == OP_REC && !ensure_fork(p)) return MGR_ECUDA;
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return MGR_ECUDA;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const mgr::PipeCtx pc{p->pipe_h2d, p->pipe_d2h, p->pipe_ev.data()};
      cudaError_t e2 =
          op == OP_DEC ? mgr::enqueue_decompose_host_pipe(p, host_in, host_out, dev_in, dev_out, ws, cs, pc)
                       : mgr::enqueue_recompose_host_pipe(p, host_in, host_out, dev_in, dev_out, ws, cs, pc,
                                                          mgr::ForkCtx{p->side, p->fork_ev.data(), p->side2});
      e = cudaStreamEndCapture(cs, &graph);
      if (e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return MGR_ECUDA;
    }
    if (p->graphs.size() >= 8) {
      cudaGraphExecDestroy(p->graphs.front().exec);
      p->graphs.erase(p->graphs.begin());
    }
    mgr_plan::GraphEntry ge{key, host_in, host_out, ws, 0.0, nullptr, exec};
    ge.din = dev_in;
    ge.dout = dev_out;
    p->graphs.push_back(ge);
  }
  if (cudaGraphLaunch(exec, st) != cudaSuccess) return MGR_ECUDA;
  return mgr::debug_after(st);
}

int run_host(const mgr_plan* p, int op, const void* host_in, void* host_out, void* dev_in, void* dev_out, void* ws,
             cudaStream_t st) {
  if (!p || !host_in || !host_out || !dev_in || !dev_out) return MGR_EINVAL;
  const size_t bytes = size_t(p->count) * p->elem;
  if ((op == OP_DEC || op == OP_REC) && !ranges_overlap(host_in, bytes, host_out, bytes) &&
      mgr::pipe_eligible(p, dev_in, dev_out) && host_pinned(host_in) && host_pinned(host_out)) {
    // an operation that can overlap its copies with its kernels; not while the
    // caller's stream is being captured
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return MGR_ECUDA;
    if (cap == cudaStreamCaptureStatusNone)
      return run_host_pipe(const_cast<mgr_plan*>(p), op, host_in, host_out, dev_in, dev_out, ws, st);
  }
  if (cudaMemcpyAsync(dev_in, host_in, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return MGR_ECUDA;
  int rc = run_op(p, op, dev_in, dev_out, ws, st);
  if (rc != MGR_OK) return rc;
  if (cudaMemcpyAsync(host_out, dev_out, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) return MGR_ECUDA;
  return mgr::debug_after(st);
}

}  // namespace

extern "C" {

const char* mgr_strerror(int code) {
  switch (code) {
    case MGR_OK: return "ok";
    case MGR_EINVAL: return "invalid argument";
    case MGR_ENOMEM: return "out of memory";
    case MGR_EBUDGET: return "request exceeds the memory budget";
    case MGR_ECUDA: return "CUDA error";
    case MGR_EPENDING: return "pending";
    case MGR_ETIMEDOUT: return "timed out";
    case MGR_EDEVICE: return "device-side error reported";
    case MGR_ENOTFOUND: return "not found";
    case MGR_EBUSY: return "queue full";
    default: return "unknown error";
  }
}

const char* mgr_version(void) { return "0.1.0"; }

int mgr_init(int device, size_t mem_budget_bytes, mgr_ctx** ctx) {
  if (!ctx) return MGR_EINVAL;
  *ctx = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) {
    cudaGetLastError();
    return MGR_ECUDA;
  }
  if (device < 0 || device >= n) return MGR_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return MGR_ECUDA;
  mgr_ctx* c = new (std::nothrow) mgr_ctx();
  if (!c) return MGR_ENOMEM;
  c->device = device;
  c->budget = mem_budget_bytes;
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
  c->num_sms = v;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  c->smem_optin = size_t(v);
  *ctx = c;
  return MGR_OK;
}

int mgr_shutdown(mgr_ctx* ctx) {
  if (!ctx) return MGR_EINVAL;
  if (ctx->live_plans.load() != 0) return MGR_EINVAL;
  cudaSetDevice(ctx->device);
  mgr::batch_destroy(ctx);
  cudaDeviceSynchronize();
  delete ctx;
  return MGR_OK;
}

int mgr_batch_submit(mgr_ctx* ctx, const mgr_request* reqs, int n, uint64_t* ticket) {
  try {
    return mgr::batch_submit(ctx, reqs, n, ticket);
  } catch (const std::bad_alloc&) {
    return MGR_ENOMEM;
  }
}

int mgr_batch_poll(mgr_ctx* ctx, uint64_t ticket, int64_t timeout_us, int* n_done) {
  return mgr::batch_poll(ctx, ticket, timeout_us, n_done);
}

int mgr_batch_tuning(mgr_ctx* ctx, char* buf, size_t len) {
  if (!ctx) return MGR_EINVAL;
  return mgr::batch_tuning(ctx, buf, len);
}

int mgr_max_levels(const mgr_desc* desc, int* levels) {
  if (!levels) return MGR_EINVAL;
  return mgr::resolve_levels(desc, nullptr, levels, nullptr);
}

int mgr_default_levels(const mgr_desc* desc, int* levels) {
  if (!levels) return MGR_EINVAL;
  return mgr::resolve_levels(desc, nullptr, nullptr, levels);
}

int mgr_plan_tables_host(const mgr_desc* desc, int level, int axis, int* n, int* m, double* wa, double* wb,
                         double* k, double* ta, double* tb, int cap) {
  if (!desc || !n || !m) return MGR_EINVAL;
  int L = 0;
  int rc = mgr::resolve_levels(desc, &L, nullptr, nullptr);
  if (rc != MGR_OK) return rc;
  if (level < 1 || level > L || axis < 0 || axis >= desc->ndim) return MGR_EINVAL;
  mgr_plan p;
  p.desc = *desc;
  for (int a = desc->ndim; a < 4; ++a) {
    p.desc.shape[a] = 0;
    p.desc.coords[a] = nullptr;
  }
  p.levels = L;
  try {
    rc = mgr::build_plan_tables(&p);
  } catch (const std::bad_alloc&) {
    return MGR_ENOMEM;
  }
  if (rc != MGR_OK) return rc;
  // desc axis -> internal axis: 4D puts time apart; fewer than three spatial
  // dimensions are the fastest internal axes
  const bool st = desc->ndim == 4;
  const int lead = mgr::kAxes - (st ? 3 : desc->ndim);
  const mgr::AxisLevel& ax = (st && axis == 0) ? p.geom[level].tax : p.geom[level].ax[(st ? axis - 1 : axis) + lead];
  *n = ax.n;
  *m = ax.m;
  if (!wa && !wb && !k && !ta && !tb) return MGR_OK;
  if (cap < std::max(ax.n, 5 * ax.m)) return MGR_EINVAL;
  const double* T = p.tables.host.data();
  if (wa) std::copy(T + ax.o_wa, T + ax.o_wa + ax.n, wa);
  if (wb) std::copy(T + ax.o_wb, T + ax.o_wb + ax.n, wb);
  if (k) std::copy(T + ax.o_k, T + ax.o_k + 5 * ax.m, k);
  if (ta) std::copy(T + ax.o_ta, T + ax.o_ta + ax.m, ta);
  if (tb) std::copy(T + ax.o_tb, T + ax.o_tb + ax.m, tb);
  return MGR_OK;
}

int mgr_plan_create(mgr_ctx* ctx, const mgr_desc* desc, mgr_plan** plan) {
  if (!ctx || !desc || !plan) return MGR_EINVAL;
  *plan = nullptr;
  if (desc->dtype != MGR_F32 && desc->dtype != MGR_F64) return MGR_EINVAL;
  if (desc->prec != MGR_PREC_NATIVE && desc->prec != MGR_PREC_MIXED) return MGR_EINVAL;
  if (desc->prec == MGR_PREC_MIXED && desc->dtype != MGR_F32) return MGR_EINVAL;
  int L = 0;
  int rc = mgr::resolve_levels(desc, &L, nullptr, nullptr);
  if (rc != MGR_OK) return rc;
  mgr_plan* p = new (std::nothrow) mgr_plan();
  if (!p) return MGR_ENOMEM;
  p->ctx = ctx;
  p->desc = *desc;
  for (int k = desc->ndim; k < 4; ++k) {
    p->desc.shape[k] = 0;
    p->desc.coords[k] = nullptr;
  }
  p->levels = L;
  p->form = desc->dtype == MGR_F64 ? mgr::kFormF64 : (desc->prec == MGR_PREC_MIXED ? mgr::kFormMixed : mgr::kFormF32);
  p->elem = desc->dtype == MGR_F64 ? 8 : 4;
  p->welem = (p->form == mgr::kFormF32) ? 4 : 8;
  p->count = 1;
  for (int k = 0; k < desc->ndim; ++k) p->count *= desc->shape[k];
  try {
    rc = mgr::build_plan_tables(p);
  } catch (const std::bad_alloc&) {
    rc = MGR_ENOMEM;
  }
  // the coordinate pointers are not kept: the tables hold everything needed
  for (int k = 0; k < 4; ++k) p->desc.coords[k] = nullptr;
  if (rc != MGR_OK) {
    delete p;
    return rc;
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    delete p;
    return MGR_ECUDA;
  }
  const size_t nt = std::max<size_t>(p->tables.host.size(), 4);
  std::vector<float> f32(nt, 0.0f);
  for (size_t i = 0; i < p->tables.host.size(); ++i) f32[i] = float(p->tables.host[i]);
  std::vector<double> f64(nt, 0.0);
  std::copy(p->tables.host.begin(), p->tables.host.end(), f64.begin());
  if (cudaMalloc(&p->tables.d64, nt * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&p->tables.d32, nt * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p->tables.d64);
    cudaFree(p->tables.d32);
    delete p;
    return MGR_ENOMEM;
  }
  if (cudaMemcpy(p->tables.d64, f64.data(), nt * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->tables.d32, f32.data(), nt * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(p->tables.d64);
    cudaFree(p->tables.d32);
    delete p;
    return MGR_ECUDA;
  }
  if (L >= 1) {
    p->ws_a = align_up(size_t(p->geom[L].coarse_count()) * p->welem);
    p->ws_b = L >= 2 ? align_up(size_t(p->geom[L - 1].coarse_count()) * p->welem) : 0;
    // one load-vector buffer per level, so a recomposition can compute every
    // level's load vector ahead of its solves
    p->f_off.assign(L + 1, 0);
    size_t off = 0;
    for (int l = L; l >= 1; --l) {
      p->f_off[l] = off;
      off += align_up(size_t(p->geom[l].coarse_count()) * p->welem);
    }
    p->ws_f = off;
  }
  if (L >= 1 && desc->ndim == 4)
    p->ws_g = align_up(size_t(p->geom[L].tax.n) * size_t(p->geom[L].space_coarse()) * p->welem);
  p->ws_bytes = p->ws_a + p->ws_b + p->ws_f + p->ws_g;
  ctx->live_plans.fetch_add(1);
  *plan = p;
  return MGR_OK;
}

int mgr_plan_destroy(mgr_plan* p) {
  if (!p) return MGR_EINVAL;
  cudaSetDevice(p->ctx->device);
  {
    std::lock_guard<std::mutex> lk(p->graph_mu);
    for (auto& g : p->graphs) cudaGraphExecDestroy(g.exec);
    p->graphs.clear();
    for (cudaEvent_t e : p->fork_ev) cudaEventDestroy(e);
    if (p->side) cudaStreamDestroy(p->side);
    if (p->side2) cudaStreamDestroy(p->side2);
    for (cudaEvent_t e : p->pipe_ev) cudaEventDestroy(e);
    if (p->pipe_h2d) cudaStreamDestroy(p->pipe_h2d);
    if (p->pipe_d2h) cudaStreamDestroy(p->pipe_d2h);
  }
  cudaFree(p->tables.d64);
  cudaFree(p->tables.d32);
  p->ctx->live_plans.fetch_sub(1);
  delete p;
  return MGR_OK;
}

int mgr_plan_levels(const mgr_plan* p, int* levels) {
  if (!p || !levels) return MGR_EINVAL;
  *levels = p->levels;
  return MGR_OK;
}

int mgr_workspace_size(const mgr_plan* p, size_t* bytes) {
  if (!p || !bytes) return MGR_EINVAL;
  *bytes = p->ws_bytes;
  return MGR_OK;
}

int mgr_decompose(const mgr_plan* p, const void* in, void* out, void* ws, mgr_stream_t stream) {
  return run_op(p, OP_DEC, in, out, ws, reinterpret_cast<cudaStream_t>(stream));
}

int mgr_recompose(const mgr_plan* p, const void* in, void* out, void* ws, mgr_stream_t stream) {
  return run_op(p, OP_REC, in, out, ws, reinterpret_cast<cudaStream_t>(stream));
}

int mgr_decompose_packed(const mgr_plan* p, const void* in, void* out, void* ws, mgr_stream_t stream) {
  return run_op(p, OP_DEC_PACKED, in, out, ws, reinterpret_cast<cudaStream_t>(stream));
}

int mgr_recompose_packed(const mgr_plan* p, const void* in, int nclasses, void* out, void* ws,
                         mgr_stream_t stream) {
  if (!p || nclasses < 1 || nclasses > p->levels + 1) return MGR_EINVAL;
  return run_op(p, OP_REC_PACKED | (nclasses << 8), in, out, ws, reinterpret_cast<cudaStream_t>(stream));
}

int mgr_quant_bins(const mgr_plan* p, double tau, double* bins, int cap) {
  if (!p || (cap > 0 && !bins) || p->desc.ndim == 4) return MGR_EINVAL;
  std::vector<double> b;
  int rc;
  try {
    rc = mgr::quant_bins(const_cast<mgr_plan*>(p), tau, b);
  } catch (const std::bad_alloc&) {
    return MGR_ENOMEM;
  }
  if (rc != MGR_OK) return rc;
  for (int i = 0; i < std::min(cap, int(b.size())); ++i) bins[i] = b[i];
  return MGR_OK;
}

int mgr_decompose_quantized(const mgr_plan* p, const void* in, int32_t* codes, double tau, void* ws,
                            unsigned long long* saturated, mgr_stream_t stream) {
  Extra x;
  x.tau = tau;
  x.sat = saturated;
  return run_op(p, OP_DEC_QUANT, in, codes, ws, reinterpret_cast<cudaStream_t>(stream), x);
}

int mgr_recompose_dequantized(const mgr_plan* p, const int32_t* codes, int nclasses, double tau, void* out, void* ws,
                              mgr_stream_t stream) {
  if (!p || nclasses < 1 || nclasses > p->levels + 1) return MGR_EINVAL;
  Extra x;
  x.tau = tau;
  return run_op(p, OP_REC_DEQ | (nclasses << 8), codes, out, ws, reinterpret_cast<cudaStream_t>(stream), x);
}

int mgr_decompose_host(const mgr_plan* p, const void* host_in, void* host_out, void* dev_in, void* dev_out, void* ws,
                       mgr_stream_t stream) {
  return run_host(p, OP_DEC, host_in, host_out, dev_in, dev_out, ws, reinterpret_cast<cudaStream_t>(stream));
}

int mgr_recompose_host(const mgr_plan* p, const void* host_in, void* host_out, void* dev_in, void* dev_out, void* ws,
                       mgr_stream_t stream) {
  return run_host(p, OP_REC, host_in, host_out, dev_in, dev_out, ws, reinterpret_cast<cudaStream_t>(stream));
}

int mgr_profile(const mgr_plan* p, int op, const void* in, void* out, void* ws, mgr_stream_t stream,
                mgr_kernel_time* times, int cap, int* n) {
  if (!n || (cap > 0 && !times) || op < OP_DEC || op > OP_REC_PACKED || !p) return MGR_EINVAL;
  if (p->desc.ndim == 4 && packed_op(op)) return MGR_EINVAL;
  if (op == OP_REC_PACKED) op |= (p->levels + 1) << 8;
  int rc = check_op_args(p, in, out, ws, !packed_op(op));
  if (rc != MGR_OK) return rc;
  if ((rc = check_sticky()) != MGR_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  mgr::Recorder rec;
  mgr::t_recorder = &rec;
  cudaError_t e = enqueue(p, op, in, out, ws, st);
  mgr::t_recorder = nullptr;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  *n = int(rec.launches.size());
  for (size_t i = 0; i < rec.launches.size(); ++i) {
    mgr::LaunchRecord& r = rec.launches[i];
    float ms = 0.f;
    if (e == cudaSuccess && r.stop) cudaEventElapsedTime(&ms, r.start, r.stop);
    if (int(i) < cap) {
      std::memcpy(times[i].name, r.name, sizeof(times[i].name));
      times[i].level = r.level;
      times[i].ms = ms;
      times[i].bytes = r.bytes;
      times[i].flops = r.flops;
    }
    cudaEventDestroy(r.start);
    if (r.stop) cudaEventDestroy(r.stop);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return MGR_ECUDA;
  }
  return mgr::debug_after(st);
}

int mgr_debug_bounds(void) {
#ifdef MGR_DEBUG_BOUNDS
  return 1;
#else
  return 0;
#endif
}

int mgr_debug_last(int* code, int64_t* index, int64_t* extent) {
  std::lock_guard<std::mutex> lk(mgr::g_dbg_mu);
  if (!mgr::g_dbg_have) return MGR_ENOTFOUND;
  if (code) *code = mgr::g_dbg_last.code;
  if (index) *index = mgr::g_dbg_last.index;
  if (extent) *extent = mgr::g_dbg_last.extent;
  return MGR_OK;
}

}  // extern "C"
