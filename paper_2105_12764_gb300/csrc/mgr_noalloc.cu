// mgr_noalloc.cu -- decomposition that allocates no device memory.
//
// mgr_decompose needs a caller-provided workspace.  Some callers cannot
// obtain one: code whose device memory is entirely owned by another
// allocator (a framework's caching pool that has reserved the device),
// plug-ins that are handed only their input and output buffers, or
// latency-critical paths where an allocation (which may synchronise the
// device) is not acceptable.  For them, mgr_decompose_noalloc runs the same
// level loop with its workspace in a fixed area that is part of this
// library's device image.
//
// The area is a file-scope __device__ array of kNoallocScratchBytes; every
// GPU that loads the library holds it until the process exits.  Host code
// cannot use the array's name as a device address (it names a host-side
// stand-in), so its device address is looked up once per device, with that
// device current, by cudaGetSymbolAddress, and passed to the kernels.
#include <cuda_runtime.h>

#include <mutex>

#include "mgr_internal.h"

namespace {

constexpr size_t kNoallocScratchBytes = size_t(MGR_NOALLOC_SCRATCH_BYTES);

// Workspace of mgr_decompose_noalloc (coarse-grid buffers and load vector).
// Its contents persist between calls; the decomposition writes every byte it
// later reads, so nothing has to start at zero.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on `device`, looked up on first use
// (with `device` current: the caller checked that it is).  A first use while
// `stream` is being captured is refused: the lookup may load the library's
// device image, which a capture does not allow.
int scratch_address(int device, cudaStream_t stream, void** out) {
  if (device < 0 || device >= kMaxDevices) return MGR_EINVAL;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[device]) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) {
      cudaGetLastError();
      return MGR_ECUDA;
    }
    if (cap != cudaStreamCaptureStatusNone) return MGR_EINVAL;
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return MGR_ECUDA;
    }
    g_scratch_ptr[device] = p;
  }
  *out = g_scratch_ptr[device];
  return MGR_OK;
}

bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + nb && pb < pa + na;
}

}  // namespace

extern "C" int mgr_decompose_noalloc(const mgr_plan* plan, const void* in, void* out, mgr_stream_t stream) {
  if (!plan || !in || !out) return MGR_EINVAL;
  if (plan->ws_bytes > kNoallocScratchBytes) return MGR_EINVAL;  // field too large for the scratch area
  const size_t bytes = size_t(plan->count) * plan->elem;
  if ((reinterpret_cast<uintptr_t>(in) % plan->elem) || (reinterpret_cast<uintptr_t>(out) % plan->elem))
    return MGR_EINVAL;
  // in place only where mgr_decompose allows it: never for 4D plans, whose
  // time passes read neighbouring slices after their coefficients are written
  const bool alias_ok = plan->desc.ndim != 4;
  if ((in != out || !alias_ok) && overlap(in, bytes, out, bytes)) return MGR_EINVAL;
  // the kernels run on the current device and use that device's copy of the
  // scratch array: it must be the plan's device
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return MGR_ECUDA;
  }
  if (cur != plan->ctx->device) return MGR_EINVAL;
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  void* ws = nullptr;
  const int rc = scratch_address(cur, st, &ws);
  if (rc != MGR_OK) return rc;
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return MGR_ECUDA;
  }
  const cudaError_t e = mgr::enqueue_decompose(plan, in, out, ws, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return MGR_ECUDA;
  }
  return mgr::debug_after(st);
}
