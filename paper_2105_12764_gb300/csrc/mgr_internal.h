// mgr_internal.h -- internal types of the GB300 multigrid refactoring library.
//
// Axes are always handled as three: axis 0 (slowest) .. axis 2 (fastest).  A
// field with ndim < 3 is embedded with leading axes of length 1 that never
// coarsen ("inactive").  A 4D (spatiotemporal) field has one more axis, time,
// slower than the three spatial ones; it is kept apart (LevelGeom::tax) so the
// spatial kernels see every time slice as a 3D field.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstddef>
#include <cstdint>
#include <mutex>
#include <vector>

#include "mgr.h"

namespace mgr {

constexpr int kAxes = 3;
constexpr int kMaxLevels = 60;

// Element type combination of one plan ("form").
enum Form : int {
  kFormF64 = 0,    // FP64 field, every step in FP64
  kFormF32 = 1,    // FP32 field, every step in FP32
  kFormMixed = 2,  // FP32 field, FP32 stencils, FP64 solves/accumulation/coarse workspace
};

// One axis at one level.  Level-l node i of this axis sits at full-grid index
// min(i * s, N - 1) (the keep-last nesting of the hierarchy).
struct AxisLevel {
  int n = 1;            // nodes on this axis at level l
  int m = 1;            // nodes at level l-1
  int64_t s = 1;        // full-grid stride 2^(L-l)
  int64_t N = 1;        // full-grid length of the axis
  bool active = false;  // coarsens at this level (n >= 3)
  // element offsets into the plan's weight tables
  int64_t o_wa = 0, o_wb = 0;  // interpolation weights, indexed by fine node (n entries)
  int64_t o_k = 0;             // 5 * m mass-transfer taps, row q at offsets -2..2 around node min(2q, n-1),
                               // each row scaled by 1/u_q of the coarse mass matrix's LU factors
  int64_t o_ta = 0, o_tb = 0;  // scaled Thomas recurrences, m entries each
};

struct LevelGeom {
  AxisLevel ax[kAxes];
  AxisLevel tax;  // time axis of a 4D field (inactive, n = m = 1, otherwise)
  int64_t space_fine() const { return (int64_t)ax[0].n * ax[1].n * ax[2].n; }
  int64_t space_coarse() const { return (int64_t)ax[0].m * ax[1].m * ax[2].m; }
  int64_t fine_count() const { return space_fine() * tax.n; }
  int64_t coarse_count() const { return space_coarse() * tax.m; }
};

// Host-side FP64 tables of a plan (built from the coordinates) and their
// device copies in FP64 and FP32.
struct Tables {
  std::vector<double> host;
  double* d64 = nullptr;
  float* d32 = nullptr;
};

}  // namespace mgr

struct mgr_ctx {
  int device = 0;
  size_t budget = 0;
  int num_sms = 0;
  size_t smem_optin = 0;
  std::atomic<int> live_plans{0};
  void* batch = nullptr;  // batch / serving state (mgr_batch.cu)
};

struct mgr_plan {
  mgr_ctx* ctx = nullptr;
  mgr_desc desc{};
  int form = 0;
  int levels = 0;                     // L
  int64_t full[mgr::kAxes] = {1, 1, 1};
  int64_t full_t = 1;                 // time axis length (4D fields), else 1
  int64_t count = 0;                  // prod(shape)
  size_t elem = 0;                    // bytes per field element
  size_t welem = 0;                   // bytes per workspace element
  std::vector<mgr::LevelGeom> geom;   // geom[l] for l = 1..L (geom[0] unused)
  int64_t coarsest[mgr::kAxes] = {1, 1, 1};
  int64_t coarsest_t = 1;
  // class-packed layout: class c (0 = coarsest grid, l = coefficients of level
  // l) starts at class_off[c]; class_off[L+1] = count
  std::vector<int64_t> class_off;
  // quantization: |Z_l|_inf of each level's correction operator (built on
  // first use, under quant_mu)
  std::mutex quant_mu;
  std::vector<double> znorm;
  mgr::Tables tables;
  // workspace layout (bytes)
  size_t ws_a = 0, ws_b = 0, ws_f = 0, ws_g = 0, ws_bytes = 0;  // ws_g: 4D time-slice load vectors
  std::vector<size_t> f_off;  // byte offset of level l's load vector in the F region (l = 1..L)
  // side stream and events of the forked recomposition graph (created on the
  // first capture, under graph_mu)
  cudaStream_t side = nullptr, side2 = nullptr;
  std::vector<cudaEvent_t> fork_ev;
  // copy streams and events of the pipelined host-buffer decomposition
  // (created on its first capture, under graph_mu)
  cudaStream_t pipe_h2d = nullptr, pipe_d2h = nullptr;
  std::vector<cudaEvent_t> pipe_ev;
  // launch-sequence cache: one CUDA graph per (op, in, out, workspace)
  std::mutex graph_mu;
  struct GraphEntry {
    int op;
    const void* in;
    void* out;
    void* ws;
    double tau;   // quantized operations: tolerance
    void* aux;    // quantized decomposition: saturation counter
    cudaGraphExec_t exec;
    const void* din = nullptr;  // host-buffer operations: the device buffers
    void* dout = nullptr;
  };
  std::vector<GraphEntry> graphs;
};

namespace mgr {

// Per-launch instrumentation used by mgr_profile (events around every launch).
struct LaunchRecord {
  cudaEvent_t start = nullptr, stop = nullptr;
  char name[32] = {0};
  int level = 0;
  double bytes = 0, flops = 0;
};
struct Recorder {
  std::vector<LaunchRecord> launches;
};
extern thread_local Recorder* t_recorder;

// Algorithmic work of one launch: compulsory bytes and floating-point
// operations (fused multiply-add = 2) of the arithmetic the kernel must do.
struct Work {
  double bytes = 0, flops = 0;
};
Work work_level_load(const mgr_plan* p, int l, bool decompose);
Work work_solve(const mgr_plan* p, int l, int axis, bool final_op);
Work work_interp(const mgr_plan* p, int l);

// NVTX range over host-side enqueue work: one per operation and one per
// level, so a profiler's timeline groups the launches of each level.  A CUDA
// graph replay runs no host code, so its launches fall under the ranges of
// the capture that built the graph.  Costs a few nanoseconds when no
// profiler is attached.
struct NvtxRange {
  explicit NvtxRange(const char* fmt, ...) {
    char buf[64];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    nvtxRangePushA(buf);
  }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Device-side record of the first out-of-bounds index a bounds-checking build
// (MGR_DEBUG_BOUNDS) met, one per translation unit with kernels; codes name
// the access (kDbg* below).
struct DebugRecord {
  unsigned long long count;
  int code;
  int pad;
  long long index;
  long long extent;
};
enum : int {
  kDbgLevelIn = 1, kDbgLevelY = 2, kDbgLevelW = 3, kDbgLevelF = 4, kDbgLevelStage = 5, kDbgLevelTile = 6,
  kDbgInterpC = 11, kDbgInterpW = 12, kDbgInterpOut = 13, kDbgInterpStage = 14,
  kDbgSolveF = 21, kDbgSolveW = 22, kDbgSolveSmem = 23,
  kDbgSmallIn = 31, kDbgSmallOut = 32, kDbgCoarsestY = 41, kDbgCoarsestW = 42,
};
// Read and clear the records of every translation unit (bounds-checking
// builds; others report nothing): returns the number of violations since the
// last call and the first one of them in *first.
unsigned long long debug_take(DebugRecord* first);
unsigned long long debug_take_core(DebugRecord* first);
unsigned long long debug_take_batch(DebugRecord* first);
unsigned long long debug_take_st(DebugRecord* first);
// After an operation is enqueued on `st`: bounds-checking builds wait for it
// (unless `st` is being captured) and return MGR_EDEVICE for a recorded
// out-of-bounds access (kept for mgr_debug_last); other builds return MGR_OK.
int debug_after(cudaStream_t st);
extern std::mutex g_dbg_mu;
extern DebugRecord g_dbg_last;
extern bool g_dbg_have;

// Host-side fault injection for tests (no GPU fault is involved): true when
// the comma-separated list in the environment variable MGR_FAULT_INJECT
// names `what` ("alloc": device allocations of the batch / serving layers
// fail; "launch": operations fail before any kernel is launched; "admit":
// serving admission refuses requests).  Read on every call.
bool fault_injected(const char* what);

// Raise the dynamic shared-memory limit of kernel `fn` on the current device
// to at least `bytes`.  The limit only ever grows: a launch captured into a
// graph (or issued from another thread) with a larger request than the
// current one is never left above a lowered limit.  Requests that fit, with
// the kernel's static shared memory, in the 48 KB every kernel may use
// without the attribute need no call.
cudaError_t raise_smem_limit(const void* fn, size_t bytes);
template <typename F>
inline cudaError_t raise_smem_limit(F* fn, size_t bytes) {
  return raise_smem_limit(reinterpret_cast<const void*>(fn), bytes);
}

// mgr_plan.cpp
int build_plan_tables(mgr_plan* p);
int resolve_levels(const mgr_desc* d, int* levels, int* max_levels, int* default_levels);

// mgr_batch.cu: batched refactoring (context-owned state in mgr_ctx::batch).
int batch_submit(mgr_ctx* ctx, const mgr_request* reqs, int n, uint64_t* ticket);
int batch_poll(mgr_ctx* ctx, uint64_t ticket, int64_t timeout_us, int* n_done);
int batch_tuning(mgr_ctx* ctx, char* buf, size_t len);
void batch_destroy(mgr_ctx* ctx);

// mgr_core.cu: enqueue one whole operation (all levels) on `st` (no graph).
cudaError_t enqueue_decompose(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st);
cudaError_t enqueue_recompose(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st);
// mgr_st.cu: the 4D (spatiotemporal) form of the two operations
cudaError_t enqueue_decompose_st(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st);
cudaError_t enqueue_recompose_st(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st);
// A recomposition captured into a graph may run the load-vector passes of all
// levels on `side`, concurrently with the solve / interpolation chain (they
// depend only on the coefficients); ev: L + 1 events.
struct ForkCtx {
  cudaStream_t side;
  cudaEvent_t* ev;
  cudaStream_t side2;  // the finest level's pass (may be null: everything on side)
};
cudaError_t enqueue_recompose_fork(const mgr_plan* p, int op, const void* in, int ncls, const double* bins, void* out,
                                   void* ws, cudaStream_t st, const ForkCtx& fk);
// Decomposition with pinned host buffers, pipelined (graph capture only): the
// input planes go to the device in slabs on `h2d`; the finest level pass runs
// in parts, each as soon as its planes are there; the planes a part finishes
// that are fine in z (they hold only finest-level coefficients, final once the
// part is done) go back on `d2h` while the coarser levels run; the other
// planes follow at the end.  ev: kPipeEvents events.
constexpr int kPipeParts = 8;
constexpr int kPipeEvents = 2 * kPipeParts + 3;
struct PipeCtx {
  cudaStream_t h2d, d2h;
  cudaEvent_t* ev;
};
// whether a decomposition from host_in into host_out through dev_in / dev_out
// can run pipelined (3D nodal plan with a tiled finest level, distinct device
// buffers, enough planes)
bool pipe_eligible(const mgr_plan* p, const void* dev_in, const void* dev_out);
cudaError_t enqueue_decompose_host_pipe(const mgr_plan* p, const void* host_in, void* host_out, const void* dev_in,
                                        void* dev_out, void* ws, cudaStream_t st, const PipeCtx& pc);
// The recomposition likewise: the coefficients of the coarser levels (the
// even planes) first, the odd planes in slabs that release parts of the
// finest load-vector pass (run on fk.side), and the output planes copied back
// as the parts of the finest interpolation finish.
cudaError_t enqueue_recompose_host_pipe(const mgr_plan* p, const void* host_in, void* host_out, const void* dev_in,
                                        void* dev_out, void* ws, cudaStream_t st, const PipeCtx& pc,
                                        const ForkCtx& fk);
// class-packed output / input (recompose from classes 0..ncls-1)
cudaError_t enqueue_decompose_packed(const mgr_plan* p, const void* in, void* out, void* ws, cudaStream_t st);
cudaError_t enqueue_recompose_packed(const mgr_plan* p, const void* in, int ncls, void* out, void* ws,
                                     cudaStream_t st);
// quantized class-packed forms: int32 codes with bin widths bins[0..L]
cudaError_t enqueue_decompose_quantized(const mgr_plan* p, const void* in, int* codes, const double* bins,
                                        unsigned long long* sat, void* ws, cudaStream_t st);
cudaError_t enqueue_recompose_dequantized(const mgr_plan* p, const int* codes, int ncls, const double* bins,
                                          void* out, void* ws, cudaStream_t st);
// mgr_plan.cpp: bin widths for the max-norm tolerance tau (L+1 entries)
int quant_bins(mgr_plan* p, double tau, std::vector<double>& bins);
// mgr_classes.cu: layout conversion nodal <-> class-packed
cudaError_t enqueue_pack_classes(const mgr_plan* p, const void* nodal, void* packed, cudaStream_t st);
cudaError_t enqueue_unpack_classes(const mgr_plan* p, const void* packed, int ncls, void* nodal, cudaStream_t st);

}  // namespace mgr
