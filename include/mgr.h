/*
 * mgr.h -- C ABI of the GB300 (sm_103a) multigrid hierarchical data
 * refactoring library: decomposition of a structured-grid field into
 * hierarchical coefficients and its inverse recomposition
 * (arXiv 2105.12764, Sec. II.A, Eq. (1) and Eq. (2)).
 *
 * Conventions shared by every entry point
 *   - Every function returns int: MGR_OK (0) on success, a negative MGR_E*
 *     code otherwise; mgr_strerror() names it.  No C++ exception crosses the
 *     ABI.  A failing call leaves caller-owned buffers untouched unless it
 *     says otherwise.
 *   - Pointers named `in`, `out`, `workspace` are DEVICE pointers on the
 *     context's device (cudaMalloc, torch, ...), owned by the caller.  Pointers
 *     in mgr_desc.coords are HOST pointers, copied at plan creation.
 *   - Arrays are row-major: shape[ndim-1] is the fastest (contiguous) axis.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     enqueued on it and the call returns without waiting, unless stated.
 *
 * Output layout ("nodal"): decomposition output has the input's shape.  The
 * node sets of the hierarchy are nested, N_0 c N_1 c ... c N_L (all nodes);
 * every node of N_l \ N_{l-1} holds its level-l coefficient
 * (I - Pi_{l-1}) Q_l u (Sec. II.A.1), and the nodes of N_0 hold the coarsest
 * nodal values Q_0 u.  Per dimension, the level-(l-1) node list keeps every
 * other node of the level-l list starting with the first one, plus the last
 * node if it was skipped; for n = 2^k+1 this is the paper's dyadic hierarchy.
 */
#ifndef MGR_H
#define MGR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */
#define MGR_OK 0
#define MGR_EINVAL (-1)    /* invalid argument (shape, levels, alias, NULL, ...)   */
#define MGR_ENOMEM (-2)    /* host or device allocation failed                     */
#define MGR_EBUDGET (-3)   /* request can never fit the context's memory budget    */
#define MGR_ECUDA (-4)     /* a CUDA runtime call failed (sticky errors included)  */
#define MGR_EPENDING (-5)  /* poll: work not finished yet                          */
#define MGR_ETIMEDOUT (-6) /* poll/wait: the timeout expired                       */
#define MGR_EDEVICE (-7)   /* reserved for device-reported errors; not returned now  */
#define MGR_ENOTFOUND (-8) /* unknown ticket / resident handle                     */
#define MGR_EBUSY (-9)     /* queue full: retry after polling                      */

typedef struct CUstream_st* mgr_stream_t; /* same type as cudaStream_t */

typedef enum { MGR_F32 = 0, MGR_F64 = 1 } mgr_dtype;

typedef enum {
  /* every step in the field's dtype */
  MGR_PREC_NATIVE = 0,
  /* the precision pattern: coefficients and mass-transfer stencils in FP32,
     tridiagonal solves, correction accumulation and the coarse-grid
     workspace in FP64.  Requires dtype MGR_F32. */
  MGR_PREC_MIXED = 1
} mgr_precision;

/* Problem description (Sec. II.A: a d-dimensional field on a rectilinear
   grid; Sec. IV.A: FP32 or FP64 nodal values).  ndim = 4 is the
   spatiotemporal (3+1)-D form of Sec. III.E: shape[0] is time, decomposed
   with the other three axes as one more tensor-product dimension.  4D plans
   run mgr_decompose / mgr_recompose (and their _host and _noalloc forms and
   the serving layer) out of place (in == out is MGR_EINVAL) in the nodal
   layout; the class-packed, quantized and batched forms are 1D-3D only. */
typedef struct {
  int ndim;                /* 1..4                                                   */
  int64_t shape[4];        /* shape[0..ndim-1], each >= 2 and <= 2^30; shape[ndim-1]
                              fastest; shape[ndim-2] * shape[ndim-1] < 2^31 (and, for
                              4D, shape[1] * shape[2] * shape[3] < 2^31)              */
  const double* coords[4]; /* HOST, strictly increasing, length shape[k]; NULL means
                              uniform unit spacing x_i = i.  Copied at plan time;
                              spacings are formed in FP64 on the host.               */
  int levels;              /* -1: default depth (smallest dimension reaches 3 nodes);
                              0..mgr_max_levels(): explicit depth                    */
  mgr_dtype dtype;
  mgr_precision prec;
} mgr_desc;

typedef struct mgr_ctx mgr_ctx;
typedef struct mgr_plan mgr_plan;

const char* mgr_strerror(int code);

/* Library version, "major.minor.patch". */
const char* mgr_version(void);

/* Create a context on CUDA device `device` (made current on this thread).
   mem_budget_bytes caps the device memory the context's batch / serving
   layer may hold (0 = no cap).  Owns the streams, graphs, autotune cache and
   resident pool.  *ctx is NULL on failure. */
int mgr_init(int device, size_t mem_budget_bytes, mgr_ctx** ctx);
/* Synchronises the context's streams and frees everything it owns.  Plans
   created from it must be destroyed first. */
int mgr_shutdown(mgr_ctx* ctx);

/* Deepest explicit depth (smallest dimension reaches 2 nodes) and the default
   depth (smallest dimension reaches 3 nodes) for a description. */
int mgr_max_levels(const mgr_desc* desc, int* levels);
int mgr_default_levels(const mgr_desc* desc, int* levels);

/* The FP64 tables a plan for `desc` would hold for one axis at one level,
   built on the host only (no context, no device, nothing allocated on a GPU):
   the inspection point of the operators of Sec. II.A / III.A.
     level     1..L of the resolved depth (desc->levels = -1: the default)
     axis      0..ndim-1 in the order of desc->shape (ndim-1 fastest; axis 0
               of a 4D field is time)
     n, m      out: nodes of this axis at level `level` and at level-1
     wa, wb    n entries: interpolation weights of each fine node on its left
               and right coarse neighbours (Sec. II.A.1); 0 at coarse nodes
     k         5*m entries: row q holds the mass-transfer taps K = P^T M
               (Sec. III.A.2) at fine nodes min(2q, n-1)-2 .. +2, scaled by
               1/u_q, u_q the pivots of the coarse mass matrix's LU factors
               (Sec. III.A.3); taps outside 0..n-1 are 0
     ta, tb    m entries: the scaled Thomas recurrences, forward
               y_q = f'_q - ta_q y_{q-1}, backward z_q = y_q - tb_q z_{q+1}
     cap       capacity of each of wa, wb, k, ta, tb in doubles
   With all five arrays NULL only n and m are returned.  MGR_EINVAL for an
   invalid description, level or axis, or when cap < max(n, 5*m) with any
   array given.  An axis that does not coarsen at this level reports
   n = m = 1 and the identity stencil. */
int mgr_plan_tables_host(const mgr_desc* desc, int level, int axis, int* n, int* m, double* wa, double* wb,
                         double* k, double* ta, double* tb, int cap);

/* Build a plan: the hierarchy, every interpolation weight, the mass-transfer
   stencils K = P^T M (Sec. III.A.2, formed as P^T M in FP64 from the
   coordinates) and the factors of the coarse mass matrices for the Thomas
   solves (Sec. III.A.3), uploaded once to the device.  The plan owns these
   device arrays; it holds no field data. */
int mgr_plan_create(mgr_ctx* ctx, const mgr_desc* desc, mgr_plan** plan);
int mgr_plan_destroy(mgr_plan* plan);
/* Depth the plan runs (levels = -1 resolved). */
int mgr_plan_levels(const mgr_plan* plan, int* levels);
/* Bytes of device workspace one mgr_decompose / mgr_recompose call needs
   (coarse-grid buffers: about 0.28 x the field's element count, in the
   solve precision).  May be 0 when levels = 0. */
int mgr_workspace_size(const mgr_plan* plan, size_t* bytes);

/* Decompose (Sec. II.A, finest to coarsest): for l = L..1 compute the level-l
   coefficients (interpolation residuals), the load vector f = (x_k P_k^T M_k) c,
   the correction z from the tensor-product coarse mass matrix by Thomas
   solves along every dimension, and add z to the coarse nodes.
     in        DEVICE, prod(shape) elements of dtype, row-major
     out       DEVICE, same size and type, nodal layout (above); out == in
               (exact alias) is allowed, partial overlap returns MGR_EINVAL
     workspace DEVICE, >= mgr_workspace_size() bytes, 256-byte aligned; its
               contents on entry do not matter
   Asynchronous on `stream`; the buffers must stay valid until the stream
   reaches this point.  Concurrent calls that share a workspace race. */
int mgr_decompose(const mgr_plan* plan, const void* in, void* out, void* workspace, mgr_stream_t stream);

/* Recompose (Sec. II.A, coarsest to finest): the inverse of mgr_decompose.
   For l = 1..L recompute z from the level-l coefficients, subtract it from
   the coarse nodes, and add the interpolant of the coarse nodes to the
   coefficients.  Arguments as for mgr_decompose (in = nodal coefficients,
   out = field). */
int mgr_recompose(const mgr_plan* plan, const void* in, void* out, void* workspace, mgr_stream_t stream);

/* End-to-end forms for callers that hold the field in HOST memory: copy
   host_in to dev_in, run the operation from dev_in into dev_out, and copy
   dev_out back to host_out, all on `stream` (pinned host memory makes the
   copies asynchronous).  dev_in, dev_out: DEVICE, field-sized; they may be
   the same buffer.  Returns after enqueueing; synchronise `stream` before
   reading host_out.  With pinned, non-overlapping host buffers, distinct
   device buffers and a 3D plan of at least 32 planes whose finest level is
   tiled, the copies overlap the kernels (copies by slabs of planes, the
   finest level in parts as its planes arrive, finished planes copied back
   early); the results are the same bits as the plain sequence.  The call
   takes the plan's graph lock like mgr_decompose. */
int mgr_decompose_host(const mgr_plan* plan, const void* host_in, void* host_out, void* dev_in, void* dev_out,
                       void* workspace, mgr_stream_t stream);
int mgr_recompose_host(const mgr_plan* plan, const void* host_in, void* host_out, void* dev_in, void* dev_out,
                       void* workspace, mgr_stream_t stream);

/* ------------------------------------------------ coefficient classes */

/* Class-packed layout (Sec. I: the refactored data are a series of
   hierarchically organised coefficient classes, and an approximation of a
   chosen fidelity is rebuilt from the first few of them).  Class 0 holds the
   coarsest nodal values Q_0 u on N_0; class l (1..L) holds the level-l
   coefficients on N_l \ N_{l-1}.  The classes are stored one after another,
   coarsest first, each in row-major order of its level grid with the nodes
   of N_{l-1} left out, so the first k classes are a prefix of the buffer.
   Total size: prod(shape) elements, like the nodal layout. */

/* offsets[c] = first element of class c for c = 0..L, offsets[L+1] =
   prod(shape); writes min(cap, L+2) entries and sets *nclasses = L+1.
   Host-only (no device work). */
int mgr_class_offsets(const mgr_plan* plan, int64_t* offsets, int cap, int* nclasses);

/* Decompose into the class-packed layout: the same operation as
   mgr_decompose, with the level pass writing each coefficient straight to its
   class position (no extra pass).  out: DEVICE, prod(shape) elements; it must
   not overlap `in` (MGR_EINVAL).  Workspace as for mgr_decompose. */
int mgr_decompose_packed(const mgr_plan* plan, const void* in, void* out, void* workspace, mgr_stream_t stream);

/* Progressive recomposition: rebuild the field from classes 0..nclasses-1 of
   a class-packed decomposition, the dropped classes taken as zero.  The
   result is Q_{nclasses-1} u, interpolated to the full grid; nclasses = L+1
   is the exact inverse of mgr_decompose_packed.  Levels whose class is
   dropped have a zero correction and run as interpolation only.
     in        DEVICE; only its first offsets[nclasses] elements are read
     nclasses  1..L+1 (else MGR_EINVAL)
     out       DEVICE, prod(shape) elements, not overlapping in[0..N)
   Workspace and stream as for mgr_recompose. */
int mgr_recompose_packed(const mgr_plan* plan, const void* in, int nclasses, void* out, void* workspace,
                         mgr_stream_t stream);

/* Layout conversions, one launch each, no workspace.  pack: nodal -> class-
   packed (a permutation).  unpack: classes 0..nclasses-1 of a class-packed
   buffer -> nodal layout, with the nodes of dropped classes set to 0
   (nclasses 1..L+1; only the first offsets[nclasses] elements are read).
   The two buffers must not overlap. */
int mgr_pack_classes(const mgr_plan* plan, const void* nodal, void* packed, mgr_stream_t stream);
int mgr_unpack_classes(const mgr_plan* plan, const void* packed, int nclasses, void* nodal, mgr_stream_t stream);

/* ------------------------------------------------ linear quantization */

/* The quantization stage that follows refactoring in a lossy compressor
   (Sec. V "Lossy compression": refactoring, quantization and entropy coding;
   quantization and dequantization run on the GPU next to the refactoring).
   The paper does not state the quantizer; this library uses uniform bins per
   coefficient class with widths chosen so that the recomposed field is
   within `tau` of the input in the maximum norm:
     q_0 = 2 tau / (L+1),  q_l = 2 tau / ((L+1) (1 + |Z_l|_inf)),
   Z_l the level-l correction operator (x_k M_{l-1,k})^-1 (x_k P_k^T M_k).
   (A perturbation d_l of class l reaches the field through
   e_l = d_l + P_l (e_{l-1} - Z_l d_l) with |P_l|_inf = 1, and rounding to
   the nearest code gives |d_l| <= q_l / 2.)  Codes are int32,
   k = round-half-even(c * (1/q)) with the product and the rounding in the
   stencil precision of the plan (FP64 for MGR_F64, FP32 for the FP32 forms;
   class 0 in the solve precision), in the class-packed layout. */

/* bins[c] = bin width of class c for tolerance tau > 0 (writes min(cap, L+1)
   entries).  Host-only; the first call on a plan evaluates the operator
   norms (O(n_k^2) per axis and level). */
int mgr_quant_bins(const mgr_plan* plan, double tau, double* bins, int cap);

/* Decompose and quantize in the same pass: the level pass writes the int32
   code of each coefficient to its class-packed position (no coefficient
   array is written).
     codes      DEVICE, prod(shape) int32, not overlapping `in`
     tau        max-norm tolerance of the recomposed field, > 0
     saturated  DEVICE counter or NULL: the call adds the number of values
                whose code does not fit in int32 (they are stored as
                +-(2^31-1), and the tolerance no longer holds); zero it first
   Workspace and stream as for mgr_decompose. */
int mgr_decompose_quantized(const mgr_plan* plan, const void* in, int32_t* codes, double tau, void* workspace,
                            unsigned long long* saturated, mgr_stream_t stream);

/* Dequantize and recompose from classes 0..nclasses-1 of quantized codes
   (nclasses = L+1: every class; the error is then at most tau plus
   rounding).  Codes are read and scaled inside the level kernels.  Only the
   first offsets[nclasses] codes are read.  `out`: DEVICE field, not
   overlapping the codes. */
int mgr_recompose_dequantized(const mgr_plan* plan, const int32_t* codes, int nclasses, double tau, void* out,
                              void* workspace, mgr_stream_t stream);

/* ------------------------------------------------------------ no-alloc form */

/* Measured FP64 fused multiply-add throughput of `device`, in FMAs per second:
   the roofline denominator of the plain FP64 form, whose level passes are
   bound by the FP64 pipe rather than by HBM.  Every thread runs eight
   independent FMA chains over four 256-thread CTAs per SM; the best of three
   timed launches (after a warm-up launch, about 10 ms each on a GB300) is
   returned in *fma_per_second (2 flops each).  The paper has no counterpart:
   this is a measurement helper.  Synchronous; allocates and frees a small
   device buffer; MGR_EINVAL for a bad device or a null pointer, MGR_ECUDA if
   a CUDA call fails.  The current device is restored. */
int mgr_fp64_fma_rate(int device, double* fma_per_second);

/* Bounds-checking builds.  A library compiled with MGR_DEBUG_BOUNDS checks,
   in every kernel of the level loop (level pass, interpolation, solves,
   one-CTA coarse levels, coarsest copy; single-field, batched, served and 4D
   forms), each global index against the extent of the buffer it addresses
   and the level pass's shared-tile indices against the tile.  A violation
   is recorded in a device error record and the access is skipped (no trap:
   the context stays usable); the operation then waits for its stream
   (unless the stream is being captured) and returns MGR_EDEVICE, batched
   polls and served waits likewise.  The paper has no counterpart: this is
   a debugging aid of this library.
   mgr_debug_bounds: 1 in such a build, 0 otherwise.
   mgr_debug_last: the first out-of-bounds access of the last operation that
   returned MGR_EDEVICE -- a code naming the access, its index and the
   buffer's extent in elements; MGR_ENOTFOUND if none was recorded. */
int mgr_debug_bounds(void);
int mgr_debug_last(int* code, int64_t* index, int64_t* extent);

/* Size of the fixed device scratch area used by mgr_decompose_noalloc. */
#define MGR_NOALLOC_SCRATCH_BYTES (32u << 20)

/* Decomposition for callers that cannot allocate device memory (their
   device memory is entirely owned by another allocator, they are handed
   only their input and output buffers, or an allocation -- which may
   synchronise the device -- is not acceptable on their path).  The paper
   has no counterpart: this is a calling convention of this library.
   Same operation and arguments as mgr_decompose, without the workspace:
   the workspace is a fixed MGR_NOALLOC_SCRATCH_BYTES area in this library's
   device image, which every GPU that loads the library holds until the
   process exits.  The call allocates nothing (no cudaMalloc / cudaFree) and
   launches the kernels directly on `stream`.
     - Returns MGR_EINVAL when the plan's mgr_workspace_size() exceeds
       MGR_NOALLOC_SCRATCH_BYTES (for example FP64 fields of more than about
       15 million nodes), and for the argument errors of mgr_decompose
       (among them in == out for a 4D plan, which runs out of place only).
     - The plan's device must be the calling thread's current device (the
       kernels use that device's copy of the area); MGR_EINVAL otherwise.
     - The first call on a device looks up the area's device address; make
       that first call before any stream capture.  A first call made while
       `stream` is being captured returns MGR_EINVAL and leaves the capture
       untouched.
     - Every call on a device shares the one area, which keeps the previous
       call's contents (nothing in it needs to start at zero).  Calls whose
       work overlaps on the GPU (different streams, or other host threads)
       race on it: serialise them. */
int mgr_decompose_noalloc(const mgr_plan* plan, const void* in, void* out, mgr_stream_t stream);

/* ------------------------------------------------------------ batching */

#define MGR_OP_DECOMPOSE 0
#define MGR_OP_RECOMPOSE 1

/* One field of a batch. */
typedef struct {
  int op;               /* MGR_OP_DECOMPOSE or MGR_OP_RECOMPOSE                      */
  const mgr_plan* plan; /* the field's plan; every request of a submit shares the
                           plan's dtype and precision                                */
  const void* in;       /* DEVICE, field-sized                                       */
  void* out;            /* DEVICE, field-sized, distinct from `in`                   */
  uint64_t user_tag;    /* caller's bookkeeping; not interpreted                     */
  int keep_resident;    /* serving layer only (mgr_serve_*); ignored by a batch      */
} mgr_request;

/* Batched refactoring of many independent fields of uneven sizes (the
   batching pattern of the hot path): all fields advance level by level
   together, each phase of the level loop (level pass, x/y/z solves,
   interpolation) is ONE persistent launch whose CTAs walk a list of work
   items across all fields, and the phase sequence is captured once into a
   CUDA graph and replayed on later submits of the same request list.  The
   level-pass tile shape and z-chunk length are chosen by the autotuner on
   the first submit of a batch shape (analytic model ranks the candidates,
   the top three are timed).  Decompositions run before recompositions; the
   requests of one submit must be independent (no request reads another's
   output).  The context allocates the workspaces (counted against its
   memory budget; MGR_EBUDGET when a batch can never fit) and runs the work
   on its own stream.  Returns after enqueueing; *ticket identifies the
   submit for mgr_batch_poll. */
int mgr_batch_submit(mgr_ctx* ctx, const mgr_request* reqs, int n, uint64_t* ticket);

/* Wait up to timeout_us microseconds (0: do not wait, < 0: no limit) for a
   submit.  MGR_OK with *n_done = its request count when finished (the ticket
   is then released), MGR_EPENDING (timeout 0) or MGR_ETIMEDOUT otherwise,
   MGR_ENOTFOUND for an unknown or released ticket. */
int mgr_batch_poll(mgr_ctx* ctx, uint64_t ticket, int64_t timeout_us, int* n_done);

/* Text report of the autotuner's decisions (candidate tile shapes and their
   measured times per batch shape).  Writes at most len bytes including the
   terminating NUL; returns the full length. */
int mgr_batch_tuning(mgr_ctx* ctx, char* buf, size_t len);

/* ------------------------------------------------------------ serving */

/* The serving pattern: a request loop that admits decompose / recompose
   requests of mixed sizes by device-memory budget and keeps hierarchies
   resident.  Requests enter a FIFO queue; a dispatcher admits the head as
   soon as one of `slots` execution slots is free and its device memory (its
   workspace, plus the hierarchy for a decomposition) fits the context's
   budget, evicting least recently used resident hierarchies that no request
   references.  Admitted requests run on a pool of `streams` streams, so work
   of requests that arrive while others run overlaps on the device
   (continuous batching).  A decomposition writes its hierarchy (nodal
   coefficients) into library memory; with keep_resident it stays resident
   under a handle equal to the request id, for later recompositions. */
typedef struct mgr_server mgr_server;

typedef struct {
  int op;               /* MGR_OP_DECOMPOSE: in -> resident hierarchy;
                           MGR_OP_RECOMPOSE: resident hierarchy `src` -> out */
  const mgr_plan* plan; /* field description (the plan must outlive the request) */
  const void* in;       /* decompose: DEVICE field, read while the request runs */
  uint64_t src;         /* recompose: handle of a finished resident hierarchy  */
  void* out;            /* recompose: DEVICE field buffer                      */
  int keep_resident;    /* decompose: keep the hierarchy after completion      */
  double arrival;       /* arrival time (mgr_serve_now() clock); 0 = now       */
} mgr_serve_request;

typedef struct {
  int status;      /* MGR_OK, or the request's error (MGR_EBUDGET, MGR_ECUDA, ...) */
  double arrival;  /* seconds, mgr_serve_now() clock                               */
  double admitted; /* when it was launched                                        */
  double done;     /* when its completion was observed                             */
  uint64_t handle; /* resident hierarchy handle (decompose with keep_resident)     */
} mgr_serve_result;

/* Steady clock in seconds used for the request time stamps. */
double mgr_serve_now(void);
int mgr_serve_start(mgr_ctx* ctx, int slots, int streams, mgr_server** server);
/* Queue a request.  MGR_EBUDGET if it can never fit the budget, MGR_ENOTFOUND
   for an unknown hierarchy, MGR_EPENDING if that hierarchy is not finished. */
int mgr_serve_enqueue(mgr_server* server, const mgr_serve_request* req, uint64_t* id);
/* Wait up to timeout_us (0: poll, < 0: no limit) for request `id`; on MGR_OK
   fills *res and forgets the request.  MGR_EPENDING / MGR_ETIMEDOUT otherwise. */
int mgr_serve_wait(mgr_server* server, uint64_t id, int64_t timeout_us, mgr_serve_result* res);
/* Device pointer of a finished resident hierarchy (nodal layout of its plan). */
int mgr_serve_hierarchy(mgr_server* server, uint64_t handle, const void** ptr);
/* Copy a finished resident hierarchy into the caller's DEVICE buffer `dst`
   (field-sized) on `stream`. */
int mgr_serve_read(mgr_server* server, uint64_t handle, void* dst, mgr_stream_t stream);
/* Drop a resident hierarchy (MGR_EPENDING while a request still uses it). */
int mgr_serve_release(mgr_server* server, uint64_t handle);
int mgr_serve_stats(mgr_server* server, size_t* used_bytes, int* queued, int* running, int* resident);
/* Finish all queued and running requests, free every resident hierarchy. */
int mgr_serve_stop(mgr_server* server);

/* ------------------------------------------------------------ profiling */

/* One kernel launch of an operation, timed by CUDA events recorded on the
   launching stream immediately before and after it. */
typedef struct {
  char name[32]; /* kernel role: level_load_dec, level_load_rec, solve_x/y/z, interp,
                    interp_zero (a dropped class), coarsest, coef_inplace          */
  int level;     /* level l of the launch (0 for the coarsest-grid copy)            */
  float ms;      /* event-to-event duration                                         */
  double bytes;  /* compulsory bytes of the launch's inputs and outputs             */
  double flops;  /* floating-point operations of its minimal arithmetic (FMA = 2)   */
} mgr_kernel_time;

#define MGR_OP_DECOMPOSE_PACKED 2 /* mgr_profile only: mgr_decompose_packed                */
#define MGR_OP_RECOMPOSE_PACKED 3 /* mgr_profile only: mgr_recompose_packed, every class   */

/* Run one decomposition (op = 0) or recomposition (op = 1), or their
   class-packed forms (op = 2, 3), exactly as mgr_decompose / mgr_recompose /
   mgr_decompose_packed / mgr_recompose_packed would, but launched directly (no graph) with
   a pair of CUDA events around every kernel, and wait for it.  Writes up to
   `cap` records to `times` and the number of launches to *n (which may exceed
   cap).  Not part of the hot path: it synchronises `stream`. */
int mgr_profile(const mgr_plan* plan, int op, const void* in, void* out, void* workspace, mgr_stream_t stream,
                mgr_kernel_time* times, int cap, int* n);

#ifdef __cplusplus
}
#endif

#endif /* MGR_H */
