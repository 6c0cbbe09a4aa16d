// mgr_device.cuh -- small device helpers shared by the kernels of this
// library (index maps of the nested hierarchy and cp.async wrappers).
// Included inside an anonymous namespace of each translation unit.
#pragma once

__device__ __forceinline__ int pidx(int q, int n) { return min(2 * q, n - 1); }
__device__ __forceinline__ bool is_coarse(int i, int n) { return ((i & 1) == 0) || (i == n - 1); }
__device__ __forceinline__ int cidx(int i) { return (i + 1) >> 1; }
// first fine node of the stencil region of coarse node q0, moved down to a coarse node
__device__ __forceinline__ int region_start(int q0, int n) {
  const int r = pidx(q0, n) - 2;
  return (r & 1) ? r - 1 : r;
}
__device__ __forceinline__ int64_t fmap(int i, int64_t s, int64_t N) {
  int64_t f = int64_t(i) * s;
  return f < N - 1 ? f : N - 1;
}

// Asynchronous global -> shared copy of 4, 8 or 16 bytes (both addresses
// aligned to the copy size).
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes) {
  unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
  else if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// The same copy of `bytes` (4, 8 or 16) that reads nothing and writes zeros
// when `valid` is false (the copy's source-size operand): a branch-free
// predicated load.  `gmem` must be a valid address either way.
__device__ __forceinline__ void cp_async_zf(void* smem, const void* gmem, int bytes, bool valid) {
  unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  const unsigned n = valid ? unsigned(bytes) : 0u;
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(n) : "memory");
  else if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(n) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}


// ---------------------------------------------------------------------------
// Bounds-checking builds (MGR_DEBUG_BOUNDS): every checked access tests its
// index against the extent of the buffer it addresses; a violation is
// recorded in this translation unit's device record (the first one's code,
// index and extent, and a count) and the access is skipped -- no trap, the
// context stays usable.  The host reads and clears the record after each
// operation and returns MGR_EDEVICE.  In other builds a check is `true` and
// compiles away.
// ---------------------------------------------------------------------------
#ifdef MGR_DEBUG_BOUNDS
static __device__ DebugRecord g_debug_record;
__device__ __forceinline__ bool dbg_in(long long i, long long n, int code) {
  if (i >= 0 && i < n) return true;
  if (atomicAdd(&g_debug_record.count, 1ull) == 0ull) {
    g_debug_record.code = code;
    g_debug_record.index = i;
    g_debug_record.extent = n;
  }
  return false;
}
#define MGR_IN(i, n, code) dbg_in((long long)(i), (long long)(n), (code))
#else
#define MGR_IN(i, n, code) true
#endif
// pointer p inside [base, base + n)
#define MGR_PIN(p, base, n, code) MGR_IN((p) - (base), (n), (code))
// the statement(s) after `check`, run only where the check holds; other builds
// run them unconditionally and do not evaluate `check` at all
#ifdef MGR_DEBUG_BOUNDS
#define MGR_GUARD(check, ...) \
  do {                        \
    if (check) {              \
      __VA_ARGS__;            \
    }                         \
  } while (0)
#else
#define MGR_GUARD(check, ...) \
  do {                        \
    __VA_ARGS__;              \
  } while (0)
#endif
