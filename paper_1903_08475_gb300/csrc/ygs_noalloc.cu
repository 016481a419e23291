// ygs_solve_static: the FP64 solve (projection, radial scans, synthesis) with
// its split-K partial sums and the moments B and M held in one file-scope
// device array instead of workspaces from the device allocator.
//
// Who needs this: callers that may not allocate device memory at the moment
// they solve -- a host framework that has handed all free device memory to
// its own pool, or a time-stepping loop that forbids allocator calls (and the
// synchronisation some of them imply) once it is running.  The plan itself is
// still made by ygs_create beforehand; this entry point adds no allocation of
// its own: no cudaMalloc, no cudaFree, no library routine that allocates.
//
// The array is shared by every call in the process on a given device: two of
// these calls whose GPU work overlaps (different streams without ordering,
// different host threads) race on it and give wrong results.  Nothing in it
// needs to start at zero: every element a kernel reads was written earlier in
// the same call (each split-K chunk writes its whole [n_r][K] plane, the
// scan writes all of B and M).
#include <string>

#include "ygs_internal.h"

namespace ygs {
namespace {

constexpr size_t kScratchDoubles = (size_t)YGS_STATIC_SCRATCH_BYTES / sizeof(double);

// Layout of one call: S split-K planes of [n_r][K], then B [n_r][K], then M [n_r][K].
static __device__ __align__(256) double g_scratch[kScratchDoubles];

// Device address of g_scratch on the current device.  Looked up on every
// call rather than cached: a cached address would outlive a reset of the
// device or a new primary context, and cudaGetSymbolAddress costs little once
// the module is loaded (ygs_create loads it, see prepare_static_scratch).
cudaError_t scratch_address(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  *out = (double*)p;
  return e;
}

struct CurrentDevice {
  int prev = -1;
  bool ok = true;
  explicit CurrentDevice(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = (cudaSetDevice(dev) == cudaSuccess);
  }
  ~CurrentDevice() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

ygs_status fail(ygs_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

}  // namespace

cudaError_t prepare_static_scratch() {
  double* base = nullptr;
  return scratch_address(&base);
}

long long static_scratch_bytes(const ygs_plan* p) {
  return (long long)(p->S + 2) * p->n_r * (long long)p->K * (long long)sizeof(double);
}

}  // namespace ygs

using namespace ygs;

extern "C" size_t ygs_static_scratch_capacity(void) { return (size_t)YGS_STATIC_SCRATCH_BYTES; }

extern "C" ygs_status ygs_solve_static(ygs_plan* p, const double* d_rho, double* d_phi, void* stream) {
  if (!p) return fail(YGS_ERR_INVALID_ARG, "plan is NULL");
  if (!d_rho || !d_phi) return fail(YGS_ERR_INVALID_ARG, "field pointer is NULL");
  if (((uintptr_t)d_rho & 15) || ((uintptr_t)d_phi & 15))
    return fail(YGS_ERR_INVALID_ARG, "field pointers must be 16-byte aligned");
  const size_t bytes = (size_t)p->n_cells * sizeof(double);
  const char* ca = (const char*)d_rho;
  const char* cb = (const char*)d_phi;
  if (ca < cb + bytes && cb < ca + bytes) return fail(YGS_ERR_INVALID_ARG, "input and output fields overlap");
  const size_t need = (size_t)static_scratch_bytes(p);
  if (need > (size_t)YGS_STATIC_SCRATCH_BYTES)
    return fail(YGS_ERR_UNSUPPORTED, "ygs_solve_static: this plan needs " + std::to_string(need) +
                                         " bytes of scratch ((fp64_split_k + 2) * n_r * K doubles = (" +
                                         std::to_string(p->S) + " + 2) * " + std::to_string(p->n_r) + " * " +
                                         std::to_string(p->K) + "), more than the static " +
                                         std::to_string((size_t)YGS_STATIC_SCRATCH_BYTES) +
                                         " bytes; use ygs_solve");
  CurrentDevice cur(p->device);
  if (!cur.ok) return fail(YGS_ERR_CUDA, "cudaSetDevice failed");
  double* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return fail(YGS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  const size_t plane = (size_t)p->n_r * p->K;
  double* part = base;
  double* B = base + (size_t)p->S * plane;
  double* M = B + plane;
  cudaStream_t s = (cudaStream_t)stream;
  if ((e = launch_project_fp64(p, d_rho, p->U, part, s)) != cudaSuccess ||
      (e = launch_scan_fwd(p, part, p->S, B, M, s)) != cudaSuccess ||
      (e = launch_synth_fp64(p, M, p->Q, d_phi, s)) != cudaSuccess)
    return fail(YGS_ERR_CUDA, std::string("ygs_solve_static launch: ") + cudaGetErrorString(e));
  return YGS_OK;
}
