// pit_solve_noalloc: pit_solve for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or have torch or another allocator do it) at the point
// where they want a solve: serving loops whose device memory budget is fixed when they start,
// plug-ins that run inside another framework's memory manager with no device allocator of their
// own, and real-time hosts that forbid allocation -- and the device synchronisation cudaMalloc
// can bring -- once initialised.  For them this entry point runs the same solver with its
// scratch space in a fixed, file-scope device array instead of a caller-provided workspace.
//
// The array is kStaticScratchBytes (64 MiB) and, like any __device__ variable, every GPU that
// loads the library holds it until the process exits.  Its device address is obtained once per
// device (cudaGetSymbolAddress with that device current) on the first call made on that device
// and kept for the life of the process; do not reset the device after it (a new context could
// place the array elsewhere).  All calls
// share the one array and it keeps the previous call's contents; the solver initialises every
// scratch region it reads (the trajectory, residuals, aggregates and its scalar accumulators),
// so nothing has to start at zero.  Calls whose device work overlaps -- on different streams,
// or from different host threads -- race on the array: serialise them.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "pit_internal.h"

namespace pit {
namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the static scratch array on the current device (set up once per device).
int static_scratch(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error(std::string("pit_solve_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    return PIT_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("pit_solve_noalloc: device ordinal out of range");
    return PIT_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("pit_solve_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return PIT_ECUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return PIT_OK;
}

}  // namespace
}  // namespace pit

using namespace pit;

extern "C" int32_t pit_solve_noalloc(const pit_ode* ode, const pit_grid* grid, int32_t q,
                                     const double* y0, const pit_opts* opts,
                                     const void* init_traj, void* mean, void* sqrtcov,
                                     pit_solve_info* info, void* stream) {
  size_t need = 0;
  int32_t st = pit_solve_workspace_size(ode, grid, q, opts, &need);
  if (st != PIT_OK) return st;
  if (need > kStaticScratchBytes) {
    set_error("pit_solve_noalloc: this problem needs " + std::to_string(need) +
              " bytes of scratch; the static scratch array holds " +
              std::to_string(kStaticScratchBytes) + " bytes (use pit_solve with a workspace)");
    return PIT_ENOMEM;
  }
  void* ws = nullptr;
  st = static_scratch(&ws);
  if (st != PIT_OK) return st;
  return pit_solve(ode, grid, q, y0, opts, init_traj, mean, sqrtcov, info, ws,
                   kStaticScratchBytes, stream);
}
