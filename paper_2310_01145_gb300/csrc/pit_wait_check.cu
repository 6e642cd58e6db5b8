// pit_check_wait: runs the bounded cross-block wait of the single-launch iteration kernel
// (group_wait in pit_fused.cuh) once, on a flag word the caller provides, so that its timeout
// path can be exercised without a faulted or stalled block: with a flag that nothing sets the
// wait must give up after `poll_limit` polls, set the timeout bit and return.
#include "pit_fused.cuh"
#include "pit_internal.h"

namespace pit {
namespace {

// words[0] = flag, words[1] = status, words[2] = result (1: flag seen, 0: gave up)
__global__ void k_wait_check(unsigned* words, unsigned target, long long limit) {
  Grp<float, 8, 8, 1> g;
  g.init();
  if (threadIdx.x >= 8) return;
  const bool ok = group_wait(g, words + 0, target, words + 1, limit);
  if (g.gl == 0) words[2] = ok ? 1u : 0u;
}

}  // namespace
}  // namespace pit

using namespace pit;

extern "C" int32_t pit_check_wait(int64_t poll_limit, uint32_t target, void* words,
                                  void* stream) {
  if (poll_limit < 0 || !words || reinterpret_cast<uintptr_t>(words) % 4 != 0) {
    set_error("pit_check_wait: poll_limit must be >= 0 and words a 4-byte aligned device pointer");
    return PIT_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned* w = static_cast<unsigned*>(words);
  PIT_CUDA_TRY(cudaMemsetAsync(w + 1, 0, 2 * sizeof(unsigned), s));
  PIT_LAUNCH(KC_ITERATION, s, k_wait_check<<<1, 32, 0, s>>>(w, target, poll_limit));
  PIT_CUDA_TRY(cudaGetLastError());
  unsigned host[3] = {0, 0, 0};
  PIT_CUDA_TRY(cudaMemcpyAsync(host, w, sizeof(host), cudaMemcpyDeviceToHost, s));
  PIT_CUDA_TRY(cudaStreamSynchronize(s));
  if (host[2] == 1u && !(host[1] & kStatusTimeout)) return PIT_OK;
  if (host[2] == 0u && (host[1] & kStatusTimeout)) {
    set_error("pit_check_wait: the wait gave up after the poll limit and set the timeout bit");
    return PIT_ETIMEOUT;
  }
  set_error("pit_check_wait: inconsistent result of the bounded wait");
  return PIT_EINTERNAL;
}
