// pit_check_dgemm_tc: one thread block computes an FP64 product through the tensor-core digit
// GEMM of the large-state solver (cta_dgemm in pit_tc.cuh), so that its accuracy, its operand
// layouts and its bounded wait can be checked on their own against an FP64 product.
#include <algorithm>
#include <string>

#include "pit_internal.h"
#include "pit_tc.cuh"

namespace pit {
namespace {

template <bool TA, bool TB>
__global__ void __launch_bounds__(512, 1)
k_tc_dgemm(int m, int n, int k, double alpha, const double* __restrict__ A, int lda,
           const double* __restrict__ B, int ldb, double beta, double* __restrict__ C, int ldc,
           unsigned* status) {
  extern __shared__ __align__(128) unsigned char smem_tc[];
  tc::tc_setup();
  const tc::TcCtx c{smem_tc, status, tc::kTcWaitNs};
  tc::cta_dgemm<TA, TB>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
  if (threadIdx.x == 0 && tc::tc_state().fail) status[1] = tc::tc_state().where;
  tc::tc_teardown();
}

// Waits once on the block's mbarrier with nothing committed to it: the wait must give up after
// wait_ns, set the timeout bit and still free the tensor memory.
__global__ void __launch_bounds__(512, 1) k_tc_wait(unsigned* status, unsigned long long wait_ns) {
  extern __shared__ __align__(128) unsigned char smem_tc[];
  tc::tc_setup();
  const tc::TcCtx c{smem_tc, status, wait_ns};
  tc::tc_wait(c);
  __syncthreads();
  if (threadIdx.x == 0) status[1] = tc::tc_state().fail ? tc::tc_state().where : 0u;
  tc::tc_teardown();
}

template <bool TA, bool TB>
int launch(int m, int n, int k, double alpha, const double* A, int lda, const double* B, int ldb,
           double beta, double* C, int ldc, unsigned* status, cudaStream_t s) {
  const int sm = static_cast<int>(tc::stage_bytes());
  PIT_CUDA_TRY(cudaFuncSetAttribute(k_tc_dgemm<TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  PIT_LAUNCH(KC_ITERATION, s,
             (k_tc_dgemm<TA, TB><<<1, 512, sm, s>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, status)));
  PIT_CUDA_TRY(cudaGetLastError());
  return PIT_OK;
}

}  // namespace
}  // namespace pit

using namespace pit;

extern "C" int32_t pit_check_dgemm_tc(int32_t m, int32_t n, int32_t k, int32_t trans_a,
                                      int32_t trans_b, double alpha, const void* A, int32_t lda,
                                      const void* B, int32_t ldb, double beta, void* C,
                                      int32_t ldc, void* status, void* stream) {
  set_error("");
  const int rows_a = trans_a ? k : m, cols_a = trans_a ? m : k;
  const int rows_b = trans_b ? n : k, cols_b = trans_b ? k : n;
  if (m < 0 || n < 0 || k < 0 || m > 4096 || n > 4096 || k > 4096 || (trans_a & ~1) ||
      (trans_b & ~1) || lda < std::max(1, cols_a) || ldb < std::max(1, cols_b) ||
      ldc < std::max(1, n) || !status || reinterpret_cast<uintptr_t>(status) % 4 != 0 ||
      (m * k > 0 && !A) || (k * n > 0 && !B) || (m * n > 0 && !C)) {
    set_error("pit_check_dgemm_tc: need 0 <= m, n, k <= 4096, trans flags 0/1, leading dimensions "
              "at least the row lengths, device pointers and a 4-byte aligned status word pair");
    return PIT_EINVAL;
  }
  (void)rows_a;
  (void)rows_b;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned* st = static_cast<unsigned*>(status);
  PIT_CUDA_TRY(cudaMemsetAsync(st, 0, 2 * sizeof(unsigned), s));
  const double* a = static_cast<const double*>(A);
  const double* b = static_cast<const double*>(B);
  double* cc = static_cast<double*>(C);
  int rc;
  if (trans_a) rc = trans_b ? launch<true, true>(m, n, k, alpha, a, lda, b, ldb, beta, cc, ldc, st, s)
                            : launch<true, false>(m, n, k, alpha, a, lda, b, ldb, beta, cc, ldc, st, s);
  else rc = trans_b ? launch<false, true>(m, n, k, alpha, a, lda, b, ldb, beta, cc, ldc, st, s)
                    : launch<false, false>(m, n, k, alpha, a, lda, b, ldb, beta, cc, ldc, st, s);
  if (rc != PIT_OK) return rc;
  unsigned host[2] = {0, 0};
  PIT_CUDA_TRY(cudaMemcpyAsync(host, st, sizeof(host), cudaMemcpyDeviceToHost, s));
  PIT_CUDA_TRY(cudaStreamSynchronize(s));
  if (host[0] & tc::kTcTimeoutBit) {
    set_error("pit_check_dgemm_tc: a tensor-core wait gave up (product " +
              std::to_string(host[1]) + ")");
    return PIT_ETIMEOUT;
  }
  return PIT_OK;
}

extern "C" int32_t pit_check_tc_wait(int64_t wait_ns, void* status, void* stream) {
  set_error("");
  if (wait_ns < 0 || wait_ns > 4000000000ll || !status ||
      reinterpret_cast<uintptr_t>(status) % 4 != 0) {
    set_error("pit_check_tc_wait: need 0 <= wait_ns <= 4e9 and a 4-byte aligned status word pair");
    return PIT_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned* st = static_cast<unsigned*>(status);
  const int sm = static_cast<int>(tc::stage_bytes());
  PIT_CUDA_TRY(cudaFuncSetAttribute(k_tc_wait, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  PIT_CUDA_TRY(cudaMemsetAsync(st, 0, 2 * sizeof(unsigned), s));
  PIT_LAUNCH(KC_ITERATION, s, (k_tc_wait<<<1, 512, sm, s>>>(st, static_cast<unsigned long long>(wait_ns))));
  PIT_CUDA_TRY(cudaGetLastError());
  unsigned host[2] = {0, 0};
  PIT_CUDA_TRY(cudaMemcpyAsync(host, st, sizeof(host), cudaMemcpyDeviceToHost, s));
  PIT_CUDA_TRY(cudaStreamSynchronize(s));
  if ((host[0] & tc::kTcTimeoutBit) && host[1] == 1u) {
    set_error("pit_check_tc_wait: the wait gave up and set the timeout bit");
    return PIT_ETIMEOUT;
  }
  set_error("pit_check_tc_wait: the wait on an mbarrier that nothing arrives on returned");
  return PIT_EINTERNAL;
}
