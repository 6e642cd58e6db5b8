// Large-state solver, FP32 arithmetic (double-float trajectory).
#include "pit_dense_impl.cuh"

namespace pit {
namespace {
int solve_dense_f32(const SolveArgs& a, size_t* w, bool e) { return dn::DenseSolver<float>::run(a, w, e); }
DenseRegistrar reg_dense_f32(PIT_F32, solve_dense_f32);
}  // namespace
}  // namespace pit
