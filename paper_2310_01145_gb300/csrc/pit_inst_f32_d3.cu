// Kernel instantiations for F32 arithmetic, ODE dimension d = 3 (generated list; one
// translation unit per (dtype, d) so that the build compiles them in parallel).
#include "pit_solve_impl.cuh"

namespace pit {
namespace {
int solve_3_1(const SolveArgs& a, size_t* w, bool e) {
  return SolverImpl<float, 3, 2, 8, 1>::run(a, w, e);
}
Registrar reg_3_1(PIT_F32, 3, 1, 0, solve_3_1);
int solve_3_1_v1(const SolveArgs& a, size_t* w, bool e) {
  return SolverImpl<float, 3, 2, 4, 2, 8, 1>::run(a, w, e);
}
Registrar reg_3_1_v1(PIT_F32, 3, 1, 1, solve_3_1_v1);
int solve_3_2(const SolveArgs& a, size_t* w, bool e) {
  return SolverImpl<float, 3, 3, 16, 1>::run(a, w, e);
}
Registrar reg_3_2(PIT_F32, 3, 2, 0, solve_3_2);
}  // namespace
}  // namespace pit
