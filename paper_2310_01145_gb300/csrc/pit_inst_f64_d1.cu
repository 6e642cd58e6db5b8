// Kernel instantiations for F64 arithmetic, ODE dimension d = 1 (generated list; one
// translation unit per (dtype, d) so that the build compiles them in parallel).
#include "pit_solve_impl.cuh"

namespace pit {
namespace {
int solve_1_1(const SolveArgs& a, size_t* w, bool e) {
  return SolverImpl<double, 1, 2, 4, 1>::run(a, w, e);
}
Registrar reg_1_1(PIT_F64, 1, 1, 0, solve_1_1);
int solve_1_2(const SolveArgs& a, size_t* w, bool e) {
  return SolverImpl<double, 1, 3, 4, 1>::run(a, w, e);
}
Registrar reg_1_2(PIT_F64, 1, 2, 0, solve_1_2);
int solve_1_3(const SolveArgs& a, size_t* w, bool e) {
  return SolverImpl<double, 1, 4, 4, 1>::run(a, w, e);
}
Registrar reg_1_3(PIT_F64, 1, 3, 0, solve_1_3);
}  // namespace
}  // namespace pit
