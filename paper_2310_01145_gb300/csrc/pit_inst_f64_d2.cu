// Kernel instantiations for F64 arithmetic, ODE dimension d = 2 (generated list; one
// translation unit per (dtype, d) so that the build compiles them in parallel).
#include "pit_solve_impl.cuh"

namespace pit {
namespace {
int solve_2_1(const SolveArgs& a, size_t* w, bool e) {
  return SolverImpl<double, 2, 2, 4, 1>::run(a, w, e);
}
Registrar reg_2_1(PIT_F64, 2, 1, 0, solve_2_1);
int solve_2_2(const SolveArgs& a, size_t* w, bool e) {
  return SolverImpl<double, 2, 3, 8, 1>::run(a, w, e);
}
Registrar reg_2_2(PIT_F64, 2, 2, 0, solve_2_2);
int solve_2_2_v1(const SolveArgs& a, size_t* w, bool e) {
  return SolverImpl<double, 2, 3, 4, 2, 8, 1>::run(a, w, e);
}
Registrar reg_2_2_v1(PIT_F64, 2, 2, 1, solve_2_2_v1);
int solve_2_3(const SolveArgs& a, size_t* w, bool e) {
  return SolverImpl<double, 2, 4, 8, 1>::run(a, w, e);
}
Registrar reg_2_3(PIT_F64, 2, 3, 0, solve_2_3);
int solve_2_3_v1(const SolveArgs& a, size_t* w, bool e) {
  return SolverImpl<double, 2, 4, 4, 2, 8, 1>::run(a, w, e);
}
Registrar reg_2_3_v1(PIT_F64, 2, 3, 1, solve_2_3_v1);
}  // namespace
}  // namespace pit
