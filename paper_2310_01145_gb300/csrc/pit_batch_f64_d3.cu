// Segmented-solve engines for F64 arithmetic, ODE dimension d = 3 (one translation
// unit per (dtype, d) so that the build compiles them in parallel).
#include "pit_batch.cuh"

namespace pit {
namespace {
SegRegistrar seg_3_1(PIT_F64, 3, 1, &SegEngineImpl<double, 3, 2, 8, 1>::make);
SegRegistrar seg_3_2(PIT_F64, 3, 2, &SegEngineImpl<double, 3, 3, 16, 1>::make);
}  // namespace
}  // namespace pit
