// Segmented-solve engines for F64 arithmetic, ODE dimension d = 1 (one translation
// unit per (dtype, d) so that the build compiles them in parallel).
#include "pit_batch.cuh"

namespace pit {
namespace {
SegRegistrar seg_1_1(PIT_F64, 1, 1, &SegEngineImpl<double, 1, 2, 4, 1>::make);
SegRegistrar seg_1_2(PIT_F64, 1, 2, &SegEngineImpl<double, 1, 3, 4, 1>::make);
SegRegistrar seg_1_3(PIT_F64, 1, 3, &SegEngineImpl<double, 1, 4, 4, 1>::make);
}  // namespace
}  // namespace pit
