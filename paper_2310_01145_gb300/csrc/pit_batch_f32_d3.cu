// Segmented-solve engines for F32 arithmetic, ODE dimension d = 3 (one translation
// unit per (dtype, d) so that the build compiles them in parallel).
#include "pit_batch.cuh"

namespace pit {
namespace {
SegRegistrar seg_3_1(PIT_F32, 3, 1, &SegEngineImpl<float, 3, 2, 8, 1>::make);
SegRegistrar seg_3_2(PIT_F32, 3, 2, &SegEngineImpl<float, 3, 3, 16, 1>::make);
}  // namespace
}  // namespace pit
