// Segmented-solve engines for F32 arithmetic, ODE dimension d = 2 (one translation
// unit per (dtype, d) so that the build compiles them in parallel).
#include "pit_batch.cuh"

namespace pit {
namespace {
SegRegistrar seg_2_1(PIT_F32, 2, 1, &SegEngineImpl<float, 2, 2, 4, 1>::make);
SegRegistrar seg_2_2(PIT_F32, 2, 2, &SegEngineImpl<float, 2, 3, 8, 1>::make);
SegRegistrar seg_2_3(PIT_F32, 2, 3, &SegEngineImpl<float, 2, 4, 8, 1>::make);
}  // namespace
}  // namespace pit
