// Generic element-scan instantiations (pit_filter_scan / pit_smooth_scan), F32.
#include "pit_solve_impl.cuh"

namespace pit {
namespace {
int fscan_2(const ScanArgs& a, size_t* w) { return ScanImpl<float, 2, 4, 1>::filter(a, w); }
int sscan_2(const ScanArgs& a, size_t* w) { return ScanImpl<float, 2, 4, 1>::smooth(a, w); }
ScanRegistrar sreg_2(PIT_F32, 2, fscan_2, sscan_2);
int fscan_3(const ScanArgs& a, size_t* w) { return ScanImpl<float, 3, 4, 1>::filter(a, w); }
int sscan_3(const ScanArgs& a, size_t* w) { return ScanImpl<float, 3, 4, 1>::smooth(a, w); }
ScanRegistrar sreg_3(PIT_F32, 3, fscan_3, sscan_3);
int fscan_4(const ScanArgs& a, size_t* w) { return ScanImpl<float, 4, 4, 1>::filter(a, w); }
int sscan_4(const ScanArgs& a, size_t* w) { return ScanImpl<float, 4, 4, 1>::smooth(a, w); }
ScanRegistrar sreg_4(PIT_F32, 4, fscan_4, sscan_4);
int fscan_6(const ScanArgs& a, size_t* w) { return ScanImpl<float, 6, 8, 1>::filter(a, w); }
int sscan_6(const ScanArgs& a, size_t* w) { return ScanImpl<float, 6, 8, 1>::smooth(a, w); }
ScanRegistrar sreg_6(PIT_F32, 6, fscan_6, sscan_6);
int fscan_8(const ScanArgs& a, size_t* w) { return ScanImpl<float, 8, 8, 1>::filter(a, w); }
int sscan_8(const ScanArgs& a, size_t* w) { return ScanImpl<float, 8, 8, 1>::smooth(a, w); }
ScanRegistrar sreg_8(PIT_F32, 8, fscan_8, sscan_8);
}  // namespace
}  // namespace pit
