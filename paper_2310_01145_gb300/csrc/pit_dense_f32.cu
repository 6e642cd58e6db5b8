// Large-state solver, FP32 arithmetic (FP64 trajectory).
#include "pit_dense_impl.cuh"

namespace pit {
namespace {
int solve_dense_f32(const SolveArgs& a, size_t* w, bool e) { return dn::DenseSolver<float>::run(a, w, e); }
DenseRegistrar reg_dense_f32(PIT_F32, solve_dense_f32);
int scan_f_f32(const ScanArgs& a, size_t* w) { return dn::DenseScan<float>::filter(a, a.D, w); }
int scan_s_f32(const ScanArgs& a, size_t* w) { return dn::DenseScan<float>::smooth(a, a.D, w); }
DenseRegistrar reg_dense_scan_f32(PIT_F32, scan_f_f32, scan_s_f32);
LargeSession* make_session_f32() { return new dn::DenseSession<float>(); }
LargeSessionRegistrar reg_session_f32(PIT_F32, make_session_f32);
}  // namespace
size_t large_session_bytes_f32(const Problem& pb, const pit_opts& o) {
  return dn::DenseSession<float>::bytes(pb, o);
}
int dense_linearize_f32(const Problem& pb, int lin_mode, const void* traj, void* H, void* dv,
                        cudaStream_t s) {
  return dn::dense_linearize<float>(pb, lin_mode, traj, H, dv, s);
}
}  // namespace pit
