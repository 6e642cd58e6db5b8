// Large-state solver, FP64 arithmetic.
#include "pit_dense_impl.cuh"

namespace pit {
namespace {
int solve_dense_f64(const SolveArgs& a, size_t* w, bool e) { return dn::DenseSolver<double>::run(a, w, e); }
DenseRegistrar reg_dense_f64(PIT_F64, solve_dense_f64);
int scan_f_f64(const ScanArgs& a, size_t* w) { return dn::DenseScan<double>::filter(a, a.D, w); }
int scan_s_f64(const ScanArgs& a, size_t* w) { return dn::DenseScan<double>::smooth(a, a.D, w); }
DenseRegistrar reg_dense_scan_f64(PIT_F64, scan_f_f64, scan_s_f64);
LargeSession* make_session_f64() { return new dn::DenseSession<double>(); }
LargeSessionRegistrar reg_session_f64(PIT_F64, make_session_f64);
}  // namespace
size_t large_session_bytes_f64(const Problem& pb, const pit_opts& o) {
  return dn::DenseSession<double>::bytes(pb, o);
}
int dense_linearize_f64(const Problem& pb, int lin_mode, const void* traj, void* H, void* dv,
                        cudaStream_t s) {
  return dn::dense_linearize<double>(pb, lin_mode, traj, H, dv, s);
}
}  // namespace pit
