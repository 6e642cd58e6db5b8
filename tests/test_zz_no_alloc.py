"""pit_solve_noalloc: the solver for callers that cannot allocate device memory.

Serving loops with a device memory budget fixed at start-up, plug-ins running under another
framework's memory manager and real-time hosts that forbid allocation after initialisation may
be unable to call cudaMalloc for a workspace.
pit_solve_noalloc runs the same solver on a fixed scratch array that the library holds in
device memory.  This test calls it through the C ABI twice in a row (the second call finds the
first call's leftovers in the shared array) and checks both results against pit_solve with a
caller-provided workspace, at the tolerances of the other GPU tests.  It sits in a file of its
own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import workloads as W  # noqa: E402


def _noalloc(pit, p, opts, mean, cov):
    lib = pit.load()
    ode = pit.ode_from_problem(p).c()
    grid = pit._Grid(p.t0, p.t1, p.N)
    y0 = np.ascontiguousarray(p.y0, dtype=np.float64)
    info = pit._Info()
    st = lib.pit_solve_noalloc(ctypes.byref(ode), ctypes.byref(grid), p.q, pit._dptr(y0),
                               ctypes.byref(opts), None, ctypes.c_void_p(mean.data_ptr()),
                               ctypes.c_void_p(cov.data_ptr()), ctypes.byref(info),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, info


@pytest.mark.parametrize("p,dtype,tol,extra", [
    (W.van_der_pol(N=1000, q=2), torch.float64, 1e-10, {}),
    (W.fitzhugh_nagumo(N=3000, q=3), torch.float32, 1e-5, {}),
    # coarse-grid start: the coarse solve's workspace is carved out of the same array
    (W.fitzhugh_nagumo(N=4000, q=3), torch.float64, 1e-10, {"init_coarse": 128}),
    # d > 3 goes to the large-state solver, whose scratch also lives in the array
    (W.lorenz96(d=8, N=1000, q=2), torch.float64, 1e-10, {"max_iter": 8}),
], ids=lambda x: getattr(x, "name", str(x)))
def test_noalloc_matches_workspace_solve_twice(p, dtype, tol, extra):
    import paper_2310_01145_gb300 as pit
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    pit.load()
    kw = dict(max_iter=60, atol_delta=1e-10)
    kw.update(extra)
    opts = pit.make_opts(dtype=dtype, **kw)
    ref = pit.pit_solve(pit.ode_from_problem(p), p.y0, p.t0, p.t1, p.N, p.q, opts)
    torch.cuda.synchronize()
    ref_mean = ref.mean.double().cpu().numpy()
    ref_cov = ref.sqrtcov.double().cpu().numpy()
    ref_c = np.einsum("nij,nkj->nik", ref_cov, ref_cov)
    for call in range(2):
        mean = torch.full((p.N + 1, p.D), float("nan"), dtype=dtype, device="cuda")
        cov = torch.full((p.N + 1, p.D, p.D), float("nan"), dtype=dtype, device="cuda")
        st, info = _noalloc(pit, p, opts, mean, cov)
        assert st == 0, pit.load().pit_last_error()
        assert info.iterations == ref.iterations
        m = mean.double().cpu().numpy()
        c = cov.double().cpu().numpy()
        assert np.max(np.abs(m - ref_mean)) <= tol * np.max(np.abs(ref_mean)), call
        cc = np.einsum("nij,nkj->nik", c, c)
        assert np.max(np.abs(cc - ref_c)) <= tol * np.max(np.abs(ref_c)), call


def test_noalloc_rejects_problem_larger_than_static_scratch():
    import paper_2310_01145_gb300 as pit
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    p = W.fitzhugh_nagumo(N=2 ** 20, q=3)
    opts = pit.make_opts(dtype=torch.float32)
    mean = torch.empty((1, 1), device="cuda")
    st, _ = _noalloc(pit, p, opts, mean, mean)
    assert st == 2
    assert b"static scratch array holds" in pit.load().pit_last_error()
