"""C ABI checks that need no GPU: the library builds and loads, exports every function
include/pit.h declares, and its host-only entry points (FP64 prior, exact initial state,
argument validation, workspace queries) agree with the oracle / reject bad input."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import prior, taylor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pit.h")


@pytest.fixture(scope="module")
def pit():
    import paper_2310_01145_gb300 as P
    from paper_2310_01145_gb300.build import LIB, build
    if not os.path.exists(LIB):
        build()
    P.load()
    return P


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(pit_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pit_prior", "pit_linearize", "pit_filter_scan", "pit_smooth_scan",
                     "pit_solve", "pit_solve_workspace_size", "pit_status_string",
                     "pit_last_error", "pit_eks_sequential"):
        assert required in names


def test_library_exports_every_declared_symbol(pit):
    lib = ctypes.CDLL(pit.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the Python binding wraps exactly these names
    assert set(pit.SIGNATURES) == set(declared_functions())


@pytest.mark.parametrize("q", [1, 2, 3, 5])
@pytest.mark.parametrize("h", [1e-4, 0.03, 0.9])
def test_host_prior_matches_oracle(pit, q, h):
    out = pit.pit_prior(q, h)
    Phi, Q = prior.iwp_1d(q, h)
    Pb, Qb = prior.preconditioned_1d(q)
    np.testing.assert_allclose(out["Phi"], Phi, rtol=1e-14, atol=0)
    np.testing.assert_allclose(out["Q"], Q, rtol=1e-13, atol=0)
    np.testing.assert_allclose(out["Phibar"], Pb, rtol=0, atol=0)
    np.testing.assert_allclose(out["sqrtQbar"] @ out["sqrtQbar"].T, Qb, rtol=1e-13)
    assert np.allclose(np.triu(out["sqrtQbar"], 1), 0)
    np.testing.assert_allclose(out["Tdiag"], prior.preconditioner_1d(q, h), rtol=1e-14)


@pytest.mark.parametrize("problem", [W.logistic(q=3), W.fitzhugh_nagumo(q=3), W.rigid_body(q=2),
                                     W.van_der_pol(q=3), W.lotka_volterra(q=2),
                                     W.affine([[0.0, 1.0], [-1.0, -0.1]], [0.3, 0.0], [1.0, 0.5], q=3),
                                     W.lorenz96(d=8, q=2)],
                         ids=lambda p: p.name)
def test_host_initial_state_matches_oracle(pit, problem):
    mu = pit.pit_init_state(pit.ode_from_problem(problem), problem.q, problem.y0)
    ref = taylor.initial_state(problem.kind, problem.params, problem.y0, problem.q)
    np.testing.assert_allclose(mu, ref, rtol=1e-13, atol=1e-15)


def test_validation_errors(pit):
    ode = pit.Ode(W.LOGISTIC, 1, np.array([3.0]))
    with pytest.raises(pit.PitError) as e:
        pit.pit_init_state(pit.Ode(W.LOGISTIC, 1, np.array([3.0, 1.0])), 2, [0.1])
    assert e.value.status == 1
    with pytest.raises(pit.PitError):
        pit.pit_init_state(ode, 0, [0.1])
    with pytest.raises(pit.PitError):
        pit.pit_init_state(ode, 2, [float("nan")])
    with pytest.raises(pit.PitError):
        pit.pit_init_state(pit.Ode(W.FITZHUGH_NAGUMO, 3, np.array([0.2, 0.2, 3.0])), 2, [0, 0, 0])
    with pytest.raises(pit.PitError):
        pit.pit_prior(0, 0.1)
    with pytest.raises(pit.PitError):
        pit.pit_prior(2, -1.0)
    lib = pit.load()
    c = ode.c()
    sz = ctypes.c_size_t(0)
    bad_grid = pit._Grid(1.0, 0.0, 10)
    st = lib.pit_solve_workspace_size(ctypes.byref(c), ctypes.byref(bad_grid), 2,
                                      ctypes.byref(pit.make_opts()), ctypes.byref(sz))
    assert st == 1 and b"t0 < t1" in lib.pit_last_error()
    good = pit._Grid(0.0, 1.0, 10)
    bad_opts = pit.make_opts()
    bad_opts.max_iter = 0
    assert lib.pit_solve_workspace_size(ctypes.byref(c), ctypes.byref(good), 2,
                                        ctypes.byref(bad_opts), ctypes.byref(sz)) == 1
    # d / q outside the compiled kernel set
    st = lib.pit_solve_workspace_size(ctypes.byref(c), ctypes.byref(good), 5,
                                      ctypes.byref(pit.make_opts()), ctypes.byref(sz))
    assert st == 8
    assert lib.pit_status_string(8) == b"configuration not compiled"


def test_workspace_queries_scale_with_n(pit):
    lib = pit.load()
    ode = pit.ode_from_problem(W.fitzhugh_nagumo(q=3))
    c = ode.c()
    sizes = []
    for N in (1, 1000, 2 ** 20):
        g = pit._Grid(0.0, 20.0, N)
        sz = ctypes.c_size_t(0)
        assert lib.pit_solve_workspace_size(ctypes.byref(c), ctypes.byref(g), 3,
                                            ctypes.byref(pit.make_opts(dtype="f32")),
                                            ctypes.byref(sz)) == 0
        sizes.append(sz.value)
    assert sizes[0] < sizes[1] < sizes[2]
    # dominated by the smoothing elements: (N+1) (D^2 + D) + (N+1) D^2 (covariance pass) floats
    D = 8
    assert sizes[2] >= (2 ** 20 + 1) * (2 * D * D + 3 * D) * 4
    sz = ctypes.c_size_t(0)
    assert lib.pit_filter_scan_workspace_size(1000, 8, 0, ctypes.byref(sz)) == 0 and sz.value > 0
    # D outside the lane-group set runs on the large-state kernels, up to 256
    assert lib.pit_filter_scan_workspace_size(1000, 5, 0, ctypes.byref(sz)) == 0 and sz.value > 0
    assert lib.pit_filter_scan_workspace_size(1000, 300, 0, ctypes.byref(sz)) == 8


def test_batched_validation_on_host(pit):
    """pit_solve_batched rejects mixed families and bad sizes before any device work."""
    import ctypes
    P = pit
    lv = P.Ode(W.LOTKA_VOLTERRA, 2, np.array([1.5, 1.0, 3.0, 1.0]))
    fhn = P.Ode(W.FITZHUGH_NAGUMO, 2, np.array([0.2, 0.2, 3.0]))
    opts = P.make_opts(dtype="f32")
    cs = (P._Ode * 2)(lv.c(), fhn.c())
    gs = (P._Grid * 2)(P._Grid(0.0, 1.0, 10), P._Grid(0.0, 1.0, 12))
    sz = ctypes.c_size_t(0)
    lib = P.load()
    assert lib.pit_solve_batched_workspace_size(2, cs, gs, 2, ctypes.byref(opts), ctypes.byref(sz)) == 1
    cs2 = (P._Ode * 2)(lv.c(), lv.c())
    assert lib.pit_solve_batched_workspace_size(2, cs2, gs, 2, ctypes.byref(opts), ctypes.byref(sz)) == 0
    assert sz.value > 0
    # workspace grows with the instances' lengths
    gs3 = (P._Grid * 2)(P._Grid(0.0, 1.0, 1000), P._Grid(0.0, 1.0, 12))
    sz3 = ctypes.c_size_t(0)
    assert lib.pit_solve_batched_workspace_size(2, cs2, gs3, 2, ctypes.byref(opts), ctypes.byref(sz3)) == 0
    assert sz3.value > sz.value
    assert lib.pit_solve_batched_workspace_size(0, cs2, gs, 2, ctypes.byref(opts), ctypes.byref(sz)) == 1
    bad = (P._Grid * 2)(P._Grid(0.0, 1.0, 10), P._Grid(1.0, 0.0, 12))
    assert lib.pit_solve_batched_workspace_size(2, cs2, bad, 2, ctypes.byref(opts), ctypes.byref(sz)) == 1
    assert b"instance 1" in lib.pit_last_error()
    # q = 4 has no compiled segmented kernels
    assert lib.pit_solve_batched_workspace_size(2, cs2, gs, 4, ctypes.byref(opts), ctypes.byref(sz)) == 8


def test_server_config_validation_on_host(pit):
    """pit_server_create rejects invalid configurations before touching the device."""
    import ctypes
    P = pit
    lib = P.load()
    cfg = P._ServerConfig()
    lib.pit_server_config_default(ctypes.byref(cfg))
    assert cfg.dtype == 0 and cfg.max_iter == 20 and cfg.max_requests == 1024
    h = ctypes.c_void_p()
    for field, bad in (("dtype", 7), ("max_iter", 0), ("max_points", 1), ("max_requests", 0),
                       ("hbm_budget_bytes", 1000), ("atol_objective", -1.0),
                       ("rtol_objective", float("nan"))):
        c = P._ServerConfig()
        lib.pit_server_config_default(ctypes.byref(c))
        setattr(c, field, bad)
        assert lib.pit_server_create(ctypes.byref(c), ctypes.byref(h)) == 1, field
        assert not h.value
    assert lib.pit_server_clock() > 0


def test_solve_grid_validation(pit):
    """pit_solve_grid checks its grid on the host: strictly increasing, finite points."""
    import ctypes
    lib = pit.load()
    p = W.lorenz96(d=8, N=10, q=2)
    c = pit.ode_from_problem(p).c()
    opts = pit.make_opts()
    sz = ctypes.c_size_t(0)
    good = np.linspace(0.0, 1.0, 11)
    st = lib.pit_solve_grid_workspace_size(ctypes.byref(c), good.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           10, 2, ctypes.byref(opts), ctypes.byref(sz))
    assert st == 0 and sz.value > 0
    for bad in (np.r_[0.0, 0.5, 0.5, np.linspace(0.6, 1.0, 8)],
                np.r_[np.linspace(0.0, 1.0, 10), np.nan]):
        bad = np.ascontiguousarray(bad)
        st = lib.pit_solve_grid_workspace_size(ctypes.byref(c), bad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                               10, 2, ctypes.byref(opts), ctypes.byref(sz))
        assert st == 1
        assert b"strictly increasing" in lib.pit_last_error()


def test_binding_fails_loudly_without_the_library():
    """No CPU fallback: the binding raises when libpit.so is absent (fresh process)."""
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import paper_2310_01145_gb300 as P\n"
            "try:\n"
            "    P.load('/nonexistent/libpit.so')\n"
            "except ImportError as e:\n"
            "    print('raised', e)\n") % ROOT
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert "raised" in out.stdout, out.stdout + out.stderr


def test_tensor_core_options_and_checks_on_host(pit):
    """pit_opts.tensor_cores is validated and sizes the FP64 large-state workspace (the trias'
    product buffer); the tensor-core checks and pit_linearize_approx reject bad arguments on the
    host, before any device work."""
    import ctypes
    lib = pit.load()
    p = W.lorenz96(d=64, N=100, q=2)
    c = pit.ode_from_problem(p).c()
    g = pit._Grid(p.t0, p.t1, p.N)
    sizes = {}
    for dt in ("f64", "f32"):
        for tcores in (0, 1):
            o = pit.make_opts(dtype=pit.PIT_F64 if dt == "f64" else pit.PIT_F32,
                              tensor_cores=tcores)
            sz = ctypes.c_size_t(0)
            assert lib.pit_solve_workspace_size(ctypes.byref(c), ctypes.byref(g), p.q,
                                                ctypes.byref(o), ctypes.byref(sz)) == 0
            sizes[dt, tcores] = sz.value
    assert sizes["f64", 1] > sizes["f64", 0]          # W and W T of the trias, per block
    assert sizes["f32", 1] == sizes["f32", 0]          # FP32 solves never use them
    bad = pit.make_opts(tensor_cores=3)
    sz = ctypes.c_size_t(0)
    assert lib.pit_solve_workspace_size(ctypes.byref(c), ctypes.byref(g), p.q, ctypes.byref(bad),
                                        ctypes.byref(sz)) == 1
    assert lib.pit_check_dgemm_tc(-1, 1, 1, 0, 0, 1.0, None, 1, None, 1, 0.0, None, 1, None,
                                  None) == 1
    assert lib.pit_check_dgemm_tc(4, 4, 4, 2, 0, 1.0, None, 4, None, 4, 0.0, None, 4, None,
                                  None) == 1
    assert lib.pit_check_tc_wait(-1, None, None) == 1
    assert lib.pit_linearize_approx(ctypes.byref(c), ctypes.byref(g), p.q, 0, 3, None, None,
                                    None, None) == 1
