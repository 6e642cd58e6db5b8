"""Python binding of the GB300 parallel-in-time probabilistic ODE solver (libpit.so).

Argument marshalling only: every step of the solver runs in the CUDA library behind the C ABI
of include/pit.h.  PyTorch provides device memory and streams.  Function names mirror the C
entry points (pit_solve, pit_filter_scan, ...).  If libpit.so is missing this module raises on
first use -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpit.so")

PIT_F32, PIT_F64 = 0, 1

STATUS = {0: "PIT_OK", 1: "PIT_EINVAL", 2: "PIT_ENOMEM", 3: "PIT_ECUDA", 4: "PIT_ENOCONV",
          5: "PIT_ETIMEOUT", 6: "PIT_ENONFINITE", 7: "PIT_EINTERNAL", 8: "PIT_EUNSUPPORTED"}


class PitError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Ode(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("d", ctypes.c_int32),
                ("params", ctypes.POINTER(ctypes.c_double)), ("n_params", ctypes.c_int32)]


class _Grid(ctypes.Structure):
    _fields_ = [("t0", ctypes.c_double), ("t1", ctypes.c_double), ("N", ctypes.c_int64)]


class _Opts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("fixed_iters", ctypes.c_int32),
                ("atol_delta", ctypes.c_double), ("rtol_delta", ctypes.c_double),
                ("dtype", ctypes.c_int32), ("calibrate", ctypes.c_int32),
                ("want_cov", ctypes.c_int32), ("chain_len", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("linearization", ctypes.c_int32),
                ("objective", ctypes.c_int32), ("atol_objective", ctypes.c_double),
                ("rtol_objective", ctypes.c_double), ("init_coarse", ctypes.c_int32),
                ("scan", ctypes.c_int32), ("tensor_cores", ctypes.c_int32)]


class _Info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("last_delta", ctypes.c_double), ("sigma2", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("deltas", ctypes.c_double * 64),
                ("objective", ctypes.c_double), ("objectives", ctypes.c_double * 65)]


LINEARIZATIONS = {"ek1": 0, "diag": 1, "diagonal_ek1": 1, "ek0": 2}
_OPT_KEYS = ("dtype", "max_iter", "fixed_iters", "atol_delta", "rtol_delta", "calibrate",
             "want_cov", "chain_len", "variant", "linearization", "objective", "atol_objective",
             "rtol_objective", "init_coarse", "scan", "tensor_cores")


class _BatchInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("status", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("last_delta", ctypes.c_double), ("sigma2", ctypes.c_double),
                ("objective", ctypes.c_double)]


class _ServerConfig(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("atol_delta", ctypes.c_double), ("rtol_delta", ctypes.c_double),
                ("calibrate", ctypes.c_int32), ("chain_len", ctypes.c_int32),
                ("max_points", ctypes.c_int64), ("max_requests", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_size_t),
                ("atol_objective", ctypes.c_double), ("rtol_objective", ctypes.c_double)]


class _ServerResult(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_int64), ("tag", ctypes.c_uint64),
                ("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("last_delta", ctypes.c_double), ("sigma2", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("objective", ctypes.c_double)]


_lib = None

# exported symbols and their signatures (declared in include/pit.h)
_P, _I32, _I64, _SZ, _D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_double
_DP = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "pit_version": (ctypes.c_char_p, []),
    "pit_status_string": (ctypes.c_char_p, [_I32]),
    "pit_last_error": (ctypes.c_char_p, []),
    "pit_launch_count": (_I64, []),
    "pit_opts_default": (None, [ctypes.POINTER(_Opts)]),
    "pit_profile_enable": (None, [_I32]),
    "pit_profile_reset": (None, []),
    "pit_profile_read": (_I32, [_I32, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_int64)]),
    "pit_prior": (_I32, [_I32, _D, _DP, _DP, _DP, _DP, _DP]),
    "pit_init_state": (_I32, [ctypes.POINTER(_Ode), _I32, _DP, _DP]),
    "pit_linearize": (_I32, [ctypes.POINTER(_Ode), ctypes.POINTER(_Grid), _I32, _I32, _P, _P, _P, _P]),
    "pit_linearize_approx": (_I32, [ctypes.POINTER(_Ode), ctypes.POINTER(_Grid), _I32, _I32, _I32,
                                    _P, _P, _P, _P]),
    "pit_filter_scan_workspace_size": (_I32, [_I64, _I32, _I32, ctypes.POINTER(_SZ)]),
    "pit_filter_scan": (_I32, [_I64, _I32, _I32, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "pit_smooth_scan_workspace_size": (_I32, [_I64, _I32, _I32, _I32, ctypes.POINTER(_SZ)]),
    "pit_smooth_scan": (_I32, [_I64, _I32, _I32, _P, _P, _P, _I32, _P, _SZ, _P]),
    "pit_solve_workspace_size": (_I32, [ctypes.POINTER(_Ode), ctypes.POINTER(_Grid), _I32,
                                        ctypes.POINTER(_Opts), ctypes.POINTER(_SZ)]),
    "pit_solve": (_I32, [ctypes.POINTER(_Ode), ctypes.POINTER(_Grid), _I32, _DP,
                         ctypes.POINTER(_Opts), _P, _P, _P, ctypes.POINTER(_Info), _P, _SZ, _P]),
    "pit_solve_grid_workspace_size": (_I32, [ctypes.POINTER(_Ode), _DP, _I64, _I32,
                                             ctypes.POINTER(_Opts), ctypes.POINTER(_SZ)]),
    "pit_solve_grid": (_I32, [ctypes.POINTER(_Ode), _DP, _I64, _I32, _DP, ctypes.POINTER(_Opts),
                              _P, _P, _P, ctypes.POINTER(_Info), _P, _SZ, _P]),
    "pit_solve_noalloc": (_I32, [ctypes.POINTER(_Ode), ctypes.POINTER(_Grid), _I32, _DP,
                                 ctypes.POINTER(_Opts), _P, _P, _P, ctypes.POINTER(_Info), _P]),
    "pit_check_wait": (_I32, [_I64, ctypes.c_uint32, _P, _P]),
    "pit_check_dgemm_tc": (_I32, [_I32, _I32, _I32, _I32, _I32, ctypes.c_double, _P, _I32, _P,
                                  _I32, ctypes.c_double, _P, _I32, _P, _P]),
    "pit_check_tc_wait": (_I32, [_I64, _P, _P]),
    "pit_eks_workspace_size": (_I32, [ctypes.POINTER(_Ode), ctypes.POINTER(_Grid), _I32,
                                      ctypes.POINTER(_Opts), ctypes.POINTER(_SZ)]),
    "pit_eks_sequential": (_I32, [ctypes.POINTER(_Ode), ctypes.POINTER(_Grid), _I32, _DP,
                                  ctypes.POINTER(_Opts), _P, _P, ctypes.POINTER(_Info), _P, _SZ,
                                  _P]),
    "pit_solve_batched_workspace_size": (_I32, [_I32, ctypes.POINTER(_Ode),
                                                ctypes.POINTER(_Grid), _I32,
                                                ctypes.POINTER(_Opts), ctypes.POINTER(_SZ)]),
    "pit_solve_batched": (_I32, [_I32, ctypes.POINTER(_Ode), ctypes.POINTER(_Grid), _I32, _DP,
                                 ctypes.POINTER(_Opts), _P, _P, ctypes.POINTER(_BatchInfo), _P,
                                 _SZ, _P]),
    "pit_server_config_default": (None, [ctypes.POINTER(_ServerConfig)]),
    "pit_server_clock": (ctypes.c_double, []),
    "pit_server_create": (_I32, [ctypes.POINTER(_ServerConfig), ctypes.POINTER(ctypes.c_void_p)]),
    "pit_server_submit": (_I32, [_P, ctypes.POINTER(_Ode), ctypes.POINTER(_Grid), _I32, _DP, _P,
                                 ctypes.c_uint64, ctypes.POINTER(ctypes.c_int64)]),
    "pit_server_submit_cov": (_I32, [_P, ctypes.POINTER(_Ode), ctypes.POINTER(_Grid), _I32, _DP,
                                     _P, _P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int64)]),
    "pit_server_step": (_I32, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "pit_server_poll": (_I32, [_P, ctypes.POINTER(_ServerResult), _I32, ctypes.POINTER(_I32)]),
    "pit_server_stats": (_I32, [_P, ctypes.POINTER(_SZ), ctypes.POINTER(_I32)]),
    "pit_server_destroy": (None, [_P]),
}


def load(path: str = LIB_PATH):
    """Load libpit.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with paper_2310_01145_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st: int, what: str):
    if st != 0:
        raise PitError(st, f"{what}: {load().pit_last_error().decode()}")


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _tptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _dtype_code(dtype) -> int:
    import torch
    if dtype in (torch.float64, "f64", "float64", PIT_F64):
        return PIT_F64
    if dtype in (torch.float32, "f32", "float32", PIT_F32):
        return PIT_F32
    raise ValueError(f"unsupported dtype {dtype}")


def _torch_dtype(code: int):
    import torch
    return torch.float64 if code == PIT_F64 else torch.float32


@dataclasses.dataclass
class Ode:
    """Vector field description (see pit_ode_kind in pit.h)."""
    kind: int
    d: int
    params: np.ndarray

    def c(self):
        self._p = np.ascontiguousarray(self.params, dtype=np.float64)
        return _Ode(self.kind, self.d,
                    self._p.ctypes.data_as(_DP) if self._p.size else ctypes.cast(None, _DP),
                    int(self._p.size))


def ode_from_problem(problem) -> Ode:
    return Ode(problem.kind, problem.d, np.asarray(problem.params, dtype=np.float64))


def pit_opts_default() -> _Opts:
    o = _Opts()
    load().pit_opts_default(ctypes.byref(o))
    return o


def make_opts(dtype=PIT_F64, max_iter=20, fixed_iters=0, atol_delta=1e-10, rtol_delta=0.0,
              calibrate=True, want_cov=True, chain_len=0, variant=0, linearization="ek1",
              objective=False, atol_objective=0.0, rtol_objective=0.0,
              init_coarse=0, scan=0, tensor_cores=1) -> _Opts:
    o = pit_opts_default()
    o.max_iter, o.fixed_iters = int(max_iter), int(fixed_iters)
    o.atol_delta, o.rtol_delta = float(atol_delta), float(rtol_delta)
    o.dtype = _dtype_code(dtype)
    o.calibrate, o.want_cov, o.chain_len = int(bool(calibrate)), int(bool(want_cov)), int(chain_len)
    o.variant = int(variant)
    o.linearization = (LINEARIZATIONS[linearization] if isinstance(linearization, str)
                       else int(linearization))
    o.objective = int(bool(objective))
    o.atol_objective, o.rtol_objective = float(atol_objective), float(rtol_objective)
    o.init_coarse = int(init_coarse)
    o.scan = int(scan)
    o.tensor_cores = int(tensor_cores)
    return o


def pit_version() -> str:
    return load().pit_version().decode()


def pit_launch_count() -> int:
    return int(load().pit_launch_count())


def pit_profile_enable(on: bool = True) -> None:
    load().pit_profile_enable(1 if on else 0)


def pit_profile_reset() -> None:
    load().pit_profile_reset()


def pit_profile_read() -> dict:
    """{kernel class: (total device ms, launches)} accumulated since the last reset."""
    lib = load()
    n = lib.pit_profile_read(0, None, None, None)
    names = ctypes.create_string_buffer(32 * n)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    lib.pit_profile_read(n, names, ms, cnt)
    out = {}
    for i in range(n):
        nm = names.raw[32 * i: 32 * (i + 1)].split(b"\0")[0].decode()
        out[nm] = (float(ms[i]), int(cnt[i]))
    return out


def pit_prior(q: int, h: float):
    """Host FP64 prior blocks: dict of Phi, Q, Phibar, sqrtQbar ((q+1)^2) and Tdiag (q+1)."""
    K = q + 1
    out = {k: np.zeros((K, K)) for k in ("Phi", "Q", "Phibar", "sqrtQbar")}
    out["Tdiag"] = np.zeros(K)
    _check(load().pit_prior(q, h, _dptr(out["Phi"]), _dptr(out["Q"]), _dptr(out["Phibar"]),
                            _dptr(out["sqrtQbar"]), _dptr(out["Tdiag"])), "pit_prior")
    return out


def pit_init_state(ode: Ode, q: int, y0) -> np.ndarray:
    y = np.ascontiguousarray(y0, dtype=np.float64)
    mu0 = np.zeros(ode.d * (q + 1))
    c = ode.c()
    _check(load().pit_init_state(ctypes.byref(c), q, _dptr(y), _dptr(mu0)), "pit_init_state")
    return mu0


def pit_linearize(ode: Ode, t0: float, t1: float, N: int, q: int, traj, stream=None,
                  linearization="ek1"):
    """H (N, d, D) and dvec (N, d) at the device trajectory traj ((N+1, D)); `linearization`
    picks the exact Jacobian ("ek1"), its diagonal ("diag") or zero ("ek0")."""
    import torch
    code = _dtype_code(traj.dtype)
    D = ode.d * (q + 1)
    H = torch.empty((N, ode.d, D), dtype=traj.dtype, device=traj.device)
    dv = torch.empty((N, ode.d), dtype=traj.dtype, device=traj.device)
    c, gr = ode.c(), _Grid(t0, t1, N)
    mode = LINEARIZATIONS[linearization] if isinstance(linearization, str) else int(linearization)
    lib = load()
    if mode == 0:
        st = lib.pit_linearize(ctypes.byref(c), ctypes.byref(gr), q, code,
                               _tptr(traj.contiguous()), _tptr(H), _tptr(dv), _stream_ptr(stream))
    else:
        st = lib.pit_linearize_approx(ctypes.byref(c), ctypes.byref(gr), q, code, mode,
                                      _tptr(traj.contiguous()), _tptr(H), _tptr(dv),
                                      _stream_ptr(stream))
    _check(st, "pit_linearize")
    return H, dv


def _workspace(nbytes: int, device):
    import torch
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def pit_filter_scan(A, b, C, eta, J, stream=None):
    """In-place inclusive scan of filtering elements (tensors on one CUDA device)."""
    N, D = b.shape
    code = _dtype_code(b.dtype)
    sz = ctypes.c_size_t(0)
    _check(load().pit_filter_scan_workspace_size(N, D, code, ctypes.byref(sz)),
           "pit_filter_scan_workspace_size")
    ws = _workspace(sz.value, b.device)
    for t in (A, b, C, eta, J):
        assert t.is_contiguous() and t.dtype == b.dtype
    _check(load().pit_filter_scan(N, D, code, _tptr(A), _tptr(b), _tptr(C), _tptr(eta), _tptr(J),
                                  _tptr(ws), ws.numel(), _stream_ptr(stream)), "pit_filter_scan")
    return A, b, C, eta, J


def pit_smooth_scan(E, g, L=None, stream=None):
    """In-place reverse inclusive scan of smoothing elements."""
    N, D = g.shape
    code = _dtype_code(g.dtype)
    want_L = 1 if L is not None else 0
    sz = ctypes.c_size_t(0)
    _check(load().pit_smooth_scan_workspace_size(N, D, code, want_L, ctypes.byref(sz)),
           "pit_smooth_scan_workspace_size")
    ws = _workspace(sz.value, g.device)
    _check(load().pit_smooth_scan(N, D, code, _tptr(E), _tptr(g), _tptr(L), want_L, _tptr(ws),
                                  ws.numel(), _stream_ptr(stream)), "pit_smooth_scan")
    return E, g, L


@dataclasses.dataclass
class SolveResult:
    mean: "object"          # torch tensor (N+1, D)
    sqrtcov: "object"       # torch tensor (N+1, D, D) or None
    iterations: int
    converged: bool
    last_delta: float
    sigma2: float
    kernel_launches: int
    status: int


def _solve_like(fn_ws, fn_run, ode: Ode, y0, t0, t1, N, q, opts: _Opts, init_traj=None,
                device=None, stream=None, workspace=None, out=None, allow_noconv=True,
                is_eks=False):
    import torch
    device = device or torch.device("cuda", torch.cuda.current_device())
    c, gr = ode.c(), _Grid(float(t0), float(t1), int(N))
    sz = ctypes.c_size_t(0)
    _check(fn_ws(ctypes.byref(c), ctypes.byref(gr), int(q), ctypes.byref(opts), ctypes.byref(sz)),
           "workspace_size")
    if workspace is None or workspace.numel() < sz.value:
        workspace = _workspace(sz.value, device)
    tdt = _torch_dtype(opts.dtype)
    D = ode.d * (q + 1)
    if out is None:
        mean = torch.empty((N + 1, D), dtype=tdt, device=device)
        cov = torch.empty((N + 1, D, D), dtype=tdt, device=device) if opts.want_cov else None
    else:
        mean, cov = out
    y = np.ascontiguousarray(y0, dtype=np.float64)
    info = _Info()
    if is_eks:
        st = fn_run(ctypes.byref(c), ctypes.byref(gr), int(q), _dptr(y), ctypes.byref(opts),
                    _tptr(mean), _tptr(cov), ctypes.byref(info), _tptr(workspace),
                    workspace.numel(), _stream_ptr(stream))
    else:
        st = fn_run(ctypes.byref(c), ctypes.byref(gr), int(q), _dptr(y), ctypes.byref(opts),
                    _tptr(init_traj), _tptr(mean), _tptr(cov), ctypes.byref(info),
                    _tptr(workspace), workspace.numel(), _stream_ptr(stream))
    if not (st == 0 or (st == 4 and allow_noconv)):
        _check(st, "pit_solve")
    res = SolveResult(mean, cov, info.iterations, bool(info.converged), info.last_delta,
                      info.sigma2, int(info.kernel_launches), int(st))
    res.deltas = [float(info.deltas[i]) for i in range(min(info.iterations, 64))]
    res.objective = float(info.objective)
    res.objectives = [float(info.objectives[i]) for i in range(min(info.iterations, 64) + 1)]
    return res


def pit_solve(ode: Ode, y0, t0: float, t1: float, N: int, q: int, opts: Optional[_Opts] = None,
              init_traj=None, device=None, stream=None, workspace=None, out=None,
              allow_noconv=True) -> SolveResult:
    """ParaIEKS (Algorithm 2) through the C ABI; outputs are torch tensors on `device`."""
    lib = load()
    return _solve_like(lib.pit_solve_workspace_size, lib.pit_solve, ode, y0, t0, t1, N, q,
                       opts or make_opts(), init_traj, device, stream, workspace, out,
                       allow_noconv)


def pit_check_dgemm_tc(A, B, C, alpha=1.0, beta=0.0, trans_a=False, trans_b=False, stream=None):
    """C = alpha op(A) op(B) + beta C through the tensor-core digit product (FP64 torch tensors on
    the device, row-major and contiguous); returns C.  Raises PitError (status PIT_ETIMEOUT when a
    wait for the tensor cores gave up)."""
    import torch
    m, n = C.shape
    k = A.shape[0] if trans_a else A.shape[1]
    for t in (A, B, C):
        assert t.dtype == torch.float64 and t.is_contiguous()
    status = torch.zeros(2, dtype=torch.int32, device=C.device)
    _check(load().pit_check_dgemm_tc(m, n, k, int(trans_a), int(trans_b), float(alpha), _tptr(A),
                                     max(1, A.shape[1]), _tptr(B), max(1, B.shape[1]),
                                     float(beta), _tptr(C), max(1, C.shape[1]), _tptr(status),
                                     _stream_ptr(stream)),
           "pit_check_dgemm_tc")
    return C


def pit_check_tc_wait(wait_ns: int, device="cuda:0", stream=None) -> int:
    """Bounded wait of the tensor-core product on an mbarrier nothing arrives on; returns the
    status (PIT_ETIMEOUT: it gave up and set the timeout bit)."""
    import torch
    status = torch.zeros(2, dtype=torch.int32, device=device)
    return int(load().pit_check_tc_wait(int(wait_ns), _tptr(status), _stream_ptr(stream)))


def pit_check_wait(poll_limit: int, target: int, words, stream=None) -> int:
    """Run the bounded cross-block wait once on words[0] (a torch int32 tensor of >= 3 entries
    on the device); returns the status (PIT_OK: flag seen, PIT_ETIMEOUT: gave up)."""
    return int(load().pit_check_wait(int(poll_limit), int(target), _tptr(words),
                                     _stream_ptr(stream)))


def pit_eks_sequential(ode: Ode, y0, t0: float, t1: float, N: int, q: int,
                       opts: Optional[_Opts] = None, device=None, stream=None,
                       workspace=None, out=None) -> SolveResult:
    """Sequential EKS with local linearisation (GPU baseline) through the C ABI."""
    lib = load()
    return _solve_like(lib.pit_eks_workspace_size, lib.pit_eks_sequential, ode, y0, t0, t1, N,
                       q, opts or make_opts(), None, device, stream, workspace, out, True,
                       is_eks=True)


def pit_solve_grid(ode: Ode, y0, ts, q: int, opts: Optional[_Opts] = None, init_traj=None,
                   device=None, stream=None, workspace=None, out=None,
                   allow_noconv=True) -> SolveResult:
    """ParaIEKS on the non-uniform grid ts (N+1 increasing points) through the C ABI."""
    import torch
    lib = load()
    opts = opts or make_opts()
    t = np.ascontiguousarray(ts, dtype=np.float64)
    N = t.size - 1
    device = device or torch.device("cuda", torch.cuda.current_device())
    c = ode.c()
    sz = ctypes.c_size_t(0)
    _check(lib.pit_solve_grid_workspace_size(ctypes.byref(c), _dptr(t), N, int(q),
                                             ctypes.byref(opts), ctypes.byref(sz)),
           "workspace_size")
    if workspace is None or workspace.numel() < sz.value:
        workspace = _workspace(sz.value, device)
    tdt = _torch_dtype(opts.dtype)
    D = ode.d * (q + 1)
    if out is None:
        mean = torch.empty((N + 1, D), dtype=tdt, device=device)
        cov = torch.empty((N + 1, D, D), dtype=tdt, device=device) if opts.want_cov else None
    else:
        mean, cov = out
    y = np.ascontiguousarray(y0, dtype=np.float64)
    info = _Info()
    st = lib.pit_solve_grid(ctypes.byref(c), _dptr(t), N, int(q), _dptr(y), ctypes.byref(opts),
                            _tptr(init_traj), _tptr(mean), _tptr(cov), ctypes.byref(info),
                            _tptr(workspace), workspace.numel(), _stream_ptr(stream))
    if not (st == 0 or (st == 4 and allow_noconv)):
        _check(st, "pit_solve_grid")
    res = SolveResult(mean, cov, info.iterations, bool(info.converged), info.last_delta,
                      info.sigma2, int(info.kernel_launches), int(st))
    res.deltas = [float(info.deltas[i]) for i in range(min(info.iterations, 64))]
    return res


def solve_problem(problem, **kw) -> SolveResult:
    """Convenience wrapper for a workloads.Problem (a non-uniform grid goes to pit_solve_grid)."""
    opts = kw.pop("opts", None) or make_opts(**{k: kw.pop(k) for k in list(kw)
                                                if k in _OPT_KEYS})
    if getattr(problem, "ts", None) is not None:
        return pit_solve_grid(ode_from_problem(problem), problem.y0, problem.ts, problem.q, opts,
                              **kw)
    return pit_solve(ode_from_problem(problem), problem.y0, problem.t0, problem.t1, problem.N,
                     problem.q, opts, **kw)


@dataclasses.dataclass
class BatchResult:
    mean: "object"          # torch tensor (sum_i (N_i + 1), D)
    sqrtcov: "object"       # torch tensor (sum_i (N_i + 1), D, D) or None
    rows: np.ndarray        # first row of each instance
    iterations: np.ndarray
    converged: np.ndarray
    status: np.ndarray      # per-instance pit_status
    last_delta: np.ndarray
    sigma2: np.ndarray
    call_status: int
    objective: Optional[np.ndarray] = None   # V of each instance's last iterate, when evaluated

    def instance(self, i: int):
        """(mean, sqrtcov) views of instance i."""
        a, b = int(self.rows[i]), int(self.rows[i + 1])
        return self.mean[a:b], (self.sqrtcov[a:b] if self.sqrtcov is not None else None)


def pit_solve_batched(odes: Sequence[Ode], y0s, grids: Sequence[tuple], q: int,
                      opts: Optional[_Opts] = None, device=None, stream=None, workspace=None,
                      allow_noconv=True, allow_diverged=False) -> BatchResult:
    """Batched ParaIEKS over instances of one ODE family (see pit_solve_batched in pit.h).
    grids: (t0, t1, N) per instance; y0s: (B, d)."""
    import torch
    lib = load()
    opts = opts or make_opts()
    device = device or torch.device("cuda", torch.cuda.current_device())
    B = len(odes)
    cs = (_Ode * B)(*[o.c() for o in odes])
    keep = [o._p for o in odes]  # parameter arrays referenced by cs
    gs = (_Grid * B)(*[_Grid(float(t0), float(t1), int(N)) for (t0, t1, N) in grids])
    sz = ctypes.c_size_t(0)
    _check(lib.pit_solve_batched_workspace_size(B, cs, gs, int(q), ctypes.byref(opts),
                                                ctypes.byref(sz)), "batched workspace_size")
    if workspace is None or workspace.numel() < sz.value:
        workspace = _workspace(sz.value, device)
    d = odes[0].d
    D = d * (q + 1)
    Ns = np.array([int(g[2]) for g in grids], dtype=np.int64)
    rows = np.concatenate([[0], np.cumsum(Ns + 1)])
    M = int(rows[-1])
    tdt = _torch_dtype(opts.dtype)
    mean = torch.empty((M, D), dtype=tdt, device=device)
    cov = torch.empty((M, D, D), dtype=tdt, device=device) if opts.want_cov else None
    y = np.ascontiguousarray(np.asarray(y0s, dtype=np.float64).reshape(B, d))
    info = (_BatchInfo * B)()
    st = lib.pit_solve_batched(B, cs, gs, int(q), _dptr(y), ctypes.byref(opts), _tptr(mean),
                               _tptr(cov), info, _tptr(workspace), workspace.numel(),
                               _stream_ptr(stream))
    del keep
    if not (st == 0 or (st == 4 and allow_noconv) or (st == 6 and allow_diverged)):
        _check(st, "pit_solve_batched")
    return BatchResult(mean, cov, rows,
                       np.array([info[i].iterations for i in range(B)]),
                       np.array([bool(info[i].converged) for i in range(B)]),
                       np.array([info[i].status for i in range(B)]),
                       np.array([info[i].last_delta for i in range(B)]),
                       np.array([info[i].sigma2 for i in range(B)]), int(st),
                       np.array([info[i].objective for i in range(B)]))


def solve_problems_batched(problems, **kw) -> BatchResult:
    """Batched solve of workloads.Problem instances (same family, d and q)."""
    opts = kw.pop("opts", None) or make_opts(**{k: kw.pop(k) for k in list(kw)
                                                if k in _OPT_KEYS})
    q = problems[0].q
    return pit_solve_batched([ode_from_problem(p) for p in problems],
                             np.stack([np.asarray(p.y0, dtype=np.float64) for p in problems]),
                             [(p.t0, p.t1, p.N) for p in problems], q, opts, **kw)


class Server:
    """Solve server with continuous batching (pit_server_* in pit.h).  submit() queues a
    workloads.Problem and returns its request id; step() admits, iterates once and retires;
    poll() returns the retired requests as dicts (with their device means)."""

    def __init__(self, dtype="f32", max_iter=20, atol_delta=1e-10, rtol_delta=1e-6,
                 calibrate=True, chain_len=0, max_points=1 << 22, max_requests=1024,
                 hbm_budget_bytes=8 << 30, device=None, atol_objective=0.0,
                 rtol_objective=0.0):
        import torch
        lib = load()
        cfg = _ServerConfig()
        lib.pit_server_config_default(ctypes.byref(cfg))
        cfg.dtype = _dtype_code(dtype)
        cfg.max_iter, cfg.atol_delta, cfg.rtol_delta = int(max_iter), float(atol_delta), float(rtol_delta)
        cfg.calibrate, cfg.chain_len = int(bool(calibrate)), int(chain_len)
        cfg.max_points, cfg.max_requests = int(max_points), int(max_requests)
        cfg.hbm_budget_bytes = int(hbm_budget_bytes)
        cfg.atol_objective, cfg.rtol_objective = float(atol_objective), float(rtol_objective)
        self.cfg = cfg
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self._h = ctypes.c_void_p()
        _check(lib.pit_server_create(ctypes.byref(cfg), ctypes.byref(self._h)), "pit_server_create")
        self._outs = {}
        self._covs = {}

    @staticmethod
    def clock() -> float:
        return float(load().pit_server_clock())

    def submit(self, problem, tag: int = 0, out=None, cov: bool = False) -> int:
        """Queue a request; cov=True also delivers its square-root covariances
        (pit_server_submit_cov), returned by poll() as "sqrtcov"."""
        import torch
        ode = ode_from_problem(problem)
        c = ode.c()
        gr = _Grid(float(problem.t0), float(problem.t1), int(problem.N))
        y = np.ascontiguousarray(problem.y0, dtype=np.float64)
        dt = _torch_dtype(self.cfg.dtype)
        if out is None:
            out = torch.empty((problem.N + 1, problem.D), dtype=dt, device=self.device)
        rid = ctypes.c_int64(0)
        if cov:
            S = torch.empty((problem.N + 1, problem.D, problem.D), dtype=dt, device=self.device)
            _check(load().pit_server_submit_cov(self._h, ctypes.byref(c), ctypes.byref(gr),
                                                int(problem.q), _dptr(y), _tptr(out), _tptr(S),
                                                int(tag), ctypes.byref(rid)),
                   "pit_server_submit_cov")
            self._covs[rid.value] = S
        else:
            _check(load().pit_server_submit(self._h, ctypes.byref(c), ctypes.byref(gr),
                                            int(problem.q), _dptr(y), _tptr(out), int(tag),
                                            ctypes.byref(rid)),
                   "pit_server_submit")
        self._outs[rid.value] = out
        return rid.value

    def step(self):
        fl, qu = _I32(0), _I32(0)
        _check(load().pit_server_step(self._h, ctypes.byref(fl), ctypes.byref(qu)),
               "pit_server_step")
        return fl.value, qu.value

    def poll(self, max_results: int = 4096):
        buf = (_ServerResult * max_results)()
        n = _I32(0)
        _check(load().pit_server_poll(self._h, buf, max_results, ctypes.byref(n)), "pit_server_poll")
        out = []
        for i in range(n.value):
            r = buf[i]
            out.append({"request_id": r.request_id, "tag": r.tag, "status": r.status,
                        "iterations": r.iterations, "last_delta": r.last_delta,
                        "sigma2": r.sigma2, "t_submit": r.t_submit, "t_admit": r.t_admit,
                        "t_done": r.t_done, "objective": r.objective,
                        "mean": self._outs.pop(r.request_id),
                        "sqrtcov": self._covs.pop(r.request_id, None)})
        return out

    def stats(self):
        used, ncls = _SZ(0), _I32(0)
        _check(load().pit_server_stats(self._h, ctypes.byref(used), ctypes.byref(ncls)),
               "pit_server_stats")
        return {"pool_used": used.value, "classes": ncls.value}

    def close(self):
        if self._h:
            load().pit_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._outs.clear()
            self._covs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
