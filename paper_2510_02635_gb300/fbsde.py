"""Thin Python binding of the C ABI in ``include/fbsde.h`` (ctypes).

Argument marshalling only: every step of the method runs in the CUDA library
``_build/libfbsde_gb300.so``.  Torch tensors supply device memory and the current
CUDA stream.  There is no CPU fallback: if the library is missing or no GPU is
present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfbsde_gb300.so")

FBSDE_OK, FBSDE_ERR_ARG, FBSDE_ERR_WORKSPACE, FBSDE_ERR_CUDA = 0, 1, 2, 3
FBSDE_ERR_NEWTON, FBSDE_ERR_CG, FBSDE_ERR_TIMEOUT, FBSDE_ERR_NONFINITE = 4, 5, 6, 7
FBSDE_FP32, FBSDE_FP64 = 0, 1
FBSDE_MAX_D = 16384

KINDS = {
    "ac_manufactured": 0,
    "logistic_grad": 1,
    "hjb_logquad": 2,
    "affine_test": 3,
    "cubic_test": 4,
    "ac_doublewell": 5,
    "cos_linear_test": 6,
    "drift_ac": 7,
    "drift_quad": 8,
}
PRECISIONS = {"fp32": FBSDE_FP32, "fp64": FBSDE_FP64}


class fbsde_problem(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("d", C.c_int32), ("N", C.c_int32), ("precision", C.c_int32),
        ("M", C.c_int64), ("sigma", C.c_double), ("T", C.c_double), ("theta", C.c_void_p),
        ("A", C.c_double), ("c0", C.c_double), ("c1", C.c_double), ("c2", C.c_double),
        ("c3", C.c_double), ("h", C.c_double), ("ridge_rel", C.c_double),
        ("cg_tol", C.c_double), ("cg_max_iter", C.c_int32), ("newton_max_iter", C.c_int32),
        ("newton_tol", C.c_double), ("ctas", C.c_int32), ("reserved", C.c_int32),
        ("mu0", C.c_double), ("mu1", C.c_double), ("sig1", C.c_double),
    ]


class fbsde_trace(C.Structure):
    _fields_ = [("alpha", C.c_void_p), ("alpha_x", C.c_void_p), ("cg_iters", C.c_void_p),
                ("newton_iters", C.c_void_p), ("x_N", C.c_void_p), ("y_N", C.c_void_p)]


class fbsde_instance(C.Structure):
    _fields_ = [("problem", fbsde_problem), ("Q", C.c_int32), ("solve_index0", C.c_uint32),
                ("seed", C.c_uint64), ("x0", C.c_void_p), ("u0", C.c_void_p),
                ("grad_u0", C.c_void_p)]


class fbsde_kernel_stats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("timed", C.c_int64), ("total_ms", C.c_double)]


class fbsde_diag(C.Structure):
    _fields_ = [("status", C.c_int32), ("solves_cg_exhausted", C.c_int32),
                ("max_newton_iters", C.c_int32), ("cg_iters_total", C.c_int32)]


EXPORTS = ["fbsde_workspace_bytes", "fbsde_solve", "fbsde_solve_host",
           "fbsde_host_staging_bytes", "fbsde_diagnostics", "fbsde_philox4x32_10",
           "fbsde_normals", "fbsde_status_string", "fbsde_abi_version",
           "fbsde_profile_start", "fbsde_profile_select", "fbsde_profile_stop", "fbsde_kernel_name",
           "fbsde_solve_noalloc", "fbsde_adjoint", "fbsde_adjoint_workspace_bytes",
           "fbsde_plan_workspace_bytes", "fbsde_plan_create", "fbsde_plan_launch",
           "fbsde_plan_diagnostics", "fbsde_plan_destroy", "fbsde_plan_instance_diagnostics",
           "fbsde_anchored_workspace_bytes", "fbsde_solve_anchored", "fbsde_solve_batch",
           "fbsde_solve_batch_direct", "fbsde_anchored_diagnostics", "fbsde_check_bounded_wait"]
FBSDE_NOALLOC_MAX_BYTES = 64 << 20
FBSDE_NUM_KERNELS = 13
FBSDE_MAX_D_FP64 = 10240
FBSDE_BATCH_DIRECT_MAX_D = 128
FBSDE_PROFILED_EAGER_PASSES = 48   # the header constant of the same name

_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing: run "
                               "`python -c 'import __graft_entry__ as g; g.build()'` first")
        lib = C.CDLL(path)
        P, V, I32, I64, U32, U64, SZ = (C.POINTER(fbsde_problem), C.c_void_p, C.c_int32,
                                        C.c_int64, C.c_uint32, C.c_uint64, C.c_size_t)
        lib.fbsde_workspace_bytes.argtypes = [P, I32]
        lib.fbsde_workspace_bytes.restype = SZ
        lib.fbsde_solve.argtypes = [P, I32, V, U64, U32, V, V, C.POINTER(fbsde_trace), V, SZ, V]
        lib.fbsde_solve.restype = C.c_int
        lib.fbsde_solve_host.argtypes = [P, I32, V, U64, U32, V, V, V, SZ, V]
        lib.fbsde_solve_host.restype = C.c_int
        lib.fbsde_host_staging_bytes.argtypes = [P, I32]
        lib.fbsde_host_staging_bytes.restype = SZ
        lib.fbsde_diagnostics.argtypes = [P, I32, V, C.POINTER(fbsde_diag), V]
        lib.fbsde_diagnostics.restype = C.c_int
        lib.fbsde_philox4x32_10.argtypes = [V, V, V, I64, V]
        lib.fbsde_philox4x32_10.restype = C.c_int
        lib.fbsde_normals.argtypes = [U64, U32, U32, U32, I32, I32, I32, V, V]
        lib.fbsde_normals.restype = C.c_int
        lib.fbsde_status_string.argtypes = [C.c_int]
        lib.fbsde_status_string.restype = C.c_char_p
        lib.fbsde_profile_start.argtypes = [I32]
        lib.fbsde_profile_start.restype = C.c_int
        lib.fbsde_profile_select.argtypes = [C.c_uint32]
        lib.fbsde_profile_select.restype = C.c_int
        lib.fbsde_profile_stop.argtypes = [C.POINTER(fbsde_kernel_stats)]
        lib.fbsde_profile_stop.restype = C.c_int
        lib.fbsde_kernel_name.argtypes = [C.c_int]
        lib.fbsde_kernel_name.restype = C.c_char_p
        lib.fbsde_solve_noalloc.argtypes = [P, I32, V, U64, U32, V, V, V]
        lib.fbsde_solve_noalloc.restype = C.c_int
        lib.fbsde_anchored_workspace_bytes.argtypes = [P]
        lib.fbsde_anchored_workspace_bytes.restype = SZ
        lib.fbsde_solve_anchored.argtypes = [P, I32, V, U64, U32, V, V, V, SZ, V]
        lib.fbsde_solve_anchored.restype = C.c_int
        lib.fbsde_solve_batch.argtypes = [P, C.c_int64, I32, V, U64, U32, V, V, V, SZ, V]
        lib.fbsde_solve_batch.restype = C.c_int
        lib.fbsde_solve_batch_direct.argtypes = [P, C.c_int64, I32, V, U64, U32, V, V, V, SZ, V]
        lib.fbsde_solve_batch_direct.restype = C.c_int
        lib.fbsde_anchored_diagnostics.argtypes = [P, V, C.POINTER(fbsde_diag), V]
        lib.fbsde_anchored_diagnostics.restype = C.c_int
        lib.fbsde_check_bounded_wait.argtypes = [I64, V, C.POINTER(C.c_int64), V]
        lib.fbsde_check_bounded_wait.restype = C.c_int
        lib.fbsde_adjoint_workspace_bytes.argtypes = [P, I32]
        lib.fbsde_adjoint_workspace_bytes.restype = SZ
        lib.fbsde_adjoint.argtypes = [P, I32, V, U64, U32, V, V, V, V, V, V, SZ, V]
        lib.fbsde_adjoint.restype = C.c_int
        IP = C.POINTER(fbsde_instance)
        lib.fbsde_plan_workspace_bytes.argtypes = [I32, IP]
        lib.fbsde_plan_workspace_bytes.restype = SZ
        lib.fbsde_plan_create.argtypes = [C.POINTER(C.c_void_p), I32, IP, I32, V, SZ]
        lib.fbsde_plan_create.restype = C.c_int
        lib.fbsde_plan_launch.argtypes = [V, V]
        lib.fbsde_plan_launch.restype = C.c_int
        lib.fbsde_plan_diagnostics.argtypes = [V, C.POINTER(fbsde_diag), V]
        lib.fbsde_plan_diagnostics.restype = C.c_int
        lib.fbsde_plan_instance_diagnostics.argtypes = [V, I32, C.POINTER(fbsde_diag), V]
        lib.fbsde_plan_instance_diagnostics.restype = C.c_int
        lib.fbsde_plan_destroy.argtypes = [V]
        lib.fbsde_plan_destroy.restype = None
        lib.fbsde_abi_version.argtypes = []
        lib.fbsde_abi_version.restype = C.c_int
        _lib = lib
        return lib


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_problem(kind: str, d: int, N: int, M: int, sigma: float, T: float,
                 precision: str = "fp32", theta=None, A: float = 0.0, c0: float = 0.0,
                 c1: float = 0.0, c2: float = 0.0, c3: float = 0.0, h: float = 2.0,
                 ridge_rel: float = 1e-3, cg_tol: float = 1e-6, cg_max_iter: int = 0,
                 newton_max_iter: int = 0, newton_tol: float = 0.0,
                 ctas: int = 0, mu0: float = 0.0, mu1: float = 0.0,
                 sig1: float = 0.0) -> fbsde_problem:
    """Fill the C problem struct; theta is a device tensor (or host array for the
    host-buffer entry point) whose storage must outlive the call.  mu0, mu1, sig1: the
    forward SDE's drift mu0 + mu1 x_i and diffusion sigma + sig1 x_i (zero: driftless)."""
    return fbsde_problem(KINDS[kind], int(d), int(N), PRECISIONS[precision], int(M),
                         float(sigma), float(T), _ptr(theta), float(A), float(c0), float(c1),
                         float(c2), float(c3), float(h), float(ridge_rel), float(cg_tol),
                         int(cg_max_iter), int(newton_max_iter), float(newton_tol), int(ctas),
                         0, float(mu0), float(mu1), float(sig1))


def fbsde_workspace_bytes(problem: fbsde_problem, Q: int) -> int:
    return int(load_library().fbsde_workspace_bytes(C.byref(problem), int(Q)))


def fbsde_host_staging_bytes(problem: fbsde_problem, Q: int) -> int:
    return int(load_library().fbsde_host_staging_bytes(C.byref(problem), int(Q)))


def fbsde_solve(problem: fbsde_problem, Q: int, x0, seed: int, solve_index0: int, u0,
                grad_u0, workspace, trace: fbsde_trace | None = None, stream=None) -> int:
    """x0 [Q, d], u0 [Q], grad_u0 [Q, d] (or None) and workspace are CUDA tensors."""
    return int(load_library().fbsde_solve(
        C.byref(problem), int(Q), _ptr(x0), int(seed), int(solve_index0), _ptr(u0),
        _ptr(grad_u0), C.byref(trace) if trace is not None else None, _ptr(workspace),
        workspace.numel() * workspace.element_size(), _stream(stream)))


def fbsde_solve_host(problem: fbsde_problem, Q: int, x0: np.ndarray, seed: int,
                     solve_index0: int, u0: np.ndarray, grad_u0: np.ndarray | None, workspace,
                     stream=None) -> int:
    """Host-buffer variant: x0, u0, grad_u0 (and problem.theta) are host arrays."""
    for a in (x0, u0, grad_u0):
        if a is not None:
            assert a.dtype == np.float64 and a.flags.c_contiguous
    return int(load_library().fbsde_solve_host(
        C.byref(problem), int(Q), _ptr(x0), int(seed), int(solve_index0), _ptr(u0),
        _ptr(grad_u0), _ptr(workspace), workspace.numel() * workspace.element_size(),
        _stream(stream)))


def fbsde_solve_noalloc(problem: fbsde_problem, Q: int, x0, seed: int, solve_index0: int,
                        u0, grad_u0, stream=None) -> int:
    """The solve on the library's built-in scratch array (no workspace argument)."""
    return int(load_library().fbsde_solve_noalloc(
        C.byref(problem), int(Q), _ptr(x0), int(seed), int(solve_index0), _ptr(u0),
        _ptr(grad_u0), _stream(stream)))


def fbsde_anchored_workspace_bytes(problem: fbsde_problem) -> int:
    return int(load_library().fbsde_anchored_workspace_bytes(C.byref(problem)))


def fbsde_solve_anchored(problem: fbsde_problem, Q: int, x0, seed: int, solve_index0: int,
                         u0, grad_u0, workspace, stream=None) -> int:
    """Algorithm 1 with one regression per particle anchor (asynchronous on the stream;
    the device status through fbsde_anchored_diagnostics)."""
    return int(load_library().fbsde_solve_anchored(
        C.byref(problem), int(Q), _ptr(x0), int(seed), int(solve_index0), _ptr(u0),
        _ptr(grad_u0), _ptr(workspace), workspace.numel() * workspace.element_size(),
        _stream(stream)))


def fbsde_solve_batch(problem: fbsde_problem, K: int, Q: int, x0, seed: int, solve_index0: int,
                      u0, grad_u0, workspace, stream=None) -> int:
    """Algorithm 1 per anchor over a batch of K particles (cyclic window; asynchronous)."""
    return int(load_library().fbsde_solve_batch(
        C.byref(problem), int(K), int(Q), _ptr(x0), int(seed), int(solve_index0), _ptr(u0),
        _ptr(grad_u0), _ptr(workspace), workspace.numel() * workspace.element_size(),
        _stream(stream)))


def fbsde_solve_batch_direct(problem: fbsde_problem, K: int, Q: int, x0, seed: int,
                             solve_index0: int, u0, grad_u0, workspace, stream=None) -> int:
    """The batch reading with each anchor's regression solved directly (L D L^T of its
    operator; d <= FBSDE_BATCH_DIRECT_MAX_D; asynchronous)."""
    return int(load_library().fbsde_solve_batch_direct(
        C.byref(problem), int(K), int(Q), _ptr(x0), int(seed), int(solve_index0), _ptr(u0),
        _ptr(grad_u0), _ptr(workspace), workspace.numel() * workspace.element_size(),
        _stream(stream)))


def fbsde_anchored_diagnostics(problem: fbsde_problem, workspace, stream=None) -> fbsde_diag:
    out = fbsde_diag()
    check(load_library().fbsde_anchored_diagnostics(C.byref(problem), _ptr(workspace),
                                                    C.byref(out), _stream(stream)),
          "fbsde_anchored_diagnostics")
    return out


def solve_anchored(problem: fbsde_problem, x0, seed: int, solve_index0: int = 0,
                   K: int | None = None, direct: bool = False) -> dict:
    """Per-anchor solve of the CUDA tensor x0 [Q, d]; returns u0 [Q], grad [Q, d], status.
    With K, each anchor's regression runs over its batch of K particles (fbsde_solve_batch),
    or, with direct, is solved directly (fbsde_solve_batch_direct)."""
    import torch
    Q = x0.shape[0]
    nbytes = fbsde_anchored_workspace_bytes(problem)
    if nbytes == 0:
        raise ValueError("invalid problem for the per-anchor solve")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=x0.device)
    u = torch.empty(Q, dtype=torch.float64, device=x0.device)
    g = torch.empty(Q, problem.d, dtype=torch.float64, device=x0.device)
    if K is None:
        check(fbsde_solve_anchored(problem, Q, x0, seed, solve_index0, u, g, ws),
              "fbsde_solve_anchored")
    elif direct:
        check(fbsde_solve_batch_direct(problem, K, Q, x0, seed, solve_index0, u, g, ws),
              "fbsde_solve_batch_direct")
    else:
        check(fbsde_solve_batch(problem, K, Q, x0, seed, solve_index0, u, g, ws),
              "fbsde_solve_batch")
    dg = fbsde_anchored_diagnostics(problem, ws)
    return {"u0": u, "grad": g, "status": int(dg.status), "cg_passes": int(dg.cg_iters_total)}


def fbsde_adjoint_workspace_bytes(problem: fbsde_problem, Q: int) -> int:
    return int(load_library().fbsde_adjoint_workspace_bytes(C.byref(problem), int(Q)))


def fbsde_adjoint(problem: fbsde_problem, Q: int, x0, seed: int, solve_index0: int, u0_bar,
                  u0, grad_u0, x0_bar, theta_bar, workspace, stream=None) -> int:
    """Reverse sweep: x0_bar = u0_bar du/dx0, theta_bar = sum_q u0_bar_q du_q/dtheta."""
    return int(load_library().fbsde_adjoint(
        C.byref(problem), int(Q), _ptr(x0), int(seed), int(solve_index0), _ptr(u0_bar),
        _ptr(u0), _ptr(grad_u0), _ptr(x0_bar), _ptr(theta_bar), _ptr(workspace),
        workspace.numel() * workspace.element_size(), _stream(stream)))


def fbsde_diagnostics(problem: fbsde_problem, Q: int, workspace, stream=None) -> fbsde_diag:
    out = fbsde_diag()
    st = load_library().fbsde_diagnostics(C.byref(problem), int(Q), _ptr(workspace),
                                          C.byref(out), _stream(stream))
    if st != FBSDE_OK:
        raise RuntimeError(f"fbsde_diagnostics: {fbsde_status_string(st)}")
    return out


def fbsde_philox4x32_10(ctr, key, out, stream=None) -> int:
    """ctr [n, 4], key [2], out [n, 4]: uint32 data in int32 CUDA tensors."""
    n = ctr.shape[0]
    return int(load_library().fbsde_philox4x32_10(_ptr(ctr), _ptr(key), _ptr(out), n,
                                                  _stream(stream)))


def fbsde_normals(seed: int, s: int, k: int, j0: int, nj: int, d: int, precision: str, out,
                  stream=None) -> int:
    return int(load_library().fbsde_normals(int(seed), int(s), int(k), int(j0), int(nj),
                                            int(d), PRECISIONS[precision], _ptr(out),
                                            _stream(stream)))


def fbsde_check_bounded_wait(limit_ns: int, scratch, stream=None) -> tuple[int, int]:
    """(status, waited nanoseconds) of one bounded wait on an mbarrier that nothing
    arrives on; FBSDE_ERR_TIMEOUT is the expected status."""
    waited = C.c_int64(0)
    st = load_library().fbsde_check_bounded_wait(int(limit_ns), _ptr(scratch), C.byref(waited),
                                                 _stream(stream))
    return int(st), int(waited.value)


def fbsde_status_string(status: int) -> str:
    return load_library().fbsde_status_string(int(status)).decode()


def fbsde_profile_start(max_timed_launches: int) -> int:
    return int(load_library().fbsde_profile_start(int(max_timed_launches)))


def fbsde_profile_select(families) -> int:
    """Time only the named kernel families (e.g. ["matvec"]); the others are counted."""
    lib = load_library()
    names = [lib.fbsde_kernel_name(f).decode() for f in range(FBSDE_NUM_KERNELS)]
    mask = 0
    for fam in families:
        mask |= 1 << names.index(fam)
    return int(lib.fbsde_profile_select(mask))


def fbsde_profile_stop() -> dict:
    """Per kernel family: launches, timed launches and summed event milliseconds."""
    lib = load_library()
    arr = (fbsde_kernel_stats * FBSDE_NUM_KERNELS)()
    check(lib.fbsde_profile_stop(arr), "fbsde_profile_stop")
    return {lib.fbsde_kernel_name(i).decode(): {"launches": int(arr[i].launches),
                                                  "timed": int(arr[i].timed),
                                                  "total_ms": float(arr[i].total_ms)}
            for i in range(FBSDE_NUM_KERNELS)}


def fbsde_abi_version() -> int:
    return int(load_library().fbsde_abi_version())


def check(status: int, what: str = "fbsde") -> None:
    if status != FBSDE_OK:
        raise RuntimeError(f"{what}: {fbsde_status_string(status)} ({status})")


class Solver:
    """Owns the device workspace for one problem shape and runs solves on it."""

    def __init__(self, kind: str, d: int, N: int, M: int, sigma: float, T: float, Q: int,
                 precision: str = "fp32", theta=None, device="cuda", **params):
        import torch
        self.torch = torch
        self.Q = int(Q)
        self.device = torch.device(device)
        self.theta = None
        if theta is not None:
            self.theta = torch.as_tensor(np.asarray(theta, dtype=np.float64), device=self.device)
        self.problem = make_problem(kind, d, N, M, sigma, T, precision, theta=self.theta,
                                    **params)
        nbytes = fbsde_workspace_bytes(self.problem, self.Q)
        if nbytes == 0:
            raise ValueError("invalid problem parameters")
        self.ws_bytes = nbytes
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        off = (-self.workspace.data_ptr()) % 256
        self.workspace = self.workspace[off:off + nbytes]

    def _adjoint_workspace(self):
        if getattr(self, "adj_workspace", None) is None:
            n = fbsde_adjoint_workspace_bytes(self.problem, self.Q)
            self.adj_workspace = self.torch.empty(n, dtype=self.torch.uint8, device=self.device)
        return self.adj_workspace

    def adjoint(self, x0, seed: int, u0_bar=None, solve_index0: int = 0,
                with_theta: bool = False, check_status: bool = True) -> dict:
        """u(0,x0), grad u (method), and the reverse-sweep derivatives du/dx0, du/dtheta."""
        torch = self.torch
        p = self.problem
        x0 = torch.as_tensor(x0, dtype=torch.float64, device=self.device).contiguous()
        ub = (torch.ones(self.Q, dtype=torch.float64, device=self.device) if u0_bar is None
              else torch.as_tensor(u0_bar, dtype=torch.float64, device=self.device).contiguous())
        out = {"u0": torch.empty(self.Q, dtype=torch.float64, device=self.device),
               "grad": torch.empty(self.Q, p.d, dtype=torch.float64, device=self.device),
               "x0_bar": torch.empty(self.Q, p.d, dtype=torch.float64, device=self.device),
               "theta_bar": (torch.empty(p.d, dtype=torch.float64, device=self.device)
                             if with_theta else None)}
        ws = self._adjoint_workspace()
        check(fbsde_adjoint(p, self.Q, x0, seed, solve_index0, ub, out["u0"], out["grad"],
                            out["x0_bar"], out["theta_bar"], ws), "fbsde_adjoint")
        if check_status:
            out["status"] = int(fbsde_diagnostics(p, self.Q, ws).status)
        return out

    def solve(self, x0, seed: int, solve_index0: int = 0, trace: bool = False,
              trace_forward: bool = False, check_status: bool = True) -> dict:
        torch = self.torch
        p = self.problem
        x0 = torch.as_tensor(x0, dtype=torch.float64, device=self.device).contiguous()
        assert x0.shape == (self.Q, p.d)
        u0 = torch.empty(self.Q, dtype=torch.float64, device=self.device)
        grad = torch.empty(self.Q, p.d, dtype=torch.float64, device=self.device)
        out = {"u0": u0, "grad": grad}
        tr = None
        if trace or trace_forward:
            tr = fbsde_trace()
        if trace:
            out["alpha"] = torch.full((self.Q, p.N), math.nan, dtype=torch.float64,
                                      device=self.device)
            out["alpha_x"] = torch.full((self.Q, p.N, p.d), math.nan, dtype=torch.float64,
                                        device=self.device)
            out["cg_iters"] = torch.zeros(self.Q, p.N, dtype=torch.int32, device=self.device)
            out["newton_iters"] = torch.zeros(self.Q, p.N, dtype=torch.int32, device=self.device)
            tr.alpha, tr.alpha_x = _ptr(out["alpha"]), _ptr(out["alpha_x"])
            tr.cg_iters, tr.newton_iters = _ptr(out["cg_iters"]), _ptr(out["newton_iters"])
        if trace_forward:
            out["x_N"] = torch.empty(self.Q, p.M, p.d, dtype=torch.float64, device=self.device)
            out["y_N"] = torch.empty(self.Q, p.M, dtype=torch.float64, device=self.device)
            tr.x_N, tr.y_N = _ptr(out["x_N"]), _ptr(out["y_N"])
        check(fbsde_solve(p, self.Q, x0, seed, solve_index0, u0, grad, self.workspace, tr),
              "fbsde_solve")
        if check_status:
            dg = fbsde_diagnostics(p, self.Q, self.workspace)
            out["status"] = int(dg.status)
            out["max_newton_iters"] = int(dg.max_newton_iters)
            out["solves_cg_exhausted"] = int(dg.solves_cg_exhausted)
        return out


class Plan:
    """A batch of (possibly heterogeneous) solves captured once into a CUDA graph.

    instances: list of dicts with keys problem (fbsde_problem), Q, x0 (CUDA tensor
    [Q, d]), seed, solve_index0 (default 0), grad (bool, default True).  Outputs are
    allocated here; launch() replays the graph; x0 tensors may be refilled in place."""

    def __init__(self, instances, branches: int = 0, device="cuda"):
        import torch
        self.torch = torch
        lib = load_library()
        n = len(instances)
        self.keep = []
        arr = (fbsde_instance * n)()
        self.u0, self.grad = [], []
        for i, spec in enumerate(instances):
            p = spec["problem"]
            Q = int(spec["Q"])
            x0 = spec["x0"]
            assert x0.is_cuda and x0.dtype == torch.float64 and x0.is_contiguous()
            u = torch.empty(Q, dtype=torch.float64, device=device)
            g = (torch.empty(Q, p.d, dtype=torch.float64, device=device)
                 if spec.get("grad", True) else None)
            self.u0.append(u)
            self.grad.append(g)
            self.keep += [x0, u, g, spec.get("theta")]
            arr[i] = fbsde_instance(p, Q, int(spec.get("solve_index0", 0)), int(spec["seed"]),
                                    x0.data_ptr(), u.data_ptr(), _ptr(g))
        self.arr = arr
        nbytes = int(lib.fbsde_plan_workspace_bytes(n, arr))
        if nbytes == 0:
            raise ValueError("invalid plan instances")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        h = C.c_void_p()
        check(lib.fbsde_plan_create(C.byref(h), n, arr, int(branches), _ptr(self.workspace),
                                    nbytes), "fbsde_plan_create")
        self.handle = h

    def launch(self, stream=None) -> None:
        check(load_library().fbsde_plan_launch(self.handle, _stream(stream)), "fbsde_plan_launch")

    def diagnostics(self, stream=None) -> fbsde_diag:
        out = fbsde_diag()
        check(load_library().fbsde_plan_diagnostics(self.handle, C.byref(out), _stream(stream)),
              "fbsde_plan_diagnostics")
        return out

    def instance_diagnostics(self, index: int, stream=None) -> fbsde_diag:
        out = fbsde_diag()
        check(load_library().fbsde_plan_instance_diagnostics(self.handle, int(index),
                                                             C.byref(out), _stream(stream)),
              "fbsde_plan_instance_diagnostics")
        return out

    def close(self) -> None:
        if getattr(self, "handle", None):
            load_library().fbsde_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _make_function():
    import torch

    class FBSDEValue(torch.autograd.Function):
        """u(0, x0) of every query as a differentiable function of x0 [Q, d] and (for the
        kinds with terminal coefficients) theta [d]; backward runs fbsde_adjoint."""

        @staticmethod
        def forward(ctx, x0, theta, solver, seed, solve_index0):
            x0 = x0.detach().contiguous()
            if theta is not None:
                solver.theta = theta.detach().to(torch.float64).contiguous()
                solver.problem.theta = solver.theta.data_ptr()
            out = solver.solve(x0, seed=seed, solve_index0=solve_index0, check_status=False)
            ctx.solver, ctx.seed, ctx.solve_index0 = solver, seed, solve_index0
            ctx.has_theta = theta is not None
            ctx.save_for_backward(x0)
            return out["u0"]

        @staticmethod
        def backward(ctx, grad_u0):
            (x0,) = ctx.saved_tensors
            adj = ctx.solver.adjoint(x0, ctx.seed, u0_bar=grad_u0.contiguous(),
                                     solve_index0=ctx.solve_index0,
                                     with_theta=ctx.has_theta, check_status=False)
            return adj["x0_bar"], adj["theta_bar"], None, None, None

    return FBSDEValue


_FUNCTION = None


def fbsde_value(solver: "Solver", x0, seed: int, theta=None, solve_index0: int = 0):
    """Differentiable u(0, x0) (torch.autograd): gradients flow to x0 and theta."""
    global _FUNCTION
    if _FUNCTION is None:
        _FUNCTION = _make_function()
    return _FUNCTION.apply(x0, theta, solver, seed, solve_index0)


def _main(argv=None) -> None:
    """One solve of a seeded synthetic problem (used for profiling small cases)."""
    import argparse
    import time

    import torch

    ap = argparse.ArgumentParser(description="one fbsde_solve on cuda:0")
    ap.add_argument("--kind", default="ac_manufactured", choices=sorted(KINDS))
    ap.add_argument("--d", type=int, default=10000)
    ap.add_argument("--M", type=int, default=4096)
    ap.add_argument("--N", type=int, default=3)
    ap.add_argument("--Q", type=int, default=4)
    ap.add_argument("--T", type=float, default=1.0)
    ap.add_argument("--sigma", type=float, default=1.0)
    ap.add_argument("--precision", default="fp32", choices=sorted(PRECISIONS))
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--cg-tol", type=float, default=1e-6)
    ap.add_argument("--cg-max-iter", type=int, default=0)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--x0", default="uniform", choices=["uniform", "zero"],
                    help="query points: U[-1,1]^d from the seed, or the origin")
    ap.add_argument("--anchored", action="store_true",
                    help="Algorithm 1 with one regression per particle anchor "
                         "(fbsde_solve_anchored)")
    ap.add_argument("--K", type=int, default=0,
                    help="with --anchored: each anchor's regression over its batch of K "
                         "particles (fbsde_solve_batch)")
    ap.add_argument("--direct", action="store_true",
                    help="with --anchored --K: solve each batch regression directly "
                         "(fbsde_solve_batch_direct)")
    ap.add_argument("--time-products", action="store_true",
                    help="run the launch profiler on the product kernel (the first "
                         "FBSDE_PROFILED_EAGER_PASSES CG passes of each level are then launched "
                         "one by one, outside CUDA graphs, e.g. for a kernel profiler)")
    ap.add_argument("--mu0", type=float, default=0.0, help="drift mu0 + mu1 x_i")
    ap.add_argument("--mu1", type=float, default=0.0)
    ap.add_argument("--sig1", type=float, default=0.0, help="diffusion sigma + sig1 x_i")
    ap.add_argument("--time-family", default=None,
                    help="time the launches of one kernel family (e.g. step), or of "
                         "every family (all), with the library's launch profiler")
    ap.add_argument("--kernel-table", action="store_true",
                    help="after the timed solves, one more solve under the CUDA activity "
                         "profiler (torch.profiler): device time per kernel, including the "
                         "kernels that CUDA graphs launch")
    a = ap.parse_args(argv)
    if a.K and not a.anchored:
        ap.error("--K needs --anchored")
    if a.direct and not a.K:
        ap.error("--direct needs --K")
    rng = np.random.default_rng(a.seed)
    x0 = torch.tensor(rng.uniform(-1.0, 1.0, size=(a.Q, a.d)) if a.x0 == "uniform"
                      else np.zeros((a.Q, a.d)), device="cuda")
    theta = rng.uniform(0.5, 1.5, size=a.d) if a.kind in ("hjb_logquad", "affine_test") else None
    solver = Solver(a.kind, a.d, a.N, a.M, a.sigma, a.T, Q=a.Q, precision=a.precision,
                    theta=theta, cg_tol=a.cg_tol, cg_max_iter=a.cg_max_iter, mu0=a.mu0,
                    mu1=a.mu1, sig1=a.sig1)
    if a.kernel_table:
        # the activity API is set up before the first solve instantiates its CUDA graphs:
        # kernels of graphs instantiated earlier may be recorded for one loop iteration only
        from torch.profiler import ProfilerActivity, profile
        with profile(activities=[ProfilerActivity.CUDA]):
            torch.cuda.synchronize()
    if a.time_products or a.time_family:
        fbsde_profile_start(1 << 20)
        if a.time_family != "all":
            fbsde_profile_select([a.time_family or "matvec"])
    for r in range(a.repeat):
        t0 = time.perf_counter()
        out = (solve_anchored(solver.problem, x0, a.seed, K=a.K or None, direct=a.direct)
               if a.anchored else solver.solve(x0, seed=a.seed))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        print(f"solve {r}: {dt * 1e3:.1f} ms status={out['status']} "
              f"u0[0]={float(out['u0'][0]):.12f}")
    if a.kernel_table:
        from torch.profiler import ProfilerActivity, profile
        run = ((lambda: solve_anchored(solver.problem, x0, a.seed, K=a.K or None,
                                       direct=a.direct)) if a.anchored
               else (lambda: solver.solve(x0, seed=a.seed)))
        with profile(activities=[ProfilerActivity.CUDA]) as kp:
            run()
            torch.cuda.synchronize()
        print(kp.key_averages().table(sort_by="cuda_time_total", row_limit=16,
                                      max_name_column_width=64))
    if a.time_products or a.time_family:
        prof = fbsde_profile_stop()
        for fam in (prof if a.time_family == "all" else [a.time_family or "matvec"]):
            mv = prof[fam]
            if mv["launches"]:
                print(f"{fam} launches {mv['launches']}, timed {mv['timed']}, "
                      f"{mv['total_ms']:.3f} ms")


if __name__ == "__main__":
    _main()
