"""FP64 CPU oracle of the localized stochastic FBSDE scheme (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` are the only callers.  The CUDA
library and its Python binding never import this package, and this package
imports nothing from them.

The arithmetic lives in ``fbsde_oracle.c`` (plain C, FP64, OpenMP only over
independent outputs); this file compiles it with gcc on first use and marshals
numpy arrays.  Every function names the passage of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fbsde_oracle.c")
_SRC_SDE = os.path.join(_HERE, "fbsde_oracle_sde.c")   # the scheme with a drift (same library)
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

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
STATUS = {0: "ok", 1: "bad argument", 4: "newton not converged", 5: "cg not converged",
          7: "non-finite result", 8: "out of memory"}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(_SRC_SDE))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", _SRC, _SRC_SDE, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("d", C.c_int32), ("sigma", C.c_double), ("T", C.c_double),
        ("N", C.c_int32), ("cg_max_iter", C.c_int32), ("M", C.c_int64),
        ("theta", C.POINTER(C.c_double)), ("A", C.c_double), ("c0", C.c_double),
        ("c1", C.c_double), ("c2", C.c_double), ("c3", C.c_double), ("h", C.c_double),
        ("ridge_rel", C.c_double),
        ("cg_tol", C.c_double), ("newton_tol", C.c_double), ("newton_max_iter", C.c_int32),
        ("pad_", C.c_int32),
    ]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_up = C.POINTER(C.c_uint32)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            lib.orc_philox4x32_10.argtypes = [_up, _up, _up]
            lib.orc_philox4x32_10.restype = None
            lib.orc_uniform.argtypes = [C.c_uint32]
            lib.orc_uniform.restype = C.c_double
            lib.orc_normals.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                        C.c_int32, _dp]
            lib.orc_normals.restype = None
            lib.orc_g.argtypes = [C.POINTER(_Problem), _dp]
            lib.orc_g.restype = C.c_double
            lib.orc_f.argtypes = [C.POINTER(_Problem), C.c_double, _dp, C.c_double, _dp, _dp]
            lib.orc_f.restype = C.c_double
            lib.orc_newton.argtypes = [C.POINTER(_Problem), C.c_double, C.c_double, C.c_double,
                                       _ip]
            lib.orc_newton.restype = C.c_double
            lib.orc_f_feature.argtypes = [C.POINTER(_Problem), C.c_double, _dp, _dp]
            lib.orc_f_feature.restype = C.c_double
            lib.orc_llr.argtypes = [C.c_int32, C.c_int64, _dp, _dp, C.c_double, C.c_double,
                                    C.c_double, C.c_double, C.c_int32, _dp, _dp, _dp, _ip]
            lib.orc_llr.restype = C.c_int
            lib.orc_solve.argtypes = [C.POINTER(_Problem), _dp, C.c_uint64, C.c_uint32,
                                      C.c_int32, _dp, _dp, _dp, _dp, _ip, _ip, _dp, _dp, _dp,
                                      _dp]
            lib.orc_solve.restype = C.c_int
            lib.orc_solve_anchored.argtypes = [C.POINTER(_Problem), _dp, C.c_uint64,
                                               C.c_uint32, _dp, _dp]
            lib.orc_solve_anchored.restype = C.c_int
            lib.orc_solve_neighbours.argtypes = [C.POINTER(_Problem), C.c_int64, _dp, C.c_uint64,
                                                 C.c_uint32, _dp, _dp]
            lib.orc_solve_neighbours.restype = C.c_int
            lib.orc_solve_batch.argtypes = [C.POINTER(_Problem), C.c_int64, _dp, C.c_uint64,
                                            C.c_uint32, _dp, _dp]
            lib.orc_solve_batch.restype = C.c_int
            lib.orc_adjoint.argtypes = [C.POINTER(_Problem), _dp, C.c_uint64, C.c_uint32, _dp,
                                        _dp, _dp, _dp]
            lib.orc_adjoint.restype = C.c_int
            lib.orc_path.argtypes = [C.POINTER(_Problem), _dp, C.c_uint64, C.c_uint32, C.c_int64,
                                     _dp]
            lib.orc_path.restype = C.c_int
            lib.orc_g_grad.argtypes = [C.POINTER(_Problem), _dp, _dp, _dp]
            lib.orc_g_grad.restype = None
            lib.orc_f_grads.argtypes = [C.POINTER(_Problem), C.c_double, _dp, C.c_double, _dp,
                                        _dp, _dp]
            lib.orc_f_grads.restype = None
            lib.orc_max_threads.argtypes = []
            lib.orc_max_threads.restype = C.c_int
            lib.orc_solve_sde.argtypes = [C.POINTER(_Problem), C.c_void_p, _dp, C.c_uint64,
                                          C.c_uint32, _dp, _dp, _dp, _dp, _ip, _dp]
            lib.orc_solve_sde.restype = C.c_int
            lib.orc_sde_g.argtypes = [C.POINTER(_Problem), _dp]
            lib.orc_sde_g.restype = C.c_double
            lib.orc_sde_f.argtypes = [C.POINTER(_Problem), C.c_void_p, C.c_double, _dp, C.c_double,
                                      _dp, _dp]
            lib.orc_sde_f.restype = C.c_double
            _lib = lib
    return _lib


def _ptr(a, ty=_dp):
    if a is None:
        return None
    return a.ctypes.data_as(ty)


@dataclass
class Problem:
    """Parameters of one problem of the form (2.1) with mu = 0 and scalar sigma."""
    kind: str
    d: int
    sigma: float
    T: float
    N: int
    M: int
    theta: np.ndarray | None = None
    A: float = 0.0
    c0: float = 0.0
    c1: float = 0.0
    c2: float = 0.0
    c3: float = 0.0
    h: float = 2.0
    ridge_rel: float = 1e-3
    cg_tol: float = 1e-12
    cg_max_iter: int = 0          # 0: 10 d
    newton_tol: float = 1e-13
    newton_max_iter: int = 50
    _keep: list = field(default_factory=list, repr=False)

    def c_struct(self) -> _Problem:
        th = None
        if self.theta is not None:
            th = np.ascontiguousarray(self.theta, dtype=np.float64)
            assert th.shape == (self.d,)
            self._keep = [th]
        return _Problem(KINDS[self.kind], int(self.d), float(self.sigma), float(self.T),
                        int(self.N), int(self.cg_max_iter or 10 * self.d), int(self.M),
                        _ptr(th), float(self.A), float(self.c0), float(self.c1),
                        float(self.c2), float(self.c3), float(self.h), float(self.ridge_rel),
                        float(self.cg_tol),
                        float(self.newton_tol), int(self.newton_max_iter), 0)


def max_threads() -> int:
    return int(_load().orc_max_threads())


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of Salmon et al. (SC'11) on one counter (4 words) and key (2 words)."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c, _up), _ptr(k, _up), _ptr(out, _up))
    return out


def uniform(x: int) -> float:
    return float(_load().orc_uniform(int(x) & 0xFFFFFFFF))


def normals(seed: int, s: int, k: int, j: int, d: int) -> np.ndarray:
    """xi_{s,k,j,0..d-1}: the standard normals of particle j at level k (k = N: the end
    point of its Brownian path, 1 <= k < N: the bridge step to level k)."""
    out = np.zeros(d, dtype=np.float64)
    _load().orc_normals(seed, s, k, j, d, _ptr(out))
    return out


def path(prob: Problem, x0, seed: int, s: int, j: int) -> np.ndarray:
    """Positions X_0..X_N ([N+1, d]) of particle j of solve s: the Brownian path of
    Eq. 2.7 drawn backwards by the Brownian bridge, as the solve and the adjoint draw it."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    out = np.zeros((prob.N + 1, prob.d))
    ps = prob.c_struct()
    st = _load().orc_path(C.byref(ps), _ptr(x0), seed, s, j, _ptr(out))
    if st != 0:
        raise RuntimeError(f"orc_path: status {st}")
    return out


def g(prob: Problem, x) -> float:
    """Terminal condition g of (2.1) for the problem kind."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    ps = prob.c_struct()
    return float(_load().orc_g(C.byref(ps), _ptr(x)))


def f(prob: Problem, t: float, x, y: float, z) -> tuple[float, float]:
    """Driver f(t,x,y,z) of (2.1) and its derivative in y."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    ps = prob.c_struct()
    dfdy = C.c_double()
    val = _load().orc_f(C.byref(ps), t, _ptr(x), y, _ptr(z), C.byref(dfdy))
    return float(val), float(dfdy.value)


def newton(prob: Problem, E_hat: float, dt: float, t: float, x, z) -> tuple[float, int]:
    """Root of F(Y) = Y - E_hat - dt f(t,x,Y,z) by the Newton iteration (2.16)-(2.17)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    ps = prob.c_struct()
    lib = _load()
    feat = lib.orc_f_feature(C.byref(ps), t, _ptr(x), _ptr(z))
    it = C.c_int32()
    y = lib.orc_newton(C.byref(ps), E_hat, dt, feat, C.byref(it))
    return float(y), int(it.value)


def llr(D, Y, rho_ref: float, h: float = 2.0, ridge_rel: float = 1e-3, cg_tol: float = 1e-12,
        cg_max_iter: int = 0):
    """One weighted local linear regression, Eqs. (2.10)-(2.15) with Remark 2.2's ridge,
    solved on the Schur complement of Lemma 3.7.  Returns (alpha, alpha_x, w, iters, status)."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    M, d = D.shape
    assert Y.shape == (M,)
    ax = np.zeros(d)
    w = np.zeros(M)
    alpha = C.c_double()
    it = C.c_int32()
    st = _load().orc_llr(d, M, _ptr(D), _ptr(Y), rho_ref, h, ridge_rel, cg_tol,
                         int(cg_max_iter or 10 * d), C.byref(alpha), _ptr(ax), _ptr(w),
                         C.byref(it))
    return float(alpha.value), ax, w, int(it.value), int(st)


def solve(prob: Problem, x0, seed: int, solve_index: int = 0, max_levels: int | None = None,
          trace: bool = False, keep_forward: bool = False, keep_levels_y: bool = False) -> dict:
    """Algorithm 1 for one query point x0.  Returns a dict with u0, grad, status and,
    on request, the per-level trace (alpha, alpha_x, CG and Newton iterations), the
    forward-sweep end state (X_N, Y_N) and Y_k^j at every level."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    assert x0.shape == (prob.d,)
    N, M, d = prob.N, prob.M, prob.d
    L = N if max_levels is None else int(max_levels)
    u0 = C.c_double(math.nan)
    grad = np.zeros(d)
    a_lv = np.full(N, np.nan) if trace else None
    ax_lv = np.full((N, d), np.nan) if trace else None
    cg_lv = np.zeros(N, dtype=np.int32) if trace else None
    nt_lv = np.zeros(N, dtype=np.int32) if trace else None
    xN = np.zeros((M, d)) if keep_forward else None
    yN = np.zeros(M) if keep_forward else None
    y_lv = np.full((N + 1, M), np.nan) if keep_levels_y else None
    phase = np.zeros(2)
    ps = prob.c_struct()
    st = _load().orc_solve(C.byref(ps), _ptr(x0), int(seed), int(solve_index), L,
                           C.byref(u0), _ptr(grad), _ptr(a_lv), _ptr(ax_lv),
                           _ptr(cg_lv, _ip), _ptr(nt_lv, _ip), _ptr(xN), _ptr(yN), _ptr(y_lv),
                           _ptr(phase))
    out = {"u0": float(u0.value), "grad": grad, "status": int(st),
           "forward_s": float(phase[0]), "backward_s": float(phase[1]), "levels": L}
    if trace:
        out.update(alpha=a_lv, alpha_x=ax_lv, cg_iters=cg_lv, newton_iters=nt_lv)
    if keep_forward:
        out.update(X_N=xN, Y_N=yN)
    if keep_levels_y:
        out.update(Y_levels=y_lv)
    return out


class _SdeCoef(C.Structure):
    _fields_ = [("mu0", C.c_double), ("mu1", C.c_double), ("sig1", C.c_double)]


def solve_sde(prob: Problem, x0, seed: int, solve_index: int = 0, mu0: float = 0.0,
              mu1: float = 0.0, sig1: float = 0.0, trace: bool = False,
              keep_paths: bool = False) -> dict:
    """Algorithm 1 with the drift mu_i(x) = mu0 + mu1 x_i and the diffusion
    sigma(x) = diag(prob.sigma + sig1 x_i) (the forward SDE of Sec. 2.1, Euler-Maruyama
    paths (2.7), anchor on the drift path of x0, Z = sigma(X)^T alpha_x per particle):
    u0, grad, status and, on request, the per-level alpha, alpha_x, CG iterations and the
    paths X_0..X_N [N+1, M, d]."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    assert x0.shape == (prob.d,)
    N, M, d = prob.N, prob.M, prob.d
    u0 = C.c_double(math.nan)
    grad = np.zeros(d)
    a_lv = np.full(N, np.nan) if trace else None
    ax_lv = np.full((N, d), np.nan) if trace else None
    cg_lv = np.zeros(N, dtype=np.int32) if trace else None
    xs = np.zeros((N + 1, M, d)) if keep_paths else None
    ps = prob.c_struct()
    coef = _SdeCoef(float(mu0), float(mu1), float(sig1))
    st = _load().orc_solve_sde(C.byref(ps), C.byref(coef), _ptr(x0), int(seed), int(solve_index),
                               C.byref(u0), _ptr(grad), _ptr(a_lv), _ptr(ax_lv), _ptr(cg_lv, _ip),
                               _ptr(xs))
    out = {"u0": float(u0.value), "grad": grad, "status": int(st)}
    if trace:
        out.update(alpha=a_lv, alpha_x=ax_lv, cg_iters=cg_lv)
    if keep_paths:
        out["paths"] = xs
    return out


def sde_g(prob: Problem, x) -> float:
    """g of the problem table of the scheme with a drift (kinds 7, 8 and the driftless ones)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(_load().orc_sde_g(C.byref(prob.c_struct()), _ptr(x)))


def sde_f(prob: Problem, t: float, x, y: float, z, mu0: float = 0.0, mu1: float = 0.0,
          sig1: float = 0.0) -> tuple[float, float]:
    """f(t, x, y, z) and df/dy of the scheme with a drift (the coefficients enter the
    manufactured sources of kinds 7 and 8)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    dfdy = C.c_double()
    coef = _SdeCoef(float(mu0), float(mu1), float(sig1))
    v = _load().orc_sde_f(C.byref(prob.c_struct()), C.byref(coef), float(t), _ptr(x), float(y),
                          _ptr(z), C.byref(dfdy))
    return float(v), float(dfdy.value)


def solve_anchored(prob: Problem, x0, seed: int, solve_index: int = 0) -> dict:
    """Algorithm 1 with one regression per particle anchor (each particle's own position
    at level k).  Returns u0, grad (alpha_x of level 0) and status."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    assert x0.shape == (prob.d,)
    u0 = C.c_double(math.nan)
    grad = np.zeros(prob.d)
    ps = prob.c_struct()
    st = _load().orc_solve_anchored(C.byref(ps), _ptr(x0), int(seed), int(solve_index),
                                    C.byref(u0), _ptr(grad))
    return {"u0": float(u0.value), "grad": grad, "status": int(st)}


def solve_neighbours(prob: Problem, K: int, x0, seed: int, solve_index: int = 0) -> dict:
    """Algorithm 1 with one regression per particle anchor over the anchor's K nearest
    particles only (the subset reading of Remark 2.1).  K = M is solve_anchored."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    assert x0.shape == (prob.d,)
    u0 = C.c_double(math.nan)
    grad = np.zeros(prob.d)
    ps = prob.c_struct()
    st = _load().orc_solve_neighbours(C.byref(ps), int(K), _ptr(x0), int(seed), int(solve_index),
                                      C.byref(u0), _ptr(grad))
    return {"u0": float(u0.value), "grad": grad, "status": int(st)}


def solve_batch(prob: Problem, K: int, x0, seed: int, solve_index: int = 0) -> dict:
    """Algorithm 1 with one regression per particle anchor over a batch of K particles, the
    cyclic window j = (m + q) mod M of anchor m (the random-batch reading of Remark 2.1; the
    paths are i.i.d., so the window holds the anchor's own path and a random sample of K - 1
    others).  K = M is solve_anchored."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    assert x0.shape == (prob.d,)
    u0 = C.c_double(math.nan)
    grad = np.zeros(prob.d)
    ps = prob.c_struct()
    st = _load().orc_solve_batch(C.byref(ps), int(K), _ptr(x0), int(seed), int(solve_index),
                                 C.byref(u0), _ptr(grad))
    return {"u0": float(u0.value), "grad": grad, "status": int(st)}


def g_grad(prob: Problem, x) -> tuple[np.ndarray, np.ndarray]:
    """(dg/dx, dg/dtheta) of the terminal condition at x."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    gx, gt = np.zeros(prob.d), np.zeros(prob.d)
    ps = prob.c_struct()
    _load().orc_g_grad(C.byref(ps), _ptr(x), _ptr(gx), _ptr(gt))
    return gx, gt


def f_grads(prob: Problem, t: float, x, y: float, z) -> tuple[np.ndarray, np.ndarray]:
    """(df/dx, df/dz) of the driver at (t, x, y, z)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    fx, fz = np.zeros(prob.d), np.zeros(prob.d)
    ps = prob.c_struct()
    _load().orc_f_grads(C.byref(ps), t, _ptr(x), y, _ptr(z), _ptr(fx), _ptr(fz))
    return fx, fz


def adjoint(prob: Problem, x0, seed: int, solve_index: int = 0, trace: bool = False) -> dict:
    """Reverse-mode derivatives of the estimator u(0,x0) with respect to x0 and theta for
    the same random increments (a plain tape over the levels of Algorithm 1).  With trace,
    also v_levels [N, d]: the solution of each level's adjoint regression solve."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    u0 = C.c_double(math.nan)
    dx, dth = np.zeros(prob.d), np.zeros(prob.d)
    vl = np.full((prob.N, prob.d), np.nan) if trace else None
    ps = prob.c_struct()
    st = _load().orc_adjoint(C.byref(ps), _ptr(x0), int(seed), int(solve_index), C.byref(u0),
                             _ptr(dx), _ptr(dth), _ptr(vl))
    out = {"u0": float(u0.value), "du_dx0": dx, "du_dtheta": dth, "status": int(st)}
    if trace:
        out["v_levels"] = vl
    return out
