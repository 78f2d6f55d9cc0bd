"""Named workloads and their seeded synthetic inputs.

This module holds no arithmetic of the method.  It only names the problem
parameters of each workload and draws the query points x0 (and the terminal
coefficients theta) from numpy's seeded generator, so that the CUDA path, the
CPU oracle, the tests and the benchmark all see identical inputs.  The Brownian
increments of the method itself are not drawn here: both implementations
regenerate them from the counter-based Philox4x32-10 stream.

The paper has no dataset: all its experiments are manufactured closed-form
problems (Sec. 4), and these workloads are of the same kind.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    kind: str            # problem kind (see the C-ABI header for the formulas)
    d: int
    sigma: float
    T: float
    N: int
    M: int
    Q: int               # number of independent query points (solves)
    seed: int            # Philox seed of the Brownian increments and of the inputs
    x0_law: str          # "zero", "normal_1/d" (N(0, I/d)), "uniform_pm1" (U[-1,1]^d)
    precision: str = "fp32"   # "fp32": FP32 streams + FP64 solve/Newton; "fp64": FP64 throughout
    h: float = 2.0
    ridge_rel: float = 1e-3
    cg_tol: float = 1e-6
    cg_max_iter: int = 0  # 0: library default
    newton_tol: float = 1e-13
    newton_max_iter: int = 50
    A: float = 0.0
    c0: float = 0.0
    c1: float = 0.0
    theta_law: str | None = None   # "uniform_0.5_1.5" for the log-quadratic terminal
    extra: dict = field(default_factory=dict)

    @property
    def particle_dim_updates(self) -> int:
        """Q * M * d * N: particle-dimension updates of one whole solve."""
        return self.Q * self.M * self.d * self.N

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def inputs(w: Workload) -> dict:
    """Seeded query points x0 [Q, d] (float64) and, if the terminal needs them,
    coefficients theta [d]."""
    rng = np.random.default_rng(w.seed)
    theta = None
    if w.theta_law == "uniform_0.5_1.5":
        theta = rng.uniform(0.5, 1.5, size=w.d)
    if w.x0_law == "zero":
        x0 = np.zeros((w.Q, w.d))
    elif w.x0_law == "normal_1/d":
        x0 = rng.standard_normal((w.Q, w.d)) / math.sqrt(w.d)
    elif w.x0_law == "uniform_pm1":
        x0 = rng.uniform(-1.0, 1.0, size=(w.Q, w.d))
    else:
        raise ValueError(f"unknown x0 law {w.x0_law!r}")
    if w.extra.get("theta_affine"):
        theta = rng.uniform(-1.0, 1.0, size=w.d)
    return {"x0": np.ascontiguousarray(x0), "theta": theta}


def exact_solution(w: Workload, x0) -> tuple[float, np.ndarray] | None:
    """u(0, x0) and grad u(0, x0) of the workload's manufactured closed form, or None for
    kinds without one.  These are properties of the test problems (checked against the PDE
    (2.1) symbolically by the oracle tests), not arithmetic of the scheme:
      Allen-Cahn with manufactured source: u = e^{t - T} (1/d) sum_i cos x_i;
      gradient-dependent logistic driver (sigma = d): u = 1 / (1 + exp(-(t + sum_i x_i / d)));
      drift kinds (any affine drift and diffusion): u = e^{t - T} (1/d) sum_i cos x_i, or
      e^{t - T} (1/d) sum_i x_i^2.
    """
    x0 = np.asarray(x0, dtype=np.float64)
    if w.kind in ("ac_manufactured", "drift_ac"):
        e = math.exp(-w.T)
        return e * float(np.mean(np.cos(x0))), -e * np.sin(x0) / w.d
    if w.kind == "logistic_grad" and w.sigma == float(w.d):
        u = 1.0 / (1.0 + math.exp(-float(np.sum(x0)) / w.d))
        return u, np.full(w.d, u * (1.0 - u) / w.d)
    if w.kind == "drift_quad":
        e = math.exp(-w.T)
        return e * float(np.mean(x0 * x0)), 2.0 * e * x0 / w.d
    return None


# Plain scheme at d = 100, FP64 throughout (Allen-Cahn with manufactured source).
C0_AC_D100 = Workload("ac_manufactured_d100_M2048_N10_Q1_fp64", "ac_manufactured", d=100,
                      sigma=1.0, T=0.5, N=10, M=2048, Q=1, seed=0, x0_law="zero",
                      precision="fp64", cg_tol=1e-12)
# Gradient-dependent driver at d = 1000; sigma = d makes the logistic closed form exact.
C1_LOGISTIC_D1000 = Workload("logistic_grad_d1000_M4096_N20_Q64", "logistic_grad", d=1000,
                             sigma=1000.0, T=1.0, N=20, M=4096, Q=64, seed=1,
                             x0_law="normal_1/d")
# Very high dimension: the Allen-Cahn problem of C0 at d = 10^4.
C2_AC_D10000 = Workload("ac_manufactured_d10000_M16384_N50_Q16", "ac_manufactured", d=10000,
                        sigma=1.0, T=1.0, N=50, M=16384, Q=16, seed=2, x0_law="uniform_pm1")
# Log-quadratic terminal with the quadratic-gradient driver (Cole-Hopf solvable).
C4_HJB_D1000 = Workload("hjb_logquad_d1000_M4096_N20_Q1", "hjb_logquad", d=1000,
                        sigma=math.sqrt(2.0), T=1.0, N=20, M=4096, Q=1, seed=4,
                        x0_law="normal_1/d", theta_law="uniform_0.5_1.5")
# Forward SDE with an Ornstein-Uhlenbeck drift and a state-dependent diffusion (drift
# mu_i = 0.1 - 0.8 x_i, diffusion 0.5 + 0.2 x_i), manufactured Allen-Cahn-type source.
F4_DRIFT_AC_D1000 = Workload("drift_ac_ou_d1000_M4096_N20_Q16", "drift_ac", d=1000, sigma=0.5,
                             T=0.6, N=20, M=4096, Q=16, seed=6, x0_law="normal_1/d",
                             extra={"mu0": 0.1, "mu1": -0.8, "sig1": 0.2})
# Sec. 4.1, case 1 of the paper: double-well Allen-Cahn, d = 100, T = 0.3, x0 = 0,
# generator Lap u (sigma = sqrt 2); printed reference u(0,0) ~ 0.0528.
AC_CASE1_D100 = Workload("ac_doublewell_d100_T0.3", "ac_doublewell", d=100,
                         sigma=math.sqrt(2.0), T=0.3, N=10, M=2048, Q=1, seed=5, x0_law="zero")

ALL = {w.name: w for w in (C0_AC_D100, C1_LOGISTIC_D1000, C2_AC_D10000, C4_HJB_D1000,
                           AC_CASE1_D100)}


# Batched uneven instances: 512 independent solves in one plan, d log-uniform in
# [100, 10^4], M in {512, 2048, 8192, 16384}, N in {10, 20, 50}, kinds alternating
# between the Allen-Cahn problem (sigma = 1, T = 0.5) and the logistic-gradient problem
# (sigma = d, T = 1), x0 ~ N(0, I/d), seed 3, FP32.
BATCH_NAME = "batch512_ac_logistic_d100-10000"


def batch_instances(n: int = 512, seed: int = 3, precision: str = "fp32",
                    cg_max_iter: int = 3000) -> list[Workload]:
    """The n instances of the batched workload (Q = 1 each); instance i uses Philox solve
    index i.  d, M and N are drawn in instance order from one numpy generator; the query
    points come from batch_x0."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        d = int(round(math.exp(rng.uniform(math.log(100.0), math.log(10000.0)))))
        M = int(rng.choice([512, 2048, 8192, 16384]))
        N = int(rng.choice([10, 20, 50]))
        if i % 2 == 0:
            kind, sigma, T = "ac_manufactured", 1.0, 0.5
        else:
            kind, sigma, T = "logistic_grad", float(d), 1.0
        out.append(Workload(f"{BATCH_NAME}_{i}", kind, d=d, sigma=sigma, T=T, N=N, M=M, Q=1,
                            seed=seed, x0_law="normal_1/d", precision=precision,
                            cg_max_iter=cg_max_iter, extra={"index": i}))
    return out


def batch_x0(instances: list[Workload], seed: int = 3) -> list[np.ndarray]:
    """x0 of each batched instance ([1, d] each), from a second seeded stream."""
    rng = np.random.default_rng(seed + 1_000_003)
    return [rng.standard_normal((1, w.d)) / math.sqrt(w.d) for w in instances]
