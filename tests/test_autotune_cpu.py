"""Host-side pieces of the batched driver: the condition-number estimate that routes
instances between the FP32 and FP64 paths, checked against the eigenvalues of actual
Gaussian clouds (numpy), and the routing itself."""
import numpy as np
import pytest

from paper_2510_02635_gb300 import autotune, fbsde
from paper_2510_02635_gb300 import workloads as W


def _w(d, M, ridge=1e-3):
    return W.Workload("k", "ac_manufactured", d=d, sigma=1.0, T=1.0, N=1, M=M, Q=1, seed=0,
                      x0_law="zero", ridge_rel=ridge)


@pytest.mark.parametrize("d,M", [(100, 400), (200, 220), (300, 60), (80, 2000)])
def test_kappa_estimate_tracks_sample_covariance(d, M):
    rng = np.random.default_rng(d + M)
    D = rng.standard_normal((M, d))
    S = D.mean(axis=0)
    G = D.T @ D / M - np.outer(S, S)
    lam = 1e-3 * np.trace(G) / d
    ev = np.linalg.eigvalsh(G + lam * np.eye(d))
    kappa = ev[-1] / ev[0]
    est = autotune.kappa_estimate(_w(d, M))
    assert est / 2.5 <= kappa <= est * 2.5, (kappa, est)


def test_route_precision_moves_only_ill_conditioned_fp32_instances():
    inst = [_w(100, 4000), _w(5000, 512), _w(5000, 512).with_(precision="fp64"),
            _w(9000, 512), _w(12000, 512)]
    out = autotune.route_precision(inst)
    # the last is too wide for the FP64 path (d > 10240) and stays FP32
    assert [w.precision for w in out] == ["fp32", "fp64", "fp64", "fp64", "fp32"]
    assert autotune.kappa_estimate(inst[0]) < autotune.KAPPA_FP32_MAX
    assert autotune.kappa_estimate(inst[1]) > autotune.KAPPA_FP32_MAX


def test_routing_covers_every_ill_conditioned_instance_of_the_batch():
    """With the FP64 path up to d = 10240, every FP32 instance of the 512-instance batch
    whose estimated condition number exceeds the FP32 limit goes to FP64 (the batch's d
    stops at 10^4), so the accuracy of every instance is that of the FP64 path or of an
    FP32 regression within the limit."""
    inst = W.batch_instances()
    routed = autotune.route_precision(inst)
    assert max(w.d for w in inst) <= fbsde.FBSDE_MAX_D_FP64
    for w, r in zip(inst, routed):
        hot = autotune.kappa_estimate(w) > autotune.KAPPA_FP32_MAX
        assert r.precision == ("fp64" if hot else "fp32")
    assert sum(r.precision == "fp64" for r in routed) == sum(
        autotune.kappa_estimate(w) > autotune.KAPPA_FP32_MAX for w in inst)
