"""Algorithm 1 with one regression per particle anchor: the CUDA path against the oracle's
literal per-anchor solve on the same seeds (FP64 within 1e-10, FP32 within 1e-4), and, with
uniform weights, against the single-anchor entry point; the same for each anchor's
regression over a batch of K particles (fbsde_solve_batch, and fbsde_solve_batch_direct with
each regression solved directly, against the oracle's subset loop).  Sizes are ragged with
respect to the 64 x 64 tiles of the SIMT contractions, the 128 x 128 tiles of the tensor-core ones
(M >= 1024, FP32) and the 16-byte row chunks."""
import math

import numpy as np
import pytest

import oracle
from helpers import TOL_FP32, TOL_FP64

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    ("ac_manufactured", 10, 150, 4, {}),
    ("ac_manufactured", 37, 200, 3, {"h": 1.0}),
    ("logistic_grad", 12, 97, 3, {"sigma": 12.0, "T": 1.0}),
    ("hjb_logquad", 9, 130, 3, {"sigma": math.sqrt(2.0), "T": 1.0, "theta": True}),
    ("ac_doublewell", 16, 65, 4, {"sigma": math.sqrt(2.0), "T": 0.3}),
    ("cos_linear_test", 5, 64, 3, {"c1": 0.4}),
]


def _run(fb, kind, d, M, N, prec, extra, Q=2, seed=13, K=None, direct=False):
    extra = dict(extra)
    sigma, T, h = extra.pop("sigma", 1.0), extra.pop("T", 0.5), extra.pop("h", 2.0)
    rng = np.random.default_rng(d * 1000 + M)
    theta = rng.uniform(0.5, 1.5, d) if extra.pop("theta", False) else None
    x0 = rng.normal(scale=0.4, size=(Q, d))
    tol = 1e-13 if prec == "fp64" else 1e-7
    th_dev = torch.tensor(theta, device="cuda") if theta is not None else None
    p = fb.make_problem(kind, d, N, M, sigma, T, prec, theta=th_dev, h=h, cg_tol=tol,
                        cg_max_iter=1000, **extra)
    out = fb.solve_anchored(p, torch.tensor(x0, device="cuda"), seed, 0, K=K, direct=direct)
    torch.cuda.synchronize()
    op = oracle.Problem(kind, d, sigma, T, N, M, theta=theta, h=h, cg_tol=1e-13,
                        cg_max_iter=1000, **extra)
    if K is None:
        refs = [oracle.solve_anchored(op, x0[q], seed, q) for q in range(Q)]
    else:
        refs = [oracle.solve_batch(op, K, x0[q], seed, q) for q in range(Q)]
    return out, refs, p, x0, th_dev


def _check(out, refs, tol):
    assert out["status"] == 0
    for q, ref in enumerate(refs):
        assert ref["status"] == 0
        u, g = float(out["u0"][q]), out["grad"][q].cpu().numpy()
        assert abs(u - ref["u0"]) <= tol * abs(ref["u0"]), (q, u, ref["u0"])
        scale = max(np.linalg.norm(ref["grad"]), abs(ref["u0"]))
        assert np.linalg.norm(g - ref["grad"]) <= tol * scale, q


@pytest.mark.parametrize("kind,d,M,N,extra", CASES)
def test_fp64_matches_oracle(kind, d, M, N, extra):
    from paper_2510_02635_gb300 import fbsde as fb
    out, refs, *_ = _run(fb, kind, d, M, N, "fp64", extra)
    _check(out, refs, TOL_FP64)


@pytest.mark.parametrize("kind,d,M,N,extra", CASES)
def test_fp32_matches_oracle(kind, d, M, N, extra):
    from paper_2510_02635_gb300 import fbsde as fb
    out, refs, *_ = _run(fb, kind, d, M, N, "fp32", extra)
    _check(out, refs, TOL_FP32)


@pytest.mark.parametrize("kind,d,M,N,extra", [
    ("ac_manufactured", 21, 1030, 2, {}),
    ("logistic_grad", 12, 1100, 2, {"sigma": 12.0, "T": 1.0}),
])
def test_fp32_tensor_core_products_match_oracle(kind, d, M, N, extra):
    """From M = 1024 particles on, the FP32 contractions run on the tensor cores (split
    TF32); M is ragged with respect to their 128 x 128 tiles and 16-wide k stages."""
    from paper_2510_02635_gb300 import fbsde as fb
    out, refs, *_ = _run(fb, kind, d, M, N, "fp32", extra, Q=1)
    _check(out, refs, TOL_FP32)


@pytest.mark.parametrize("prec,tol", [("fp64", TOL_FP64), ("fp32", TOL_FP32)])
def test_uniform_weights_equal_the_single_anchor_solve(prec, tol):
    """h = inf: every anchor's fit is the single-anchor fit shifted, so u and grad u are
    the single-anchor entry point's."""
    from paper_2510_02635_gb300 import fbsde as fb
    d, M, N, Q = 20, 180, 4, 2
    x0 = torch.tensor(np.random.default_rng(3).normal(scale=0.4, size=(Q, d)), device="cuda")
    p = fb.make_problem("ac_manufactured", d, N, M, 1.0, 0.5, prec, h=math.inf,
                        cg_tol=1e-13 if prec == "fp64" else 1e-7, cg_max_iter=1000)
    a = fb.solve_anchored(p, x0, 21, 0)
    ws = torch.empty(fb.fbsde_workspace_bytes(p, Q), dtype=torch.uint8, device="cuda")
    u = torch.empty(Q, dtype=torch.float64, device="cuda")
    g = torch.empty(Q, d, dtype=torch.float64, device="cuda")
    fb.check(fb.fbsde_solve(p, Q, x0, 21, 0, u, g, ws))
    torch.cuda.synchronize()
    assert a["status"] == 0
    assert torch.all(torch.abs(a["u0"] - u) <= tol * torch.abs(u))
    scale = torch.maximum(torch.linalg.norm(g, dim=1), torch.abs(u))
    assert torch.all(torch.linalg.norm(a["grad"] - g, dim=1) <= tol * scale)


@pytest.mark.parametrize("prec,tol,d", [("fp32", TOL_FP32, 4096), ("fp32", TOL_FP32, 4100),
                                        ("fp64", TOL_FP64, 2048), ("fp64", TOL_FP64, 2052)])
def test_uniform_weights_on_both_sides_of_the_register_row_limit(prec, tol, d):
    """Rows of 1024 16-byte chunks (FP32 d = 4096, FP64 d = 2048) are the longest whose CG
    pass keeps the anchor's vectors in registers (eight warps of four chunks per thread);
    one chunk more takes the streaming warp-per-anchor pass.  Both equal the single-anchor
    solve under uniform weights.  M < d, so the ridge is the mean eigenvalue."""
    from paper_2510_02635_gb300 import fbsde as fb
    M, N, Q = 180, 3, 2
    x0 = torch.tensor(np.random.default_rng(d).normal(scale=0.02, size=(Q, d)), device="cuda")
    p = fb.make_problem("ac_manufactured", d, N, M, 1.0, 0.5, prec, h=math.inf, ridge_rel=1.0,
                        cg_tol=1e-13 if prec == "fp64" else 1e-7, cg_max_iter=1000)
    a = fb.solve_anchored(p, x0, 5, 0)
    ws = torch.empty(fb.fbsde_workspace_bytes(p, Q), dtype=torch.uint8, device="cuda")
    u = torch.empty(Q, dtype=torch.float64, device="cuda")
    g = torch.empty(Q, d, dtype=torch.float64, device="cuda")
    fb.check(fb.fbsde_solve(p, Q, x0, 5, 0, u, g, ws))
    torch.cuda.synchronize()
    assert a["status"] == 0
    assert torch.all(torch.abs(a["u0"] - u) <= tol * torch.abs(u))
    scale = torch.maximum(torch.linalg.norm(g, dim=1), torch.abs(u))
    assert torch.all(torch.linalg.norm(a["grad"] - g, dim=1) <= tol * scale)


def test_argument_errors():
    from paper_2510_02635_gb300 import fbsde as fb
    fb.load_library()
    assert fb.fbsde_anchored_workspace_bytes(
        fb.make_problem("ac_manufactured", 10, 3, 40000, 1.0, 0.5, "fp32")) == 0   # M > 32768
    p = fb.make_problem("hjb_logquad", 10, 3, 64, 1.0, 0.5, "fp32")   # theta missing
    ws = torch.empty(fb.fbsde_anchored_workspace_bytes(p), dtype=torch.uint8, device="cuda")
    x0 = torch.zeros(1, 10, dtype=torch.float64, device="cuda")
    u = torch.empty(1, dtype=torch.float64, device="cuda")
    assert fb.fbsde_solve_anchored(p, 1, x0, 0, 0, u, None, ws) == fb.FBSDE_ERR_ARG


# Drivers whose Newton derivative stays away from 0 on small batches (a gradient-dependent
# driver with a large sigma makes F' = 1 - dt sum_i z_i, built from a few noisy slopes, pass
# near 0, where both sides' Newton iterations are at the mercy of rounding).
BATCH_CASES = [
    ("ac_manufactured", 10, 150, 3, 40, {}),
    ("cos_linear_test", 5, 97, 3, 31, {"c1": 0.4}),
    ("hjb_logquad", 9, 130, 3, 64, {"sigma": math.sqrt(2.0), "T": 1.0, "theta": True}),
    ("ac_doublewell", 16, 65, 3, 33, {"sigma": math.sqrt(2.0), "T": 0.3}),
]


@pytest.mark.parametrize("kind,d,M,N,K,extra", BATCH_CASES)
@pytest.mark.parametrize("prec,tol", [("fp64", TOL_FP64), ("fp32", TOL_FP32)])
def test_batch_matches_oracle(kind, d, M, N, K, extra, prec, tol):
    """Each anchor's regression over its batch of K particles (the cyclic window, the
    random-batch reading of Remark 2.1) against the oracle's literal subset loop."""
    from paper_2510_02635_gb300 import fbsde as fb
    out, refs, *_ = _run(fb, kind, d, M, N, prec, extra, K=K)
    _check(out, refs, tol)


def test_smallest_batch_fp64_matches_oracle():
    """K = 2 < d: each anchor's regression is underdetermined and held by the ridge."""
    from paper_2510_02635_gb300 import fbsde as fb
    out, refs, *_ = _run(fb, "ac_doublewell", 16, 65, 3, "fp64",
                         {"sigma": math.sqrt(2.0), "T": 0.3}, K=2)
    _check(out, refs, TOL_FP64)


def test_batch_on_the_tensor_core_path_matches_oracle():
    from paper_2510_02635_gb300 import fbsde as fb
    out, refs, *_ = _run(fb, "ac_manufactured", 21, 1030, 2, "fp32", {}, Q=1, K=300)
    _check(out, refs, TOL_FP32)


@pytest.mark.parametrize("prec,tol,M,K", [("fp64", TOL_FP64, 700, 50), ("fp32", TOL_FP32, 700, 50),
                                          ("fp32", TOL_FP32, 1300, 40)])
def test_banded_products_match_oracle(prec, tol, M, K):
    """Narrow windows (K << M): the products cover only the band of (particle, anchor)
    entries the windows use, skipping most tiles of the M x M products and most K-splits
    of the tall ones (SIMT tiles at M = 700, tensor-core tiles at M = 1300; the band wraps
    around the last anchors).  Same bar as the full batch solve."""
    from paper_2510_02635_gb300 import fbsde as fb
    out, refs, *_ = _run(fb, "ac_manufactured", 24, M, 2, prec, {}, Q=1, K=K)
    _check(out, refs, tol)


@pytest.mark.parametrize("kind,d,M,N,K,extra", BATCH_CASES)
@pytest.mark.parametrize("prec,tol", [("fp64", TOL_FP64), ("fp32", TOL_FP32)])
def test_direct_batch_matches_oracle(kind, d, M, N, K, extra, prec, tol):
    """Each anchor's batch regression solved directly (its operator's L D L^T) against the
    oracle's literal subset loop, on the cases of the CG form."""
    from paper_2510_02635_gb300 import fbsde as fb
    out, refs, *_ = _run(fb, kind, d, M, N, prec, extra, K=K, direct=True)
    _check(out, refs, tol)
    assert out["cg_passes"] == 0


@pytest.mark.parametrize("prec,tol,d,M,K", [
    ("fp64", TOL_FP64, 16, 65, 2),       # K = 2 < d: held by the ridge
    ("fp32", TOL_FP32, 21, 1030, 300),   # tensor-core products of the level
    ("fp32", TOL_FP32, 24, 1300, 40),    # banded products, the band wrapping around
    ("fp64", TOL_FP64, 128, 160, 48),    # the largest d: three 4 x 4 blocks per thread
    ("fp32", TOL_FP32, 127, 200, 150),   # ragged d, padding inside the last block
])
def test_direct_batch_edges_match_oracle(prec, tol, d, M, K):
    from paper_2510_02635_gb300 import fbsde as fb
    out, refs, *_ = _run(fb, "ac_manufactured", d, M, 2, prec, {}, Q=1, K=K, direct=True)
    _check(out, refs, tol)


@pytest.mark.parametrize("prec,tol", [("fp64", TOL_FP64), ("fp32", TOL_FP32)])
def test_direct_and_cg_batch_solve_the_same_regressions(prec, tol):
    """The two forms of the batch reading agree (the CG to its tolerance, the direct solve
    to rounding), on a window wider than d."""
    from paper_2510_02635_gb300 import fbsde as fb
    d, M, N, Q, K = 50, 600, 3, 2, 200
    x0 = torch.tensor(np.random.default_rng(8).normal(scale=0.3, size=(Q, d)), device="cuda")
    p = fb.make_problem("ac_manufactured", d, N, M, 1.0, 0.5, prec,
                        cg_tol=1e-13 if prec == "fp64" else 1e-7, cg_max_iter=1000)
    a = fb.solve_anchored(p, x0, 4, 0, K=K)
    b = fb.solve_anchored(p, x0, 4, 0, K=K, direct=True)
    assert a["status"] == 0 and b["status"] == 0
    assert torch.all(torch.abs(a["u0"] - b["u0"]) <= tol * torch.abs(a["u0"]))
    scale = torch.maximum(torch.linalg.norm(a["grad"], dim=1), torch.abs(a["u0"]))
    assert torch.all(torch.linalg.norm(a["grad"] - b["grad"], dim=1) <= tol * scale)


def test_direct_batch_argument_errors():
    from paper_2510_02635_gb300 import fbsde as fb
    Q = 1
    for d, ridge in ((fb.FBSDE_BATCH_DIRECT_MAX_D + 1, 1e-3), (16, 0.0)):
        p = fb.make_problem("ac_manufactured", d, 2, 100, 1.0, 0.5, "fp32", ridge_rel=ridge)
        ws = torch.empty(fb.fbsde_anchored_workspace_bytes(p), dtype=torch.uint8, device="cuda")
        x0 = torch.zeros(Q, d, dtype=torch.float64, device="cuda")
        u = torch.empty(Q, dtype=torch.float64, device="cuda")
        g = torch.empty(Q, d, dtype=torch.float64, device="cuda")
        assert fb.fbsde_solve_batch_direct(p, 50, Q, x0, 1, 0, u, g, ws) == fb.FBSDE_ERR_ARG
        assert fb.fbsde_solve_batch_direct(p, 1, Q, x0, 1, 0, u, g, ws) == fb.FBSDE_ERR_ARG


@pytest.mark.parametrize("prec,M", [("fp64", 300), ("fp32", 1100)])
def test_per_anchor_call_is_asynchronous_and_capturable(prec, M):
    """The call enqueues its work and returns: captured by the caller into a CUDA graph (no
    host synchronisation may occur during capture) and replayed, it gives the bits of the
    eager call, which replays its own cached graph.  M = 1100 in FP32 takes the tensor-core
    products with the fused column pass inside the conditional CG loop."""
    from paper_2510_02635_gb300 import fbsde as fb
    d, N, Q, seed = 24, 3, 2, 5
    x0 = torch.tensor(np.random.default_rng(8).normal(scale=0.4, size=(Q, d)), device="cuda")
    p = fb.make_problem("ac_manufactured", d, N, M, 1.0, 0.5, prec,
                        cg_tol=1e-13 if prec == "fp64" else 1e-7, cg_max_iter=1000)
    ws = torch.empty(fb.fbsde_anchored_workspace_bytes(p), dtype=torch.uint8, device="cuda")
    u = torch.empty(Q, dtype=torch.float64, device="cuda")
    g = torch.empty(Q, d, dtype=torch.float64, device="cuda")
    fb.check(fb.fbsde_solve_anchored(p, Q, x0, seed, 0, u, g, ws))
    torch.cuda.synchronize()
    assert fb.fbsde_anchored_diagnostics(p, ws).status == 0
    u_ref, g_ref = u.clone(), g.clone()
    fb.check(fb.fbsde_solve_anchored(p, Q, x0, seed, 0, u, g, ws))   # the cached graph
    torch.cuda.synchronize()
    assert torch.equal(u, u_ref) and torch.equal(g, g_ref)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s, capture_error_mode="thread_local"):
        fb.check(fb.fbsde_solve_anchored(p, Q, x0, seed, 0, u, g, ws,
                                         stream=torch.cuda.current_stream()))
    for _ in range(2):
        u.zero_()
        g.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(u, u_ref) and torch.equal(g, g_ref)
    assert fb.fbsde_anchored_diagnostics(p, ws).status == 0


def test_per_anchor_status_reports_exhausted_cg():
    """Three CG passes per level, far from the tolerance: the call itself returns
    FBSDE_OK (it only enqueues), and the device status read afterwards is FBSDE_ERR_CG, with
    three passes per level and query."""
    from paper_2510_02635_gb300 import fbsde as fb
    d, M, N, Q = 16, 200, 3, 2
    x0 = torch.zeros(Q, d, dtype=torch.float64, device="cuda")
    p = fb.make_problem("ac_manufactured", d, N, M, 1.0, 0.5, "fp64", cg_tol=1e-15,
                        cg_max_iter=3)
    ws = torch.empty(fb.fbsde_anchored_workspace_bytes(p), dtype=torch.uint8, device="cuda")
    u = torch.empty(Q, dtype=torch.float64, device="cuda")
    assert fb.fbsde_solve_anchored(p, Q, x0, 1, 0, u, None, ws) == fb.FBSDE_OK
    dg = fb.fbsde_anchored_diagnostics(p, ws)
    assert dg.status == fb.FBSDE_ERR_CG
    assert dg.cg_iters_total == 3 * N * Q
