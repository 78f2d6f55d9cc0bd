"""fbsde_solve_noalloc: the solve for callers that cannot allocate device memory (it
runs on the library's own fixed scratch array).  Its results must agree with the
workspace entry point fbsde_solve on the same inputs, on two calls in a row (the
scratch array keeps the previous call's contents between calls)."""
import math

import numpy as np
import pytest

from helpers import TOL_FP32, TOL_FP64

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _reference(fb, p, Q, x0, seed):
    ws = torch.empty(fb.fbsde_workspace_bytes(p, Q), dtype=torch.uint8, device="cuda")
    u = torch.empty(Q, dtype=torch.float64, device="cuda")
    g = torch.empty(Q, p.d, dtype=torch.float64, device="cuda")
    fb.check(fb.fbsde_solve(p, Q, x0, seed, 0, u, g, ws), "fbsde_solve")
    torch.cuda.synchronize()
    return u.cpu().numpy(), g.cpu().numpy()


@pytest.mark.parametrize("prec,tol", [("fp32", TOL_FP32), ("fp64", TOL_FP64)])
def test_noalloc_matches_workspace_entry_point_twice(prec, tol):
    from paper_2510_02635_gb300 import fbsde as fb
    d, N, M, Q, seed = 200, 5, 1500, 3, 11
    rng = np.random.default_rng(4)
    theta = torch.tensor(rng.uniform(0.5, 1.5, d), device="cuda")
    x0 = torch.tensor(rng.standard_normal((Q, d)) / math.sqrt(d), device="cuda")
    cases = [fb.make_problem("ac_manufactured", d, N, M, 1.0, 0.5, prec, cg_tol=1e-10),
             fb.make_problem("hjb_logquad", d, N, M, math.sqrt(2.0), 1.0, prec, theta=theta,
                             cg_tol=1e-10)]
    for p in cases:
        assert 0 < fb.fbsde_workspace_bytes(p, Q) <= fb.FBSDE_NOALLOC_MAX_BYTES
        u_ref, g_ref = _reference(fb, p, Q, x0, seed)
        for _ in range(2):
            u = torch.full((Q,), math.nan, dtype=torch.float64, device="cuda")
            g = torch.full((Q, d), math.nan, dtype=torch.float64, device="cuda")
            fb.check(fb.fbsde_solve_noalloc(p, Q, x0, seed, 0, u, g), "fbsde_solve_noalloc")
            torch.cuda.synchronize()
            u, g = u.cpu().numpy(), g.cpu().numpy()
            assert np.all(np.abs(u - u_ref) <= tol * np.abs(u_ref))
            scale = np.maximum(np.linalg.norm(g_ref, axis=1), np.abs(u_ref))
            assert np.all(np.linalg.norm(g - g_ref, axis=1) <= tol * scale)


def test_noalloc_call_allocates_no_device_memory():
    """The defining property: once the library's module is loaded on the device (the
    first call does that, and looks up the scratch array's address), a call leaves the
    device's free memory exactly where it was."""
    from paper_2510_02635_gb300 import fbsde as fb
    d, N, M, Q, seed = 300, 4, 2000, 2, 5
    rng = np.random.default_rng(6)
    x0 = torch.tensor(rng.standard_normal((Q, d)) / math.sqrt(d), device="cuda")
    u = torch.empty(Q, dtype=torch.float64, device="cuda")
    g = torch.empty(Q, d, dtype=torch.float64, device="cuda")
    p = fb.make_problem("ac_manufactured", d, N, M, 1.0, 0.5, "fp32", cg_tol=1e-8)
    fb.check(fb.fbsde_solve_noalloc(p, Q, x0, seed, 0, u, g), "fbsde_solve_noalloc")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        fb.check(fb.fbsde_solve_noalloc(p, Q, x0, seed, 0, u, g), "fbsde_solve_noalloc")
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    assert bool(torch.isfinite(u).all())


def test_noalloc_rejects_problems_beyond_its_scratch():
    from paper_2510_02635_gb300 import fbsde as fb
    p = fb.make_problem("ac_manufactured", 4000, 5, 8192, 1.0, 0.5, "fp32")
    assert fb.fbsde_workspace_bytes(p, 1) > fb.FBSDE_NOALLOC_MAX_BYTES
    x0 = torch.zeros(1, 4000, dtype=torch.float64, device="cuda")
    u = torch.empty(1, dtype=torch.float64, device="cuda")
    assert fb.fbsde_solve_noalloc(p, 1, x0, 0, 0, u, None) == fb.FBSDE_ERR_WORKSPACE
