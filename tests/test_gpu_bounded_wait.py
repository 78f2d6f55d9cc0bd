"""Every device wait of the kernels (the mbarrier waits of the product ring, the fused step
and the tensor-core pipeline) gives up after a time limit and records FBSDE_ERR_TIMEOUT
instead of hanging.  The check makes one such wait run out on purpose, with a short limit,
on an mbarrier that nothing arrives on (no fault, no trap: the wait returns), and then
checks that the context is still usable by running a solve."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_wait_gives_up_after_its_limit_and_the_context_stays_usable():
    from paper_2510_02635_gb300 import fbsde as fb
    scratch = torch.zeros(4, dtype=torch.int32, device="cuda")
    for limit in (1_000_000, 50_000_000):
        st, waited = fb.fbsde_check_bounded_wait(limit, scratch)
        assert st == fb.FBSDE_ERR_TIMEOUT
        # the first wait runs to its limit; the second, after the first timeout, only polls
        assert limit <= waited < limit + 20_000_000, (limit, waited)
    d, N, M, Q = 32, 3, 256, 1
    solver = fb.Solver("ac_manufactured", d, N, M, 1.0, 0.5, Q=Q, precision="fp32",
                       cg_tol=1e-7)
    x0 = torch.tensor(np.linspace(-0.5, 0.5, d)[None, :], device="cuda")
    out = solver.solve(x0, seed=3)
    torch.cuda.synchronize()
    assert out["status"] == 0 and math.isfinite(float(out["u0"][0]))
