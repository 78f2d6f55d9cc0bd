"""Plans (CUDA graph with device-side CG loops): one instance and heterogeneous batches
give the same bits as the eager entry point, launch after launch."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _instance(fb, kind, d, M, N, Q, prec, seed, sigma=1.0, T=0.5, theta=None, sidx=0):
    rng = np.random.default_rng(seed)
    th = None if theta is None else torch.tensor(theta, device="cuda")
    p = fb.make_problem(kind, d, N, M, sigma, T, prec, theta=th,
                        cg_tol=1e-12 if prec == "fp64" else 1e-6, cg_max_iter=300)
    x0 = torch.tensor(rng.standard_normal((Q, d)) / math.sqrt(d), device="cuda")
    return {"problem": p, "Q": Q, "x0": x0, "seed": seed, "solve_index0": sidx, "theta": th}


def _eager(fb, spec):
    p, Q = spec["problem"], spec["Q"]
    ws = torch.empty(fb.fbsde_workspace_bytes(p, Q), dtype=torch.uint8, device="cuda")
    u = torch.empty(Q, dtype=torch.float64, device="cuda")
    g = torch.empty(Q, p.d, dtype=torch.float64, device="cuda")
    fb.check(fb.fbsde_solve(p, Q, spec["x0"], spec["seed"], spec["solve_index0"], u, g, ws))
    status = fb.fbsde_diagnostics(p, Q, ws).status
    return u.cpu(), g.cpu(), status


def test_single_instance_plan_matches_eager_bits():
    from paper_2510_02635_gb300 import fbsde as fb
    for spec in [_instance(fb, "ac_manufactured", 300, 1200, 6, 3, "fp32", 1),
                 _instance(fb, "ac_manufactured", 100, 2048, 5, 1, "fp64", 2)]:
        ref = _eager(fb, spec)
        plan = fb.Plan([spec])
        for _ in range(2):
            plan.launch()
            torch.cuda.synchronize()
            assert torch.equal(plan.u0[0].cpu(), ref[0])
            assert torch.equal(plan.grad[0].cpu(), ref[1])
        assert plan.diagnostics().status == 0
        plan.close()


def test_heterogeneous_batch_plan_matches_per_instance_solves():
    from paper_2510_02635_gb300 import fbsde as fb
    rng = np.random.default_rng(9)
    specs = []
    for i in range(12):
        d = int(round(math.exp(rng.uniform(math.log(20), math.log(2000)))))
        M = int(rng.choice([256, 512, 1024]))
        N = int(rng.choice([3, 5, 8]))
        kind = "ac_manufactured" if i % 2 == 0 else "logistic_grad"
        sigma, T = (1.0, 0.5) if kind == "ac_manufactured" else (float(d), 1.0)
        specs.append(_instance(fb, kind, d, M, N, int(rng.integers(1, 4)),
                               "fp32" if i % 3 else "fp64", 100 + i, sigma, T, sidx=7 * i))
    theta = rng.uniform(0.5, 1.5, 64)
    specs.append(_instance(fb, "hjb_logquad", 64, 700, 4, 2, "fp32", 5, math.sqrt(2.0), 1.0,
                           theta=theta))
    refs = [_eager(fb, s) for s in specs]
    plan = fb.Plan(specs, branches=5)
    plan.launch()
    torch.cuda.synchronize()
    for i, (u, g, _) in enumerate(refs):
        assert torch.equal(plan.u0[i].cpu(), u), i
        assert torch.equal(plan.grad[i].cpu(), g), i
    # refill the bound inputs in place and launch again
    specs[0]["x0"].mul_(0.5)
    ref0 = _eager(fb, specs[0])
    plan.launch()
    torch.cuda.synchronize()
    assert torch.equal(plan.u0[0].cpu(), ref0[0])
    # instances with M close to d may exhaust cg_max_iter (status 5) in both modes alike
    first_bad = next((st for *_, st in refs if st != 0), 0)
    assert plan.diagnostics().status == first_bad
    plan.close()
