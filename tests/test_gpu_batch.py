"""The batched workload (512 uneven instances in one autotuned plan, FP32) against the
oracle on sampled instances, and one instance of the per-instance FP64 form."""
import numpy as np
import pytest

import oracle
from helpers import TOL_FP32, TOL_FP64, oracle_problem, rel_errors
from paper_2510_02635_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sample(instances):
    """Small instances of both kinds, including one with M close to d (slow CG)."""
    cost = np.array([w.M * w.d * w.N for w in instances])
    picks = []
    for kind in ("ac_manufactured", "logistic_grad"):
        idx = [i for i in np.argsort(cost) if instances[i].kind == kind]
        picks += idx[:2]
    near = [i for i in np.argsort(cost) if 0.8 * instances[i].d < instances[i].M < 1.25 * instances[i].d]
    picks += near[:1]
    return [int(i) for i in picks]


def test_batched_plan_matches_oracle_on_sampled_instances():
    from paper_2510_02635_gb300 import autotune
    inst = autotune.route_precision(W.batch_instances())
    x0s = W.batch_x0(inst)
    table = autotune.tune(inst)
    batch = autotune.Batch(inst, x0s, table)
    batch.launch()
    torch.cuda.synchronize()
    assert batch.plan.diagnostics().status == 0
    u, g = batch.results()
    assert all(np.isfinite(u))
    for i in _sample(inst):
        w = inst[i]
        ref = oracle.solve(oracle_problem(w, cg_tol=1e-11), x0s[i][0], w.seed, i)
        assert ref["status"] == 0
        ru, rg = rel_errors(u[i], g[i], ref)
        assert ru <= TOL_FP32 and rg <= TOL_FP32, (i, w.d, w.M, w.N, ru, rg)
    batch.close()


def test_per_instance_fp64_form_matches_oracle():
    from paper_2510_02635_gb300 import autotune, fbsde
    inst = W.batch_instances(precision="fp64")
    x0s = W.batch_x0(inst)
    i = _sample(inst)[0]
    w = inst[i].with_(cg_tol=1e-12)
    x0 = torch.tensor(x0s[i], device="cuda")
    plan = fbsde.Plan([{"problem": autotune.problem_of(w), "Q": 1, "x0": x0, "seed": w.seed,
                        "solve_index0": i}])
    plan.launch()
    torch.cuda.synchronize()
    ref = oracle.solve(oracle_problem(w), x0s[i][0], w.seed, i)
    ru, rg = rel_errors(float(plan.u0[0][0]), plan.grad[0][0].cpu().numpy(), ref)
    assert ru <= TOL_FP64 and rg <= TOL_FP64
    plan.close()


def test_routed_batch_has_the_accuracy_of_the_fp64_form():
    """The first 32 batch instances, precision routed by conditioning (FP32 where the
    regression's estimated condition number allows it), against each instance solved
    alone in FP64: u and grad u within 1e-4 relative for every instance."""
    from paper_2510_02635_gb300 import autotune, fbsde
    inst = autotune.route_precision(W.batch_instances())[:32]
    assert any(w.precision == "fp64" for w in inst) and any(w.precision == "fp32" for w in inst)
    x0s = W.batch_x0(W.batch_instances())[:32]
    batch = autotune.Batch(inst, x0s, None)
    batch.launch()
    torch.cuda.synchronize()
    u32, g32 = batch.results()
    batch.close()
    for i, w in enumerate(W.batch_instances(precision="fp64")[:32]):
        plan = fbsde.Plan([{"problem": autotune.problem_of(w), "Q": 1, "seed": w.seed,
                            "x0": torch.tensor(x0s[i], device="cuda"), "solve_index0": i}])
        plan.launch()
        torch.cuda.synchronize()
        u64, g64 = float(plan.u0[0][0]), plan.grad[0][0].cpu().numpy()
        plan.close()
        scale = max(np.linalg.norm(g64), abs(u64))
        assert abs(u32[i] - u64) <= TOL_FP32 * abs(u64), (i, w.d, w.M)
        assert np.linalg.norm(g32[i] - g64) <= TOL_FP32 * scale, (i, w.d, w.M)
