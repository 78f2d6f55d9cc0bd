"""Accuracy of the GPU scheme against the closed-form solution at the full-size workloads
that have one: the Allen-Cahn problem with manufactured source at d = 10^4 (16 queries,
M = 16384, N = 50; u* = e^{-T} mean_i cos x0_i) and the logistic gradient-dependent driver
at d = 1000 (64 queries, M = 4096, N = 20, sigma = d; u* = logistic(sum_i x0_i / d)).

The bar is the scheme's own error, not the parity tolerance: the error of the estimator
(Theorem 3.1's O(dt) time discretisation, the localisation and ridge bias of the
regression, and the Monte-Carlo spread of its particle cloud), measured by the FP64 oracle
over independent Philox streams and stored with its rule in
tests/golden/closed_form_bounds.json (written by make_closed_form_bounds.py beside it).
Every query of the GPU solve is one more independent stream, so each must lie within
|mean error| + 4 std of the oracle's streams."""
import hashlib
import json
import os

import numpy as np
import pytest

from helpers import gpu_solver
from paper_2510_02635_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BOUNDS = os.path.join(ROOT, "tests", "golden", "closed_form_bounds.json")


def _bounds(w):
    ref = json.load(open(BOUNDS))
    src = hashlib.sha256(open(os.path.join(ROOT, "oracle", "fbsde_oracle.c"), "rb").read()).hexdigest()
    assert ref["oracle_source_sha256"] == src, "closed_form_bounds.json is stale: rerun its script"
    return ref["workloads"][w.name]


@pytest.mark.parametrize("w", [W.C2_AC_D10000, W.C1_LOGISTIC_D1000], ids=lambda w: w.name)
def test_gpu_error_against_closed_form_within_the_schemes_bound(w):
    b = _bounds(w)
    inp = W.inputs(w)
    out = gpu_solver(w, theta=inp["theta"]).solve(torch.tensor(inp["x0"], device="cuda"),
                                                  seed=w.seed)
    torch.cuda.synchronize()
    assert out["status"] == 0
    eu, eg = [], []
    for q in range(w.Q):
        us, gs = W.exact_solution(w, inp["x0"][q])
        eu.append(abs(float(out["u0"][q]) - us) / abs(us))
        eg.append(float(np.linalg.norm(out["grad"][q].cpu().numpy() - gs) / np.linalg.norm(gs)))
    assert max(eu) <= b["u"]["bound"], (max(eu), b["u"])
    assert max(eg) <= b["grad"]["bound"], (max(eg), b["grad"])
    # query 0 is the oracle's stream 0 itself: the GPU reproduces its error
    r0 = b["runs"][0]
    assert abs(float(out["u0"][0]) - r0["u0"]) <= 1e-4 * abs(r0["u0"])
