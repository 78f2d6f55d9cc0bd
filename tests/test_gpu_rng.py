"""GPU random stream vs the oracle: Philox4x32-10 words bit for bit, normals within
the rounding of the stream precision (FP32 logf/sincospif vs FP64 log/cos)."""
import os

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


@pytest.fixture(scope="module")
def fb():
    from paper_2510_02635_gb300 import fbsde
    fbsde.load_library()
    return fbsde


def _gpu_philox(fb, ctr, key):
    c = torch.tensor(np.asarray(ctr, dtype=np.uint32).view(np.int32), device="cuda")
    k = torch.tensor(np.asarray(key, dtype=np.uint32).view(np.int32), device="cuda")
    out = torch.zeros_like(c)
    fb.check(fb.fbsde_philox4x32_10(c, k, out))
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


def test_philox_known_answers_on_gpu(fb):
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        v = [int(t, 16) for t in line.split()]
        out = _gpu_philox(fb, [v[0:4]], v[4:6])
        assert list(out[0]) == v[6:10]


def test_philox_bit_exact_against_oracle(fb):
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:16] = np.arange(64, dtype=np.uint32).reshape(16, 4)   # small counters too
    key = rng.integers(0, 2 ** 32, size=2, dtype=np.uint64).astype(np.uint32)
    out = _gpu_philox(fb, ctr, key)
    for i in range(ctr.shape[0]):
        assert np.array_equal(out[i], oracle.philox4x32_10(ctr[i], key)), i


@pytest.mark.parametrize("prec,tol", [("fp32", 4e-6), ("fp64", 1e-13)])
@pytest.mark.parametrize("d", [1, 7, 100, 1001])
def test_normals_match_oracle(fb, prec, tol, d):
    seed, s, k, j0, nj = 0x0123456789ABCDEF, 5, 3, 17, 40
    dt = torch.float32 if prec == "fp32" else torch.float64
    out = torch.empty(nj, d, dtype=dt, device="cuda")
    fb.check(fb.fbsde_normals(seed, s, k, j0, nj, d, prec, out))
    torch.cuda.synchronize()
    z = out.double().cpu().numpy()
    ref = np.stack([oracle.normals(seed, s, k, j0 + jj, d) for jj in range(nj)])
    err = np.abs(z - ref) / (1.0 + np.abs(ref))
    assert err.max() <= tol
