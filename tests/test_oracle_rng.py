"""Pins of the oracle's random-number stream (Philox4x32-10 + uniform map + Box-Muller).

The Brownian increments Delta W_k^j ~ N(0, dt I) of Eq. (2.7) are regenerated, not
stored, so both implementations derive them from the same counter-based generator.
These tests pin the oracle's generator to published known answers, to an
independent library implementation, and to the normal distribution.
"""
import ctypes
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    assert list(oracle.philox4x32_10(ctr, key)) == expect


def _curand_host():
    for path in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(path)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator():
    """cuRAND's host-side Philox4_32_10 generator (a library run, no GPU) emits, for
    seed s, blocks of 4 words equal to Philox(counter = (0, 0, n, 0), key = s)."""
    lib = _curand_host()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:  # PHILOX4_32_10
        pytest.skip("cuRAND host generator unavailable")
    try:
        seed = 0xFEDCBA9876543210
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n = 4 * 64
        out = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint)),
                                  ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for b in range(n // 4):
        assert list(oracle.philox4x32_10([0, 0, b, 0], key)) == list(out[4 * b:4 * b + 4])


def test_uniform_map_exact_in_binary32_and_open_interval():
    words = [0, 1, 511, 512, 0x7FFFFFFF, 0x80000000, 0xFFFFFE00, 0xFFFFFFFF, 0x12345678]
    for x in words:
        u = oracle.uniform(x)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u          # same value in FP32 and FP64
    assert oracle.uniform(0) == 2.0 ** -24
    assert oracle.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    # 512 consecutive words share one uniform value, the map is monotone in x >> 9
    assert oracle.uniform(0x1FF) == oracle.uniform(0)
    assert oracle.uniform(0x200) > oracle.uniform(0x1FF)


def test_normals_distribution():
    """Mean 0, variance 1, zero skew, kurtosis 3 and a Kolmogorov-Smirnov test."""
    scipy_stats = pytest.importorskip("scipy.stats")
    d = 1000
    z = np.concatenate([oracle.normals(11, s, k, j, d)
                        for s in range(2) for k in range(4) for j in range(25)])
    n = z.size
    assert abs(z.mean()) < 4.0 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 4.0 * math.sqrt(2.0 / n)
    assert abs(scipy_stats.skew(z)) < 4.0 * math.sqrt(6.0 / n)
    assert abs(scipy_stats.kurtosis(z)) < 4.0 * math.sqrt(24.0 / n)
    assert scipy_stats.kstest(z, "norm").pvalue > 1e-3


def test_normals_independent_across_counter_fields():
    """Streams for different dimension, particle, level, solve and seed are uncorrelated."""
    d = 4096
    base = oracle.normals(3, 1, 2, 5, d)
    others = [oracle.normals(3, 1, 2, 6, d),   # particle
              oracle.normals(3, 1, 3, 5, d),   # level
              oracle.normals(3, 2, 2, 5, d),   # solve
              oracle.normals(4, 1, 2, 5, d)]   # seed
    for o in others:
        assert abs(np.corrcoef(base, o)[0, 1]) < 4.0 / math.sqrt(d)
    # lag-1 correlation inside one vector (within and across Box-Muller pairs)
    assert abs(np.corrcoef(base[:-1], base[1:])[0, 1]) < 4.0 / math.sqrt(d)
    # ragged dimension counts are prefixes of the same stream
    assert np.array_equal(oracle.normals(3, 1, 2, 5, 7), base[:7])


def test_normals_use_the_documented_counter_layout():
    """Dimension i of particle j at level k of solve s uses counter (i // 4, j, k, s) and
    key (seed lo, seed hi); words (0,1) feed dimensions 4q, 4q+1 and words (2,3) feed
    4q+2, 4q+3 (each pair shares the Box-Muller radius sqrt(-2 ln u))."""
    seed, s, k, j, d = 0x1122334455667788, 7, 3, 11, 12
    z = oracle.normals(seed, s, k, j, d)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for q in range(3):
        w = oracle.philox4x32_10([q, j, k, s], key)
        for pair in range(2):
            r2 = -2.0 * math.log(oracle.uniform(int(w[2 * pair])))
            zz = z[4 * q + 2 * pair: 4 * q + 2 * pair + 2]
            assert zz[0] ** 2 + zz[1] ** 2 == pytest.approx(r2, rel=1e-12)
