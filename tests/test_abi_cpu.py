"""The C-ABI library builds, loads and exports every entry point of include/fbsde.h;
its host-side argument checks and workspace sizing behave as documented.  No test
here launches GPU work (argument errors return before any CUDA call)."""
import ctypes as C
import math
import os
import re

import pytest

from paper_2510_02635_gb300 import build as gbuild
from paper_2510_02635_gb300 import fbsde

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fbsde.h")


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return fbsde.load_library()


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"FBSDE_API\s+[\w\s\*]+?\b(fbsde_\w+)\s*\(", text)))


def test_every_declared_entry_point_is_exported(lib):
    names = _declared()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(fbsde.EXPORTS)


def test_binding_constants_match_the_header():
    text = open(HEADER).read()
    for name in ("FBSDE_PROFILED_EAGER_PASSES", "FBSDE_NOALLOC_MAX_BYTES", "FBSDE_MAX_D",
                 "FBSDE_MAX_D_FP64"):
        m = re.search(r"#define\s+" + name + r"\s+\(?(\d+)u?(?:\s*<<\s*(\d+))?", text)
        assert m, name
        val = int(m.group(1)) << int(m.group(2) or 0)
        assert getattr(fbsde, name) == val, name
    m = re.search(r"FBSDE_NUM_KERNELS\s*=\s*(\d+)", text)
    assert int(m.group(1)) == fbsde.FBSDE_NUM_KERNELS


def test_abi_version_and_status_strings(lib):
    assert fbsde.fbsde_abi_version() == 1
    assert fbsde.fbsde_status_string(0) == "ok"
    assert "argument" in fbsde.fbsde_status_string(1)
    assert fbsde.fbsde_status_string(99) == "unknown status"


def _prob(**kw):
    base = dict(kind="ac_manufactured", d=100, N=10, M=2048, sigma=1.0, T=0.5)
    base.update(kw)
    return fbsde.make_problem(**base)


def test_workspace_sizing(lib):
    p = _prob()
    n1 = fbsde.fbsde_workspace_bytes(p, 1)
    n4 = fbsde.fbsde_workspace_bytes(p, 4)
    assert n1 >= 2048 * 100 * 4 and n4 >= 4 * 2048 * 100 * 4 and n4 > n1
    p64 = _prob(precision="fp64")
    assert fbsde.fbsde_workspace_bytes(p64, 1) >= 2048 * 100 * 8
    big = _prob(d=10000, M=16384, N=50)
    assert fbsde.fbsde_workspace_bytes(big, 16) >= 16 * 16384 * 10000 * 4
    assert fbsde.fbsde_workspace_bytes(big, 16) < 16 * 16384 * 10000 * 4 * 1.05
    assert fbsde.fbsde_host_staging_bytes(p, 3) >= 3 * 100 * 8 * 2


@pytest.mark.parametrize("bad", [dict(d=0), dict(d=fbsde.FBSDE_MAX_D + 1), dict(M=1),
                                 dict(N=0), dict(sigma=0.0), dict(sigma=math.nan), dict(T=-1.0),
                                 dict(cg_tol=0.0), dict(ridge_rel=-1.0),
                                 dict(precision="fp64", d=9000)])
def test_invalid_problems_are_rejected(lib, bad):
    p = _prob(**bad)
    assert fbsde.fbsde_workspace_bytes(p, 1) == 0


def test_invalid_kind_precision_and_count(lib):
    p = _prob()
    p.kind = 42
    assert fbsde.fbsde_workspace_bytes(p, 1) == 0
    p = _prob()
    p.precision = 7
    assert fbsde.fbsde_workspace_bytes(p, 1) == 0
    assert fbsde.fbsde_workspace_bytes(_prob(), 0) == 0


def test_solve_argument_errors_return_synchronously(lib):
    p = _prob()
    L = lib
    # missing x0 / u0 -> FBSDE_ERR_ARG; missing or small workspace -> FBSDE_ERR_WORKSPACE
    assert L.fbsde_solve(C.byref(p), 1, None, 0, 0, None, None, None, None, 0, None) == 1
    fake = C.c_void_p(256)
    assert L.fbsde_solve(C.byref(p), 1, fake, 0, 0, fake, None, None, None, 0, None) == 2
    assert L.fbsde_solve(C.byref(p), 1, fake, 0, 0, fake, None, None, fake, 16, None) == 2
    unaligned = C.c_void_p(257)
    n = fbsde.fbsde_workspace_bytes(p, 1)
    assert L.fbsde_solve(C.byref(p), 1, fake, 0, 0, fake, None, None, unaligned, n, None) == 2
    # kinds that read theta need it
    ph = _prob(kind="hjb_logquad")
    assert L.fbsde_solve(C.byref(ph), 1, fake, 0, 0, fake, None, None, fake, 1 << 40, None) == 1
    assert L.fbsde_solve(None, 1, fake, 0, 0, fake, None, None, fake, 1 << 40, None) == 1
    assert L.fbsde_philox4x32_10(None, None, None, 4, None) == 1
    assert L.fbsde_normals(0, 0, 0, 0, 4, 0, 0, fake, None) == 1
    assert L.fbsde_normals(0, 0, 0, 0, 4, 8, 3, fake, None) == 1
