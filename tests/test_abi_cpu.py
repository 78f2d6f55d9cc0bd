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
    assert fbsde.fbsde_abi_version() == 3
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
                                 dict(precision="fp64", d=10241)])
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


def test_anchored_workspace_sizing(lib):
    """Three M x M stream-precision matrices dominate at large M (the rest is O(M d) plus
    the M^2/64 column-pass partials); M beyond 32768 (or below 2) and invalid problems
    give 0."""
    for M in (2048, 16384):
        n = fbsde.fbsde_anchored_workspace_bytes(_prob(M=M))
        assert n >= 3 * M * M * 4
    n16 = fbsde.fbsde_anchored_workspace_bytes(_prob(M=16384))
    assert n16 < 1.1 * 3 * 16384 ** 2 * 4
    n32 = fbsde.fbsde_anchored_workspace_bytes(_prob(M=32768))
    assert 3.8 < n32 / n16 < 4.1
    assert fbsde.fbsde_anchored_workspace_bytes(_prob(M=2048, precision="fp64")) >= 3 * 2048 ** 2 * 8
    assert fbsde.fbsde_anchored_workspace_bytes(_prob(M=32768)) > 0
    for bad in (dict(M=32769), dict(M=1), dict(sigma=0.0), dict(d=0)):
        assert fbsde.fbsde_anchored_workspace_bytes(_prob(**bad)) == 0


def test_anchored_argument_errors_return_synchronously(lib):
    p = _prob(M=256)
    n = fbsde.fbsde_anchored_workspace_bytes(p)
    fake, unaligned = C.c_void_p(1 << 20), C.c_void_p((1 << 20) + 8)
    L = lib
    assert L.fbsde_solve_anchored(C.byref(p), 1, None, 0, 0, fake, None, fake, n, None) == 1
    assert L.fbsde_solve_anchored(C.byref(p), 1, fake, 0, 0, None, None, fake, n, None) == 1
    assert L.fbsde_solve_anchored(C.byref(p), 0, fake, 0, 0, fake, None, fake, n, None) == 1
    ph = _prob(kind="hjb_logquad", M=256)
    assert L.fbsde_solve_anchored(C.byref(ph), 1, fake, 0, 0, fake, None, fake, 1 << 40, None) == 1
    assert L.fbsde_solve_anchored(C.byref(p), 1, fake, 0, 0, fake, None, None, n, None) == 2
    assert L.fbsde_solve_anchored(C.byref(p), 1, fake, 0, 0, fake, None, fake, n - 1, None) == 2
    assert L.fbsde_solve_anchored(C.byref(p), 1, fake, 0, 0, fake, None, unaligned, n, None) == 2


def test_adjoint_workspace_and_argument_errors(lib):
    """The adjoint workspace holds the solve's plus the tape; theta_bar only for kinds with
    terminal coefficients; theta required for them; workspace checks as for the solve."""
    p = _prob(M=512, N=6)
    ns, na = fbsde.fbsde_workspace_bytes(p, 2), fbsde.fbsde_adjoint_workspace_bytes(p, 2)
    assert na > ns
    assert na - ns >= 6 * 2 * 512 * 4   # per level and query: the M taped weights at least
    assert fbsde.fbsde_adjoint_workspace_bytes(_prob(sigma=-1.0), 1) == 0
    fake, L = C.c_void_p(1 << 20), lib
    args = lambda pr, **kw: [C.byref(pr), 1, kw.get("x0", fake), 0, 0, kw.get("ub", fake), fake,
                             None, kw.get("xb", fake), kw.get("tb"), kw.get("ws", fake),
                             kw.get("n", 1 << 40), None]
    assert L.fbsde_adjoint(*args(p, x0=None)) == 1
    assert L.fbsde_adjoint(*args(p, ub=None)) == 1
    assert L.fbsde_adjoint(*args(p, xb=None)) == 1
    assert L.fbsde_adjoint(*args(p, tb=fake)) == 1            # no theta in this kind
    assert L.fbsde_adjoint(*args(_prob(kind="hjb_logquad"))) == 1   # theta missing
    na1 = fbsde.fbsde_adjoint_workspace_bytes(p, 1)   # the calls above and below use Q = 1
    assert L.fbsde_adjoint(*args(p, ws=None)) == 2
    assert L.fbsde_adjoint(*args(p, n=na1 - 1)) == 2
    assert L.fbsde_adjoint(*args(p, ws=C.c_void_p((1 << 20) + 16), n=na1)) == 2


def test_plan_workspace_is_the_aligned_sum_of_the_instances(lib):
    fake = (1 << 20)
    pa, pb = _prob(M=512), _prob(d=37, M=300, precision="fp64")
    arr = (fbsde.fbsde_instance * 2)()
    arr[0] = fbsde.fbsde_instance(pa, 2, 0, 1, fake, fake, None)
    arr[1] = fbsde.fbsde_instance(pb, 1, 0, 2, fake, fake, fake)
    total = int(lib.fbsde_plan_workspace_bytes(2, arr))
    a, b = fbsde.fbsde_workspace_bytes(pa, 2), fbsde.fbsde_workspace_bytes(pb, 1)
    up = lambda x: (x + 255) // 256 * 256
    assert total == up(up(a) + b)
    assert int(lib.fbsde_plan_workspace_bytes(0, arr)) == 0
    arr[1] = fbsde.fbsde_instance(pb, 1, 0, 2, None, fake, None)   # x0 missing
    assert int(lib.fbsde_plan_workspace_bytes(2, arr)) == 0
    h = C.c_void_p()
    assert lib.fbsde_plan_create(None, 1, arr, 0, None, 0) == 1
    assert lib.fbsde_plan_create(C.byref(h), 1, arr, 0, None, 0) == 2
    assert lib.fbsde_plan_create(C.byref(h), 1, arr, 0, C.c_void_p(fake), up(a) - 1) == 2
    assert h.value is None


def test_batch_argument_errors_return_synchronously(lib):
    p = _prob(M=256)
    n = fbsde.fbsde_anchored_workspace_bytes(p)
    fake = C.c_void_p(1 << 20)
    for K in (1, 0, 257, -5):
        assert lib.fbsde_solve_batch(C.byref(p), K, 1, fake, 0, 0, fake, None, fake, n, None) == 1
    assert lib.fbsde_solve_batch(C.byref(p), 64, 1, None, 0, 0, fake, None, fake, n, None) == 1
    assert lib.fbsde_solve_batch(C.byref(p), 64, 1, fake, 0, 0, fake, None, fake, n - 1, None) == 2
    assert lib.fbsde_solve_batch(None, 64, 1, fake, 0, 0, fake, None, fake, n, None) == 1


def test_direct_batch_argument_errors_return_synchronously(lib):
    """The direct form takes the batch form's checks, and also needs d <= 128 and a positive
    ridge (the ridge bounds every pivot of its factorisation below)."""
    fake = C.c_void_p(1 << 20)
    p = _prob(M=256)
    n = fbsde.fbsde_anchored_workspace_bytes(p)
    for K in (1, 0, 257):
        assert lib.fbsde_solve_batch_direct(C.byref(p), K, 1, fake, 0, 0, fake, None, fake, n,
                                            None) == 1
    assert lib.fbsde_solve_batch_direct(C.byref(p), 64, 1, fake, 0, 0, fake, None, fake, n - 1,
                                        None) == 2
    for bad in (dict(d=fbsde.FBSDE_BATCH_DIRECT_MAX_D + 1), dict(ridge_rel=0.0)):
        pb = _prob(M=256, **bad)
        nb = fbsde.fbsde_anchored_workspace_bytes(pb)
        assert nb > 0   # the CG form takes these problems
        assert lib.fbsde_solve_batch_direct(C.byref(pb), 64, 1, fake, 0, 0, fake, None, fake, nb,
                                            None) == 1


def test_forward_sde_workspace_and_argument_checks(lib):
    """A drift, a state-dependent diffusion or a drift kind adds the stored levels of the
    Euler-Maruyama rows (checkpoints every s = ceil(sqrt N) levels below N plus one segment
    of s - 1 levels) and the anchor offsets [Q][N+1][ld]; the driftless problem is
    unchanged.  HJB_LOGQUAD needs sig1 = 0, the coefficients must be finite, and the
    adjoint and per-anchor entry points take only the driftless scheme."""
    Q, d, M, N = 2, 100, 2048, 10
    base = fbsde.fbsde_workspace_bytes(_prob(d=d, M=M, N=N), Q)
    s = math.ceil(math.sqrt(N))
    slots = (N - 1) // s + s - 1
    slab = Q * M * d * 4
    for kw in (dict(mu0=0.1), dict(mu1=-0.5), dict(sig1=0.2), dict(kind="drift_ac"),
               dict(kind="drift_quad")):
        n = fbsde.fbsde_workspace_bytes(_prob(d=d, M=M, N=N, **kw), Q)
        # (the driftless FP32 problem sizes its partials for the fused step; the drift
        # path does not use it, so the rest of the layout differs by a little)
        assert slots * slab < n - base <= slots * slab + 2 * Q * (N + 1) * d * 4 + 4096
    # FP64 (no fused step either way): exactly the stored slabs plus the anchor offsets
    up = lambda x: (x + 255) // 256 * 256
    for N1, slots1 in ((1, 0), (2, 1), (4, 2), (9, 4), (10, 5), (17, 7)):
        n0 = fbsde.fbsde_workspace_bytes(_prob(d=d, M=M, N=N1, precision="fp64"), Q)
        n1 = fbsde.fbsde_workspace_bytes(_prob(d=d, M=M, N=N1, precision="fp64", mu1=-1.0), Q)
        assert n1 - n0 == up(slots1 * Q * M * d * 8) + up(Q * (N1 + 1) * d * 8), N1
    assert fbsde.fbsde_workspace_bytes(_prob(kind="hjb_logquad", sig1=0.1), 1) == 0
    assert fbsde.fbsde_workspace_bytes(_prob(kind="hjb_logquad", mu0=0.1), 1) > 0
    for bad in (dict(mu0=math.nan), dict(mu1=math.inf), dict(sig1=-math.inf)):
        assert fbsde.fbsde_workspace_bytes(_prob(**bad), 1) == 0
    assert fbsde.fbsde_anchored_workspace_bytes(_prob(mu1=-0.3)) == 0
    assert fbsde.fbsde_anchored_workspace_bytes(_prob(kind="drift_ac")) == 0
    fake = C.c_void_p(1 << 20)
    p = _prob(mu0=0.2)
    assert lib.fbsde_adjoint(C.byref(p), 1, fake, 0, 0, fake, fake, None, fake, None, fake,
                             1 << 40, None) == 1


def test_bounded_wait_check_argument_errors(lib):
    """Argument errors of the wait check return before any CUDA call."""
    fake = C.c_void_p(1 << 20)
    assert lib.fbsde_check_bounded_wait(0, fake, None, None) == 1
    assert lib.fbsde_check_bounded_wait(2_000_000_000, fake, None, None) == 1
    assert lib.fbsde_check_bounded_wait(1000, None, None, None) == 1
    assert lib.fbsde_check_bounded_wait(1000, C.c_void_p((1 << 20) + 4), None, None) == 1


@pytest.mark.parametrize("argv", [["--K", "64"], ["--anchored", "--direct"], ["--direct"]])
def test_cli_rejects_batch_options_without_their_form(argv):
    """The CLI's batch options apply to the per-anchor form only: --K needs --anchored and
    --direct needs --K (an argument error before any device work)."""
    with pytest.raises(SystemExit) as e:
        fbsde._main(argv)
    assert e.value.code == 2
