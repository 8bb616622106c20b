"""Host-side checks of the C ABI (no GPU needed).

* librexi.so builds for sm_103a and exports every function include/rexi.h declares;
* the library's double-double FCF construction (Algorithms 1-2) agrees with the
  oracle's 60-digit tables;
* the default R1 rule (largest R1 with 2 sigma_{K+1} <= 1e-9) gives the radii of
  the oracle tables;
* argument validation happens before any device call.
"""

import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import tables

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1912_03312_gb300 import build, _native
    build.build()
    return _native.load()


def header_functions():
    text = open(os.path.join(ROOT, "include", "rexi.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(rexi_\w+)\s*\(", text, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 15
    for nm in names:
        assert hasattr(lib, nm), nm


def test_debug_build_exports_the_same_symbols_and_says_so(lib):
    # librexi_debug.so (index checks in the Lanczos kernel) is the same ABI
    from paper_1912_03312_gb300 import _native as N
    dbg = C.CDLL(N.DEBUG_LIB_PATH)
    for nm in header_functions():
        assert hasattr(dbg, nm), nm
    dbg.rexi_debug_checks.restype = C.c_int
    assert dbg.rexi_debug_checks() == 1 and lib.rexi_debug_checks() == 0
    rec = (C.c_longlong * 4)()
    assert lib.rexi_plan_debug_record(None, rec) == N.REXI_EINVAL
    assert lib.rexi_plan_debug_trip(None, 1) == N.REXI_EINVAL
    assert "REXI_EBOUNDS" in N.status_string(N.REXI_EBOUNDS)


def test_binding_covers_header():
    from paper_1912_03312_gb300 import _native
    assert sorted(_native.SIGNATURES) == header_functions()


def test_struct_sizes_match_header(lib):
    # rexi_options_default writes sizeof(rexi_options) bytes: a canary after the
    # ctypes struct must survive.
    from paper_1912_03312_gb300 import _native as N

    class Guarded(C.Structure):
        _fields_ = [("o", N.Options), ("canary", C.c_uint64)]

    g = Guarded()
    g.canary = 0x5A5A5A5A5A5A5A5A
    assert lib.rexi_options_default(C.byref(g.o)) == 0
    assert g.canary == 0x5A5A5A5A5A5A5A5A
    assert g.o.restart_m == 30 and g.o.precision == N.REXI_MIXED and g.o.allow_substeps == 1


@pytest.mark.parametrize("K,R1", [(8, 8.0), (12, 14.0), (16, 10.0), (16, 24.0), (32, 68.0)])
def test_library_fcf_matches_oracle_tables(lib, K, R1):
    import paper_1912_03312_gb300 as R
    s, b, info = R.fcf(K, R1)
    so, bo, meta = tables.poles(K, R1)
    idx = [int(np.argmin(np.abs(so - x))) for x in s]
    assert len(set(idx)) == K
    assert np.max(np.abs(s - so[idx]) / np.abs(so[idx])) < 1e-13
    assert np.max(np.abs(b - bo[idx]) / np.abs(bo[idx])) < 1e-12
    assert abs(info["sigma_K1"] - meta["sigma_K+1"]) < 1e-6 * meta["sigma_K+1"]


def test_default_radius_rule(lib):
    import paper_1912_03312_gb300 as R
    assert R.fcf(16)[2]["R1"] == 24.0
    assert R.fcf(32)[2]["R1"] == 68.0


def test_status_strings(lib):
    from paper_1912_03312_gb300 import _native as N
    for code in (0, -1, -2, -3, -4, -5, -6, 1):
        assert N.status_string(code).startswith("REXI_")


def test_argument_validation_before_device(lib):
    from paper_1912_03312_gb300 import _native as N
    g = N.Grid()
    g.ndim = 1
    g.n[0] = 8
    g.lo[0] = -1.0
    g.hi[0] = 1.0
    g.hbar = 1.0
    g.mass = 1.0
    V = (C.c_double * 8)(*([0.0] * 8))
    h = C.c_void_p()
    assert lib.rexi_plan_create(C.byref(h), C.byref(g), V, 0.1, 0, None) == N.REXI_EINVAL      # K = 0
    assert lib.rexi_plan_create(C.byref(h), C.byref(g), V, -0.1, 4, None) == N.REXI_EINVAL     # dt < 0
    V[3] = float("nan")
    assert lib.rexi_plan_create(C.byref(h), C.byref(g), V, 0.1, 4, None) == N.REXI_EINVAL      # NaN in V
    V[3] = 0.0
    g.hi[0] = -2.0
    assert lib.rexi_plan_create(C.byref(h), C.byref(g), V, 0.1, 4, None) == N.REXI_EINVAL      # empty box
    g.hi[0] = 1.0
    o = N.Options()
    lib.rexi_options_default(C.byref(o))
    o.restart_m = 64
    assert lib.rexi_plan_create(C.byref(h), C.byref(g), V, 0.1, 4, C.byref(o)) == N.REXI_EINVAL
    o.restart_m = N.REXI_MAX_RESTART_FULL + 1  # full delayed CGS2 keeps m+1 dots in registers
    assert o.ortho == 1 and o.window == 0
    assert lib.rexi_plan_create(C.byref(h), C.byref(g), V, 0.1, 4, C.byref(o)) == N.REXI_EINVAL
    o.restart_m = N.REXI_MAX_RESTART + 1
    o.window = 2
    assert lib.rexi_plan_create(C.byref(h), C.byref(g), V, 0.1, 4, C.byref(o)) == N.REXI_EINVAL
    o.window = 0
    o.ortho = 2
    o.restart_m = 30
    assert lib.rexi_plan_create(C.byref(h), C.byref(g), V, 0.1, 4, C.byref(o)) == N.REXI_EINVAL
    o.ortho = 1
    o.window = 1                              # a window needs at least the two previous vectors
    assert lib.rexi_plan_create(C.byref(h), C.byref(g), V, 0.1, 4, C.byref(o)) == N.REXI_EINVAL
    o.window = 3
    o.ortho = 0                               # windows are a delayed-CGS2 option
    assert lib.rexi_plan_create(C.byref(h), C.byref(g), V, 0.1, 4, C.byref(o)) == N.REXI_EINVAL
    # the double-float recurrence is the Lanczos kernel's: the item engine refuses it
    o.window = 0
    o.restart_m = 30
    for ortho in (0, 1):
        o.ortho = ortho
        o.precision = N.REXI_DF64
        assert lib.rexi_plan_create(C.byref(h), C.byref(g), V, 0.1, 4, C.byref(o)) == N.REXI_EINVAL
    o.precision = 7                           # not a precision form
    assert lib.rexi_plan_create(C.byref(h), C.byref(g), V, 0.1, 4, C.byref(o)) == N.REXI_EINVAL
    # the Lanczos path (ortho = 2): FP64 or double-float, no window, Krylov dimension <= REXI_MAX_KRYLOV
    o.ortho = 2
    o.window = 0
    o.precision = N.REXI_MIXED
    assert lib.rexi_plan_create(C.byref(h), C.byref(g), V, 0.1, 4, C.byref(o)) == N.REXI_EINVAL
    o.precision = N.REXI_DF64
    o.window = 2
    assert lib.rexi_plan_create(C.byref(h), C.byref(g), V, 0.1, 4, C.byref(o)) == N.REXI_EINVAL
    o.precision = N.REXI_FP64
    o.window = 2
    assert lib.rexi_plan_create(C.byref(h), C.byref(g), V, 0.1, 4, C.byref(o)) == N.REXI_EINVAL
    o.window = 0
    o.restart_m = 513
    assert lib.rexi_plan_create(C.byref(h), C.byref(g), V, 0.1, 4, C.byref(o)) == N.REXI_EINVAL
    o.restart_m = 256
    o.ortho = 3
    assert lib.rexi_plan_create(C.byref(h), C.byref(g), V, 0.1, 4, C.byref(o)) == N.REXI_EINVAL
    assert h.value is None


def test_no_device_is_an_error_not_a_fallback(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1912_03312_gb300 import _native as N
    g = N.Grid()
    g.ndim = 1
    g.n[0] = 8
    g.lo[0] = -1.0
    g.hi[0] = 1.0
    g.hbar = 1.0
    g.mass = 1.0
    V = (C.c_double * 8)(*([0.0] * 8))
    h = C.c_void_p()
    assert lib.rexi_plan_create(C.byref(h), C.byref(g), V, 0.1, 8, None) == N.REXI_ECUDA


def test_grid_size_overflow_is_rejected_before_any_device_call(lib):
    # Three extents whose product exceeds 2^63 (and 2^30 long before): both
    # entry points that take a grid reject it with REXI_EINVAL before any
    # allocation, copy or launch, so a wrapped point count can never size a
    # buffer that the stencil then indexes past.
    from paper_1912_03312_gb300 import _native as N
    g = N.Grid()
    g.ndim = 3
    g.n[0], g.n[1], g.n[2] = 1 << 22, 1 << 22, 1 << 20
    for d in range(3):
        g.lo[d], g.hi[d] = -1.0, 1.0
    g.hbar = g.mass = 1.0
    V = (C.c_double * 8)(*([0.0] * 8))
    h = C.c_void_p()
    assert lib.rexi_plan_create(C.byref(h), C.byref(g), V, 0.1, 4, None) == N.REXI_EINVAL
    assert h.value is None
    o = N.Options()
    lib.rexi_options_default(C.byref(o))
    o.tol = 1e-12
    z = (C.c_double * 8)(*([0.0] * 8))
    a0 = (C.c_double * 2)(0.0, 0.0)
    dummy = C.c_void_p(16)                      # never dereferenced: validation comes first
    call = lambda grid, opt: lib.rexi_substep_static(C.byref(grid), dummy, 0.1, 0.0, 4, z, z, a0, opt,
                                                      dummy, dummy, None, None)
    assert call(g, C.byref(o)) == N.REXI_EINVAL
    # a grid whose extent is not finite, a missing or non-finite option set
    g.n[0], g.n[1], g.n[2] = 8, 8, 8
    g.hi[1] = float("inf")
    assert call(g, C.byref(o)) == N.REXI_EINVAL
    g.hi[1] = 1.0
    assert call(g, None) == N.REXI_EINVAL
    o.tol = float("nan")
    assert call(g, C.byref(o)) == N.REXI_EINVAL
    o.tol = 1e-12
    o.inner_tol = -1.0
    assert call(g, C.byref(o)) == N.REXI_EINVAL
    o.inner_tol = 1e-5
    o.precision = N.REXI_DF64                   # the allocation-free entry point runs the item engine
    assert call(g, C.byref(o)) == N.REXI_EINVAL


def test_binding_precision_names():
    # the Python option names map onto the header's precision forms; an
    # unknown name is refused before any call
    from paper_1912_03312_gb300 import _native as N
    from paper_1912_03312_gb300.rexi import options
    assert (N.REXI_FP64, N.REXI_MIXED, N.REXI_DF64) == (0, 1, 2)
    assert options(precision="fp64").precision == N.REXI_FP64
    assert options(precision="mixed").precision == N.REXI_MIXED
    assert options(precision="df64", ortho="lanczos").precision == N.REXI_DF64
    with pytest.raises(ValueError):
        options(precision="fp32")
