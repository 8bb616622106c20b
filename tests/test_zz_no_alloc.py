"""The allocation-free entry point rexi_substep_static, through the C ABI.

Some callers cannot allocate device memory (code inside an allocator callback,
hosts that reserve all GPU memory up front, sandboxes without cudaMalloc).  For
them the library runs one rational evaluation with its workspace in a fixed
static device array.  This test checks that call against the ordinary plan
entry point (rexi_step on a plan with one substep) on two calls in a row, with
the tolerance of the step parity tests, and that an oversized problem is
rejected.  It lives in its own file, collected last, and passes alone or after
the other tests.
"""

import ctypes as C

import numpy as np
import pytest

import workloads as wl

from _common import library_plan, relerr, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_03312_gb300 import build
    build.build()


def _static_call(lp, V_dev, psi_in, psi_out, tol, precision):
    from paper_1912_03312_gb300 import _native as N
    lib = N.load()
    info = lp.info()
    z, alpha, a0, ns = lp.poles()
    zz = np.ascontiguousarray(z.view(np.float64))
    aa = np.ascontiguousarray(alpha.view(np.float64))
    a0a = np.array([a0.real, a0.imag])
    o = N.Options()
    lib.rexi_options_default(C.byref(o))
    o.precision = N.REXI_MIXED if precision == "mixed" else N.REXI_FP64
    o.tol = tol
    st = N.Stats()
    dptr = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.rexi_substep_static(C.byref(lp.grid), C.c_void_p(V_dev.data_ptr()), info["tau"], info["c"], lp.K,
                                 dptr(zz), dptr(aa), dptr(a0a), C.byref(o), C.c_void_p(psi_in.data_ptr()),
                                 C.c_void_p(psi_out.data_ptr()), stream, C.byref(st))
    return rc, st


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_static_substep_matches_plan_step_twice(precision):
    g, V, psi = wl.random_problem(71, (64, 48), box=8.0)
    _, _, psi2 = wl.random_problem(72, (64, 48), box=8.0)
    K, R1, dt, tol = 16, 24.0, 0.5, 1e-13
    lp = library_plan(g, V, dt, K, R1, precision=precision, tol=tol)
    info = lp.info()
    assert info["n_sub"] == 1
    bound = max(1e-10 if precision == "fp64" else 1e-6, 2.0 * info["amplification"] * tol)
    V_dev = torch.from_numpy(np.ascontiguousarray(V, dtype=np.float64)).cuda()
    for state in (psi, psi2):                      # two calls in a row share the static workspace
        ref = lp.step(to_dev(state)).cpu().numpy()
        x_in = to_dev(state)
        x_out = torch.empty_like(x_in)
        rc, st = _static_call(lp, V_dev, x_in, x_out, tol, precision)
        assert rc == 0 and st.status == 0, (rc, st.status)
        assert relerr(x_out.cpu().numpy(), ref) < bound


def test_static_substep_in_place():
    # psi_in and psi_out may be the same buffer: the call reads the state into
    # its workspace before it writes the result.  In place and out of place run
    # the same launch, so the results are equal bit for bit.
    g, V, psi = wl.random_problem(73, (64, 48), box=8.0)
    K, R1, dt, tol = 16, 24.0, 0.5, 1e-13
    lp = library_plan(g, V, dt, K, R1, precision="fp64", tol=tol)
    V_dev = torch.from_numpy(np.ascontiguousarray(V, dtype=np.float64)).cuda()
    x_in = to_dev(psi)
    x_out = torch.empty_like(x_in)
    rc, st = _static_call(lp, V_dev, x_in, x_out, tol, "fp64")
    assert rc == 0 and st.status == 0
    buf = to_dev(psi)
    rc, st = _static_call(lp, V_dev, buf, buf, tol, "fp64")
    assert rc == 0 and st.status == 0
    assert np.array_equal(buf.cpu().numpy(), x_out.cpu().numpy())
    info = lp.info()
    ref = lp.step(to_dev(psi)).cpu().numpy()
    assert relerr(buf.cpu().numpy(), ref) < max(1e-10, 2.0 * info["amplification"] * tol)


def test_static_substep_rejects_oversized_problem():
    from paper_1912_03312_gb300 import _native as N
    g = wl.make_grid((512, 512), (-30.0, -30.0), (30.0, 30.0))
    V = np.zeros((512, 512))
    lp = library_plan(wl.make_grid((32, 32), (-30.0, -30.0), (30.0, 30.0)), np.zeros((32, 32)), 0.5, 32, 68.0)
    V_dev = torch.from_numpy(V).cuda()
    psi = torch.zeros((512, 512), dtype=torch.complex128, device="cuda")
    big = lp.grid.__class__()
    big.ndim = 2
    big.n[0] = big.n[1] = 512
    big.lo[0] = big.lo[1] = -30.0
    big.hi[0] = big.hi[1] = 30.0
    big.hbar = big.mass = 1.0
    lib = N.load()
    z = np.zeros(64)
    a0 = np.zeros(2)
    o = N.Options()
    lib.rexi_options_default(C.byref(o))
    o.tol = 1e-12
    dptr = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    rc = lib.rexi_substep_static(C.byref(big), C.c_void_p(V_dev.data_ptr()), 0.25, 0.0, 32, dptr(z), dptr(z),
                                 dptr(a0), C.byref(o), C.c_void_p(psi.data_ptr()), C.c_void_p(psi.data_ptr()),
                                 None, None)
    assert rc == N.REXI_EINVAL
    del g
