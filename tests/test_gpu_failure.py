"""Failure detection on the device without a GPU fault: every device-side wait
of the engine (grid barriers, bulk-copy completions) is bounded.  With the
plan's wait limit set to 1 ns, the CTAs that wait at a grid barrier give up
at once: the launch ends with REXI_ETIMEOUT instead of hanging, and the same
plan then steps normally with the default limit (the context stays usable,
and the result is bitwise the one of a launch before the failure)."""

import numpy as np
import pytest

import workloads as wl

from _common import library_plan, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_03312_gb300 import build
    build.build()


def test_wait_limit_expiry_reports_timeout_and_plan_recovers():
    from paper_1912_03312_gb300 import _native as N
    g, V, psi = wl.random_problem(95, (130, 101), box=8.0)
    lp = library_plan(g, V, 0.5, 16, 24.0, precision="fp64", tol=1e-13, window=2, restart=64)
    x = to_dev(psi)
    ref = lp.step(x).cpu().numpy()
    cheb_ref, _ = lp.cheb_step(x, tol=1e-12)
    cheb_ref = cheb_ref.cpu().numpy()

    lp.set_timeout(1e-9)
    with pytest.raises(N.RexiError) as e:
        lp.step(x, stats=True)
    assert e.value.code == N.REXI_ETIMEOUT
    lp.cheb_step(x, tol=1e-12)                       # asynchronous: the status reports it
    assert lp.last_status() == N.REXI_ETIMEOUT

    lp.set_timeout(0.0)                              # back to the default limit
    out, st = lp.step(x, stats=True)
    assert st["status"] == 0 and lp.last_status() == 0
    assert np.array_equal(out.cpu().numpy(), ref)
    c2, _ = lp.cheb_step(x, tol=1e-12)
    assert lp.last_status() == 0
    assert np.array_equal(c2.cpu().numpy(), cheb_ref)


def test_wait_limit_validation():
    from paper_1912_03312_gb300 import _native as N
    g, V, psi = wl.random_problem(96, (40, 30), box=6.0)
    lp = library_plan(g, V, 0.5, 8, 8.0)
    for bad in (float("nan"), 7200.0):
        with pytest.raises(N.RexiError) as e:
            lp.set_timeout(bad)
        assert e.value.code == N.REXI_EINVAL
    lp.set_timeout(10.0)
    lp.set_timeout(-1.0)
