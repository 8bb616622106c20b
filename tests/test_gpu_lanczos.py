"""Parity of the shared-basis Lanczos path (``ortho="lanczos"``) against the
oracle, through the C ABI.

That path is a kernel of its own: one Krylov basis per substep for all K poles,
built by the three-term recurrence of tau (H - c) with real coefficients, the
update recomputed on every tile's halo so one grid barrier per step suffices,
per-pole Givens least squares on the shared basis (control CTA), and the pole
sum as one pass over the basis.  Cases: 1D/2D/3D grids, degenerate dimensions
(length 1 and 2), tiles that wrap on both sides, ragged tiles, K = 8/16/32,
several substeps; per-pole solutions to 1e-10; steps to max(1e-10, 2 A tol)
with tol chosen so that bound stays below the metric's 1e-6; plane wave and
zero state at 512^2; states far outside the FP32 range (scale invariance);
NaN input, too few iterations, the bounded waits, graph
capture, reproducibility, in place, host buffers, the adjoint on the item
engine, tile settings, and several problems in one batched launch.
"""

import numpy as np
import pytest

import workloads as wl
from oracle import step as ostep

from _common import OraclePlan, library_plan, log_parity, relerr, solve_tol, step_bound, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_03312_gb300 import build
    build.build()


def lz_plan(g, V, dt, K, R1, **kw):
    kw.setdefault("precision", "fp64")
    return library_plan(g, V, dt, K, R1, ortho="lanczos", **kw)


CASES = [                                   # grid, box, K, R1, dt
    ((300,), 8.0, 16, 24.0, 1.0),           # 1D, many substeps
    ((5000,), 250.0, 16, 24.0, 1.0),        # 1D, ragged tiles
    ((37,), 6.0, 8, 8.0, 0.3),              # 1D, tiny
    ((130, 101), 8.0, 16, 24.0, 0.5),       # 2D, ragged in both directions
    ((96, 80), 8.0, 32, 68.0, 0.5),         # 2D, K = 32
    ((2, 17), 6.0, 8, 8.0, 0.3),            # a dimension of length 2
    ((33, 20), 6.0, 8, 8.0, 0.3),
    ((16, 12), 8.0, 16, 24.0, 0.5),         # tiles wrap on both sides
    ((20, 18, 14), 8.0, 16, 24.0, 0.3),     # 3D
    ((9, 7, 5), 8.0, 8, 8.0, 0.2),
    ((5, 1, 3), 6.0, 8, 8.0, 0.3),          # a dimension of length 1
]


@pytest.mark.parametrize("n,box,K,R1,dt", CASES)
def test_lanczos_step_matches_oracle(n, box, K, R1, dt):
    g, V, psi = wl.random_problem(91, n, box=box)
    orc = OraclePlan(g, V, dt, K, R1)
    tol = solve_tol(orc.A * orc.n_sub)
    lp = lz_plan(g, V, dt, K, R1, tol=tol)
    out, st = lp.step(to_dev(psi), stats=True)
    assert st["status"] == 0 and st["n_sub"] == orc.n_sub
    ref, _ = ostep.step(V, orc.h, psi, orc.tau, orc.n_sub, orc.z, orc.alpha, orc.alpha0, tol=1e-14)
    bound = step_bound(orc.A * orc.n_sub, tol, "fp64")
    err = relerr(out.cpu().numpy(), ref)
    log_parity("lanczos_step[%s,K%d]" % ("x".join(map(str, n)), K), err, bound, A=orc.A, tol=tol,
               iters=max(st["iters"]))
    assert err < bound, (err, bound)
    # every pole stopped on its bound within the plan's tolerance
    assert max(st["resid"]) <= tol
    # the same launch again is bitwise reproducible
    assert np.array_equal(lp.step(to_dev(psi)).cpu().numpy(), out.cpu().numpy())


@pytest.mark.parametrize("n,box,K,R1,dt", [CASES[0], CASES[3], CASES[4], CASES[8], CASES[10]])
def test_lanczos_solve_poles_match_oracle(n, box, K, R1, dt):
    g, V, psi = wl.random_problem(92, n, box=box)
    lp = lz_plan(g, V, dt, K, R1, tol=1e-13)
    orc = OraclePlan(g, V, dt, K, R1)
    x, st = lp.solve_poles(to_dev(psi), stats=True)
    assert st["status"] == 0
    x = x.cpu().numpy()
    z, _, _, _ = lp.poles()
    for k in range(K):
        kk = int(np.argmin(np.abs(orc.z - z[k])))
        xo, _ = ostep.solve_pole(V, orc.h, psi, orc.tau, orc.z[kk], tol=1e-14)
        err = relerr(x[k], xo)
        log_parity("lanczos_pole[%s,K%d,%d]" % ("x".join(map(str, n)), K, k), err, 1e-10)
        assert err < 1e-10, (k, err)
        assert st["resid"][k] <= 1e-13


@pytest.mark.parametrize("scale_exp", [-500, -200, 200, 450])
def test_lanczos_step_is_scale_invariant(scale_exp):
    # psi of any finite norm: sweep 0 forms its inner products in FP64 (the
    # later vectors are normalised), so 2^e psi steps to 2^e times the step
    # of psi, far outside the FP32 range of the compensated products
    g, V, psi = wl.random_problem(95, (130, 101), box=8.0)
    K, R1, dt = 16, 24.0, 0.5
    lp = lz_plan(g, V, dt, K, R1, tol=1e-13)
    ref, st = lp.step(to_dev(psi), stats=True)
    assert st["status"] == 0
    s = 2.0 ** scale_exp
    out, st2 = lp.step(to_dev(psi * s), stats=True)
    # the same Krylov columns up to the rounding of the rescaled vectors
    assert st2["status"] == 0 and abs(st2["total_iters"] - st["total_iters"]) <= K
    err = relerr(out.cpu().numpy() / s, ref.cpu().numpy())
    log_parity("lanczos_scale[2^%d]" % scale_exp, err, 1e-13)
    assert err < 1e-13, err


def test_lanczos_tiles_and_grid_settings_agree():
    # the result does not depend on the tile box or the CTAs per SM beyond the
    # summation order of the inner products
    from paper_1912_03312_gb300 import autotune
    g, V, psi = wl.random_problem(93, (200, 150), box=8.0)
    K, R1, dt = 16, 24.0, 0.5
    orc = OraclePlan(g, V, dt, K, R1)
    tol = solve_tol(orc.A * orc.n_sub)
    lp = lz_plan(g, V, dt, K, R1, tol=tol)
    outs = []
    for gt, cps in ((2048, 2), (512, 2), (1024, 1), (256, 1)):
        autotune.apply(lp, {"pole_tile": 1024, "group_tile": gt, "ctas_per_sm": cps})
        o, st = lp.step(to_dev(psi), stats=True)
        assert st["status"] == 0
        outs.append(o.cpu().numpy())
    bound = step_bound(orc.A * orc.n_sub, tol, "fp64")
    for o in outs[1:]:
        assert relerr(o, outs[0]) < bound


def test_lanczos_plane_wave_and_zero_state_512():
    # A plane wave is an eigenvector: the shared recurrence breaks down after
    # one step (||u_1|| at rounding level) and every pole stops on its first
    # column; the step multiplies the wave by the scalar of Eq. (4)-(5).  The
    # zero state stops before any column and stays exactly zero.
    n = (512, 512)
    g = wl.make_grid(n, (-30.0, -30.0), (30.0, 30.0))
    V = np.full((512, 512), -0.8)
    lp = lz_plan(g, V, 0.5, 32, 68.0)
    X = wl.coords(g)
    mx, my = -7, 4
    psi = np.exp(1j * (2 * np.pi * mx * (X[0] + 30.0) / 60.0 + 2 * np.pi * my * (X[1] + 30.0) / 60.0))
    out, st = lp.step(to_dev(psi), stats=True)
    assert st["status"] == 0
    z, alpha, a0, ns = lp.poles()
    h = 60.0 / 512
    lam = -0.8 + 0.5 * ((2 - 2 * np.cos(2 * np.pi * mx / 512)) + (2 - 2 * np.cos(2 * np.pi * my / 512))) / h ** 2
    tau = lp.info()["tau"]
    r = a0 + np.sum(alpha / (tau * lam - z))
    info = lp.info()
    out = out.cpu().numpy()
    assert np.all(np.isfinite(out))
    bound = max(1e-9, 2.0 * info["amplification"] * info["tol"] * ns)
    err = relerr(out, psi * r ** ns)
    log_parity("lanczos_plane_wave_512", err, bound)
    assert err < bound
    assert max(st["iters"]) <= 40 * ns
    zero, stz = lp.step(torch.zeros_like(to_dev(psi)), stats=True)
    assert stz["status"] == 0 and float(zero.abs().max()) == 0.0


def test_lanczos_in_place_and_host_buffers_agree():
    g, V, psi = wl.random_problem(94, (64, 48), box=8.0)
    lp = lz_plan(g, V, 0.5, 16, 24.0, tol=1e-12)
    a = lp.step(to_dev(psi)).cpu().numpy()
    buf = to_dev(psi)
    lp.step(buf, out=buf)
    assert np.array_equal(a, buf.cpu().numpy())
    assert np.array_equal(a, lp.step_host(psi))


def test_lanczos_failures_are_reported_and_plan_recovers():
    from paper_1912_03312_gb300._native import RexiError
    g, V, psi = wl.random_problem(95, (64, 40), box=8.0)
    lp = lz_plan(g, V, 0.5, 16, 24.0, tol=1e-13)
    good = lp.step(to_dev(psi)).cpu().numpy()
    bad = psi.copy()
    bad[3, 4] = np.nan
    with pytest.raises(RexiError) as e:
        lp.step(to_dev(bad), stats=True)
    assert e.value.code == -4                       # REXI_ENOCONV
    # too small a Krylov dimension
    short = lz_plan(g, V, 0.5, 16, 24.0, tol=1e-13, max_iters=3)
    with pytest.raises(RexiError) as e:
        short.step(to_dev(psi), stats=True)
    assert e.value.code == -4
    # bounded waits that run out: REXI_ETIMEOUT, then the plan steps again
    lp.set_timeout(1e-9)
    with pytest.raises(RexiError) as e:
        lp.step(to_dev(psi), stats=True)
    assert e.value.code == -5
    lp.set_timeout(0.0)
    again, st = lp.step(to_dev(psi), stats=True)
    assert st["status"] == 0 and np.array_equal(again.cpu().numpy(), good)


def test_lanczos_step_captured_in_cuda_graph():
    g, V, psi = wl.random_problem(96, (96, 80), box=8.0)
    lp = lz_plan(g, V, 0.5, 16, 24.0, tol=1e-12)
    x = to_dev(psi)
    eager = lp.step(x).clone()
    out = torch.empty_like(x)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        lp.step(x, out=out)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        lp.step(x, out=out)
    for _ in range(2):
        out.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, eager)


def test_lanczos_plan_adjoint_and_batched_rules():
    # the adjoint of a Lanczos plan runs on the item engine (allocated at its
    # first call); the batched call rejects Lanczos plans
    from paper_1912_03312_gb300 import step_batched
    from paper_1912_03312_gb300._native import RexiError
    g, V, psi = wl.random_problem(97, (40, 36), box=8.0)
    K, R1, dt = 16, 24.0, 0.5
    lp = lz_plan(g, V, dt, K, R1, tol=1e-13)
    orc = OraclePlan(g, V, dt, K, R1)
    rng = np.random.default_rng(3)
    G = rng.normal(size=psi.shape) + 1j * rng.normal(size=psi.shape)
    dV = torch.zeros(lp.n, dtype=torch.float64, device="cuda")
    gin = lp.step_backward(to_dev(psi), to_dev(G), dV)
    Go = G.copy()
    states = ostep.evolve(V, orc.h, psi, orc.tau, orc.n_sub, 1, orc.z, orc.alpha, orc.alpha0, tol=1e-14)
    dVo = np.zeros(V.shape)
    for s_ in range(orc.n_sub - 1, -1, -1):
        Go, dvs = ostep.substep_adjoint(V, orc.h, states[s_], Go, orc.tau, orc.z, orc.alpha, orc.alpha0, tol=1e-14)
        dVo += dvs
    bound = max(1e-9, 2.0 * orc.A * 1e-13 * orc.n_sub)
    assert relerr(gin.cpu().numpy(), Go) < bound
    assert relerr(dV.cpu().numpy().reshape(V.shape), dVo) < 10 * bound
    # forward still on the Lanczos kernel after the adjoint workspace exists
    out, st = lp.step(to_dev(psi), stats=True)
    assert st["status"] == 0
    # a batch must not mix Lanczos and item-engine plans, nor repeat a plan
    le = library_plan(g, V, dt, K, R1, precision="fp64", tol=1e-13)
    for plans in ([lp, le], [le, lp], [lp, lp]):
        with pytest.raises(RexiError):
            step_batched(plans, [to_dev(psi)] * len(plans))


def test_lanczos_batched_matches_singles_and_oracle():
    # several problems (1D, 2D, 3D; K = 16 and 32; different substep counts)
    # in one launch of the Lanczos kernel, each on its share of the CTAs:
    # every step agrees with the problem's single launch and with the oracle
    # to the step bound, repeats bit for bit, and leaves the plans usable alone
    from paper_1912_03312_gb300 import step_batched
    cases = [((300,), 8.0, 16, 24.0, 1.0), ((130, 101), 8.0, 16, 24.0, 0.5), ((96, 80), 8.0, 32, 68.0, 0.5),
             ((20, 18, 14), 8.0, 16, 24.0, 0.3), ((64, 48), 8.0, 16, 24.0, 0.5), ((2, 17), 6.0, 8, 8.0, 0.3)]
    plans, psis, singles, refs, bounds = [], [], [], [], []
    for i, (n, box, K, R1, dt) in enumerate(cases):
        g, V, psi = wl.random_problem(130 + i, n, box=box)
        orc = OraclePlan(g, V, dt, K, R1)
        tol = solve_tol(orc.A * orc.n_sub)
        lp = lz_plan(g, V, dt, K, R1, tol=tol)
        plans.append(lp)
        psis.append(to_dev(psi))
        singles.append(lp.step(to_dev(psi)).cpu().numpy())
        refs.append(ostep.step(V, orc.h, psi, orc.tau, orc.n_sub, orc.z, orc.alpha, orc.alpha0, tol=1e-14)[0])
        bounds.append(step_bound(orc.A * orc.n_sub, tol, "fp64"))
    outs, sts = step_batched(plans, psis, stats=True)
    for i, (o, s_, r, b) in enumerate(zip(outs, sts, refs, bounds)):
        assert s_["status"] == 0, (i, s_["status"])
        o = o.cpu().numpy()
        err = relerr(o, r)
        log_parity("lanczos_batched[%s]" % "x".join(map(str, cases[i][0])), err, b)
        assert err < b, (i, err, b)
        assert relerr(o, singles[i]) < b, i
    again = step_batched(plans, psis)
    assert all(np.array_equal(a.cpu().numpy(), o.cpu().numpy()) for a, o in zip(again, outs))
    for lp, p_, s1 in zip(plans, psis, singles):
        assert np.array_equal(lp.step(p_).cpu().numpy(), s1)


def test_lanczos_work_counts():
    # the kernel's own count of the algorithmic bytes and FP64 flops matches
    # the per-sweep formula for the Krylov dimensions it reports
    g, V, psi = wl.random_problem(98, (128, 96), box=8.0)
    lp = lz_plan(g, V, 0.5, 16, 24.0, tol=1e-13)
    out, st = lp.step(to_dev(psi), stats=True)
    assert st["status"] == 0
    assert st["bytes"] > 0 and st["flops64"] > 0
    n = 128 * 96
    # at least one sweep of 40 bytes per point per substep and the pole sums
    assert st["bytes"] >= st["n_sub"] * n * (40 + 32)
