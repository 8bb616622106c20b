"""Parity of the Lanczos path with its recurrence in double-float pairs
(``precision="df64"``, ``ortho="lanczos"``) against the oracle, through the C ABI.

In that mode every vector of the three-term recurrence from u_1 on (the
stencil input on the tile's extended box, B u / f, the update's operands and
the stored basis) is a pair of floats per component and every operation runs on
the FP32 pipe; sweep 0 (the caller's state at any scale), the tridiagonal
matrix, the per-pole least squares, the combined coefficients and the input
state's term stay in FP64.  The recurrence's rounding (a few 2^-48 of each
result's largest term) enters psi' through the combined coefficients
sum_k alpha_k y_k, whose magnitudes sum to O(10), not through the individual
weights alpha_k (the pole-sum amplification A ~ 1e7 at K = 32): its effect is
near 1e-13, so the step bounds are those of the FP64 path, max(1e-10, 2 A tol),
and per-pole solutions agree with the oracle to 1e-10.

Cases: 1D/2D/3D grids, grids of equal spacings (every stencil ratio -1: the
unit neighbour pairs) and of unequal spacings (ratios as pairs), a dimension of
length 1 in x (the first stencil dimension is then y) and elsewhere, ragged and
wrapping tiles, resident tiles and streamed tiles (several tiles per CTA, the
basis read back from memory), several substeps, K = 8/16/32; states far outside
the FP32 range; the FP64 path on the same problems; one batched launch mixing
FP64 and double-float plans; graph capture.
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


def df_plan(g, V, dt, K, R1, tiles=None, **kw):
    lp = library_plan(g, V, dt, K, R1, ortho="lanczos", precision=kw.pop("precision", "df64"), **kw)
    if tiles == STREAMED:
        # more tiles than tile CTAs: every CTA streams several tiles per sweep
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        assert int(np.prod(g["n"])) > STREAMED[0] * (sms * STREAMED[1] - 1)
    if tiles is not None:
        from paper_1912_03312_gb300 import autotune
        autotune.apply(lp, {"pole_tile": 1024, "group_tile": tiles[0], "ctas_per_sm": tiles[1]})
    return lp


STREAMED = (256, 1)        # tile boxes of at most 256 points, one CTA per SM: several tiles per CTA on
                           # grids above 256 x (SMs - 1) points (asserted)

CASES = [                                              # grid, box, K, R1, dt, tiles
    ((300,), 8.0, 16, 24.0, 1.0, None),                # 1D, many substeps
    ((5000,), 250.0, 16, 24.0, 1.0, None),             # 1D, ragged tiles
    ((60000,), 3000.0, 16, 24.0, 1.0, STREAMED),       # the same spacing, streamed
    ((37,), 6.0, 8, 8.0, 0.3, None),                   # 1D, tiny
    ((130, 101), 8.0, 16, 24.0, 0.5, None),            # 2D, unequal spacings, ragged both ways
    ((250, 200), 15.0, 16, 24.0, 0.5, STREAMED),        # unequal spacings, streamed
    ((96, 80), 8.0, 32, 68.0, 0.5, None),              # 2D, K = 32
    ((64, 64), 8.0, 16, 24.0, 0.5, None),              # 2D, equal spacings (unit ratios)
    ((224, 224), 28.0, 16, 24.0, 0.5, STREAMED),        # equal spacings, streamed
    ((2, 17), 6.0, 8, 8.0, 0.3, None),                 # a dimension of length 2
    ((1, 40), 6.0, 8, 8.0, 0.3, None),                 # x of length 1: y is the first stencil dimension
    ((16, 12), 8.0, 16, 24.0, 0.5, None),              # tiles wrap on both sides
    ((20, 18, 14), 8.0, 16, 24.0, 0.3, None),          # 3D
    ((40, 36, 30), 16.0, 16, 24.0, 0.3, STREAMED),      # 3D, streamed
    ((12, 12, 12), 8.0, 16, 24.0, 0.3, None),          # 3D, equal spacings
    ((5, 1, 3), 6.0, 8, 8.0, 0.3, None),               # y of length 1
]


def _case_id(c):
    return "x".join(map(str, c[0])) + ("_streamed" if c[5] else "")


@pytest.mark.parametrize("n,box,K,R1,dt,tiles", CASES, ids=[_case_id(c) for c in CASES])
def test_df64_step_matches_oracle(n, box, K, R1, dt, tiles):
    g, V, psi = wl.random_problem(91, n, box=box)
    orc = OraclePlan(g, V, dt, K, R1)
    tol = solve_tol(orc.A * orc.n_sub)
    lp = df_plan(g, V, dt, K, R1, tiles, tol=tol)
    assert lp.info()["precision"] == 2
    out, st = lp.step(to_dev(psi), stats=True)
    assert st["status"] == 0 and st["n_sub"] == orc.n_sub
    ref, _ = ostep.step(V, orc.h, psi, orc.tau, orc.n_sub, orc.z, orc.alpha, orc.alpha0, tol=1e-14)
    bound = step_bound(orc.A * orc.n_sub, tol, "fp64")
    err = relerr(out.cpu().numpy(), ref)
    log_parity("lanczos_df64_step[%s,K%d]" % (_case_id((n, 0, 0, 0, 0, tiles)), K), err, bound, A=orc.A, tol=tol,
               iters=max(st["iters"]))
    assert err < bound, (err, bound)
    assert max(st["resid"]) <= tol
    # the same launch again is bitwise reproducible
    assert np.array_equal(lp.step(to_dev(psi)).cpu().numpy(), out.cpu().numpy())
    # and the FP64 recurrence on the same problem agrees to the same bound
    l64 = df_plan(g, V, dt, K, R1, tiles, tol=tol, precision="fp64")
    o64, st64 = l64.step(to_dev(psi), stats=True)
    assert st64["status"] == 0
    d = relerr(out.cpu().numpy(), o64.cpu().numpy())
    log_parity("lanczos_df64_vs_fp64[%s,K%d]" % (_case_id((n, 0, 0, 0, 0, tiles)), K), d, bound)
    assert d < bound, d


POLE_CASES = [CASES[0], CASES[4], CASES[5], CASES[7], CASES[12], CASES[13]]


@pytest.mark.parametrize("n,box,K,R1,dt,tiles", POLE_CASES, ids=[_case_id(c) for c in POLE_CASES])
def test_df64_solve_poles_match_oracle(n, box, K, R1, dt, tiles):
    g, V, psi = wl.random_problem(92, n, box=box)
    lp = df_plan(g, V, dt, K, R1, tiles, tol=1e-13)
    orc = OraclePlan(g, V, dt, K, R1)
    x, st = lp.solve_poles(to_dev(psi), stats=True)
    assert st["status"] == 0
    x = x.cpu().numpy()
    z, _, _, _ = lp.poles()
    worst = 0.0
    for k in range(K):
        kk = int(np.argmin(np.abs(orc.z - z[k])))
        xo, _ = ostep.solve_pole(V, orc.h, psi, orc.tau, orc.z[kk], tol=1e-14)
        worst = max(worst, relerr(x[k], xo))
        assert st["resid"][k] <= 1e-13
    log_parity("lanczos_df64_poles[%s,K%d]" % (_case_id((n, 0, 0, 0, 0, tiles)), K), worst, 1e-10)
    assert worst < 1e-10, worst


@pytest.mark.parametrize("tiles", [None, STREAMED])
@pytest.mark.parametrize("scale_exp", [-500, -200, 200, 450])
def test_df64_step_is_scale_invariant(scale_exp, tiles):
    # sweep 0 runs in FP64 on the caller's state and s_1 brings u_1 to unit
    # scale before it is rounded to pairs, so 2^e psi steps to 2^e times the
    # step of psi although 2^e psi is far outside the FP32 range
    n, box = ((250, 200), 15.0) if tiles == STREAMED else ((130, 101), 8.0)
    g, V, psi = wl.random_problem(95, n, box=box)
    K, R1, dt = 16, 24.0, 0.5
    lp = df_plan(g, V, dt, K, R1, tiles, tol=1e-13)
    ref, st = lp.step(to_dev(psi), stats=True)
    assert st["status"] == 0
    s = 2.0 ** scale_exp
    out, st2 = lp.step(to_dev(psi * s), stats=True)
    assert st2["status"] == 0 and abs(st2["total_iters"] - st["total_iters"]) <= K
    err = relerr(out.cpu().numpy() / s, ref.cpu().numpy())
    log_parity("lanczos_df64_scale[2^%d,%s]" % (scale_exp, "streamed" if tiles else "resident"), err, 1e-10)
    assert err < 1e-10, err


def test_df64_plane_wave_and_zero_state():
    # a plane wave on a constant potential is an eigenvector of H: the
    # recurrence breaks down after one column and the step is the scalar
    # rational function; the zero state steps to zero
    g = wl.make_grid((128, 128), (-8.0, -8.0), (8.0, 8.0))
    V0 = -0.4
    V = np.full((128, 128), V0)
    K, R1, dt = 16, 24.0, 0.5
    lp = df_plan(g, V, dt, K, R1, tol=1e-13)
    X = wl.coords(g)
    m = (3, -2)
    ph = sum(2 * np.pi * m[d] * (X[d] + 8.0) / 16.0 for d in range(2))
    wave = np.exp(1j * ph)
    out, st = lp.step(to_dev(wave), stats=True)
    assert st["status"] == 0
    h = 16.0 / 128
    lam = V0 + 0.5 * sum(2 - 2 * np.cos(2 * np.pi * m[d] / 128) for d in range(2)) / h ** 2
    zz, aa, a0, ns = lp.poles()
    r = a0 + np.sum(aa / (lp.info()["tau"] * lam - zz))
    wi = lp.info()
    bound = max(1e-9, 2.0 * wi["amplification"] * wi["tol"] * ns)
    err = relerr(out.cpu().numpy(), wave * r ** ns)
    log_parity("lanczos_df64_plane_wave", err, bound)
    assert err < bound
    oz, st = lp.step(torch.zeros_like(to_dev(wave)), stats=True)
    assert st["status"] == 0 and float(oz.abs().max()) == 0.0


def test_df64_batched_with_fp64_plans():
    # one launch of the Lanczos kernel with double-float and FP64 plans side by
    # side (each problem on its own CTAs, in its own arithmetic): against the
    # single launches of the same plans
    from paper_1912_03312_gb300 import step_batched
    plans, psis, bounds = [], [], []
    for i, (n, box, K, R1, dt, _) in enumerate([CASES[0], CASES[4], CASES[7], CASES[12], CASES[6]]):
        g, V, psi = wl.random_problem(150 + i, n, box=box)
        orc = OraclePlan(g, V, dt, K, R1)
        tol = solve_tol(orc.A * orc.n_sub)
        plans.append(df_plan(g, V, dt, K, R1, tol=tol, precision="df64" if i % 2 == 0 else "fp64"))
        psis.append(to_dev(psi))
        bounds.append(step_bound(orc.A * orc.n_sub, tol, "fp64"))
    singles = [p.step(x).cpu().numpy() for p, x in zip(plans, psis)]
    outs, sts = step_batched(plans, psis, stats=True)
    for i, (o, s, b) in enumerate(zip(outs, sts, bounds)):
        assert s["status"] == 0
        err = relerr(o.cpu().numpy(), singles[i])
        log_parity("lanczos_df64_batched[%d]" % i, err, b)
        assert err < b, (i, err, b)


def test_df64_step_captured_in_cuda_graph():
    g, V, psi = wl.random_problem(96, (96, 80), box=8.0)
    lp = df_plan(g, V, 0.5, 16, 24.0, tol=1e-12)
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


def test_df64_is_refused_outside_lanczos():
    # the double-float form is the Lanczos kernel's; the item engine refuses it
    from paper_1912_03312_gb300 import _native as N
    g, V, psi = wl.random_problem(97, (33, 20), box=6.0)
    with pytest.raises(N.RexiError) as e:
        library_plan(g, V, 0.3, 8, 8.0, precision="df64")
    assert e.value.code == N.REXI_EINVAL
