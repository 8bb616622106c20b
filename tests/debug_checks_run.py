"""Runs the Lanczos kernel of the index-checked build (librexi_debug.so) on the
parity cases and on every check site made to fail; prints one JSON line.

Started by tests/test_gpu_debug_checks.py in a child process with REXI_DEBUG=1
(the binding then loads the checked build).  Exit status 0 when:

* every case (the recurrence in FP64, and in double-float pairs on resident
  and streamed tiles) runs with status 0, no failed check recorded, and the step (or
  each pole's solution) agrees with the oracle to the bounds of the release
  tests: steps to max(1e-10, 2 A tol), poles to 1e-10;
* a batched launch of several of these problems (each on its share of the
  CTAs) runs with no failed check and agrees with the single launches;
* for every check site s = 1 .. 11 made to fail (rexi_plan_debug_trip), the
  launch ends with REXI_EBOUNDS and the record names s; afterwards the same
  plan, with no site tripped, reproduces the clean result bit for bit.
"""

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import ctypes as C  # noqa: E402

import torch  # noqa: E402

import workloads as wl  # noqa: E402
from oracle import step as ostep  # noqa: E402
from _common import OraclePlan, library_plan, relerr, solve_tol, step_bound, to_dev  # noqa: E402

from paper_1912_03312_gb300 import _native as N  # noqa: E402
from paper_1912_03312_gb300 import autotune  # noqa: E402

STEP_CASES = [                              # grid, box, K, R1, dt, tiles (group_tile, ctas_per_sm)
    ((300,), 8.0, 16, 24.0, 1.0, None),
    ((60000,), 3000.0, 16, 24.0, 1.0, (256, 1)),    # several tiles per CTA (streamed)
    ((130, 101), 8.0, 16, 24.0, 0.5, None),
    ((130, 101), 8.0, 16, 24.0, 0.5, (256, 1)),
    ((96, 80), 8.0, 32, 68.0, 0.5, None),
    ((2, 17), 6.0, 8, 8.0, 0.3, None),
    ((16, 12), 8.0, 16, 24.0, 0.5, None),
    ((20, 18, 14), 8.0, 16, 24.0, 0.3, None),
    ((20, 18, 14), 8.0, 16, 24.0, 0.3, (256, 2)),
    ((5, 1, 3), 6.0, 8, 8.0, 0.3, None),
]
# the recurrence in double-float pairs (precision "df64"): resident and
# streamed tiles, unequal and equal spacings
DF_CASES = [
    ((130, 101), 8.0, 16, 24.0, 0.5, None),
    ((250, 200), 15.0, 16, 24.0, 0.5, (256, 1)),    # streamed (more tiles than CTAs)
    ((64, 64), 8.0, 16, 24.0, 0.5, None),
    ((60000,), 3000.0, 16, 24.0, 1.0, (256, 1)),    # streamed
    ((40, 36, 30), 16.0, 16, 24.0, 0.3, (256, 1)),  # streamed
    ((12, 12, 12), 8.0, 16, 24.0, 0.3, None),
]
POLE_CASES = [((130, 101), 8.0, 16, 24.0, 0.5), ((20, 18, 14), 8.0, 16, 24.0, 0.3)]


def record(lp):
    rec = (C.c_longlong * 4)()
    N.check(N.load().rexi_plan_debug_record(lp.handle, rec), "rexi_plan_debug_record")
    return [int(v) for v in rec]


def plan(g, V, dt, K, R1, tiles=None, precision="fp64", **kw):
    lp = library_plan(g, V, dt, K, R1, precision=precision, ortho="lanczos", **kw)
    if tiles is not None:
        autotune.apply(lp, {"pole_tile": 1024, "group_tile": tiles[0], "ctas_per_sm": tiles[1]})
    return lp


def main():
    torch.cuda.set_device(0)
    lib = N.load()
    assert N.LIB_PATH == N.DEBUG_LIB_PATH and lib.rexi_debug_checks() == 1, "not the index-checked build"
    out = {"steps": [], "poles": [], "trips": []}
    cases = [c + ("fp64",) for c in STEP_CASES] + [c + ("df64",) for c in DF_CASES]
    for n, box, K, R1, dt, tiles, prec in cases:
        g, V, psi = wl.random_problem(91, n, box=box)
        orc = OraclePlan(g, V, dt, K, R1)
        tol = solve_tol(orc.A * orc.n_sub)
        lp = plan(g, V, dt, K, R1, tiles, precision=prec, tol=tol)
        res, st = lp.step(to_dev(psi), stats=True)
        rec = record(lp)
        ref, _ = ostep.step(V, orc.h, psi, orc.tau, orc.n_sub, orc.z, orc.alpha, orc.alpha0, tol=1e-14)
        err = relerr(res.cpu().numpy(), ref)
        bound = step_bound(orc.A * orc.n_sub, tol, "fp64")
        out["steps"].append({"case": "x".join(map(str, n)), "tiles": tiles, "precision": prec,
                             "status": st["status"], "record": rec, "err": err, "bound": bound})
        assert st["status"] == 0 and rec == [0, 0, 0, 0], (n, tiles, st["status"], rec)
        assert err < bound, (n, tiles, err, bound)
    for n, box, K, R1, dt in POLE_CASES:
        g, V, psi = wl.random_problem(92, n, box=box)
        orc = OraclePlan(g, V, dt, K, R1)
        lp = plan(g, V, dt, K, R1, tol=1e-13)
        x, st = lp.solve_poles(to_dev(psi), stats=True)
        rec = record(lp)
        assert st["status"] == 0 and rec == [0, 0, 0, 0], (n, st["status"], rec)
        x = x.cpu().numpy()
        z, _, _, _ = lp.poles()
        worst = 0.0
        for k in range(K):
            kk = int(np.argmin(np.abs(orc.z - z[k])))
            xo, _ = ostep.solve_pole(V, orc.h, psi, orc.tau, orc.z[kk], tol=1e-14)
            worst = max(worst, relerr(x[k], xo))
        out["poles"].append({"case": "x".join(map(str, n)), "max_err": worst})
        assert worst < 1e-10, (n, worst)
    # several problems in one batched launch (each on its own range of CTAs)
    from paper_1912_03312_gb300 import step_batched
    bplans, bpsis, bsingle, bbound = [], [], [], []
    for i, (n, box, K, R1, dt, tiles) in enumerate(STEP_CASES[:6]):
        g, V, psi = wl.random_problem(140 + i, n, box=box)
        orc = OraclePlan(g, V, dt, K, R1)
        tol = solve_tol(orc.A * orc.n_sub)
        lp = plan(g, V, dt, K, R1, precision="df64" if i % 2 else "fp64", tol=tol)
        bplans.append(lp)
        bpsis.append(to_dev(psi))
        bsingle.append(lp.step(to_dev(psi)).cpu().numpy())
        bbound.append(step_bound(orc.A * orc.n_sub, tol, "fp64"))
    bouts, bsts = step_batched(bplans, bpsis, stats=True)
    for i, (o, st_, lp) in enumerate(zip(bouts, bsts, bplans)):
        rec = record(lp)
        assert st_["status"] == 0 and rec == [0, 0, 0, 0], (i, st_["status"], rec)
        assert relerr(o.cpu().numpy(), bsingle[i]) < bbound[i], i
    out["batched"] = {"problems": len(bplans), "records": "clean"}
    # every site made to fail (FP64 and double-float recurrences): REXI_EBOUNDS
    # with the site recorded, then recovery
    g, V, psi = wl.random_problem(94, (130, 101), box=8.0)
    for prec in ("fp64", "df64"):
        lp = plan(g, V, 0.5, 16, 24.0, precision=prec, tol=1e-13)
        clean = lp.step(to_dev(psi)).cpu().numpy()
        assert lp.step(to_dev(psi), stats=True)[1]["status"] == 0
        for site in sorted(N.LZ_SITES):
            N.check(lib.rexi_plan_debug_trip(lp.handle, site), "rexi_plan_debug_trip")
            try:
                lp.step(to_dev(psi), stats=True)
                code = 0
            except N.RexiError as e:
                code = e.code
            rec = record(lp)
            N.check(lib.rexi_plan_debug_trip(lp.handle, 0), "rexi_plan_debug_trip")
            again = lp.step(to_dev(psi)).cpu().numpy()
            out["trips"].append({"precision": prec, "site": site, "name": N.LZ_SITES[site], "status": code,
                                 "record": rec, "recovered": bool(np.array_equal(again, clean))})
            assert code == N.REXI_EBOUNDS and rec[0] == site and rec[3] >= 1, (prec, site, code, rec)
            assert np.array_equal(again, clean), (prec, site)
    # a site out of range and a plan of the item engine are refused
    assert lib.rexi_plan_debug_trip(lp.handle, len(N.LZ_SITES) + 1) == N.REXI_EINVAL
    le = library_plan(g, V, 0.5, 16, 24.0, precision="fp64")
    assert lib.rexi_plan_debug_trip(le.handle, 1) == N.REXI_EINVAL
    print(json.dumps(out))


if __name__ == "__main__":
    main()
