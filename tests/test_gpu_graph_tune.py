"""CUDA-graph capture of the persistent launch, and the autotuner.

* rexi_step (no statistics) only enqueues memsets and one cooperative launch,
  so it can be captured in a CUDA graph; replays must reproduce the eager result.
* rexi_step_batched likewise.
* Every tile/occupancy setting gives the same step up to summation order.
"""

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


def test_step_captured_in_cuda_graph():
    g, V, psi = wl.random_problem(81, (96, 80), box=8.0)
    lp = library_plan(g, V, 0.5, 16, 24.0, precision="mixed", tol=1e-12)
    x = to_dev(psi)
    eager = lp.step(x).clone()
    out = torch.empty_like(x)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        lp.step(x, out=out)                          # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        lp.step(x, out=out)
    for _ in range(2):
        out.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, eager)


def test_batched_captured_in_cuda_graph():
    from paper_1912_03312_gb300 import step_batched
    plans, ins, eager = [], [], []
    for i, n in enumerate([(64, 48), (40,), (20, 16, 12)]):
        g, V, psi = wl.random_problem(82 + i, n, box=8.0)
        lp = library_plan(g, V, 0.4, 16, 24.0, precision="mixed", tol=1e-12)
        plans.append(lp)
        ins.append(to_dev(psi))
        eager.append(lp.step(ins[-1]).clone())
    outs = [torch.empty_like(t) for t in ins]
    step_batched(plans, ins, outs)                  # builds the cached descriptor set
    torch.cuda.synchronize()
    eager_b = [o.clone() for o in outs]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step_batched(plans, ins, outs)
    for o in outs:
        o.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for o, eb, e, lp in zip(outs, eager_b, eager, plans):
        assert torch.equal(o, eb)                   # the replay is the batched launch, bit for bit
        # against the single-problem launches: same solves, reductions split differently
        A = lp.info()["amplification"]
        assert relerr(o.cpu().numpy(), e.cpu().numpy()) < max(1e-6, 2.0 * A * 1e-12)


def test_tile_settings_agree_and_autotune(tmp_path, monkeypatch):
    from paper_1912_03312_gb300 import autotune
    monkeypatch.setenv("REXI_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    g, V, psi = wl.random_problem(85, (200, 150), box=10.0)
    lp = library_plan(g, V, 0.5, 16, 24.0, precision="mixed", tol=1e-13)
    x = to_dev(psi)
    ref = lp.step(x).cpu().numpy()
    A = lp.info()["amplification"]
    for pt, gt, c in [(256, 256, 1), (1024, 2048, 2), (2048, 512, 0), (1792, 1536, 1), (768, 1280, 0)]:
        autotune.apply(lp, {"pole_tile": pt, "group_tile": gt, "ctas_per_sm": c})
        got = lp.step(x).cpu().numpy()
        assert relerr(got, ref) < max(1e-6, 2.0 * A * 1e-13)
    # the FP64 windowed path (direct pole sum) under the same settings
    lw = library_plan(g, V, 0.5, 16, 24.0, precision="fp64", tol=1e-13, window=2, restart=64)
    refw = lw.step(x).cpu().numpy()
    for pt, gt, c in [(1792, 1792, 1), (1024, 1536, 2), (256, 512, 0)]:
        autotune.apply(lw, {"pole_tile": pt, "group_tile": gt, "ctas_per_sm": c})
        assert relerr(lw.step(x).cpu().numpy(), refw) < max(1e-10, 2.0 * A * 1e-13)
    with pytest.raises(Exception):
        autotune.apply(lw, {"pole_tile": 300, "group_tile": 512, "ctas_per_sm": 0})   # not a multiple of 256
    cfg = autotune.autotune(lp, x, steps=1)
    assert not cfg["cached"] and cfg["ms"] > 0
    cfg2 = autotune.autotune(lp, x, steps=1)
    assert cfg2["cached"] and cfg2["pole_tile"] == cfg["pole_tile"]
