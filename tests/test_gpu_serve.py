"""Serving loop: requests arriving over time are admitted under a device-memory
budget, advanced together in batched launches while others keep running, and each
result equals the same run served alone (bitwise: the batched kernels compute every
problem independently).  A second check: the loop never holds more than its budget
while a run is active."""
import math

import pytest

from paper_2110_03732_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def small_stream(seed=3, n=9):
    reqs = P.request_stream(seed, n, rate=400.0, tube_cells=(100, 160), vortex_side=(24, 48), star_side=(14, 20),
                            steps_2d3d=12)
    from paper_2110_03732_gb300.serve import Request
    out = []
    for i, (t, pr, steps) in enumerate(reqs):
        out.append(Request(i, t, pr, steps, t_end=pr.t_end if pr.ndim == 1 else None))
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_served_results_equal_alone(precision):
    from paper_2110_03732_gb300 import build, serve
    build.build()
    reqs = small_stream()
    srv = serve.Server(budget_bytes=60e6, precision=precision, keep_results=True)
    results, stats = srv.run(reqs, realtime=True)
    assert stats["requests"] == len(reqs)
    assert stats["peak_bytes"] <= 60e6 or stats["peak_bytes"] == max(serve.request_bytes(r.problem) for r in reqs)
    by_id = {r.rid: r for r in results}
    for req in reqs:
        ref = serve.run_alone(req, precision=precision)
        got = by_id[req.rid].state
        for a, b in zip(got, ref):
            assert torch.equal(a, b), (precision, req.rid, req.problem.name)
    assert stats["p50_tts_s"] > 0 and stats["p99_tts_s"] >= stats["p50_tts_s"]


def test_budget_limits_concurrency():
    from paper_2110_03732_gb300 import build, serve
    build.build()
    reqs = small_stream(seed=5, n=6)
    one = max(serve.request_bytes(r.problem) for r in reqs)
    srv = serve.Server(budget_bytes=1.5 * one, precision="fp64")
    results, stats = srv.run(reqs, realtime=False)
    assert stats["requests"] == len(reqs)
    assert stats["peak_bytes"] <= 1.5 * one
