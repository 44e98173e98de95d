"""The seeded synthetic workloads (paper_2110_03732_gb300/problems.py) are
reproducible and follow their recipes: the batched Orszag-Tang set (sides from the
given list, eta log-uniform in its range, phases in [0, 2 pi)) and the Poisson request
stream (increasing arrivals at the given mean rate, the three kinds, step counts)."""
import math

import numpy as np

from paper_2110_03732_gb300 import problems as P


def test_ot_batch_is_seeded_and_follows_its_recipe():
    a = P.ot_batch(seed=0, n_boxes=6, sizes=(8, 16, 24))
    b = P.ot_batch(seed=0, n_boxes=6, sizes=(8, 16, 24))
    c = P.ot_batch(seed=1, n_boxes=6, sizes=(8, 16, 24))
    assert [p.n for p in a] == [p.n for p in b]
    assert [p.eta_u for p in a] == [p.eta_u for p in b]
    for pa, pb in zip(a, b):
        for x, y in zip(pa.prim, pb.prim):
            assert np.array_equal(x, y)
    assert [p.eta_u for p in a] != [p.eta_u for p in c]
    for p in a:
        assert p.ndim == 2 and p.n[0] == p.n[1] and p.n[0] in (8, 16, 24)
        assert 1e-6 <= p.eta_u <= 1.0


def test_request_stream_is_seeded_poisson_with_three_kinds():
    kw = dict(n_requests=60, rate=400.0, tube_cells=(100, 160), vortex_side=(8, 12), star_side=(6, 8))
    r1 = P.request_stream(3, **kw)
    r2 = P.request_stream(3, **kw)
    assert [(t, s) for t, _, s in r1] == [(t, s) for t, _, s in r2]
    times = np.array([t for t, _, _ in r1])
    assert np.all(np.diff(times) > 0)
    # mean inter-arrival of 60 exponential gaps at 400/s: 2.5 ms within 4 standard errors
    gaps = np.diff(np.concatenate([[0.0], times]))
    assert abs(gaps.mean() - 1 / 400.0) < 4 * (1 / 400.0) / math.sqrt(len(gaps))
    kinds = {p.ndim for _, p, _ in r1}
    assert kinds == {1, 2, 3}
    for _, p, steps in r1:
        assert steps >= 1
        if p.ndim == 1:
            assert 100 <= p.n[0] <= 160
            # run to t = 0.4 at the CFL step of the tube
            dt = p.cfl * (p.hi[0] - p.lo[0]) / p.n[0]
            assert (steps - 1) * dt < p.t_end <= steps * dt + 1e-12
        else:
            assert steps == 100
