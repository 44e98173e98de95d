"""Host logic of the continuous-batching server (paper_2110_03732_gb300/serve.py) that
needs no GPU: the per-request device-memory estimate that admission charges against
the HBM budget, and the shortest-remaining-work-first choice of the bulk lane."""
import os
import shutil

import pytest

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


@pytest.fixture(scope="module")
def serve():
    from paper_2110_03732_gb300 import build
    build.build()
    from paper_2110_03732_gb300 import serve as S
    return S


def test_request_bytes_counts_state_scratch_and_fields(serve):
    from paper_2110_03732_gb300 import grmhd
    from paper_2110_03732_gb300 import problems as P
    for pr in (P.orszag_tang(64), P.orszag_tang(128), P.shock_tube(400), P.star(32)):
        N = pr.N
        ncell = N[0] * N[1] * N[2]
        g = grmhd.make_grid(pr.ndim, pr.n, pr.lo, pr.hi, pr.bc)
        scratch = grmhd.scratch_bytes(g, grmhd.ssp2())
        extra = (2 if pr.alpha is not None else 0) + (1 if pr.eta is not None else 0)
        assert serve.request_bytes(pr) == 8 * ncell * (11 + extra) + scratch
        # the scratch alone holds more than the state: stage bases, fluxes, EMFs, history
        assert scratch > 11 * 8 * ncell
    # a 4x larger grid needs about 4x the memory
    r = serve.request_bytes(P.orszag_tang(256)) / serve.request_bytes(P.orszag_tang(128))
    assert 3.5 < r < 4.5
    # the metric arrays of the star are charged
    st = P.star(32)
    assert st.alpha is not None


class _Bulk:
    def __init__(self, runs):
        self.runs = list(runs)
        self.dirty = False


def _run(rid, cells, left):
    return {"rid": rid, "cells": cells, "left": left}


def test_select_takes_shortest_remaining_work_within_the_cell_cap(serve):
    s = serve.Server(budget_bytes=1e9, device="cpu", bulk_cells=1000)
    a, b, c, d = _run(0, 600, 10), _run(1, 300, 5), _run(2, 500, 1), _run(3, 200, 50)
    bulk = _Bulk([a, b])
    rest = s._select(bulk, [c, d])
    # work = cells x steps left: c 500, b 1500, a 6000, d 10000.  c and b fit (800 cells),
    # a would exceed 1000, d (200 more) still fits
    assert [r["rid"] for r in bulk.runs] == [2, 1, 3]
    assert bulk.dirty
    assert sorted(r["rid"] for r in rest) == [0]


def test_select_always_takes_the_first_run_and_keeps_an_unchanged_batch_clean(serve):
    s = serve.Server(budget_bytes=1e9, device="cpu", bulk_cells=100)
    big = _run(0, 5000, 3)
    bulk = _Bulk([big])
    rest = s._select(bulk, [])
    # a run larger than the cap still runs (alone), and re-selecting it changes nothing
    assert [r["rid"] for r in bulk.runs] == [0]
    assert not bulk.dirty
    assert rest == []
    later = _run(1, 10, 100)
    rest = s._select(bulk, [later])
    # 5000 x 3 = 15000 against 10 x 100 = 1000: the small run goes first, then the big one
    # no longer fits under the cap and waits
    assert [r["rid"] for r in bulk.runs] == [1]
    assert bulk.dirty
    assert [r["rid"] for r in rest] == [0]
