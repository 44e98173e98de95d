"""The window construction used by the full-size GPU parity tests, checked on the
oracle alone: the oracle stepped on a window of a problem reproduces, in the window's
core, the oracle stepped on the whole problem.  This pins the dependency radius the
windows assume (an IMEX-SSP2 step reaches at most 6 cells; the core keeps 14 cells
from every cut side for two steps) and the cropping of the padded arrays, edge
potentials and metric."""
import numpy as np
import pytest

import oracle
from parity_tools import padded, window, window_core
from paper_2110_03732_gb300 import problems as P


@pytest.fixture(scope="module")
def star64():
    pr = P.star(n=64)
    st = oracle.from_problem(pr)
    dt = oracle.cfl_dt(st.grid, pr.cfl, pr.alpha, pr.psi)
    for _ in range(2):
        st.step(dt)
    return pr, st, dt


@pytest.mark.parametrize("start", [(14, 14, 14), (0, 0, 0), (28, 0, 14)])
def test_window_core_equals_whole_problem(star64, start):
    pr, st, dt = star64
    size = (36, 36, 36)
    wp = window(pr, start, size)
    ws = oracle.from_problem(wp)
    for _ in range(2):
        ws.step(dt)
    loc, glob = window_core(pr, start, size, 2)
    Iw, Ig = padded(loc, wp.ng), padded(glob, pr.ng)
    assert ws.fails == 0 and st.fails == 0
    for v in range(8):
        a, b = ws.q[v][Iw], st.q[v][Ig]
        assert a.size >= 8 ** 3
        assert np.abs(a - b).max() <= 1e-14 * max(np.abs(b).max(), 1e-300), v
    for d in range(3):
        a, b = ws.bf[d][Iw], st.bf[d][Ig]
        assert np.abs(a - b).max() <= 1e-14 * max(np.abs(b).max(), 1e-300), d


def test_window_too_close_to_a_cut_side_differs(star64):
    """The check above has teeth: cells next to a cut side do differ from the whole
    problem's after two steps (the window's outflow ghosts are not the neighbours)."""
    pr, st, dt = star64
    start, size = (14, 14, 14), (36, 36, 36)
    wp = window(pr, start, size)
    ws = oracle.from_problem(wp)
    for _ in range(2):
        ws.step(dt)
    loc = [slice(0, 36)] * 3
    glob = [slice(s, s + 36) for s in start]
    diff = max(np.abs(ws.q[v][padded(loc, wp.ng)] - st.q[v][padded(glob, pr.ng)]).max() for v in range(8))
    assert diff > 0.0


def test_window_of_a_periodic_box_keeps_the_cell_width():
    """A window of the 2-D periodic Orszag-Tang box (cell width 2 pi / 96, not dyadic)
    away from the boundary: its core after two steps equals the whole box's."""
    pr = P.orszag_tang(96)
    st = oracle.from_problem(pr)
    dt = oracle.cfl_dt(st.grid, pr.cfl)
    for _ in range(2):
        st.step(dt)
    start, size = (20, 41, 0), (36, 36, 1)
    wp = window(pr, start, size)
    assert wp.dx == pr.dx
    ws = oracle.from_problem(wp)
    for _ in range(2):
        ws.step(dt)
    loc, glob = window_core(pr, start, size, 2)
    Iw, Ig = padded(loc, wp.ng), padded(glob, pr.ng)
    for v in range(8):
        assert np.array_equal(ws.q[v][Iw], st.q[v][Ig]), v
    for d in range(3):
        assert np.array_equal(ws.bf[d][Iw], st.bf[d][Ig]), d
    with pytest.raises(AssertionError):
        window(pr, (0, 41, 0), size)   # would cut the periodic boundary
