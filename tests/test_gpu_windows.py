"""Oracle parity at the full sizes of the 3-D star and the 256-box batch, on sampled
windows.  The oracle cannot step a 256^3 grid in seconds, but the value of a cell
after a step depends only on the cells around it (an IMEX-SSP2 step reaches at most
6 cells), so the oracle is stepped on windows of the full problem, each cut from the
same padded arrays, and the GPU's full-size result is compared with it in each
window's core: the cells more than 14 cells (two steps) from every cut side.
tests/test_oracle_windows.py checks on the CPU that such cores equal the oracle's
whole-problem result.

The GPU side is the full problem in the launch configuration the benchmark times (the
single-problem step for the star, FP64 and mixed; the batched step of all 256 boxes).
FP64 bounds: relative L1 <= 1e-10 and the per-element bound of parity_tools.  Mixed
bounds: relative L1 of D and tau <= 1e-5 (the mixed path's density target)."""
import numpy as np
import pytest

import oracle
from parity_tools import check, padded, rel_l1, window, window_core
from paper_2110_03732_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NSTEPS = 2
W = 36
# the star at 256^3 on [-20, 20]^3 (dx = 0.15625, surface radius R = 12.53 = 80 cells):
# the centre, the surface crossing on +x (eta jumps from 1e-6 to 1, the atmosphere
# begins), an off-axis point inside the field, and two corners on the outflow boundary
STAR_WINDOWS = [(110, 110, 110), (190, 110, 110), (140, 96, 150), (0, 0, 0), (220, 220, 220)]


@pytest.fixture(scope="module")
def G():
    from paper_2110_03732_gb300 import build, grmhd
    build.build()
    return grmhd


@pytest.fixture(scope="module")
def star256():
    return P.star(n=256)


def cpu(t):
    return t.detach().cpu().numpy()


def oracle_window(pr, start, size, dt):
    wp = window(pr, start, size)
    ws = oracle.from_problem(wp)
    for _ in range(NSTEPS):
        ws.step(dt)
    assert ws.fails == 0
    loc, glob = window_core(pr, start, size, NSTEPS)
    return ws, padded(loc, wp.ng), padded(glob, pr.ng)


def star_run(G, pr, precision):
    S = G.Solver.from_problem(pr, precision=precision)
    dt = S.compute_dt()
    for _ in range(NSTEPS):
        S.step(dt)
    torch.cuda.synchronize()
    divb, _, nf = S.diagnostics()
    assert nf == 0
    return S, dt


def test_star_full_size_windows_fp64(G, star256):
    pr = star256
    S, dt = star_run(G, pr, "fp64")
    for start in STAR_WINDOWS:
        ws, Iw, Ig = oracle_window(pr, start, (W, W, W), dt)
        for v in range(8):
            check(cpu(S.q[v][Ig]), ws.q[v][Iw], f"star 256^3 window {start} q[{v}]")
        for d in range(3):
            check(cpu(S.bf[d][Ig]), ws.bf[d][Iw], f"star 256^3 window {start} bf[{d}]")


def test_star_full_size_windows_mixed(G, star256):
    pr = star256
    S, dt = star_run(G, pr, "mixed")
    for start in STAR_WINDOWS:
        ws, Iw, Ig = oracle_window(pr, start, (W, W, W), dt)
        for v in (0, 4):
            e = rel_l1(cpu(S.q[v][Ig]), ws.q[v][Iw])
            assert e <= 1e-5, (start, v, e)


def test_batch_full_size_members_vs_oracle(G):
    """All 256 boxes in one batched mixed-precision step, as the benchmark runs them:
    the smallest boxes whole, and windows of the largest (periodic, so the windows stay
    off the boundary), against the oracle."""
    probs = P.ot_batch(0, 256)
    solvers = [G.Solver.from_problem(pr, precision="mixed") for pr in probs]
    B = G.Batch(solvers)
    dts = [s.compute_dt() for s in solvers]
    B.set_dt(dts)
    for _ in range(NSTEPS):
        B.step()
    torch.cuda.synchronize()
    sides = [pr.n[0] for pr in probs]
    small = [i for i, n in enumerate(sides) if n == 64][:2]
    large = [i for i, n in enumerate(sides) if n == 512][:2]
    assert small and large
    for i in small:
        pr = probs[i]
        st = oracle.from_problem(pr)
        for _ in range(NSTEPS):
            st.step(dts[i])
        I = st.grid.interior()
        for v in (0, 4):
            assert rel_l1(cpu(solvers[i].q[v])[I], st.q[v][I]) <= 1e-5, (i, v)
    for i in large:
        pr = probs[i]
        for start in ((100, 300, 0), (400, 37, 0)):
            ws, Iw, Ig = oracle_window(pr, start, (W, W, 1), dts[i])
            for v in (0, 4):
                assert rel_l1(cpu(solvers[i].q[v][Ig]), ws.q[v][Iw]) <= 1e-5, (i, start, v)
