"""GPU parity of the marching flux and edge-EMF kernels on grids large enough that each
thread marches several faces or edges (the chunk length grows with the grid, up to 8),
so the line reconstructions carry state across faces, ragged chunk ends included
(513 faces per line at 512^2).  The small-grid parity tests run chunks of one.
Relative L1 <= 1e-10 per variable against the oracle's per-face reconstruction."""
import numpy as np
import pytest

import oracle
from parity_tools import check, rel_max
from paper_2110_03732_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def G():
    from paper_2110_03732_gb300 import build, grmhd
    build.build()
    return grmhd


def rel_l1(a, b):
    den = max(np.abs(b).sum(), 1e-3 * b.size)
    return np.abs(a - b).sum() / den


def cpu(t):
    return t.detach().cpu().numpy()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda").contiguous()


def check_L(st, Lg, Lo):
    I = st.grid.interior()
    for v in range(8):
        check(cpu(Lg[v])[I], Lo[v][I], f"L[{v}]")
    for d in range(3):
        sl = list(I)
        ax = 2 - d
        if st.grid.ndim > d and st.grid.bc[d] != 0:
            sl[ax] = slice(st.grid.ng[d], st.grid.ng[d] + st.grid.n[d] + 1)
        sl = tuple(sl)
        check(cpu(Lg[8 + d])[sl], Lo[8 + d][sl], f"L_B[{d}]")


@pytest.mark.parametrize("rec", ["mc", "ppm"])
def test_march_2d_512(G, rec):
    pr = P.random_box(7, 2, [512, 512], bc="periodic")
    st = oracle.from_problem(pr, rec=rec)
    Lo = oracle.explicit_L(st.grid, st.prim, st.bf, pr.alpha, pr.psi)
    S = G.Solver.from_problem(pr, rec=rec)
    Lg = S.explicit_L([dev(a) for a in st.prim], [dev(a) for a in st.bf])
    torch.cuda.synchronize()
    check_L(st, Lg, Lo)


@pytest.mark.parametrize("rec", ["mc", "ppm"])
def test_march_3d_metric(G, rec):
    n = [64, 60, 56] if rec == "mc" else [48, 44, 40]
    pr = P.random_box(8, 3, n, bc="outflow", metric=True)
    st = oracle.from_problem(pr, rec=rec)
    Lo = oracle.explicit_L(st.grid, st.prim, st.bf, pr.alpha, pr.psi)
    S = G.Solver.from_problem(pr, rec=rec)
    Lg = S.explicit_L([dev(a) for a in st.prim], [dev(a) for a in st.bf])
    torch.cuda.synchronize()
    check_L(st, Lg, Lo)


def test_march_glm_512(G):
    pr = P.random_box(9, 2, [512, 512], bc="outflow", glm=True, kappa=1.5)
    st = oracle.from_problem_glm(pr)
    Lo = oracle.explicit_L_glm(st.grid, pr.kappa, st.prim, st.qB, st.qphi, pr.alpha, pr.psi)
    S = G.Solver.from_problem(pr, divb="glm")
    Lg = S.explicit_L_glm([dev(a) for a in st.prim], [dev(a) for a in st.qB], dev(st.qphi))
    torch.cuda.synchronize()
    I = st.grid.interior()
    for v in range(12):
        check(cpu(Lg[v])[I], Lo[v][I], f"L[{v}]")


def test_march_3d_metric_step(G):
    """One full step (implicit solves, marched fluxes and EMFs, update) on a 3-D metric
    box large enough to march."""
    pr = P.random_box(10, 3, [64, 48, 40], bc="outflow", metric=True)
    st = oracle.from_problem(pr)
    S = G.Solver.from_problem(pr)
    dt = oracle.cfl_dt(st.grid, pr.cfl, pr.alpha, pr.psi)
    st.step(dt)
    S.step(dt)
    torch.cuda.synchronize()
    I = st.grid.interior()
    for v in range(8):
        check(cpu(S.q[v])[I], st.q[v][I], v)
    for d in range(3):
        check(cpu(S.bf[d])[I], st.bf[d][I], ("B", d))
