"""GPU parity of the ideal-limit edge EMF (App. A) against the oracle: explicit
operator and full steps, relative L1 <= 1e-10 per variable, on 1-D/2-D/3-D,
periodic/outflow and flat/metric boxes, and the advected field loop."""
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


CASES = [
    (1, [37], "outflow", False),
    (1, [24], "periodic", True),
    (2, [21, 17], "periodic", False),
    (2, [18, 11], "outflow", True),
    (3, [10, 9, 7], "periodic", False),
    (3, [8, 7, 9], "outflow", True),
]


@pytest.mark.parametrize("ndim,n,bc,metric", CASES)
def test_ideal_emf_explicit_L_parity(G, ndim, n, bc, metric):
    pr = P.random_box(80 + ndim, ndim, n, bc=bc, metric=metric)
    st = oracle.from_problem(pr, emf="ideal")
    Lo = oracle.explicit_L(st.grid, st.prim, st.bf, pr.alpha, pr.psi)
    S = G.Solver.from_problem(pr, emf="ideal")
    pg = [torch.as_tensor(a, device="cuda").contiguous() for a in st.prim]
    bg = [torch.as_tensor(a, device="cuda").contiguous() for a in st.bf]
    Lg = S.explicit_L(pg, bg)
    torch.cuda.synchronize()
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


def _steps(G, pr, nsteps):
    st = oracle.from_problem(pr, emf="ideal")
    S = G.Solver.from_problem(pr, emf="ideal")
    dt = oracle.cfl_dt(st.grid, pr.cfl, pr.alpha, pr.psi)
    I = st.grid.interior()
    for k in range(nsteps):
        st.step(dt)
        S.step(dt)
        torch.cuda.synchronize()
        for v in range(8):
            check(cpu(S.q[v])[I], st.q[v][I], (k, v))
        for d in range(3):
            check(cpu(S.bf[d])[I], st.bf[d][I], (k, "B", d))
    divb, _, nf = S.diagnostics()
    assert nf == 0 and st.fails == 0
    return S


def test_ideal_emf_steps(G):
    _steps(G, P.random_box(91, 2, [19, 13], bc="periodic"), 3)
    _steps(G, P.random_box(92, 3, [9, 8, 7], bc="outflow", metric=True), 3)
    S = _steps(G, P.orszag_tang(64, eta=1e-8), 3)
    divb, _, _ = S.diagnostics()
    assert divb[2] < 1e-12


def test_ideal_emf_rejected_where_unsupported(G):
    pr = P.random_box(93, 2, [8, 8], bc="fixed")
    with pytest.raises(G.GrmhdError):
        G.Solver.from_problem(pr, emf="ideal")
    pr = P.random_box(94, 2, [8, 8], bc="periodic")
    with pytest.raises(G.GrmhdError):
        G.Solver.from_problem(pr, emf="ideal", precision="mixed")
    S = G.Solver.from_problem(pr, emf="ideal")
    with pytest.raises(G.GrmhdError):
        G.Batch([S])


def test_ideal_emf_orszag_tang_full_size_two_steps(G):
    """The ideal-limit UCT on the 512^2 Orszag-Tang workload in the launch configuration
    the benchmark times: two steps against the oracle."""
    S = _steps(G, P.orszag_tang(512), 2)
    divb, _, _ = S.diagnostics()
    assert divb[2] < 1e-12
