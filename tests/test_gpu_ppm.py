"""GPU parity of the PPM reconstruction against the oracle: the explicit operators (CT
with the resistive EMF, and GLM) and full steps, relative L1 <= 1e-10 per variable, on
1-D/2-D/3-D, periodic/outflow/fixed (whose stencil reads past the two ghost layers) and
flat/metric boxes."""
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


CASES = [
    (1, [37], "outflow", False),
    (1, [24], "periodic", True),
    (2, [21, 17], "periodic", False),
    (2, [18, 11], "outflow", True),
    (2, [12, 14], "fixed", False),
    (3, [10, 9, 7], "periodic", False),
    (3, [8, 7, 9], "outflow", True),
    (3, [7, 8, 6], "fixed", True),
]


@pytest.mark.parametrize("ndim,n,bc,metric", CASES)
def test_ppm_explicit_L_parity(G, ndim, n, bc, metric):
    pr = P.random_box(100 + ndim, ndim, n, bc=bc, metric=metric)
    st = oracle.from_problem(pr, rec="ppm")
    Lo = oracle.explicit_L(st.grid, st.prim, st.bf, pr.alpha, pr.psi)
    S = G.Solver.from_problem(pr, rec="ppm")
    Lg = S.explicit_L([dev(a) for a in st.prim], [dev(a) for a in st.bf])
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


@pytest.mark.parametrize("ndim,n,bc,metric", [(1, [30], "periodic", True), (2, [19, 15], "fixed", False),
                                              (3, [9, 8, 7], "outflow", True)])
def test_ppm_glm_explicit_L_parity(G, ndim, n, bc, metric):
    pr = P.random_box(110 + ndim, ndim, n, bc=bc, metric=metric, glm=True, kappa=1.5)
    st = oracle.from_problem_glm(pr, rec="ppm")
    Lo = oracle.explicit_L_glm(st.grid, pr.kappa, st.prim, st.qB, st.qphi, pr.alpha, pr.psi)
    S = G.Solver.from_problem(pr, divb="glm", rec="ppm")
    Lg = S.explicit_L_glm([dev(a) for a in st.prim], [dev(a) for a in st.qB], dev(st.qphi))
    torch.cuda.synchronize()
    I = st.grid.interior()
    for v in range(12):
        check(cpu(Lg[v])[I], Lo[v][I], f"L[{v}]")


def test_ppm_steps(G):
    for pr in (P.random_box(121, 2, [19, 13], bc="periodic"),
               P.random_box(122, 3, [9, 8, 7], bc="outflow", metric=True),
               P.random_box(123, 2, [12, 10], bc="fixed")):
        st = oracle.from_problem(pr, rec="ppm")
        S = G.Solver.from_problem(pr, rec="ppm")
        dt = oracle.cfl_dt(st.grid, pr.cfl, pr.alpha, pr.psi)
        I = st.grid.interior()
        for k in range(3):
            st.step(dt)
            S.step(dt)
            torch.cuda.synchronize()
            for v in range(8):
                check(cpu(S.q[v])[I], st.q[v][I], (pr.name, k, v))
            for d in range(3):
                check(cpu(S.bf[d])[I], st.bf[d][I], (pr.name, k, "B", d))
        assert S.diagnostics()[2] == 0 and st.fails == 0
    # GLM with PPM
    pr = P.random_box(124, 2, [17, 14], bc="outflow", glm=True, kappa=2.0)
    st = oracle.from_problem_glm(pr, rec="ppm")
    S = G.Solver.from_problem(pr, divb="glm", rec="ppm")
    dt = oracle.cfl_dt(st.grid, pr.cfl)
    I = st.grid.interior()
    for k in range(3):
        st.step(dt)
        S.step(dt)
        torch.cuda.synchronize()
        for v in range(8):
            check(cpu(S.q[v])[I], st.q[v][I], ("glm", k, v))
        check(cpu(S.phi)[I], st.qphi[I])


def test_ppm_rejected_where_unsupported(G):
    pr = P.random_box(125, 2, [8, 8], bc="periodic")
    with pytest.raises(G.GrmhdError):
        G.Solver.from_problem(pr, rec="ppm", emf="ideal")
    S = G.Solver.from_problem(pr, rec="ppm")
    with pytest.raises(G.GrmhdError):
        G.Batch([S])


def test_ppm_mixed_vs_fp64(G):
    """PPM on the mixed-precision path (FP32 reconstruction, HLL and edge EMF): against
    the FP64 PPM path after 100 steps of Orszag-Tang 128^2 the density agrees to 1e-5
    (relative L1), div B stays at FP64 round-off and the periodic totals are kept."""
    pr = P.orszag_tang(128)
    S64 = G.Solver.from_problem(pr, rec="ppm")
    Sm = G.Solver.from_problem(pr, rec="ppm", precision="mixed")
    dt = S64.compute_dt()
    _, tot0, _ = Sm.diagnostics()
    for _ in range(100):
        S64.step(dt)
        Sm.step(dt)
    torch.cuda.synchronize()
    I = S64.interior()
    r64 = cpu(S64.get_prims()[0])[I]
    rm = cpu(Sm.get_prims()[0])[I]
    err = np.abs(rm - r64).sum() / np.abs(r64).sum()
    divb, tot1, nf = Sm.diagnostics()
    assert nf == 0 and err <= 1e-5, err
    assert divb[2] <= 1e-12
    scale = max(abs(x) for x in tot0[:5])
    for v in range(5):
        assert abs(tot1[v] - tot0[v]) <= 1e-12 * scale


def test_ppm_orszag_tang_full_size_two_steps(G):
    """PPM on the 512^2 Orszag-Tang workload in the launch configuration the benchmark
    times: two steps against the oracle, FP64 bounds; then the mixed-precision PPM path
    on the same workload against the same oracle (relative L1 of D and tau <= 1e-5)."""
    pr = P.orszag_tang(512)
    st = oracle.from_problem(pr, rec="ppm")
    S = G.Solver.from_problem(pr, rec="ppm")
    Sm = G.Solver.from_problem(pr, rec="ppm", precision="mixed")
    dt = oracle.cfl_dt(st.grid, pr.cfl)
    I = st.grid.interior()
    for k in range(2):
        st.step(dt)
        S.step(dt)
        Sm.step(dt)
        torch.cuda.synchronize()
        for v in range(8):
            check(cpu(S.q[v])[I], st.q[v][I], ("ppm 512^2", k, v))
        for d in range(3):
            check(cpu(S.bf[d])[I], st.bf[d][I], ("ppm 512^2", k, "B", d))
        for v in (0, 4):
            assert rel_l1(cpu(Sm.q[v])[I], st.q[v][I]) <= 1e-5, ("ppm mixed 512^2", k, v)
    assert S.diagnostics()[2] == 0 and Sm.diagnostics()[2] == 0 and st.fails == 0
