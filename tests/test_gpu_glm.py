"""GPU parity of the GLM hyperbolic-cleaning variant (Sec. 3.1; cell-centred q_B and
q_Phi) through the C ABI against the CPU oracle on the same seeded inputs: relative
L1 error per variable <= 1e-10 (the FP64 bar of the staggered scheme)."""
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
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = max(np.abs(b).sum(), 1e-3 * b.size)
    return np.abs(a - b).sum() / den


def cpu(t):
    return t.detach().cpu().numpy()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda").contiguous()


def compare(st, S, tol=TOL, tag=""):
    """Relative L1 <= tol and the per-element bound (parity_tools) scaled with it."""
    I = st.grid.interior()
    tm = max(1e-8, 100 * tol)
    for v in range(8):
        check(cpu(S.q[v])[I], st.q[v][I], f"{tag} q[{v}]", tol, tm)
    for d in range(3):
        check(cpu(S.bf[d])[I], st.qB[d][I], f"{tag} qB[{d}]", tol, tm)
    check(cpu(S.phi)[I], st.qphi[I], f"{tag} qphi", tol, tm)


CASES_L = [
    (1, [37], "outflow", False),
    (1, [24], "periodic", True),
    (2, [21, 17], "periodic", False),
    (2, [18, 11], "outflow", True),
    (2, [12, 14], "fixed", False),
    (3, [10, 9, 7], "periodic", False),
    (3, [8, 7, 9], "outflow", True),
]


@pytest.mark.parametrize("ndim,n,bc,metric", CASES_L)
def test_glm_explicit_L_parity(G, ndim, n, bc, metric):
    pr = P.random_box(41 + ndim, ndim, n, bc=bc, metric=metric, glm=True, kappa=2.5)
    st = oracle.from_problem_glm(pr)
    Lo = oracle.explicit_L_glm(st.grid, pr.kappa, st.prim, st.qB, st.qphi, pr.alpha, pr.psi)
    S = G.Solver.from_problem(pr, divb="glm")
    Lg = S.explicit_L_glm([dev(a) for a in st.prim], [dev(a) for a in st.qB], dev(st.qphi))
    torch.cuda.synchronize()
    I = st.grid.interior()
    for v in range(12):
        check(cpu(Lg[v])[I], Lo[v][I], f"L[{v}]")


def test_glm_init_and_implicit_parity(G):
    pr = P.orszag_tang(40, kappa=1.0)
    st = oracle.from_problem_glm(pr)
    S = G.Solver.from_problem(pr, divb="glm")
    torch.cuda.synchronize()
    I = st.grid.interior()
    for d in range(3):   # central curl of the cell potential
        np.testing.assert_allclose(cpu(S.bf[d])[I], st.qB[d][I], rtol=1e-13, atol=1e-13)
    compare(st, S, tag="init")
    pr = P.random_box(51, 3, [9, 8, 7], bc="periodic", metric=True, glm=True)
    st = oracle.from_problem_glm(pr)
    rng = np.random.default_rng(2)
    q = [a.copy() for a in st.q]
    for k in range(3):
        q[5 + k] = q[5 + k] + 0.05 * rng.normal(size=q[5 + k].shape)
    for a_dt in (1e-3, 3e-2):
        qo = [a.copy() for a in q]
        po, Ro, fails, _ = oracle.implicit_cc(st.grid, a_dt, qo, st.qB, pr.alpha, pr.psi, pr.eta, pr.eta_u,
                                              [a.copy() for a in st.prim])
        assert fails == 0
        S = G.Solver.from_problem(pr, divb="glm")
        qg = [dev(a) for a in q]
        pg = [dev(a) for a in st.prim]
        Rg = S.implicit(a_dt, qg, [dev(a) for a in st.qB], pg)
        torch.cuda.synchronize()
        for v in range(8):
            check(cpu(pg[v])[I], po[v][I], (a_dt, "prim", v))
        for v in range(3):
            assert rel_l1(cpu(Rg[v])[I], Ro[v][I]) <= 1e-9, (a_dt, "R", v)


def _steps(G, pr, nsteps, tol=TOL):
    st = oracle.from_problem_glm(pr)
    S = G.Solver.from_problem(pr, divb="glm")
    compare(st, S, tag="init")
    dt = oracle.cfl_dt(st.grid, pr.cfl, pr.alpha, pr.psi)
    assert abs(S.compute_dt() - dt) <= 1e-14 * dt
    for k in range(nsteps):
        st.step(dt)
        S.step(dt)
        torch.cuda.synchronize()
        compare(st, S, tol, tag=f"step {k}")
    _, _, nf = S.diagnostics()
    assert nf == 0 and st.fails == 0
    return st, S


def test_glm_step_random_boxes(G):
    _steps(G, P.random_box(61, 2, [19, 13], bc="periodic", glm=True, kappa=3.0), 3)
    _steps(G, P.random_box(62, 3, [9, 7, 6], bc="outflow", metric=True, glm=True, kappa=1.0), 3)
    _steps(G, P.random_box(63, 2, [12, 10], bc="fixed", glm=True, kappa=0.5), 3)
    _steps(G, P.random_box(64, 1, [31], bc="periodic", metric=True, glm=True, xi=0.3), 3)


def test_glm_step_wave_and_monopole(G):
    _steps(G, P.glm_wave(n=48, kappa=1.0), 4)
    st, S = _steps(G, P.monopole(n=20, ndim=3, kappa=5.0), 3)
    divb, _, _ = S.diagnostics()
    ref = oracle.divb_cc(st.grid, st.qB)
    np.testing.assert_allclose(divb, ref, rtol=1e-10)


def test_glm_orszag_tang_full_size_two_steps(G):
    """Orszag-Tang at 512^2 with GLM cleaning: two steps against the oracle."""
    _steps(G, P.orszag_tang(512, kappa=1.0), 2)


def test_glm_rejected_by_batch(G):
    pr = P.random_box(65, 2, [8, 8], bc="periodic", glm=True)
    S = G.Solver.from_problem(pr, divb="glm")
    with pytest.raises(G.GrmhdError):
        G.Batch([S])
