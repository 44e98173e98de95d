"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same
seeded inputs.  Tolerance (FP64 path): relative L1 error per variable <= 1e-10 per
step (the target for the FP64 path), with a floor of 1e-3 per cell on the
denominator for variables that are identically ~0."""
import math

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


def gpu_solver(G, pr):
    return G.Solver.from_problem(pr)


def compare_state(st, S, tol=TOL, tag=""):
    """Relative L1 <= tol per variable and the per-element bound (parity_tools), scaled
    with tol; returns the worst relative L1."""
    I = st.grid.interior()
    tm = max(1e-8, 100 * tol)
    worst = 0.0
    for v in range(8):
        worst = max(worst, check(cpu(S.q[v])[I], st.q[v][I], f"{tag} q[{v}]", tol, tm))
    for d in range(3):
        worst = max(worst, check(cpu(S.bf[d])[I], st.bf[d][I], f"{tag} bf[{d}]", tol, tm))
    return worst


# ---------------------------------------------------------------------------
# cell-local implicit solve
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("ndim,n,metric", [(2, [19, 13], False), (3, [9, 7, 6], True)])
def test_implicit_parity(G, ndim, n, metric):
    pr = P.random_box(31, ndim, n, bc="periodic", metric=metric)
    st = oracle.from_problem(pr)
    rng = np.random.default_rng(5)
    q = [a.copy() for a in st.q]
    # perturb E* away from the state so that the solve has work to do
    for k in range(3):
        q[5 + k] = q[5 + k] + 0.05 * rng.normal(size=q[5 + k].shape)
    for a_dt in (1e-3, 3e-2, 0.0):
        qo = [a.copy() for a in q]
        po = [a.copy() for a in st.prim]
        po, Ro, fails, _ = oracle.implicit(st.grid, a_dt, qo, st.bf, pr.alpha, pr.psi, pr.eta, pr.eta_u, po)
        assert fails == 0
        S = gpu_solver(G, pr)
        qg = [torch.as_tensor(a, device="cuda").contiguous() for a in q]
        pg = [torch.as_tensor(a, device="cuda").contiguous() for a in st.prim]
        bg = [torch.as_tensor(a, device="cuda").contiguous() for a in st.bf]
        Rg = S.implicit(a_dt, qg, bg, pg)
        torch.cuda.synchronize()
        I = st.grid.interior()
        for v in range(8):
            check(cpu(pg[v])[I], po[v][I], (a_dt, "prim", v))
        for v in range(3):
            check(cpu(qg[5 + v])[I], qo[5 + v][I], (a_dt, "qE", v))
            if a_dt > 0:
                assert rel_l1(cpu(Rg[v])[I], Ro[v][I]) <= 1e-9, (a_dt, "R", v)
        _, _, nf = S.diagnostics()
        assert nf == 0


# ---------------------------------------------------------------------------
# explicit operator
# ---------------------------------------------------------------------------

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
def test_explicit_L_parity(G, ndim, n, bc, metric):
    pr = P.random_box(7 + ndim, ndim, n, bc=bc, metric=metric)
    st = oracle.from_problem(pr)
    Lo = oracle.explicit_L(st.grid, st.prim, st.bf, pr.alpha, pr.psi)
    S = gpu_solver(G, pr)
    pg = [torch.as_tensor(a, device="cuda").contiguous() for a in st.prim]
    bg = [torch.as_tensor(a, device="cuda").contiguous() for a in st.bf]
    Lg = S.explicit_L(pg, bg)
    torch.cuda.synchronize()
    I = st.grid.interior()
    for v in range(8):
        check(cpu(Lg[v])[I], Lo[v][I], f"L[{v}]")
    # face rates: compare on the faces the step updates (interior + the upper
    # boundary face of non-periodic directions)
    for d in range(3):
        sl = list(I)
        ax = 2 - d
        if st.grid.ndim > d and st.grid.bc[d] != 0:
            sl[ax] = slice(st.grid.ng[d], st.grid.ng[d] + st.grid.n[d] + 1)
        sl = tuple(sl)
        check(cpu(Lg[8 + d])[sl], Lo[8 + d][sl], f"L_B[{d}]")


# ---------------------------------------------------------------------------
# full steps
# ---------------------------------------------------------------------------

def _steps(G, pr, nsteps, dt=None, tol=TOL):
    st = oracle.from_problem(pr)
    S = gpu_solver(G, pr)
    compare_state(st, S, tag="init")
    dt = dt or oracle.cfl_dt(st.grid, pr.cfl, pr.alpha, pr.psi)
    dtg = S.compute_dt()
    assert abs(dtg - oracle.cfl_dt(st.grid, pr.cfl, pr.alpha, pr.psi)) <= 1e-14 * dtg
    worst = 0.0
    for k in range(nsteps):
        st.step(dt)
        S.step(dt)
        torch.cuda.synchronize()
        worst = max(worst, compare_state(st, S, tol, tag=f"step {k}"))
    divb, tot, nf = S.diagnostics()
    assert nf == 0 and st.fails == 0
    return st, S, worst


def test_step_shock_tube_ragged(G):
    _steps(G, P.shock_tube(67), 5)


def test_step_shock_tube_full_size(G):
    """The 1-D shock tube at its full 400 cells, the whole run to t = 0.4."""
    pr = P.shock_tube(400)
    st = oracle.from_problem(pr)
    S = gpu_solver(G, pr)
    dt = oracle.cfl_dt(st.grid, pr.cfl)
    nsteps = int(round(pr.t_end / dt))
    for _ in range(nsteps):
        st.step(dt)
        S.step(dt)
    torch.cuda.synchronize()
    # 400 steps: allow the per-step bound to accumulate
    compare_state(st, S, tol=400 * TOL, tag="t=0.4")


def test_step_orszag_tang_ragged(G):
    pr = P.orszag_tang(37)
    pr2 = P.orszag_tang(37)
    _steps(G, pr, 4)
    # also a non-square, ragged box with a per-cell resistivity field
    pr2 = P.random_box(2, 2, [29, 23], bc="periodic")
    _steps(G, pr2, 3)


def test_step_3d_metric(G):
    _steps(G, P.random_box(4, 3, [11, 9, 8], bc="outflow", metric=True), 3)


def test_step_charged_vortex_fixed(G):
    _steps(G, P.charged_vortex(24), 4)


def test_step_star_small(G):
    _steps(G, P.star(n=20), 3)


def test_step_telegraph(G):
    """Telegraph set-up of Sec. 5: rho = 1e12 with p = 0.  The recovered pressure
    p = (w_t/W - rho)/Gamma_hat is then round-off of a 1e12 quantity (about 1e-4 on
    both sides, different on each), and it enters S and tau through the pressure
    flux: those are compared against that conditioning bound, the determined
    quantities (D, E, B) at the FP64 tolerance."""
    pr = P.telegraph(32)
    st = oracle.from_problem(pr)
    S = gpu_solver(G, pr)
    dt = oracle.cfl_dt(st.grid, pr.cfl)
    I = st.grid.interior()
    for k in range(4):
        st.step(dt)
        S.step(dt)
        torch.cuda.synchronize()
        for v in (0, 5, 6, 7):
            check(cpu(S.q[v])[I], st.q[v][I], (k, v))
        for d in range(3):
            check(cpu(S.bf[d])[I], st.bf[d][I], (k, "B", d))
        noise = 8 * 2.2e-16 * 1e12          # pressure round-off
        bound = (k + 1) * 2 * noise * dt / st.grid.dx[0] * 10
        for v in (1, 2, 3, 4):
            assert np.abs(cpu(S.q[v])[I] - st.q[v][I]).max() <= bound, (k, v)


def test_orszag_tang_full_size_two_steps(G):
    """The 2-D Orszag-Tang workload at its full 512^2 size, in the launch configuration
    the benchmark times: two steps against the oracle, element by element."""
    pr = P.orszag_tang(512)
    _steps(G, pr, 2)


def test_star_full_size_invariants(G):
    """The 3-D star at its full 256^3 size (the oracle cannot follow it in seconds):
    two steps keep div B at round-off, every Newton solve converges and all fields stay
    finite; parity at this size is covered by the small-star case above."""
    pr = P.star(n=256)
    S = gpu_solver(G, pr)
    dt = S.compute_dt()
    for _ in range(2):
        S.step(dt)
    torch.cuda.synchronize()
    divb, tot, nf = S.diagnostics()
    bmax = max(float(b.abs().max()) for b in S.bf)
    assert nf == 0
    assert divb[2] < 1e-12 * bmax * 256 / 40.0
    for t in S.q:
        assert bool(torch.isfinite(t).all())


# ---------------------------------------------------------------------------
# invariants and host-visible results on the GPU
# ---------------------------------------------------------------------------

def test_gpu_conservation_and_divb(G):
    pr = P.orszag_tang(64)
    S = gpu_solver(G, pr)
    dt = S.compute_dt()
    _, tot0, _ = S.diagnostics()
    for _ in range(20):
        S.step(dt)
    divb, tot1, nf = S.diagnostics()
    assert nf == 0
    scale = max(abs(x) for x in tot0[:5])
    for v in range(5):
        assert abs(tot1[v] - tot0[v]) <= 1e-12 * scale
    assert divb[2] < 1e-12


def test_gpu_get_prims_matches_oracle(G):
    pr = P.orszag_tang(33)
    st = oracle.from_problem(pr)
    S = gpu_solver(G, pr)
    dt = oracle.cfl_dt(st.grid, 0.4)
    st.step(dt)
    S.step(dt)
    po = st.con2prim()
    pg = S.get_prims()
    torch.cuda.synchronize()
    I = st.grid.interior()
    for v in range(8):
        check(cpu(pg[v])[I], po[v][I])


def test_minimal_grids(G):
    """Degenerate sizes: two cells in a periodic direction, one cell in an outflow one."""
    for pr in (P.random_box(3, 2, [2, 5], bc="periodic"), P.random_box(3, 2, [1, 6], bc="outflow"),
               P.random_box(3, 3, [2, 3, 2], bc="periodic")):
        _steps(G, pr, 2, dt=0.01)


def test_step_dynamo(G):
    """Mean-field dynamo (xi != 0): the 1-D helical test and a 3-D box with a metric.
    The helical test freezes the matter with rho = 1e12, which makes tau = rho h W^2 - p - D
    round-off of a 1e12 quantity on both sides (as in the telegraph case); the parity run
    takes rho = 10, where every variable is well conditioned and the dynamo terms
    still dominate the field evolution."""
    _steps(G, P.dynamo_1d(k=1, n=48, rho=10.0), 4)
    _steps(G, P.random_box(13, 3, [9, 8, 7], bc="periodic", metric=True, xi=0.4), 3)


def test_implicit_parity_dynamo(G):
    pr = P.random_box(33, 2, [17, 15], bc="periodic", xi=0.7)
    st = oracle.from_problem(pr)
    rng = np.random.default_rng(9)
    q = [a.copy() for a in st.q]
    for k in range(3):
        q[5 + k] = q[5 + k] + 0.05 * rng.normal(size=q[5 + k].shape)
    for a_dt in (1e-3, 3e-2):
        qo = [a.copy() for a in q]
        po = [a.copy() for a in st.prim]
        po, Ro, fails, _ = oracle.implicit(st.grid, a_dt, qo, st.bf, pr.alpha, pr.psi, pr.eta, pr.eta_u, po)
        assert fails == 0
        S = gpu_solver(G, pr)
        qg = [torch.as_tensor(a, device="cuda").contiguous() for a in q]
        pg = [torch.as_tensor(a, device="cuda").contiguous() for a in st.prim]
        bg = [torch.as_tensor(a, device="cuda").contiguous() for a in st.bf]
        S.implicit(a_dt, qg, bg, pg)
        torch.cuda.synchronize()
        I = st.grid.interior()
        for v in range(8):
            check(cpu(pg[v])[I], po[v][I], (a_dt, v))
