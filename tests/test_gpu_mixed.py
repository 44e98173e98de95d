"""Mixed precision (MC reconstruction, HLL fluxes, the UCT edge EMF and the non-stiff
sources in FP32, the flux divergence in double-word arithmetic; the implicit E +
velocity solve, CT face update and stage combination in FP64) against the FP64
oracle.  Bounds (the targets for the mixed path): relative
L1 error of the density <= 1e-5 after 100 steps, div B at FP64 round-off
(<= 1e-12), conservation of the periodic totals at FP64 round-off (each FP32 face
flux and edge EMF value is shared by both sides)."""
import numpy as np
import pytest

import oracle
from paper_2110_03732_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2110_03732_gb300 import build, grmhd
    build.build()
    return grmhd


def rel_l1(a, b):
    return np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300)


def cpu(t):
    return t.detach().cpu().numpy()


def test_mixed_orszag_tang_100_steps_vs_oracle(G):
    pr = P.orszag_tang(128)
    st = oracle.from_problem(pr)
    S = G.Solver.from_problem(pr, precision="mixed")
    dt = oracle.cfl_dt(st.grid, pr.cfl)
    _, tot0, _ = S.diagnostics()
    for _ in range(100):
        st.step(dt)
        S.step(dt)
    torch.cuda.synchronize()
    I = st.grid.interior()
    rho_o = st.con2prim()[0][I]
    rho_g = cpu(S.get_prims()[0])[I]
    err_rho = rel_l1(rho_g, rho_o)
    err_D = rel_l1(cpu(S.q[0])[I], st.q[0][I])
    divb, tot1, nf = S.diagnostics()
    print(f"mixed OT 128^2 after 100 steps: rel L1 rho {err_rho:.2e}, D {err_D:.2e}, div B max {divb[2]:.2e}")
    assert nf == 0
    assert err_rho <= 1e-5 and err_D <= 1e-5
    assert divb[2] <= 1e-12
    scale = max(abs(x) for x in tot0[:5])
    for v in range(5):
        assert abs(tot1[v] - tot0[v]) <= 1e-12 * scale


def test_mixed_explicit_operator_vs_oracle(G):
    """One FP32 evaluation of the explicit operator: single-precision accuracy."""
    for ndim, n, bc, metric in ((2, [24, 20], "periodic", False), (3, [10, 9, 8], "outflow", True),
                                (1, [40], "outflow", False)):
        pr = P.random_box(17, ndim, n, bc=bc, metric=metric)
        st = oracle.from_problem(pr)
        Lo = oracle.explicit_L(st.grid, st.prim, st.bf, pr.alpha, pr.psi)
        S = G.Solver.from_problem(pr, precision="mixed")
        pg = [torch.as_tensor(a, device="cuda").contiguous() for a in st.prim]
        bg = [torch.as_tensor(a, device="cuda").contiguous() for a in st.bf]
        Lg = S.explicit_L(pg, bg)
        torch.cuda.synchronize()
        I = st.grid.interior()
        for v in range(8):
            scale = max(np.abs(Lo[v][I]).sum(), 1e-3 * Lo[v][I].size)
            assert np.abs(cpu(Lg[v])[I] - Lo[v][I]).sum() / scale <= 2e-5, (ndim, v)


def test_mixed_full_size_vs_fp64(G):
    """The 512^2 workload: mixed against the FP64 path (itself held to the oracle at
    1e-10 per step) after 100 steps, and div B."""
    pr = P.orszag_tang(512)
    S64 = G.Solver.from_problem(pr)
    Sm = G.Solver.from_problem(pr, precision="mixed")
    dt = S64.compute_dt()
    for _ in range(100):
        S64.step(dt)
        Sm.step(dt)
    torch.cuda.synchronize()
    I = S64.interior()
    err = rel_l1(cpu(Sm.q[0])[I], cpu(S64.q[0])[I])
    divb, _, nf = Sm.diagnostics()
    print(f"mixed vs FP64 OT 512^2 after 100 steps: rel L1 D {err:.2e}, div B max {divb[2]:.2e}")
    assert nf == 0 and err <= 1e-5 and divb[2] <= 1e-12


def test_mixed_star_small_runs(G):
    """3-D star (metric, atmosphere, per-cell eta) in mixed precision against FP64."""
    pr = P.star(n=20)
    st = oracle.from_problem(pr)
    S = G.Solver.from_problem(pr, precision="mixed")
    dt = oracle.cfl_dt(st.grid, pr.cfl, pr.alpha, pr.psi)
    for _ in range(5):
        st.step(dt)
        S.step(dt)
    torch.cuda.synchronize()
    I = st.grid.interior()
    assert rel_l1(cpu(S.q[0])[I], st.q[0][I]) <= 1e-5
    divb, _, nf = S.diagnostics()
    assert nf == 0


def test_mixed_star_64_after_100_steps(G):
    """The 64^3 star (fixed metric, outflow, atmosphere, eta 1e-6 inside and 1 outside)
    after 100 steps in mixed precision against the FP64 path: relative L1 of D and tau
    <= 1e-5 over the interior, and div B at FP64 round-off of the field scale in both
    (every FP32 edge EMF is shared by the faces around it)."""
    pr = P.star(n=64)
    S64 = G.Solver.from_problem(pr)
    Sm = G.Solver.from_problem(pr, precision="mixed")
    dt = S64.compute_dt()
    for _ in range(100):
        S64.step(dt)
        Sm.step(dt)
    torch.cuda.synchronize()
    I = S64.interior()
    errD = rel_l1(cpu(Sm.q[0])[I], cpu(S64.q[0])[I])
    errT = rel_l1(cpu(Sm.q[4])[I], cpu(S64.q[4])[I])
    dm, _, nfm = Sm.diagnostics()
    d64, _, nf64 = S64.diagnostics()
    bscale = max(float(b[I].abs().max()) for b in S64.bf) / min(pr.dx[:3])
    print(f"mixed vs FP64 star 64^3 after 100 steps: rel L1 D {errD:.2e}, tau {errT:.2e}, "
          f"div B max {dm[2]:.2e} (FP64 {d64[2]:.2e}, field scale {bscale:.2e})")
    assert nfm == 0 and nf64 == 0
    assert errD <= 1e-5 and errT <= 1e-5
    assert dm[2] <= 1e-12 * bscale and d64[2] <= 1e-12 * bscale
