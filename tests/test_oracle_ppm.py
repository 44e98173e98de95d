"""Pins of the oracle's PPM reconstruction (named in Sec. 5 for the star runs; read as
Colella & Woodward's interface interpolation with their monotonicity constraints):

* it is exact for the cell averages of a cubic (every direction), where MC is not;
* its face states never leave the range of the two cells beside the face (no new
  extrema), for every boundary kind, the fixed one reading past its two ghost layers;
* a smooth monotone front carried by a uniform flow (no extrema, where both limiters
  clip) is reproduced with a several times smaller error than with MC, converging
  faster;
* the half-turn symmetry (resistive and ideal EMFs, whose edge reconstructions use it
  too), the constant-metric rescaling and the 1-D embedding (GLM) hold with PPM."""
import math

import numpy as np
import pytest

import oracle
from paper_2110_03732_gb300 import problems as P


def _cubic(x):
    return 0.3 * x + 0.2 * x ** 2 + 0.1 * x ** 3


def _cubic_int(x):
    return 0.15 * x ** 2 + 0.2 / 3 * x ** 3 + 0.025 * x ** 4


@pytest.mark.parametrize("d", [0, 1, 2])
def test_ppm_exact_for_cubic_averages(d):
    n = [8, 8, 8]
    n[d] = 30
    dxs = [0.05, 0.03, 0.04]
    g = oracle.Grid(3, n, dxs, ["outflow"] * 3, 5.0 / 3.0, rec="ppm")
    gm = oracle.Grid(3, n, dxs, ["outflow"] * 3, 5.0 / 3.0)
    dx = dxs[d]
    xf = (np.arange(g.N[d]) - 2) * dx
    avg = (_cubic_int(xf + dx) - _cubic_int(xf)) / dx
    shape = [1, 1, 1]
    shape[2 - d] = g.N[d]
    a = np.ascontiguousarray(np.broadcast_to(avg.reshape(shape), g.shape))
    L, R = oracle.face_states(g, a, d)
    Lm, _ = oracle.face_states(gm, a, d)
    sl = [slice(2, -2)] * 3
    sl[2 - d] = slice(5, n[d])          # faces whose 6-cell stencil lies in the interior
    sl = tuple(sl)
    exact = np.broadcast_to(_cubic(xf).reshape(shape), g.shape)[sl]
    assert np.abs(L[sl] - exact).max() < 1e-13
    assert np.abs(R[sl] - exact).max() < 1e-13
    assert np.abs(Lm[sl] - exact).max() > 1e-6          # MC is only exact for lines


@pytest.mark.parametrize("bc", ["periodic", "outflow", "fixed"])
def test_ppm_no_new_extrema(bc):
    g = oracle.Grid(1, [50], [0.1], [bc], 5.0 / 3.0, rec="ppm")
    rng = np.random.default_rng(4)
    worst = 0.0
    for _ in range(20):
        a = rng.normal(size=g.shape)
        L, R = oracle.face_states(g, a, 0)
        for i in range(2, 53):
            lo, hi = min(a[0, 0, i - 1], a[0, 0, i]), max(a[0, 0, i - 1], a[0, 0, i])
            for v in (L[0, 0, i], R[0, 0, i]):
                worst = max(worst, lo - v, v - hi)
    assert worst <= 1e-15, worst


def _front(n, rec, T=0.4, v=0.5, w=0.08, x0=0.3):
    """A smooth monotone density front rho = 1 + tanh((x - x0)/w)/2 (as exact cell
    averages) carried by a uniform flow between outflow boundaries; returns the mean
    error against the exact translated averages away from the boundaries."""
    F = lambda x: x + 0.5 * w * np.log(np.cosh((x - x0) / w))      # integral of rho
    xl = (np.arange(n + 4) - 2) / n
    rho = ((F(xl + 1.0 / n) - F(xl)) * n)[None, None]
    z = np.zeros_like(rho)
    W = 1.0 / math.sqrt(1 - v * v)
    prim = [rho, np.full_like(z, W * v), z.copy(), z.copy(), np.ones_like(z), z.copy(), z.copy(), z.copy()]
    pr = P.Problem("front", 1, [n, 1, 1], [0.0, 0.0, 0.0], [1.0, 1.0, 1.0], ["outflow"] * 3, 5.0 / 3.0, prim,
                   bface=[z.copy(), z.copy(), z.copy()], eta_u=1.0, cfl=0.4)
    st = oracle.from_problem(pr, rec=rec)
    dt0 = oracle.cfl_dt(st.grid, pr.cfl)
    ns = int(math.ceil(T / dt0))
    for _ in range(ns):
        st.step(T / ns)
    assert st.fails == 0
    xa = np.arange(n) / n
    exact = (F(xa + 1.0 / n - v * T) - F(xa - v * T)) * n
    keep = (xa > 0.1) & (xa + 1.0 / n < 0.9)
    return np.abs(st.prim[0][0, 0, 2:-2] - exact)[keep].mean()


def test_ppm_front_beats_mc():
    """Away from extrema (where both limiters clip) PPM's higher order shows: on the
    monotone front its error is several times below MC's and falls faster."""
    for n in (32, 64):
        e_ppm, e_mc = _front(n, "ppm"), _front(n, "mc")
        assert e_ppm < 0.3 * e_mc, (n, e_ppm, e_mc)
    assert _front(32, "ppm") / _front(64, "ppm") > 6.0


@pytest.mark.parametrize("emf", ["resistive", "ideal"])
def test_ppm_half_turn(emf):
    n0, n1 = 12, 10
    pr = P.random_box(17, 2, [n0, n1], bc="periodic")
    st = oracle.from_problem(pr, emf=emf, rec="ppm")
    g = st.grid
    I = g.interior()

    def pad(core):
        return np.ascontiguousarray(np.pad(core, [(0, 0), (2, 2), (2, 2)], mode="wrap"))

    cell = lambda a: pad(a[I][:, ::-1, ::-1])
    xface = lambda a: pad(np.roll(a[I][:, ::-1, ::-1], 1, axis=2))
    yface = lambda a: pad(np.roll(a[I][:, ::-1, ::-1], 1, axis=1))
    sp = [1, -1, -1, 1, 1, -1, -1, 1]
    prim_R = [s * cell(a) for s, a in zip(sp, st.prim)]
    bf_R = [-xface(st.bf[0]), -yface(st.bf[1]), cell(st.bf[2])]
    L = oracle.explicit_L(g, st.prim, st.bf)
    LR = oracle.explicit_L(g, prim_R, bf_R)
    want = [s * cell(L[v]) for v, s in enumerate(sp)] + [-xface(L[8]), -yface(L[9]), cell(L[10])]
    for k in range(11):
        np.testing.assert_allclose(LR[k][I], want[k][I], rtol=1e-12, atol=1e-11 * np.abs(L[k][I]).max(),
                                   err_msg=str(k))
    # PPM really changes the operator
    gm = oracle.Grid(2, [n0, n1], g.dx[:2], ["periodic"] * 2, pr.gamma, emf=emf)
    Lm = oracle.explicit_L(gm, st.prim, st.bf)
    assert np.abs(Lm[0][I] - L[0][I]).max() > 1e-3 * np.abs(L[0][I]).max()


def test_ppm_constant_metric_is_a_rescaling():
    al, ps = 0.8, 1.1
    p2, p4, p6, p8 = ps ** 2, ps ** 4, ps ** 6, ps ** 8
    pr = P.random_box(31, 2, [14, 12], bc="outflow")
    sf = oracle.from_problem(pr, rec="ppm")
    gm = oracle.Grid(2, pr.n, [d / p2 for d in pr.dx], pr.bc, pr.gamma, rec="ppm")
    alpha, psi = np.full(pr.shape, al), np.full(pr.shape, ps)
    prim_m = [pr.prim[0]] + [pr.prim[1 + i] / p2 for i in range(3)] + [pr.prim[4]] + \
             [pr.prim[5 + i] / p2 for i in range(3)]
    sm = oracle.State(gm, prim_m, [p4 * b for b in sf.bf], alpha, psi, pr.eta, pr.eta_u)
    dtf = oracle.cfl_dt(sf.grid, pr.cfl)
    for _ in range(2):
        sf.step(dtf)
        sm.step(dtf / al)
    I = sf.grid.interior()
    scale = [p6, p8, p8, p8, p6, p4, p4, p4]
    for v in range(8):
        np.testing.assert_allclose(sm.q[v][I], scale[v] * sf.q[v][I], rtol=1e-12,
                                   atol=1e-13 * np.abs(sm.q[v]).max())


@pytest.mark.parametrize("axis", [0, 2])
def test_ppm_glm_1d_problem_embedded_in_3d(axis):
    n = 20
    pr1 = P.random_box(23, 1, [n], bc="periodic", glm=True, kappa=2.0)
    st1 = oracle.from_problem_glm(pr1, rec="ppm")
    shape3 = [4, 4, 4]
    shape3[axis] = n
    g3 = oracle.Grid(3, shape3, [pr1.dx[0]] * 3, ["periodic"] * 3, pr1.gamma, rec="ppm")

    def embed(a1):
        out = np.empty(g3.shape)
        np.moveaxis(out, 2 - axis, 2)[...] = a1[0, 0, :]
        return out

    perm = [(axis + k) % 3 for k in range(3)]
    prim3 = [None] * 8
    prim3[0] = embed(pr1.prim[0])
    prim3[4] = embed(pr1.prim[4])
    qB3 = [None] * 3
    for k in range(3):
        prim3[1 + perm[k]] = embed(pr1.prim[1 + k])
        prim3[5 + perm[k]] = embed(pr1.prim[5 + k])
        qB3[perm[k]] = embed(st1.qB[k])
    st3 = oracle.GLMState(g3, prim3, qB3, embed(st1.qphi), pr1.kappa, eta=embed(pr1.eta), eta_u=pr1.eta_u)
    dt = 0.2 * pr1.dx[0]
    for _ in range(2):
        st1.step(dt)
        st3.step(dt)
    sl3 = g3.interior()
    line3 = lambda a: np.moveaxis(a[sl3], 2 - axis, 2)[0, 0, :]
    l1 = lambda a: a[st1.grid.interior()][0, 0, :]
    for k in range(3):
        np.testing.assert_allclose(line3(st3.q[1 + perm[k]]), l1(st1.q[1 + k]), rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(line3(st3.qB[perm[k]]), l1(st1.qB[k]), rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(line3(st3.qphi), l1(st1.qphi), rtol=1e-11, atol=1e-12)
