"""GPU diagnostics against the oracle: grmhd_diagnostics' div B norms (Sec. 3.2:
staggered differences on a CT context, central differences of the cell fields on a
GLM context) and the volume totals of the 8 conserved variables, on seeded noisy
states whose field is far from divergence-free, for every boundary kind in 1-D, 2-D
and 3-D.  The oracle's diagnostics are pinned to closed forms in
test_oracle_diagnostics.py.

Tolerance: 1e-12 relative for the mean and rms (the GPU adds per block, then over
blocks, in another order than the oracle's single loop), 1e-13 for the maximum (the
GPU multiplies by 1/dx where the oracle divides by dx), and the totals to 1e-12 of
the volume sum of |q| (noise totals can be near zero)."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2110_03732_gb300 import build, grmhd
    build.build()
    return grmhd


CASES = [
    (1, [37], "outflow"),
    (2, [48, 40], "periodic"),
    (2, [33, 21], "fixed"),
    (3, [20, 14, 11], "outflow"),
    (3, [12, 10, 9], "periodic"),
    (3, [11, 9, 8], "fixed"),
]


def _setup(G, ndim, n, bc, glm, seed):
    lo = [-0.3, 0.1, -1.0]
    hi = [0.9, 1.6, 0.4]
    S = G.Solver(ndim, n, lo, hi, [bc] * 3, 4.0 / 3.0, divb="glm" if glm else "ct")
    dx = [(hi[d] - lo[d]) / n[d] if d < ndim else 1.0 for d in range(3)]
    g = oracle.Grid(ndim, n, dx, [bc] * 3, 4.0 / 3.0)
    rng = np.random.default_rng(seed)
    q = [rng.normal(0.0, 1.0, g.shape) + (2.0 if v in (0, 4) else 0.0) for v in range(8)]
    bf = [rng.normal(0.0, 1.0, g.shape) + 0.5 * d for d in range(3)]
    for v in range(8):
        S.q[v].copy_(torch.as_tensor(q[v]))
    for d in range(3):
        S.bf[d].copy_(torch.as_tensor(bf[d]))
    torch.cuda.synchronize()
    return S, g, q, bf


def _check(S, g, q, want_div):
    div, tot, nf = S.diagnostics()
    assert nf == 0
    div = np.array(div)
    np.testing.assert_allclose(div[:2], want_div[:2], rtol=1e-12, atol=0)
    np.testing.assert_allclose(div[2], want_div[2], rtol=1e-13, atol=0)
    want_tot = oracle.totals(g, q)
    vol_abs = oracle.totals(g, [np.abs(a) for a in q])
    assert np.all(np.abs(np.array(tot) - want_tot) <= 1e-12 * vol_abs), (tot, want_tot)
    assert want_div[0] > 1.0   # the fields are far from divergence-free


@pytest.mark.parametrize("ndim,n,bc", CASES)
def test_ct_diagnostics_match_oracle(G, ndim, n, bc):
    S, g, q, bf = _setup(G, ndim, n, bc, glm=False, seed=11 + ndim)
    _check(S, g, q, oracle.divb(g, bf))


@pytest.mark.parametrize("ndim,n,bc", CASES)
def test_glm_diagnostics_match_oracle(G, ndim, n, bc):
    S, g, q, bf = _setup(G, ndim, n, bc, glm=True, seed=23 + ndim)
    _check(S, g, q, oracle.divb_cc(g, bf))


def test_diagnostics_of_a_run_match_oracle(G):
    """After a few steps of a 3-D metric box on both sides the GPU's diagnostics of
    its own state equal the oracle's diagnostics of the oracle's state (div B at
    round-off on both, totals to the step parity)."""
    from paper_2110_03732_gb300 import problems as P
    pr = P.random_box(5, 3, [14, 12, 10], bc="outflow", metric=True)
    st = oracle.from_problem(pr)
    S = G.Solver.from_problem(pr)
    dt = S.compute_dt()
    for _ in range(3):
        st.step(dt)
        S.step(dt)
    div, tot, nf = S.diagnostics()
    assert nf == 0
    want_tot = oracle.totals(st.grid, st.q)
    vol_abs = oracle.totals(st.grid, [np.abs(a) for a in st.q])
    assert np.all(np.abs(np.array(tot) - want_tot) <= 1e-10 * vol_abs)
    bmax = max(np.abs(b).max() for b in st.bf)
    scale = bmax / min(st.grid.dx[:3])
    want_div = oracle.divb(st.grid, st.bf)
    assert want_div[2] < 1e-12 * scale and div[2] < 1e-12 * scale
