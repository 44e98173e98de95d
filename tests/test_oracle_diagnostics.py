"""Pins of the oracle's diagnostics (Sec. 3.2 div B, the volume totals of the
conserved variables of Sec. 2.1) against closed forms.

div B.  The discrete divergence of a staggered field is, per cell, the sum over the
active directions of (face value above - face value below) / dx.  For face values
that are a quadratic in their own coordinate the centred difference is the exact
derivative at the cell centre; for a cubic it is the derivative plus h^2 with h half
the cell width; for sin(k x + phi) it is 2 cos(k x_c + phi) sin(k h) / dx.  Terms
that do not depend on a face's own coordinate cancel.  The tests build such fields
on every padded face (ghosts included, or NaN where the boundary rule must replace
them) and compare the oracle's (mean |div|, rms, max) with the same norms of the
closed-form per-cell values.  A missing 1/dx, a difference taken towards the lower
neighbour, a difference along the wrong axis, a ghost counted as interior or a norm
mixed up changes the result.

Totals.  The total of a uniform state is its value times the interior volume; the
total of a linear profile is the volume times its value at the box centre.  Ghost
cells are filled with a huge value so that counting them shows.  With a constant
conformal factor psi (gamma_ij = psi^4 delta_ij) the densitised conserved variables
of a uniform state are psi^k times their flat-space values in the local orthonormal
frame, with k fixed by the tensor type (rest mass and energy densities: the volume
element psi^6; the covariant momentum: one more psi^2; the contravariant E: psi^-2),
so the totals pin the psi powers of prim2con as well."""
import numpy as np
import pytest

import oracle


def _positions(grid, d, face):
    """Coordinates along direction d of the padded index: cells at (i - ng + 1/2) dx,
    lower faces at (i - ng) dx (the box starts at 0)."""
    N, ng, dx = grid.N[d], grid.ng[d], grid.dx[d]
    i = np.arange(N, dtype=np.float64)
    return (i - ng + (0.0 if face else 0.5)) * dx


def _mesh(grid, d_face):
    """(X, Y, Z) on the padded (N2, N1, N0) array, with the positions of direction
    d_face taken at the lower faces (d_face = None: all at cell centres)."""
    ax = [_positions(grid, d, face=(d == d_face)) for d in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return X, Y, Z


def _norms(div):
    a = np.abs(div)
    return np.array([a.mean(), np.sqrt((div * div).mean()), a.max()])


POLY = {  # per direction: (coefficient, power) of the face value's own coordinate
    0: (0.7, 2),
    1: (-1.3, 3),
    2: (2.1, 2),
}


def _poly_face(grid, d):
    X, Y, Z = _mesh(grid, d)
    r = (X, Y, Z)[d]
    a, p = POLY[d]
    # plus a term that does not depend on the face's own coordinate (it must cancel)
    other = [(Y, Z), (Z, X), (X, Y)][d]
    return a * r ** p + np.sin(3.0 * other[0] + 0.4) * np.cos(other[1] - 0.2) + 0.25


def _poly_div_exact(grid):
    X, Y, Z = _mesh(grid, None)
    div = np.zeros(grid.shape)
    for d in range(grid.ndim):
        r = (X, Y, Z)[d]
        a, p = POLY[d]
        h = 0.5 * grid.dx[d]
        div += a * (2.0 * r) if p == 2 else a * (3.0 * r * r + h * h)
    return div[grid.interior()]


@pytest.mark.parametrize("ndim,n,dx", [(1, [19], [0.3]), (2, [13, 9], [0.3, 0.7]),
                                       (3, [7, 6, 5], [0.3, 0.7, 1.1])])
def test_divb_of_polynomial_faces_fixed_boundaries(ndim, n, dx):
    """FIXED boundaries keep every ghost as given, so the faces are the closed form
    everywhere and each interior cell's divergence is known exactly."""
    g = oracle.Grid(ndim, n, dx, ["fixed"] * 3, 4.0 / 3.0)
    bf = [_poly_face(g, d) for d in range(3)]
    got = oracle.divb(g, bf)
    want = _norms(_poly_div_exact(g))
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=0)
    assert want[0] < want[1] < want[2]   # the three norms differ: a mix-up shows


@pytest.mark.parametrize("ndim,n,dx", [(2, [12, 10], [0.4, 0.25]), (3, [8, 7, 6], [0.4, 0.25, 0.6])])
def test_divb_of_polynomial_faces_outflow_ignores_ghosts(ndim, n, dx):
    """OUTFLOW: the n + 1 faces bounding the interior along each direction are real,
    every other padded face is replaced by the boundary rule, so NaN there must not
    reach the result."""
    g = oracle.Grid(ndim, n, dx, ["outflow"] * 3, 4.0 / 3.0)
    bf = []
    for d in range(3):
        b = _poly_face(g, d)
        keep = np.zeros(g.shape, dtype=bool)
        sl = []
        for e in (2, 1, 0):
            lo, hi = g.ng[e], g.ng[e] + g.n[e] + (1 if (e == d and e < ndim) else 0)
            sl.append(slice(lo, hi))
        keep[tuple(sl)] = True
        b[~keep] = np.nan
        bf.append(b)
    got = oracle.divb(g, bf)
    np.testing.assert_allclose(got, _norms(_poly_div_exact(g)), rtol=1e-12, atol=0)


@pytest.mark.parametrize("ndim,n", [(1, [24]), (2, [16, 12]), (3, [10, 8, 6])])
def test_divb_of_periodic_modes(ndim, n):
    """PERIODIC on [0, 2 pi): face values sin(k_d x_d + phi_d) (plus terms that do not
    depend on x_d).  Per cell the discrete divergence is
    sum_d 2 cos(k_d x_d + phi_d) sin(k_d dx_d / 2) / dx_d.  Ghost faces are NaN: the
    periodic rule must replace all of them, including the upper boundary face."""
    dx = [2 * np.pi / n[d] for d in range(ndim)]
    g = oracle.Grid(ndim, n, dx, ["periodic"] * 3, 4.0 / 3.0)
    k = [2.0, 1.0, 3.0]
    ph = [0.3, -1.1, 0.8]
    bf = []
    for d in range(3):
        X, Y, Z = _mesh(g, d)
        r = (X, Y, Z)[d]
        other = [(Y, Z), (Z, X), (X, Y)][d]
        b = np.sin(k[d] * r + ph[d]) + 0.5 * np.cos(other[0]) * np.sin(other[1] + 0.1)
        if d < ndim:
            keep = np.zeros(g.shape, dtype=bool)
            keep[g.interior()] = True
            b[~keep] = np.nan
        bf.append(b)
    X, Y, Z = _mesh(g, None)
    div = np.zeros(g.shape)
    for d in range(ndim):
        r = (X, Y, Z)[d]
        div += 2.0 * np.cos(k[d] * r + ph[d]) * np.sin(0.5 * k[d] * dx[d]) / dx[d]
    np.testing.assert_allclose(oracle.divb(g, bf), _norms(div[g.interior()]), rtol=1e-12, atol=1e-15)


def test_divb_ignores_the_inactive_direction():
    """In 2-D the z 'face' array is the cell value of B^z and has no z derivative."""
    g = oracle.Grid(2, [10, 8], [0.5, 0.5], ["fixed"] * 3, 4.0 / 3.0)
    bf = [_poly_face(g, d) for d in range(3)]
    d0 = oracle.divb(g, bf)
    bf[2] = np.random.default_rng(1).normal(size=g.shape)
    np.testing.assert_array_equal(oracle.divb(g, bf), d0)


def _filled(grid, interior_values, ghost=1e12):
    a = np.full(grid.shape, ghost)
    a[grid.interior()] = interior_values
    return a


@pytest.mark.parametrize("ndim,n,dx", [(1, [17], [0.25, 7.0, 5.0]), (2, [11, 6], [0.3, 0.125, 7.0]),
                                       (3, [5, 4, 3], [0.3, 0.125, 0.75])])
def test_totals_of_uniform_state(ndim, n, dx):
    """A uniform value c_v in every interior cell totals c_v times the interior volume
    (the product of n_d dx_d over the active directions only).  Ghosts hold 1e12."""
    g = oracle.Grid(ndim, n, dx, ["outflow"] * 3, 4.0 / 3.0)
    c = np.array([1.5, -0.25, 0.75, 2.0, 3.5, -1.0, 0.5, 0.125])
    q = [_filled(g, c[v]) for v in range(8)]
    vol = np.prod([n[d] * dx[d] for d in range(ndim)])
    np.testing.assert_allclose(oracle.totals(g, q), c * vol, rtol=1e-14, atol=0)


@pytest.mark.parametrize("ndim,n,dx", [(2, [12, 7], [0.3, 0.2]), (3, [6, 5, 4], [0.3, 0.2, 0.45])])
def test_totals_of_linear_profiles(ndim, n, dx):
    """q_v = c_v + a_v x + b_v y + e_v z over the interior totals the volume times the
    value at the centre of the box [0, n_d dx_d] (cell centres are symmetric about
    it).  Different coefficients per variable catch a variable-index mix-up."""
    g = oracle.Grid(ndim, n, dx, ["periodic"] * 3, 4.0 / 3.0)
    X, Y, Z = _mesh(g, None)
    I = g.interior()
    rng = np.random.default_rng(7)
    coef = rng.uniform(-2, 2, size=(8, 4))
    L = [n[d] * dx[d] if d < ndim else 0.0 for d in range(3)]
    vol = np.prod([n[d] * dx[d] for d in range(ndim)])
    q, want = [], []
    for v in range(8):
        c, a, b, e = coef[v]
        prof = c + a * X + b * Y + (e * Z if ndim == 3 else 0.0)
        q.append(_filled(g, prof[I]))
        want.append(vol * (c + a * L[0] / 2 + b * L[1] / 2 + (e * L[2] / 2 if ndim == 3 else 0.0)))
    np.testing.assert_allclose(oracle.totals(g, q), want, rtol=1e-13, atol=1e-13 * vol)


@pytest.mark.parametrize("psi", [1.0, 1.3])
def test_totals_of_uniform_state_with_conformal_factor(psi):
    """Uniform state on a constant conformal factor: rho, p, u^x, E^z and a uniform
    face field q_B^y = b.  In the local orthonormal frame (e_i = psi^-2 d_i) the
    state is the flat special-relativistic one with u_hat = psi^2 u^x,
    E_hat = psi^2 E^z, B_hat = psi^2 B^y = b / psi^4, and its flat conserved values
    are D = rho W, S_x = rho h W u_hat + (E x B)_x = rho h W u_hat - E_hat B_hat,
    tau = rho h W^2 - p + (E_hat^2 + B_hat^2)/2 - D, E = E_hat.  Densitised
    coordinate components carry psi^6 (volume element) times psi^2 for the covariant
    S_x and psi^-2 for the contravariant E^z."""
    gam = 4.0 / 3.0
    g = oracle.Grid(3, [4, 3, 5], [0.5, 0.25, 0.2], ["periodic"] * 3, gam)
    rho, p, u, Ez, b = 1.7, 0.6, 0.45, 0.3, 0.8
    prim = [np.full(g.shape, x) for x in (rho, u, 0.0, 0.0, p, 0.0, 0.0, Ez)]
    bf = [np.zeros(g.shape), np.full(g.shape, b), np.zeros(g.shape)]
    ps = np.full(g.shape, psi)
    q = oracle.prim2con(g, prim, bf, ps)
    uh, Eh, Bh = psi ** 2 * u, psi ** 2 * Ez, b / psi ** 4
    W = np.sqrt(1.0 + uh * uh)
    h = 1.0 + gam / (gam - 1.0) * p / rho
    flat = np.array([rho * W, rho * h * W * uh - Eh * Bh, 0.0, 0.0,
                     rho * h * W * W - p + 0.5 * (Eh * Eh + Bh * Bh) - rho * W, 0.0, 0.0, Eh])
    powers = np.array([6, 8, 8, 8, 6, 4, 4, 4])
    vol = 4 * 0.5 * 3 * 0.25 * 5 * 0.2
    np.testing.assert_allclose(oracle.totals(g, q), vol * psi ** powers * flat, rtol=1e-13, atol=1e-15)


# ---------------------------------------------------------------------------
# the CFL time step (Sec. 2.5: characteristic speeds alpha sqrt(gamma^dd) with beta = 0;
# the multi-dimensional rule of reading c14: dt = CFL / max over cells of sum_d c_d / dx_d)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("ndim,n,dx", [(1, [16], [0.1]), (2, [12, 9], [0.1, 0.25]), (3, [6, 5, 7], [0.5, 0.2, 0.125])])
def test_cfl_dt_flat_is_the_light_crossing_bound(ndim, n, dx):
    """Flat space: light moves at 1 in every direction, and the bound for a
    dimensionally unsplit step is CFL / sum_d (1 / dx_d)."""
    g = oracle.Grid(ndim, n, dx, ["periodic"] * 3, 4.0 / 3.0)
    want = 0.4 / sum(1.0 / dx[d] for d in range(ndim))
    assert abs(oracle.cfl_dt(g, 0.4) - want) <= 1e-15 * want


@pytest.mark.parametrize("alpha,psi", [(0.5, 2.0), (0.8, 1.25), (1.0, 0.5)])
def test_cfl_dt_constant_metric_is_a_rescaling(alpha, psi):
    """On a constant lapse alpha and conformal factor psi (gamma_ij = psi^4 delta_ij) the
    coordinate light speed is alpha / psi^2, so the step is the flat one times
    psi^2 / alpha.  The ghost cells carry extreme metric values that must be ignored."""
    g = oracle.Grid(2, [10, 7], [0.1, 0.3], ["outflow"] * 3, 4.0 / 3.0)
    a = np.full(g.shape, alpha)
    p = np.full(g.shape, psi)
    I = g.interior()
    ghost = np.ones(g.shape, dtype=bool)
    ghost[I] = False
    a[ghost] = 1e6
    p[ghost] = 1e-3
    flat = oracle.cfl_dt(g, 0.4)
    assert abs(oracle.cfl_dt(g, 0.4, a, p) - flat * psi * psi / alpha) <= 1e-14 * flat * psi * psi / alpha


def test_cfl_dt_takes_the_fastest_cell():
    """One interior cell with twice the lapse (light twice as fast there) halves the
    step; the same cell with psi = 2 instead slows light four-fold and leaves the step
    to the other cells."""
    g = oracle.Grid(3, [5, 4, 6], [0.2, 0.2, 0.4], ["outflow"] * 3, 5.0 / 3.0)
    flat = oracle.cfl_dt(g, 0.4)
    a = np.ones(g.shape)
    a[3, 4, 5] = 2.0   # an interior cell (padded indices, two ghosts each side)
    assert abs(oracle.cfl_dt(g, 0.4, a, None) - flat / 2.0) <= 1e-15 * flat
    p = np.ones(g.shape)
    p[3, 4, 5] = 2.0
    assert abs(oracle.cfl_dt(g, 0.4, None, p) - flat) <= 1e-15 * flat
