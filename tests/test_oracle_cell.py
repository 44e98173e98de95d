"""Pins of the oracle's cell-local arithmetic (implicit E + velocity solve, Sec. 2.4)
against what the paper and the mathematics fix, independently of the oracle's own
formulas: Ohm's law as printed in Sec. 2.2 (restated here in plain vector form),
closed forms of special cases, limits, and finite differences."""
import math

import numpy as np
import pytest

import oracle

GAMS = [4.0 / 3.0, 5.0 / 3.0, 2.0]


def p2c(rho, u, p, E, B, psi, gam):
    """Sec. 2.1 conserved variables (undensitised) for gamma_ij = psi^4 delta_ij,
    written here in orthonormal components (X_hat = psi^2 X^i for vectors)."""
    g = psi ** 4
    W = math.sqrt(1.0 + g * (u @ u))
    h = 1.0 + gam / (gam - 1.0) * p / rho
    uh, Eh, Bh = psi * psi * u, psi * psi * E, psi * psi * B
    S_hat = rho * h * W * uh + np.cross(Eh, Bh)
    tau = rho * h * W * W - p + 0.5 * (Eh @ Eh + Bh @ Bh) - rho * W
    return rho * W, S_hat * psi * psi, tau  # S_i covariant = psi^2 S_hat


def stiff_rhs(u, E, B, psi, eta):
    """-(W/eta)[E + v x B - (E.v) v] in orthonormal components (Ohm's law, Sec. 2.2,
    stiff part, xi = 0), returned as a contravariant coordinate vector."""
    g = psi ** 4
    W = math.sqrt(1.0 + g * (u @ u))
    vh, Eh, Bh = psi * psi * u / W, psi * psi * E, psi * psi * B
    J = W / eta * (Eh + np.cross(vh, Bh) - (Eh @ vh) * vh)
    return -J / (psi * psi)


def random_state(rng, psi):
    rho = 10 ** rng.uniform(-1, 1)
    p = 10 ** rng.uniform(-2, 1)
    u = rng.normal(0, 0.6, 3)
    E = rng.normal(0, 0.5, 3)
    B = rng.normal(0, 1.0, 3)
    return rho, u, p, E, B


@pytest.mark.parametrize("gam", GAMS)
@pytest.mark.parametrize("psi", [1.0, 1.25])
def test_con2prim_roundtrip(gam, psi):
    """E held fixed: the solve inverts the Sec. 2.1 definitions."""
    rng = np.random.default_rng(1)
    for _ in range(40):
        rho, u, p, E, B = random_state(rng, psi)
        D, S, tau = p2c(rho, u, p, E, B, psi, gam)
        it, uu, EE, r, pp = oracle.solve_cell(D, S, tau, E, B, psi, -1.0, gam)
        assert it > 0
        np.testing.assert_allclose(uu, u, rtol=1e-11, atol=1e-12)
        assert abs(r - rho) <= 1e-11 * rho
        assert abs(pp - p) <= 1e-10 * max(p, rho)
        np.testing.assert_array_equal(EE, E)


@pytest.mark.parametrize("gam", GAMS)
@pytest.mark.parametrize("psi", [1.0, 1.3])
def test_implicit_constructed_root(gam, psi):
    """A known root: pick the stage solution (rho, u, p, E, B) and eta_t, build E* from
    the implicit equation E* = E + (1/eta_t) W [E + v x B - (E.v) v] (Sec. 2.4 with the
    sign that makes the printed A_k consistent) and (D, S, tau) from the Sec. 2.1
    definitions; the solve must return that solution."""
    rng = np.random.default_rng(2)
    for k in range(60):
        rho, u, p, _, B = random_state(rng, psi)
        etat = 10 ** rng.uniform(-4, 3)
        # a stage solution as it arises in a run: E = -v x B plus a non-ideal part that
        # the relaxation keeps of order eta_t (so that E* - E stays of order one)
        W = math.sqrt(1 + psi ** 4 * (u @ u))
        E = -np.cross(psi * psi * u / W, psi * psi * B) / (psi * psi) \
            + min(0.5, etat) * rng.normal(0, 1, 3)
        D, S, tau = p2c(rho, u, p, E, B, psi, gam)
        Es = E - (1.0 / etat) * stiff_rhs(u, E, B, psi, 1.0)
        # the solve starts from the previous stage's velocity in a run: a nearby guess
        guess = u + rng.normal(0, 0.05, 3)
        it, uu, EE, r, pp = oracle.solve_cell(D, S, tau, Es, B, psi, etat, gam, guess)
        assert it > 0, k
        np.testing.assert_allclose(uu, u, rtol=1e-10, atol=1e-11)
        np.testing.assert_allclose(EE, E, rtol=1e-10, atol=1e-11 * (1 + np.abs(B).max()))
        assert abs(r - rho) <= 1e-10 * rho
        assert abs(pp - p) <= 1e-9 * max(p, rho)


def test_implicit_from_rest_weak_field():
    """From rest (the fallback guess) the solve finds the root of weakly magnetised
    states, stiff or not."""
    rng = np.random.default_rng(12)
    gam, psi = 4.0 / 3.0, 1.1
    for k in range(40):
        rho, u, p, _, B = random_state(rng, psi)
        B *= 0.3
        rho, p = rho + 1.0, p + 0.5
        etat = 10 ** rng.uniform(-4, 3)
        W = math.sqrt(1 + psi ** 4 * (u @ u))
        E = -np.cross(psi * psi * u / W, psi * psi * B) / (psi * psi) + min(0.5, etat) * rng.normal(0, 1, 3)
        D, S, tau = p2c(rho, u, p, E, B, psi, gam)
        Es = E - (1.0 / etat) * stiff_rhs(u, E, B, psi, 1.0)
        it, uu, EE, r, pp = oracle.solve_cell(D, S, tau, Es, B, psi, etat, gam)
        assert it > 0, k
        np.testing.assert_allclose(uu, u, rtol=1e-10, atol=1e-11)
        np.testing.assert_allclose(EE, E, rtol=1e-10, atol=1e-11)


def test_implicit_unphysical_base_is_reported():
    """A base state with no physical root must be reported as a failure (-1), not
    returned as a spurious root at W -> infinity."""
    gam, psi = 4.0 / 3.0, 1.0
    rng = np.random.default_rng(7)
    seen_fail = 0
    for _ in range(60):
        rho, u, p, E0, B = random_state(rng, psi)
        D, S, tau = p2c(rho, u, p, E0, B, psi, gam)
        Es = E0 + rng.normal(0, 0.3, 3)
        etat = 10 ** rng.uniform(-4, 3)
        it, uu, EE, r, pp = oracle.solve_cell(D, S, tau, Es, B, psi, etat, gam)
        if it < 0:
            seen_fail += 1
            continue
        # whatever is returned as converged must satisfy the stage equations
        D2, S2, tau2 = p2c(r, uu, pp, EE, B, psi, gam)
        assert abs(D2 - D) <= 1e-10 * D
        assert abs(tau2 - tau) <= 1e-9 * (tau + D)
        lhs = EE - Es
        rhs = (1.0 / etat) * stiff_rhs(uu, EE, B, psi, 1.0)
        np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-9 * (1 + np.abs(Es).max() + np.abs(B).max()))
    assert seen_fail < 60


@pytest.mark.parametrize("psi", [1.0, 1.2])
def test_static_closed_form(psi):
    """u = 0 (a static root): E = eta_t E*/(1 + eta_t) from A_0 = W + eta_t at W = 1."""
    rng = np.random.default_rng(3)
    gam = 5.0 / 3.0
    for _ in range(20):
        rho, _, p, E, B = random_state(rng, psi)
        etat = 10 ** rng.uniform(-3, 2)
        u0 = np.zeros(3)
        D, S, tau = p2c(rho, u0, p, E, B, psi, gam)
        Es = E * (1.0 + etat) / etat
        it, uu, EE, r, pp = oracle.solve_cell(D, S, tau, Es, B, psi, etat, gam)
        np.testing.assert_allclose(uu, 0.0, atol=1e-12)
        np.testing.assert_allclose(EE, E, rtol=1e-12, atol=1e-13)
        assert abs(pp - p) < 1e-10 * max(p, rho)


def test_limits():
    """eta_t -> infinity: E -> E* (the plain con2prim); eta_t -> 0: E -> -v x B."""
    rng = np.random.default_rng(4)
    gam, psi = 4.0 / 3.0, 1.0
    for _ in range(20):
        rho, u, p, E, B = random_state(rng, psi)
        D, S, tau = p2c(rho, u, p, E, B, psi, gam)
        it, uu, EE, r, pp = oracle.solve_cell(D, S, tau, E, B, psi, 1e14, gam)
        np.testing.assert_allclose(EE, E, atol=1e-9)
        np.testing.assert_allclose(uu, u, atol=1e-9)
        it, uu, EE, r, pp = oracle.solve_cell(D, S, tau, E, B, psi, 1e-12, gam)
        W = math.sqrt(1 + uu @ uu)
        np.testing.assert_allclose(EE, -np.cross(uu / W, B), atol=1e-9)


@pytest.mark.parametrize("psi", [1.0, 1.3])
def test_jacobian_finite_difference(psi):
    """The analytic Jacobian of Sec. 2.4 (with the E-field derivative) matches central
    differences of the residual."""
    rng = np.random.default_rng(5)
    gam = 5.0 / 3.0
    for _ in range(20):
        rho, u, p, E, B = random_state(rng, psi)
        D, S, tau = p2c(rho, u, p, E, B, psi, gam)
        Es = E + rng.normal(0, 0.3, 3)
        etat = 10 ** rng.uniform(-2, 2)
        ut = u + rng.normal(0, 0.2, 3)
        f, J, _ = oracle.residual_cell(D, S, tau, Es, B, psi, etat, gam, ut)
        Jfd = np.zeros((3, 3))
        for j in range(3):
            h = 1e-6 * (1 + abs(ut[j]))
            up, um = ut.copy(), ut.copy()
            up[j] += h
            um[j] -= h
            fp, _, _ = oracle.residual_cell(D, S, tau, Es, B, psi, etat, gam, up)
            fm, _, _ = oracle.residual_cell(D, S, tau, Es, B, psi, etat, gam, um)
            Jfd[:, j] = (fp - fm) / (2 * h)
        np.testing.assert_allclose(J, Jfd, rtol=1e-6, atol=1e-6 * np.abs(J).max())


def test_ssp2_tableau_order_conditions():
    """IMEX-SSP2(2,2,2): both parts second order, c_i consistent, gamma = 1 - 1/sqrt 2."""
    At, A, wt, w = oracle.ssp2_tableau()
    g = 1 - 1 / math.sqrt(2)
    assert abs(A[0, 0] - g) < 1e-16 and abs(A[1, 1] - g) < 1e-16
    for M, b in ((At, wt), (A, w)):
        c = M.sum(axis=1)
        assert abs(b.sum() - 1) < 1e-15
        assert abs(b @ c - 0.5) < 1e-15
    # coupling condition of IMEX order 2: wt.c = w.ct = 1/2
    assert abs(wt @ A.sum(axis=1) - 0.5) < 1e-15 and abs(w @ At.sum(axis=1) - 0.5) < 1e-15
    # L-stability: stability function of the implicit part vanishes at infinity
    # R(z) = 1 + z w^T (I - z A)^{-1} 1 -> 1 - w^T A^{-1} 1
    assert abs(1 - w @ np.linalg.solve(A, np.ones(2))) < 1e-14


def stiff_rhs_xi(u, E, B, psi, xi):
    """-W{[E + v x B - (E.v)v] - xi [B - v x E - (B.v)v]} (Ohm's law with the
    mean-field dynamo, Sec. 2.2; eta = 1), orthonormal components -> contravariant."""
    g = psi ** 4
    W = math.sqrt(1.0 + g * (u @ u))
    vh, Eh, Bh = psi * psi * u / W, psi * psi * E, psi * psi * B
    J = W * ((Eh + np.cross(vh, Bh) - (Eh @ vh) * vh) - xi * (Bh - np.cross(vh, Eh) - (Bh @ vh) * vh))
    return -J / (psi * psi)


@pytest.mark.parametrize("xi", [0.1, 0.5, 2.0])
@pytest.mark.parametrize("psi", [1.0, 1.2])
def test_dynamo_constructed_root(xi, psi):
    """Sec. 2.4 with xi != 0: the printed A_k(W) must give back a constructed root of
    E = E* - (W/eta_t){[E + v x B - (E.v)v] - xi[B - v x E - (B.v)v]}.  A strong dynamo
    (xi = 2) can have a second physical root; a solve that lands there must still
    satisfy every stage equation, and that may happen only rarely."""
    rng = np.random.default_rng(21)
    gam = 4.0 / 3.0
    other = 0
    for k in range(40):
        rho, u, p, _, B = random_state(rng, psi)
        etat = 10 ** rng.uniform(-3, 3)
        W = math.sqrt(1 + psi ** 4 * (u @ u))
        E = -np.cross(psi * psi * u / W, psi * psi * B) / (psi * psi) + min(0.5, etat) * rng.normal(0, 1, 3)
        D, S, tau = p2c(rho, u, p, E, B, psi, gam)
        Es = E - (1.0 / etat) * stiff_rhs_xi(u, E, B, psi, xi)
        guess = u + rng.normal(0, 0.05, 3)
        it, uu, EE, r, pp = oracle.solve_cell(D, S, tau, Es, B, psi, etat, gam, guess, xi=xi)
        assert it > 0, k
        if np.abs(uu - u).max() > 1e-8 and xi > 1.0:
            other += 1
            D2, S2, tau2 = p2c(r, uu, pp, EE, B, psi, gam)
            assert abs(D2 - D) <= 1e-12 * D and abs(tau2 - tau) <= 1e-11 * (tau + D)
            res = EE - Es - (1.0 / etat) * stiff_rhs_xi(uu, EE, B, psi, xi)
            assert np.abs(res).max() <= 1e-10 * (1 + np.abs(Es).max()) and r > 0 and pp > 0
            continue
        np.testing.assert_allclose(uu, u, rtol=1e-10, atol=1e-11)
        np.testing.assert_allclose(EE, E, rtol=1e-10, atol=1e-10 * (1 + np.abs(B).max()))
    assert other <= 2


@pytest.mark.parametrize("xi", [0.3, 1.5])
def test_dynamo_jacobian_finite_difference(xi):
    rng = np.random.default_rng(8)
    gam, psi = 5.0 / 3.0, 1.15
    for _ in range(15):
        rho, u, p, E, B = random_state(rng, psi)
        D, S, tau = p2c(rho, u, p, E, B, psi, gam)
        Es = E + rng.normal(0, 0.3, 3)
        etat = 10 ** rng.uniform(-2, 2)
        ut = u + rng.normal(0, 0.2, 3)
        f, J, _ = oracle.residual_cell(D, S, tau, Es, B, psi, etat, gam, ut, xi=xi)
        Jfd = np.zeros((3, 3))
        for j in range(3):
            h = 1e-6 * (1 + abs(ut[j]))
            up, um = ut.copy(), ut.copy()
            up[j] += h
            um[j] -= h
            fp, _, _ = oracle.residual_cell(D, S, tau, Es, B, psi, etat, gam, up, xi=xi)
            fm, _, _ = oracle.residual_cell(D, S, tau, Es, B, psi, etat, gam, um, xi=xi)
            Jfd[:, j] = (fp - fm) / (2 * h)
        np.testing.assert_allclose(J, Jfd, rtol=1e-6, atol=1e-6 * np.abs(J).max())
