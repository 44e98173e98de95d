"""Exact solution of the 1-D special-relativistic Riemann problem for an ideal gas
with zero tangential velocity (Marti & Mueller 1994, J. Fluid Mech. 258, 317;
Pons, Marti & Mueller 2000, J. Fluid Mech. 422, 125), written here from the published
method: shocks from the Taub adiabat and the relativistic jump conditions,
rarefactions from the Riemann invariant

    arctanh(v) +/- (2/sqrt(Gamma-1)) arctanh(c_s/sqrt(Gamma-1)) = const

along the isentrope p = K rho^Gamma.  Used as an independent pin for the oracle's
hydrodynamics at B = E = 0 (the ideal-limit shock tube).  Self-checks of this file
against the jump conditions and the invariant's ODE are in test_oracle_physics.py
(test_exact_riemann_solver_self_checks).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


def enthalpy(rho, p, gam):
    return 1.0 + gam / (gam - 1.0) * p / rho


def sound_speed(rho, p, gam):
    return math.sqrt(gam * p / (rho * enthalpy(rho, p, gam)))


def rarefaction(rho_a, p_a, v_a, p, gam, sign):
    """State behind a rarefaction at pressure p (< p_a).  sign = -1 for the left
    (leftward-facing) wave, +1 for the right one.  Returns (rho, v, c_s)."""
    K = p_a / rho_a ** gam
    rho = (p / K) ** (1.0 / gam)
    A = math.sqrt(gam - 1.0)
    cs_a = sound_speed(rho_a, p_a, gam)
    cs = sound_speed(rho, p, gam)
    # left wave keeps J+ = arctanh(v) + I(rho); right wave keeps J- = arctanh(v) - I(rho)
    I_a = 2.0 / A * math.atanh(cs_a / A)
    I_b = 2.0 / A * math.atanh(cs / A)
    if sign < 0:
        w = math.atanh(v_a) + I_a - I_b
    else:
        w = math.atanh(v_a) - I_a + I_b
    return rho, math.tanh(w), cs


def shock(rho_a, p_a, v_a, p, gam, sign):
    """State behind a shock of pressure p (> p_a) moving into state a.
    sign = -1 for a left-moving shock, +1 for a right-moving one.
    Returns (rho_b, v_b, V_shock)."""
    h_a = enthalpy(rho_a, p_a, gam)
    dp = p - p_a
    # Taub adiabat [h^2] = (h_a/rho_a + h_b/rho_b)(p_b - p_a), ideal gas h_b/rho_b from h_b, p_b
    c2 = 1.0 - (gam - 1.0) * dp / (gam * p)
    c1 = (gam - 1.0) * dp / (gam * p)
    c0 = -h_a * h_a - h_a * dp / rho_a
    h_b = (-c1 + math.sqrt(c1 * c1 - 4.0 * c2 * c0)) / (2.0 * c2)
    rho_b = gam * p / ((gam - 1.0) * (h_b - 1.0))
    j2 = -dp / (h_b / rho_b - h_a / rho_a)
    j = sign * math.sqrt(j2)
    W_a = 1.0 / math.sqrt(1.0 - v_a * v_a)
    D2 = rho_a * rho_a * W_a * W_a
    # shock speed from j = W_s rho_a W_a (V_s - v_a)
    Vs = (D2 * v_a + sign * math.sqrt(j2) * math.sqrt(j2 + rho_a * rho_a)) / (D2 + j2)
    W_s = 1.0 / math.sqrt(1.0 - Vs * Vs)
    v_b = (h_a * W_a * v_a + W_s * dp / j) / (h_a * W_a + dp * (W_s * v_a / j + 1.0 / (rho_a * W_a)))
    return rho_b, v_b, Vs


def _behind(state, p, gam, sign):
    rho_a, p_a, v_a = state
    if p > p_a:
        rb, vb, _ = shock(rho_a, p_a, v_a, p, gam, sign)
    else:
        rb, vb, _ = rarefaction(rho_a, p_a, v_a, p, gam, sign)
    return rb, vb


def solve(left, right, gam):
    """(rho, p, v) left/right -> p*, v*, rho*_L, rho*_R."""
    pl, pr = left[1], right[1]

    def mismatch(p):
        return _behind(left, p, gam, -1)[1] - _behind(right, p, gam, +1)[1]

    lo, hi = 1e-12 * min(pl, pr), 10.0 * max(pl, pr)
    ps = brentq(mismatch, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    rl, vs = _behind(left, ps, gam, -1)
    rr, _ = _behind(right, ps, gam, +1)
    return ps, vs, rl, rr


def sample(left, right, gam, xi):
    """Self-similar solution (rho, p, v) at xi = x/t (array)."""
    ps, vs, rls, rrs = solve(left, right, gam)
    rhoL, pL, vL = left
    rhoR, pR, vR = right
    out_rho = np.empty_like(xi)
    out_p = np.empty_like(xi)
    out_v = np.empty_like(xi)
    csL, csR = sound_speed(rhoL, pL, gam), sound_speed(rhoR, pR, gam)
    # left wave
    if ps > pL:
        _, _, VsL = shock(rhoL, pL, vL, ps, gam, -1)
        headL = tailL = VsL
    else:
        headL = (vL - csL) / (1.0 - vL * csL)
        cs_s = sound_speed(rls, ps, gam)
        tailL = (vs - cs_s) / (1.0 - vs * cs_s)
    if ps > pR:
        _, _, VsR = shock(rhoR, pR, vR, ps, gam, +1)
        headR = tailR = VsR
    else:
        headR = (vR + csR) / (1.0 + vR * csR)
        cs_s = sound_speed(rrs, ps, gam)
        tailR = (vs + cs_s) / (1.0 + vs * cs_s)
    for n, x in enumerate(xi):
        if x < headL:
            r, p, v = rhoL, pL, vL
        elif x < tailL:
            # inside the left fan: xi = (v - c_s)/(1 - v c_s) on the isentrope
            def g(pp):
                rr, vv, cc = rarefaction(rhoL, pL, vL, pp, gam, -1)
                return (vv - cc) / (1.0 - vv * cc) - x
            p = brentq(g, ps, pL, xtol=1e-15, rtol=1e-15)
            r, v, _ = rarefaction(rhoL, pL, vL, p, gam, -1)
        elif x < vs:
            r, p, v = rls, ps, vs
        elif x < tailR:
            r, p, v = rrs, ps, vs
        elif x < headR:
            def g(pp):
                rr, vv, cc = rarefaction(rhoR, pR, vR, pp, gam, +1)
                return (vv + cc) / (1.0 + vv * cc) - x
            p = brentq(g, ps, pR, xtol=1e-15, rtol=1e-15)
            r, v, _ = rarefaction(rhoR, pR, vR, p, gam, +1)
        else:
            r, p, v = rhoR, pR, vR
        out_rho[n], out_p[n], out_v[n] = r, p, v
    return out_rho, out_p, out_v
