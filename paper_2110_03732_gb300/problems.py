"""Seeded, synthetic initial data for the resistive-MHD workloads.

This module holds initial conditions only: closed-form profiles evaluated at cell
centres, staggered faces or edges of the padded grid, plus a seeded generator of
random physical cell states.  It holds none of the method's arithmetic: no
conserved variables, no curl, no reconstruction, no solver.  Both the CUDA path and
the CPU oracle read it, and each converts the primitives with its own code.

Layout: every array has shape ``(N2, N1, N0)`` (x fastest) with ``ng = 2`` ghost
cells on each side of every active direction (none in an inactive one).  Padded
index ``i`` along an active direction has cell centre ``lo + (i - ng + 1/2) dx`` and
lower face ``lo + (i - ng) dx``.  Face arrays hold q_B on the lower face of cell
``i``; edge arrays hold A_c on the lower corner edge (lower in both transverse
directions).

Primitive order: rho, u^1, u^2, u^3 (u^i = W v^i), p, E^1, E^2, E^3.

Workloads (the paper's section or table is given for each):
  * ``shock_tube``      - resistive relativistic shock tube, Sec. 5 (Balsara test 1
                          states, Gamma = 2), 400 cells on [-0.5, 0.5].
  * ``orszag_tang``     - 2-D resistive relativistic Orszag-Tang vortex (not in the
                          paper), periodic [0, 2 pi]^2, Gamma = 4/3.
  * ``star``            - 3-D magnetised static star on a fixed conformally flat
                          metric (synthetic stand-in for the paper's neutron-star runs).
  * ``current_sheet``   - self-similar current sheet, Sec. 5.
  * ``telegraph``       - 2-D telegraph-equation plane wave, Sec. 5.
  * ``charged_vortex``  - stationary charged vortex, Sec. 5.
  * ``random_cells``    - seeded random physical states for cell-local tests.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from math import erf as _erf

_verf = np.vectorize(_erf)


@dataclass
class Problem:
    """One resistive-MHD problem on a padded Cartesian grid."""

    name: str
    ndim: int
    n: list            # interior cells per direction (length 3; 1 where inactive)
    lo: list
    hi: list
    bc: list           # "periodic" | "outflow" | "fixed" per direction
    gamma: float       # ideal-gas adiabatic index
    prim: list         # 8 padded arrays (rho, u^1..3, p, E^1..3), ghosts included
    bface: list = None  # 3 padded arrays of face q_B, or None
    A_edge: list = None  # 3 padded arrays of edge A_c, or None (then bface is used)
    alpha: np.ndarray = None
    psi: np.ndarray = None
    eta: np.ndarray = None   # per-cell resistivity, or None (then eta_u)
    eta_u: float = 0.0
    cfl: float = 0.4
    xi: float = 0.0          # mean-field dynamo parameter
    # GLM variant (cell-centred B): potential at cell centres or q_B at cell centres,
    # initial Phi (None: 0) and the damping kappa_B
    A_cell: list = None
    bcell: list = None
    phi: np.ndarray = None
    kappa: float = 0.0
    rho_atm: float = 0.0     # atmosphere floor density (0: no atmosphere treatment)
    p_atm: float = 0.0
    t_end: float = 0.0
    steps: int = 0
    info: dict = field(default_factory=dict)

    @property
    def ng(self):
        return [2 if d < self.ndim else 0 for d in range(3)]

    @property
    def N(self):
        return [self.n[d] + 2 * self.ng[d] for d in range(3)]

    @property
    def shape(self):
        N = self.N
        return (N[2], N[1], N[0])

    @property
    def dx(self):
        return [(self.hi[d] - self.lo[d]) / self.n[d] for d in range(3)]

    @property
    def cells(self):
        return self.n[0] * self.n[1] * self.n[2]


def _axes(ndim, n, lo, hi):
    ng = [2 if d < ndim else 0 for d in range(3)]
    dx = [(hi[d] - lo[d]) / n[d] for d in range(3)]
    centre = []
    face = []
    for d in range(3):
        i = np.arange(n[d] + 2 * ng[d], dtype=np.float64)
        centre.append(lo[d] + (i - ng[d] + 0.5) * dx[d])
        face.append(lo[d] + (i - ng[d]) * dx[d])
    return centre, face


def _mesh(x, y, z):
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def _pad_shape(ndim, n):
    ng = [2 if d < ndim else 0 for d in range(3)]
    return (n[2] + 2 * ng[2], n[1] + 2 * ng[1], n[0] + 2 * ng[0])


def _lorentz_u(vx, vy, vz):
    W = 1.0 / np.sqrt(1.0 - (vx * vx + vy * vy + vz * vz))
    return W * vx, W * vy, W * vz


# --------------------------------------------------------------------------
# benchmark workloads (shock tube, Orszag-Tang, magnetised star)
# --------------------------------------------------------------------------

def shock_tube(n=400, eta=1e-3, with_B=True):
    """Resistive shock tube (Sec. 5): (rho, p, B^x, B^y) = (1, 1, .5, 1) for x < 0 and
    (.125, .1, .5, -1) for x > 0, v = E = 0, Gamma = 2, outflow, t_end = 0.4.
    ``with_B=False`` gives the same hydrodynamic states with B = 0 (exact
    relativistic Riemann problem)."""
    ndim, nn, lo, hi = 1, [n, 1, 1], [-0.5, 0.0, 0.0], [0.5, 1.0, 1.0]
    c, f = _axes(ndim, nn, lo, hi)
    X, _, _ = _mesh(c[0], c[1], c[2])
    left = X < 0.0
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    z = np.zeros_like(X)
    prim = [rho, z.copy(), z.copy(), z.copy(), p, z.copy(), z.copy(), z.copy()]
    bx = np.full_like(X, 0.5 if with_B else 0.0)
    by = np.where(left, 1.0, -1.0) if with_B else z.copy()
    bface = [bx, by, z.copy()]
    return Problem("shock_tube_1d", ndim, nn, lo, hi, ["outflow"] * 3, 2.0, prim, bface=bface,
                   eta_u=eta, cfl=0.4, t_end=0.4)


def orszag_tang(n=512, eta=1e-4, phase=(0.0, 0.0), gamma=4.0 / 3.0, eta_field=False, kappa=1.0):
    """2-D resistive relativistic Orszag-Tang vortex on periodic [0, 2 pi]^2:
    rho = 1, p = 1, v = (-0.5 sin y, 0.5 sin x), B = (-sin y, sin 2x) from the edge
    potential A_z = cos y + cos(2x)/2, E = -v x B.  ``phase`` shifts x and y.  The
    potential is also given at cell centres, with ``kappa`` the damping of the GLM
    variant."""
    ndim, nn = 2, [n, n, 1]
    lo, hi = [0.0, 0.0, 0.0], [2 * math.pi, 2 * math.pi, 1.0]
    c, f = _axes(ndim, nn, lo, hi)
    px, py = phase
    X, Y, _ = _mesh(c[0] + px, c[1] + py, c[2])
    vx, vy = -0.5 * np.sin(Y), 0.5 * np.sin(X)
    Bx, By = -np.sin(Y), np.sin(2 * X)
    ux, uy, uz = _lorentz_u(vx, vy, np.zeros_like(vx))
    Ez = -(vx * By - vy * Bx)
    z = np.zeros_like(X)
    prim = [np.ones_like(X), ux, uy, uz, np.ones_like(X), z.copy(), z.copy(), Ez]
    FX, FY, _ = _mesh(f[0] + px, f[1] + py, c[2])
    Az = np.cos(FY) + 0.5 * np.cos(2 * FX)
    A = [z.copy(), z.copy(), Az]
    # the same potential at cell centres, for the cell-centred (GLM) variant
    A_cell = [z.copy(), z.copy(), np.cos(Y) + 0.5 * np.cos(2 * X)]
    eta_arr = np.full_like(X, eta) if eta_field else None
    return Problem("orszag_tang_2d", ndim, nn, lo, hi, ["periodic"] * 3, gamma, prim, A_edge=A,
                   eta=eta_arr, eta_u=eta, cfl=0.4, steps=1000, A_cell=A_cell, kappa=kappa)


def star(n=256, L=20.0, K=100.0, gamma=2.0, rho_c=1.28e-3, M=1.4, atm_frac=1e-10, b_frac=1e-3,
         eta_in=1e-6, eta_out=1.0):
    """3-D magnetised static star on a fixed conformally flat metric, [-L, L]^3.
    Density: Newtonian n = 1 polytrope rho = rho_c sin(xi)/xi, xi = pi r / R,
    R = pi sqrt(K / (2 pi)), p = K rho^Gamma, atmosphere rho_c * atm_frac outside.
    Metric: rbar = sqrt(r^2 + 4 M^2), alpha = 1 - 2M/(rbar + M), psi = 1 + M/(2 rbar).
    Field: A_phi = A_b max(p - 0.04 p_max, 0) varpi^2, i.e. A = A_b f (-y, x, 0) on
    edges, with A_b set so the continuum central field has B^2/(2 p_c) = b_frac.
    Resistivity eta_in inside the surface and eta_out outside."""
    ndim, nn, lo, hi = 3, [n, n, n], [-L, -L, -L], [L, L, L]
    c, f = _axes(ndim, nn, lo, hi)
    R = math.pi * math.sqrt(K / (2 * math.pi))
    rho_atm = rho_c * atm_frac
    p_c = K * rho_c ** gamma

    def rho_of(r):
        xi = np.pi * r / R
        s = np.where(xi > 1e-12, np.sin(xi) / np.where(xi > 1e-12, xi, 1.0), 1.0)
        return np.where(r < R, np.maximum(rho_c * s, rho_atm), rho_atm)

    X, Y, Z = _mesh(c[0], c[1], c[2])
    r = np.sqrt(X * X + Y * Y + Z * Z)
    rho = rho_of(r)
    p = K * rho ** gamma
    rbar = np.sqrt(r * r + 4 * M * M)
    alpha = 1.0 - 2.0 * M / (rbar + M)
    psi = 1.0 + M / (2.0 * rbar)
    z = np.zeros_like(X)
    prim = [rho, z.copy(), z.copy(), z.copy(), p, z.copy(), z.copy(), z.copy()]
    A_b = math.sqrt(2.0 * b_frac * p_c) / (2.0 * 0.96 * p_c)

    def fpot(xx, yy, zz):
        rr = np.sqrt(xx * xx + yy * yy + zz * zz)
        pp = K * rho_of(rr) ** gamma
        return A_b * np.maximum(pp - 0.04 * p_c, 0.0)

    # A_x on x-edges: centre in x, lower face in y and z
    Xa, Ya, Za = _mesh(c[0], f[1], f[2])
    Ax = -Ya * fpot(Xa, Ya, Za)
    Xb, Yb, Zb = _mesh(f[0], c[1], f[2])
    Ay = Xb * fpot(Xb, Yb, Zb)
    A = [Ax, Ay, z.copy()]
    eta = np.where(r < R, eta_in, eta_out)
    return Problem("star_3d", ndim, nn, lo, hi, ["outflow"] * 3, gamma, prim, A_edge=A, alpha=alpha,
                   psi=psi, eta=eta, eta_u=eta_in, cfl=0.4, steps=500, rho_atm=rho_atm, p_atm=K * rho_atm ** gamma,
                   info={"R": R, "rho_atm": rho_atm, "p_c": p_c})


# --------------------------------------------------------------------------
# paper test problems (pins)
# --------------------------------------------------------------------------

def current_sheet(n=256, eta=0.01, t0=1.0, rho=1.0, p=5000.0, gamma=4.0 / 3.0):
    """Self-similar current sheet (Sec. 5): B^y = erf(x / (2 sqrt(eta t))),
    E^z = sqrt(eta/(pi t)) exp(-x^2/(4 eta t)) at t = t0, on [-1.5, 1.5], outflow."""
    ndim, nn, lo, hi = 1, [n, 1, 1], [-1.5, 0.0, 0.0], [1.5, 1.0, 1.0]
    c, f = _axes(ndim, nn, lo, hi)
    X, _, _ = _mesh(c[0], c[1], c[2])
    z = np.zeros_like(X)
    By = _verf(X / (2.0 * math.sqrt(eta * t0)))
    Ez = math.sqrt(eta / (math.pi * t0)) * np.exp(-X * X / (4.0 * eta * t0))
    prim = [np.full_like(X, rho), z.copy(), z.copy(), z.copy(), np.full_like(X, p), z.copy(), z.copy(), Ez]
    bface = [z.copy(), By, z.copy()]
    return Problem("current_sheet_1d", ndim, nn, lo, hi, ["outflow"] * 3, gamma, prim, bface=bface,
                   eta_u=eta, cfl=0.4, t_end=10.0 - t0, info={"t0": t0})


def telegraph_exact(X, Y, t, sigma=1.0, B1=1.0, Lx=1.0, Ly=0.5):
    """Rotated plane-wave solution of the telegraph problem (Sec. 5): returns
    (E^x, E^y, B^z)."""
    ta = Lx / Ly
    al = math.atan(ta)
    kx = 2 * math.pi / Lx
    k = kx * math.sqrt(1 + ta * ta)
    mu = math.sqrt(k * k - sigma * sigma / 4.0)
    ph = kx * X + kx * ta * Y - mu * t
    damp = B1 * math.exp(-sigma * t / 2.0)
    Bz = damp * np.cos(ph)
    Ey0 = damp * (mu / k * np.cos(ph) + sigma / (2 * k) * np.sin(ph))
    return -math.sin(al) * Ey0, math.cos(al) * Ey0, Bz


def telegraph_period(sigma=1.0, Lx=1.0, Ly=0.5):
    kx = 2 * math.pi / Lx
    k = kx * math.sqrt(1 + (Lx / Ly) ** 2)
    return 2 * math.pi / math.sqrt(k * k - sigma * sigma / 4.0)


def telegraph(nx=64, sigma=1.0, rho=1e12, gamma=4.0 / 3.0):
    """Telegraph equation test (Sec. 5): Lx x Ly = 1 x 0.5, periodic, Nx x Nx/2,
    sigma_c = 1 (eta = 1), B1 = 1, rho = 1e12, p = 0, v = 0, tan(alpha) = 2."""
    ndim, nn, lo, hi = 2, [nx, nx // 2, 1], [0.0, 0.0, 0.0], [1.0, 0.5, 1.0]
    c, f = _axes(ndim, nn, lo, hi)
    X, Y, _ = _mesh(c[0], c[1], c[2])
    Ex, Ey, Bz = telegraph_exact(X, Y, 0.0, sigma)
    z = np.zeros_like(X)
    prim = [np.full_like(X, rho), z.copy(), z.copy(), z.copy(), z.copy(), Ex, Ey, z.copy()]
    bface = [z.copy(), z.copy(), Bz]
    return Problem("telegraph_2d", ndim, nn, lo, hi, ["periodic"] * 3, gamma, prim, bface=bface,
                   eta_u=1.0 / sigma, cfl=0.4, t_end=telegraph_period(sigma))


def charged_vortex_fields(X, Y, q0=0.7, p0=0.1, rho=1.0, gamma=4.0 / 3.0):
    """Stationary charged vortex (Sec. 5): returns (E^x, E^y, v^x, v^y, B^z, p, rho_e)."""
    R2 = X * X + Y * Y
    R = np.sqrt(R2)
    ER = 0.5 * q0 * R / (R2 + 1.0)
    root = np.sqrt((R2 + 1.0) ** 2 - q0 * q0 / 4.0)
    Bz = root / (R2 + 1.0)
    vphi = -0.5 * q0 * R / root
    g1 = (gamma - 1.0) / gamma
    p = -rho * g1 + (p0 + rho * g1) * ((4 * R2 + 4 - q0 * q0) / ((R2 + 1.0) * (4 - q0 * q0))) ** (
        gamma / (2 * (gamma - 1.0)))
    safe = np.where(R > 0, R, 1.0)
    cx, cy = np.where(R > 0, X / safe, 0.0), np.where(R > 0, Y / safe, 0.0)
    rho_e = q0 / (R2 + 1.0) ** 2
    return ER * cx, ER * cy, -vphi * cy, vphi * cx, Bz, p, rho_e


def charged_vortex(n=64, q0=0.7, p0=0.1, rho=1.0, gamma=4.0 / 3.0, eta=1e-3):
    """Stationary charged vortex on [-10, 10]^2, boundary values held fixed, t_end = 10."""
    ndim, nn, lo, hi = 2, [n, n, 1], [-10.0, -10.0, 0.0], [10.0, 10.0, 1.0]
    c, f = _axes(ndim, nn, lo, hi)
    X, Y, _ = _mesh(c[0], c[1], c[2])
    Ex, Ey, vx, vy, Bz, p, _ = charged_vortex_fields(X, Y, q0, p0, rho, gamma)
    ux, uy, uz = _lorentz_u(vx, vy, np.zeros_like(vx))
    z = np.zeros_like(X)
    prim = [np.full_like(X, rho), ux, uy, uz, p, Ex, Ey, z.copy()]
    bface = [z.copy(), z.copy(), Bz]
    return Problem("charged_vortex_2d", ndim, nn, lo, hi, ["fixed"] * 3, gamma, prim, bface=bface,
                   eta_u=eta, cfl=0.4, t_end=10.0)


# --------------------------------------------------------------------------
# random states
# --------------------------------------------------------------------------

def random_prims(seed, shape, u_scale=0.5, e_scale=0.5, b_scale=1.0):
    """Seeded random physical primitives: rho in [0.1, 10] and p in [0.01, 10]
    (log-uniform), u^i ~ N(0, u_scale^2), E^i ~ N(0, e_scale^2), cell B^i ~ N(0, b_scale^2).
    Returns (prim[8], B[3])."""
    rng = np.random.default_rng(seed)
    rho = 10.0 ** rng.uniform(-1, 1, shape)
    p = 10.0 ** rng.uniform(-2, 1, shape)
    u = [rng.normal(0, u_scale, shape) for _ in range(3)]
    E = [rng.normal(0, e_scale, shape) for _ in range(3)]
    B = [rng.normal(0, b_scale, shape) for _ in range(3)]
    return [rho, *u, p, *E], B


def random_box(seed, ndim, n, bc="periodic", gamma=5.0 / 3.0, amp=0.2, eta=1e-2, metric=False, xi=0.0,
               glm=False, kappa=2.0):
    """A small seeded box of smooth-plus-noise states for stencil parity tests: every
    field is a constant plus a few random Fourier modes plus noise of relative size
    ``amp``; face B from a random edge potential.  ``metric=True`` adds a smooth lapse
    and conformal factor.  ``glm=True`` adds cell-centred q_B (not divergence-free)
    and a Phi field for the GLM variant (drawn after everything else, so the other
    fields do not change)."""
    rng = np.random.default_rng(seed)
    nn = [n[d] if d < ndim else 1 for d in range(3)]
    lo, hi = [0.0] * 3, [1.0] * 3
    c, f = _axes(ndim, nn, lo, hi)
    X, Y, Z = _mesh(c[0], c[1], c[2])
    shp = X.shape

    def smooth(base, scale, XX=X, YY=Y, ZZ=Z):
        out = np.full(XX.shape, base, dtype=np.float64)
        for _ in range(3):
            k = rng.integers(1, 3, 3) * 2 * math.pi
            ph = rng.uniform(0, 2 * math.pi)
            out += scale * rng.normal() * np.sin(k[0] * XX + (k[1] * YY if ndim > 1 else 0)
                                                 + (k[2] * ZZ if ndim > 2 else 0) + ph)
        return out

    rho = smooth(1.0, 0.3 * amp) * (1 + amp * 0.1 * rng.uniform(-1, 1, shp))
    p = smooth(1.0, 0.3 * amp) * (1 + amp * 0.1 * rng.uniform(-1, 1, shp))
    u = [smooth(0.0, 0.5) + 0.05 * rng.normal(size=shp) for _ in range(3)]
    E = [smooth(0.0, 0.3) + 0.05 * rng.normal(size=shp) for _ in range(3)]
    prim = [rho, *u, p, *E]
    ng = [2 if d < ndim else 0 for d in range(3)]

    def edge_noise():
        # noise that repeats with the grid period, so that a periodic grid keeps a
        # periodic potential
        core = rng.normal(size=(nn[2], nn[1], nn[0]))
        pad = [(ng[2], ng[2]), (ng[1], ng[1]), (ng[0], ng[0])]
        return np.pad(core, pad, mode="wrap" if bc == "periodic" else "edge")

    A = []
    for cdir in range(3):
        coords = [f[d] if d != cdir else c[d] for d in range(3)]
        XX, YY, ZZ = _mesh(*coords)
        A.append(smooth(0.0, 0.1, XX, YY, ZZ) + 0.002 * edge_noise())
    bface = None
    if ndim == 1:
        # no curl can make B^x in 1-D: set the faces directly (B^x constant)
        bface = [np.full(shp, 0.7), smooth(0.3, 0.5), smooth(-0.2, 0.5)]
        A = None
    alpha = psi = None
    if metric:
        alpha = smooth(0.8, 0.05)
        psi = smooth(1.1, 0.05)
    eta_arr = 10.0 ** rng.uniform(math.log10(eta) - 1, math.log10(eta) + 1, shp)
    bcell = phi = None
    if glm:
        # cell-centred fields for the GLM variant (with a divergence), and a Phi
        bcell = [smooth(0.3 * (d - 1), 0.5) + 0.05 * rng.normal(size=shp) for d in range(3)]
        phi = smooth(0.0, 0.1) + 0.01 * rng.normal(size=shp)
    return Problem(f"random_box_{ndim}d", ndim, nn, lo, hi, [bc] * 3, gamma, prim, bface=bface, A_edge=A,
                   alpha=alpha, psi=psi, eta=eta_arr, eta_u=eta, cfl=0.4, xi=xi, bcell=bcell, phi=phi,
                   kappa=kappa)


# --------------------------------------------------------------------------
# batched and served workloads
# --------------------------------------------------------------------------

def ot_batch(seed=0, n_boxes=256, sizes=(64, 128, 256, 512), eta_range=(-6.0, 0.0)):
    """Independent 2-D Orszag-Tang boxes: side drawn uniformly from `sizes`, eta
    log-uniform in 10^eta_range, phase shifts uniform in [0, 2 pi)^2 (seeded)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_boxes):
        n = int(rng.choice(sizes))
        eta = 10.0 ** rng.uniform(*eta_range)
        ph = tuple(rng.uniform(0, 2 * math.pi, 2))
        out.append(orszag_tang(n, eta=eta, phase=ph))
    return out


def request_stream(seed=0, n_requests=64, rate=200.0, tube_cells=(400, 4096), vortex_side=(128, 512),
                   star_side=(64, 128), eta_range=(-6.0, 0.0), steps_2d3d=100):
    """Seeded Poisson stream of runs: (arrival time [s], Problem, number of steps).
    Kinds drawn uniformly: 1-D shock tube (cells in `tube_cells`, run to t = 0.4),
    2-D Orszag-Tang (side in `vortex_side`, `steps_2d3d` steps), 3-D star (side in
    `star_side`, `steps_2d3d` steps); eta log-uniform in 10^eta_range for every run.
    Each Problem's info records the drawn eta and its kind."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += rng.exponential(1.0 / rate)
        kind = int(rng.integers(0, 3))
        eta = 10.0 ** rng.uniform(*eta_range)
        if kind == 0:
            n = int(rng.integers(tube_cells[0], tube_cells[1] + 1))
            pr = shock_tube(n, eta=eta)
            steps = int(math.ceil(pr.t_end / (pr.cfl * (pr.hi[0] - pr.lo[0]) / n) - 1e-9))
        elif kind == 1:
            n = int(rng.integers(vortex_side[0], vortex_side[1] + 1))
            pr = orszag_tang(n, eta=eta, phase=tuple(rng.uniform(0, 2 * math.pi, 2)))
            steps = steps_2d3d
        else:
            n = int(rng.integers(star_side[0], star_side[1] + 1))
            pr = star(n=n, eta_in=eta)
            steps = steps_2d3d
        pr.info["eta"] = eta
        pr.info["kind"] = ("tube", "vortex", "star")[kind]
        out.append((t, pr, steps))
    return out


def dynamo_1d(k=1, n=64, eta=0.1, xi=0.5, rho=1e12, p=1.0, gamma=4.0 / 3.0):
    """One-dimensional steady dynamo (Sec. 5): B = 0.1 (0, sin kx, -cos kx), E = 0, v = 0
    on periodic [-pi, pi], uniform eta and dynamo parameter xi.  The paper freezes the
    matter; a density of 1e12 keeps it at rest here.  Frozen-matter growth rate of
    the helical mode: the positive root of lambda^2 + lambda/eta + k^2 - k xi/eta = 0."""
    ndim, nn, lo, hi = 1, [n, 1, 1], [-math.pi, 0.0, 0.0], [math.pi, 1.0, 1.0]
    c, f = _axes(ndim, nn, lo, hi)
    X, _, _ = _mesh(c[0], c[1], c[2])
    z = np.zeros_like(X)
    prim = [np.full_like(X, rho), z.copy(), z.copy(), z.copy(), np.full_like(X, p), z.copy(), z.copy(), z.copy()]
    bface = [z.copy(), 0.1 * np.sin(k * X), -0.1 * np.cos(k * X)]
    return Problem("dynamo_1d", ndim, nn, lo, hi, ["periodic"] * 3, gamma, prim, bface=bface, eta_u=eta, xi=xi,
                   cfl=0.4, t_end=6.0)


def dynamo_growth_rate(k, eta, xi):
    """Positive root of lambda^2 + lambda/eta + k^2 - k xi/eta = 0."""
    return 0.5 * (-1.0 / eta + math.sqrt(1.0 / eta ** 2 + 4.0 * (k * xi / eta - k * k)))


# --------------------------------------------------------------------------
# GLM hyperbolic cleaning workloads (Sec. 3.1, Sec. 5)
# --------------------------------------------------------------------------

def glm_wave(n=64, k=1, b=1e-3, kappa=1.0, rho=1.0, p=1.0, gamma=4.0 / 3.0, eta=1.0):
    """1-D (B^x, Phi) mode on periodic [0, 2 pi]: cell-centred B^x = b cos(kx), Phi = 0,
    matter at rest, E = 0.  For small b the GLM subsystem is the damped wave
    f'' + kappa f' + k^2 f = 0 for the amplitude f(t) of B^x (see glm_wave_amplitude)."""
    ndim, nn, lo, hi = 1, [n, 1, 1], [0.0, 0.0, 0.0], [2 * math.pi, 1.0, 1.0]
    c, f = _axes(ndim, nn, lo, hi)
    X, _, _ = _mesh(c[0], c[1], c[2])
    z = np.zeros_like(X)
    prim = [np.full_like(X, rho), z.copy(), z.copy(), z.copy(), np.full_like(X, p), z.copy(), z.copy(), z.copy()]
    bcell = [b * np.cos(k * X), z.copy(), z.copy()]
    return Problem("glm_wave_1d", ndim, nn, lo, hi, ["periodic"] * 3, gamma, prim, bcell=bcell, phi=z.copy(),
                   kappa=kappa, eta_u=eta, cfl=0.4, info={"k": k, "b": b})


def glm_wave_amplitude(t, k, kappa):
    """Amplitude of B^x for f'' + kappa f' + k^2 f = 0, f(0) = 1, f'(0) = 0 (k > kappa/2)."""
    w = math.sqrt(k * k - 0.25 * kappa * kappa)
    return math.exp(-0.5 * kappa * t) * (math.cos(w * t) + 0.5 * kappa / w * math.sin(w * t))


def monopole(n=64, ndim=3, kappa=1.0, R=0.2, L=2.0, rho=1.0, eps=0.1, gamma=5.0 / 3.0, eta=1e-16):
    """Magnetic monopole test for hyperbolic cleaning (Sec. 5): cell-centred
    B^x = exp(-r^2/R^2) - exp(-1) for r < R, else 0 (a Gaussian monopole), rho = 1,
    eps = 0.1 (p = (Gamma - 1) rho eps), Gamma = 5/3, v = E = 0, eta = 1e-16, on
    [-L, L]^ndim with outflow boundaries (the paper's run is 3-D, 64^3)."""
    nn = [n if d < ndim else 1 for d in range(3)]
    lo = [-L if d < ndim else 0.0 for d in range(3)]
    hi = [L if d < ndim else 1.0 for d in range(3)]
    c, f = _axes(ndim, nn, lo, hi)
    X, Y, Z = _mesh(c[0], c[1], c[2])
    r2 = X * X + (Y * Y if ndim > 1 else 0.0) + (Z * Z if ndim > 2 else 0.0)
    bx = np.where(r2 < R * R, np.exp(-r2 / (R * R)) - math.exp(-1.0), 0.0)
    z = np.zeros_like(X)
    prim = [np.full_like(X, rho), z.copy(), z.copy(), z.copy(), np.full_like(X, (gamma - 1.0) * rho * eps),
            z.copy(), z.copy(), z.copy()]
    return Problem(f"monopole_{ndim}d", ndim, nn, lo, hi, ["outflow"] * 3, gamma, prim, bcell=[bx, z.copy(), z.copy()],
                   phi=z.copy(), kappa=kappa, eta_u=eta, cfl=0.4)
