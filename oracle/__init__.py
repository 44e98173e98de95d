"""CPU oracle for one IMEX-RK step of resistive (GR)MHD with staggered CT.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  It shares no code with the CUDA path in ``paper_2110_03732_gb300``; the
only module both sides use is ``paper_2110_03732_gb300.problems`` (seeded
initial data, none of the method's arithmetic).

The arithmetic lives in ``grmhd_oracle.c`` (plain C99, FP64, compiled with
``-O2 -ffp-contract=off`` so that no multiply-add is fused); this file compiles it
with gcc on first use and marshals numpy arrays.  Arrays are padded grids of shape
``(N2, N1, N0)`` (x fastest) with two ghost layers in each active direction; see
``grid_shape``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "grmhd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libgrmhd_oracle.so")
_lock = threading.Lock()
_lib = None

BC = {"periodic": 0, "outflow": 1, "fixed": 2}
GAMMA_SSP2 = 1.0 - 1.0 / np.sqrt(2.0)


def compile_library(src: str, out: str) -> None:
    """gcc, plain C99, FP64, no fused multiply-add contraction."""
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", src, "-o", out, "-lm"]
    subprocess.run(cmd, check=True)


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        compile_library(_SRC, tmp)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    """The loaded oracle library.  ``GRMHD_ORACLE_LIB`` names another build of the oracle
    source to load instead (tests/test_oracle_mutations.py loads copies with planted
    mistakes that way); it is then loaded as it is, never rebuilt."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("GRMHD_ORACLE_LIB")
            if not path:
                build()
                path = _LIB
            L = C.CDLL(path)
            dp = C.POINTER(C.c_double)
            dpp = C.POINTER(dp)
            ip = C.POINTER(C.c_int)
            L.orc_curl_A.argtypes = [ip, dp, dpp, dpp]
            L.orc_prim2con.argtypes = [ip, dp, dpp, dpp, dp, dpp]
            L.orc_solve_cell.argtypes = [dp, C.c_double, C.c_double, C.c_double, dp, dp, dp, dp]
            L.orc_solve_cell.restype = C.c_int
            L.orc_residual_cell.argtypes = [dp, C.c_double, C.c_double, C.c_double, dp, dp, dp, dp]
            L.orc_implicit.argtypes = [ip, dp, C.c_double, dpp, dpp, dp, dp, dp, C.c_double, dpp, dpp, ip]
            L.orc_implicit.restype = C.c_int
            L.orc_explicit_L.argtypes = [ip, dp, dpp, dpp, dp, dp, dpp]
            L.orc_step.argtypes = [ip, dp, C.c_int, dp, dp, dp, dp, C.c_double, dpp, dpp, dp, dp, dp,
                                   C.c_double, dpp, ip]
            L.orc_step.restype = C.c_int
            L.orc_dt.argtypes = [ip, dp, dp, dp, C.c_double]
            L.orc_dt.restype = C.c_double
            L.orc_divb.argtypes = [ip, dp, dpp, dp]
            L.orc_totals.argtypes = [ip, dp, dpp, dp]
            L.orc_curl_A_cc.argtypes = [ip, dp, dpp, dpp]
            L.orc_prim2con_cc.argtypes = [ip, dp, dpp, dpp, dp, dpp]
            L.orc_implicit_cc.argtypes = [ip, dp, C.c_double, dpp, dpp, dp, dp, dp, C.c_double, dpp, dpp, ip]
            L.orc_implicit_cc.restype = C.c_int
            L.orc_explicit_L_glm.argtypes = [ip, dp, C.c_double, dpp, dpp, dp, dp, dp, dpp]
            L.orc_step_glm.argtypes = [ip, dp, C.c_int, dp, dp, dp, dp, C.c_double, C.c_double, dpp, dpp, dp,
                                       dp, dp, dp, C.c_double, dpp, ip]
            L.orc_step_glm.restype = C.c_int
            L.orc_divb_cc.argtypes = [ip, dp, dpp, dp]
            L.orc_face_states.argtypes = [ip, dp, dp, C.c_int, dp, dp]
            _lib = L
    return _lib


# --------------------------------------------------------------------------
# marshalling
# --------------------------------------------------------------------------

def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _dpp(arrs):
    ptrs = (C.POINTER(C.c_double) * len(arrs))(*[_dp(a) for a in arrs])
    return C.cast(ptrs, C.POINTER(C.POINTER(C.c_double))), ptrs


class Grid:
    """Uniform Cartesian grid: ``ndim`` active directions, ``n`` interior cells,
    cell widths ``dx``, boundary kinds ``bc`` (periodic / outflow / fixed), ideal-gas
    ``gamma``, atmosphere floor ``rho_atm``/``p_atm`` (0: none).  Inactive directions
    have one cell and no ghosts."""

    def __init__(self, ndim, n, dx, bc, gamma, rho_atm=0.0, p_atm=0.0, xi=0.0, emf="resistive", rec="mc"):
        n = list(n) + [1] * (3 - len(n))
        dx = list(dx) + [1.0] * (3 - len(dx))
        bc = list(bc) + ["periodic"] * (3 - len(bc))
        self.ndim = ndim
        self.n = [int(v) if d < ndim else 1 for d, v in enumerate(n)]
        self.dx = [float(v) for v in dx]
        self.bc = [BC[b] if isinstance(b, str) else int(b) for b in bc]
        self.gamma = float(gamma)
        self.ng = [2 if d < ndim else 0 for d in range(3)]
        self.N = [self.n[d] + 2 * self.ng[d] for d in range(3)]
        self._gi = (C.c_int * 7)(ndim, *self.n, *self.bc)
        self.rho_atm, self.p_atm, self.xi = float(rho_atm), float(p_atm), float(xi)
        self.emf = {"resistive": 0, "ideal": 1}[emf] if isinstance(emf, str) else int(emf)
        self.rec = {"mc": 0, "ppm": 1}[rec] if isinstance(rec, str) else int(rec)
        self._gd = (C.c_double * 9)(*self.dx, self.gamma, self.rho_atm, self.p_atm, self.xi, float(self.emf),
                                    float(self.rec))

    @property
    def shape(self):
        return (self.N[2], self.N[1], self.N[0])

    def interior(self):
        """Slices of the interior cells in a padded ``(N2, N1, N0)`` array."""
        return tuple(slice(self.ng[d], self.ng[d] + self.n[d]) for d in (2, 1, 0))

    def zeros(self, k=None):
        if k is None:
            return np.zeros(self.shape)
        return [np.zeros(self.shape) for _ in range(k)]

    @property
    def gi(self):
        return C.cast(self._gi, C.POINTER(C.c_int))

    @property
    def gd(self):
        return C.cast(self._gd, C.POINTER(C.c_double))


def curl_A(grid, A):
    """Face q_B = curl of the edge vector potential (Sec. 4); faces whose stencil
    leaves the array stay zero."""
    bf = grid.zeros(3)
    pa, ka = _dpp(A)
    pb, kb = _dpp(bf)
    lib().orc_curl_A(grid.gi, grid.gd, pa, pb)
    return bf


def prim2con(grid, prim, bf, psi=None):
    """Densitised conserved (D, S_j, tau, E^j) at every padded cell."""
    q = grid.zeros(8)
    pp, k1 = _dpp(prim)
    pb, k2 = _dpp(bf)
    pq, k3 = _dpp(q)
    lib().orc_prim2con(grid.gi, grid.gd, pp, pb, _dp(psi), pq)
    return q


def solve_cell(D, S, tau, Es, B, psi, etat, gamma, guess=None, xi=0.0):
    """One-cell implicit solve (Sec. 2.4).  ``etat < 0`` holds E fixed; ``guess`` is
    the initial velocity (default: rest); ``xi`` the dynamo parameter.  Returns
    (iterations, u[3], E[3], rho, p)."""
    inp = np.array([D, *S, tau, *Es, *B, xi], dtype=np.float64)
    g = None if guess is None else np.ascontiguousarray(guess, dtype=np.float64)
    u = np.zeros(3)
    E = np.zeros(3)
    rp = np.zeros(2)
    it = lib().orc_solve_cell(_dp(inp), psi, etat, gamma, _dp(g), _dp(u), _dp(E), _dp(rp))
    return it, u, E, rp[0], rp[1]


def residual_cell(D, S, tau, Es, B, psi, etat, gamma, u, xi=0.0):
    """Residual f_i, analytic Jacobian J_ij and E^i(u) at velocity ``u``."""
    inp = np.array([D, *S, tau, *Es, *B, xi], dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    f = np.zeros(3)
    J = np.zeros(9)
    E = np.zeros(3)
    lib().orc_residual_cell(_dp(inp), psi, etat, gamma, _dp(u), _dp(f), _dp(J), _dp(E))
    return f, J.reshape(3, 3), E


def implicit(grid, a_dt, q, bf, alpha=None, psi=None, eta=None, eta_u=0.0, prim=None):
    """Implicit stage solve over the interior; ``q`` is modified (q_E replaced).
    Returns (prim[8], R[3], fails, max_iters)."""
    prim = grid.zeros(8) if prim is None else prim
    R = grid.zeros(3)
    st = (C.c_int * 2)(0, 0)
    pq, k1 = _dpp(q)
    pb, k2 = _dpp(bf)
    pp, k3 = _dpp(prim)
    pr, k4 = _dpp(R)
    f = lib().orc_implicit(grid.gi, grid.gd, a_dt, pq, pb, _dp(alpha), _dp(psi), _dp(eta), eta_u, pp, pr,
                           C.cast(st, C.POINTER(C.c_int)))
    return prim, R, f, st[1]


def explicit_L(grid, prim, bf, alpha=None, psi=None):
    """The explicit operator: 8 cell-centred + 3 face arrays."""
    L = grid.zeros(11)
    pp, k1 = _dpp(prim)
    pb, k2 = _dpp(bf)
    pl, k3 = _dpp(L)
    lib().orc_explicit_L(grid.gi, grid.gd, pp, pb, _dp(alpha), _dp(psi), pl)
    return L


def ssp2_tableau():
    """IMEX-SSP2(2,2,2), Sec. 2.3 table: explicit (At, wt), implicit (A, w)."""
    g = GAMMA_SSP2
    At = np.array([[0.0, 0.0], [1.0, 0.0]])
    A = np.array([[g, 0.0], [1.0 - 2.0 * g, g]])
    wt = np.array([0.5, 0.5])
    w = np.array([0.5, 0.5])
    return At, A, wt, w


def step(grid, dt, q, bf, prim, alpha=None, psi=None, eta=None, eta_u=0.0, tableau=None):
    """One IMEX step in place on ``q`` (8) and ``bf`` (3); ``prim`` (8) receives the
    last stage's primitives (its ghosts are read for fixed boundaries).
    Returns (fails, max_iters)."""
    At, A, wt, w = ssp2_tableau() if tableau is None else tableau
    s = len(wt)
    At = np.ascontiguousarray(At, dtype=np.float64).ravel()
    A = np.ascontiguousarray(A, dtype=np.float64).ravel()
    wt = np.ascontiguousarray(wt, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    st = (C.c_int * 2)(0, 0)
    pq, k1 = _dpp(q)
    pb, k2 = _dpp(bf)
    pp, k3 = _dpp(prim)
    rc = lib().orc_step(grid.gi, grid.gd, s, _dp(At), _dp(A), _dp(wt), _dp(w), dt, pq, pb, _dp(alpha),
                        _dp(psi), _dp(eta), eta_u, pp, C.cast(st, C.POINTER(C.c_int)))
    if rc != 0:
        raise ValueError("oracle: tableau must be diagonally implicit with a_ii > 0")
    return st[0], st[1]


def cfl_dt(grid, cfl, alpha=None, psi=None):
    return lib().orc_dt(grid.gi, grid.gd, _dp(alpha), _dp(psi), cfl)


def divb(grid, bf):
    """(mean |div q_B|, rms, max) over interior cells."""
    out = np.zeros(3)
    pb, k = _dpp(bf)
    lib().orc_divb(grid.gi, grid.gd, pb, _dp(out))
    return out


def totals(grid, q):
    out = np.zeros(8)
    pq, k = _dpp(q)
    lib().orc_totals(grid.gi, grid.gd, pq, _dp(out))
    return out


class State:
    """An oracle run: grid, conserved q (8), face q_B (3), primitives (8), metric, eta."""

    def __init__(self, grid, prim, bf, alpha=None, psi=None, eta=None, eta_u=0.0):
        self.grid = grid
        self.bf = [np.ascontiguousarray(b, dtype=np.float64).copy() for b in bf]
        self.prim = [np.ascontiguousarray(p, dtype=np.float64).copy() for p in prim]
        self.alpha = None if alpha is None else np.ascontiguousarray(alpha, dtype=np.float64)
        self.psi = None if psi is None else np.ascontiguousarray(psi, dtype=np.float64)
        self.eta = None if eta is None else np.ascontiguousarray(eta, dtype=np.float64)
        self.eta_u = float(eta_u)
        self.q = prim2con(grid, self.prim, self.bf, self.psi)
        self.t = 0.0
        self.fails = 0
        self.max_iters = 0

    def step(self, dt, tableau=None):
        f, it = step(self.grid, dt, self.q, self.bf, self.prim, self.alpha, self.psi, self.eta, self.eta_u,
                     tableau)
        self.fails += f
        self.max_iters = max(self.max_iters, it)
        self.t += dt

    def run(self, t_end, cfl):
        dt0 = cfl_dt(self.grid, cfl, self.alpha, self.psi)
        while self.t < t_end * (1 - 1e-14):
            self.step(min(dt0, t_end - self.t))

    def con2prim(self):
        """Primitives of the current conserved state with E held fixed."""
        q = [a.copy() for a in self.q]
        prim = [a.copy() for a in self.prim]
        implicit(self.grid, 0.0, q, self.bf, self.alpha, self.psi, self.eta, self.eta_u, prim)
        return prim


def from_problem(prob, emf="resistive", rec="mc"):
    """Oracle state from a ``paper_2110_03732_gb300.problems.Problem``: face q_B from
    the edge potential (oracle curl) or taken as given.  ``emf="ideal"`` takes the
    ideal-limit edge EMF of App. A."""
    grid = Grid(prob.ndim, prob.n, prob.dx, prob.bc, prob.gamma, prob.rho_atm, prob.p_atm, getattr(prob, "xi", 0.0),
                emf, rec)
    if prob.A_edge is not None:
        bf = curl_A(grid, [np.ascontiguousarray(a, dtype=np.float64) for a in prob.A_edge])
    else:
        bf = [np.ascontiguousarray(b, dtype=np.float64).copy() for b in prob.bface]
    return State(grid, prob.prim, bf, prob.alpha, prob.psi, prob.eta, prob.eta_u)


# --------------------------------------------------------------------------
# GLM hyperbolic cleaning variant (Sec. 3.1): cell-centred q_B (3) and q_Phi
# --------------------------------------------------------------------------

def curl_A_cc(grid, A):
    """Cell-centred q_B from a cell-centred potential (central differences)."""
    qB = grid.zeros(3)
    pa, k1 = _dpp(A)
    pb, k2 = _dpp(qB)
    lib().orc_curl_A_cc(grid.gi, grid.gd, pa, pb)
    return qB


def prim2con_cc(grid, prim, qB, psi=None):
    q = grid.zeros(8)
    pp, k1 = _dpp(prim)
    pb, k2 = _dpp(qB)
    pq, k3 = _dpp(q)
    lib().orc_prim2con_cc(grid.gi, grid.gd, pp, pb, _dp(psi), pq)
    return q


def implicit_cc(grid, a_dt, q, qB, alpha=None, psi=None, eta=None, eta_u=0.0, prim=None):
    """The implicit solve with cell-centred q_B given directly."""
    prim = grid.zeros(8) if prim is None else prim
    R = grid.zeros(3)
    st = (C.c_int * 2)(0, 0)
    pq, k1 = _dpp(q)
    pb, k2 = _dpp(qB)
    pp, k3 = _dpp(prim)
    pr, k4 = _dpp(R)
    f = lib().orc_implicit_cc(grid.gi, grid.gd, a_dt, pq, pb, _dp(alpha), _dp(psi), _dp(eta), eta_u, pp, pr,
                              C.cast(st, C.POINTER(C.c_int)))
    return prim, R, f, st[1]


def explicit_L_glm(grid, kappa, prim, qB, qphi, alpha=None, psi=None):
    """GLM explicit operator: 12 cell-centred arrays (8 + q_B^1..3 + q_Phi)."""
    L = grid.zeros(12)
    pp, k1 = _dpp(prim)
    pb, k2 = _dpp(qB)
    pl, k3 = _dpp(L)
    lib().orc_explicit_L_glm(grid.gi, grid.gd, float(kappa), pp, pb, _dp(qphi), _dp(alpha), _dp(psi), pl)
    return L


def step_glm(grid, dt, kappa, q, qB, qphi, prim, alpha=None, psi=None, eta=None, eta_u=0.0, tableau=None):
    """One IMEX step of the GLM variant in place on q (8), qB (3), qphi."""
    At, A, wt, w = ssp2_tableau() if tableau is None else tableau
    s = len(wt)
    At = np.ascontiguousarray(At, dtype=np.float64).ravel()
    A = np.ascontiguousarray(A, dtype=np.float64).ravel()
    wt = np.ascontiguousarray(wt, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    st = (C.c_int * 2)(0, 0)
    pq, k1 = _dpp(q)
    pb, k2 = _dpp(qB)
    pp, k3 = _dpp(prim)
    rc = lib().orc_step_glm(grid.gi, grid.gd, s, _dp(At), _dp(A), _dp(wt), _dp(w), dt, float(kappa), pq, pb,
                            _dp(qphi), _dp(alpha), _dp(psi), _dp(eta), eta_u, pp, C.cast(st, C.POINTER(C.c_int)))
    if rc != 0:
        raise ValueError("oracle: tableau must be diagonally implicit with a_ii > 0")
    return st[0], st[1]


def divb_cc(grid, qB):
    """(mean |div q_B|, rms, max) of cell-centred fields by central differences."""
    out = np.zeros(3)
    pb, k = _dpp(qB)
    lib().orc_divb_cc(grid.gi, grid.gd, pb, _dp(out))
    return out


class GLMState:
    """An oracle run of the GLM variant: q (8), cell-centred qB (3), qphi."""

    def __init__(self, grid, prim, qB, qphi, kappa, alpha=None, psi=None, eta=None, eta_u=0.0):
        self.grid = grid
        self.kappa = float(kappa)
        self.qB = [np.ascontiguousarray(b, dtype=np.float64).copy() for b in qB]
        self.qphi = np.ascontiguousarray(qphi, dtype=np.float64).copy()
        self.prim = [np.ascontiguousarray(p, dtype=np.float64).copy() for p in prim]
        self.alpha = None if alpha is None else np.ascontiguousarray(alpha, dtype=np.float64)
        self.psi = None if psi is None else np.ascontiguousarray(psi, dtype=np.float64)
        self.eta = None if eta is None else np.ascontiguousarray(eta, dtype=np.float64)
        self.eta_u = float(eta_u)
        self.q = prim2con_cc(grid, self.prim, self.qB, self.psi)
        self.t = 0.0
        self.fails = 0
        self.max_iters = 0

    def step(self, dt, tableau=None):
        f, it = step_glm(self.grid, dt, self.kappa, self.q, self.qB, self.qphi, self.prim, self.alpha, self.psi,
                         self.eta, self.eta_u, tableau)
        self.fails += f
        self.max_iters = max(self.max_iters, it)
        self.t += dt


def face_states(grid, a, d):
    """Left/right states at the lower d-face of every cell (test export of the
    reconstruction)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    L = grid.zeros()
    R = grid.zeros()
    lib().orc_face_states(grid.gi, grid.gd, _dp(a), int(d), _dp(L), _dp(R))
    return L, R


def from_problem_glm(prob, kappa=None, rec="mc"):
    """GLM oracle state from a Problem: cell-centred q_B from ``prob.A_cell`` (oracle
    central curl) or ``prob.bcell``; q_Phi = psi^6 ``prob.phi`` (0 if None)."""
    grid = Grid(prob.ndim, prob.n, prob.dx, prob.bc, prob.gamma, prob.rho_atm, prob.p_atm, getattr(prob, "xi", 0.0),
                rec=rec)
    if prob.A_cell is not None:
        qB = curl_A_cc(grid, [np.ascontiguousarray(a, dtype=np.float64) for a in prob.A_cell])
    else:
        qB = [np.ascontiguousarray(b, dtype=np.float64).copy() for b in prob.bcell]
    qphi = grid.zeros()
    if prob.phi is not None:
        sg = 1.0 if prob.psi is None else prob.psi ** 6
        qphi = np.ascontiguousarray(sg * prob.phi, dtype=np.float64)
    k = prob.kappa if kappa is None else kappa
    return GLMState(grid, prob.prim, qB, qphi, k, prob.alpha, prob.psi, prob.eta, prob.eta_u)
