"""Thin ctypes binding of ``libgrmhd.so`` (the C ABI in ``include/grmhd.h``).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  Importing this module fails
loudly when the library has not been built (``paper_2110_03732_gb300.build``); there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build as _build

_lib = None

GRMHD_OK = 0
GRMHD_WARN_C2P_FAILED = 1
GRMHD_ERR_ARG = -1
GRMHD_ERR_TIMEOUT = -4
BC = {"periodic": 0, "outflow": 1, "fixed": 2}


class GrmhdError(RuntimeError):
    pass


class Grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("bc", C.c_int * 3)]


class Tableau(C.Structure):
    _fields_ = [("s", C.c_int), ("At", C.c_double * 16), ("A", C.c_double * 16), ("wt", C.c_double * 4),
                ("w", C.c_double * 4)]


class Params(C.Structure):
    _fields_ = [("gamma_eos", C.c_double), ("cfl", C.c_double), ("newton_tol", C.c_double),
                ("newton_kmax", C.c_int), ("precision", C.c_int), ("rho_atm", C.c_double), ("p_atm", C.c_double),
                ("divb", C.c_int), ("kappa_b", C.c_double), ("emf", C.c_int), ("rec", C.c_int)]

EMF = {"resistive": 0, "ideal": 1}
REC = {"mc": 0, "ppm": 1}

DIVB = {"ct": 0, "glm": 1}


def library_path():
    return _build.LIB


def lib():
    """Load ``libgrmhd.so``; raises if it is missing (build it first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise GrmhdError(f"{path} is missing: run paper_2110_03732_gb300.build.build() (nvcc, sm_103a)")
    L = C.CDLL(path)
    vp = C.c_void_p
    dpp = C.POINTER(C.c_void_p)
    L.grmhd_tableau_ssp2.argtypes = [C.POINTER(Tableau)]
    L.grmhd_scratch_bytes.argtypes = [C.POINTER(Grid), C.POINTER(Tableau), C.POINTER(C.c_size_t)]
    L.grmhd_create.argtypes = [C.POINTER(Grid), C.POINTER(Params), C.POINTER(Tableau), C.POINTER(vp)]
    L.grmhd_destroy.argtypes = [vp]
    L.grmhd_bind.argtypes = [vp, dpp, dpp, vp, C.c_size_t]
    L.grmhd_set_metric.argtypes = [vp, vp, vp]
    L.grmhd_set_eta.argtypes = [vp, vp, C.c_double]
    L.grmhd_set_dynamo.argtypes = [vp, C.c_double]
    L.grmhd_init_from_prims.argtypes = [vp, dpp, dpp, vp]
    L.grmhd_compute_dt.argtypes = [vp, C.POINTER(C.c_double), vp]
    L.grmhd_stage.argtypes = [vp, C.c_int, C.c_double, vp]
    L.grmhd_step.argtypes = [vp, C.c_double, vp]
    L.grmhd_get_prims.argtypes = [vp, dpp, vp]
    L.grmhd_implicit.argtypes = [vp, C.c_double, dpp, dpp, dpp, dpp, vp]
    L.grmhd_explicit_L.argtypes = [vp, dpp, dpp, dpp, vp]
    L.grmhd_explicit_L_glm.argtypes = [vp, dpp, dpp, vp, dpp, vp]
    L.grmhd_bind_phi.argtypes = [vp, vp]
    L.grmhd_clean_scratch_bytes.argtypes = [C.POINTER(Grid), C.POINTER(C.c_size_t)]
    L.grmhd_clean_divb.argtypes = [vp, C.c_int, vp, C.c_size_t, vp]
    L.grmhd_diagnostics.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_longlong), vp]
    L.grmhd_set_timing.argtypes = [vp, C.c_int]
    L.grmhd_set_launch_overlap.argtypes = [vp, C.c_int]
    L.grmhd_kernel_times.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
    L.grmhd_batch_scratch_bytes.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(C.c_size_t)]
    L.grmhd_batch_create.argtypes = [C.POINTER(vp), C.c_int, vp, C.c_size_t, C.POINTER(vp)]
    L.grmhd_batch_set_dt.argtypes = [vp, C.POINTER(C.c_double), vp]
    L.grmhd_batch_step.argtypes = [vp, vp]
    L.grmhd_batch_autotune.argtypes = [vp, C.c_int, vp]
    L.grmhd_batch_config.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.grmhd_batch_destroy.argtypes = [vp]
    L.grmhd_batch_step_persistent.argtypes = [vp, C.c_int, C.c_int, vp]
    L.grmhd_batch_set_wait_limit.argtypes = [vp, C.c_double]
    L.grmhd_batch_persistent_status.argtypes = [vp, vp]
    L.grmhd_launch_count.argtypes = [vp]
    L.grmhd_launch_count.restype = C.c_longlong
    L.grmhd_start_bytes.argtypes = [vp, C.POINTER(C.c_size_t)]
    L.grmhd_save_start.argtypes = [vp, vp, C.c_size_t, vp]
    L.grmhd_load_start.argtypes = [vp, vp, C.c_size_t, vp]
    L.grmhd_fp64_fma_rate.argtypes = [C.POINTER(C.c_double), vp]
    L.grmhd_bounds_violations.argtypes = [C.POINTER(C.c_longlong), C.c_int]
    L.grmhd_numerics_eval.argtypes = [C.c_int, vp, vp, C.c_longlong, vp]
    L.grmhd_last_error.restype = C.c_char_p
    for name in ("grmhd_tableau_ssp2", "grmhd_scratch_bytes", "grmhd_create", "grmhd_destroy", "grmhd_bind",
                 "grmhd_set_metric", "grmhd_set_eta", "grmhd_set_dynamo", "grmhd_init_from_prims", "grmhd_compute_dt", "grmhd_stage",
                 "grmhd_step", "grmhd_get_prims", "grmhd_implicit", "grmhd_explicit_L", "grmhd_diagnostics",
                 "grmhd_set_timing", "grmhd_set_launch_overlap", "grmhd_kernel_times", "grmhd_batch_scratch_bytes", "grmhd_batch_create",
                 "grmhd_batch_set_dt", "grmhd_batch_step", "grmhd_batch_autotune", "grmhd_batch_config",
                 "grmhd_batch_destroy", "grmhd_explicit_L_glm", "grmhd_bind_phi", "grmhd_clean_scratch_bytes",
                 "grmhd_clean_divb", "grmhd_start_bytes", "grmhd_save_start", "grmhd_load_start",
                 "grmhd_fp64_fma_rate", "grmhd_bounds_violations", "grmhd_batch_step_persistent",
                 "grmhd_batch_set_wait_limit", "grmhd_batch_persistent_status", "grmhd_numerics_eval"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def check(status, what=""):
    if status < 0:
        msg = lib().grmhd_last_error().decode()
        raise GrmhdError(f"{what}: status {status}: {msg}")
    return status


def _ptrs(tensors):
    arr = (C.c_void_p * len(tensors))(*[None if t is None else t.data_ptr() for t in tensors])
    return C.cast(arr, C.POINTER(C.c_void_p)), arr


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def make_grid(ndim, n, lo, hi, bc):
    g = Grid()
    g.ndim = ndim
    for d in range(3):
        g.n[d] = int(n[d]) if d < ndim else 1
        g.lo[d] = float(lo[d])
        g.hi[d] = float(hi[d])
        b = bc[d]
        g.bc[d] = BC[b] if isinstance(b, str) else int(b)
    return g


def bounds_violations(reset=False):
    """Array-index bounds violations counted since the last reset (synchronises the
    device); -1 when the loaded library is the normal build, which has no checks.
    Load the checked copy by pointing build.LIB at build.LIB_CHECKED before the
    first use of the library."""
    n = C.c_longlong(0)
    check(lib().grmhd_bounds_violations(C.byref(n), int(bool(reset))), "bounds_violations")
    return n.value


def fp64_fma_rate(stream=None):
    """FP64 fused multiply-add rate of the current device in TFLOP/s (a register-only
    probe kernel timed with CUDA events; measurement only)."""
    r = C.c_double(0.0)
    check(lib().grmhd_fp64_fma_rate(C.byref(r), _stream(stream)), "fp64_fma_rate")
    return r.value


# ops of grmhd_numerics_eval: (value, inputs per element, outputs per element)
NUMERIC_OPS = {
    "rsqrt_ge1": (0, 1, 1), "rcp_pos": (1, 1, 1), "d2f": (2, 1, 1), "f2d": (3, 1, 1),
    "dw_split": (4, 1, 2), "dw_add": (5, 2, 2), "dw_mul": (6, 2, 2), "dw_rcp": (7, 1, 2),
    "dw_sqrt": (8, 1, 2), "quarter": (9, 1, 1), "twice": (10, 1, 1), "minmod3": (11, 3, 1),
    "minmod3_f32": (12, 3, 1), "prod_sign": (13, 2, 1), "ppm_limit": (14, 3, 2), "tests": (15, 1, 1),
}


def numerics_eval(name, x, stream=None):
    """The library's device arithmetic helper `name` (NUMERIC_OPS) on the float64 CUDA
    tensor x of shape (n,) or (n, arity); returns (n,) or (n, 2) (testing only)."""
    import torch
    op, ar, no = NUMERIC_OPS[name]
    x = x.to(torch.float64).contiguous()
    n = x.shape[0]
    if x.numel() != n * ar:
        raise GrmhdError(f"numerics_eval {name}: expected {ar} inputs per element")
    out = torch.empty((n, no) if no > 1 else (n,), dtype=torch.float64, device=x.device)
    check(lib().grmhd_numerics_eval(op, x.data_ptr() if n else None, out.data_ptr() if n else None, n,
                                    _stream(stream)), "numerics_eval")
    return out


def ssp2():
    t = Tableau()
    check(lib().grmhd_tableau_ssp2(C.byref(t)), "tableau")
    return t


def scratch_bytes(grid, tab):
    n = C.c_size_t(0)
    check(lib().grmhd_scratch_bytes(C.byref(grid), C.byref(tab), C.byref(n)), "scratch_bytes")
    return n.value


class Solver:
    """One resistive-MHD problem resident on the GPU: state, scratch and context.

    ``q`` (8 tensors) and ``bf`` (3 tensors) are the padded, densitised conserved
    cell and face fields; the library updates them in place.  With ``divb="glm"``
    (GLM cleaning, Sec. 3.1) ``bf`` holds cell-centred q_B and ``phi`` the evolved
    q_Phi; ``kappa`` is the damping kappa_B.  ``launch_overlap`` launches the stage
    kernels with programmatic dependent launch (bitwise the same results)."""

    def __init__(self, ndim, n, lo, hi, bc, gamma, cfl=0.4, tableau=None, device="cuda", newton_tol=0.0,
                 newton_kmax=0, rho_atm=0.0, p_atm=0.0, precision="fp64", divb="ct", kappa=0.0, emf="resistive",
                 rec="mc", launch_overlap=True):
        self.L = lib()
        self.grid = make_grid(ndim, n, lo, hi, bc)
        self.tab = ssp2() if tableau is None else tableau
        prec = {"fp64": 0, "mixed": 1}[precision] if isinstance(precision, str) else int(precision)
        self.precision = prec
        self.glm = (DIVB[divb] if isinstance(divb, str) else int(divb)) == DIVB["glm"]
        self.par = Params(float(gamma), float(cfl), float(newton_tol), int(newton_kmax), prec, float(rho_atm),
                          float(p_atm), DIVB["glm"] if self.glm else DIVB["ct"], float(kappa),
                          EMF[emf] if isinstance(emf, str) else int(emf), REC[rec] if isinstance(rec, str) else int(rec))
        self.device = torch.device(device)
        ng = [2 if d < ndim else 0 for d in range(3)]
        self.N = [self.grid.n[d] + 2 * ng[d] for d in range(3)]
        self.shape = (self.N[2], self.N[1], self.N[0])
        self.ndim = ndim
        self.ng = ng
        self.cells = self.grid.n[0] * self.grid.n[1] * self.grid.n[2]
        opts = dict(dtype=torch.float64, device=self.device)
        # the state in one block (q 0..7, the three field arrays, q_Phi for GLM), so that
        # it moves between host and device in one copy; q, bf and phi are views into it
        self.state = torch.zeros((12 if self.glm else 11,) + self.shape, **opts)
        self.q = [self.state[v] for v in range(8)]
        self.bf = [self.state[8 + d] for d in range(3)]
        nbytes = scratch_bytes(self.grid, self.tab)
        # torch's caching allocator returns 512-byte aligned blocks
        self.scratch = torch.zeros(nbytes, dtype=torch.uint8, device=self.device)
        ctx = C.c_void_p()
        with torch.cuda.device(self.device):
            check(self.L.grmhd_create(C.byref(self.grid), C.byref(self.par), C.byref(self.tab), C.byref(ctx)),
                  "create")
        self.ctx = ctx
        self.set_launch_overlap(launch_overlap)
        pq, self._kq = _ptrs(self.q)
        pb, self._kb = _ptrs(self.bf)
        check(self.L.grmhd_bind(ctx, pq, pb, C.c_void_p(self.scratch.data_ptr()), nbytes), "bind")
        self.phi = None
        if self.glm:
            self.phi = self.state[11]
            check(self.L.grmhd_bind_phi(ctx, C.c_void_p(self.phi.data_ptr())), "bind_phi")
        self.alpha = self.psi = self.eta = None
        self.eta_u = 0.0

    def __del__(self):
        try:
            if getattr(self, "ctx", None):
                self.L.grmhd_destroy(self.ctx)
                self.ctx = None
        except Exception:
            pass

    # -- configuration -------------------------------------------------------
    def set_metric(self, alpha=None, psi=None):
        self.alpha = None if alpha is None else self._dev(alpha)
        self.psi = None if psi is None else self._dev(psi)
        check(self.L.grmhd_set_metric(self.ctx, self._vp(self.alpha), self._vp(self.psi)), "set_metric")

    def set_eta(self, eta=None, eta_u=0.0):
        self.eta = None if eta is None else self._dev(eta)
        self.eta_u = float(eta_u)
        check(self.L.grmhd_set_eta(self.ctx, self._vp(self.eta), self.eta_u), "set_eta")

    def set_dynamo(self, xi):
        check(self.L.grmhd_set_dynamo(self.ctx, float(xi)), "set_dynamo")

    def init_from_prims(self, prim, A_edge=None, bface=None, stream=None, phi=None):
        """Initial state.  CT: A_edge on edges (curl -> faces) or face q_B in bface.
        GLM: A_edge is a cell-centred potential (central curl), or bface holds the
        cell-centred q_B; phi is the initial primitive Phi (None: zero), which the
        library densitises into q_Phi."""
        prim = [self._dev(p) for p in prim]
        if bface is not None:
            for d in range(3):
                self.bf[d].copy_(self._dev(bface[d]))
        if self.glm:
            prim = prim + [None if phi is None else self._dev(phi)]
        A = None if A_edge is None else [self._dev(a) for a in A_edge]
        pp, k1 = _ptrs(prim)
        pa, k2 = _ptrs(A) if A is not None else (None, None)
        check(self.L.grmhd_init_from_prims(self.ctx, pp, pa, _stream(stream)), "init_from_prims")
        self._keep = (prim, A)

    @classmethod
    def from_problem(cls, prob, device="cuda", **kw):
        kw.setdefault("rho_atm", prob.rho_atm)
        kw.setdefault("p_atm", prob.p_atm)
        if kw.get("divb") == "glm":
            kw.setdefault("kappa", prob.kappa)
        s = cls(prob.ndim, prob.n, prob.lo, prob.hi, prob.bc, prob.gamma, prob.cfl, device=device, **kw)
        s.set_metric(prob.alpha, prob.psi)
        s.set_eta(prob.eta, prob.eta_u if prob.eta is None else (prob.eta_u or 1.0))
        if getattr(prob, "xi", 0.0):
            s.set_dynamo(prob.xi)
        if s.glm:
            # cell-centred fields: the potential at cell centres, else q_B given at cells
            s.init_from_prims(prob.prim, A_edge=prob.A_cell, bface=None if prob.A_cell is not None else prob.bcell,
                              phi=prob.phi)
        else:
            s.init_from_prims(prob.prim, A_edge=prob.A_edge, bface=None if prob.A_edge is not None else prob.bface)
        return s

    # -- stepping ------------------------------------------------------------
    def compute_dt(self, stream=None):
        dt = C.c_double(0.0)
        check(self.L.grmhd_compute_dt(self.ctx, C.byref(dt), _stream(stream)), "compute_dt")
        return dt.value

    def stage(self, i, dt, stream=None):
        return check(self.L.grmhd_stage(self.ctx, int(i), float(dt), _stream(stream)), "stage")

    def step(self, dt, stream=None, clean_cycles=0):
        """One IMEX step; with clean_cycles > 0 the field is then cleaned (Sec. 3.3)."""
        r = check(self.L.grmhd_step(self.ctx, float(dt), _stream(stream)), "step")
        if clean_cycles:
            self.clean_divb(clean_cycles, stream)
        return r

    def clean_divb(self, cycles=10, stream=None):
        """Elliptic cleaning of the bound field arrays (multigrid, `cycles` V-cycles)."""
        if getattr(self, "_mg_scratch", None) is None:
            n = C.c_size_t(0)
            check(self.L.grmhd_clean_scratch_bytes(C.byref(self.grid), C.byref(n)), "clean_scratch_bytes")
            self._mg_scratch = torch.empty(max(n.value, 1), dtype=torch.uint8, device=self.device)
        check(self.L.grmhd_clean_divb(self.ctx, int(cycles), C.c_void_p(self._mg_scratch.data_ptr()),
                                      self._mg_scratch.numel(), _stream(stream)), "clean_divb")

    def get_prims(self, stream=None):
        out = [torch.zeros(self.shape, dtype=torch.float64, device=self.device) for _ in range(8)]
        po, k = _ptrs(out)
        check(self.L.grmhd_get_prims(self.ctx, po, _stream(stream)), "get_prims")
        return out

    def implicit(self, a_dt, q, bface, prim, stream=None):
        """Implicit solve on caller tensors (q is modified; prim in/out). Returns R."""
        R = [torch.zeros(self.shape, dtype=torch.float64, device=self.device) for _ in range(3)]
        pq, k1 = _ptrs(q)
        pb, k2 = _ptrs(bface)
        pp, k3 = _ptrs(prim)
        pr, k4 = _ptrs(R)
        check(self.L.grmhd_implicit(self.ctx, float(a_dt), pq, pb, pp, pr, _stream(stream)), "implicit")
        return R

    def explicit_L_glm(self, prim, qB, qphi, stream=None):
        """GLM explicit operator: 12 arrays (8 cell-centred, q_B^1..3, q_Phi)."""
        Lt = [torch.zeros(self.shape, dtype=torch.float64, device=self.device) for _ in range(12)]
        pp, k1 = _ptrs(prim)
        pb, k2 = _ptrs(qB)
        pl, k3 = _ptrs(Lt)
        check(self.L.grmhd_explicit_L_glm(self.ctx, pp, pb, self._vp(qphi), pl, _stream(stream)), "explicit_L_glm")
        return Lt

    def explicit_L(self, prim, bface, stream=None):
        Lt = [torch.zeros(self.shape, dtype=torch.float64, device=self.device) for _ in range(11)]
        pp, k1 = _ptrs(prim)
        pb, k2 = _ptrs(bface)
        pl, k3 = _ptrs(Lt)
        check(self.L.grmhd_explicit_L(self.ctx, pp, pb, pl, _stream(stream)), "explicit_L")
        return Lt

    def diagnostics(self, stream=None):
        divb = (C.c_double * 3)()
        tot = (C.c_double * 8)()
        nf = C.c_longlong(0)
        check(self.L.grmhd_diagnostics(self.ctx, divb, tot, C.byref(nf), _stream(stream)), "diagnostics")
        return list(divb), list(tot), nf.value

    def launch_count(self):
        return int(self.L.grmhd_launch_count(self.ctx))

    # -- checkpoint / resume -------------------------------------------------
    def checkpoint(self, stream=None):
        """Everything a bitwise resume needs, as CPU tensors: the state q^n, the face
        (or cell) q_B, q_Phi for GLM, and the context's Newton start blob
        (grmhd_save_start).  The grid, parameters, metric and eta are the caller's
        set-up and are not included."""
        n = C.c_size_t()
        check(self.L.grmhd_start_bytes(self.ctx, C.byref(n)), "start_bytes")
        blob = torch.empty(n.value, dtype=torch.uint8, device=self.device)
        check(self.L.grmhd_save_start(self.ctx, C.c_void_p(blob.data_ptr()), n.value, _stream(stream)), "save_start")
        ck = {"q": [t.cpu() for t in self.q], "bf": [t.cpu() for t in self.bf], "start": blob.cpu()}
        if self.phi is not None:
            ck["phi"] = self.phi.cpu()
        return ck

    def restore(self, ck, stream=None):
        """Load a checkpoint taken from a solver of the same grid, tableau and scheme
        (the library checks the start blob's size first)."""
        blob = ck["start"].to(self.device)
        check(self.L.grmhd_load_start(self.ctx, C.c_void_p(blob.data_ptr()), blob.numel(), _stream(stream)),
              "load_start")
        for t, s in zip(self.q, ck["q"]):
            t.copy_(s)
        for t, s in zip(self.bf, ck["bf"]):
            t.copy_(s)
        if self.phi is not None:
            self.phi.copy_(ck["phi"])
        torch.cuda.current_stream(self.device).synchronize()

    KERNEL_KINDS = ("implicit", "flux", "emf", "update")

    def set_timing(self, on=True):
        check(self.L.grmhd_set_timing(self.ctx, int(on)), "set_timing")

    def set_launch_overlap(self, on=True):
        """Programmatic dependent launch of the stage kernels (bitwise the same results)."""
        check(self.L.grmhd_set_launch_overlap(self.ctx, int(on)), "set_launch_overlap")

    def kernel_times(self):
        """Cumulative (ms, launches) per kernel kind since timing was enabled."""
        ms = (C.c_double * 4)()
        n = (C.c_longlong * 4)()
        check(self.L.grmhd_kernel_times(self.ctx, ms, n), "kernel_times")
        return {k: (ms[i], n[i]) for i, k in enumerate(self.KERNEL_KINDS)}

    # -- helpers -------------------------------------------------------------
    def _dev(self, a):
        if isinstance(a, torch.Tensor):
            t = a.to(device=self.device, dtype=torch.float64)
        else:
            t = torch.as_tensor(a, dtype=torch.float64).to(self.device)
        return t.contiguous()

    @staticmethod
    def _vp(t):
        return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(None)

    def interior(self):
        return tuple(slice(self.ng[d], self.ng[d] + self.grid.n[d]) for d in (2, 1, 0))


class Batch:
    """Many Solver problems advanced together (grmhd_batch_*): one launch per kernel
    kind and stage covers all of them.  Each problem's results are bitwise those of
    stepping it alone.  The solvers must share the tableau and the precision."""

    KINDS = ("implicit", "flux_x", "flux_y", "flux_z", "emf_x", "emf_y", "emf_z", "update")

    def __init__(self, solvers):
        self.L = lib()
        self.solvers = list(solvers)
        n = len(self.solvers)
        arr = (C.c_void_p * n)(*[s.ctx.value for s in self.solvers])
        self._arr = arr
        nb = C.c_size_t(0)
        check(self.L.grmhd_batch_scratch_bytes(arr, n, C.byref(nb)), "batch_scratch_bytes")
        dev = self.solvers[0].device
        self.scratch = torch.zeros(max(nb.value, 1), dtype=torch.uint8, device=dev)
        b = C.c_void_p()
        check(self.L.grmhd_batch_create(arr, n, C.c_void_p(self.scratch.data_ptr()), nb.value, C.byref(b)),
              "batch_create")
        self.b = b
        self.n = n

    def __del__(self):
        try:
            if getattr(self, "b", None):
                self.L.grmhd_batch_destroy(self.b)
                self.b = None
        except Exception:
            pass

    def set_dt(self, dts, stream=None):
        arr = (C.c_double * self.n)(*[float(x) for x in dts])
        check(self.L.grmhd_batch_set_dt(self.b, arr, _stream(stream)), "batch_set_dt")

    def step(self, stream=None):
        return check(self.L.grmhd_batch_step(self.b, _stream(stream)), "batch_step")

    def autotune(self, reps=3, stream=None):
        check(self.L.grmhd_batch_autotune(self.b, int(reps), _stream(stream)), "batch_autotune")
        return self.config()

    def config(self):
        th = (C.c_int * 8)()
        it = (C.c_int * 8)()
        check(self.L.grmhd_batch_config(self.b, th, it), "batch_config")
        return {k: (th[i], it[i]) for i, k in enumerate(self.KINDS)}

    def step_persistent(self, nsteps=1, synchronize=True, stream=None):
        """nsteps steps of every problem in one cooperative launch (bitwise the same
        results as step()); with synchronize, raises GrmhdError on a wait that ran out
        (status GRMHD_ERR_TIMEOUT)."""
        return check(self.L.grmhd_batch_step_persistent(self.b, int(nsteps), int(bool(synchronize)),
                                                        _stream(stream)), "batch_step_persistent")

    def set_wait_limit(self, seconds):
        check(self.L.grmhd_batch_set_wait_limit(self.b, float(seconds)), "batch_set_wait_limit")

    def persistent_status(self, stream=None):
        """GRMHD_OK, or GRMHD_ERR_TIMEOUT if a barrier wait of the last persistent launch
        ran out (synchronises; does not raise)."""
        return int(self.L.grmhd_batch_persistent_status(self.b, _stream(stream)))
