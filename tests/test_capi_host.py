"""Host-side checks of the C ABI that need no GPU: the library builds for sm_103a,
exports every function that include/grmhd.h declares, and rejects invalid grids,
tableaux and parameters before touching the device."""
import ctypes as C
import math
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "grmhd.h")

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


@pytest.fixture(scope="module")
def lib():
    from paper_2110_03732_gb300 import build
    path = build.build()
    return C.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(grmhd_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_no_device_allocation_symbols_in_sources():
    """The library allocates no device memory: the caller passes all buffers."""
    csrc = os.path.join(ROOT, "paper_2110_03732_gb300", "csrc")
    for f in os.listdir(csrc):
        s = open(os.path.join(csrc, f)).read()
        assert "cudaMalloc" not in s and "cudaFree" not in s, f


def _grid(ndim=2, n=(8, 8, 1), bc=(0, 0, 0), lo=(0, 0, 0), hi=(1, 1, 1)):
    from paper_2110_03732_gb300.grmhd import Grid
    g = Grid()
    g.ndim = ndim
    for d in range(3):
        g.n[d] = n[d]
        g.lo[d] = lo[d]
        g.hi[d] = hi[d]
        g.bc[d] = bc[d]
    return g


def test_ssp2_tableau_values(lib):
    from paper_2110_03732_gb300.grmhd import Tableau
    t = Tableau()
    assert lib.grmhd_tableau_ssp2(C.byref(t)) == 0
    g = 1 - 1 / math.sqrt(2)
    assert t.s == 2
    assert list(t.At[:4]) == [0, 0, 1, 0]
    assert abs(t.A[0] - g) < 1e-16 and abs(t.A[2] - (1 - 2 * g)) < 1e-16 and abs(t.A[3] - g) < 1e-16
    assert list(t.wt[:2]) == [0.5, 0.5] and list(t.w[:2]) == [0.5, 0.5]


def test_scratch_bytes_formula(lib):
    from paper_2110_03732_gb300.grmhd import Tableau
    t = Tableau()
    lib.grmhd_tableau_ssp2(C.byref(t))
    for ndim, n in ((1, (400, 1, 1)), (2, (512, 512, 1)), (3, (20, 12, 9))):
        g = _grid(ndim, n)
        b = C.c_size_t()
        assert lib.grmhd_scratch_bytes(C.byref(g), C.byref(t), C.byref(b)) == 0
        ncell = 1
        for d in range(3):
            ncell *= n[d] + 4 if d < ndim else 1
        arr = -(-8 * ncell // 256) * 256
        # FP64: primitives, stiff rates, later stage bases, running sum, fluxes, edge
        # EMFs and two transport-velocity arrays per direction (ideal-limit EMF)
        narr = 8 + 3 + 11 * (t.s - 1) + 11 + 8 * ndim + 3 + 2 * ndim
        arr32 = -(-4 * ncell // 256) * 256
        # FP32: stage primitives + cell q_B, and per stage the Newton start history (last
        # root and its change, 3 components each)
        narr32 = 11 + 6 * t.s
        small = -(-8 * 1024 * 11 // 256) * 256 + 256 + 256
        ct = narr * arr + narr32 * arr32 + small
        # GLM layout: 12 cell-centred variables per stage base, running sum and flux
        # direction, no edge EMFs; of the FP32 arrays only the start history
        glm = (8 + 3 + 12 * (t.s - 1) + 12 + 12 * ndim) * arr + 6 * t.s * arr32 + small
        assert b.value == max(ct, glm)


@pytest.mark.parametrize("field,value", [("ndim", 0), ("ndim", 4), ("n", 0), ("hi", -1.0), ("bc", 7),
                                         ("periodic1", 1)])
def test_invalid_grid_rejected(lib, field, value):
    from paper_2110_03732_gb300.grmhd import Tableau
    t = Tableau()
    lib.grmhd_tableau_ssp2(C.byref(t))
    g = _grid()
    if field == "ndim":
        g.ndim = value
    elif field == "n":
        g.n[1] = value
    elif field == "hi":
        g.hi[0] = value
    elif field == "bc":
        g.bc[0] = value
    elif field == "periodic1":
        g.n[0] = 1
    b = C.c_size_t()
    assert lib.grmhd_scratch_bytes(C.byref(g), C.byref(t), C.byref(b)) == -1
    lib.grmhd_last_error.restype = C.c_char_p
    assert len(lib.grmhd_last_error()) > 0


def test_invalid_tableau_and_params_rejected(lib):
    from paper_2110_03732_gb300.grmhd import Params, Tableau
    g = _grid()
    b = C.c_size_t()
    t = Tableau()
    lib.grmhd_tableau_ssp2(C.byref(t))
    t.A[3] = 0.0  # a_22 = 0: not diagonally implicit
    assert lib.grmhd_scratch_bytes(C.byref(g), C.byref(t), C.byref(b)) == -1
    lib.grmhd_tableau_ssp2(C.byref(t))
    t.At[1] = 0.3  # explicit part not strictly lower
    assert lib.grmhd_scratch_bytes(C.byref(g), C.byref(t), C.byref(b)) == -1
    lib.grmhd_tableau_ssp2(C.byref(t))
    t.s = 5
    assert lib.grmhd_scratch_bytes(C.byref(g), C.byref(t), C.byref(b)) == -1
    lib.grmhd_tableau_ssp2(C.byref(t))
    p = Params(1.0, 0.4, 0.0, 0, 0, 0.0, 0.0)   # Gamma must exceed 1
    ctx = C.c_void_p()
    assert lib.grmhd_create(C.byref(g), C.byref(p), C.byref(t), C.byref(ctx)) == -1
    assert not ctx.value


@pytest.mark.parametrize("case", ["bad_divb", "glm_mixed", "glm_negative_kappa"])
def test_invalid_divergence_scheme_rejected(lib, case):
    from paper_2110_03732_gb300.grmhd import Params, Tableau
    g = _grid()
    t = Tableau()
    lib.grmhd_tableau_ssp2(C.byref(t))
    p = Params(5.0 / 3.0, 0.4, 0.0, 0, 0, 0.0, 0.0, 1, 1.0)
    if case == "bad_divb":
        p.divb = 3
    elif case == "glm_mixed":
        p.precision = 1
    else:
        p.kappa_b = -1.0
    ctx = C.c_void_p()
    assert lib.grmhd_create(C.byref(g), C.byref(p), C.byref(t), C.byref(ctx)) == -1
    assert not ctx.value
    lib.grmhd_last_error.restype = C.c_char_p
    assert len(lib.grmhd_last_error()) > 0


def test_clean_scratch_bytes(lib):
    """Multigrid plan of the elliptic cleaning: phi and rhs on every level (each
    halving all active extents while they are even and >= 4), three CG vectors of the
    coarsest level, 1024 partial sums and the mean; too coarse a grid is refused."""
    for ndim, n, levels in (((2, (512, 512, 1), [512 * 512 // 4 ** k for k in range(9)]),
                             (1, (400, 1, 1), [400, 200, 100, 50, 25]),
                             (3, (19, 13, 7), [19 * 13 * 7]))):
        g = _grid(ndim, n)
        b = C.c_size_t()
        assert lib.grmhd_clean_scratch_bytes(C.byref(g), C.byref(b)) == 0
        want = 8 * (2 * sum(levels) + 3 * levels[-1] + 1024 + 1)
        assert b.value == -(-want // 256) * 256, (ndim, b.value, want)
    g = _grid(2, (1000, 1000, 1))     # coarsest 125 x 125 cells
    b = C.c_size_t()
    assert lib.grmhd_clean_scratch_bytes(C.byref(g), C.byref(b)) == -1


@pytest.mark.parametrize("case", ["bad_emf", "ideal_mixed", "ideal_glm", "ideal_fixed"])
def test_invalid_emf_rejected(lib, case):
    from paper_2110_03732_gb300.grmhd import Params, Tableau
    g = _grid()
    t = Tableau()
    lib.grmhd_tableau_ssp2(C.byref(t))
    p = Params(5.0 / 3.0, 0.4, 0.0, 0, 0, 0.0, 0.0, 0, 0.0, 1, 0)
    if case == "bad_emf":
        p.emf = 2
    elif case == "ideal_mixed":
        p.precision = 1
    elif case == "ideal_glm":
        p.divb = 1
    else:
        g.bc[1] = 2
    ctx = C.c_void_p()
    assert lib.grmhd_create(C.byref(g), C.byref(p), C.byref(t), C.byref(ctx)) == -1
    assert not ctx.value


@pytest.mark.parametrize("case", ["bad_rec", "ppm_ideal"])
def test_invalid_reconstruction_rejected(lib, case):
    from paper_2110_03732_gb300.grmhd import Params, Tableau
    g = _grid()
    t = Tableau()
    lib.grmhd_tableau_ssp2(C.byref(t))
    p = Params(5.0 / 3.0, 0.4, 0.0, 0, 0, 0.0, 0.0, 0, 0.0, 0, 1)
    if case == "bad_rec":
        p.rec = 5
    else:
        p.emf = 1
    ctx = C.c_void_p()
    assert lib.grmhd_create(C.byref(g), C.byref(p), C.byref(t), C.byref(ctx)) == -1
    assert not ctx.value


def test_null_context_is_refused_by_every_call(lib):
    """Every call that takes a context returns GRMHD_ERR_ARG (-1) with a message for a
    NULL one, before touching the device."""
    vp = C.c_void_p
    null = vp(None)
    buf = (C.c_double * 8)()
    ptrs = (vp * 11)()
    sz = C.c_size_t(0)
    ll = (C.c_longlong * 4)()
    calls = {
        "grmhd_set_timing": (null, C.c_int(1)),
        "grmhd_set_launch_overlap": (null, C.c_int(1)),
        "grmhd_kernel_times": (null, buf, ll),
        "grmhd_bind": (null, ptrs, ptrs, vp(1), C.c_size_t(0)),
        "grmhd_bind_phi": (null, vp(1)),
        "grmhd_set_metric": (null, null, null),
        "grmhd_set_eta": (null, null, C.c_double(1.0)),
        "grmhd_set_dynamo": (null, C.c_double(0.1)),
        "grmhd_init_from_prims": (null, ptrs, ptrs, null),
        "grmhd_compute_dt": (null, buf, null),
        "grmhd_stage": (null, C.c_int(0), C.c_double(1e-3), null),
        "grmhd_step": (null, C.c_double(1e-3), null),
        "grmhd_get_prims": (null, ptrs, null),
        "grmhd_implicit": (null, C.c_double(1e-3), ptrs, ptrs, ptrs, ptrs, null),
        "grmhd_explicit_L": (null, ptrs, ptrs, ptrs, null),
        "grmhd_explicit_L_glm": (null, ptrs, ptrs, vp(1), ptrs, null),
        "grmhd_diagnostics": (null, buf, buf, ll, null),
        "grmhd_clean_divb": (null, C.c_int(1), vp(1), C.c_size_t(0), null),
        "grmhd_start_bytes": (null, C.byref(sz)),
        "grmhd_save_start": (null, vp(1), C.c_size_t(0), null),
        "grmhd_load_start": (null, vp(1), C.c_size_t(0), null),
    }
    lib.grmhd_last_error.restype = C.c_char_p
    for name, args in calls.items():
        f = getattr(lib, name)
        f.restype = C.c_int
        assert f(*args) == -1, name
        assert lib.grmhd_last_error(), name
    lib.grmhd_launch_count.restype = C.c_longlong
    assert lib.grmhd_launch_count(null) == 0
    lib.grmhd_destroy.restype = C.c_int
    assert lib.grmhd_destroy(null) == 0


def test_ctypes_structs_match_the_header_layout(tmp_path):
    """The binding's ctypes Structures have the sizes and field offsets that a C
    compiler gives the header's structs (a mismatch would silently corrupt them)."""
    from paper_2110_03732_gb300.grmhd import Grid, Params, Tableau
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"grmhd_grid": Grid, "grmhd_params": Params, "grmhd_tableau": Tableau}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "grmhd.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    import subprocess
    # grmhd.h refers to cudaStream_t only through an opaque struct pointer
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True, timeout=120)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=30).stdout.split("\n")
    got = {}
    for ln in out:
        parts = ln.split()
        if len(parts) == 3:
            got[(parts[0], parts[1])] = int(parts[2])
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_normal_build_reports_no_bounds_checks():
    """The normal build has no index checks: grmhd_bounds_violations reports -1 (and
    needs no device for that)."""
    import ctypes as C
    from paper_2110_03732_gb300 import build as _b
    L = C.CDLL(_b.build())
    L.grmhd_bounds_violations.argtypes = [C.POINTER(C.c_longlong), C.c_int]
    L.grmhd_bounds_violations.restype = C.c_int
    n = C.c_longlong(7)
    assert L.grmhd_bounds_violations(C.byref(n), 0) == 0 and n.value == -1
    assert L.grmhd_bounds_violations(None, 0) == -1


def test_numerics_eval_checks_arguments_on_the_host():
    """grmhd_numerics_eval refuses an unknown op, a negative count and NULL arrays, and
    launches nothing for n = 0 -- all before any device call."""
    import ctypes as C
    from paper_2110_03732_gb300 import build as _b
    L = C.CDLL(_b.build())
    f = L.grmhd_numerics_eval
    f.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p]
    f.restype = C.c_int
    assert f(-1, None, None, 0, None) == -1
    assert f(16, None, None, 0, None) == -1
    assert f(0, None, None, -1, None) == -1
    assert f(0, None, None, 4, None) == -1
    assert f(0, None, None, 0, None) == 0


def test_mixed_precision_refuses_a_tolerance_below_1e_11():
    """The mixed path accepts Newton roots by a double-word residual (~1e-14 of the
    momentum scale): grmhd_create refuses newton_tol in (0, 1e-11) for it, before any
    device call; FP64 takes any tolerance."""
    import ctypes as C
    from paper_2110_03732_gb300 import build as _b
    from paper_2110_03732_gb300.grmhd import Params, Tableau
    L = C.CDLL(_b.build())
    L.grmhd_create.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    L.grmhd_create.restype = C.c_int
    L.grmhd_tableau_ssp2.argtypes = [C.c_void_p]
    L.grmhd_last_error.restype = C.c_char_p
    t = Tableau()
    L.grmhd_tableau_ssp2(C.byref(t))
    g = _grid(2, (8, 8, 1))
    p = Params(4.0 / 3.0, 0.4, 1e-12, 0, 1, 0.0, 0.0, 0, 0.0, 0, 0)
    ctx = C.c_void_p()
    assert L.grmhd_create(C.byref(g), C.byref(p), C.byref(t), C.byref(ctx)) == -1
    assert b"newton_tol" in L.grmhd_last_error()
