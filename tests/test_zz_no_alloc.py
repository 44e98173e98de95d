"""grmhd_divb_noalloc: the div B check for callers that cannot allocate device
memory (their device memory is owned by a pool or arena of their own, or their loop
must not allocate after start-up), so they cannot give a context its scratch.  The
call keeps its partial sums in a fixed array inside the library instead.

The test calls it through the C ABI twice in a row on the same face fields and
compares both results with grmhd_diagnostics (the entry point that uses
caller-provided scratch): the maximum must agree exactly (order-independent), the
mean and rms to 1e-12 relative (the two reductions add in different orders).  Both
are also compared with the oracle's div B on the same fields (maximum to 1e-13: the
oracle divides by dx where the GPU multiplies by 1/dx).  It also checks that a grid
above the array's stated limit, or with an infinite extent, is refused, and that
the array of an inactive direction may be NULL.  This file is collected last on
purpose."""
import ctypes as C

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _divb_noalloc(lib, grid, bf, out):
    arr = (C.c_void_p * 3)(*[b.data_ptr() for b in bf])
    return lib.grmhd_divb_noalloc(C.byref(grid), C.cast(arr, C.POINTER(C.c_void_p)), C.c_void_p(out.data_ptr()),
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("case", ["ot_2d", "random_3d_outflow"])
def test_divb_noalloc_matches_diagnostics(case):
    from paper_2110_03732_gb300 import build, grmhd
    from paper_2110_03732_gb300 import problems as P
    build.build()
    lib = grmhd.lib()
    lib.grmhd_divb_noalloc.argtypes = [C.POINTER(grmhd.Grid), C.POINTER(C.c_void_p), C.c_void_p, C.c_void_p]
    lib.grmhd_divb_noalloc.restype = C.c_int
    if case == "ot_2d":
        pr = P.orszag_tang(96)
    else:
        pr = P.random_box(6, 3, [20, 14, 11], bc="outflow")
    S = grmhd.Solver.from_problem(pr)
    og = oracle.Grid(pr.ndim, pr.n, [(pr.hi[d] - pr.lo[d]) / pr.n[d] if d < pr.ndim else 1.0 for d in range(3)],
                     pr.bc, pr.gamma)
    dt = S.compute_dt()
    for _ in range(3):
        S.step(dt)
    # face fields with a clearly non-zero divergence as well as the solver's own
    rng = np.random.default_rng(3)
    noisy = [b + torch.as_tensor(rng.normal(0, 1e-3, b.shape), device=b.device) for b in S.bf]
    for fields in (S.bf, noisy):
        if fields is not S.bf:
            for d in range(3):
                S.bf[d].copy_(fields[d])
        ref, _, _ = S.diagnostics()
        outs = []
        for _ in range(2):
            out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
            assert _divb_noalloc(lib, S.grid, S.bf, out) == 0
            torch.cuda.synchronize()
            outs.append(out.cpu().numpy())
        want = oracle.divb(og, [b.cpu().numpy() for b in S.bf])
        for o in outs:
            assert o[2] == ref[2]
            np.testing.assert_allclose(o[:2], ref[:2], rtol=1e-12, atol=0)
            if fields is noisy:
                np.testing.assert_allclose(o[:2], want[:2], rtol=1e-12, atol=0)
                np.testing.assert_allclose(o[2], want[2], rtol=1e-13, atol=0)
            else:   # a CT run: both at round-off of the field scale
                scale = float(max(b.abs().max() for b in S.bf)) / min(og.dx[:pr.ndim])
                assert o[2] < 1e-12 * scale and want[2] < 1e-12 * scale
        np.testing.assert_array_equal(outs[0], outs[1])


def test_divb_noalloc_inactive_direction_may_be_null_and_extents_must_be_finite():
    from paper_2110_03732_gb300 import build, grmhd
    build.build()
    lib = grmhd.lib()
    lib.grmhd_divb_noalloc.argtypes = [C.POINTER(grmhd.Grid), C.POINTER(C.c_void_p), C.c_void_p, C.c_void_p]
    lib.grmhd_divb_noalloc.restype = C.c_int
    n = [24, 18]
    g = grmhd.make_grid(2, n, [0.0, -1.0, 0.0], [2.0, 0.5, 1.0], ["outflow"] * 3)
    og = oracle.Grid(2, n, [2.0 / n[0], 1.5 / n[1]], ["outflow"] * 3, 4.0 / 3.0)
    rng = np.random.default_rng(5)
    bf = [torch.as_tensor(rng.normal(size=og.shape), device="cuda") for _ in range(2)]
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    arr = (C.c_void_p * 3)(bf[0].data_ptr(), bf[1].data_ptr(), None)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.grmhd_divb_noalloc(C.byref(g), C.cast(arr, C.POINTER(C.c_void_p)), C.c_void_p(out.data_ptr()), st) == 0
    torch.cuda.synchronize()
    want = oracle.divb(og, [b.cpu().numpy() for b in bf] + [np.zeros(og.shape)])
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-12, atol=0)
    # an active direction's array may not be NULL
    arr0 = (C.c_void_p * 3)(bf[0].data_ptr(), None, None)
    assert lib.grmhd_divb_noalloc(C.byref(g), C.cast(arr0, C.POINTER(C.c_void_p)), C.c_void_p(out.data_ptr()), st) == -1
    for bad in (float("inf"), float("-inf"), float("nan")):
        gb = grmhd.make_grid(2, n, [0.0, -1.0, 0.0], [bad, 0.5, 1.0], ["outflow"] * 3)
        assert lib.grmhd_divb_noalloc(C.byref(gb), C.cast(arr, C.POINTER(C.c_void_p)), C.c_void_p(out.data_ptr()),
                                      st) == -1
        assert b"invalid grid" in lib.grmhd_last_error()
    gb = grmhd.make_grid(2, n, [float("-inf"), -1.0, 0.0], [2.0, 0.5, 1.0], ["outflow"] * 3)
    assert lib.grmhd_divb_noalloc(C.byref(gb), C.cast(arr, C.POINTER(C.c_void_p)), C.c_void_p(out.data_ptr()),
                                  st) == -1


def test_divb_noalloc_rejects_grids_above_its_limit():
    from paper_2110_03732_gb300 import build, grmhd
    build.build()
    lib = grmhd.lib()
    lib.grmhd_divb_noalloc.argtypes = [C.POINTER(grmhd.Grid), C.POINTER(C.c_void_p), C.c_void_p, C.c_void_p]
    lib.grmhd_divb_noalloc.restype = C.c_int
    g = grmhd.make_grid(3, [130, 130, 130], [0, 0, 0], [1, 1, 1], ["periodic"] * 3)  # 2.197e6 cells
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    bf = [t, t, t]
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    assert _divb_noalloc(lib, g, bf, out) == -1   # GRMHD_ERR_ARG
    assert b"too large" in lib.grmhd_last_error()
